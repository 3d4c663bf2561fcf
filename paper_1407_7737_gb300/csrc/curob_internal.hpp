// curob_internal.hpp -- host-side declarations shared by libcurob's .cu files.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "curob_device.cuh"

namespace curob {

// What the generator needs to know about one rotated block.
struct GaussJob {
  long long r_off;  // destination in the FP64 rotation pool
  int n;            // block size
  int fid;          // function the block belongs to (RNG counter word 2)
  int comp;         // component index within the function (RNG counter word 3)
  int blk;          // block index within the component (RNG counter word 1)
};

// One component to shift and permute.
struct PermJob {
  long long base;   // offset of its o / S / o[S] vectors
  int fid, comp;
  int origin;       // x^opt = 0 (third member of a composition, Sec. 6)
  int identity;     // unrotated: S = identity
  int nblk;
  int blk_off[5], blk_n[5];  // non-empty blocks in z order
};

// Per-variable table request for one segment.
struct AuxJob {
  long long aux_off;
  int kind, n, gn, gpos;
};

// curob_setup.cu
cudaError_t launch_shift_perm(const PermJob* d_jobs, int njobs, int D, uint64_t seed, double* o,
                              int* S, double* operm, uint64_t* tmp_words, int* tmp_mark,
                              cudaStream_t st);
cudaError_t launch_gauss_gs(const GaussJob* d_jobs, int njobs, int max_n, uint64_t seed, double* R,
                            int* status, cudaStream_t st);
cudaError_t launch_aux(const AuxJob* d_jobs, int njobs, double* aux, float* aux32,
                       cudaStream_t st);
cudaError_t launch_split_f32(const double* src, float* hi, float* lo, long long n,
                             cudaStream_t st);
cudaError_t launch_transpose_block(long long r_off, int n, const double* R, const float* Rh,
                                   const float* Rl, double* Rt, float* Rht, float* Rlt,
                                   cudaStream_t st);
cudaError_t launch_operm(const PermJob* d_jobs, int njobs, int D, const double* o, const int* S,
                         double* operm, cudaStream_t st);

// curob_simt64.cu / curob_simt32.cu
cudaError_t launch_simt_f64(const Tables& tb, const Function& F, const double* x, int N,
                            double* out, cudaStream_t st);
cudaError_t launch_simt_f32(const Tables& tb, const Function& F, const float* x, int N,
                            float* out, cudaStream_t st);

// curob_small64.cu / curob_small32.cu: one CTA per candidate and one warp
// per block, for small populations; blocks up to 128 wide, at most 16 blocks
// per function, the CTA's tables within 160 KB of shared memory.
struct SmallArgs;  // curob_small.cuh
bool small_supports(const Function& F, int D);
cudaError_t launch_small_f64(const SmallArgs& a, const double* x, int N, double* out,
                             cudaStream_t st);
cudaError_t launch_small_f32(const SmallArgs& a, const float* x, int N, float* out,
                             cudaStream_t st);

}  // namespace curob

// curob_mma.hpp -- the tensor-core (tcgen05) evaluator of curob_evaluatef.
#pragma once

#include <vector>

#include "../../include/curob.h"
#include "curob_internal.hpp"

namespace curob {

struct MmaPlan {
  float* img = nullptr;      // operand images of every rotation block (TF32 then BF16)
  long long img_floats = 0;
  float* ohi = nullptr;      // o[S[k]] split into FP32 hi/lo words, per component
  float* olo = nullptr;
  long long o_entries = 0;
  float* tau = nullptr;      // EXACT: power-of-two row scales of every block
  float* onat = nullptr;     // o per component in natural order, FP32
  bool sm103 = false;        // the device runs tcgen05
  bool ready = false;
  cudaMemPool_t pool = nullptr;  // stream-ordered scratch of split launches (kept warm)
};

// Lays out and fills the operand images (sets Segment::img_off / npad).
curob_status mma_prepare(MmaPlan& p, std::vector<Segment>& segs, const Tables& tb, float* prev);
// Rebuilds the images of the given segments after their R changed.
curob_status mma_refresh(MmaPlan& p, const std::vector<Segment>& segs, const std::vector<int>& ids,
                         const Tables& tb);
void mma_release(MmaPlan& p);
// True when every block of F fits the tensor-core kernel.
bool mma_supports(const MmaPlan& p, const Function& F);
// Precision AUTO picks for F (CUROB_PRECISION_TF32X3, _EXACT or _MIXED).
int mma_auto_mode(const MmaPlan& p, const Function& F);
// AUTO for a composition whose members differ: the members with a kind that
// magnifies contraction error on EXACT, the others on TF32X3, then the
// finish kernel (heavy kinds, composition): three launches on `st`.
cudaError_t launch_mma_mixed(const MmaPlan& p, const Tables& tb, const Function& F,
                             const float* x, int N, float* out, cudaStream_t st);
// One CTA whose wait on an mbarrier nothing completes runs out (2 s) and
// writes DEV_TIMEOUT to *status.
cudaError_t launch_wait_selftest(int* status, cudaStream_t st);
// mode: CUROB_PRECISION_TF32X3, _BF16X3, _FP16X3 or _EXACT.  A function with
// heavy-kind blocks (kind_is_heavy) takes a second launch (finish kernel).
cudaError_t launch_mma(const MmaPlan& p, const Tables& tb, const Function& F, int mode,
                       const float* x, int N, float* out, cudaStream_t st);

// One launch of the tensor-core kernel over all of F's components, every
// kind closed in its epilogue (the tile arithmetic of the persistent batch
// kernel, launch by launch).
cudaError_t launch_mma_fused(const MmaPlan& p, const Tables& tb, const Function& F, int mode,
                             const float* x, int N, float* out, cudaStream_t st);
// Kernel launches launch_mma / launch_mma_mixed make for F at N candidates
// (mode CUROB_PRECISION_MIXED for the latter).
int mma_launch_count(const Function& F, int mode, int N);

// Persistent launches over a ragged batch, in CUROB_PRECISION_EXACT or
// _TF32X3 (every item of one launch in the launch's precision).
size_t mma_args_bytes();
// Writes the device-side argument block of one batch item into dst (host).
// npad_max: the widest block (rounded up to 32) among the items of the
// launch the item belongs to (TF32X3 sizes its stages by it).
void mma_fill_args(void* dst, const MmaPlan& p, const Tables& tb, const Function& F,
                   const float* x, float* out, int N, int mode = CUROB_PRECISION_EXACT,
                   int npad_max = 512);
// Launches the persistent kernel on `grid` CTAs over nwork (item, tile)
// pairs; *d_counter must be 0; mode and npad_max as the items' argument
// blocks were filled with.
cudaError_t launch_mma_batch(const void* d_args, const int2* d_work, int nwork, int* d_counter,
                             int grid, cudaStream_t st, int mode = CUROB_PRECISION_EXACT,
                             int npad_max = 512);
// Largest block width the tensor-core kernels take.
int mma_max_block();

}  // namespace curob

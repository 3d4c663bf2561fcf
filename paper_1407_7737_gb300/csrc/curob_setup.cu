// curob_setup.cu -- instance generation on the GPU (General Setup section):
// shifts x^opt ~ U[-70,70]^D, a random split of the variables into blocks,
// Gaussian blocks orthonormalised by Gram-Schmidt, per-variable tables.
// Not timed: runs once per curob_initialize.  Compiled with -fmad=false so
// that the shift 140 u - 70 rounds exactly like its two-operation statement.
#include <algorithm>

#include "curob_internal.hpp"

namespace curob {

namespace {

__device__ inline double u53(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

// o (or 0) and the Fisher-Yates words, one thread per variable.
__global__ void shift_words_kernel(const PermJob* jobs, int D, uint64_t seed, double* o,
                                   uint64_t* words) {
  const PermJob J = jobs[blockIdx.y];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < D; k += gridDim.x * blockDim.x) {
    double v = 0.0;
    if (!J.origin) {
      double t = 140.0 * u53(rng_word(seed, P_SHIFT, 0, J.fid, J.comp, (uint64_t)k));
      v = t - 70.0;
    }
    o[J.base + k] = v;
    words[(long long)blockIdx.y * D + k] = rng_word(seed, P_PERM, 0, J.fid, J.comp, (uint64_t)k);
  }
}

// Fisher-Yates over the D variables, then each block's indices in increasing
// order.  Sequential by nature: one thread per component.
__global__ void permute_kernel(const PermJob* jobs, int njobs, int D, const uint64_t* words, int* S,
                               int* mark) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= njobs) return;
  const PermJob J = jobs[j];
  int* s = S + J.base;
  for (int k = 0; k < D; ++k) s[k] = k;
  if (J.identity) return;
  const uint64_t* w = words + (long long)j * D;
  for (int i = D - 1; i >= 1; --i) {
    int r = (int)__umul64hi(w[i], (uint64_t)(i + 1));
    int t = s[i];
    s[i] = s[r];
    s[r] = t;
  }
  int* mk = mark + (long long)j * D;
  for (int b = 0; b < J.nblk; ++b)
    for (int k = J.blk_off[b]; k < J.blk_off[b] + J.blk_n[b]; ++k) mk[s[k]] = b;
  int cur[5];
  for (int b = 0; b < J.nblk; ++b) cur[b] = J.blk_off[b];
  for (int v = 0; v < D; ++v) s[cur[mk[v]]++] = v;
}

__global__ void operm_kernel(const PermJob* jobs, int D, const double* o, const int* S,
                             double* operm) {
  const PermJob J = jobs[blockIdx.y];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < D; k += gridDim.x * blockDim.x)
    operm[J.base + k] = o[J.base + S[J.base + k]];
}

// Standard normal entries by Box-Muller (cos branch) from words 2t, 2t+1.
__global__ void gauss_kernel(const GaussJob* jobs, uint64_t seed, double* R) {
  const GaussJob J = jobs[blockIdx.x];
  const long long nn = (long long)J.n * J.n;
  for (long long t = threadIdx.x; t < nn; t += blockDim.x) {
    uint64_t w1 = rng_word(seed, P_GAUSS, J.blk, J.fid, J.comp, (uint64_t)(2 * t));
    uint64_t w2 = rng_word(seed, P_GAUSS, J.blk, J.fid, J.comp, (uint64_t)(2 * t + 1));
    double u1 = (double)((w1 >> 11) + 1) * 0x1.0p-53;
    double u2 = (double)(w2 >> 11) * 0x1.0p-53;
    double r = sqrt(-2.0 * log(u1));
    R[J.r_off + t] = r * cos(2.0 * kPi * u2);
  }
}

// Gram-Schmidt over the rows of each block (General Setup: the Gaussian
// matrix orthonormalised), modified form with a full second pass: row r is
// reduced against rows 0..r-1 one at a time, twice, then normalised.  Every
// dot product and the norm are summed sequentially in index order, each
// product rounded before it is added (this file is compiled without FMA
// contraction), so the rows are the same function of the Gaussian entries
// whatever the launch shape.  One warp per block: the lanes form the products
// and apply the updates, lane 0 adds the products in order.  Sequential by
// nature (O(n^3) dependent additions per block); setup only.  A CTA holds
// four warps, each with a block of its own, so that every warp has an FP64
// pipe to itself (one per scheduler); the largest blocks come first.
constexpr int kGsWarps = 4;
__global__ void __launch_bounds__(32 * kGsWarps) gram_schmidt_kernel(const GaussJob* jobs,
                                                                     int njobs, int max_n,
                                                                     double* Rall, int* status) {
  extern __shared__ double smem_gs[];
  const int job = blockIdx.x * kGsWarps + (threadIdx.x >> 5);
  if (job >= njobs) return;  // uniform over the warp; the kernel has no CTA barrier
  const GaussJob J = jobs[job];
  const int n = J.n;
  double* R = Rall + J.r_off;
  double* v = smem_gs + (size_t)(threadIdx.x >> 5) * 2 * max_n;  // the row being orthonormalised
  double* p = v + n;                                             // products of a dot product
  const int lane = threadIdx.x & 31;
  // sum_c p[c] in index order, starting from 0 (lane 0), sent to every lane
  auto ordered_sum = [&]() -> double {
    __syncwarp();
    double d = 0.0;
    if (lane == 0) {
#pragma unroll 8
      for (int c = 0; c < n; ++c) d = d + p[c];
    }
    d = __shfl_sync(0xffffffffu, d, 0);
    __syncwarp();
    return d;
  };
  for (int r = 0; r < n; ++r) {
    for (int c = lane; c < n; c += 32) v[c] = R[(long long)r * n + c];
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = 0; q < r; ++q) {
        const double* e = R + (long long)q * n;
        for (int c = lane; c < n; c += 32) p[c] = v[c] * e[c];
        const double d = ordered_sum();
        for (int c = lane; c < n; c += 32) v[c] = v[c] - d * e[c];
      }
    }
    for (int c = lane; c < n; c += 32) p[c] = v[c] * v[c];
    double nrm = sqrt(ordered_sum());
    if (!(nrm > 1e-10)) {  // a degenerate Gaussian draw (probability zero)
      if (lane == 0) atomicExch(status, DEV_BAD_ARG);
      nrm = 1.0;
    }
    for (int c = lane; c < n; c += 32) R[(long long)r * n + c] = v[c] / nrm;
    __syncwarp();  // row r is read back by every lane for the next rows
  }
}

// Per-variable tables: Elliptic weights (1e6)^(i/(n-1)), Different-Powers
// exponents 2 + 4 i/(n-1), Griewank divisors sqrt(i) (Sec. 3.3, 3.6, 4.3).
__global__ void aux_kernel(const AuxJob* jobs, double* aux, float* aux32) {
  const AuxJob J = jobs[blockIdx.x];
  for (int i = threadIdx.x; i < J.n; i += blockDim.x) {
    const int gi = J.gpos + i;
    double v = 0.0;
    if (J.kind == K_ELLIPTIC)
      v = (J.gn > 1) ? pow(1.0e6, (double)gi / (double)(J.gn - 1)) : 1.0;
    else if (J.kind == K_POWERS)
      v = 2.0 + ((J.gn > 1) ? 4.0 * ((double)gi / (double)(J.gn - 1)) : 0.0);
    else if (J.kind == K_GRIEWANK)
      v = sqrt((double)(gi + 1));
    aux[J.aux_off + i] = v;
    aux32[J.aux_off + i] = (float)v;
  }
}

// FP32 hi/lo words of an FP64 array: hi = fl32(v), lo = fl32(v - hi).
__global__ void split_f32_kernel(const double* src, float* hi, float* lo, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = src[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

// Column-major copies of one rotation block (FP64 and the FP32 hi/lo words)
// for the small-population kernels, whose lane i walks row i of the block:
// in the copy, the lanes of one step read consecutive addresses.
__global__ void transpose_block_kernel(long long r_off, int n, const double* R, const float* Rh,
                                       const float* Rl, double* Rt, float* Rht, float* Rlt) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e - i * n;
    Rt[r_off + j * n + i] = R[r_off + e];
    Rht[r_off + j * n + i] = Rh[r_off + e];
    Rlt[r_off + j * n + i] = Rl[r_off + e];
  }
}

}  // namespace

cudaError_t launch_transpose_block(long long r_off, int n, const double* R, const float* Rh,
                                   const float* Rl, double* Rt, float* Rht, float* Rlt,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long nn = (long long)n * n;
  const int blocks = (int)std::min<long long>((nn + 255) / 256, 1024);
  transpose_block_kernel<<<blocks, 256, 0, st>>>(r_off, n, R, Rh, Rl, Rt, Rht, Rlt);
  return cudaGetLastError();
}

cudaError_t launch_shift_perm(const PermJob* d_jobs, int njobs, int D, uint64_t seed, double* o,
                              int* S, double* operm, uint64_t* tmp_words, int* tmp_mark,
                              cudaStream_t st) {
  if (njobs == 0) return cudaSuccess;
  dim3 g((D + 255) / 256, njobs);
  shift_words_kernel<<<g, 256, 0, st>>>(d_jobs, D, seed, o, tmp_words);
  permute_kernel<<<(njobs + 63) / 64, 64, 0, st>>>(d_jobs, njobs, D, tmp_words, S, tmp_mark);
  operm_kernel<<<g, 256, 0, st>>>(d_jobs, D, o, S, operm);
  return cudaGetLastError();
}

cudaError_t launch_operm(const PermJob* d_jobs, int njobs, int D, const double* o, const int* S,
                         double* operm, cudaStream_t st) {
  if (njobs == 0) return cudaSuccess;
  dim3 g((D + 255) / 256, njobs);
  operm_kernel<<<g, 256, 0, st>>>(d_jobs, D, o, S, operm);
  return cudaGetLastError();
}

cudaError_t launch_gauss_gs(const GaussJob* d_jobs, int njobs, int max_n, uint64_t seed, double* R,
                            int* status, cudaStream_t st) {
  if (njobs == 0) return cudaSuccess;
  gauss_kernel<<<njobs, 256, 0, st>>>(d_jobs, seed, R);
  size_t smem = kGsWarps * 2 * (size_t)max_n * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gram_schmidt_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  gram_schmidt_kernel<<<(njobs + kGsWarps - 1) / kGsWarps, 32 * kGsWarps, smem, st>>>(
      d_jobs, njobs, max_n, R, status);
  return cudaGetLastError();
}

cudaError_t launch_aux(const AuxJob* d_jobs, int njobs, double* aux, float* aux32,
                       cudaStream_t st) {
  if (njobs == 0) return cudaSuccess;
  aux_kernel<<<njobs, 256, 0, st>>>(d_jobs, aux, aux32);
  return cudaGetLastError();
}

cudaError_t launch_split_f32(const double* src, float* hi, float* lo, long long n,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  split_f32_kernel<<<(int)blocks, 256, 0, st>>>(src, hi, lo, n);
  return cudaGetLastError();
}

}  // namespace curob

// curob_small32.cu -- the small-population evaluator of the FP32 path
// (curob_evaluatef for small N): compensated FP32 dot products, FP64 sums.
#define CUROB_SMALL_F32
#include "curob_small.cuh"

namespace curob {
namespace {
// One CTA per candidate, one warp per segment of the function (blockDim =
// 32 F.nseg).
__global__ void __launch_bounds__(32 * kSmallMaxWarps)
eval_small_f32_kernel(const __grid_constant__ SmallArgs a, const float* __restrict__ x, int N,
                      float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double Gs[kMaxComponents], D2s[kMaxComponents];
  const long long row = blockIdx.x;
  if (row >= N) return;  // uniform over the CTA
  const Function& F = a.F;
  const int D = a.tb.D;
  const SmallSmem L = small_smem_layout<float>(F, D);
  float* xs = reinterpret_cast<float*>(smem + L.x);
  float* U = reinterpret_cast<float*>(smem + L.z);
  float* Yh = reinterpret_cast<float*>(smem + L.y);
  float* Yl = reinterpret_cast<float*>(smem + L.yl);
  double* P = reinterpret_cast<double*>(smem + L.p);
  double* d2s = reinterpret_cast<double*>(smem + L.d2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* xr = x + row * (long long)D;
  for (int k = threadIdx.x; k < D; k += blockDim.x) xs[k] = xr[k];  // the candidate, coalesced
  __syncthreads();
  {
    const Segment& sg = a.seg[warp];
    const size_t co = (size_t)(sg.comp - F.comp0) * D;
    small_block_f32(a.tb, sg, a.comp[sg.comp - F.comp0], xs, U + co, Yh + co, Yl + co,
                    P + 4 * warp, d2s + warp);
  }
  __syncthreads();
  if (warp < F.ncomp && lane == 0) {
    double d2 = 0.0;
    Gs[warp] = small_close_f32(a, a.comp[warp], U + (size_t)warp * D, P, d2s, &d2);
    D2s[warp] = d2;
  }
  __syncthreads();
  if (warp == 0) {
    const double f = F.composition ? compose_warp(a.comp, F.ncomp, Gs, D2s, D) : Gs[0];
    if (lane == 0) out[row] = (float)(f + kFopt);
  }
}
}  // namespace

cudaError_t launch_small_f32(const SmallArgs& a, const float* x, int N, float* out,
                             cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  if (!small_supports(a.F, a.tb.D)) return cudaErrorInvalidValue;
  const size_t smem = small_smem_layout<float>(a.F, a.tb.D).total;
  cudaError_t e = cudaFuncSetAttribute(eval_small_f32_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eval_small_f32_kernel<<<N, 32 * a.F.nseg, smem, st>>>(a, x, N, out);
  return cudaGetLastError();
}
}  // namespace curob

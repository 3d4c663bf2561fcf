// curob_small32.cu -- the small-population evaluator of the FP32 path
// (curob_evaluatef for small N): compensated FP32 dot products, FP64 sums.
#define CUROB_SMALL_F32
#include "curob_small.cuh"

namespace curob {
namespace {
// One CTA per candidate, one warp per segment of the function (blockDim =
// 32 F.nseg).
__global__ void __launch_bounds__(32 * kSmallMaxWarps)
eval_small_f32_kernel(Tables tb, Function F, const float* __restrict__ x, int N,
                      float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double Gs[kMaxComponents], D2s[kMaxComponents];
  const long long row = blockIdx.x;
  if (row >= N) return;  // uniform over the CTA
  const int D = tb.D;
  const SmallSmem L = small_smem_layout<float>(F, D);
  float* U = reinterpret_cast<float*>(smem + L.z);
  float* Yh = reinterpret_cast<float*>(smem + L.y);
  float* Yl = reinterpret_cast<float*>(smem + L.yl);
  double* P = reinterpret_cast<double*>(smem + L.p);
  double* d2s = reinterpret_cast<double*>(smem + L.d2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg_base = tb.comp[F.comp0].seg0;
  const float* xr = x + row * (long long)D;
  {
    const Segment sg = tb.seg[seg_base + warp];
    const size_t co = (size_t)(sg.comp - F.comp0) * D;
    small_block_f32(tb, sg, tb.comp[sg.comp], xr, U + co, Yh + co, Yl + co, P + 4 * warp,
                    d2s + warp);
  }
  __syncthreads();
  if (warp < F.ncomp && lane == 0) {
    double d2 = 0.0;
    Gs[warp] = small_close_f32(tb, tb.comp[F.comp0 + warp], seg_base, U + (size_t)warp * D, P,
                               d2s, &d2);
    D2s[warp] = d2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double f = F.composition ? compose(tb.comp + F.comp0, F.ncomp, Gs, D2s, D) : Gs[0];
    out[row] = (float)(f + kFopt);
  }
}
}  // namespace

cudaError_t launch_small_f32(const Tables& tb, const Function& F, const float* x, int N,
                             float* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  if (!small_supports(F, tb.D)) return cudaErrorInvalidValue;
  const size_t smem = small_smem_layout<float>(F, tb.D).total;
  cudaError_t e = cudaFuncSetAttribute(eval_small_f32_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eval_small_f32_kernel<<<N, 32 * F.nseg, smem, st>>>(tb, F, x, N, out);
  return cudaGetLastError();
}
}  // namespace curob

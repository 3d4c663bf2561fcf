// curob_small64.cu -- the small-population FP64 evaluator (curob_evaluate
// for small N).  Compiled with -fmad=false, like the batched FP64 kernel:
// every expression rounds as written and the dot products take their
// explicit fma() per term in index order.
#define CUROB_SMALL_F64
#include "curob_small.cuh"

namespace curob {
namespace {
// One CTA per candidate, one warp per segment of the function (blockDim =
// 32 F.nseg).
__global__ void __launch_bounds__(32 * kSmallMaxWarps)
eval_small_f64_kernel(const __grid_constant__ SmallArgs a, const double* __restrict__ x, int N,
                      double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double Gs[kMaxComponents], D2s[kMaxComponents];
  const long long row = blockIdx.x;
  if (row >= N) return;  // uniform over the CTA
  const Function& F = a.F;
  const int D = a.tb.D;
  const SmallSmem L = small_smem_layout<double>(F, D);
  double* xs = reinterpret_cast<double*>(smem + L.x);
  double* Z = reinterpret_cast<double*>(smem + L.z);
  double* Y = reinterpret_cast<double*>(smem + L.y);
  double* Tt = reinterpret_cast<double*>(smem + L.t);
  double* d2s = reinterpret_cast<double*>(smem + L.d2);
  double* Wall = reinterpret_cast<double*>(smem + L.w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* xr = x + row * (long long)D;
  for (int k = threadIdx.x; k < D; k += blockDim.x) xs[k] = xr[k];  // the candidate, coalesced
  __syncthreads();
  {
    const Segment& sg = a.seg[warp];
    const int c = sg.comp - F.comp0;
    // the spread Weierstrass series of this warp, if its block is one
    int wi = 0;
    for (int w = 0; w < warp; ++w) wi += a.seg[w].kind == K_WEIERSTRASS ? 1 : 0;
    small_block_f64(a.tb, sg, a.comp[c], xs, Z + (size_t)c * D, Y + (size_t)c * D,
                    Tt + (size_t)c * 3 * D, Wall + (size_t)wi * kWeierK * kWeierChunk,
                    d2s + warp);
  }
  __syncthreads();
  if (warp < F.ncomp && lane == 0) {
    double d2 = 0.0;
    Gs[warp] = small_close_f64(a, a.comp[warp], Z + (size_t)warp * D, Tt + (size_t)warp * 3 * D,
                               d2s, &d2);
    D2s[warp] = d2;
  }
  __syncthreads();
  if (warp == 0) {
    const double f = F.composition ? compose_warp(a.comp, F.ncomp, Gs, D2s, D) : Gs[0];
    if (lane == 0) out[row] = f + kFopt;
  }
}
}  // namespace

bool small_supports(const Function& F, int D) {
  return F.max_n <= kSmallMaxN && F.nseg <= kSmallMaxWarps &&
         small_smem_layout<double>(F, D).total <= 160 * 1024;
}

cudaError_t launch_small_f64(const SmallArgs& a, const double* x, int N, double* out,
                             cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  if (!small_supports(a.F, a.tb.D)) return cudaErrorInvalidValue;
  const size_t smem = small_smem_layout<double>(a.F, a.tb.D).total;
  cudaError_t e = cudaFuncSetAttribute(eval_small_f64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eval_small_f64_kernel<<<N, 32 * a.F.nseg, smem, st>>>(a, x, N, out);
  return cudaGetLastError();
}
}  // namespace curob

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
eval_small_f64_kernel(Tables tb, Function F, const double* __restrict__ x, int N,
                      double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double Gs[kMaxComponents], D2s[kMaxComponents];
  const long long row = blockIdx.x;
  if (row >= N) return;  // uniform over the CTA
  const int D = tb.D;
  const SmallSmem L = small_smem_layout<double>(F, D);
  double* Z = reinterpret_cast<double*>(smem + L.z);
  double* Y = reinterpret_cast<double*>(smem + L.y);
  double* Tt = reinterpret_cast<double*>(smem + L.t);
  double* d2s = reinterpret_cast<double*>(smem + L.d2);
  double* Wall = reinterpret_cast<double*>(smem + L.w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg_base = tb.comp[F.comp0].seg0;
  const double* xr = x + row * (long long)D;
  {
    const Segment sg = tb.seg[seg_base + warp];
    const int c = sg.comp - F.comp0;
    // the spread Weierstrass series of this warp, if its block is one
    int wi = 0;
    for (int w = 0; w < warp; ++w) wi += tb.seg[seg_base + w].kind == K_WEIERSTRASS ? 1 : 0;
    small_block_f64(tb, sg, tb.comp[sg.comp], xr, Z + (size_t)c * D, Y + (size_t)c * D,
                    Tt + (size_t)c * 3 * D, Wall + (size_t)wi * kWeierK * kWeierChunk,
                    d2s + warp);
  }
  __syncthreads();
  if (warp < F.ncomp && lane == 0) {
    double d2 = 0.0;
    Gs[warp] = small_close_f64(tb, tb.comp[F.comp0 + warp], seg_base, Z + (size_t)warp * D,
                               Tt + (size_t)warp * 3 * D, d2s, &d2);
    D2s[warp] = d2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double f = F.composition ? compose(tb.comp + F.comp0, F.ncomp, Gs, D2s, D) : Gs[0];
    out[row] = f + kFopt;
  }
}
}  // namespace

bool small_supports(const Function& F, int D) {
  return F.max_n <= kSmallMaxN && F.nseg <= kSmallMaxWarps &&
         small_smem_layout<double>(F, D).total <= 160 * 1024;
}

cudaError_t launch_small_f64(const Tables& tb, const Function& F, const double* x, int N,
                             double* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  if (!small_supports(F, tb.D)) return cudaErrorInvalidValue;
  const size_t smem = small_smem_layout<double>(F, tb.D).total;
  cudaError_t e = cudaFuncSetAttribute(eval_small_f64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eval_small_f64_kernel<<<N, 32 * F.nseg, smem, st>>>(tb, F, x, N, out);
  return cudaGetLastError();
}
}  // namespace curob

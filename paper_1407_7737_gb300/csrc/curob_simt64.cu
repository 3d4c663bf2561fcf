// curob_simt64.cu -- FP64 evaluator (curob_evaluate).  Compiled with
// -fmad=false: every expression rounds exactly as written, and the rotation's
// dot products take their explicit fma() per term in index order.
#define CUROB_SIMT_F64
#include "curob_simt.cuh"

namespace curob {
cudaError_t launch_simt_f64(const Tables& tb, const Function& F, const double* x, int N,
                            double* out, cudaStream_t st) {
  return launch_simt<double, 2>(eval_simt_f64_kernel, tb, F, x, N, out, st);
}
}  // namespace curob

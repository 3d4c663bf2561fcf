// curob_simt64.cu -- FP64 evaluator (curob_evaluate).  Compiled with
// -fmad=false: every expression rounds exactly as written, and the rotation's
// dot products take their explicit fma() per term in index order.
#include "curob_simt.cuh"

namespace curob {
cudaError_t launch_simt_f64(const Tables& tb, const Function& F, const double* x, int N,
                            double* out, cudaStream_t st) {
  return launch_simt<double, double>(tb, F, x, N, out, st);
}
}  // namespace curob

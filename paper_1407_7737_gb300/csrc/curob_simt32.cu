// curob_simt32.cu -- FP32 CUDA-core evaluator (curob_evaluatef for blocks the
// tensor-core kernel does not take).  Shift in FP64, rotation and transforms
// in FP32, reductions across lanes in FP64.
#include "curob_simt.cuh"

namespace curob {
cudaError_t launch_simt_f32(const Tables& tb, const Function& F, const float* x, int N,
                            float* out, cudaStream_t st) {
  return launch_simt<float, float>(tb, F, x, N, out, st);
}
}  // namespace curob

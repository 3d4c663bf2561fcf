// curob_simt32.cu -- FP32 CUDA-core evaluator (curob_evaluatef for blocks the
// tensor-core kernel does not take, or CUROB_PRECISION_SIMT).
#define CUROB_SIMT_F32
#include "curob_simt.cuh"

namespace curob {
cudaError_t launch_simt_f32(const Tables& tb, const Function& F, const float* x, int N,
                            float* out, cudaStream_t st) {
  return launch_simt<float, 3>(eval_simt_f32_kernel, tb, F, x, N, out, st);
}
}  // namespace curob

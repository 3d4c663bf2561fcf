// curob_mma.cu -- tensor-core evaluator (not yet enabled: every function runs
// on the CUDA-core path until this module reports support).
#include "curob_mma.hpp"

namespace curob {

curob_status mma_prepare(MmaPlan& p, std::vector<Segment>& segs, const Tables& tb, float* prev) {
  (void)segs; (void)tb; (void)prev;
  p.img = nullptr;
  p.img_floats = 0;
  p.ready = false;
  return CUROB_OK;
}
curob_status mma_refresh(MmaPlan& p, const std::vector<Segment>& segs, const std::vector<int>& ids,
                         const Tables& tb) {
  (void)p; (void)segs; (void)ids; (void)tb;
  return CUROB_OK;
}
void mma_release(MmaPlan& p) {
  cudaFree(p.img);
  p.img = nullptr;
  p.ready = false;
}
bool mma_supports(const MmaPlan& p, const Function& F) { (void)F; return p.ready; }
int mma_auto_mode(const MmaPlan& p, const Function& F) { (void)p; (void)F; return CUROB_PRECISION_TF32X3; }
cudaError_t launch_mma(const MmaPlan& p, const Tables& tb, const Function& F, bool bf16,
                       const float* x, int N, float* out, cudaStream_t st) {
  (void)p; (void)tb; (void)F; (void)bf16; (void)x; (void)N; (void)out; (void)st;
  return cudaErrorNotSupported;
}

}  // namespace curob

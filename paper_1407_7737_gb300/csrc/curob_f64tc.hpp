// curob_f64tc.hpp -- the tensor-core evaluator of curob_evaluate (FP64).
#pragma once

#include <vector>

#include "../../include/curob.h"
#include "curob_internal.hpp"

namespace curob {

// Output columns of one chunk of a block (the N of one product): six FP32
// accumulators of this width fill 480 of the 512 TMEM columns.
constexpr int kF64Nw = 80;

// One chunk of output columns of one rotated block: the work of one CTA per
// tile of 128 candidates.
struct F64Chunk {
  long long b_off;  // byte offset of the chunk's digit image (K step 0) in the R digit pool
  int comp;         // component index within the function (z scratch plane)
  int zcol;         // first z column of the chunk within its component
  int nwc;          // chunk width rounded up to 16 (<= kF64Nw)
  int nvalid;       // columns of the chunk that exist
  int nk;           // K steps of 16 over the block
  int ksg;          // the block's first K step in a tile's row of the y digit image
  int sslot;        // the block's slot among its function's rotated blocks
  int rexp_off;     // exponent of the chunk's first row in the row exponent pool
  int pad_;
  double offset;    // c of the block
};

struct F64Plan {
  uint8_t* rimg = nullptr;     // BF16 digit images of every rotated block's chunks
  int* rexp = nullptr;         // power-of-two exponent of every rotated block row
  F64Chunk* chunks = nullptr;  // every function's chunks (device)
  int2* seginfo = nullptr;     // per segment: (rotated slot, first K step), slot -1 if identity
  int chunk0[kNumFunctions] = {}, nchunk[kNumFunctions] = {};
  int nrot[kNumFunctions] = {};      // rotated blocks of the function
  int ks_total[kNumFunctions] = {};  // K steps over them
  std::vector<long long> seg_img;    // host copies: per segment, digit image offset (-1 none)
  std::vector<long long> seg_rexp;   // per segment, first row exponent
  int nsm = 0;                       // persistent grid of the tensor-core launch
  bool ready = false;
};

// Lays out and fills the R digit images of every rotated block.
curob_status f64_prepare(F64Plan& p, const std::vector<Segment>& segs,
                         const std::vector<Component>& comps, const Function* funcs,
                         const bool* func_ok, const Tables& tb);
// Rebuilds the digit images of the given segments after their R changed.
curob_status f64_refresh(F64Plan& p, const std::vector<Segment>& segs, const std::vector<int>& ids,
                         const Tables& tb);
void f64_release(F64Plan& p);
// True when the tensor-core FP64 evaluator can run fid.
bool f64_supports(const F64Plan& p, int fid);
// curob_evaluate on the tensor cores: per slice of candidates, a launch that
// shifts, scales and cuts y into digits, a tensor-core launch over the
// rotated blocks (none if the function has none) and a finish launch; scratch
// taken stream-ordered from `pool` (the device's default pool if null).
cudaError_t launch_f64tc(const F64Plan& p, cudaMemPool_t pool, const Tables& tb,
                         const Function& F, int fid, const double* x, int N, double* out,
                         cudaStream_t st);
// Kernel launches launch_f64tc makes for fid at N candidates.
int f64_launch_count(const F64Plan& p, const Function& F, int fid, int D, int N);

}  // namespace curob

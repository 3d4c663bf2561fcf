// curob_instance.hpp -- one instance of the suite at a dimension D: every
// function's components, blocks and generated data (General Setup), on the
// current device.
#pragma once

#include <vector>

#include "../../include/curob.h"
#include "curob_internal.hpp"
#include "curob_f64tc.hpp"
#include "curob_mma.hpp"

namespace curob {

// Host bookkeeping for one component.
struct CompHost {
  int fid, idx;            // function and member index (RNG counter words 2, 3)
  int rotated;
  std::vector<int> sizes;  // all blocks, including empty ones, in z order
  std::vector<int> segs;   // segment ids of the non-empty blocks
};

class Instance {
 public:
  int D = 0;
  uint64_t seed = 0;
  bool func_ok[kNumFunctions] = {};
  Function func[kNumFunctions] = {};
  std::vector<Segment> segs;
  std::vector<Component> comps;
  std::vector<CompHost> chost;
  // device memory
  Segment* d_seg = nullptr;
  Component* d_comp = nullptr;
  double *d_o = nullptr, *d_operm = nullptr, *d_R = nullptr, *d_aux = nullptr;
  int* d_S = nullptr;
  float *d_R32 = nullptr, *d_R32lo = nullptr, *d_aux32 = nullptr;
  double* d_Rt = nullptr;  // column-major copies of the blocks
  float *d_R32t = nullptr, *d_R32lot = nullptr;
  int* d_status = nullptr;
  long long r_total = 0, aux_total = 0;
  MmaPlan mma;  // tensor-core operand images
  F64Plan f64;  // digit images of the tensor-core FP64 evaluator

  // Builds every function's instance for (D, seed) on the current device.
  curob_status create(int D, uint64_t seed);
  void release();
  bool ready() const { return d_seg != nullptr; }
  Tables tables() const;
  int find_comp(int fid, int comp) const;
  // Copies component data in / out (host pointers, layout of curob.h).
  curob_status get_component(int fid, int comp, double* o, int* S, double* R) const;
  curob_status set_component(int fid, int comp, const double* o, const int* S, const double* R);

 private:
  void build_tables();
  curob_status generate_all();
};

bool needs_d10(int fid);

// The small-population kernels' by-value copy of a function's segments and
// components (curob_small.cuh).
void fill_small_args(SmallArgs& a, const Instance& I, const Function& F);

}  // namespace curob

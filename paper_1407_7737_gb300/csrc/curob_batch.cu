// curob_batch.cu -- ragged batches (include/curob.h, curob_batch_*): many
// (function, D, seed, population) items evaluated by persistent tensor-core
// launches, scheduled by a small autotuner and replayed from a CUDA graph.
//
// Each item takes the precision curob_evaluatef's AUTO rule gives its
// function: TF32X3 where no kind magnifies contraction error, EXACT otherwise
// (a composition whose members differ runs whole on EXACT, and so does a
// function with blocks narrower than 16, which AUTO sends to the CUDA-core
// kernel).  The items of each precision form one persistent launch.  The
// tuner times three work orders per launch on a full grid, then whether the
// two launches run one after the other or side by side on a split of the SMs
// (the split from the estimated costs, and its two neighbours), and against
// them one launch with every item on EXACT (which meets the FP32 bar
// everywhere); it keeps the fastest and captures it in a CUDA graph.
#include <algorithm>
#include <map>
#include <memory>
#include <numeric>
#include <utility>
#include <vector>

#include "../../include/curob.h"
#include "curob_instance.hpp"
#include "curob_mma.hpp"
#include "curob_small.cuh"

namespace curob {
bool device_accessible(const void* p);
}

using namespace curob;

namespace {
constexpr int kGroups = 2;        // 0: EXACT items, 1: TF32X3 items (2: every item on EXACT)
constexpr int kSmallAuto = 512;   // AUTO's small-population limit (curob_set_small_batch default)

struct Group {
  int mode = CUROB_PRECISION_EXACT;
  std::vector<int2> work_host[3];  // (item, tile) in each candidate order
  int2* d_work[3] = {nullptr, nullptr, nullptr};
  int nwork = 0;
  int* d_counter = nullptr;
  int npad_max = 32;               // widest block of the group's items, rounded up to 32
  double cost = 0.0;               // estimated cost of the group's tiles
  int order = 0, grid = 0;
};
}  // namespace

struct curob_batch_st {
  std::vector<curob_batch_item> items;
  std::map<std::pair<int, uint64_t>, std::unique_ptr<Instance>> inst;
  std::vector<Instance*> item_inst;
  std::vector<int> item_group;       // 0 EXACT, 1 TF32X3
  std::vector<double> tile_cost;     // estimated cost of one tile of each item
  std::vector<SmallArgs> small;      // per item, for curob_batch_run_auto
  Group grp[kGroups + 1];
  void* d_args = nullptr;            // per item, at its group's precision
  void* d_args_all = nullptr;        // per item, on EXACT (group 2)
  int all_exact = 0;                 // the tuner chose group 2
  int nsm = 0;
  bool tuned = false;
  int concurrent = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t priv = nullptr, priv2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

namespace {

bool heavy_kind(int k) {
  return k == K_POWERS || k == K_WEIERSTRASS || k == K_GRIEWANK || k == K_SCHAFFER7 ||
         k == K_EGR || k == K_SCHWEFEL || k == K_KATSUURA || k == K_SCHAFFER6;
}

// Cost of one 128-candidate tile: tensor work (npad^2 per block and
// product: 10 on EXACT, 3 on TF32X3) plus the epilogue's per-variable work
// (heavier for transcendental kinds).
double tile_cost(const Instance& I, int fid, int group) {
  const Function& F = I.func[fid];
  const double prod = group == 0 ? 10.0 : 3.0;
  double c = 0.0;
  for (int ci = 0; ci < F.ncomp; ++ci) {
    const Component& C = I.comps[F.comp0 + ci];
    for (int si = 0; si < C.nseg; ++si) {
      const Segment& s = I.segs[C.seg0 + si];
      const int npad = (s.n + 31) / 32 * 32;
      c += (double)npad * npad * prod / 64.0 + (double)s.n * (heavy_kind(s.kind) ? 40.0 : 4.0);
    }
  }
  return c;
}

void free_batch(curob_batch b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->priv) cudaStreamDestroy(b->priv);
  if (b->priv2) cudaStreamDestroy(b->priv2);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  cudaFree(b->d_args);
  cudaFree(b->d_args_all);
  for (Group& g : b->grp) {
    for (int o = 0; o < 3; ++o) cudaFree(g.d_work[o]);
    cudaFree(g.d_counter);
  }
  for (auto& kv : b->inst) kv.second->release();
  delete b;
}

cudaError_t launch_group(curob_batch b, int gi, int order, int grid, cudaStream_t st) {
  Group& g = b->grp[gi];
  cudaError_t e = cudaMemsetAsync(g.d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return launch_mma_batch(gi == kGroups ? b->d_args_all : b->d_args, g.d_work[order], g.nwork,
                          g.d_counter,
                          std::min(grid, std::max(1, g.nwork)), st, g.mode, g.npad_max);
}

// Issues a schedule on b->priv: the groups in sequence, or side by side (the
// TF32X3 group on priv2, forked from and joined back into priv).
cudaError_t issue(curob_batch b, const int* order, const int* grid, bool concurrent,
                  int all_order = -1) {
  if (all_order >= 0) return launch_group(b, kGroups, all_order, b->nsm, b->priv);
  const bool both = b->grp[0].nwork > 0 && b->grp[1].nwork > 0;
  cudaError_t e = cudaSuccess;
  if (concurrent && both) {
    e = cudaEventRecord(b->fork, b->priv);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->priv2, b->fork, 0);
    if (e == cudaSuccess) e = launch_group(b, 0, order[0], grid[0], b->priv);
    if (e == cudaSuccess) e = launch_group(b, 1, order[1], grid[1], b->priv2);
    if (e == cudaSuccess) e = cudaEventRecord(b->join, b->priv2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->priv, b->join, 0);
    return e;
  }
  for (int gi = 0; gi < kGroups && e == cudaSuccess; ++gi)
    if (b->grp[gi].nwork > 0) e = launch_group(b, gi, order[gi], grid[gi], b->priv);
  return e;
}

// Time one schedule (ms): two runs, the second measured.
float time_schedule(curob_batch b, const int* order, const int* grid, bool concurrent,
                    int all_order = -1) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = -1.f;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0, b->priv);
    if (issue(b, order, grid, concurrent, all_order) != cudaSuccess) {
      ms = -1.f;
      break;
    }
    cudaEventRecord(e1, b->priv);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

curob_status tune_and_capture(curob_batch b) {
  int order[kGroups] = {0, 0}, grid[kGroups] = {b->nsm, b->nsm};
  // the work order of each launch, alone on a full grid
  for (int gi = 0; gi < kGroups; ++gi) {
    if (b->grp[gi].nwork == 0) continue;
    float best = 1e30f;
    int sel[kGroups] = {0, 0};
    for (int o = 0; o < 3; ++o) {
      sel[gi] = o;
      const int saved = b->grp[1 - gi].nwork;
      b->grp[1 - gi].nwork = 0;  // time this launch alone
      const float ms = time_schedule(b, sel, grid, false);
      b->grp[1 - gi].nwork = saved;
      if (ms < 0.f) return CUROB_ERR_CUDA;
      if (ms < best) {
        best = ms;
        order[gi] = o;
      }
    }
  }
  // one after the other on full grids, or side by side on a split
  float best = time_schedule(b, order, grid, false);
  if (best < 0.f) return CUROB_ERR_CUDA;
  b->concurrent = 0;
  b->grp[0].grid = grid[0];
  b->grp[1].grid = grid[1];
  if (b->grp[0].nwork > 0 && b->grp[1].nwork > 0 && b->nsm >= 4) {
    const double share = b->grp[0].cost / std::max(1e-30, b->grp[0].cost + b->grp[1].cost);
    const int g0 = (int)(share * b->nsm + 0.5);
    const int step = std::max(1, b->nsm / 8);
    for (int cand : {g0, g0 - step, g0 + step}) {
      const int gE = std::min(b->nsm - 1, std::max(1, cand));
      const int split[kGroups] = {gE, b->nsm - gE};
      const float ms = time_schedule(b, order, split, true);
      if (ms < 0.f) return CUROB_ERR_CUDA;
      if (ms < best) {
        best = ms;
        b->concurrent = 1;
        b->grp[0].grid = split[0];
        b->grp[1].grid = split[1];
      }
    }
  }
  b->grp[0].order = order[0];
  b->grp[1].order = order[1];
  // every item on EXACT, one launch
  b->all_exact = 0;
  if (b->grp[1].nwork > 0) {
    for (int o = 0; o < 3; ++o) {
      const float ms = time_schedule(b, order, grid, false, o);
      if (ms < 0.f) return CUROB_ERR_CUDA;
      if (ms < best) {
        best = ms;
        b->all_exact = 1;
        b->grp[kGroups].order = o;
        b->grp[kGroups].grid = b->nsm;
      }
    }
  }
  const int g[kGroups] = {b->grp[0].grid, b->grp[1].grid};
  if (cudaStreamBeginCapture(b->priv, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return CUROB_ERR_CUDA;
  const cudaError_t e = issue(b, order, g, b->concurrent != 0,
                              b->all_exact ? b->grp[kGroups].order : -1);
  if (cudaStreamEndCapture(b->priv, &b->graph) != cudaSuccess || e != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return CUROB_ERR_CUDA;
  b->tuned = true;
  return CUROB_OK;
}

}  // namespace

extern "C" {

curob_status curob_batch_create(const curob_batch_item* items, int n_items, curob_batch* batch) {
  if (!items || !batch) return CUROB_ERR_NULL_POINTER;
  if (n_items < 1) return CUROB_ERR_INVALID_ARGUMENT;
  *batch = nullptr;
  for (int i = 0; i < n_items; ++i) {
    const curob_batch_item& it = items[i];
    if (it.fid < 0 || it.fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
    if (it.D < 2 || (needs_d10(it.fid) && it.D < 10)) return CUROB_ERR_INVALID_DIM;
    if (it.N < 0) return CUROB_ERR_INVALID_ARGUMENT;
    if (it.N > 0) {
      if (!it.x || !it.out) return CUROB_ERR_NULL_POINTER;
      if (!device_accessible(it.x) || !device_accessible(it.out))
        return CUROB_ERR_INVALID_ARGUMENT;
    }
  }
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CUROB_ERR_CUDA;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major != 10) return CUROB_ERR_UNSUPPORTED;
  curob_batch b = new curob_batch_st();
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  b->items.assign(items, items + n_items);
  b->grp[0].mode = CUROB_PRECISION_EXACT;
  b->grp[1].mode = CUROB_PRECISION_TF32X3;
  b->small.resize(n_items);
  curob_status rc = CUROB_OK;
  for (int i = 0; i < n_items; ++i) {
    const curob_batch_item& it = b->items[i];
    auto key = std::make_pair(it.D, it.seed);
    if (!b->inst.count(key)) {
      std::unique_ptr<Instance> I(new Instance());
      rc = I->create(it.D, it.seed);
      if (rc != CUROB_OK) break;
      b->inst[key] = std::move(I);
    }
    Instance* I = b->inst[key].get();
    const Function& F = I->func[it.fid];
    if (F.max_n > mma_max_block()) {
      rc = CUROB_ERR_UNSUPPORTED;
      break;
    }
    // AUTO's precision; MIXED compositions and blocks AUTO leaves to the
    // CUDA cores go to EXACT
    const int gi = (mma_supports(I->mma, F) &&
                    mma_auto_mode(I->mma, F) == CUROB_PRECISION_TF32X3) ? 1 : 0;
    b->item_inst.push_back(I);
    b->item_group.push_back(gi);
    b->tile_cost.push_back(tile_cost(*I, it.fid, gi));
    fill_small_args(b->small[i], *I, F);
    Group& g = b->grp[gi];
    g.npad_max = std::max(g.npad_max, (F.max_n + 31) / 32 * 32);
  }
  if (rc != CUROB_OK) {
    free_batch(b);
    return rc;
  }
  // argument blocks (each in its group's precision and stage geometry) and
  // the three candidate work orders of each group
  const size_t ab = mma_args_bytes();
  std::vector<unsigned char> args(ab * n_items);
  std::vector<int> tiles(n_items);
  for (int i = 0; i < n_items; ++i) {
    const curob_batch_item& it = b->items[i];
    Instance* I = b->item_inst[i];
    Group& g = b->grp[b->item_group[i]];
    mma_fill_args(args.data() + ab * i, I->mma, I->tables(), I->func[it.fid], it.x, it.out, it.N,
                  g.mode, g.npad_max);
    tiles[i] = (it.N + 127) / 128;
    for (int t = 0; t < tiles[i]; ++t) g.work_host[2].push_back(make_int2(i, t));
    g.cost += b->tile_cost[i] * tiles[i];
  }
  {  // group 2: every item on EXACT, same tiles
    Group& g = b->grp[kGroups];
    g.mode = CUROB_PRECISION_EXACT;
    for (int i = 0; i < n_items; ++i) {
      for (int t = 0; t < tiles[i]; ++t) g.work_host[2].push_back(make_int2(i, t));
      g.cost += tile_cost(*b->item_inst[i], b->items[i].fid, 0) * tiles[i];
    }
  }
  for (Group& g : b->grp) {
    g.nwork = (int)g.work_host[2].size();
    g.work_host[0] = g.work_host[2];  // longest tile first
    std::stable_sort(g.work_host[0].begin(), g.work_host[0].end(),
                     [&](int2 a, int2 c) { return b->tile_cost[a.x] > b->tile_cost[c.x]; });
  }
  for (int t = 0;; ++t) {  // round robin over items
    bool any = false;
    for (int i = 0; i < n_items; ++i)
      if (t < tiles[i]) {
        b->grp[b->item_group[i]].work_host[1].push_back(make_int2(i, t));
        b->grp[kGroups].work_host[1].push_back(make_int2(i, t));
        any = true;
      }
    if (!any) break;
  }
  std::vector<unsigned char> args_all(ab * n_items);
  for (int i = 0; i < n_items; ++i) {
    const curob_batch_item& it = b->items[i];
    Instance* I = b->item_inst[i];
    mma_fill_args(args_all.data() + ab * i, I->mma, I->tables(), I->func[it.fid], it.x, it.out,
                  it.N, CUROB_PRECISION_EXACT, b->grp[kGroups].npad_max);
  }
  bool ok = cudaMalloc(&b->d_args, args.size()) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->priv, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->priv2, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) == cudaSuccess;
  for (Group& g : b->grp) {
    ok = ok && cudaMalloc(&g.d_counter, sizeof(int)) == cudaSuccess;
    for (int o = 0; o < 3 && ok; ++o)
      ok = cudaMalloc(&g.d_work[o], sizeof(int2) * std::max(g.nwork, 1)) == cudaSuccess &&
           (g.nwork == 0 || cudaMemcpy(g.d_work[o], g.work_host[o].data(),
                                       sizeof(int2) * g.nwork, cudaMemcpyHostToDevice) ==
                                cudaSuccess);
  }
  ok = ok && cudaMemcpy(b->d_args, args.data(), args.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_args_all, args_all.size()) == cudaSuccess &&
       cudaMemcpy(b->d_args_all, args_all.data(), args_all.size(), cudaMemcpyHostToDevice) ==
           cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_batch(b);
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  *batch = b;
  return CUROB_OK;
}

curob_status curob_batch_run(curob_batch b, curob_stream_t stream) {
  if (!b) return CUROB_ERR_NULL_POINTER;
  if (b->grp[kGroups].nwork == 0) return CUROB_OK;
  if (!b->tuned) {
    curob_status rc = tune_and_capture(b);
    if (rc != CUROB_OK) return rc;
  }
  return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? CUROB_OK : CUROB_ERR_CUDA;
}

curob_status curob_batch_run_separate(curob_batch b, curob_stream_t stream) {
  if (!b) return CUROB_ERR_NULL_POINTER;
  for (size_t i = 0; i < b->items.size(); ++i) {
    const curob_batch_item& it = b->items[i];
    if (it.N == 0) continue;
    Instance* I = b->item_inst[i];
    const int mode = b->all_exact ? CUROB_PRECISION_EXACT : b->grp[b->item_group[i]].mode;
    if (launch_mma_fused(I->mma, I->tables(), I->func[it.fid], mode, it.x, it.N, it.out,
                         (cudaStream_t)stream) != cudaSuccess)
      return CUROB_ERR_CUDA;
  }
  return CUROB_OK;
}

curob_status curob_batch_run_auto(curob_batch b, curob_stream_t stream) {
  if (!b) return CUROB_ERR_NULL_POINTER;
  const cudaStream_t st = (cudaStream_t)stream;
  for (size_t i = 0; i < b->items.size(); ++i) {
    const curob_batch_item& it = b->items[i];
    if (it.N == 0) continue;
    Instance* I = b->item_inst[i];
    const Function& F = I->func[it.fid];
    cudaError_t e;
    if (it.N <= kSmallAuto && small_supports(F, I->D)) {
      e = launch_small_f32(b->small[i], it.x, it.N, it.out, st);
    } else {
      const int m = mma_supports(I->mma, F) ? mma_auto_mode(I->mma, F) : CUROB_PRECISION_SIMT;
      if (m == CUROB_PRECISION_SIMT)
        e = launch_simt_f32(I->tables(), F, it.x, it.N, it.out, st);
      else if (m == CUROB_PRECISION_MIXED)
        e = launch_mma_mixed(I->mma, I->tables(), F, it.x, it.N, it.out, st);
      else
        e = launch_mma(I->mma, I->tables(), F, m, it.x, it.N, it.out, st);
    }
    if (e != cudaSuccess) return CUROB_ERR_CUDA;
  }
  return CUROB_OK;
}

curob_status curob_batch_schedule(curob_batch b, int* n_work, int* grid, int* order) {
  if (!b) return CUROB_ERR_NULL_POINTER;
  if (!b->tuned) return CUROB_ERR_NOT_INITIALIZED;
  const int big = b->all_exact ? kGroups : (b->grp[1].cost > b->grp[0].cost ? 1 : 0);
  if (n_work) *n_work = b->grp[kGroups].nwork;
  if (grid)
    *grid = b->all_exact ? b->grp[kGroups].grid
            : b->concurrent ? b->grp[0].grid + b->grp[1].grid
                            : std::max(b->grp[0].nwork ? b->grp[0].grid : 0,
                                       b->grp[1].nwork ? b->grp[1].grid : 0);
  if (order) *order = b->grp[big].order;
  return CUROB_OK;
}

curob_status curob_batch_plan(curob_batch b, int* items_exact, int* items_tf32, int* work_exact,
                              int* work_tf32, int* grid_exact, int* grid_tf32, int* order_exact,
                              int* order_tf32, int* concurrent) {
  if (!b) return CUROB_ERR_NULL_POINTER;
  if (!b->tuned) return CUROB_ERR_NOT_INITIALIZED;
  int ne = 0, nt = 0;
  for (int gi : b->item_group) (gi && !b->all_exact ? nt : ne) += 1;
  const Group& ge = b->grp[b->all_exact ? kGroups : 0];
  const Group& gt = b->grp[1];
  if (items_exact) *items_exact = ne;
  if (items_tf32) *items_tf32 = nt;
  if (work_exact) *work_exact = ge.nwork;
  if (work_tf32) *work_tf32 = b->all_exact ? 0 : gt.nwork;
  if (grid_exact) *grid_exact = ge.nwork ? ge.grid : 0;
  if (grid_tf32) *grid_tf32 = (!b->all_exact && gt.nwork) ? gt.grid : 0;
  if (order_exact) *order_exact = ge.order;
  if (order_tf32) *order_tf32 = gt.order;
  if (concurrent) *concurrent = b->all_exact ? 0 : b->concurrent;
  return CUROB_OK;
}

curob_status curob_batch_status(curob_batch b, curob_stream_t stream) {
  if (!b) return CUROB_ERR_NULL_POINTER;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CUROB_ERR_CUDA;
  curob_status rc = CUROB_OK;
  for (auto& kv : b->inst) {
    int st = 0;
    if (cudaMemcpy(&st, kv.second->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return CUROB_ERR_CUDA;
    if (st != DEV_OK) {
      cudaMemset(kv.second->d_status, 0, sizeof(int));
      rc = (st == DEV_TIMEOUT) ? CUROB_ERR_DEVICE_TIMEOUT : CUROB_ERR_CUDA;
    }
  }
  return rc;
}

curob_status curob_batch_destroy(curob_batch b) {
  if (!b) return CUROB_ERR_NULL_POINTER;
  cudaDeviceSynchronize();
  free_batch(b);
  return CUROB_OK;
}

}  // extern "C"

// curob_batch.cu -- ragged batches (include/curob.h, curob_batch_*): many
// (function, D, seed, population) items evaluated by one persistent
// tensor-core launch, scheduled by a small autotuner and replayed from a
// CUDA graph.
#include <algorithm>
#include <map>
#include <memory>
#include <numeric>
#include <utility>
#include <vector>

#include "../../include/curob.h"
#include "curob_instance.hpp"
#include "curob_mma.hpp"

namespace curob {
bool device_accessible(const void* p);
}

using namespace curob;

struct curob_batch_st {
  std::vector<curob_batch_item> items;
  std::map<std::pair<int, uint64_t>, std::unique_ptr<Instance>> inst;
  std::vector<Instance*> item_inst;
  std::vector<double> tile_cost;     // estimated cost of one tile of each item
  std::vector<int2> work_host[3];    // (item, tile) in each candidate order
  int nwork = 0;
  void* d_args = nullptr;
  int2* d_work[3] = {nullptr, nullptr, nullptr};
  int* d_counter = nullptr;
  int nsm = 0;
  bool tuned = false;
  int grid = 0, order = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t priv = nullptr;
};

namespace {

bool heavy_kind(int k) {
  return k == K_POWERS || k == K_WEIERSTRASS || k == K_GRIEWANK || k == K_SCHAFFER7 ||
         k == K_EGR || k == K_SCHWEFEL || k == K_KATSUURA || k == K_SCHAFFER6;
}

// Cost of one 128-candidate tile: tensor work (npad^2 per block and N chunk
// pass) plus the epilogue's per-variable work (heavier for transcendental
// kinds).
double tile_cost(const Instance& I, int fid) {
  const Function& F = I.func[fid];
  double c = 0.0;
  for (int ci = 0; ci < F.ncomp; ++ci) {
    const Component& C = I.comps[F.comp0 + ci];
    for (int si = 0; si < C.nseg; ++si) {
      const Segment& s = I.segs[C.seg0 + si];
      const int npad = (s.n + 31) / 32 * 32;
      c += (double)npad * npad * 10.0 / 64.0 + (double)s.n * (heavy_kind(s.kind) ? 40.0 : 4.0);
    }
  }
  return c;
}

void free_batch(curob_batch b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->priv) cudaStreamDestroy(b->priv);
  cudaFree(b->d_args);
  for (int o = 0; o < 3; ++o) cudaFree(b->d_work[o]);
  cudaFree(b->d_counter);
  for (auto& kv : b->inst) kv.second->release();
  delete b;
}

// Time one schedule (ms), two launches, the second measured.
float time_schedule(curob_batch b, int order, int grid) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = -1.f;
  for (int rep = 0; rep < 2; ++rep) {
    cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->priv);
    cudaEventRecord(e0, b->priv);
    if (launch_mma_batch(b->d_args, b->d_work[order], b->nwork, b->d_counter, grid, b->priv) !=
        cudaSuccess) {
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
  const int grids[2] = {b->nsm, std::max(1, b->nsm * 3 / 4)};
  float best = 1e30f;
  for (int order = 0; order < 3; ++order)
    for (int gi = 0; gi < 2; ++gi) {
      const int grid = std::min(grids[gi], std::max(1, b->nwork));
      const float ms = time_schedule(b, order, grid);
      if (ms < 0.f) return CUROB_ERR_CUDA;
      if (ms < best) {
        best = ms;
        b->order = order;
        b->grid = grid;
      }
    }
  if (cudaStreamBeginCapture(b->priv, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return CUROB_ERR_CUDA;
  cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->priv);
  launch_mma_batch(b->d_args, b->d_work[b->order], b->nwork, b->d_counter, b->grid, b->priv);
  if (cudaStreamEndCapture(b->priv, &b->graph) != cudaSuccess) return CUROB_ERR_CUDA;
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
  curob_status rc = CUROB_OK;
  for (const curob_batch_item& it : b->items) {
    auto key = std::make_pair(it.D, it.seed);
    if (!b->inst.count(key)) {
      std::unique_ptr<Instance> I(new Instance());
      rc = I->create(it.D, it.seed);
      if (rc != CUROB_OK) break;
      b->inst[key] = std::move(I);
    }
    Instance* I = b->inst[key].get();
    if (I->func[it.fid].max_n > mma_max_block()) {
      rc = CUROB_ERR_UNSUPPORTED;
      break;
    }
    b->item_inst.push_back(I);
    b->tile_cost.push_back(tile_cost(*I, it.fid));
  }
  if (rc != CUROB_OK) {
    free_batch(b);
    return rc;
  }
  // argument blocks and the three candidate work orders
  const size_t ab = mma_args_bytes();
  std::vector<unsigned char> args(ab * n_items);
  std::vector<int> tiles(n_items);
  for (int i = 0; i < n_items; ++i) {
    const curob_batch_item& it = b->items[i];
    Instance* I = b->item_inst[i];
    mma_fill_args(args.data() + ab * i, I->mma, I->tables(), I->func[it.fid], it.x, it.out, it.N);
    tiles[i] = (it.N + 127) / 128;
    for (int t = 0; t < tiles[i]; ++t) b->work_host[2].push_back(make_int2(i, t));
  }
  b->nwork = (int)b->work_host[2].size();
  b->work_host[0] = b->work_host[2];  // longest tile first
  std::stable_sort(b->work_host[0].begin(), b->work_host[0].end(),
                   [&](int2 a, int2 c) { return b->tile_cost[a.x] > b->tile_cost[c.x]; });
  for (int t = 0;; ++t) {  // round robin over items
    bool any = false;
    for (int i = 0; i < n_items; ++i)
      if (t < tiles[i]) {
        b->work_host[1].push_back(make_int2(i, t));
        any = true;
      }
    if (!any) break;
  }
  bool ok = cudaMalloc(&b->d_args, args.size()) == cudaSuccess &&
            cudaMalloc(&b->d_counter, sizeof(int)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->priv, cudaStreamNonBlocking) == cudaSuccess;
  for (int o = 0; o < 3 && ok; ++o)
    ok = cudaMalloc(&b->d_work[o], sizeof(int2) * std::max(b->nwork, 1)) == cudaSuccess &&
         (b->nwork == 0 || cudaMemcpy(b->d_work[o], b->work_host[o].data(),
                                      sizeof(int2) * b->nwork, cudaMemcpyHostToDevice) ==
                               cudaSuccess);
  ok = ok && cudaMemcpy(b->d_args, args.data(), args.size(), cudaMemcpyHostToDevice) == cudaSuccess;
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
  if (b->nwork == 0) return CUROB_OK;
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
    if (launch_mma_fused(I->mma, I->tables(), I->func[it.fid], CUROB_PRECISION_EXACT, it.x,
                         it.N, it.out, (cudaStream_t)stream) != cudaSuccess)
      return CUROB_ERR_CUDA;
  }
  return CUROB_OK;
}

curob_status curob_batch_schedule(curob_batch b, int* n_work, int* grid, int* order) {
  if (!b) return CUROB_ERR_NULL_POINTER;
  if (!b->tuned) return CUROB_ERR_NOT_INITIALIZED;
  if (n_work) *n_work = b->nwork;
  if (grid) *grid = b->grid;
  if (order) *order = b->order;
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

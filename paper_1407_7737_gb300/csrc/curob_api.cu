// curob_api.cu -- the C ABI of libcurob (include/curob.h): the library's
// instance (initialize/dispose, Sec. 1.3 "Interface"), evaluation entry
// points and the instance-data accessors.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/curob.h"
#include "curob_instance.hpp"
#include "curob_internal.hpp"
#include "curob_mma.hpp"
#include "curob_small.cuh"

namespace curob {
namespace {

// Default population limit of the small-population kernels (one warp per
// candidate and component): below it a call is latency-bound and they finish
// first; above it the batched kernels' throughput wins.
constexpr int kSmallBatchDefault = 512;

struct State {
  std::mutex mu;
  bool init = false;
  int max_conc = 0;
  int device = 0;
  int precision = CUROB_PRECISION_AUTO;
  int precision64 = CUROB_PRECISION64_AUTO;
  int small_batch = kSmallBatchDefault;  // calls with N <= this take the small kernels
  Instance inst;
  void* d_hx = nullptr;   // host-wrapper staging (max_conc x D doubles)
  void* d_hout = nullptr; // (max_conc doubles)
  cudaStream_t hstream = nullptr;         // host wrappers: chunk 0's stream
  cudaStream_t hside[3] = {};             // and the other chunks' streams
  SmallArgs small[kNumFunctions];         // launch arguments of the small kernels
};

// Host wrappers cut a call into up to kHostChunks chunks of whole 128-row
// tiles, each on its own stream (copy in, evaluate, copy out), so that a
// chunk's copy-in overlaps the kernels of the chunks before it.
constexpr int kHostChunks = 4;
constexpr int kHostMinChunk = 1024;  // candidates: smaller calls stay one chunk

State g;

Tables tables() { return g.inst.tables(); }

void free_all() {
  g.inst.release();
  cudaFree(g.d_hx);
  cudaFree(g.d_hout);
  if (g.hstream) cudaStreamDestroy(g.hstream);
  for (cudaStream_t& s : g.hside) {
    if (s) cudaStreamDestroy(s);
    s = nullptr;
  }
  g.d_hx = g.d_hout = nullptr;
  g.hstream = nullptr;
  g.init = false;
}

cudaStream_t host_stream(int k) { return k == 0 ? g.hstream : g.hside[k - 1]; }

// Copy in, evaluate (eval(x_dev, n, out_dev, stream) on each chunk), copy
// out, then wait for every chunk.  T is the element type of x and out.
template <typename T, typename Eval>
curob_status host_pipeline(const T* x, int N, T* out, Eval eval) {
  const int D = g.inst.D;
  int chunks = std::min(kHostChunks, std::max(1, N / kHostMinChunk));
  const int per = ((N + chunks - 1) / chunks + 127) / 128 * 128;
  chunks = (N + per - 1) / per;
  T* dx = static_cast<T*>(g.d_hx);
  T* dout = static_cast<T*>(g.d_hout);
  curob_status rc = CUROB_OK;
  int issued = 0;
  for (int k = 0; k < chunks && rc == CUROB_OK; ++k, ++issued) {
    const size_t r0 = (size_t)k * per;
    const int n = (int)std::min<size_t>(per, (size_t)N - r0);
    cudaStream_t st = host_stream(k);
    if (cudaMemcpyAsync(dx + r0 * D, x + r0 * D, sizeof(T) * (size_t)n * D,
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = CUROB_ERR_CUDA;
      break;
    }
    rc = eval(dx + r0 * D, n, dout + r0, st);
    if (rc == CUROB_OK && cudaMemcpyAsync(out + r0, dout + r0, sizeof(T) * (size_t)n,
                                          cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = CUROB_ERR_CUDA;
  }
  for (int k = 0; k < issued; ++k)  // nothing may still use the staging after return
    if (cudaStreamSynchronize(host_stream(k)) != cudaSuccess && rc == CUROB_OK)
      rc = CUROB_ERR_CUDA;
  return rc;
}

curob_status check_eval_args(int fid, const void* x, int N, const void* out) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  if (!g.inst.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
  if (N < 0) return CUROB_ERR_INVALID_ARGUMENT;
  if (N > g.max_conc) return CUROB_ERR_CAPACITY;
  if (N == 0) return CUROB_OK;
  if (!x || !out) return CUROB_ERR_NULL_POINTER;
  return CUROB_OK;
}

// The precision curob_evaluatef uses for F (AUTO resolved), or -1 when a
// forced tensor-core precision cannot take F's block sizes.
int resolve_precision(const Function& F) {
  int mode = g.precision;
  const bool mma_ok = mma_supports(g.inst.mma, F);
  const bool tc = mode == CUROB_PRECISION_TF32X3 || mode == CUROB_PRECISION_BF16X3 ||
                  mode == CUROB_PRECISION_EXACT || mode == CUROB_PRECISION_FP16X3;
  if (tc && !mma_ok) return -1;
  if (mode == CUROB_PRECISION_AUTO)
    mode = mma_ok ? mma_auto_mode(g.inst.mma, F) : CUROB_PRECISION_SIMT;
  return mode;
}

// The path curob_evaluate takes for fid at N candidates beyond the small
// kernels: CUROB_PRECISION64_TENSOR or _SIMT, or -1 when the tensor cores are
// forced but unavailable.
int resolve_precision64(int fid) {
  const bool tc = f64_supports(g.inst.f64, fid);
  if (g.precision64 == CUROB_PRECISION64_TENSOR) return tc ? CUROB_PRECISION64_TENSOR : -1;
  if (g.precision64 == CUROB_PRECISION64_SIMT) return CUROB_PRECISION64_SIMT;
  return tc ? CUROB_PRECISION64_TENSOR : CUROB_PRECISION64_SIMT;
}

bool use_small(const Function& F, int N);

// curob_evaluate's kernels for one batch already on the device.
curob_status eval64(int fid, const double* x, int n, double* out, cudaStream_t st) {
  const Function& F = g.inst.func[fid];
  cudaError_t e;
  if (use_small(F, n)) {
    e = launch_small_f64(g.small[fid], x, n, out, st);
  } else {
    const int path = resolve_precision64(fid);
    if (path < 0) return CUROB_ERR_UNSUPPORTED;
    e = path == CUROB_PRECISION64_TENSOR
            ? launch_f64tc(g.inst.f64, g.inst.mma.pool, tables(), F, fid, x, n, out, st)
            : launch_simt_f64(tables(), F, x, n, out, st);
  }
  return e == cudaSuccess ? CUROB_OK : CUROB_ERR_CUDA;
}

// The small kernels' by-value copy of a function's segments and components.
void make_small_args(SmallArgs& a, const Function& F) { fill_small_args(a, g.inst, F); }

// A call of N candidates takes the small-population kernels (FP64, and the
// FP32 path under AUTO) when N is within the limit and every block fits them.
bool use_small(const Function& F, int N) {
  return N <= g.small_batch && small_supports(F, g.inst.D);
}

// The instance's tables live on the device curob_initialize ran on: a
// kernel launched on another device would read them through a pointer that
// device cannot use and fault, so every evaluation requires that device to
// be current.
bool on_instance_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return dev == g.device;
}

}  // namespace

// A kernel given a pointer the GPU cannot reach would fault the context, so
// evaluations accept device memory of the instance's device, or managed
// memory, only.
bool device_accessible(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && (!g.init || a.device == g.device);
}

}  // namespace curob

using namespace curob;

extern "C" {

const char* curob_status_string(curob_status s) {
  switch (s) {
    case CUROB_OK: return "ok";
    case CUROB_ERR_NOT_INITIALIZED: return "not initialized";
    case CUROB_ERR_ALREADY_INITIALIZED: return "already initialized";
    case CUROB_ERR_INVALID_FID: return "invalid function id";
    case CUROB_ERR_INVALID_DIM: return "invalid dimension";
    case CUROB_ERR_CAPACITY: return "N exceeds max_concurrency";
    case CUROB_ERR_NULL_POINTER: return "null pointer";
    case CUROB_ERR_CUDA: return "CUDA error";
    case CUROB_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case CUROB_ERR_OUT_OF_MEMORY: return "out of device memory";
    case CUROB_ERR_INVALID_ARGUMENT: return "invalid argument";
    case CUROB_ERR_UNSUPPORTED: return "unsupported size";
  }
  return "unknown status";
}

curob_status curob_initialize(int D, int max_concurrency, uint64_t seed) {
  std::lock_guard<std::mutex> lk(g.mu);
  if (g.init) return CUROB_ERR_ALREADY_INITIALIZED;
  if (D < 2) return CUROB_ERR_INVALID_DIM;
  if (max_concurrency < 1) return CUROB_ERR_INVALID_ARGUMENT;
  if (cudaGetDevice(&g.device) != cudaSuccess) return CUROB_ERR_CUDA;
  g.max_conc = max_concurrency;
  if (cudaMalloc(&g.d_hx, sizeof(double) * (size_t)max_concurrency * D) != cudaSuccess ||
      cudaMalloc(&g.d_hout, sizeof(double) * (size_t)max_concurrency) != cudaSuccess) {
    cudaGetLastError();
    free_all();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  bool streams_ok = cudaStreamCreateWithFlags(&g.hstream, cudaStreamNonBlocking) == cudaSuccess;
  for (cudaStream_t& s : g.hside)
    streams_ok = streams_ok && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
  if (!streams_ok) {
    free_all();
    return CUROB_ERR_CUDA;
  }
  curob_status rc = g.inst.create(D, seed);
  if (rc != CUROB_OK) {
    free_all();
    return rc;
  }
  g.precision = CUROB_PRECISION_AUTO;
  g.precision64 = CUROB_PRECISION64_AUTO;
  g.small_batch = kSmallBatchDefault;
  for (int fid = 0; fid < kNumFunctions; ++fid)
    if (g.inst.func_ok[fid]) make_small_args(g.small[fid], g.inst.func[fid]);
  g.init = true;
  return CUROB_OK;
}

curob_status curob_dispose(void) {
  std::lock_guard<std::mutex> lk(g.mu);
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  cudaDeviceSynchronize();
  free_all();
  return CUROB_OK;
}

curob_status curob_evaluate(int fid, const double* x, int N, double* out, curob_stream_t stream) {
  curob_status rc = check_eval_args(fid, x, N, out);
  if (rc != CUROB_OK || N == 0) return rc;
  if (!on_instance_device()) return CUROB_ERR_INVALID_ARGUMENT;
  if (!device_accessible(x) || !device_accessible(out)) return CUROB_ERR_INVALID_ARGUMENT;
  return eval64(fid, x, N, out, (cudaStream_t)stream);
}

curob_status curob_evaluatef(int fid, const float* x, int N, float* out, curob_stream_t stream) {
  curob_status rc = check_eval_args(fid, x, N, out);
  if (rc != CUROB_OK || N == 0) return rc;
  if (!on_instance_device()) return CUROB_ERR_INVALID_ARGUMENT;
  if (!device_accessible(x) || !device_accessible(out)) return CUROB_ERR_INVALID_ARGUMENT;
  const Function& F = g.inst.func[fid];
  const int mode = resolve_precision(F);
  if (mode < 0) return CUROB_ERR_UNSUPPORTED;
  cudaError_t e;
  if (g.precision == CUROB_PRECISION_AUTO && use_small(F, N))
    e = launch_small_f32(g.small[fid], x, N, out, (cudaStream_t)stream);
  else if (mode == CUROB_PRECISION_SIMT)
    e = launch_simt_f32(tables(), F, x, N, out, (cudaStream_t)stream);
  else if (mode == CUROB_PRECISION_MIXED)
    e = launch_mma_mixed(g.inst.mma, tables(), F, x, N, out, (cudaStream_t)stream);
  else
    e = launch_mma(g.inst.mma, tables(), F, mode, x, N, out, (cudaStream_t)stream);
  return e == cudaSuccess ? CUROB_OK : CUROB_ERR_CUDA;
}

curob_status curob_h_evaluate(int fid, const double* x, int N, double* out) {
  curob_status rc = check_eval_args(fid, x, N, out);
  if (rc != CUROB_OK || N == 0) return rc;
  // the staging buffers and the streams are shared: one host call at a time
  std::lock_guard<std::mutex> lk(g.mu);
  if (!on_instance_device()) return CUROB_ERR_INVALID_ARGUMENT;
  return host_pipeline<double>(x, N, out, [&](const double* dx, int n, double* dout,
                                              cudaStream_t st) {
    return eval64(fid, dx, n, dout, st);
  });
}

curob_status curob_h_evaluatef(int fid, const float* x, int N, float* out) {
  curob_status rc = check_eval_args(fid, x, N, out);
  if (rc != CUROB_OK || N == 0) return rc;
  std::lock_guard<std::mutex> lk(g.mu);
  if (!on_instance_device()) return CUROB_ERR_INVALID_ARGUMENT;
  return host_pipeline<float>(x, N, out, [&](const float* dx, int n, float* dout,
                                             cudaStream_t st) {
    return curob_evaluatef(fid, dx, n, dout, st);
  });
}

curob_status curob_set_precision(int mode) {
  if (mode < CUROB_PRECISION_AUTO || mode > CUROB_PRECISION_FP16X3 ||
      mode == CUROB_PRECISION_MIXED)
    return CUROB_ERR_INVALID_ARGUMENT;
  g.precision = mode;
  return CUROB_OK;
}

curob_status curob_set_small_batch(int max_n) {
  if (max_n < 0) return CUROB_ERR_INVALID_ARGUMENT;
  g.small_batch = max_n;
  return CUROB_OK;
}

curob_status curob_query_small(int fid, int N, int* small) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  if (!g.inst.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
  if (!small) return CUROB_ERR_NULL_POINTER;
  if (N < 0) return CUROB_ERR_INVALID_ARGUMENT;
  *small = (N > 0 && use_small(g.inst.func[fid], N)) ? 1 : 0;
  return CUROB_OK;
}

curob_status curob_query_precision(int fid, int* mode) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  if (!g.inst.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
  if (!mode) return CUROB_ERR_NULL_POINTER;
  const int m = resolve_precision(g.inst.func[fid]);
  if (m < 0) return CUROB_ERR_UNSUPPORTED;
  *mode = m;
  return CUROB_OK;
}

curob_status curob_query_component_precision(int fid, int comp, int* mode) {
  int m = 0;
  curob_status rc = curob_query_precision(fid, &m);
  if (rc != CUROB_OK) return rc;
  const Function& F = g.inst.func[fid];
  if (comp < 0 || comp >= F.ncomp) return CUROB_ERR_INVALID_ARGUMENT;
  if (m == CUROB_PRECISION_MIXED)
    m = (F.sens_mask >> comp & 1) ? CUROB_PRECISION_EXACT : CUROB_PRECISION_TF32X3;
  *mode = m;
  return CUROB_OK;
}

curob_status curob_query_launches(int fid, int N, int* launches) {
  int m = 0;
  curob_status rc = curob_query_precision(fid, &m);
  if (rc != CUROB_OK) return rc;
  if (!launches) return CUROB_ERR_NULL_POINTER;
  if (N < 0) return CUROB_ERR_INVALID_ARGUMENT;
  if (N == 0) *launches = 0;
  else if (m == CUROB_PRECISION_SIMT) *launches = 1;
  else if (g.precision == CUROB_PRECISION_AUTO && use_small(g.inst.func[fid], N)) *launches = 1;
  else *launches = mma_launch_count(g.inst.func[fid], m, N);
  return CUROB_OK;
}

curob_status curob_set_precision64(int mode) {
  if (mode < CUROB_PRECISION64_AUTO || mode > CUROB_PRECISION64_TENSOR)
    return CUROB_ERR_INVALID_ARGUMENT;
  g.precision64 = mode;
  return CUROB_OK;
}

curob_status curob_query_precision64(int fid, int* mode) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  if (!g.inst.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
  if (!mode) return CUROB_ERR_NULL_POINTER;
  const int path = resolve_precision64(fid);
  if (path < 0) return CUROB_ERR_UNSUPPORTED;
  *mode = path;
  return CUROB_OK;
}

curob_status curob_query_launches64(int fid, int N, int* launches) {
  int m = 0;
  curob_status rc = curob_query_precision64(fid, &m);
  if (rc != CUROB_OK) return rc;
  if (!launches) return CUROB_ERR_NULL_POINTER;
  if (N < 0) return CUROB_ERR_INVALID_ARGUMENT;
  const Function& F = g.inst.func[fid];
  if (N == 0) *launches = 0;
  else if (use_small(F, N) || m == CUROB_PRECISION64_SIMT) *launches = 1;
  else *launches = f64_launch_count(g.inst.f64, F, fid, g.inst.D, N);
  return CUROB_OK;
}

curob_status curob_selftest_bounded_wait(curob_stream_t stream) {
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CUROB_ERR_CUDA;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major != 10) return CUROB_ERR_UNSUPPORTED;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int h = -1;
  const bool ok = cudaMemsetAsync(d, 0, sizeof(int), st) == cudaSuccess &&
                  launch_wait_selftest(d, st) == cudaSuccess &&
                  cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(d);
  if (!ok) return CUROB_ERR_CUDA;
  return h == DEV_TIMEOUT ? CUROB_ERR_DEVICE_TIMEOUT : (h == DEV_OK ? CUROB_OK : CUROB_ERR_CUDA);
}

curob_status curob_get_device_status(curob_stream_t stream) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CUROB_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, g.inst.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (st == DEV_OK) return CUROB_OK;
  cudaMemset(g.inst.d_status, 0, sizeof(int));
  return st == DEV_TIMEOUT ? CUROB_ERR_DEVICE_TIMEOUT : CUROB_ERR_CUDA;
}

curob_status curob_get_config(int* D, int* max_concurrency) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (!D || !max_concurrency) return CUROB_ERR_NULL_POINTER;
  *D = g.inst.D;
  *max_concurrency = g.max_conc;
  return CUROB_OK;
}

curob_status curob_num_components(int fid, int* ncomp) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  if (!g.inst.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
  if (!ncomp) return CUROB_ERR_NULL_POINTER;
  *ncomp = g.inst.func[fid].ncomp;
  return CUROB_OK;
}

curob_status curob_component_layout(int fid, int comp, int* n_blocks, int sizes[5], int* rotated) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  int c = g.inst.find_comp(fid, comp);
  if (c < 0) return g.inst.func_ok[fid] ? CUROB_ERR_INVALID_ARGUMENT : CUROB_ERR_INVALID_DIM;
  if (!n_blocks || !sizes || !rotated) return CUROB_ERR_NULL_POINTER;
  const CompHost& ch = g.inst.chost[c];
  for (int i = 0; i < 5; ++i) sizes[i] = 0;
  if (ch.rotated) {
    *n_blocks = (int)ch.sizes.size();
    for (size_t i = 0; i < ch.sizes.size(); ++i) sizes[i] = ch.sizes[i];
  } else {
    *n_blocks = 1;
    sizes[0] = g.inst.D;
  }
  *rotated = ch.rotated;
  return CUROB_OK;
}

curob_status curob_component_kinds(int fid, int comp, int* n_blocks, int kinds[5]) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  int c = g.inst.find_comp(fid, comp);
  if (c < 0) return g.inst.func_ok[fid] ? CUROB_ERR_INVALID_ARGUMENT : CUROB_ERR_INVALID_DIM;
  if (!n_blocks || !kinds) return CUROB_ERR_NULL_POINTER;
  const CompHost& ch = g.inst.chost[c];
  int k = 0;
  for (int i = 0; i < 5; ++i) kinds[i] = -1;
  for (int id : ch.segs)
    if (k < 5) kinds[k++] = g.inst.segs[id].kind;
  *n_blocks = k;
  return CUROB_OK;
}

curob_status curob_get_component(int fid, int comp, double* o, int* S, double* R) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  return g.inst.get_component(fid, comp, o, S, R);
}

curob_status curob_set_component(int fid, int comp, const double* o, const int* S, const double* R) {
  std::lock_guard<std::mutex> lk(g.mu);
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  return g.inst.set_component(fid, comp, o, S, R);
}

curob_status curob_get_optimum(int fid, double* xopt) {
  if (!xopt) return CUROB_ERR_NULL_POINTER;
  return curob_get_component(fid, 0, xopt, nullptr, nullptr);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free evaluation of several functions in one launch.
//
// For callers that may not allocate device memory at evaluation time: code
// that reserves all of its GPU memory up front under a fixed budget (an
// optimizer embedded in a real-time or safety-constrained loop), or a plugin
// whose host framework owns every device allocation.  The work list, the
// per-function argument blocks and the work counter of the persistent kernel
// live in this file's static device array instead of cudaMalloc'd memory; the
// caller passes candidates and outputs, and the instance is the one
// curob_initialize built.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoAllocMaxItems = 64;       // functions per call
constexpr int kNoAllocMaxTiles = 16384;    // 128-candidate tiles per call
constexpr size_t kNoAllocArgsBytes = 64 * 512;
constexpr size_t kNoAllocWorkOff = 256 + kNoAllocArgsBytes;
constexpr size_t kNoAllocBytes = kNoAllocWorkOff + kNoAllocMaxTiles * sizeof(int2);
constexpr int kNoAllocMaxDevices = 64;

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};        // device address of the array, per device
unsigned char g_noalloc_args[kNoAllocArgsBytes];      // host staging (no host allocation either)
int2 g_noalloc_work[kNoAllocMaxTiles];
}  // namespace

// 160 KB on every device that loads the library, held until the process exits.
// Layout: [work counter | 256 B][argument blocks | 32 KB][work list | 128 KB].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

extern "C" curob_status curob_evaluatef_multi_noalloc(const int* fids, const float* const* x,
                                                      const int* N, float* const* out,
                                                      int n_items, curob_stream_t stream) {
  using namespace curob;
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (!fids || !x || !N || !out) return CUROB_ERR_NULL_POINTER;
  if (n_items < 1) return CUROB_ERR_INVALID_ARGUMENT;
  if (n_items > kNoAllocMaxItems) return CUROB_ERR_CAPACITY;
  if (mma_args_bytes() * (size_t)n_items > kNoAllocArgsBytes) return CUROB_ERR_CAPACITY;
  long long tiles = 0;
  for (int i = 0; i < n_items; ++i) {
    const int fid = fids[i];
    if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
    if (!g.inst.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
    if (N[i] < 0) return CUROB_ERR_INVALID_ARGUMENT;
    if (N[i] > g.max_conc) return CUROB_ERR_CAPACITY;
    if (!mma_supports(g.inst.mma, g.inst.func[fid])) return CUROB_ERR_UNSUPPORTED;
    if (N[i] > 0) {
      if (!x[i] || !out[i]) return CUROB_ERR_NULL_POINTER;
      if (!device_accessible(x[i]) || !device_accessible(out[i]))
        return CUROB_ERR_INVALID_ARGUMENT;
    }
    tiles += (N[i] + 127) / 128;
  }
  if (tiles > kNoAllocMaxTiles) return CUROB_ERR_CAPACITY;
  if (tiles == 0) return CUROB_OK;

  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
    return CUROB_ERR_CUDA;
  // the argument blocks point at the instance's tables, which live on the
  // device curob_initialize ran on; another current device would fault
  if (dev != g.device) return CUROB_ERR_INVALID_ARGUMENT;
  if (!g_noalloc_addr[dev]) {  // first call on this device: look the array up once
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CUROB_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  const size_t ab = mma_args_bytes();
  int nwork = 0;
  for (int i = 0; i < n_items; ++i) {
    mma_fill_args(g_noalloc_args + ab * i, g.inst.mma, g.inst.tables(), g.inst.func[fids[i]],
                  x[i], out[i], N[i]);
  }
  // round robin over the functions, so every CTA sees a mix of them
  for (int t = 0; nwork < tiles; ++t)
    for (int i = 0; i < n_items; ++i)
      if (t < (N[i] + 127) / 128) g_noalloc_work[nwork++] = make_int2(i, t);
  cudaStream_t st = (cudaStream_t)stream;
  // the counter must start at 0; the rest is overwritten before use
  if (cudaMemsetAsync(base, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemcpyAsync(base + 256, g_noalloc_args, ab * n_items, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(base + kNoAllocWorkOff, g_noalloc_work, sizeof(int2) * nwork,
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return CUROB_ERR_CUDA;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(nsm, nwork));
  if (launch_mma_batch(base + 256, reinterpret_cast<const int2*>(base + kNoAllocWorkOff), nwork,
                       reinterpret_cast<int*>(base), grid, st) != cudaSuccess)
    return CUROB_ERR_CUDA;
  return CUROB_OK;
}

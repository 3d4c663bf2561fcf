// curob_api.cu -- the C ABI of libcurob (include/curob.h): instance
// construction (initialize/dispose, Sec. 1.3 "Interface"), evaluation entry
// points and the instance-data accessors.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/curob.h"
#include "curob_internal.hpp"
#include "curob_mma.hpp"

namespace curob {
namespace {

// ---------------------------------------------------------------------------
// The suite (Table 1 and Sec. 3-6).  Scale s and offset c of each basic kind:
// z = R(s (x - o)) + c, as printed under each function.
// ---------------------------------------------------------------------------
struct KindInfo { double scale, offset; };
const KindInfo kKind[K_COUNT] = {
    {1.0, 0.0},      // sphere            Sec. 3.1
    {1.0, 0.0},      // ellipsoid         Sec. 3.2
    {1.0, 0.0},      // elliptic          Sec. 3.3
    {1.0, 0.0},      // discus            Sec. 3.4
    {1.0, 0.0},      // bent cigar        Sec. 3.5
    {0.01, 0.0},     // different powers  Sec. 3.6
    {1.0, 0.0},      // sharp valley      Sec. 3.7
    {1.0, 0.0},      // step              Sec. 4.1
    {0.005, 0.0},    // weierstrass       Sec. 4.2
    {6.0, 0.0},      // griewank          Sec. 4.3
    {0.0512, 0.0},   // rastrigin         Sec. 4.4, 4.5
    {1.0, 0.0},      // schaffer F7       Sec. 4.6
    {0.05, 1.0},     // expanded griewank+rosenbrock  Sec. 4.7
    {0.02048, 1.0},  // rosenbrock        Sec. 4.8
    {10.0, 0.0},     // modified schwefel Sec. 4.9, 4.10 (420.97 lives in g1)
    {0.05, 0.0},     // katsuura          Sec. 4.11
    {0.1, 2.5},      // lunacek           Sec. 4.12 (2.5 read outside R)
    {1.0, 0.0},      // ackley            Sec. 4.13
    {0.05, -1.0},    // happycat          Sec. 4.14
    {0.05, -1.0},    // hgbat             Sec. 4.15
    {1.0, 0.0},      // expanded schaffer F6  Sec. 4.16
};

// A member of a function: a basic kind (rotated or not) or a hybrid.
struct Member {
  int kind;     // basic kind, or -1 for a hybrid member
  int rotated;
  int hybrid;   // hybrid function id (23..28) when kind < 0
};
struct HybridInfo { int n; int kind[5]; int pct[5]; };
struct CompInfo { int n; Member m[5]; double sigma[5], lambda[5], bias[5]; };

// Sec. 5.1-5.6 (Hybrid Function 2 read as N = 3: three p's and three G's).
const HybridInfo kHybrid[6] = {
    {3, {K_SCHWEFEL, K_RASTRIGIN, K_ELLIPTIC}, {30, 30, 40}},
    {3, {K_CIGAR, K_HGBAT, K_RASTRIGIN}, {30, 30, 40}},
    {4, {K_GRIEWANK, K_WEIERSTRASS, K_ROSENBROCK, K_SCHAFFER6}, {20, 20, 30, 30}},
    {4, {K_HGBAT, K_DISCUS, K_EGR, K_RASTRIGIN}, {20, 20, 30, 30}},
    {5, {K_SCHAFFER6, K_HGBAT, K_ROSENBROCK, K_SCHWEFEL, K_ELLIPTIC}, {10, 20, 20, 20, 30}},
    {5, {K_KATSUURA, K_HAPPYCAT, K_EGR, K_SCHWEFEL, K_ACKLEY}, {10, 20, 20, 20, 30}},
};

Member B(int k, int r) { return Member{k, r, -1}; }
Member Hm(int h) { return Member{-1, 1, h}; }

// Sec. 6.1-6.8.  Members not called "Rotated" are unrotated; "Expanded
// Schwefel" is the unrotated Modified Schwefel; Composition Function 5 takes
// its G's in list order.
CompInfo comp_info(int fid) {
  switch (fid) {
    case 29: return {5, {B(K_ROSENBROCK, 1), B(K_ELLIPTIC, 0), B(K_CIGAR, 1), B(K_DISCUS, 1), B(K_ELLIPTIC, 0)},
                     {10, 20, 30, 40, 50}, {1e-10, 1e-6, 1e-26, 1e-6, 1e-6}, {0, 100, 200, 300, 400}};
    case 30: return {3, {B(K_SCHWEFEL, 0), B(K_RASTRIGIN, 1), B(K_HGBAT, 1)},
                     {15, 15, 15}, {1, 1, 1}, {0, 100, 200}};
    case 31: return {3, {B(K_SCHWEFEL, 1), B(K_RASTRIGIN, 1), B(K_ELLIPTIC, 1)},
                     {20, 50, 40}, {0.25, 1, 1e-7}, {0, 100, 200}};
    case 32: return {5, {B(K_SCHWEFEL, 1), B(K_HAPPYCAT, 1), B(K_ELLIPTIC, 1), B(K_WEIERSTRASS, 1), B(K_GRIEWANK, 1)},
                     {20, 15, 10, 10, 40}, {2.5e-2, 0.1, 1e-8, 0.25, 1}, {0, 100, 200, 300, 400}};
    case 33: return {5, {B(K_HGBAT, 1), B(K_RASTRIGIN, 1), B(K_SCHWEFEL, 1), B(K_WEIERSTRASS, 1), B(K_ELLIPTIC, 1)},
                     {15, 15, 15, 15, 15}, {10, 10, 2.5, 2.5, 1e-6}, {0, 100, 200, 300, 400}};
    case 34: return {5, {B(K_EGR, 1), B(K_HAPPYCAT, 1), B(K_SCHWEFEL, 1), B(K_SCHAFFER6, 1), B(K_ELLIPTIC, 0)},
                     {10, 20, 30, 40, 50}, {2.5, 10, 2.5, 5e-4, 1e-6}, {0, 100, 200, 300, 400}};
    case 35: return {3, {Hm(23), Hm(24), Hm(25)}, {10, 30, 50}, {1, 1, 1}, {0, 100, 200}};
    case 36: return {3, {Hm(26), Hm(27), Hm(28)}, {10, 30, 50}, {1, 1, 1}, {0, 100, 200}};
    default: break;
  }
  // Table 1 rows 0..22: one member; IDs 10 and 15 are the unrotated ones.
  if (fid <= 22) {
    const int kinds[23] = {K_SPHERE, K_ELLIPSOID, K_ELLIPTIC, K_DISCUS, K_CIGAR, K_POWERS,
                           K_SHARPV, K_STEP, K_WEIERSTRASS, K_GRIEWANK, K_RASTRIGIN,
                           K_RASTRIGIN, K_SCHAFFER7, K_EGR, K_ROSENBROCK, K_SCHWEFEL,
                           K_SCHWEFEL, K_KATSUURA, K_LUNACEK, K_ACKLEY, K_HAPPYCAT, K_HGBAT,
                           K_SCHAFFER6};
    return {1, {B(kinds[fid], (fid == 10 || fid == 15) ? 0 : 1)}, {1}, {1}, {0}};
  }
  return {1, {Hm(fid)}, {1}, {1}, {0}};  // hybrids 23..28
}

bool needs_d10(int fid) { return (fid >= 23 && fid <= 28) || fid == 35 || fid == 36; }

// Block sizes of a member at dimension D (General Setup; Sec. 5 Eq. numbers).
void member_blocks(const Member& m, int D, std::vector<int>& sizes) {
  sizes.clear();
  if (m.kind < 0) {
    const HybridInfo& h = kHybrid[m.hybrid - 23];
    int used = 0;
    for (int i = 0; i < h.n - 1; ++i) {
      int v = (h.pct[i] * D + 99) / 100;  // ceil(p_i D) in integer percent
      sizes.push_back(v);
      used += v;
    }
    sizes.push_back(D - used);
  } else {
    sizes.push_back(D / 3);
    sizes.push_back(D / 3);
    sizes.push_back(D - 2 * (D / 3));
  }
}

// Host bookkeeping for one component.
struct CompHost {
  int fid, idx;        // function and member index (RNG counter words 2, 3)
  int rotated;
  std::vector<int> sizes;  // all blocks, including empty ones, in z order
  std::vector<int> segs;   // segment ids of the non-empty blocks
};

struct State {
  std::mutex mu;
  bool init = false;
  int D = 0, max_conc = 0;
  uint64_t seed = 0;
  int device = 0;
  int precision = CUROB_PRECISION_AUTO;
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
  float *d_R32 = nullptr, *d_R32lo = nullptr, *d_aux32 = nullptr, *d_img = nullptr;
  int* d_status = nullptr;
  long long r_total = 0, aux_total = 0, img_total = 0;
  void* d_hx = nullptr;   // host-wrapper staging (max_conc x D doubles)
  void* d_hout = nullptr; // (max_conc doubles)
  cudaStream_t hstream = nullptr;
  MmaPlan mma;            // tensor-core path state
};

State g;

Tables tables() {
  Tables t;
  t.seg = g.d_seg;
  t.comp = g.d_comp;
  t.o = g.d_o;
  t.S = g.d_S;
  t.operm = g.d_operm;
  t.R = g.d_R;
  t.R32 = g.d_R32;
  t.R32lo = g.d_R32lo;
  t.aux = g.d_aux;
  t.aux32 = g.d_aux32;
  t.img = g.d_img;
  t.D = g.D;
  t.status = g.d_status;
  return t;
}

void free_all() {
  cudaFree(g.d_seg); cudaFree(g.d_comp); cudaFree(g.d_o); cudaFree(g.d_operm);
  cudaFree(g.d_R); cudaFree(g.d_aux); cudaFree(g.d_S); cudaFree(g.d_R32); cudaFree(g.d_R32lo);
  cudaFree(g.d_aux32); cudaFree(g.d_status); cudaFree(g.d_hx);  // d_img belongs to g.mma
  cudaFree(g.d_hout);
  if (g.hstream) cudaStreamDestroy(g.hstream);
  mma_release(g.mma);
  g.d_seg = nullptr; g.d_comp = nullptr; g.d_o = g.d_operm = g.d_R = g.d_aux = nullptr;
  g.d_S = nullptr; g.d_R32 = g.d_R32lo = g.d_aux32 = g.d_img = nullptr; g.d_status = nullptr;
  g.d_hx = g.d_hout = nullptr; g.hstream = nullptr;
  g.segs.clear(); g.comps.clear(); g.chost.clear();
  for (int f = 0; f < kNumFunctions; ++f) g.func_ok[f] = false;
  g.init = false;
}

bool kind_has_aux(int k) { return k == K_ELLIPTIC || k == K_POWERS || k == K_GRIEWANK; }

// Builds the component and segment tables for dimension D.
void build_tables(int D) {
  g.segs.clear(); g.comps.clear(); g.chost.clear();
  long long r_total = 0, aux_total = 0;
  for (int fid = 0; fid < kNumFunctions; ++fid) {
    g.func_ok[fid] = !(needs_d10(fid) && D < 10);
    if (!g.func_ok[fid]) continue;
    CompInfo ci = comp_info(fid);
    Function F;
    F.comp0 = (int)g.comps.size();
    F.ncomp = ci.n;
    F.composition = fid >= 29;
    F.max_n = 0;
    F.sensitive = 0;
    for (int c = 0; c < ci.n; ++c) {
      const Member& m = ci.m[c];
      CompHost ch;
      ch.fid = fid;
      ch.idx = c;
      ch.rotated = m.rotated;
      member_blocks(m, D, ch.sizes);
      Component C;
      C.seg0 = (int)g.segs.size();
      C.base = (long long)g.comps.size() * D;
      C.sigma = ci.sigma[c];
      C.lambda = ci.lambda[c];
      C.bias = ci.bias[c];
      // non-empty blocks become segments
      std::vector<int> nz;
      for (size_t b = 0; b < ch.sizes.size(); ++b)
        if (ch.sizes[b] > 0) nz.push_back((int)b);
      int off = 0;
      std::vector<int> offs(ch.sizes.size());
      for (size_t b = 0; b < ch.sizes.size(); ++b) { offs[b] = off; off += ch.sizes[b]; }
      for (size_t t = 0; t < nz.size(); ++t) {
        const int b = nz[t];
        Segment s;
        s.n = ch.sizes[b];
        s.zoff = offs[b];
        if (m.kind < 0) {  // hybrid block: a function of its own
          s.kind = kHybrid[m.hybrid - 23].kind[b];
          s.gn = s.n;
          s.gpos = 0;
          s.gfirst = s.glast = 1;
        } else {
          s.kind = m.kind;
          s.gn = D;
          s.gpos = s.zoff;
          s.gfirst = (t == 0);
          s.glast = (t + 1 == nz.size());
        }
        s.identity = m.rotated ? 0 : 1;
        s.scale = kKind[s.kind].scale;
        s.offset = kKind[s.kind].offset;
        s.r_off = -1;
        if (!s.identity) { s.r_off = r_total; r_total += (long long)s.n * s.n; }
        s.aux_off = -1;
        if (kind_has_aux(s.kind)) { s.aux_off = aux_total; aux_total += s.n; }
        s.img_off = -1;
        s.npad = 0;
        s.comp = (int)g.comps.size();
        F.max_n = std::max(F.max_n, s.n);
        if (kind_is_sensitive(s.kind)) F.sensitive = 1;
        ch.segs.push_back((int)g.segs.size());
        g.segs.push_back(s);
      }
      C.nseg = (int)g.segs.size() - C.seg0;
      g.comps.push_back(C);
      g.chost.push_back(ch);
    }
    g.func[fid] = F;
  }
  g.r_total = r_total;
  g.aux_total = aux_total;
}

#define CU(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      return e_ == cudaErrorMemoryAllocation ? CUROB_ERR_OUT_OF_MEMORY : CUROB_ERR_CUDA; \
    }                                              \
  } while (0)

// Shift, permutation, rotations and tables for all components, on the GPU.
curob_status generate_all() {
  const int D = g.D;
  const int nc = (int)g.comps.size();
  std::vector<PermJob> pj(nc);
  std::vector<GaussJob> gj;
  std::vector<AuxJob> aj;
  int max_n = 1;
  for (int c = 0; c < nc; ++c) {
    const CompHost& ch = g.chost[c];
    PermJob& p = pj[c];
    memset(&p, 0, sizeof(p));
    p.base = g.comps[c].base;
    p.fid = ch.fid;
    p.comp = ch.idx;
    p.origin = (ch.fid >= 29 && ch.idx == 2) ? 1 : 0;  // Sec. 6: third optimum at 0
    p.identity = ch.rotated ? 0 : 1;
    int off = 0, k = 0;
    for (size_t b = 0; b < ch.sizes.size(); ++b) {
      if (ch.sizes[b] > 0) { p.blk_off[k] = off; p.blk_n[k] = ch.sizes[b]; ++k; }
      off += ch.sizes[b];
    }
    p.nblk = k;
    // Gaussian blocks: the block index b counts empty blocks too
    int sidx = 0;
    for (size_t b = 0; b < ch.sizes.size(); ++b) {
      if (ch.sizes[b] == 0) continue;
      const Segment& s = g.segs[ch.segs[sidx++]];
      if (!s.identity) {
        GaussJob J;
        J.r_off = s.r_off;
        J.n = s.n;
        J.fid = ch.fid;
        J.comp = ch.idx;
        J.blk = (int)b;
        gj.push_back(J);
        max_n = std::max(max_n, s.n);
      }
    }
  }
  for (const Segment& s : g.segs)
    if (s.aux_off >= 0) aj.push_back(AuxJob{s.aux_off, s.kind, s.n, s.gn, s.gpos});

  if (2 * (size_t)max_n * sizeof(double) > 220 * 1024) return CUROB_ERR_UNSUPPORTED;

  PermJob* d_pj = nullptr;
  GaussJob* d_gj = nullptr;
  AuxJob* d_aj = nullptr;
  uint64_t* d_words = nullptr;
  int* d_mark = nullptr;
  curob_status rc = CUROB_OK;
  auto fail = [&](cudaError_t e) {
    if (rc == CUROB_OK && e != cudaSuccess)
      rc = (e == cudaErrorMemoryAllocation) ? CUROB_ERR_OUT_OF_MEMORY : CUROB_ERR_CUDA;
  };
  fail(cudaMalloc(&d_pj, sizeof(PermJob) * std::max(nc, 1)));
  fail(cudaMalloc(&d_gj, sizeof(GaussJob) * std::max<size_t>(gj.size(), 1)));
  fail(cudaMalloc(&d_aj, sizeof(AuxJob) * std::max<size_t>(aj.size(), 1)));
  fail(cudaMalloc(&d_words, sizeof(uint64_t) * (size_t)nc * D));
  fail(cudaMalloc(&d_mark, sizeof(int) * (size_t)nc * D));
  if (rc == CUROB_OK) {
    fail(cudaMemcpy(d_pj, pj.data(), sizeof(PermJob) * nc, cudaMemcpyHostToDevice));
    if (!gj.empty())
      fail(cudaMemcpy(d_gj, gj.data(), sizeof(GaussJob) * gj.size(), cudaMemcpyHostToDevice));
    if (!aj.empty())
      fail(cudaMemcpy(d_aj, aj.data(), sizeof(AuxJob) * aj.size(), cudaMemcpyHostToDevice));
  }
  if (rc == CUROB_OK)
    fail(launch_shift_perm(d_pj, nc, D, g.seed, g.d_o, g.d_S, g.d_operm, d_words, d_mark, 0));
  if (rc == CUROB_OK)
    fail(launch_gauss_gs(d_gj, (int)gj.size(), max_n, g.seed, g.d_R, g.d_status, 0));
  if (rc == CUROB_OK) fail(launch_aux(d_aj, (int)aj.size(), g.d_aux, g.d_aux32, 0));
  if (rc == CUROB_OK) fail(launch_split_f32(g.d_R, g.d_R32, g.d_R32lo, g.r_total, 0));
  if (rc == CUROB_OK) fail(cudaDeviceSynchronize());
  cudaFree(d_pj); cudaFree(d_gj); cudaFree(d_aj); cudaFree(d_words); cudaFree(d_mark);
  if (rc == CUROB_OK) {
    int st = 0;
    fail(cudaMemcpy(&st, g.d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (rc == CUROB_OK && st != DEV_OK) rc = CUROB_ERR_CUDA;
  }
  return rc;
}

curob_status check_eval_args(int fid, const void* x, int N, const void* out) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  if (!g.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
  if (N < 0) return CUROB_ERR_INVALID_ARGUMENT;
  if (N > g.max_conc) return CUROB_ERR_CAPACITY;
  if (N == 0) return CUROB_OK;
  if (!x || !out) return CUROB_ERR_NULL_POINTER;
  return CUROB_OK;
}

// A kernel given a pointer the GPU cannot reach would fault the context, so
// evaluations accept device (or managed) memory only.
bool device_accessible(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The precision curob_evaluatef uses for F (AUTO resolved), or -1 when a
// forced tensor-core precision cannot take F's block sizes.
int resolve_precision(const Function& F) {
  int mode = g.precision;
  const bool mma_ok = mma_supports(g.mma, F);
  const bool tc = mode == CUROB_PRECISION_TF32X3 || mode == CUROB_PRECISION_BF16X3 ||
                  mode == CUROB_PRECISION_EXACT;
  if (tc && !mma_ok) return -1;
  if (mode == CUROB_PRECISION_AUTO) mode = mma_ok ? mma_auto_mode(g.mma, F) : CUROB_PRECISION_SIMT;
  return mode;
}

int find_comp(int fid, int comp) {
  if (fid < 0 || fid >= kNumFunctions || !g.func_ok[fid]) return -1;
  if (comp < 0 || comp >= g.func[fid].ncomp) return -1;
  return g.func[fid].comp0 + comp;
}

}  // namespace
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
  g.D = D;
  g.max_conc = max_concurrency;
  g.seed = seed;
  build_tables(D);
  const int nc = (int)g.comps.size();
  auto alloc = [&](void** p, size_t bytes) -> bool {
    return cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess;
  };
  bool ok = alloc((void**)&g.d_seg, sizeof(Segment) * g.segs.size()) &&
            alloc((void**)&g.d_comp, sizeof(Component) * nc) &&
            alloc((void**)&g.d_o, sizeof(double) * (size_t)nc * D) &&
            alloc((void**)&g.d_operm, sizeof(double) * (size_t)nc * D) &&
            alloc((void**)&g.d_S, sizeof(int) * (size_t)nc * D) &&
            alloc((void**)&g.d_R, sizeof(double) * (size_t)g.r_total) &&
            alloc((void**)&g.d_R32, sizeof(float) * (size_t)g.r_total) &&
            alloc((void**)&g.d_R32lo, sizeof(float) * (size_t)g.r_total) &&
            alloc((void**)&g.d_aux, sizeof(double) * (size_t)g.aux_total) &&
            alloc((void**)&g.d_aux32, sizeof(float) * (size_t)g.aux_total) &&
            alloc((void**)&g.d_status, sizeof(int)) &&
            alloc(&g.d_hx, sizeof(double) * (size_t)max_concurrency * D) &&
            alloc(&g.d_hout, sizeof(double) * (size_t)max_concurrency);
  if (!ok) {
    cudaGetLastError();
    free_all();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  if (cudaMemset(g.d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&g.hstream, cudaStreamNonBlocking) != cudaSuccess) {
    free_all();
    return CUROB_ERR_CUDA;
  }
  curob_status rc = generate_all();
  if (rc == CUROB_OK) {
    // tensor-core operand images (TF32/BF16 hi-lo splits of every block)
    rc = mma_prepare(g.mma, g.segs, tables(), g.d_img);
    g.d_img = g.mma.img;
  }
  if (rc == CUROB_OK) {
    if (cudaMemcpy(g.d_seg, g.segs.data(), sizeof(Segment) * g.segs.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g.d_comp, g.comps.data(), sizeof(Component) * nc, cudaMemcpyHostToDevice) !=
            cudaSuccess)
      rc = CUROB_ERR_CUDA;
  }
  if (rc != CUROB_OK) {
    free_all();
    return rc;
  }
  g.precision = CUROB_PRECISION_AUTO;
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
  if (!device_accessible(x) || !device_accessible(out)) return CUROB_ERR_INVALID_ARGUMENT;
  cudaError_t e = launch_simt_f64(tables(), g.func[fid], x, N, out, (cudaStream_t)stream);
  return e == cudaSuccess ? CUROB_OK : CUROB_ERR_CUDA;
}

curob_status curob_evaluatef(int fid, const float* x, int N, float* out, curob_stream_t stream) {
  curob_status rc = check_eval_args(fid, x, N, out);
  if (rc != CUROB_OK || N == 0) return rc;
  if (!device_accessible(x) || !device_accessible(out)) return CUROB_ERR_INVALID_ARGUMENT;
  const Function& F = g.func[fid];
  const int mode = resolve_precision(F);
  if (mode < 0) return CUROB_ERR_UNSUPPORTED;
  cudaError_t e;
  if (mode == CUROB_PRECISION_SIMT)
    e = launch_simt_f32(tables(), F, x, N, out, (cudaStream_t)stream);
  else
    e = launch_mma(g.mma, tables(), F, mode, x, N, out, (cudaStream_t)stream);
  return e == cudaSuccess ? CUROB_OK : CUROB_ERR_CUDA;
}

curob_status curob_h_evaluate(int fid, const double* x, int N, double* out) {
  curob_status rc = check_eval_args(fid, x, N, out);
  if (rc != CUROB_OK || N == 0) return rc;
  const size_t in = sizeof(double) * (size_t)N * g.D, ob = sizeof(double) * (size_t)N;
  std::lock_guard<std::mutex> lk(g.mu);
  if (cudaMemcpyAsync(g.d_hx, x, in, cudaMemcpyHostToDevice, g.hstream) != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (launch_simt_f64(tables(), g.func[fid], (const double*)g.d_hx, N, (double*)g.d_hout,
                      g.hstream) != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (cudaMemcpyAsync(out, g.d_hout, ob, cudaMemcpyDeviceToHost, g.hstream) != cudaSuccess ||
      cudaStreamSynchronize(g.hstream) != cudaSuccess)
    return CUROB_ERR_CUDA;
  return CUROB_OK;
}

curob_status curob_h_evaluatef(int fid, const float* x, int N, float* out) {
  curob_status rc = check_eval_args(fid, x, N, out);
  if (rc != CUROB_OK || N == 0) return rc;
  const size_t in = sizeof(float) * (size_t)N * g.D, ob = sizeof(float) * (size_t)N;
  if (cudaMemcpyAsync(g.d_hx, x, in, cudaMemcpyHostToDevice, g.hstream) != cudaSuccess)
    return CUROB_ERR_CUDA;
  rc = curob_evaluatef(fid, (const float*)g.d_hx, N, (float*)g.d_hout, g.hstream);
  if (rc != CUROB_OK) return rc;
  if (cudaMemcpyAsync(out, g.d_hout, ob, cudaMemcpyDeviceToHost, g.hstream) != cudaSuccess ||
      cudaStreamSynchronize(g.hstream) != cudaSuccess)
    return CUROB_ERR_CUDA;
  return CUROB_OK;
}

curob_status curob_set_precision(int mode) {
  if (mode < CUROB_PRECISION_AUTO || mode > CUROB_PRECISION_EXACT)
    return CUROB_ERR_INVALID_ARGUMENT;
  g.precision = mode;
  return CUROB_OK;
}

curob_status curob_query_precision(int fid, int* mode) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  if (!g.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
  if (!mode) return CUROB_ERR_NULL_POINTER;
  const int m = resolve_precision(g.func[fid]);
  if (m < 0) return CUROB_ERR_UNSUPPORTED;
  *mode = m;
  return CUROB_OK;
}

curob_status curob_get_device_status(curob_stream_t stream) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CUROB_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, g.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (st == DEV_OK) return CUROB_OK;
  cudaMemset(g.d_status, 0, sizeof(int));
  return st == DEV_TIMEOUT ? CUROB_ERR_DEVICE_TIMEOUT : CUROB_ERR_CUDA;
}

curob_status curob_get_config(int* D, int* max_concurrency) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (!D || !max_concurrency) return CUROB_ERR_NULL_POINTER;
  *D = g.D;
  *max_concurrency = g.max_conc;
  return CUROB_OK;
}

curob_status curob_num_components(int fid, int* ncomp) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  if (!g.func_ok[fid]) return CUROB_ERR_INVALID_DIM;
  if (!ncomp) return CUROB_ERR_NULL_POINTER;
  *ncomp = g.func[fid].ncomp;
  return CUROB_OK;
}

curob_status curob_component_layout(int fid, int comp, int* n_blocks, int sizes[5], int* rotated) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  int c = find_comp(fid, comp);
  if (c < 0) return g.func_ok[fid] ? CUROB_ERR_INVALID_ARGUMENT : CUROB_ERR_INVALID_DIM;
  if (!n_blocks || !sizes || !rotated) return CUROB_ERR_NULL_POINTER;
  const CompHost& ch = g.chost[c];
  for (int i = 0; i < 5; ++i) sizes[i] = 0;
  if (ch.rotated) {
    *n_blocks = (int)ch.sizes.size();
    for (size_t i = 0; i < ch.sizes.size(); ++i) sizes[i] = ch.sizes[i];
  } else {
    *n_blocks = 1;
    sizes[0] = g.D;
  }
  *rotated = ch.rotated;
  return CUROB_OK;
}

curob_status curob_get_component(int fid, int comp, double* o, int* S, double* R) {
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  int c = find_comp(fid, comp);
  if (c < 0) return g.func_ok[fid] ? CUROB_ERR_INVALID_ARGUMENT : CUROB_ERR_INVALID_DIM;
  const Component& C = g.comps[c];
  const CompHost& ch = g.chost[c];
  if (cudaDeviceSynchronize() != cudaSuccess) return CUROB_ERR_CUDA;
  if (o && cudaMemcpy(o, g.d_o + C.base, sizeof(double) * g.D, cudaMemcpyDeviceToHost) != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (S && cudaMemcpy(S, g.d_S + C.base, sizeof(int) * g.D, cudaMemcpyDeviceToHost) != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (R && ch.rotated) {
    long long off = 0;
    for (int sid : ch.segs) {
      const Segment& s = g.segs[sid];
      const size_t nn = (size_t)s.n * s.n;
      if (cudaMemcpy(R + off, g.d_R + s.r_off, sizeof(double) * nn, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
        return CUROB_ERR_CUDA;
      off += (long long)nn;
    }
  }
  return CUROB_OK;
}

curob_status curob_set_component(int fid, int comp, const double* o, const int* S, const double* R) {
  std::lock_guard<std::mutex> lk(g.mu);
  if (!g.init) return CUROB_ERR_NOT_INITIALIZED;
  if (fid < 0 || fid >= kNumFunctions) return CUROB_ERR_INVALID_FID;
  int c = find_comp(fid, comp);
  if (c < 0) return g.func_ok[fid] ? CUROB_ERR_INVALID_ARGUMENT : CUROB_ERR_INVALID_DIM;
  const Component& C = g.comps[c];
  const CompHost& ch = g.chost[c];
  if (!o || !S || (ch.rotated && !R)) return CUROB_ERR_NULL_POINTER;
  // S must be a permutation of 0..D-1 (it indexes x on the device)
  std::vector<char> seen(g.D, 0);
  for (int k = 0; k < g.D; ++k) {
    if (S[k] < 0 || S[k] >= g.D || seen[S[k]]) return CUROB_ERR_INVALID_ARGUMENT;
    seen[S[k]] = 1;
  }
  if (!ch.rotated)
    for (int k = 0; k < g.D; ++k)
      if (S[k] != k) return CUROB_ERR_INVALID_ARGUMENT;
  if (cudaDeviceSynchronize() != cudaSuccess) return CUROB_ERR_CUDA;
  CU(cudaMemcpy(g.d_o + C.base, o, sizeof(double) * g.D, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(g.d_S + C.base, S, sizeof(int) * g.D, cudaMemcpyHostToDevice));
  if (ch.rotated) {
    long long off = 0;
    for (int sid : ch.segs) {
      const Segment& s = g.segs[sid];
      const size_t nn = (size_t)s.n * s.n;
      CU(cudaMemcpy(g.d_R + s.r_off, R + off, sizeof(double) * nn, cudaMemcpyHostToDevice));
      CU(launch_split_f32(g.d_R + s.r_off, g.d_R32 + s.r_off, g.d_R32lo + s.r_off, (long long)nn, 0));
      off += (long long)nn;
    }
  }
  PermJob pj;
  memset(&pj, 0, sizeof(pj));
  pj.base = C.base;
  PermJob* d_pj = nullptr;
  CU(cudaMalloc(&d_pj, sizeof(PermJob)));
  cudaError_t e = cudaMemcpy(d_pj, &pj, sizeof(PermJob), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_operm(d_pj, 1, g.D, g.d_o, g.d_S, g.d_operm, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_pj);
  if (e != cudaSuccess) return CUROB_ERR_CUDA;
  curob_status rc = CUROB_OK;
  if (ch.rotated) rc = mma_refresh(g.mma, g.segs, ch.segs, tables());
  return rc;
}

curob_status curob_get_optimum(int fid, double* xopt) {
  if (!xopt) return CUROB_ERR_NULL_POINTER;
  return curob_get_component(fid, 0, xopt, nullptr, nullptr);
}

}  // extern "C"

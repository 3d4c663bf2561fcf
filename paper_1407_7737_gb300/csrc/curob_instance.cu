// curob_instance.cu -- construction of one instance of the suite (General
// Setup; Table 1; Sec. 3-6) on the current device: the function table, the
// component/block layout, the generated shifts, permutations and rotations,
// and the tensor-core operand images.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "curob_instance.hpp"
#include "curob_small.cuh"

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

}  // namespace

bool needs_d10(int fid) { return (fid >= 23 && fid <= 28) || fid == 35 || fid == 36; }

bool kind_has_aux(int k) { return k == K_ELLIPTIC || k == K_POWERS || k == K_GRIEWANK; }

// Builds the component and segment tables for dimension D.
void Instance::build_tables() {
  segs.clear(); comps.clear(); chost.clear();
  long long r_sum = 0, aux_sum = 0;
  for (int fid = 0; fid < kNumFunctions; ++fid) {
    func_ok[fid] = !(needs_d10(fid) && D < 10);
    if (!func_ok[fid]) continue;
    CompInfo ci = comp_info(fid);
    Function F;
    F.comp0 = (int)comps.size();
    F.ncomp = ci.n;
    F.composition = fid >= 29;
    F.max_n = 0;
    F.sensitive = 0;
    F.sens_mask = 0;
    F.hcols = 0;
    F.nseg = 0;
    F.nweier = 0;
    F.xcand = 0;
    for (int c = 0; c < ci.n; ++c) {
      const Member& m = ci.m[c];
      CompHost ch;
      ch.fid = fid;
      ch.idx = c;
      ch.rotated = m.rotated;
      member_blocks(m, D, ch.sizes);
      Component C;
      C.seg0 = (int)segs.size();
      C.base = (long long)comps.size() * D;
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
        if (!s.identity) { s.r_off = r_sum; r_sum += (long long)s.n * s.n; }
        s.aux_off = -1;
        if (kind_has_aux(s.kind)) { s.aux_off = aux_sum; aux_sum += s.n; }
        s.img_off = -1;
        s.npad = 0;
        s.comp = (int)comps.size();
        s.kat_e = s.kind == K_KATSUURA ? (float)(10.0 / std::pow((double)s.gn, 1.2)) : 0.f;
        s.hoff = -1;
        if (kind_is_heavy(s.kind)) {  // the blocks of a function stay consecutive
          s.hoff = F.hcols;
          F.hcols += s.n;
        }
        F.max_n = std::max(F.max_n, s.n);
        F.nseg += 1;
        F.nweier += s.kind == K_WEIERSTRASS ? 1 : 0;
        if (kind_is_sensitive(s.kind)) {
          F.sensitive = 1;
          F.sens_mask |= 1 << c;
        }
        ch.segs.push_back((int)segs.size());
        segs.push_back(s);
      }
      C.nseg = (int)segs.size() - C.seg0;
      bool from_x = !m.rotated && C.nseg > 0;
      for (int si = C.seg0; si < C.seg0 + C.nseg; ++si) from_x = from_x && kind_from_x(segs[si].kind);
      if (from_x) F.xcand |= 1 << c;
      comps.push_back(C);
      chost.push_back(ch);
    }
    func[fid] = F;
  }
  r_total = r_sum;
  aux_total = aux_sum;
}

#define CU_(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      return e_ == cudaErrorMemoryAllocation ? CUROB_ERR_OUT_OF_MEMORY : CUROB_ERR_CUDA; \
    }                                              \
  } while (0)

// Shift, permutation, rotations and tables for all components, on the GPU.
curob_status Instance::generate_all() {
  const int nc = (int)comps.size();
  std::vector<PermJob> pj(nc);
  std::vector<GaussJob> gj;
  std::vector<AuxJob> aj;
  int max_n = 1;
  for (int c = 0; c < nc; ++c) {
    const CompHost& ch = chost[c];
    PermJob& p = pj[c];
    memset(&p, 0, sizeof(p));
    p.base = comps[c].base;
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
      const Segment& s = segs[ch.segs[sidx++]];
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
  for (const Segment& s : segs)
    if (s.aux_off >= 0) aj.push_back(AuxJob{s.aux_off, s.kind, s.n, s.gn, s.gpos});

  if (8 * (size_t)max_n * sizeof(double) > 220 * 1024) return CUROB_ERR_UNSUPPORTED;
  // the longest Gram-Schmidt chains first (each block is done by one warp)
  std::stable_sort(gj.begin(), gj.end(),
                   [](const GaussJob& a, const GaussJob& b) { return a.n > b.n; });

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
    fail(launch_shift_perm(d_pj, nc, D, seed, d_o, d_S, d_operm, d_words, d_mark, 0));
  if (rc == CUROB_OK)
    fail(launch_gauss_gs(d_gj, (int)gj.size(), max_n, seed, d_R, d_status, 0));
  if (rc == CUROB_OK) fail(launch_aux(d_aj, (int)aj.size(), d_aux, d_aux32, 0));
  if (rc == CUROB_OK) fail(launch_split_f32(d_R, d_R32, d_R32lo, r_total, 0));
  for (size_t i = 0; i < gj.size() && rc == CUROB_OK; ++i)
    fail(launch_transpose_block(gj[i].r_off, gj[i].n, d_R, d_R32, d_R32lo, d_Rt, d_R32t,
                                d_R32lot, 0));
  if (rc == CUROB_OK) fail(cudaDeviceSynchronize());
  cudaFree(d_pj); cudaFree(d_gj); cudaFree(d_aj); cudaFree(d_words); cudaFree(d_mark);
  if (rc == CUROB_OK) {
    int st = 0;
    fail(cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (rc == CUROB_OK && st != DEV_OK) rc = CUROB_ERR_CUDA;
  }
  return rc;
}


Tables Instance::tables() const {
  Tables t;
  t.seg = d_seg;
  t.comp = d_comp;
  t.o = d_o;
  t.S = d_S;
  t.operm = d_operm;
  t.R = d_R;
  t.R32 = d_R32;
  t.R32lo = d_R32lo;
  t.Rt = d_Rt;
  t.R32t = d_R32t;
  t.R32lot = d_R32lot;
  t.aux = d_aux;
  t.aux32 = d_aux32;
  t.img = mma.img;
  t.D = D;
  t.status = d_status;
  return t;
}

void Instance::release() {
  cudaFree(d_seg); cudaFree(d_comp); cudaFree(d_o); cudaFree(d_operm);
  cudaFree(d_R); cudaFree(d_aux); cudaFree(d_S); cudaFree(d_R32); cudaFree(d_R32lo);
  cudaFree(d_Rt); cudaFree(d_R32t); cudaFree(d_R32lot);
  d_Rt = nullptr; d_R32t = d_R32lot = nullptr;
  cudaFree(d_aux32); cudaFree(d_status);
  mma_release(mma);
  f64_release(f64);
  d_seg = nullptr; d_comp = nullptr; d_o = d_operm = d_R = d_aux = nullptr;
  d_S = nullptr; d_R32 = d_R32lo = d_aux32 = nullptr; d_status = nullptr;
  segs.clear(); comps.clear(); chost.clear();
  for (int f = 0; f < kNumFunctions; ++f) func_ok[f] = false;
}

curob_status Instance::create(int D_, uint64_t seed_) {
  release();
  D = D_;
  seed = seed_;
  build_tables();
  const int nc = (int)comps.size();
  auto alloc = [&](void** p, size_t bytes) -> bool {
    return cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess;
  };
  bool ok = alloc((void**)&d_seg, sizeof(Segment) * segs.size()) &&
            alloc((void**)&d_comp, sizeof(Component) * nc) &&
            alloc((void**)&d_o, sizeof(double) * (size_t)nc * D) &&
            alloc((void**)&d_operm, sizeof(double) * (size_t)nc * D) &&
            alloc((void**)&d_S, sizeof(int) * (size_t)nc * D) &&
            alloc((void**)&d_R, sizeof(double) * (size_t)r_total) &&
            alloc((void**)&d_R32, sizeof(float) * (size_t)r_total) &&
            alloc((void**)&d_R32lo, sizeof(float) * (size_t)r_total) &&
            alloc((void**)&d_Rt, sizeof(double) * (size_t)r_total) &&
            alloc((void**)&d_R32t, sizeof(float) * (size_t)r_total) &&
            alloc((void**)&d_R32lot, sizeof(float) * (size_t)r_total) &&
            alloc((void**)&d_aux, sizeof(double) * (size_t)aux_total) &&
            alloc((void**)&d_aux32, sizeof(float) * (size_t)aux_total) &&
            alloc((void**)&d_status, sizeof(int));
  if (!ok) {
    cudaGetLastError();
    release();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  if (cudaMemset(d_status, 0, sizeof(int)) != cudaSuccess) {
    release();
    return CUROB_ERR_CUDA;
  }
  curob_status rc = generate_all();
  if (rc == CUROB_OK) rc = mma_prepare(mma, segs, tables(), nullptr);
  if (rc == CUROB_OK) rc = f64_prepare(f64, segs, comps, func, func_ok, tables());
  if (rc == CUROB_OK &&
      (cudaMemcpy(d_seg, segs.data(), sizeof(Segment) * segs.size(), cudaMemcpyHostToDevice) !=
           cudaSuccess ||
       cudaMemcpy(d_comp, comps.data(), sizeof(Component) * nc, cudaMemcpyHostToDevice) !=
           cudaSuccess))
    rc = CUROB_ERR_CUDA;
  if (rc != CUROB_OK) release();
  return rc;
}

int Instance::find_comp(int fid, int comp) const {
  if (fid < 0 || fid >= kNumFunctions || !func_ok[fid]) return -1;
  if (comp < 0 || comp >= func[fid].ncomp) return -1;
  return func[fid].comp0 + comp;
}

curob_status Instance::get_component(int fid, int comp, double* o, int* S, double* R) const {
  int c = find_comp(fid, comp);
  if (c < 0) return func_ok[fid] ? CUROB_ERR_INVALID_ARGUMENT : CUROB_ERR_INVALID_DIM;
  const Component& C = comps[c];
  const CompHost& ch = chost[c];
  if (cudaDeviceSynchronize() != cudaSuccess) return CUROB_ERR_CUDA;
  if (o && cudaMemcpy(o, d_o + C.base, sizeof(double) * D, cudaMemcpyDeviceToHost) != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (S && cudaMemcpy(S, d_S + C.base, sizeof(int) * D, cudaMemcpyDeviceToHost) != cudaSuccess)
    return CUROB_ERR_CUDA;
  if (R && ch.rotated) {
    long long off = 0;
    for (int sid : ch.segs) {
      const Segment& s = segs[sid];
      const size_t nn = (size_t)s.n * s.n;
      if (cudaMemcpy(R + off, d_R + s.r_off, sizeof(double) * nn, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
        return CUROB_ERR_CUDA;
      off += (long long)nn;
    }
  }
  return CUROB_OK;
}

curob_status Instance::set_component(int fid, int comp, const double* o, const int* S,
                                     const double* R) {
  int c = find_comp(fid, comp);
  if (c < 0) return func_ok[fid] ? CUROB_ERR_INVALID_ARGUMENT : CUROB_ERR_INVALID_DIM;
  const Component& C = comps[c];
  const CompHost& ch = chost[c];
  if (!o || !S || (ch.rotated && !R)) return CUROB_ERR_NULL_POINTER;
  // S must be a permutation of 0..D-1 (it indexes x on the device)
  std::vector<char> seen(D, 0);
  for (int k = 0; k < D; ++k) {
    if (S[k] < 0 || S[k] >= D || seen[S[k]]) return CUROB_ERR_INVALID_ARGUMENT;
    seen[S[k]] = 1;
  }
  if (!ch.rotated)
    for (int k = 0; k < D; ++k)
      if (S[k] != k) return CUROB_ERR_INVALID_ARGUMENT;
  if (cudaDeviceSynchronize() != cudaSuccess) return CUROB_ERR_CUDA;
  CU_(cudaMemcpy(d_o + C.base, o, sizeof(double) * D, cudaMemcpyHostToDevice));
  CU_(cudaMemcpy(d_S + C.base, S, sizeof(int) * D, cudaMemcpyHostToDevice));
  if (ch.rotated) {
    long long off = 0;
    for (int sid : ch.segs) {
      const Segment& s = segs[sid];
      const size_t nn = (size_t)s.n * s.n;
      CU_(cudaMemcpy(d_R + s.r_off, R + off, sizeof(double) * nn, cudaMemcpyHostToDevice));
      CU_(launch_split_f32(d_R + s.r_off, d_R32 + s.r_off, d_R32lo + s.r_off, (long long)nn, 0));
      CU_(launch_transpose_block(s.r_off, s.n, d_R, d_R32, d_R32lo, d_Rt, d_R32t, d_R32lot, 0));
      off += (long long)nn;
    }
  }
  PermJob pj;
  memset(&pj, 0, sizeof(pj));
  pj.base = C.base;
  PermJob* d_pj = nullptr;
  CU_(cudaMalloc(&d_pj, sizeof(PermJob)));
  cudaError_t e = cudaMemcpy(d_pj, &pj, sizeof(PermJob), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_operm(d_pj, 1, D, d_o, d_S, d_operm, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_pj);
  if (e != cudaSuccess) return CUROB_ERR_CUDA;
  std::vector<int> ids = ch.segs;
  const curob_status rc = mma_refresh(mma, segs, ids, tables());
  return rc == CUROB_OK ? f64_refresh(f64, segs, ids, tables()) : rc;
}

void fill_small_args(SmallArgs& a, const Instance& I, const Function& F) {
  memset(&a, 0, sizeof(a));
  a.tb = I.tables();
  a.F = F;
  a.seg_base = I.comps[F.comp0].seg0;
  for (int i = 0; i < F.nseg && i < kSmallMaxWarps; ++i) a.seg[i] = I.segs[a.seg_base + i];
  for (int c = 0; c < F.ncomp; ++c) a.comp[c] = I.comps[F.comp0 + c];
}

}  // namespace curob

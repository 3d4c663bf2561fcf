// curob_mma.cu -- tensor-core evaluator of curob_evaluatef (sm_103a).
//
// The block rotation z_b = R_b y_b of the General Setup is a dense
// contraction per block: for a tile of 128 candidates, Z_b (128 x n_b) =
// Y_b (128 x n_b) R_b^T, run on tcgen05 with the accumulators in tensor
// memory (TMEM), then transformed and reduced by the epilogue warps straight
// out of TMEM.  Three precisions:
//   TF32X3  y = yh + yl, R = Rh + Rl (TF32 halves), Z = Yh Rh + Yh Rl + Yl Rh,
//           one FP32 accumulator;
//   BF16X3  the same with BF16 halves;
//   EXACT   128 y / sigma_m and 128 R / tau_i (sigma, tau powers of two) cut
//           into four integer slices each (|s| <= 128: the leading one, then
//           8 more bits each), held exactly in BF16 and pre-scaled by their
//           weight (s_a 2^-8(a-1)).  The leading product s1 r1 accumulates
//           alone: every partial sum is an integer of magnitude below 2^23,
//           so its FP32 accumulation is exact whatever the tensor core's
//           rounding; the nine products of weight 2^-8 to 2^-24 share a
//           second accumulator 2^-8 below it, so its rounding (and any
//           truncation bias of the FP32 accumulation) is scaled down by
//           2^-8; dropped products weigh <= 2^-32.  z = sigma tau 2^-14
//           (A0 + A1), to ~2^-26 of the row scale.  (The error-free splitting of matrix products of
//           Ozaki, Ogita, Oishi and Rump, with BF16 integer slices.)
// The tensor core's FP32 accumulation truncates: over a 334-long block TF32X3
// loses ~2e-6 of |z| systematically, which the functions that magnify z
// errors (Discus, Weierstrass, Griewank-Rosenbrock, Katsuura) cannot absorb;
// they take EXACT.
//
// Warp roles of one CTA (one tile of 128 candidates, 1 CTA per SM):
//   warps 0-3  producers: thread = candidate row.  Per block the block's
//              index list and o hi/lo words are staged in shared memory; per
//              K stage a thread gathers its row's x at the block's variables
//              (prefetching the next stage's values), takes y = x - o in
//              double-float (exact TwoSum, then o's low word), splits or
//              slices it and stores its 64-byte rows of the A operand in the
//              64-byte-swizzled K-major layout; it also sums ||x - o||^2.
//   warps 4-7  epilogue: thread t owns row t (TMEM lane t), loads its z
//              32 columns at a time (tcgen05.ld), applies z = s z + c, the
//              per-variable transform and the running sums (FP32 per 32
//              columns, FP64 across), closes functions.
//   warp 8     allocates TMEM and issues the MMAs (one lane).
//   warp 9     loads the B operand (R_b parts, pre-laid-out in global memory
//              as the exact shared-memory image) with one bulk copy per stage
//              (cp.async.bulk, the TMA engine).
// Stages rotate through shared memory under full/empty mbarriers; the
// accumulators are handed from the MMA warp to the epilogue and back under
// tmem_full/tmem_empty.  Every wait is bounded: past ~2 s it raises
// DEV_TIMEOUT in the status word, the CTA stops, and TMEM is freed before
// exit.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "curob_mma.hpp"
#include "curob_tc.cuh"

namespace curob {
namespace {

using namespace tc;

constexpr int kTileM = 128;
constexpr int kThreads = 320;
constexpr int kPartBytes = kTileM * kRowBytes;   // 8 KB per A part
constexpr int kMaxNpad = 512;                    // TMEM columns
constexpr int kExactMaxNC = 192;                 // EXACT: widest N chunk
constexpr int kExactAcc1 = 256;                  // EXACT: TMEM column of accumulator 1
constexpr int kSigRing = 8;                      // EXACT: row scales in flight

enum Mode : int { M_TF32 = 0, M_BF16 = 1, M_EXACT = 2 };

// EXACT splits a block's npad output columns into nchunk equal chunks of at
// most kExactMaxNC (a multiple of 16 wide): accumulators 0 and 1 of a chunk
// sit at TMEM columns [0, nw) and [256, 256 + nw).
__host__ __device__ inline int exact_nchunk(int npad) {
  return (npad + kExactMaxNC - 1) / kExactMaxNC;
}
__host__ __device__ inline int exact_nw(int npad) {
  const int n = exact_nchunk(npad);
  return ((npad + n - 1) / n + 15) / 16 * 16;
}

// x - o with o = ohi + olo as a double-float (yh, yl): TwoSum(x, -ohi) is
// exact, then the low word of o.
__device__ __forceinline__ void shift_ff(float x, float ohi, float olo, float& yh, float& yl) {
  const float s = __fsub_rn(x, ohi);
  const float bb = __fsub_rn(s, x);
  const float err = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(-ohi, bb));
  const float t = __fsub_rn(err, olo);
  yh = __fadd_rn(s, t);
  yl = __fsub_rn(t, __fsub_rn(yh, s));
}

// Mode constants.
template <int kMode> struct MC {
  static constexpr int kParts = kMode == M_EXACT ? 4 : 2;  // A/B operand parts
  static constexpr int kKs = kMode == M_TF32 ? 16 : 32;    // K columns per stage
  static constexpr int kEl = kMode == M_TF32 ? 4 : 2;      // bytes per element
  static constexpr int kMmaK = kMode == M_TF32 ? 8 : 16;   // K per MMA
  static constexpr uint32_t kFmt = kMode == M_TF32 ? 2u : 1u;
};

struct MmaArgs {
  Tables tb;
  Function F;
  const float* x;
  float* out;
  int N;
  const float* ohi;      // o[S[k]] high words per component
  const float* olo;      // low words
  const uint8_t* img;    // operand images
  const float* tau;      // EXACT: row scales of R (powers of two)
  const float* onat;     // EXACT: o per component in natural order, FP32
  int nstage;
  int stage_bytes;
};

// Floats reserved per block for each precision's image (the TF32 size; BF16
// needs half).  A block's images: [TF32][BF16][EXACT].
__host__ __device__ inline long long image_floats(int npad) { return 2LL * npad * npad; }

// ------------------------------------------------------- epilogue helpers
// Running state of the open basic function of one candidate row.
struct EpiState {
  double a0 = 0, a1 = 0, a2 = 0, p = 1;
  float zfirst = 0.f, zprev = 0.f;
  __device__ void open() {
    a0 = a1 = a2 = 0.0;
    p = 1.0;
  }
  // closes the function (cyclic pair, closing map); value without f_opt
  __device__ double close(int kind, int gn) {
    if (kind_is_cyclic(kind)) a0 += (double)pair_term<float>(kind, zprev, zfirst);
    return finalize_f32(kind, a0, a1, a2, p, gn);
  }
};
struct EpiSeg {
  float s, c0, gnT, kat_e;
  const float* aux;
  int gpos, gfirst;
};

// Kinds whose per-variable term calls transcendentals with slow paths (large
// arguments): their terms are out-of-line calls on four variables at a time,
// so the unrolled chunk loop stays small while the four independent
// evaluations interleave (one epilogue warp per scheduler has no other warp
// to hide their latency); contributions come back by value (no local memory).
__host__ __device__ constexpr bool kind_is_heavy(int k) {
  return k == K_POWERS || k == K_WEIERSTRASS || k == K_GRIEWANK || k == K_SCHAFFER7 ||
         k == K_EGR || k == K_SCHWEFEL || k == K_KATSUURA || k == K_SCHAFFER6;
}
// Sums (a0, a1, a2) and product (p) of the terms of the first n <= 4 of four
// consecutive variables.
template <int KIND>
__device__ __noinline__ float4 heavy_term4(float4 z, float4 u, int gi, float gn, float4 aux,
                                           float kat_e, int n) {
  const float zs[4] = {z.x, z.y, z.z, z.w}, us[4] = {u.x, u.y, u.z, u.w};
  const float as[4] = {aux.x, aux.y, aux.z, aux.w};
  Acc<float> t[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    t[e] = acc_zero<float>();
    elem_term_f32(KIND, zs[e], us[e], gi + e, gn, as[e], kat_e, t[e]);
  }
  float4 r = make_float4(0.f, 0.f, 0.f, 1.f);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (e < n) {
      r.x += t[e].a0;
      r.y += t[e].a1;
      r.z += t[e].a2;
      r.w *= t[e].p;
    }
  }
  return r;
}
// Sum of the pair terms (zp_e, z_e) of four consecutive variables, e in
// [first, n).
template <int KIND>
__device__ __noinline__ float heavy_pair4(float4 zp, float4 z, int first, int n) {
  const float ps[4] = {zp.x, zp.y, zp.z, zp.w}, zs[4] = {z.x, z.y, z.z, z.w};
  float t[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) t[e] = pair_term<float>(KIND, ps[e], zs[e]);
  float r = 0.f;
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (e >= first && e < n) r += t[e];
  return r;
}

// 32 accumulator columns [c, c + cend) of one row, for a fixed kind: the
// loop is unrolled so the values stay in registers.
template <int KIND>
__device__ __forceinline__ void epi_chunk_k(const float* v, int c, int cend, const EpiSeg& es,
                                            EpiState& st) {
  constexpr bool kPairs = (KIND == K_SCHAFFER7 || KIND == K_EGR || KIND == K_ROSENBROCK ||
                           KIND == K_SCHAFFER6);
  constexpr bool kAux = (KIND == K_ELLIPTIC || KIND == K_POWERS || KIND == K_GRIEWANK);
  Acc<float> part = acc_zero<float>();
  if constexpr (kind_is_heavy(KIND)) {
    const bool opens = (c == 0 && es.gfirst);  // column 0 opens the function
    float zlast = st.zprev;
#pragma unroll
    for (int g = 0; g < 32; g += 4) {
      if (g < cend) {
        const int n = min(4, cend - g);
        float4 u4 = make_float4(v[g] * es.s, v[g + 1] * es.s, v[g + 2] * es.s, v[g + 3] * es.s);
        float4 z4 = make_float4(u4.x + es.c0, u4.y + es.c0, u4.z + es.c0, u4.w + es.c0);
        if constexpr (kPairs) {
          const float zp0 = g == 0 ? st.zprev : v[g > 0 ? g - 1 : 0] * es.s + es.c0;
          const float4 zp4 = make_float4(zp0, z4.x, z4.y, z4.z);
          part.a0 += heavy_pair4<KIND>(zp4, z4, (g == 0 && opens) ? 1 : 0, n);
        } else {
          float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
          if constexpr (kAux) {
            const float* ap = es.aux + c + g;
            a4 = make_float4(ap[0], n > 1 ? ap[1] : 0.f, n > 2 ? ap[2] : 0.f, n > 3 ? ap[3] : 0.f);
          }
          const float4 t = heavy_term4<KIND>(z4, u4, es.gpos + c + g, es.gnT, a4, es.kat_e, n);
          part.a0 += t.x;
          part.a1 += t.y;
          part.a2 += t.z;
          part.p *= t.w;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (e == n - 1) zlast = v[g + e] * es.s + es.c0;
      }
    }
    if (opens) st.zfirst = v[0] * es.s + es.c0;
    st.zprev = zlast;
  } else {
    float zprev = st.zprev;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k < cend) {
        const int col = c + k;
        const float u = v[k] * es.s;  // z before its offset
        const float z = u + es.c0;
        elem_term_f32(KIND, z, u, es.gpos + col, es.gnT, kAux ? es.aux[col] : 0.f, es.kat_e,
                      part);
        if (kPairs) {
          if (col == 0 && es.gfirst) st.zfirst = z;
          else part.a0 += pair_term<float>(KIND, zprev, z);
        } else if (col == 0 && es.gfirst) {
          st.zfirst = z;
        }
        zprev = z;
      }
    }
    st.zprev = zprev;
  }
  st.a0 += (double)part.a0;
  st.a1 += (double)part.a1;
  st.a2 += (double)part.a2;
  st.p *= (double)part.p;
}

__device__ __forceinline__ void epi_chunk(int kind, const float* v, int c, int cend,
                                          const EpiSeg& es, EpiState& st) {
  switch (kind) {
#define CUROB_EPI_CASE(K) \
  case K: epi_chunk_k<K>(v, c, cend, es, st); break;
    CUROB_EPI_CASE(K_SPHERE) CUROB_EPI_CASE(K_ELLIPSOID) CUROB_EPI_CASE(K_ELLIPTIC)
    CUROB_EPI_CASE(K_DISCUS) CUROB_EPI_CASE(K_CIGAR) CUROB_EPI_CASE(K_POWERS)
    CUROB_EPI_CASE(K_SHARPV) CUROB_EPI_CASE(K_STEP) CUROB_EPI_CASE(K_WEIERSTRASS)
    CUROB_EPI_CASE(K_GRIEWANK) CUROB_EPI_CASE(K_RASTRIGIN) CUROB_EPI_CASE(K_SCHAFFER7)
    CUROB_EPI_CASE(K_EGR) CUROB_EPI_CASE(K_ROSENBROCK) CUROB_EPI_CASE(K_SCHWEFEL)
    CUROB_EPI_CASE(K_KATSUURA) CUROB_EPI_CASE(K_LUNACEK) CUROB_EPI_CASE(K_ACKLEY)
    CUROB_EPI_CASE(K_HAPPYCAT) CUROB_EPI_CASE(K_HGBAT) CUROB_EPI_CASE(K_SCHAFFER6)
#undef CUROB_EPI_CASE
    default: break;
  }
}

// -------------------------------------------------------------- the kernel
// Shared-memory map of a CTA (identical for the per-launch and the
// persistent kernels).
struct Smem {
  uint8_t* stages;
  uint64_t *full, *empty, *tmem_full, *tmem_empty, *sig_full, *prod_bar, *gbar;
  uint32_t* tmem_slot;
  volatile int* abort_flag;
  double *rowG, *rowD2;
  float* rowSig;
  int* tabS;
  float *tabH, *tabL;
  int* item;  // persistent kernel: the work item of the CTA
};

__device__ inline Smem smem_map(uint8_t* smem_raw, int nstage, int stage_bytes) {
  Smem m;
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  m.stages = smem;
  uint8_t* ctrl = smem + (size_t)nstage * stage_bytes;
  m.full = reinterpret_cast<uint64_t*>(ctrl);
  m.empty = m.full + nstage;
  m.tmem_full = m.empty + nstage;
  m.tmem_empty = m.tmem_full + 1;
  m.sig_full = m.tmem_empty + 1;  // [kSigRing]
  m.prod_bar = m.sig_full + kSigRing;
  m.gbar = m.prod_bar + 1;        // [nstage]
  m.tmem_slot = reinterpret_cast<uint32_t*>(m.gbar + nstage);
  m.abort_flag = reinterpret_cast<volatile int*>(m.tmem_slot + 1);
  m.item = const_cast<int*>(reinterpret_cast<volatile int*>(m.abort_flag) + 1);
  m.rowG = reinterpret_cast<double*>(ctrl + 256);                 // [kMaxComponents][128]
  m.rowD2 = m.rowG + kMaxComponents * kTileM;                     // [kMaxComponents][128]
  m.rowSig = reinterpret_cast<float*>(m.rowD2 + kMaxComponents * kTileM);  // [kSigRing][128]
  m.tabS = reinterpret_cast<int*>(m.rowSig + kSigRing * kTileM);           // [kMaxNpad]
  m.tabH = reinterpret_cast<float*>(m.tabS + kMaxNpad);
  m.tabL = m.tabH + kMaxNpad;
  return m;
}

// Barrier-phase counters of one role, carried from tile to tile.
struct RoleState {
  uint32_t it = 0;        // K stages
  uint32_t chunk_it = 0;  // accumulator hand-offs
  uint32_t pphase = 0;    // producer group barrier uses
  uint32_t comp_it = 0;   // components (row-scale ring)
};

__device__ inline void cta_setup(const Smem& m, int nstage) {
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstage; ++s) {
      mbar_init(&m.full[s], 5);   // 4 producer warps + the B loader's expect_tx
      mbar_init(&m.empty[s], 1);  // one tcgen05.commit
      mbar_init(&m.gbar[s], 128); // producer threads' cp.async
    }
    mbar_init(m.tmem_full, 1);
    mbar_init(m.tmem_empty, 4);   // the 4 epilogue warps
    for (int s = 0; s < kSigRing; ++s) mbar_init(&m.sig_full[s], 4);
    mbar_init(m.prod_bar, 4);     // the 4 producer warps
    *m.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(m.tmem_slot)),
                 "r"(kMaxNpad));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Epilogue threads write f of their rows once every role is done with the
// tile (after a CTA barrier).
__device__ inline void write_outputs(const MmaArgs& a, const Smem& m, long long row0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 4 || warp >= 8 || *m.abort_flag) return;
  const int r = (warp - 4) * 32 + lane;
  const long long grow = row0 + r;
  if (grow >= a.N) return;
  const Function& F = a.F;
  double f;
  if (F.composition) {
    double G[kMaxComponents], d2v[kMaxComponents];
    for (int ci = 0; ci < F.ncomp; ++ci) {
      G[ci] = m.rowG[ci * kTileM + r];
      d2v[ci] = m.rowD2[ci * kTileM + r];
    }
    f = compose(a.tb.comp + F.comp0, F.ncomp, G, d2v, a.tb.D);
  } else {
    f = m.rowG[r];
  }
  a.out[grow] = (float)(f + kFopt);
}

__device__ inline void cta_teardown(const Smem& m) {
  const int warp = threadIdx.x >> 5;
  if (warp == 8) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*m.tmem_slot),
                 "r"(kMaxNpad));
  }
}

#define CUROB_ROLE_PROLOGUE                                                   \
  using C = MC<kMode>;                                                        \
  constexpr int kKs = C::kKs, kEl = C::kEl, kParts = C::kParts;               \
  constexpr int kKsteps = kKs / C::kMmaK;                                     \
  (void)kEl; (void)kParts; (void)kKsteps;                                     \
  const Tables& tb = a.tb;                                                    \
  const Function& F = a.F;                                                    \
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;                 \
  (void)lane;                                                                 \
  uint8_t* stages = m.stages;                                                 \
  uint64_t *full = m.full, *empty = m.empty, *tmem_full = m.tmem_full;        \
  uint64_t *tmem_empty = m.tmem_empty, *sig_full = m.sig_full;                \
  uint64_t *prod_bar = m.prod_bar, *gbar = m.gbar;                            \
  volatile int* abort_flag = m.abort_flag;                                    \
  double *rowG = m.rowG, *rowD2 = m.rowD2;                                    \
  float* rowSig = m.rowSig;                                                   \
  int* tabS = m.tabS;                                                         \
  float *tabH = m.tabH, *tabL = m.tabL;                                       \
  const uint32_t tmem_base = *m.tmem_slot;                                    \
  const int D = tb.D;                                                         \
  (void)full; (void)empty; (void)tmem_full; (void)tmem_empty; (void)sig_full; \
  (void)prod_bar; (void)gbar; (void)rowG; (void)rowD2; (void)rowSig;          \
  (void)tabS; (void)tabH; (void)tabL; (void)tmem_base; (void)D; (void)stages; \
  (void)warp;

template <int kMode>
__device__ void producer_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs) {
  CUROB_ROLE_PROLOGUE
    // ------------------------------------------------------------ producers
    // Thread = candidate row r.  The raw x values of a K stage are gathered
    // with 4-byte cp.async straight into the stage's own A area (row r only:
    // the first 64 bytes of part 0's row r, then part 1's), nstage - 1 stages
    // ahead; converting a stage reads the thread's own raw row back, then
    // overwrites that row of every part, so no other thread is involved.
    const int r = warp * 32 + lane;
    const long long grow = row0 + r;
    const bool vrow = grow < a.N;
    const float* xrow = a.x + (vrow ? grow : 0) * (long long)D;
    const int P = a.nstage - 1;  // gather prefetch depth (stages)
    uint32_t& it = rs.it;
    uint32_t& pphase = rs.pphase;
    bool ok = true;
    for (int ci = 0; ci < F.ncomp && ok; ++ci, ++rs.comp_it) {
      const uint32_t cg = rs.comp_it;  // component counter across tiles
      const Component Cm = tb.comp[F.comp0 + ci];
      const int* S = tb.S + Cm.base;
      const float* ohi = a.ohi + Cm.base;
      const float* olo = a.olo + Cm.base;
      double d2 = 0.0;
      float isig = 1.f;
      if constexpr (kMode == M_EXACT) {
        // row scale sigma_m = 2^e > max_j |x_j - o_j| over the component,
        // read in natural order (contiguous row, o as FP32)
        float mx = 0.f;
        if (vrow) {
          const float* on = a.onat + Cm.base;
          int k = 0;
          if ((D & 3) == 0) {
            const float4* x4 = reinterpret_cast<const float4*>(xrow);
            const float4* o4 = reinterpret_cast<const float4*>(on);
#pragma unroll 4
            for (; k < D / 4; ++k) {
              const float4 a = __ldg(x4 + k), b = __ldg(o4 + k);
              mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a.x - b.x), fabsf(a.y - b.y)),
                                   fmaxf(fabsf(a.z - b.z), fabsf(a.w - b.w))));
            }
            k *= 4;
          }
          for (; k < D; ++k) mx = fmaxf(mx, fabsf(__ldg(xrow + k) - on[k]));
        }
        int e = 0;
        if (mx > 0.f && mx < 3.0e38f) e = ilogbf(mx * 1.0009765625f) + 1;
        isig = ldexpf(1.f, -e);
        rowSig[(cg % kSigRing) * kTileM + r] = ldexpf(1.f, e);
        __syncwarp();
        if (lane == 0) mbar_arrive(&sig_full[cg % kSigRing]);
      }
      for (int si = 0; si < Cm.nseg && ok; ++si) {
        const Segment sg = tb.seg[Cm.seg0 + si];
        // stage the block's index list and o words in shared memory (the
        // previous block's readers are done at the first barrier)
        if (!producers_sync(prod_bar, pphase, abort_flag, tb.status)) { ok = false; break; }
        for (int k = r; k < sg.npad; k += kTileM) {
          const bool in = k < sg.n;
          tabS[k] = in ? S[sg.zoff + k] : 0;
          tabH[k] = in ? ohi[sg.zoff + k] : 0.f;
          tabL[k] = in ? olo[sg.zoff + k] : 0.f;
        }
        if (!producers_sync(prod_bar, pphase, abort_flag, tb.status)) { ok = false; break; }
        const int nslab = sg.npad / kKs;
        const int nchunk = kMode == M_EXACT ? exact_nchunk(sg.npad) : 1;
        const int total = nslab * nchunk;  // stages of this block
        const uint32_t it0 = it;
        // raw x of stage q, row rr: kKs floats at part 0 row rr (first 16)
        // and part 1 row rr (next 16).  Lanes walk a row's (sorted) columns,
        // so one instruction touches one or two rows' few sectors; each
        // thread's copies arrive on gbar[stage] when they land.
        const float* xbase = a.x;
        const long long nrows = a.N;
        const int nst = a.nstage, sbytes = a.stage_bytes, nvalid = sg.n;
        auto issue = [=](int q) -> bool {
          const uint32_t g = it0 + (uint32_t)q;
          const int stage = g % nst;
          if (!mbar_wait(&empty[stage], ((g / nst) & 1u) ^ 1u, abort_flag, tb.status))
            return false;
          uint8_t* A = stages + (size_t)stage * sbytes;
          const int t = q % nslab;
          constexpr int kRowsPerInst = 32 / kKs;            // 2 (TF32) or 1
          const int k = lane % kKs;                         // column of the stage
          const int j = t * kKs + k;
          const bool cin = j < nvalid;
          const int col = cin ? tabS[j] : 0;
          const uint32_t dcol = (uint32_t)((k >> 4) * kPartBytes + (k & 15) * 4);
          const uint32_t dbase = smem_u32(A) + dcol;
#pragma unroll 4
          for (int i = 0; i < 32 / kRowsPerInst; ++i) {
            const int rr = warp * 32 + i * kRowsPerInst + lane / kKs;
            const long long gr = row0 + rr;
            const bool in = cin && gr < nrows;
            const float* src = in ? xbase + gr * (long long)D + col : xbase;
            const uint32_t dst = dbase + (uint32_t)(rr * kRowBytes);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                         "r"(in ? 4 : 0)
                         : "memory");
          }
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                           smem_u32(&gbar[stage]))
                       : "memory");
          return true;
        };
        const int npre = min(P, total);
        for (int q = 0; q < npre && ok; ++q) ok = issue(q);
        for (int q = 0; q < total && ok; ++q, ++it) {
          if (!mbar_wait(&gbar[it % a.nstage], (it / a.nstage) & 1u, abort_flag, tb.status)) {
            ok = false;
            break;
          }
          const int stage = it % a.nstage;
          uint8_t* A = stages + (size_t)stage * a.stage_bytes;
          const int t = q % nslab;
          // the row's raw x of this stage, read before any part is overwritten
          float4 xr[kKs / 4];
#pragma unroll
          for (int k = 0; k < kKs; k += 4)
            xr[k / 4] = *reinterpret_cast<const float4*>(A + (k >> 4) * kPartBytes +
                                                         r * kRowBytes + (k & 15) * 4);
          constexpr int kPer = 16 / kEl;  // elements per 16-byte chunk
          float d2p = 0.f;
          // one 64-byte row per part = four 16-byte chunks, each stored whole
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float yh[kPer], yl[kPer];
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
              const int k = c * kPer + e;
              const int j = t * kKs + k;
              const float4 q4 = xr[k / 4];
              const float xv = (k & 3) == 0 ? q4.x : (k & 3) == 1 ? q4.y : (k & 3) == 2 ? q4.z : q4.w;
              if (vrow && j < sg.n) {
                shift_ff(xv, tabH[j], tabL[j], yh[e], yl[e]);
              } else {
                yh[e] = 0.f;
                yl[e] = 0.f;
              }
              d2p = fmaf(yh[e], yh[e], d2p);
            }
            const uint32_t off = swz64((uint32_t)r, (uint32_t)(c * 16));
            if constexpr (kMode == M_TF32) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const float a = yh[qq];
                hw[qq] = to_tf32(a);
                lw[qq] = to_tf32((a - __uint_as_float(hw[qq])) + yl[qq]);
              }
              *reinterpret_cast<uint4*>(A + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(A + kPartBytes + off) =
                  make_uint4(lw[0], lw[1], lw[2], lw[3]);
            } else if constexpr (kMode == M_BF16) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const float a = yh[2 * qq], b = yh[2 * qq + 1];
                hw[qq] = pack_bf16(a, b);
                const float2 hf = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&hw[qq]));
                lw[qq] = pack_bf16((a - hf.x) + yl[2 * qq], (b - hf.y) + yl[2 * qq + 1]);
              }
              *reinterpret_cast<uint4*>(A + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(A + kPartBytes + off) =
                  make_uint4(lw[0], lw[1], lw[2], lw[3]);
            } else {
              // four integer slices of 128 y / sigma (exact in BF16),
              // pre-scaled by their weight
              uint32_t w[4][4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                float sl[2][4];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                  const int k = 2 * qq + e;
                  const float v = yh[k] * isig * 128.f;
                  const float y1 = rintf(v);
                  const float v2 = ((v - y1) + yl[k] * isig * 128.f) * 256.f;
                  const float y2 = rintf(v2);
                  const float v3 = (v2 - y2) * 256.f;
                  const float y3 = rintf(v3);
                  const float y4 = rintf((v3 - y3) * 256.f);
                  sl[e][0] = y1;
                  sl[e][1] = y2 * 0.00390625f;
                  sl[e][2] = y3 * 1.52587890625e-05f;
                  sl[e][3] = y4 * 5.9604644775390625e-08f;
                }
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) w[pp][qq] = pack_bf16(sl[0][pp], sl[1][pp]);
              }
#pragma unroll
              for (int pp = 0; pp < 4; ++pp)
                *reinterpret_cast<uint4*>(A + pp * kPartBytes + off) =
                    make_uint4(w[pp][0], w[pp][1], w[pp][2], w[pp][3]);
            }
          }
          if (q < nslab) d2 += (double)d2p;  // first chunk: ||x - o||^2 of the row
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[stage]);
          if (q + P < total) ok = issue(q + P);
        }
      }
      rowD2[ci * kTileM + r] = d2;
    }
}

template <int kMode>
__device__ void epilogue_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs) {
  CUROB_ROLE_PROLOGUE
  (void)row0;
    // ------------------------------------------------------------- epilogue
    const int q = warp - 4;                 // TMEM lane quadrant
    const int r = q * 32 + lane;            // candidate row in the tile
    const uint32_t t_lane = tmem_base + ((uint32_t)(q * 32) << 16);
    uint32_t& chunk_it = rs.chunk_it;
    EpiState st;
    for (int ci = 0; ci < F.ncomp && !*abort_flag; ++ci, ++rs.comp_it) {
      const uint32_t cg = rs.comp_it;
      const Component Cm = tb.comp[F.comp0 + ci];
      double gsum = 0.0;
      float sig = 1.f;
      if constexpr (kMode == M_EXACT) {
        if (!mbar_wait(&sig_full[cg % kSigRing], (cg / kSigRing) & 1u, abort_flag, tb.status))
          break;
        sig = rowSig[(cg % kSigRing) * kTileM + r];
      }
      bool ok = true;
      for (int si = 0; si < Cm.nseg && ok; ++si) {
        const Segment sg = tb.seg[Cm.seg0 + si];
        const int kind = sg.kind;
        EpiSeg es;
        es.s = (float)sg.scale;
        es.c0 = (float)sg.offset;
        es.gnT = (float)sg.gn;
        es.kat_e = (kind == K_KATSUURA) ? (float)(10.0 / pow((double)sg.gn, 1.2)) : 0.f;
        es.aux = sg.aux_off >= 0 ? tb.aux32 + sg.aux_off : nullptr;
        es.gpos = sg.gpos;
        es.gfirst = sg.gfirst;
        const float* tau = a.tau + sg.tau_off;
        if (sg.gfirst) st.open();
        const int nchunk = kMode == M_EXACT ? exact_nchunk(sg.npad) : 1;
        const int nw = kMode == M_EXACT ? exact_nw(sg.npad) : sg.npad;
        for (int cc = 0; cc < nchunk; ++cc, ++chunk_it) {
          if (!mbar_wait(tmem_full, chunk_it & 1u, abort_flag, tb.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int c_lo = kMode == M_EXACT ? cc * nw : 0;
          const int c_hi = kMode == M_EXACT ? min(sg.n, c_lo + nw) : sg.n;
          for (int c = c_lo; c < c_hi; c += 32) {
            float v[32];
            if constexpr (kMode == M_EXACT) {
              float g1[32];
              const uint32_t lc = (uint32_t)(c - c_lo);
              tmem_ld32(t_lane + lc, v);
              tmem_ld32(t_lane + kExactAcc1 + lc, g1);
              const float base = sig * 6.103515625e-05f;  // sigma 2^-14
#pragma unroll
              for (int k = 0; k < 32; ++k)
                v[k] = (c + k < c_hi) ? (v[k] + g1[k]) * (base * tau[c + k]) : 0.f;
            } else {
              tmem_ld32(t_lane + (uint32_t)c, v);
            }
            epi_chunk(kind, v, c, min(32, c_hi - c), es, st);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tmem_empty);
        }
        if (ok && sg.glast) gsum += st.close(kind, sg.gn);
      }
      if (!ok) break;
      rowG[ci * kTileM + r] = gsum;
    }
}

template <int kMode>
__device__ void mma_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs) {
  CUROB_ROLE_PROLOGUE
  (void)row0;
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      uint32_t& it = rs.it;
      uint32_t& chunk_it = rs.chunk_it;
      bool ok = true;
      for (int ci = 0; ci < F.ncomp && ok && !*abort_flag; ++ci) {
        const Component Cm = tb.comp[F.comp0 + ci];
        for (int si = 0; si < Cm.nseg && ok; ++si) {
          const Segment sg = tb.seg[Cm.seg0 + si];
          const int nslab = sg.npad / kKs;
          const int nchunk = kMode == M_EXACT ? exact_nchunk(sg.npad) : 1;
          const int nw = kMode == M_EXACT ? exact_nw(sg.npad) : sg.npad;
          for (int cc = 0; cc < nchunk && ok; ++cc, ++chunk_it) {
            const int nc = kMode == M_EXACT ? min(nw, sg.npad - cc * nw) : sg.npad;
            const int n0 = nc > 256 ? 256 : nc;  // N per MMA <= 256
            const int n1 = nc - n0;
            const uint32_t id0 = idesc_make(C::kFmt, kTileM, (uint32_t)n0);
            const uint32_t id1 = idesc_make(C::kFmt, kTileM, (uint32_t)(n1 > 0 ? n1 : 16));
            if (!mbar_wait(tmem_empty, (chunk_it & 1u) ^ 1u, abort_flag, tb.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            for (int t = 0; t < nslab; ++t, ++it) {
              const int stage = it % a.nstage;
              const uint32_t ph = (it / a.nstage) & 1u;
              if (!mbar_wait(&full[stage], ph, abort_flag, tb.status)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_u32(stages + (size_t)stage * a.stage_bytes);
              const uint32_t sb = sa + kParts * kPartBytes;
              const uint32_t bpart = (uint32_t)(nc * kRowBytes);
#pragma unroll
              for (int kk = 0; kk < kKsteps; ++kk) {
                const uint32_t ko = (uint32_t)(kk * C::kMmaK * kEl);  // 32 B per K step
                const uint32_t first = (t == 0 && kk == 0) ? 0u : 1u;
                if constexpr (kMode == M_EXACT) {
                  // s1 r1 into accumulator 0; the pre-scaled products of
                  // weight 2^-8 to 2^-24 (a + b <= 3) into accumulator 1
                  constexpr int kPa[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
                  constexpr int kPb[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
#pragma unroll
                  for (int pq = 0; pq < 10; ++pq) {
                    const uint32_t dt = tmem_base + (pq == 0 ? 0u : (uint32_t)kExactAcc1);
                    const uint64_t da = sdesc_sw64(sa + kPa[pq] * kPartBytes + ko);
                    const uint64_t db = sdesc_sw64(sb + kPb[pq] * bpart + ko);
                    tc_mma<false>(dt, da, db, id0, (pq <= 1) ? first : 1u);
                  }
                } else {
                  const uint64_t dah = sdesc_sw64(sa + ko), dal = sdesc_sw64(sa + kPartBytes + ko);
                  for (int h = 0; h < (n1 > 0 ? 2 : 1); ++h) {
                    const uint32_t boff = (uint32_t)(h * n0 * kRowBytes) + ko;
                    const uint64_t dbh = sdesc_sw64(sb + boff), dbl = sdesc_sw64(sb + bpart + boff);
                    const uint32_t dt = tmem_base + (uint32_t)(h * n0);
                    const uint32_t idd = h ? id1 : id0;
                    tc_mma<kMode == M_TF32>(dt, dah, dbh, idd, first);
                    tc_mma<kMode == M_TF32>(dt, dah, dbl, idd, 1u);
                    tc_mma<kMode == M_TF32>(dt, dal, dbh, idd, 1u);
                  }
                }
              }
              tc_commit(&empty[stage]);  // frees the stage when these MMAs retire
            }
            if (ok) tc_commit(tmem_full);  // this chunk's accumulators complete
          }
        }
      }
    }
    __syncwarp();
}

template <int kMode>
__device__ void loader_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs) {
  CUROB_ROLE_PROLOGUE
  (void)row0;
    // ------------------------------------------------------------- B loads
    if (lane == 0) {
      uint32_t& it = rs.it;
      bool ok = true;
      for (int ci = 0; ci < F.ncomp && ok && !*abort_flag; ++ci) {
        const Component Cm = tb.comp[F.comp0 + ci];
        for (int si = 0; si < Cm.nseg && ok; ++si) {
          const Segment sg = tb.seg[Cm.seg0 + si];
          const int nslab = sg.npad / kKs;
          const int nchunk = kMode == M_EXACT ? exact_nchunk(sg.npad) : 1;
          const int nw = kMode == M_EXACT ? exact_nw(sg.npad) : sg.npad;
          const long long fl = image_floats(sg.npad);
          const uint8_t* base = a.img + ((size_t)sg.img_off + (size_t)kMode * fl) * 4;
          for (int cc = 0; cc < nchunk && ok; ++cc) {
            const int nc = kMode == M_EXACT ? min(nw, sg.npad - cc * nw) : sg.npad;
            const uint32_t bytes = (uint32_t)(kParts * nc * kRowBytes);
            const uint8_t* src = base + (size_t)cc * nslab * kParts * nw * kRowBytes;
            for (int t = 0; t < nslab; ++t, ++it) {
              const int stage = it % a.nstage;
              const uint32_t ph = (it / a.nstage) & 1u;
              if (!mbar_wait(&empty[stage], ph ^ 1u, abort_flag, tb.status)) {
                ok = false;
                break;
              }
              uint8_t* dst = stages + (size_t)stage * a.stage_bytes + kParts * kPartBytes;
              mbar_arrive_expect_tx(&full[stage], bytes);
              bulk_g2s(dst, src + (size_t)t * bytes, bytes, &full[stage]);
            }
          }
        }
      }
    }
    __syncwarp();
}

template <int kMode>
__device__ inline void run_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs) {
  const int warp = threadIdx.x >> 5;
  if (warp < 4) producer_tile<kMode>(a, m, row0, rs);
  else if (warp < 8) epilogue_tile<kMode>(a, m, row0, rs);
  else if (warp == 8) mma_tile<kMode>(a, m, row0, rs);
  else loader_tile<kMode>(a, m, row0, rs);
  // every issued MMA has been consumed by the epilogue (or the CTA aborted)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  write_outputs(a, m, row0);
}

// One launch per function: CTA b evaluates candidates [128 b, 128 b + 128).
template <int kMode>
__global__ void __launch_bounds__(kThreads, 1) mma_eval_kernel(MmaArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const Smem m = smem_map(smem_raw, args.nstage, args.stage_bytes);
  cta_setup(m, args.nstage);
  RoleState rs;
  run_tile<kMode>(args, m, (long long)blockIdx.x * kTileM, rs);
  cta_teardown(m);
}

// Persistent launch over a ragged batch: each CTA takes work items (an
// instance and one of its 128-candidate tiles) from a global counter until
// none is left; barrier phases carry over from item to item.  The counter
// must be 0 at launch.
template <int kMode>
__global__ void __launch_bounds__(kThreads, 1)
mma_batch_kernel(const MmaArgs* __restrict__ insts, const int2* __restrict__ work, int nwork,
                 int* counter, int nstage, int stage_bytes) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const Smem m = smem_map(smem_raw, nstage, stage_bytes);
  cta_setup(m, nstage);
  RoleState rs;
  for (;;) {
    if (threadIdx.x == 0) *m.item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = *m.item;
    if (w >= nwork || *m.abort_flag) break;
    const int2 W = work[w];
    run_tile<kMode>(insts[W.x], m, (long long)W.y * kTileM, rs);
    __syncthreads();  // outputs written; per-row tables free for the next item
  }
  cta_teardown(m);
}

// ----------------------------------------------------- operand image builder
// For one block (rotated or identity) writes its three images:
//   TF32/BF16: per K stage t, the hi part (npad rows x 64 B, swizzled) then
//              the lo part; hi = round(R), lo = round(R - hi) from FP64.
//   EXACT:     per N chunk of 128 rows, per K stage of 32 columns, the four
//              integer slices of R_i / tau_i (tau_i = 2^f > max_j |R_ij|),
//              nc rows x 64 B each; tau_i goes to the tau pool.
// Entries beyond n are zero.
struct ImgJob {
  long long r_off;     // FP64 block (or -1 for identity)
  long long img_off;   // destination, in floats (4-byte units)
  long long tau_off;
  int n, npad;
};

__device__ inline double r_entry(const ImgJob& J, const double* R, int row, int col) {
  if (row >= J.n || col >= J.n) return 0.0;
  return (J.r_off >= 0) ? R[J.r_off + (long long)row * J.n + col] : (row == col ? 1.0 : 0.0);
}

__global__ void build_image_kernel(const ImgJob* jobs, const double* R, uint8_t* img,
                                   float* tau) {
  const ImgJob J = jobs[blockIdx.x];
  const long long fl = image_floats(J.npad);
  uint8_t* base = img + (size_t)J.img_off * 4;
  const int npad = J.npad;
  for (int row = threadIdx.x; row < npad; row += blockDim.x) {
    double mx = 0.0;
    for (int c = 0; c < J.n; ++c) mx = fmax(mx, fabs(r_entry(J, R, row, c)));
    int e = 0;
    if (mx > 0.0) e = ilogb(mx * 1.0009765625) + 1;
    tau[J.tau_off + row] = ldexpf(1.f, e);
  }
  __syncthreads();
  const int nslab32 = npad / 32;
  const long long total = (long long)npad * npad;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int row = (int)(e / npad), col = (int)(e - (long long)row * npad);
    const double v = r_entry(J, R, row, col);
    {  // TF32: stage t = col / 16
      const int t = col / 16, k = col % 16;
      uint8_t* hi = base + (size_t)t * (2 * npad * kRowBytes);
      uint8_t* lo = hi + npad * kRowBytes;
      const uint32_t off = swz64((uint32_t)row, (uint32_t)(k * 4));
      const uint32_t h = to_tf32((float)v);
      const uint32_t l = to_tf32((float)(v - (double)__uint_as_float(h)));
      *reinterpret_cast<uint32_t*>(hi + off) = h;
      *reinterpret_cast<uint32_t*>(lo + off) = l;
    }
    {  // BF16: stage t = col / 32
      const int t = col / 32, k = col % 32;
      uint8_t* hi = base + (size_t)fl * 4 + (size_t)t * (2 * npad * kRowBytes);
      uint8_t* lo = hi + npad * kRowBytes;
      const uint32_t off = swz64((uint32_t)row, (uint32_t)(k * 2));
      const __nv_bfloat16 h = __double2bfloat16(v);
      const __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
      *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
      *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
    }
    {  // EXACT: chunk cc = row / nw, stage t = col / 32, four pre-scaled slices
      const int nw = exact_nw(npad);
      const int cc = row / nw, rr = row % nw;
      const int nc = min(nw, npad - cc * nw);
      const int t = col / 32, k = col % 32;
      uint8_t* st = base + (size_t)2 * fl * 4 +
                    ((size_t)cc * nslab32 * 4 * nw + (size_t)t * 4 * nc) * kRowBytes;
      const uint32_t off = swz64((uint32_t)rr, (uint32_t)(k * 2));
      double w = v / (double)tau[J.tau_off + row] * 128.0;  // exact: tau is 2^f
      double scale = 1.0;
      for (int s = 0; s < 4; ++s) {
        const double yv = rint(w);
        *reinterpret_cast<__nv_bfloat16*>(st + (size_t)s * nc * kRowBytes + off) =
            __double2bfloat16(yv * scale);
        w = (w - yv) * 256.0;
        scale *= 0.00390625;
      }
    }
  }
}

__global__ void split_o_kernel(const double* operm, const double* o_nat, float* ohi, float* olo,
                               float* onat, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double o = operm[i];
    const float h = (float)o;
    ohi[i] = h;
    olo[i] = (float)(o - (double)h);
    onat[i] = (float)o_nat[i];
  }
}

int npad_of(int n) { return (n + 31) / 32 * 32; }

template <int kMode>
size_t stage_bytes_for(int ncmax) {
  return (size_t)MC<kMode>::kParts * kPartBytes + (size_t)MC<kMode>::kParts * ncmax * kRowBytes;
}
size_t ctrl_bytes() {  // barriers and work item (<= 256 B) + per-row tables + block table
  return 256 + 2 * sizeof(double) * kMaxComponents * kTileM + sizeof(float) * kSigRing * kTileM +
         3 * sizeof(float) * kMaxNpad;
}

template <int kMode>
cudaError_t launch_mode(const MmaPlan& p, const Tables& tb, const Function& F, const float* x,
                        int N, float* out, cudaStream_t st) {
  const int npad_max = npad_of(F.max_n);
  const int ncmax = kMode == M_EXACT ? std::min(npad_max, kExactMaxNC) : npad_max;
  const size_t sb = stage_bytes_for<kMode>(ncmax);
  const size_t ctrl = ctrl_bytes();
  const int nstage = (int)std::min<size_t>(4, (219 * 1024 - ctrl) / sb);
  if (nstage < 2) return cudaErrorInvalidValue;
  const size_t smem = nstage * sb + ctrl + 1024;  // + alignment slack
  MmaArgs a;
  a.tb = tb;
  a.F = F;
  a.x = x;
  a.out = out;
  a.N = N;
  a.ohi = p.ohi;
  a.olo = p.olo;
  a.img = reinterpret_cast<const uint8_t*>(p.img);
  a.tau = p.tau;
  a.onat = p.onat;
  a.nstage = nstage;
  a.stage_bytes = (int)sb;
  cudaError_t e = cudaFuncSetAttribute(mma_eval_kernel<kMode>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mma_eval_kernel<kMode><<<(unsigned)((N + kTileM - 1) / kTileM), kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------- host side
curob_status mma_prepare(MmaPlan& p, std::vector<Segment>& segs, const Tables& tb, float* prev) {
  (void)prev;
  mma_release(p);
  int dev = 0, cc_major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
  p.ready = false;
  // per block: [TF32 | BF16 | EXACT] images and npad tau entries
  long long off = 0, toff = 0;
  for (Segment& s : segs) {
    s.npad = npad_of(s.n);
    if (s.npad > kMaxNpad) {
      s.img_off = -1;
      s.tau_off = 0;
      continue;
    }
    s.img_off = off;
    off += 3 * image_floats(s.npad);
    s.tau_off = toff;
    toff += s.npad;
  }
  p.img_floats = off;
  if (off > 0 && cudaMalloc(&p.img, sizeof(float) * (size_t)off) != cudaSuccess) {
    cudaGetLastError();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  if (cudaMalloc(&p.tau, sizeof(float) * (size_t)std::max<long long>(toff, 1)) != cudaSuccess) {
    cudaGetLastError();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  int max_comp = 0;
  for (const Segment& s : segs) max_comp = std::max(max_comp, s.comp + 1);
  p.o_entries = (long long)max_comp * tb.D;
  const size_t ob = sizeof(float) * (size_t)std::max<long long>(p.o_entries, 1);
  if (cudaMalloc(&p.ohi, ob) != cudaSuccess || cudaMalloc(&p.olo, ob) != cudaSuccess ||
      cudaMalloc(&p.onat, ob) != cudaSuccess) {
    cudaGetLastError();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  std::vector<int> all(segs.size());
  for (size_t i = 0; i < segs.size(); ++i) all[i] = (int)i;
  curob_status rc = mma_refresh(p, segs, all, tb);
  if (rc != CUROB_OK) return rc;
  p.sm103 = (cc_major == 10);
  p.ready = p.sm103;
  return CUROB_OK;
}

curob_status mma_refresh(MmaPlan& p, const std::vector<Segment>& segs, const std::vector<int>& ids,
                         const Tables& tb) {
  std::vector<ImgJob> jobs;
  for (int id : ids) {
    const Segment& s = segs[id];
    if (s.img_off < 0) continue;
    ImgJob J;
    J.r_off = s.identity ? -1 : s.r_off;
    J.n = s.n;
    J.npad = s.npad;
    J.img_off = s.img_off;
    J.tau_off = s.tau_off;
    jobs.push_back(J);
  }
  if (!jobs.empty()) {
    ImgJob* d = nullptr;
    const size_t bytes = sizeof(ImgJob) * jobs.size();
    if (cudaMalloc(&d, bytes) != cudaSuccess) return CUROB_ERR_OUT_OF_MEMORY;
    cudaError_t e = cudaMemcpy(d, jobs.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      build_image_kernel<<<(unsigned)jobs.size(), 256>>>(d, tb.R, (uint8_t*)p.img, p.tau);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d);
    if (e != cudaSuccess) return CUROB_ERR_CUDA;
  }
  if (p.o_entries > 0) {
    split_o_kernel<<<256, 256>>>(tb.operm, tb.o, p.ohi, p.olo, p.onat, p.o_entries);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      return CUROB_ERR_CUDA;
  }
  return CUROB_OK;
}

void mma_release(MmaPlan& p) {
  cudaFree(p.img);
  cudaFree(p.ohi);
  cudaFree(p.olo);
  cudaFree(p.tau);
  cudaFree(p.onat);
  p.img = nullptr;
  p.ohi = p.olo = p.tau = p.onat = nullptr;
  p.img_floats = 0;
  p.o_entries = 0;
  p.ready = false;
}

bool mma_supports(const MmaPlan& p, const Function& F) {
  return p.ready && F.max_n >= 16 && F.max_n <= kMaxNpad;
}

int mma_auto_mode(const MmaPlan& p, const Function& F) {
  (void)p;
  return F.sensitive ? CUROB_PRECISION_EXACT : CUROB_PRECISION_TF32X3;
}

namespace {
// Stage geometry of the EXACT persistent kernel (independent of the item).
struct BatchGeom {
  int nstage, stage_bytes;
  size_t smem;
};
BatchGeom batch_geom() {
  BatchGeom g;
  const size_t sb = stage_bytes_for<M_EXACT>(kExactMaxNC);
  g.stage_bytes = (int)sb;
  g.nstage = (int)std::min<size_t>(4, (219 * 1024 - ctrl_bytes()) / sb);
  g.smem = g.nstage * sb + ctrl_bytes() + 1024;
  return g;
}
}  // namespace

size_t mma_args_bytes() { return sizeof(MmaArgs); }

void mma_fill_args(void* dst, const MmaPlan& p, const Tables& tb, const Function& F,
                   const float* x, float* out, int N) {
  const BatchGeom g = batch_geom();
  MmaArgs a;
  a.tb = tb;
  a.F = F;
  a.x = x;
  a.out = out;
  a.N = N;
  a.ohi = p.ohi;
  a.olo = p.olo;
  a.img = reinterpret_cast<const uint8_t*>(p.img);
  a.tau = p.tau;
  a.onat = p.onat;
  a.nstage = g.nstage;
  a.stage_bytes = g.stage_bytes;
  memcpy(dst, &a, sizeof(a));
}

cudaError_t launch_mma_batch(const void* d_args, const int2* d_work, int nwork, int* d_counter,
                             int grid, cudaStream_t st) {
  const BatchGeom g = batch_geom();
  cudaError_t e = cudaFuncSetAttribute(mma_batch_kernel<M_EXACT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
  if (e != cudaSuccess) return e;
  mma_batch_kernel<M_EXACT><<<grid, kThreads, g.smem, st>>>(
      reinterpret_cast<const MmaArgs*>(d_args), d_work, nwork, d_counter, g.nstage,
      g.stage_bytes);
  return cudaGetLastError();
}

int mma_max_block() { return kMaxNpad; }

cudaError_t launch_mma(const MmaPlan& p, const Tables& tb, const Function& F, int mode,
                       const float* x, int N, float* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  switch (mode) {
    case CUROB_PRECISION_TF32X3: return launch_mode<M_TF32>(p, tb, F, x, N, out, st);
    case CUROB_PRECISION_BF16X3: return launch_mode<M_BF16>(p, tb, F, x, N, out, st);
    case CUROB_PRECISION_EXACT: return launch_mode<M_EXACT>(p, tb, F, x, N, out, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace curob

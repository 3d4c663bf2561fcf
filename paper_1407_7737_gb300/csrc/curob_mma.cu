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
//   warps 0-7  producers: warp w takes rows 32 (w % 4) .. + 31 (thread =
//              candidate row) and half w / 4 of every K stage's columns.  Per
//              block the block's index list and o hi/lo words are staged in
//              shared memory; per stage a thread gathers its row's x at the
//              block's variables (cp.async, issued stages ahead), takes
//              y = x - o in double-float (exact TwoSum, then o's low word),
//              splits or slices it and stores its rows of the A operand in the
//              swizzled K-major layout; it also sums ||x - o||^2.
//   warps 8-11 epilogue: thread t owns row t (TMEM lane t), loads its z 32
//              columns at a time (tcgen05.ld), applies z = s z + c, the
//              per-variable transform and the running sums (FP32 per 32
//              columns, FP64 across), closes functions.  Blocks of a heavy
//              kind (kind_is_heavy) instead leave z in a variable-major
//              scratch, and finish_kernel, a second launch with 8 warps per
//              16 candidates, evaluates their terms: four epilogue warps per
//              SM cannot hide the latency of long transcendental series.
//   warp 12    allocates TMEM and issues the MMAs (one lane).
//   warp 13    loads the B operand (R_b parts, pre-laid-out in global memory
//              as the exact shared-memory image) with one bulk copy per stage
//              (cp.async.bulk, the TMA engine).
// Stages rotate through shared memory under full/empty mbarriers; the
// accumulators are handed from the MMA warp to the epilogue and back under
// tmem_full/tmem_empty, alternating between the low and the high end of
// TMEM: the epilogue drains the columns the next accumulator will overwrite,
// hands TMEM back, and drains the rest while the next block's MMAs run
// (MmaArgs::acc_hi / acc_ovl).  Every wait is bounded: past ~2 s it raises
// DEV_TIMEOUT in the status word, the CTA stops, and TMEM is freed before
// exit.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "curob_mma.hpp"
#include "curob_tc.cuh"
#include "curob_tmap.hpp"

namespace curob {
namespace {

using namespace tc;

constexpr int kTileM = 128;
// Scratch of one slice of candidates: G_c and ||x - o_c||^2 (FP64) and the
// heavy-kind z (FP32) of every row; slices keep it under this many bytes.
constexpr size_t kScratchCap = size_t(256) << 20;

constexpr int kThreads = 448;  // 8 producer, 4 epilogue, MMA and loader warps
constexpr int kThreadsXT = 480;  // the same and the raw-gather warp (x^T launches)
constexpr int kMmaWarp = 12, kLoaderWarp = 13, kRawWarp = 14;
constexpr int kMaxNpad = 512;                    // TMEM columns
constexpr int kExactMaxNC = 192;                 // EXACT: widest N chunk
constexpr int kMaxStages = 6;                    // K stages in flight
constexpr int kMaxARing = 8;                     // A slots of the transposed-input rings
constexpr int kCtrlHeader = 512;                 // barrier header of the control block
constexpr size_t kSmemCap = 227 * 1024 - 1024;   // dynamic shared memory, less alignment slack
constexpr int kExactAcc1 = 256;                  // EXACT: TMEM column of accumulator 1
constexpr int kSigRing = 8;                      // EXACT: row scales in flight
constexpr size_t kTabTBytes = 2 * kMaxNpad * sizeof(float);  // epilogue's tau buffers

enum Mode : int { M_TF32 = 0, M_BF16 = 1, M_EXACT = 2, M_F16 = 3 };
// Modes whose operands are scaled per row: y by sigma_m (a power of two above
// the candidate's max_j |x_j - o_j| over the component), R by tau_i.
__host__ __device__ constexpr bool scaled_mode(int m) { return m == M_EXACT || m == M_F16; }

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
// TF32X3 and BF16X3 stage 64-byte rows (64-byte swizzle); EXACT stages
// 32-byte rows (32-byte swizzle, 16 K columns, one MMA K step per stage), so
// that its four operand parts still leave room for five stages.
template <int kMode> struct MC {
  static constexpr int kParts = kMode == M_EXACT ? 4 : 2;  // A/B operand parts
  static constexpr int kKs = (kMode == M_BF16 || kMode == M_F16) ? 32 : 16;  // K per stage
  static constexpr int kEl = kMode == M_TF32 ? 4 : 2;      // bytes per element
  static constexpr int kMmaK = kMode == M_TF32 ? 8 : 16;   // K per MMA
  static constexpr uint32_t kFmt = kMode == M_TF32 ? 2u : (kMode == M_F16 ? 0u : 1u);
  static constexpr int kRow = kMode == M_EXACT ? 32 : 64;  // bytes of a part's row
  static constexpr int kPart = kTileM * kRow;              // bytes of an A part
};
template <int kMode>
__host__ __device__ __forceinline__ uint32_t swz_m(uint32_t row, uint32_t byte_in_row) {
  return kMode == M_EXACT ? swz32(row, byte_in_row) : swz64(row, byte_in_row);
}
template <int kMode>
__device__ __forceinline__ uint64_t sdesc_m(uint32_t saddr) {
  return kMode == M_EXACT ? sdesc_sw32(saddr) : sdesc_sw64(saddr);
}

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
  // Operand rings.  Batched launches read x with gathers into the A area of
  // each stage (A and B of a stage side by side: nA = nB = nstage).  Launches
  // on the transposed copy of x (xt = 1) keep separate rings: nA A slots of
  // a_bytes (the raw gather lands in the slot it is converted in) and nB B
  // slots of b_bytes.
  int xt;
  int nA, a_bytes, nB, b_bytes;
  int nlist;                   // components evaluated, in order (all of F's, or a subset)
  int list[kMaxComponents];
  double* gout;                // split launches: G_c and ||x - o_c||^2 per component and row
  double* d2out;               // ([kMaxComponents][N] each), closed by finish_kernel
  float* zbuf;                 // heavy-kind z, variable-major ([F.hcols][N]); nullptr: the
                               // epilogue evaluates heavy kinds itself
  // Accumulator regions: hand-offs alternate between TMEM columns [0, W) and
  // [acc_hi, acc_hi + W) (acc_hi = T - W, T = 512, or 256 per EXACT
  // accumulator; W a multiple of 32 >= every hand-off's width), so the two
  // overlap in acc_ovl = 2 W - T columns (<= 0: none) and only those must be
  // drained before the next hand-off may start.
  int acc_hi;
  int acc_ovl;
  // Scaled modes: 1 when the launch reserved kTabTBytes past the control
  // block, where the epilogue stages each block's tau (else it reads them
  // from global memory).
  int tabt;
  // Scaled modes: per component, the row maxima max_j |x_j - o_j| in
  // partial form ([ntx][pm_ld] floats each: one partial per 64 variables,
  // written by the transpose of x); nullptr: the producers form them.
  const float* rowpm;
  int ntx, pm_ld;
};

// The allocation-free entry point keeps up to 64 argument blocks in 32 KB.
static_assert(sizeof(MmaArgs) <= 512, "MmaArgs outgrew the allocation-free argument area");

// Floats reserved per block for each precision's image (the TF32 size; BF16
// and FP16 need half).  A block's images: [TF32][BF16][EXACT][FP16].
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

// Heavy kinds (kind_is_heavy) evaluated in the epilogue (persistent batch
// kernel, or no z scratch): their terms are out-of-line calls on four
// variables at a time, so the unrolled chunk loop stays small while the four
// independent evaluations interleave (one epilogue warp per scheduler has no
// other warp to hide their latency); contributions come back by value (no
// local memory).
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
  } else if constexpr (KIND == K_RASTRIGIN || KIND == K_ACKLEY || KIND == K_LUNACEK) {
    // The 32 cosines first (independent of one another), then the sums in
    // column order, as elem_term_f32 forms them: with one epilogue warp per
    // scheduler nothing else hides the SFU latency of a column-by-column chain.
    float cz[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float u = v[k] * es.s;
      cz[k] = cos2pi_sfu(KIND == K_LUNACEK ? u : u + es.c0);
    }
    float zprev = st.zprev;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k < cend) {
        const int col = c + k;
        const float u = v[k] * es.s;
        const float z = u + es.c0;
        if constexpr (KIND == K_RASTRIGIN) {
          part.a0 += fmaf(z, z, 10.0f - 10.0f * cz[k]);
        } else if constexpr (KIND == K_ACKLEY) {
          part.a0 = fmaf(z, z, part.a0);
          part.a1 += cz[k];
        } else {
          const float w = u + 5.0f;
          part.a0 = fmaf(u, u, part.a0);
          part.a1 = fmaf(w, w, part.a1);
          part.a2 += cz[k];
        }
        if (col == 0 && es.gfirst) st.zfirst = z;
        zprev = z;
      }
    }
    st.zprev = zprev;
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
  st.a0 += (double)part.a0;  // FP64 operations only for the fields the kind uses
  if constexpr (kind_uses_a1(KIND)) st.a1 += (double)part.a1;
  if constexpr (kind_uses_a2(KIND)) st.a2 += (double)part.a2;
  if constexpr (kind_uses_p(KIND)) st.p *= (double)part.p;
}

// kHeavy: the build that evaluates heavy kinds in the epilogue (no z
// scratch); without it those kinds always go to the scratch, and their code,
// with the registers it needs, stays out of the kernel.
template <bool kHeavy>
__device__ __forceinline__ void epi_chunk(int kind, const float* v, int c, int cend,
                                          const EpiSeg& es, EpiState& st) {
  switch (kind) {
#define CUROB_EPI_CASE(K) \
  case K: epi_chunk_k<K>(v, c, cend, es, st); break;
#define CUROB_EPI_HEAVY(K) \
  case K: if constexpr (kHeavy) epi_chunk_k<K>(v, c, cend, es, st); break;
    CUROB_EPI_CASE(K_SPHERE) CUROB_EPI_CASE(K_ELLIPSOID) CUROB_EPI_CASE(K_ELLIPTIC)
    CUROB_EPI_CASE(K_DISCUS) CUROB_EPI_CASE(K_CIGAR) CUROB_EPI_HEAVY(K_POWERS)
    CUROB_EPI_CASE(K_SHARPV) CUROB_EPI_CASE(K_STEP) CUROB_EPI_HEAVY(K_WEIERSTRASS)
    CUROB_EPI_HEAVY(K_GRIEWANK) CUROB_EPI_CASE(K_RASTRIGIN) CUROB_EPI_HEAVY(K_SCHAFFER7)
    CUROB_EPI_HEAVY(K_EGR) CUROB_EPI_CASE(K_ROSENBROCK) CUROB_EPI_HEAVY(K_SCHWEFEL)
    CUROB_EPI_HEAVY(K_KATSUURA) CUROB_EPI_CASE(K_LUNACEK) CUROB_EPI_CASE(K_ACKLEY)
    CUROB_EPI_CASE(K_HAPPYCAT) CUROB_EPI_CASE(K_HGBAT) CUROB_EPI_HEAVY(K_SCHAFFER6)
#undef CUROB_EPI_HEAVY
#undef CUROB_EPI_CASE
    default: break;
  }
}

// -------------------------------------------------------------- the kernel
// Shared-memory map of a CTA (identical for the per-launch and the
// persistent kernels).
struct Smem {
  uint8_t* stages;
  uint8_t *a_base, *b_base;  // A slot s at a_base + s a_stride, B slot at b_base + s b_stride
  int a_stride, b_stride, nA, nB;
  uint64_t *fullB, *emptyB, *rawfull;  // B ring (aliases full/empty unless xt), raw gathers;
                                       // a stage's B copy completes on full[] of its A slot
  uint64_t *full, *empty, *tmem_full, *tmem_empty, *sig_full, *prod_bar, *gbar;
  uint32_t* tmem_slot;
  volatile int* abort_flag;
  double *rowG, *rowD2;
  float* rowSig;
  float* rowMx;  // EXACT: max_j |x_j - o_j| of each row
  int* tabS;
  float *tabH, *tabL;
  float* tabT;         // scaled modes: the epilogue's row scales tau of R, two blocks
                       // (past the control block; MmaArgs::tabt says it exists)
  uint64_t* epi_bar;   // the 4 epilogue warps
  int* item;  // persistent kernel: the work item of the CTA
};

// Ring geometry of a launch: xt = 0 (nstage stages of stage_bytes, A of
// a_bytes first in each) or xt = 1 (separate A and B rings).
struct RingGeom {
  int xt, nstage, stage_bytes, nA, a_bytes, nB, b_bytes;
};

__device__ inline Smem smem_map(uint8_t* smem_raw, const RingGeom& g) {
  Smem m;
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  m.stages = smem;
  uint8_t* ctrl;
  if (g.xt) {
    m.nA = g.nA;
    m.nB = g.nB;
    m.a_base = smem;
    m.a_stride = g.a_bytes;
    m.b_base = smem + (size_t)g.nA * g.a_bytes;
    m.b_stride = g.b_bytes;
    ctrl = m.b_base + (size_t)g.nB * g.b_bytes;
  } else {
    m.nA = m.nB = g.nstage;
    m.a_base = smem;
    m.b_base = smem + g.a_bytes;
    m.a_stride = m.b_stride = g.stage_bytes;
    ctrl = smem + (size_t)g.nstage * g.stage_bytes;
  }
  const int nA = m.nA, nB = m.nB;
  m.full = reinterpret_cast<uint64_t*>(ctrl);
  m.empty = m.full + nA;
  m.tmem_full = m.empty + nA;
  m.tmem_empty = m.tmem_full + 1;
  m.sig_full = m.tmem_empty + 1;  // [kSigRing]
  m.prod_bar = m.sig_full + kSigRing;
  m.gbar = m.prod_bar + 1;        // [nA]
  uint64_t* next = m.gbar + nA;
  if (g.xt) {
    m.fullB = next;               // [nB]
    m.emptyB = m.fullB + nB;      // [nB]
    m.rawfull = m.emptyB + nB;    // [nA]
    next = m.rawfull + nA;
  } else {
    m.fullB = m.full;
    m.emptyB = m.empty;
    m.rawfull = nullptr;
  }
  m.epi_bar = next++;
  m.tmem_slot = reinterpret_cast<uint32_t*>(next);
  m.abort_flag = reinterpret_cast<volatile int*>(m.tmem_slot + 1);
  m.item = const_cast<int*>(reinterpret_cast<volatile int*>(m.abort_flag) + 1);
  m.rowG = reinterpret_cast<double*>(ctrl + kCtrlHeader);         // [kMaxComponents][128]
  m.rowD2 = m.rowG + kMaxComponents * kTileM;                     // [2][kMaxComponents][128]
  m.rowSig = reinterpret_cast<float*>(m.rowD2 + 2 * kMaxComponents * kTileM);  // [kSigRing][128]
  m.rowMx = m.rowSig + kSigRing * kTileM;                         // [128]
  m.tabS = reinterpret_cast<int*>(m.rowMx + kTileM);              // [kMaxNpad]
  m.tabH = reinterpret_cast<float*>(m.tabS + kMaxNpad);
  m.tabL = m.tabH + kMaxNpad;
  m.tabT = m.tabL + kMaxNpad;   // [2][kMaxNpad], only where the launch reserved it (MmaArgs::tabt)
  return m;
}

// Barrier-phase counters of one role, carried from tile to tile.
struct RoleState {
  uint32_t it = 0;        // K stages
  uint32_t chunk_it = 0;  // accumulator hand-offs
  uint32_t pphase = 0;    // producer group barrier uses
  uint32_t comp_it = 0;   // components (row-scale ring)
  uint32_t b_par = 0;     // B loads: bit s = parity of the last load completing on A slot
                          // s's full barrier, bit 8 + s = used
  uint32_t r_par = 0;     // raw gathers (xt), the same bookkeeping per A slot
  uint32_t e_blk = 0;     // epilogue: blocks staged (tabT buffer parity)
  uint32_t e_phase = 0;   // epilogue group barrier uses
};

__device__ inline void cta_setup(const Smem& m, int xt) {
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < m.nA; ++s) {
      mbar_init(&m.full[s], 9);  // 8 producer warps + the B loader's expect_tx
      mbar_init(&m.empty[s], 1);          // one tcgen05.commit
      mbar_init(&m.gbar[s], 256);         // producer threads' cp.async
      if (xt) mbar_init(&m.rawfull[s], 1);  // the raw gathers' expect_tx
    }
    if (xt)
      for (int s = 0; s < m.nB; ++s) mbar_init(&m.emptyB[s], 1);  // one tcgen05.commit
    mbar_init(m.tmem_full, 1);
    mbar_init(m.tmem_empty, 4);   // the 4 epilogue warps
    for (int s = 0; s < kSigRing; ++s) mbar_init(&m.sig_full[s], 4);  // producer warps 0-3
    mbar_init(m.prod_bar, 8);     // the 8 producer warps
    mbar_init(m.epi_bar, 4);      // the 4 epilogue warps
    *m.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
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
  if (warp < 8 || warp >= 12 || *m.abort_flag) return;
  const int r = (warp - 8) * 32 + lane;
  const long long grow = row0 + r;
  if (grow >= a.N) return;
  const Function& F = a.F;
  if (a.gout) {  // split launch: the components' values for finish_kernel
    for (int li = 0; li < a.nlist; ++li) {
      const int ci = a.list[li];
      a.gout[(size_t)ci * a.N + grow] = m.rowG[ci * kTileM + r];
      a.d2out[(size_t)ci * a.N + grow] =
          m.rowD2[ci * kTileM + r] + m.rowD2[(kMaxComponents + ci) * kTileM + r];
    }
    return;
  }
  double f;
  if (F.composition) {
    double G[kMaxComponents], d2v[kMaxComponents];
    for (int ci = 0; ci < F.ncomp; ++ci) {
      G[ci] = m.rowG[ci * kTileM + r];
      d2v[ci] = m.rowD2[ci * kTileM + r] + m.rowD2[(kMaxComponents + ci) * kTileM + r];
    }
    f = compose(a.tb.comp + F.comp0, F.ncomp, G, d2v, a.tb.D);
  } else {
    f = m.rowG[r];
  }
  a.out[grow] = (float)(f + kFopt);
}

__device__ inline void cta_teardown(const Smem& m) {
  const int warp = threadIdx.x >> 5;
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*m.tmem_slot),
                 "r"(kMaxNpad));
  }
}

#define CUROB_ROLE_PROLOGUE                                                   \
  using C = MC<kMode>;                                                        \
  constexpr int kKs = C::kKs, kEl = C::kEl, kParts = C::kParts;               \
  constexpr int kKsteps = kKs / C::kMmaK;                                     \
  constexpr int kRow = C::kRow, kPart = C::kPart;                             \
  (void)kEl; (void)kParts; (void)kKsteps; (void)kRow; (void)kPart;            \
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

// kXT: x comes from its transposed copy by TMA gathers (see MmaArgs::xt);
// each producer warp then owns rows 16 w .. 16 w + 15, two lanes per row.
template <int kMode, bool kXT>
__device__ void producer_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs,
                              const CUtensorMap* xmap) {
  CUROB_ROLE_PROLOGUE
    // ------------------------------------------------------------ producers
    // Eight warps: warp w takes rows 32 (w % 4) .. + 31 (thread = candidate
    // row r) and half h = w / 4 of every stage's K columns, so two warps
    // share each row.  The raw x of a stage is gathered with 4-byte cp.async
    // straight into the A area, each half's values into the very 16-byte
    // chunks that half will overwrite with its converted operands: a thread
    // reads only its own raw values back, and no other thread touches them.
    const int h = warp >> 2;                 // half of the stage's columns
    const int r = (warp & 3) * 32 + lane;    // candidate row in the tile
    (void)xmap;
    constexpr int kHalf = kKs / 2;           // columns per half
    constexpr int kCpp = kRow / 32;          // 16-byte chunks per part row per half
    const long long grow = row0 + r;
    const bool vrow = grow < a.N;
    const float* xrow = a.x + (vrow ? grow : 0) * (long long)D;
    // Gather prefetch depth: the gather of stage q + P goes into the A area
    // of stage q + P - nstage, whose MMAs retired (nstage >= 3: P = nstage -
    // 2, issued before stage q is converted, so it never waits on the MMAs
    // of the stage just handed over).
    const bool early = a.nstage >= 3;
    const int P = early ? a.nstage - 2 : 1;
    uint32_t& it = rs.it;
    uint32_t& pphase = rs.pphase;
    bool ok = true;
    if (!kXT && vrow && h == 0) {  // bring the row into L2 now: the gathers then wait on L2
      const uintptr_t s0 = (reinterpret_cast<uintptr_t>(xrow) + 15) & ~uintptr_t(15);
      const uintptr_t s1 = reinterpret_cast<uintptr_t>(xrow + D) & ~uintptr_t(15);
      if (s1 > s0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s0), "r"((uint32_t)(s1 - s0))
                     : "memory");
    }
    for (int li = 0; li < a.nlist && ok; ++li, ++rs.comp_it) {
      const int ci = a.list[li];
      const uint32_t cg = rs.comp_it;  // component counter across tiles
      const Component Cm = tb.comp[F.comp0 + ci];
      const int* S = tb.S + Cm.base;
      const float* ohi = a.ohi + Cm.base;
      const float* olo = a.olo + Cm.base;
      double d2 = 0.0;
      // ||x - o||^2 only feeds the composition weights
      const bool need_d2 = F.composition != 0 || a.d2out != nullptr;
      float isig = 1.f;
      if (scaled_mode(kMode) && a.rowpm) {
        // max_j |x_j - o_j| of each row over the component from the
        // transpose's partial maxima (one per 64 variables), read after the
        // next producer barrier
        if (h == 0) {
          float mv = 0.f;
          if (vrow) {
            const float* pp = a.rowpm + (size_t)ci * a.ntx * a.pm_ld + grow;
            for (int t = 0; t < a.ntx; ++t) mv = fmaxf(mv, __ldg(pp + (size_t)t * a.pm_ld));
          }
          m.rowMx[r] = mv;
        }
      } else if constexpr (scaled_mode(kMode)) {
        // max_j |x_j - o_j| of each row over the component, read in natural
        // order: half h of the warp pair reads rows 16 h .. 16 h + 15 of the
        // pair's 32 with coalesced loads (o as FP32); the maxima meet in
        // rowMx and are read after the next producer barrier
        const float* on = a.onat + Cm.base;
        const bool vec = (D & 3) == 0 && (reinterpret_cast<uintptr_t>(a.x) & 15u) == 0;
        const int hm = warp >> 2;
#pragma unroll 2
        for (int rr = 16 * hm; rr < 16 * hm + 16; ++rr) {
          const int row = (warp & 3) * 32 + rr;
          const long long gr = row0 + row;
          float mv = 0.f;
          if (gr < a.N) {  // uniform across the warp
            const float* xr_ = a.x + gr * (long long)D;
            if (vec) {
              const float4* x4 = reinterpret_cast<const float4*>(xr_);
              const float4* o4 = reinterpret_cast<const float4*>(on);
#pragma unroll 4
              for (int k4 = lane; k4 < D / 4; k4 += 32) {
                const float4 u = __ldg(x4 + k4), w = __ldg(o4 + k4);
                mv = fmaxf(mv, fmaxf(fmaxf(fabsf(u.x - w.x), fabsf(u.y - w.y)),
                                     fmaxf(fabsf(u.z - w.z), fabsf(u.w - w.w))));
              }
            } else {
              for (int k = lane; k < D; k += 32) mv = fmaxf(mv, fabsf(__ldg(xr_ + k) - on[k]));
            }
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) mv = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, off));
          if (lane == 0) m.rowMx[row] = mv;
        }
      }
      for (int si = 0; si < Cm.nseg && ok; ++si) {
        const Segment sg = tb.seg[Cm.seg0 + si];
        // stage the block's index list and o words in shared memory (the
        // previous block's readers are done at the first barrier)
        if (!producers_sync(prod_bar, pphase, abort_flag, tb.status)) { ok = false; break; }
        if constexpr (scaled_mode(kMode)) {
          if (si == 0) {  // row scale sigma_m = 2^e > the row's maximum
            const float mx = m.rowMx[r];
            int e = 0;
            if (mx > 0.f && mx < 3.0e38f) e = ilogbf(mx * 1.0009765625f) + 1;
            isig = ldexpf(1.f, -e);
            if (h == 0) {
              rowSig[(cg % kSigRing) * kTileM + r] = ldexpf(1.f, e);
              __syncwarp();
              if (lane == 0) mbar_arrive(&sig_full[cg % kSigRing]);
            }
          }
        }
        for (int k = h * kTileM + r; k < sg.npad; k += 2 * kTileM) {
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
        if constexpr (kXT) {
          const int nvalid = sg.n;
          const int nA = m.nA;
          constexpr int kRawBytes = kKs * kTileM * 4;
          const uint32_t it0 = it;
          // The raw x of a stage (its kKs variables x the tile's 128
          // candidates, variable-major; gathered by the raw-gather warp) lies
          // in the last bytes of the A slot it is converted in; the producers
          // read it all, meet, and only then overwrite it with the operands.
          auto raw_ptr = [&](uint32_t g) -> uint8_t* {
            return m.a_base + (size_t)(g % nA) * m.a_stride + kParts * kPart - kRawBytes;
          };
          (void)it0;
          for (int q = 0; q < total && ok; ++q, ++it) {
            const int stage = it % nA;
            uint8_t* A = m.a_base + (size_t)stage * m.a_stride;
            const int t = q % nslab;
            const bool good = mbar_wait(&m.rawfull[stage], (it / nA) & 1u, abort_flag, tb.status);
            if (!__all_sync(0xffffffffu, good)) {
              ok = false;
              break;
            }
            // this thread's raw x: variables h kHalf + i of the stage at its row
            float xv[kHalf];
            {
              const float* raw = reinterpret_cast<const float*>(raw_ptr(it));
#pragma unroll
              for (int i = 0; i < kHalf; ++i) {
                const int v = h * kHalf + i;
                const float val = raw[v * kTileM + r];
                xv[i] = (t * kKs + v < nvalid) ? val : 0.f;  // a column past the block: x = 0
              }
            }
            // all raw values are read before any producer overwrites them
            if (!__all_sync(0xffffffffu, producers_sync(prod_bar, pphase, abort_flag, tb.status))) {
              ok = false;
              break;
            }
          constexpr int kPer = 16 / kEl;  // elements per 16-byte chunk
          float d2p = 0.f;
          // this half's kCpp chunks of 16 bytes per part row, each stored whole
#pragma unroll
          for (int cc = 0; cc < kCpp; ++cc) {
            const int c = h * kCpp + cc;  // chunk of the row
            float yh[kPer], yl[kPer], oh[kPer], ol[kPer];
            const int jc = t * kKs + h * kHalf + cc * kPer;  // first column of the chunk
#pragma unroll
            for (int q4 = 0; q4 < kPer / 4; ++q4) {  // o words, 16 bytes at a time
              const float4 a4 = *reinterpret_cast<const float4*>(tabH + jc + 4 * q4);
              const float4 b4 = *reinterpret_cast<const float4*>(tabL + jc + 4 * q4);
              oh[4 * q4] = a4.x; oh[4 * q4 + 1] = a4.y; oh[4 * q4 + 2] = a4.z; oh[4 * q4 + 3] = a4.w;
              ol[4 * q4] = b4.x; ol[4 * q4 + 1] = b4.y; ol[4 * q4 + 2] = b4.z; ol[4 * q4 + 3] = b4.w;
            }
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
              // branch-free, so that the chunk's elements interleave.  A
              // column past the block has x = 0 (zero-filled copy) and o = 0
              // (staged), so y = 0; a row past the batch is never written.
              // EXACT slices y to 2^-26 of the row scale: the exact
              // double-float shift.  The split modes keep 22 (16) bits of y:
              // x - o_hi is exact near o (Sterbenz) and one more rounding of
              // the low word of o stays below those bits.
              if constexpr (kMode == M_EXACT) {
                shift_ff(xv[cc * kPer + e], oh[e], ol[e], yh[e], yl[e]);
              } else {
                yh[e] = __fsub_rn(__fsub_rn(xv[cc * kPer + e], oh[e]), ol[e]);
                yl[e] = 0.f;
              }
              if (need_d2) d2p = fmaf(yh[e], yh[e], d2p);
            }
            const uint32_t off = swz_m<kMode>((uint32_t)r, (uint32_t)(c * 16));
            if constexpr (kMode == M_TF32) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const float a = yh[qq];
                hw[qq] = to_tf32(a);
                lw[qq] = to_tf32((a - __uint_as_float(hw[qq])) + yl[qq]);
              }
              *reinterpret_cast<uint4*>(A + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(A + kPart + off) =
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
              *reinterpret_cast<uint4*>(A + kPart + off) =
                  make_uint4(lw[0], lw[1], lw[2], lw[3]);
            } else if constexpr (kMode == M_F16) {
              // y / sigma in (-1, 1) (an exact power-of-two scaling) as FP16
              // hi + lo: 22 significant bits, as TF32 hi + lo
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const float a = yh[2 * qq] * isig, b = yh[2 * qq + 1] * isig;
                const __half2 hh = __floats2half2_rn(a, b);
                const float2 hf = __half22float2(hh);
                const __half2 ll = __floats2half2_rn(fmaf(yl[2 * qq], isig, a - hf.x),
                                                     fmaf(yl[2 * qq + 1], isig, b - hf.y));
                hw[qq] = *reinterpret_cast<const uint32_t*>(&hh);
                lw[qq] = *reinterpret_cast<const uint32_t*>(&ll);
              }
              *reinterpret_cast<uint4*>(A + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(A + kPart + off) =
                  make_uint4(lw[0], lw[1], lw[2], lw[3]);
            } else {
              // four slices of v = 128 y / sigma (exact in BF16), already at
              // their weight: s1 = rint(v), then the remainder r = v - s1
              // (plus y's low word) rounded to multiples of 2^-8, 2^-16 and
              // 2^-24 in turn.  Adding and subtracting 1.5 * 2^(23 - 8a)
              // rounds to a multiple of 2^-8a, ties to even, exactly as rintf
              // of the 2^8a-scaled value does (|v| < 128, |r| <= 2^-1, 2^-9,
              // 2^-17), and every remainder is exact
              const float s128 = isig * 128.f;
              uint32_t w[4][4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                float sl[2][4];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                  const int k = 2 * qq + e;
                  const float v = yh[k] * s128;
                  const float y1 = (v + 12582912.0f) - 12582912.0f;       // 1.5 * 2^23
                  float rr = fmaf(yl[k], s128, v - y1);
                  const float y2 = (rr + 49152.0f) - 49152.0f;            // 1.5 * 2^15
                  rr = rr - y2;
                  const float y3 = (rr + 192.0f) - 192.0f;                // 1.5 * 2^7
                  rr = rr - y3;
                  const float y4 = (rr + 0.75f) - 0.75f;                  // 1.5 * 2^-1
                  sl[e][0] = y1;
                  sl[e][1] = y2;
                  sl[e][2] = y3;
                  sl[e][3] = y4;
                }
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) w[pp][qq] = pack_bf16(sl[0][pp], sl[1][pp]);
              }
#pragma unroll
              for (int pp = 0; pp < 4; ++pp)
                *reinterpret_cast<uint4*>(A + pp * kPart + off) =
                    make_uint4(w[pp][0], w[pp][1], w[pp][2], w[pp][3]);
            }
          }
            if (q < nslab) d2 += (double)d2p;  // first chunk: ||x - o||^2 of the row
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[stage]);
          }
        } else {
        // raw x of stage q: half h's column i goes to 16-byte chunk
        // (h kCpp + (i / 4) % kCpp) of part (i / 4) / kCpp of the row, in the
        // operand's swizzle.  Lanes walk rows' (sorted) columns, so one
        // instruction touches a few rows' few sectors; each thread's copies
        // arrive on gbar[stage] when they land.
        const int nst = a.nstage, sbytes = a.stage_bytes, nvalid = sg.n;
        // Per lane: column i of the half and rows rb + v kRowsPerInst.  Both
        // swizzles repeat every 8 rows, so kPer offsets give every row's
        // destination; source offsets are 32-bit within the tile; vmask has
        // bit v for rows inside the batch.
        constexpr int kRowsPerInst = 32 / kHalf;            // 4 (16-column stages) or 2
        constexpr int kNv = 32 / kRowsPerInst;               // gathers per lane per stage
        constexpr int kPer = 8 / kRowsPerInst;               // swizzle period in v
        const int gi = lane % kHalf;                         // column of the half
        const int rb = (warp & 3) * 32 + lane / kHalf;
        const uint32_t dbyte = (uint32_t)((h * kCpp + (gi / 4) % kCpp) * 16 + (gi % 4) * 4);
        const uint32_t dpo = (uint32_t)(((gi / 4) / kCpp) * kPart);
        uint32_t dsw[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) dsw[u] = dpo + swz_m<kMode>((uint32_t)(rb + u * kRowsPerInst), dbyte);
        const float* xtile = a.x + row0 * (long long)D;
        const int roff = rb * D, rstep = kRowsPerInst * D;
        const long long nleft = a.N - row0;
        uint32_t vmask = 0;
#pragma unroll
        for (int v = 0; v < kNv; ++v)
          if (rb + v * kRowsPerInst < nleft) vmask |= 1u << v;
        auto issue = [=](int q) -> bool {
          const uint32_t g = it0 + (uint32_t)q;
          const int stage = g % nst;
          if (!mbar_wait(&empty[stage], ((g / nst) & 1u) ^ 1u, abort_flag, tb.status))
            return false;
          const uint32_t A = smem_u32(stages + (size_t)stage * sbytes);
          const int t = q % nslab;
          const int j = t * kKs + h * kHalf + gi;
          const uint32_t m = j < nvalid ? vmask : 0u;  // invalid copies fill zeros
          const float* xc = xtile + (j < nvalid ? tabS[j] : 0);
#pragma unroll
          for (int v = 0; v < kNv; ++v) {
            const bool in = (m >> v) & 1u;
            const float* src = in ? xc + (roff + v * rstep) : xtile;
            const uint32_t dst = A + dsw[v % kPer] + (uint32_t)((v / kPer) * 8 * kRow);
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
          const int stage = it % a.nstage;
          uint8_t* A = stages + (size_t)stage * a.stage_bytes;
          const int t = q % nslab;
          if (!mbar_wait(&gbar[stage], (it / a.nstage) & 1u, abort_flag, tb.status)) {
            ok = false;
            break;
          }
          if (early && q + P < total && !issue(q + P)) {
            ok = false;
            break;
          }
          // the row's raw x of this half-stage, read before it is overwritten
          float xv[kHalf];
#pragma unroll
          for (int i4 = 0; i4 < kHalf / 4; ++i4) {
            const float4 q4 = *reinterpret_cast<const float4*>(
                A + (i4 / kCpp) * kPart +
                swz_m<kMode>((uint32_t)r, (uint32_t)((h * kCpp + i4 % kCpp) * 16)));
            xv[4 * i4] = q4.x;
            xv[4 * i4 + 1] = q4.y;
            xv[4 * i4 + 2] = q4.z;
            xv[4 * i4 + 3] = q4.w;
          }
          constexpr int kPer = 16 / kEl;  // elements per 16-byte chunk
          float d2p = 0.f;
          // this half's kCpp chunks of 16 bytes per part row, each stored whole
#pragma unroll
          for (int cc = 0; cc < kCpp; ++cc) {
            const int c = h * kCpp + cc;  // chunk of the row
            float yh[kPer], yl[kPer], oh[kPer], ol[kPer];
            const int jc = t * kKs + h * kHalf + cc * kPer;  // first column of the chunk
#pragma unroll
            for (int q4 = 0; q4 < kPer / 4; ++q4) {  // o words, 16 bytes at a time
              const float4 a4 = *reinterpret_cast<const float4*>(tabH + jc + 4 * q4);
              const float4 b4 = *reinterpret_cast<const float4*>(tabL + jc + 4 * q4);
              oh[4 * q4] = a4.x; oh[4 * q4 + 1] = a4.y; oh[4 * q4 + 2] = a4.z; oh[4 * q4 + 3] = a4.w;
              ol[4 * q4] = b4.x; ol[4 * q4 + 1] = b4.y; ol[4 * q4 + 2] = b4.z; ol[4 * q4 + 3] = b4.w;
            }
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
              // branch-free, so that the chunk's elements interleave.  A
              // column past the block has x = 0 (zero-filled copy) and o = 0
              // (staged), so y = 0; a row past the batch is never written.
              // EXACT slices y to 2^-26 of the row scale: the exact
              // double-float shift.  The split modes keep 22 (16) bits of y:
              // x - o_hi is exact near o (Sterbenz) and one more rounding of
              // the low word of o stays below those bits.
              if constexpr (kMode == M_EXACT) {
                shift_ff(xv[cc * kPer + e], oh[e], ol[e], yh[e], yl[e]);
              } else {
                yh[e] = __fsub_rn(__fsub_rn(xv[cc * kPer + e], oh[e]), ol[e]);
                yl[e] = 0.f;
              }
              if (need_d2) d2p = fmaf(yh[e], yh[e], d2p);
            }
            const uint32_t off = swz_m<kMode>((uint32_t)r, (uint32_t)(c * 16));
            if constexpr (kMode == M_TF32) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const float a = yh[qq];
                hw[qq] = to_tf32(a);
                lw[qq] = to_tf32((a - __uint_as_float(hw[qq])) + yl[qq]);
              }
              *reinterpret_cast<uint4*>(A + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(A + kPart + off) =
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
              *reinterpret_cast<uint4*>(A + kPart + off) =
                  make_uint4(lw[0], lw[1], lw[2], lw[3]);
            } else if constexpr (kMode == M_F16) {
              // y / sigma in (-1, 1) (an exact power-of-two scaling) as FP16
              // hi + lo: 22 significant bits, as TF32 hi + lo
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const float a = yh[2 * qq] * isig, b = yh[2 * qq + 1] * isig;
                const __half2 hh = __floats2half2_rn(a, b);
                const float2 hf = __half22float2(hh);
                const __half2 ll = __floats2half2_rn(fmaf(yl[2 * qq], isig, a - hf.x),
                                                     fmaf(yl[2 * qq + 1], isig, b - hf.y));
                hw[qq] = *reinterpret_cast<const uint32_t*>(&hh);
                lw[qq] = *reinterpret_cast<const uint32_t*>(&ll);
              }
              *reinterpret_cast<uint4*>(A + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(A + kPart + off) =
                  make_uint4(lw[0], lw[1], lw[2], lw[3]);
            } else {
              // four slices of v = 128 y / sigma (exact in BF16), already at
              // their weight: s1 = rint(v), then the remainder r = v - s1
              // (plus y's low word) rounded to multiples of 2^-8, 2^-16 and
              // 2^-24 in turn.  Adding and subtracting 1.5 * 2^(23 - 8a)
              // rounds to a multiple of 2^-8a, ties to even, exactly as rintf
              // of the 2^8a-scaled value does (|v| < 128, |r| <= 2^-1, 2^-9,
              // 2^-17), and every remainder is exact
              const float s128 = isig * 128.f;
              uint32_t w[4][4];
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                float sl[2][4];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                  const int k = 2 * qq + e;
                  const float v = yh[k] * s128;
                  const float y1 = (v + 12582912.0f) - 12582912.0f;       // 1.5 * 2^23
                  float rr = fmaf(yl[k], s128, v - y1);
                  const float y2 = (rr + 49152.0f) - 49152.0f;            // 1.5 * 2^15
                  rr = rr - y2;
                  const float y3 = (rr + 192.0f) - 192.0f;                // 1.5 * 2^7
                  rr = rr - y3;
                  const float y4 = (rr + 0.75f) - 0.75f;                  // 1.5 * 2^-1
                  sl[e][0] = y1;
                  sl[e][1] = y2;
                  sl[e][2] = y3;
                  sl[e][3] = y4;
                }
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) w[pp][qq] = pack_bf16(sl[0][pp], sl[1][pp]);
              }
#pragma unroll
              for (int pp = 0; pp < 4; ++pp)
                *reinterpret_cast<uint4*>(A + pp * kPart + off) =
                    make_uint4(w[pp][0], w[pp][1], w[pp][2], w[pp][3]);
            }
          }
          if (q < nslab) d2 += (double)d2p;  // first chunk: ||x - o||^2 of the row
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[stage]);
          if (!early && q + P < total) ok = issue(q + P);
        }
        }
      }
      rowD2[(h * kMaxComponents + ci) * kTileM + r] = d2;  // each half's share
    }
}

template <int kMode, bool kHeavy>
__device__ void epilogue_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs) {
  CUROB_ROLE_PROLOGUE
    // ------------------------------------------------------------- epilogue
    const int q = warp - 8;                 // TMEM lane quadrant (warp % 4)
    const int r = q * 32 + lane;            // candidate row in the tile
    const uint32_t t_lane = tmem_base + ((uint32_t)(q * 32) << 16);
    uint32_t& chunk_it = rs.chunk_it;
    EpiState st;
    for (int li = 0; li < a.nlist && !*abort_flag; ++li, ++rs.comp_it) {
      const int ci = a.list[li];
      const uint32_t cg = rs.comp_it;
      const Component Cm = tb.comp[F.comp0 + ci];
      double gsum = 0.0;
      float sig = 1.f;
      if constexpr (scaled_mode(kMode)) {
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
        es.kat_e = sg.kat_e;
        es.aux = sg.aux_off >= 0 ? tb.aux32 + sg.aux_off : nullptr;
        es.gpos = sg.gpos;
        es.gfirst = sg.gfirst;
        const float* tau = a.tau + sg.tau_off;
        // scaled modes: the block's row scales of R go to shared memory once
        // (every drained column needs one, the same for all 128 rows), in one
        // of two buffers: a warp stages the next block only after its own
        // drain of this one, and the group barrier then holds it until every
        // warp has finished this block
        const float* tt = a.tabt ? m.tabT + (rs.e_blk & 1u) * kMaxNpad : tau;
        if (scaled_mode(kMode) && a.tabt) {
          float* tw = m.tabT + (rs.e_blk & 1u) * kMaxNpad;
          for (int k = r; k < sg.npad; k += kTileM) tw[k] = k < sg.n ? __ldg(tau + k) : 0.f;
          if (!producers_sync(m.epi_bar, rs.e_phase, abort_flag, tb.status)) {
            ok = false;
            break;
          }
        }
        ++rs.e_blk;
        (void)tau;
        // heavy kinds with a z scratch: the rows' z go out, variable-major
        // (a warp's store of one variable covers 32 consecutive rows)
        const bool zout = a.zbuf != nullptr && sg.hoff >= 0;
        const long long grow = row0 + r;
        float* zcol = zout ? a.zbuf + (size_t)sg.hoff * a.N + (grow < a.N ? grow : 0) : nullptr;
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
          const bool odd = (chunk_it & 1u) != 0;
          const uint32_t ab = odd ? (uint32_t)a.acc_hi : 0u;  // TMEM column of local column 0
          // local columns [l0, l1) of this hand-off, 32 at a time
          auto drain = [&](int l0, int l1) {
            for (int l = l0; l < l1; l += 32) {
              const int c = c_lo + l;
              const int cend = min(32, l1 - l);
              float v[32];
              if constexpr (kMode == M_EXACT) {
                float g1[32];
                tmem_ld32x2(t_lane + ab + (uint32_t)l, t_lane + kExactAcc1 + ab + (uint32_t)l, v, g1);
                const float base = sig * 6.103515625e-05f;  // sigma 2^-14
                if (a.tabt) {  // shared memory, 16-byte aligned (c is a multiple of 16)
#pragma unroll
                  for (int k4 = 0; k4 < 8; ++k4) {
                    const float4 t4 = *reinterpret_cast<const float4*>(tt + c + 4 * k4);
                    const float ts[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                      const int k = 4 * k4 + e;
                      v[k] = (k < cend) ? (v[k] + g1[k]) * (base * ts[e]) : 0.f;
                    }
                  }
                } else {
#pragma unroll
                  for (int k = 0; k < 32; ++k)
                    v[k] = (k < cend) ? (v[k] + g1[k]) * (base * tt[c + k]) : 0.f;
                }
              } else if constexpr (kMode == M_F16) {
                tmem_ld32(t_lane + ab + (uint32_t)l, v);
#pragma unroll
                for (int k = 0; k < 32; ++k) v[k] = (k < cend) ? v[k] * (sig * tt[c + k]) : 0.f;
              } else {
                tmem_ld32(t_lane + ab + (uint32_t)l, v);
              }
              if (zout) {
                if (grow < a.N) {
#pragma unroll
                  for (int k = 0; k < 32; ++k)
                    if (k < cend) zcol[(size_t)(c + k) * a.N] = v[k] * es.s + es.c0;
                }
              } else {
                epi_chunk<kHeavy>(kind, v, c, cend, es, st);
              }
            }
          };
          auto release = [&]() {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_empty);
          };
          const int w = c_hi - c_lo;
          // Columns the next hand-off's region covers go first, then the
          // accumulator is released and the rest drains under the next
          // block's MMAs.  Pair kinds (a chain over consecutive columns) and
          // the fused build keep column order and release at the end.
          if (zout || (!kHeavy && !kind_has_pairs(kind))) {
            int f0, f1;  // local range shared with the next hand-off's region
            if (odd) {
              f0 = 0;
              f1 = max(0, min(w, a.acc_ovl));
            } else {
              f0 = min(w, a.acc_hi);
              f1 = w;
            }
            drain(f0, f1);
            release();
            drain(0, f0);
            drain(f1, w);
          } else {
            drain(0, w);
            release();
          }
        }
        if (ok && sg.glast && !zout) gsum += st.close(kind, sg.gn);
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
    // One thread issues every MMA of the CTA, so its own instructions between
    // two stages are time the tensor pipe may stand idle: the descriptors of
    // the rings' first slots are formed once (a descriptor's address field is
    // the byte address / 16, so a slot, part or K step is a constant added to
    // it), and slot indices and barrier parities advance by counting.
    if (lane == 0) {
      uint32_t& it = rs.it;
      uint32_t& chunk_it = rs.chunk_it;
      const bool split_b = m.fullB != m.full;
      const int nA = m.nA, nB = m.nB;
      int sA = (int)(it % (uint32_t)nA), sB = (int)(it % (uint32_t)nB);
      uint32_t pA = (it / (uint32_t)nA) & 1u;
      const uint64_t dA0 = sdesc_m<kMode>(smem_u32(m.a_base));
      const uint64_t dB0 = sdesc_m<kMode>(smem_u32(m.b_base));
      const uint32_t aStr = (uint32_t)m.a_stride >> 4, bStr = (uint32_t)m.b_stride >> 4;
      uint32_t offA = (uint32_t)sA * aStr, offB = (uint32_t)sB * bStr;
      constexpr uint32_t kPart16 = (uint32_t)kPart >> 4;
      constexpr uint32_t kKo16 = (uint32_t)(C::kMmaK * kEl) >> 4;  // one MMA K step
      bool ok = true;
      for (int li = 0; li < a.nlist && ok && !*abort_flag; ++li) {
        const Component Cm = tb.comp[F.comp0 + a.list[li]];
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
            const uint32_t bpart16 = (uint32_t)(nc * kRow) >> 4;  // B part, in 16-byte units
            const uint32_t bh16 = (uint32_t)(n0 * kRow) >> 4;     // second N range of a part
            if (!mbar_wait(tmem_empty, (chunk_it & 1u) ^ 1u, abort_flag, tb.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ab = (chunk_it & 1u) ? (uint32_t)a.acc_hi : 0u;  // accumulator region
            const uint32_t dt0 = tmem_base + ab, dt1 = dt0 + (uint32_t)n0;
            for (int t = 0; t < nslab; ++t, ++it) {
              // one barrier per stage: the producers' 8 arrivals and the B
              // copy's bytes (the B ring never runs ahead of the A ring:
              // nB <= nA, so the copy of stage it cannot land on the phase
              // of stage it - nA)
              if (!mbar_wait(&full[sA], pA, abort_flag, tb.status)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint64_t da = dA0 + offA, db = dB0 + offB;
#pragma unroll
              for (int kk = 0; kk < kKsteps; ++kk) {
                const uint32_t ko = (uint32_t)kk * kKo16;
                const uint32_t first = (t == 0 && kk == 0) ? 0u : 1u;
                if constexpr (kMode == M_EXACT) {
                  // s1 r1 into accumulator 0; the pre-scaled products of
                  // weight 2^-8 to 2^-24 (a + b <= 3) into accumulator 1
                  constexpr int kPa[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
                  constexpr int kPb[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
#pragma unroll
                  for (int pq = 0; pq < 10; ++pq)
                    tc_mma<false>(pq == 0 ? dt0 : dt0 + (uint32_t)kExactAcc1,
                                  da + (uint32_t)kPa[pq] * kPart16 + ko,
                                  db + (uint32_t)kPb[pq] * bpart16 + ko, id0,
                                  (pq <= 1) ? first : 1u);
                } else {
                  const uint64_t dah = da + ko, dal = da + kPart16 + ko;
                  const uint64_t dbh = db + ko, dbl = db + bpart16 + ko;
                  tc_mma<kMode == M_TF32>(dt0, dah, dbh, id0, first);
                  tc_mma<kMode == M_TF32>(dt0, dah, dbl, id0, 1u);
                  tc_mma<kMode == M_TF32>(dt0, dal, dbh, id0, 1u);
                  if (n1 > 0) {
                    tc_mma<kMode == M_TF32>(dt1, dah, dbh + bh16, id1, first);
                    tc_mma<kMode == M_TF32>(dt1, dah, dbl + bh16, id1, 1u);
                    tc_mma<kMode == M_TF32>(dt1, dal, dbh + bh16, id1, 1u);
                  }
                }
              }
              tc_commit(&empty[sA]);  // frees the stage when these MMAs retire
              if (split_b) tc_commit(&m.emptyB[sB]);
              if (++sA == nA) {
                sA = 0;
                offA = 0;
                pA ^= 1u;
              } else {
                offA += aStr;
              }
              if (++sB == nB) {
                sB = 0;
                offB = 0;
              } else {
                offB += bStr;
              }
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
      for (int li = 0; li < a.nlist && ok && !*abort_flag; ++li) {
        const Component Cm = tb.comp[F.comp0 + a.list[li]];
        for (int si = 0; si < Cm.nseg && ok; ++si) {
          const Segment sg = tb.seg[Cm.seg0 + si];
          const int nslab = sg.npad / kKs;
          const int nchunk = kMode == M_EXACT ? exact_nchunk(sg.npad) : 1;
          const int nw = kMode == M_EXACT ? exact_nw(sg.npad) : sg.npad;
          const long long fl = image_floats(sg.npad);
          const uint8_t* base = a.img + ((size_t)sg.img_off + (size_t)kMode * fl) * 4;
          for (int cc = 0; cc < nchunk && ok; ++cc) {
            const int nc = kMode == M_EXACT ? min(nw, sg.npad - cc * nw) : sg.npad;
            const uint32_t bytes = (uint32_t)(kParts * nc * kRow);
            const uint8_t* src = base + (size_t)cc * nslab * kParts * nw * kRow;
            for (int t = 0; t < nslab; ++t, ++it) {
              const int stage = it % m.nB;
              const uint32_t ph = (it / m.nB) & 1u;
              if (!mbar_wait(&m.emptyB[stage], ph ^ 1u, abort_flag, tb.status)) {
                ok = false;
                break;
              }
              uint8_t* dst = m.b_base + (size_t)stage * m.b_stride;
              // completion goes to the full barrier of the stage's A slot
              const int sa = it % m.nA;
              const uint32_t pa = (it / m.nA) & 1u;
              mbar_arrive_expect_tx(&m.full[sa], bytes);
              rs.b_par = (rs.b_par & ~(1u << sa)) | (pa << sa) | (1u << (sa + 8));
              bulk_g2s(dst, src + (size_t)t * bytes, bytes, &m.full[sa]);
            }
          }
        }
      }
    }
    __syncwarp();
}

// x^T launches: lane 0 of the raw-gather warp walks the tile's K stages in
// the producers' order and gathers each stage's variables (rows of x^T, the
// tile's 128 candidates each, four rows per TMA gather) into the A slot the
// stage will be converted in, as soon as the MMAs of that slot's previous
// stage have retired.  The block's variable indices come straight from the
// instance, so the warp runs ahead of the producers across block
// boundaries.
template <int kMode>
__device__ void raw_loader_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs,
                                const CUtensorMap* xmap) {
  CUROB_ROLE_PROLOGUE
  constexpr int kRawBytes = kKs * kTileM * 4;
  constexpr int kGat = kKs / 4;
  if (lane == 0) {
    uint32_t& it = rs.it;
    const int nA = m.nA;
    bool ok = true;
    for (int li = 0; li < a.nlist && ok && !*abort_flag; ++li) {
      const Component Cm = tb.comp[F.comp0 + a.list[li]];
      for (int si = 0; si < Cm.nseg && ok; ++si) {
        const Segment sg = tb.seg[Cm.seg0 + si];
        const int* S = tb.S + Cm.base + sg.zoff;
        const int nslab = sg.npad / kKs;
        const int nchunk = kMode == M_EXACT ? exact_nchunk(sg.npad) : 1;
        const int total = nslab * nchunk;
        for (int q = 0; q < total; ++q, ++it) {
          const int t = q % nslab;
          int rr[kKs];  // the stage's variables (loads in flight during the wait)
#pragma unroll
          for (int e = 0; e < kKs; ++e) {
            const int j = t * kKs + e;
            rr[e] = __ldg(S + (j < sg.n ? j : 0));
          }
          const int slot = it % nA;
          if (!mbar_wait(&empty[slot], ((it / nA) & 1u) ^ 1u, abort_flag, tb.status)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&m.rawfull[slot], (uint32_t)kRawBytes);
          rs.r_par = (rs.r_par & ~(1u << slot)) | (((it / nA) & 1u) << slot) | (1u << (slot + 8));
          uint8_t* dst = m.a_base + (size_t)slot * m.a_stride + kParts * kPart - kRawBytes;
#pragma unroll
          for (int gg = 0; gg < kGat; ++gg)
            tma_gather4(dst + gg * 4 * kTileM * 4, xmap, (int)row0, rr[4 * gg], rr[4 * gg + 1],
                        rr[4 * gg + 2], rr[4 * gg + 3], &m.rawfull[slot]);
        }
      }
    }
  }
  __syncwarp();
}

template <int kMode, bool kHeavy, bool kXT>
__device__ inline void run_tile(const MmaArgs& a, const Smem& m, long long row0, RoleState& rs,
                                const CUtensorMap* xmap) {
  const int warp = threadIdx.x >> 5;
  if (warp < 8) producer_tile<kMode, kXT>(a, m, row0, rs, xmap);
  else if (warp < 12) epilogue_tile<kMode, kHeavy>(a, m, row0, rs);
  else if (warp == kMmaWarp) mma_tile<kMode>(a, m, row0, rs);
  else if (warp == kLoaderWarp) loader_tile<kMode>(a, m, row0, rs);
  else if constexpr (kXT) raw_loader_tile<kMode>(a, m, row0, rs, xmap);
  if (*m.abort_flag) {  // no copy may still be landing when the CTA moves on or exits
    const unsigned long long deadline = globaltimer() + kTimeoutNs;
    if (warp < 8) asm volatile("cp.async.wait_all;" ::: "memory");
    if (warp == kLoaderWarp && (threadIdx.x & 31) == 0)
      for (int s = 0; s < m.nA; ++s)  // B copies complete on full[] of their A slot
        if (rs.b_par >> (s + 8) & 1u) mbar_drain(&m.full[s], rs.b_par >> s & 1u, deadline);
    if (kXT && warp == kRawWarp && (threadIdx.x & 31) == 0)  // the raw gathers' issuer
      for (int s = 0; s < m.nA; ++s)
        if (rs.r_par >> (s + 8) & 1u) mbar_drain(&m.rawfull[s], rs.r_par >> s & 1u, deadline);
  }
  // every issued MMA has been consumed by the epilogue (or the CTA aborted)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  write_outputs(a, m, row0);
}

// One launch per function: CTA b evaluates candidates [128 b, 128 b + 128).
template <int kMode, bool kHeavy, bool kXT>
__global__ void __launch_bounds__(kXT ? kThreadsXT : kThreads, 1)
mma_eval_kernel(MmaArgs args, const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const Smem m = smem_map(smem_raw, RingGeom{args.xt, args.nstage, args.stage_bytes, args.nA,
                                             args.a_bytes, args.nB, args.b_bytes});
  cta_setup(m, args.xt);
  if (kXT && threadIdx.x == 0) tma_prefetch_desc(&xmap);
  RoleState rs;
  run_tile<kMode, kHeavy, kXT>(args, m, (long long)blockIdx.x * kTileM, rs, &xmap);
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
  constexpr int kA = MC<kMode>::kParts * MC<kMode>::kPart;
  const Smem m = smem_map(smem_raw, RingGeom{0, nstage, stage_bytes, nstage, kA, nstage,
                                             stage_bytes - kA});
  cta_setup(m, 0);
  RoleState rs;
  for (;;) {
    if (threadIdx.x == 0) *m.item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = *m.item;
    if (w >= nwork || *m.abort_flag) break;
    const int2 W = work[w];
    run_tile<kMode, true, false>(insts[W.x], m, (long long)W.y * kTileM, rs, nullptr);
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
    {  // FP16: stage t = col / 32, hi = fp16(R / tau_row), lo = fp16(R / tau_row - hi)
      const int t = col / 32, k = col % 32;
      uint8_t* hi = base + (size_t)3 * fl * 4 + (size_t)t * (2 * npad * kRowBytes);
      uint8_t* lo = hi + npad * kRowBytes;
      const uint32_t off = swz64((uint32_t)row, (uint32_t)(k * 2));
      const double w = v / (double)tau[J.tau_off + row];  // exact: tau is 2^f
      const __half h = __double2half(w);
      const __half l = __double2half(w - (double)__half2float(h));
      *reinterpret_cast<__half*>(hi + off) = h;
      *reinterpret_cast<__half*>(lo + off) = l;
    }
    {  // EXACT: chunk cc = row / nw, stage t = col / 16 (32-byte rows), four slices
      const int nw = exact_nw(npad);
      const int cc = row / nw, rr = row % nw;
      const int nc = min(nw, npad - cc * nw);
      const int t = col / 16, k = col % 16;
      const int nslab16 = npad / 16;
      uint8_t* st = base + (size_t)2 * fl * 4 +
                    ((size_t)cc * nslab16 * 4 * nw + (size_t)t * 4 * nc) * 32;
      const uint32_t off = swz32((uint32_t)rr, (uint32_t)(k * 2));
      double w = v / (double)tau[J.tau_off + row] * 128.0;  // exact: tau is 2^f
      double scale = 1.0;
      for (int s = 0; s < 4; ++s) {
        const double yv = rint(w);
        *reinterpret_cast<__nv_bfloat16*>(st + (size_t)s * nc * 32 + off) =
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
  return (size_t)MC<kMode>::kParts * MC<kMode>::kPart +
         (size_t)MC<kMode>::kParts * ncmax * MC<kMode>::kRow;
}
size_t ctrl_bytes() {  // barriers and work item (<= 256 B) + per-row tables + block table
  return kCtrlHeader + 3 * sizeof(double) * kMaxComponents * kTileM +
         sizeof(float) * (kSigRing + 1) * kTileM +
         3 * sizeof(float) * kMaxNpad;
}

// Self-test of the bounded waits: thread 0 waits on an mbarrier that nothing
// arrives at; after kTimeoutNs the wait gives up, sets DEV_TIMEOUT in
// *status and the kernel returns normally.
__global__ void wait_selftest_kernel(int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, &abort_flag, status);
}

// ---------------------------------------------------------- finish kernel
// Closes what split launches of the tensor-core kernel left: the basic
// functions of heavy kind, from their z in the scratch (variable-major,
// [F.hcols][N]); adds them to the component values G_c of the light kinds;
// then composes (Sec. 6) or writes f.  A block takes kFinX candidates
// (threadIdx.x: every load of one variable is two full 32-byte sectors) and
// kFinSlices slices of each block's variables (threadIdx.y); a slice sums its
// terms in FP32 (at most 32 at block widths <= 512), the slices are added in
// FP64 (shuffles within a warp, then across the warps), as the epilogue adds
// its 32-column partial sums.  The terms are latency-bound chains of
// transcendentals: 8 blocks of 8 warps per SM (32 registers, a few spilled
// to L1) beat fewer warps with no spills.
constexpr int kFinX = 16;
constexpr int kFinSlices = 16;

template <int KIND>
__device__ __forceinline__ void fin_terms(const float* zc, long long ld, int j0, int j1, int gpos,
                                          float gn, const float* aux, float kat_e,
                                          Acc<float>& acc) {
  if constexpr (kind_has_pairs(KIND)) {
    // pairs (z_{g-1}, z_g) for function positions g = gpos + j >= 1; the
    // function's blocks are consecutive in the scratch, so column j0 - 1 is
    // the previous block's last variable when j0 = 0 < gpos
    if (j0 >= j1) return;
    float zp = (gpos + j0 > 0) ? zc[(long long)(j0 - 1) * ld] : 0.f;
    for (int j = j0; j < j1; ++j) {
      const float zj = zc[(long long)j * ld];
      if (gpos + j > 0) acc.a0 += pair_term<float>(KIND, zp, zj);
      zp = zj;
    }
  } else {
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
      const float zj = zc[(long long)j * ld];
      elem_term_f32(KIND, zj, zj, gpos + j, gn, aux ? aux[j] : 0.f, kat_e, acc);
    }
  }
}

__device__ __forceinline__ void fin_dispatch(int kind, const float* zc, long long ld, int j0,
                                             int j1, int gpos, float gn, const float* aux,
                                             float kat_e, Acc<float>& acc) {
  switch (kind) {
#define CUROB_FIN_CASE(K) \
  case K: fin_terms<K>(zc, ld, j0, j1, gpos, gn, aux, kat_e, acc); break;
    CUROB_FIN_CASE(K_POWERS) CUROB_FIN_CASE(K_WEIERSTRASS) CUROB_FIN_CASE(K_GRIEWANK)
    CUROB_FIN_CASE(K_SCHAFFER7) CUROB_FIN_CASE(K_EGR) CUROB_FIN_CASE(K_SCHWEFEL)
    CUROB_FIN_CASE(K_KATSUURA) CUROB_FIN_CASE(K_SCHAFFER6)
#undef CUROB_FIN_CASE
    default: break;
  }
}

// Heavy kinds accumulate only a sum (a0) and a product (p): kind_uses_a1 and
// kind_uses_a2 are false for all of them.
static_assert(!kind_uses_a1(K_POWERS) && !kind_uses_a1(K_WEIERSTRASS) && !kind_uses_a1(K_GRIEWANK) &&
                  !kind_uses_a1(K_SCHAFFER7) && !kind_uses_a1(K_EGR) && !kind_uses_a1(K_SCHWEFEL) &&
                  !kind_uses_a1(K_KATSUURA) && !kind_uses_a1(K_SCHAFFER6) &&
                  !kind_uses_a2(K_POWERS) && !kind_uses_a2(K_WEIERSTRASS) &&
                  !kind_uses_a2(K_GRIEWANK) && !kind_uses_a2(K_SCHAFFER7) && !kind_uses_a2(K_EGR) &&
                  !kind_uses_a2(K_SCHWEFEL) && !kind_uses_a2(K_KATSUURA) && !kind_uses_a2(K_SCHAFFER6),
              "heavy kinds use a0 and p only");

// Members evaluated from x^T (Function::xcand): z_j = s y_j + c with y_j =
// (x_j - o_hi,j) - o_lo,j, as the tensor-core path forms it for an identity
// block; the slice's terms and its share of ||x - o||^2.
template <int KIND>
__device__ __forceinline__ void fin_terms_x(const float* xc, long long ld, const float* oh,
                                            const float* ol, int j0, int j1, int gpos, float gn,
                                            const float* aux, float kat_e, float s, float c0,
                                            Acc<float>& acc, float& d2) {
#pragma unroll 4
  for (int j = j0; j < j1; ++j) {
    const float y = __fsub_rn(__fsub_rn(xc[(long long)j * ld], oh[j]), ol[j]);
    const float u = y * s;
    elem_term_f32(KIND, u + c0, u, gpos + j, gn, aux ? aux[j] : 0.f, kat_e, acc);
    d2 = fmaf(y, y, d2);
  }
}
__device__ __forceinline__ void fin_dispatch_x(int kind, const float* xc, long long ld,
                                               const float* oh, const float* ol, int j0, int j1,
                                               int gpos, float gn, const float* aux, float kat_e,
                                               float s, float c0, Acc<float>& acc, float& d2) {
  switch (kind) {
#define CUROB_FINX_CASE(K) \
  case K: fin_terms_x<K>(xc, ld, oh, ol, j0, j1, gpos, gn, aux, kat_e, s, c0, acc, d2); break;
    CUROB_FINX_CASE(K_SPHERE) CUROB_FINX_CASE(K_ELLIPSOID) CUROB_FINX_CASE(K_ELLIPTIC)
    CUROB_FINX_CASE(K_POWERS) CUROB_FINX_CASE(K_STEP) CUROB_FINX_CASE(K_WEIERSTRASS)
    CUROB_FINX_CASE(K_RASTRIGIN) CUROB_FINX_CASE(K_SCHWEFEL)
#undef CUROB_FINX_CASE
    default: break;
  }
}

__device__ __forceinline__ void fin_warp_sum(double& a0, double& p) {
  // lanes tx, tx + kFinX, ... of a warp hold the same candidate
#pragma unroll
  for (int off = kFinX; off < 32; off <<= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
    p *= __shfl_xor_sync(0xffffffffu, p, off);
  }
}

__global__ void __launch_bounds__(kFinX * kFinSlices, 8)
finish_kernel(Tables tb, Function F, const float* zbuf, const double* gout, const double* d2out,
              int N, float* out, const float* xT, long long ld, const float* ohi,
              const float* olo, uint32_t xmask) {
  constexpr int kWarps = kFinX * kFinSlices / 32;
  constexpr int kSlicesPerWarp = 32 / kFinX;
  __shared__ double red[2][kWarps][kFinX];
  __shared__ double Gs[kMaxComponents][kFinX];
  __shared__ double D2s[kMaxComponents][kFinX];  // ||x - o_c||^2 of members read from x^T
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int warp = ty / kSlicesPerWarp;
  const long long i = (long long)blockIdx.x * kFinX + tx;
  const bool valid = i < N;
  const long long ic = valid ? i : 0;  // rows past N read row 0 and write nothing
  if (ty == 0)
    for (int c = 0; c < F.ncomp; ++c) Gs[c][tx] = (xmask >> c & 1u) ? 0.0 : gout[(size_t)c * N + ic];
  double a0 = 0.0, p = 1.0;
  for (int c = 0; c < F.ncomp; ++c) {
    const Component Cm = tb.comp[F.comp0 + c];
    const bool fx = (xmask >> c & 1u) != 0;  // block-uniform
    double d2acc = 0.0;
    for (int si = 0; si < Cm.nseg; ++si) {
      const Segment sg = tb.seg[Cm.seg0 + si];
      if (!fx && sg.hoff < 0) continue;  // block-uniform: every thread takes the same path
      if (sg.gfirst) {
        a0 = 0.0;
        p = 1.0;
      }
      const int L = (sg.n + kFinSlices - 1) / kFinSlices;
      const int j0 = min(sg.n, ty * L), j1 = min(sg.n, j0 + L);
      const float* aux = sg.aux_off >= 0 ? tb.aux32 + sg.aux_off : nullptr;
      Acc<float> acc = acc_zero<float>();
      if (fx) {
        float d2f = 0.f;
        fin_dispatch_x(sg.kind, xT + (size_t)sg.zoff * ld + ic, ld, ohi + Cm.base + sg.zoff,
                       olo + Cm.base + sg.zoff, j0, j1, sg.gpos, (float)sg.gn, aux, sg.kat_e,
                       (float)sg.scale, (float)sg.offset, acc, d2f);
        d2acc += (double)d2f;
      } else {
        const float* zc = zbuf + (size_t)sg.hoff * N + ic;
        fin_dispatch(sg.kind, zc, N, j0, j1, sg.gpos, (float)sg.gn, aux, sg.kat_e, acc);
      }
      a0 += (double)acc.a0;
      if (kind_uses_p(sg.kind)) p *= (double)acc.p;
      if (sg.glast) {
        fin_warp_sum(a0, p);
        if (ty % kSlicesPerWarp == 0) {
          red[0][warp][tx] = a0;
          red[1][warp][tx] = p;
        }
        __syncthreads();
        if (warp == 0) {  // lane (tx, q): warps q, q + kSlicesPerWarp, ...; then across q
          const int q = ty % kSlicesPerWarp;
          double s0 = 0.0, pp = 1.0;
          for (int w = q; w < kWarps; w += kSlicesPerWarp) {
            s0 += red[0][w][tx];
            pp *= red[1][w][tx];
          }
          fin_warp_sum(s0, pp);
          if (ty == 0) {
            if (kind_is_cyclic(sg.kind)) {  // (z_gn, z_1) closes the cycle
              const float* zf = zbuf + (size_t)(sg.hoff - sg.gpos) * N + ic;
              s0 += (double)pair_term<float>(sg.kind, zf[(size_t)(sg.gn - 1) * N], zf[0]);
            }
            Gs[c][tx] += finalize_f32(sg.kind, s0, 0.0, 0.0, pp, sg.gn);
          }
        }
        __syncthreads();
      }
    }
    if (fx && F.composition) {  // the member's ||x - o||^2 across the slices
      double one = 1.0;
      fin_warp_sum(d2acc, one);
      if (ty % kSlicesPerWarp == 0) red[0][warp][tx] = d2acc;
      __syncthreads();
      if (warp == 0) {
        const int q = ty % kSlicesPerWarp;
        double s0 = 0.0, pp = 1.0;
        for (int w = q; w < kWarps; w += kSlicesPerWarp) s0 += red[0][w][tx];
        fin_warp_sum(s0, pp);
        if (ty == 0) D2s[c][tx] = s0;
      }
      __syncthreads();
    }
  }
  if (ty != 0 || !valid) return;
  double f;
  if (F.composition) {
    double G[kMaxComponents], d2v[kMaxComponents];
    for (int c = 0; c < F.ncomp; ++c) {
      G[c] = Gs[c][tx];
      d2v[c] = (xmask >> c & 1u) ? D2s[c][tx] : d2out[(size_t)c * N + i];
    }
    f = compose(tb.comp + F.comp0, F.ncomp, G, d2v, tb.D);
  } else {
    f = Gs[0][tx];
  }
  out[i] = (float)(f + kFopt);
}

// Accumulator regions of a launch (MmaArgs::acc_hi, acc_ovl): EXACT hand-offs
// are at most kExactMaxNC wide in each 256-column half of TMEM; the others are
// a whole block, npad_max rounded up to 32, in all 512 columns.
template <int kMode>
void set_acc_regions(MmaArgs& a, int npad_max) {
  const int T = kMode == M_EXACT ? kExactAcc1 : kMaxNpad;
  const int W = kMode == M_EXACT ? kExactMaxNC : std::min(kMaxNpad, (npad_max + 31) / 32 * 32);
  a.acc_hi = T - W;
  a.acc_ovl = 2 * W - T;
}

// x^T: the transposed copy of x (D rows of ld floats, candidates inner),
// with its TMA map; when given, the producers gather rows of it.
struct XtView {
  const float* xt = nullptr;
  const CUtensorMap* map = nullptr;
  const float* pm = nullptr;  // partial row maxima per component (MmaArgs::rowpm), or nullptr
  int ntx = 0, pm_ld = 0;
};

template <int kMode>
cudaError_t launch_mode(const MmaPlan& p, const Tables& tb, const Function& F, const float* x,
                        int N, float* out, cudaStream_t st, const int* list = nullptr,
                        int nlist = 0, double* gout = nullptr, double* d2out = nullptr,
                        float* zbuf = nullptr, XtView xv = XtView()) {
  using C = MC<kMode>;
  const int npad_max = npad_of(F.max_n);
  const int ncmax = kMode == M_EXACT ? std::min(npad_max, kExactMaxNC) : npad_max;
  const size_t sb = stage_bytes_for<kMode>(ncmax);
  const size_t ctrl = ctrl_bytes();
  const int nstage = (int)std::min<size_t>(kMaxStages, (kSmemCap - ctrl) / sb);
  if (nstage < 2) return cudaErrorInvalidValue;
  // heavy kinds in the epilogue only when there is no z scratch for them
  const bool heavy = zbuf == nullptr && F.hcols > 0;
  MmaArgs a;
  a.xt = 0;
  a.nA = a.nB = nstage;
  a.a_bytes = C::kParts * C::kPart;
  a.b_bytes = (int)sb - a.a_bytes;
  size_t smem = nstage * sb + ctrl + 1024;  // + alignment slack
  if (xv.xt && !heavy) {
    // separate rings: B slots hold a whole stage of R (the larger), A slots
    // the candidates' operands with their raw gathers inside
    const size_t ab = (size_t)C::kParts * C::kPart;
    const size_t bb = (size_t)C::kParts * ncmax * C::kRow;
    auto a_slots = [&](int nb) {
      const long long room = (long long)kSmemCap - (long long)ctrl - (long long)nb * bb;
      return room > 0 ? (int)std::min<long long>(kMaxARing, room / (long long)ab) : 0;
    };
    int nB = kMode == M_EXACT ? 4 : 3;
    int nA = a_slots(nB);
    // blocks wider than 352 (hybrids' 400-variable blocks at D = 1000): two B
    // slots, so that three A slots still fit beside them
    if (nA < 3 && kMode != M_EXACT) nA = a_slots(nB = 2);
    if (nA >= std::max(3, nB)) {  // the B ring may not run ahead of the A ring
      a.xt = 1;
      a.nA = nA;
      a.nB = nB;
      a.a_bytes = (int)ab;
      a.b_bytes = (int)bb;
      smem = nA * ab + nB * bb + ctrl + 1024;
    }
  }
  // the epilogue's tau buffers, where they fit beside the rings
  a.tabt = scaled_mode(kMode) && smem - 1024 + kTabTBytes <= kSmemCap ? 1 : 0;
  if (a.tabt) smem += kTabTBytes;
  a.rowpm = scaled_mode(kMode) ? xv.pm : nullptr;
  a.ntx = xv.ntx;
  a.pm_ld = xv.pm_ld;
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
  a.nlist = list ? nlist : F.ncomp;
  for (int i = 0; i < kMaxComponents; ++i) a.list[i] = list ? (i < nlist ? list[i] : 0) : i;
  a.gout = gout;
  a.d2out = d2out;
  a.zbuf = zbuf;
  set_acc_regions<kMode>(a, npad_max);
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  const CUtensorMap& map = a.xt ? *xv.map : none;
  const auto kern = a.xt ? mma_eval_kernel<kMode, false, true>
                         : (heavy ? mma_eval_kernel<kMode, true, false>
                                  : mma_eval_kernel<kMode, false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)((N + kTileM - 1) / kTileM), a.xt ? kThreadsXT : kThreads, smem, st>>>(a, map);
  return cudaGetLastError();
}

// x (N x D, row-major) -> x^T (D rows of ld floats), zeros past N: 64 x 64
// tiles through shared memory, read and written 16 bytes per thread and
// access (both sides coalesced).  Needs D % 4 == 0 and 16-byte aligned x;
// otherwise transpose_x_scalar_kernel.
// Row maxima the scaled modes need (MmaArgs::rowpm): for each listed
// component q, max_j |x_j - o_j| over each block's 64 variables, o in FP32 in
// natural order, the producers' own expression; pm[q][blockIdx.x][row].
struct RowMaxJob {
  int nc = 0;
  const float* o[kMaxComponents];
  float* pm[kMaxComponents];
};
__global__ void __launch_bounds__(256) transpose_x_kernel(const float* __restrict__ x, int N,
                                                          int D, float* __restrict__ xt, int ld,
                                                          RowMaxJob job) {
  __shared__ float tile[64][65];
  const int c0 = blockIdx.x * 64;  // variables
  const int r0 = blockIdx.y * 64;  // candidates
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16
  for (int k = ty; k < 64; k += 16) {
    const int r = r0 + k, c = c0 + 4 * tx;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < N && c < D) v = *reinterpret_cast<const float4*>(x + (size_t)r * D + c);
    tile[k][4 * tx] = v.x;
    tile[k][4 * tx + 1] = v.y;
    tile[k][4 * tx + 2] = v.z;
    tile[k][4 * tx + 3] = v.w;
#pragma unroll
    for (int q = 0; q < kMaxComponents; ++q) {  // the 16 lanes of a half-warp hold row r's 64 variables
      if (q >= job.nc) break;
      float mv = 0.f;
      if (c < D) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(job.o[q] + c));
        mv = fmaxf(fmaxf(fabsf(v.x - w.x), fabsf(v.y - w.y)), fmaxf(fabsf(v.z - w.z), fabsf(v.w - w.w)));
      }
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) mv = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, off));
      if (tx == 0 && r < ld) job.pm[q][(size_t)blockIdx.x * ld + r] = r < N ? mv : 0.f;
    }
  }
  __syncthreads();
  for (int k = ty; k < 64; k += 16) {
    const int c = c0 + k, r = r0 + 4 * tx;
    if (c < D && r < ld)
      *reinterpret_cast<float4*>(xt + (size_t)c * ld + r) =
          make_float4(tile[4 * tx][k], tile[4 * tx + 1][k], tile[4 * tx + 2][k], tile[4 * tx + 3][k]);
  }
}
__global__ void transpose_x_scalar_kernel(const float* __restrict__ x, int N, int D,
                                          float* __restrict__ xt, int ld) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32;  // variables
  const int r0 = blockIdx.y * 32;  // candidates
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < N && c < D) ? x[(size_t)r * D + c] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (c < D && r < ld) xt[(size_t)c * ld + r] = tile[threadIdx.x][k];
  }
}

// Whether transpose_x_kernel (and with it the row maxima) serves x.
bool transpose_vec(const float* x, int D, int ld) {
  return (D & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0 && (ld & 3) == 0;
}
cudaError_t launch_transpose_x(const float* x, int n, int D, float* xt, int ld, cudaStream_t st,
                               const RowMaxJob& job = RowMaxJob()) {
  if (transpose_vec(x, D, ld))
    transpose_x_kernel<<<dim3((D + 63) / 64, (unsigned)((ld + 63) / 64)), 256, 0, st>>>(x, n, D,
                                                                                     xt, ld, job);
  else
    transpose_x_scalar_kernel<<<dim3((D + 31) / 32, (unsigned)((ld + 31) / 32)), dim3(32, 8), 0,
                                st>>>(x, n, D, xt, ld);
  return cudaGetLastError();
}

// Candidates per row of x^T, rounded so that the rows start 128 bytes apart.
inline int xt_ld(int n) { return (n + 31) / 32 * 32; }

}  // namespace

// ------------------------------------------------------------- host side
curob_status mma_prepare(MmaPlan& p, std::vector<Segment>& segs, const Tables& tb, float* prev) {
  (void)prev;
  mma_release(p);
  int dev = 0, cc_major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
  p.ready = false;
  {  // a private pool, so the split launches' scratch stays mapped between calls
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&p.pool, &props) == cudaSuccess) {
      uint64_t keep = 2 * kScratchCap;
      cudaMemPoolSetAttribute(p.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      p.pool = nullptr;  // the device's default pool serves instead
    }
  }
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
    off += 4 * image_floats(s.npad);
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
  if (p.pool) cudaMemPoolDestroy(p.pool);  // freed once outstanding scratch is returned
  p.pool = nullptr;
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
  if (!F.sensitive) return CUROB_PRECISION_TF32X3;
  const int all = (1 << F.ncomp) - 1;
  return (F.composition && F.sens_mask != all) ? CUROB_PRECISION_MIXED : CUROB_PRECISION_EXACT;
}

namespace {
// Stage geometry of a persistent launch: EXACT stages hold one N chunk of at
// most kExactMaxNC columns whatever the item; TF32X3 stages a whole block,
// sized for the widest block among the launch's items (npad_max).
struct BatchGeom {
  int nstage, stage_bytes;
  size_t smem;
};
template <int kMode>
BatchGeom batch_geom_t(int npad_max) {
  BatchGeom g;
  const int ncmax = kMode == M_EXACT ? kExactMaxNC : std::min(kMaxNpad, npad_max);
  const size_t sb = stage_bytes_for<kMode>(ncmax);
  g.stage_bytes = (int)sb;
  g.nstage = (int)std::min<size_t>(kMaxStages, (kSmemCap - ctrl_bytes()) / sb);
  g.smem = g.nstage * sb + ctrl_bytes() + 1024;
  return g;
}
BatchGeom batch_geom(int mode, int npad_max) {
  return mode == CUROB_PRECISION_TF32X3 ? batch_geom_t<M_TF32>(npad_max)
                                        : batch_geom_t<M_EXACT>(npad_max);
}
}  // namespace

size_t mma_args_bytes() { return sizeof(MmaArgs); }

void mma_fill_args(void* dst, const MmaPlan& p, const Tables& tb, const Function& F,
                   const float* x, float* out, int N, int mode, int npad_max) {
  const bool tf32 = mode == CUROB_PRECISION_TF32X3;
  const BatchGeom g = batch_geom(mode, npad_max);
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
  a.xt = 0;
  a.nA = a.nB = g.nstage;
  a.a_bytes = tf32 ? MC<M_TF32>::kParts * MC<M_TF32>::kPart
                   : MC<M_EXACT>::kParts * MC<M_EXACT>::kPart;
  a.b_bytes = g.stage_bytes - a.a_bytes;
  a.nlist = F.ncomp;
  for (int i = 0; i < kMaxComponents; ++i) a.list[i] = i;
  a.gout = nullptr;
  a.d2out = nullptr;
  a.zbuf = nullptr;
  a.tabt = 0;
  a.rowpm = nullptr;
  a.ntx = a.pm_ld = 0;
  if (tf32) set_acc_regions<M_TF32>(a, npad_of(F.max_n));
  else set_acc_regions<M_EXACT>(a, npad_of(F.max_n));
  memcpy(dst, &a, sizeof(a));
}

cudaError_t launch_mma_batch(const void* d_args, const int2* d_work, int nwork, int* d_counter,
                             int grid, cudaStream_t st, int mode, int npad_max) {
  const BatchGeom g = batch_geom(mode, npad_max);
  const auto kern = mode == CUROB_PRECISION_TF32X3 ? mma_batch_kernel<M_TF32>
                                                   : mma_batch_kernel<M_EXACT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)g.smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, g.smem, st>>>(reinterpret_cast<const MmaArgs*>(d_args), d_work, nwork,
                                       d_counter, g.nstage, g.stage_bytes);
  return cudaGetLastError();
}

int mma_max_block() { return kMaxNpad; }

cudaError_t launch_wait_selftest(int* status, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(status);
  return cudaGetLastError();
}

namespace {
// One launch of the tensor-core kernel at precision `mode` over the
// components `list` (all of F's when nullptr).
cudaError_t launch_any(int mode, const MmaPlan& p, const Tables& tb, const Function& F,
                       const float* x, int N, float* out, cudaStream_t st, const int* list,
                       int nlist, double* gout, double* d2out, float* zbuf,
                       XtView xv = XtView()) {
  switch (mode) {
    case CUROB_PRECISION_TF32X3:
      return launch_mode<M_TF32>(p, tb, F, x, N, out, st, list, nlist, gout, d2out, zbuf, xv);
    case CUROB_PRECISION_BF16X3:
      return launch_mode<M_BF16>(p, tb, F, x, N, out, st, list, nlist, gout, d2out, zbuf, xv);
    case CUROB_PRECISION_EXACT:
      return launch_mode<M_EXACT>(p, tb, F, x, N, out, st, list, nlist, gout, d2out, zbuf, xv);
    case CUROB_PRECISION_FP16X3:
      return launch_mode<M_F16>(p, tb, F, x, N, out, st, list, nlist, gout, d2out, zbuf, xv);
    default: return cudaErrorInvalidValue;
  }
}

struct SplitPlan {
  int ngroups = 0, mode[2] = {-1, -1}, list[2][kMaxComponents], nlist[2] = {0, 0};
  uint32_t xmask = 0;      // members the finish kernel evaluates from x^T
  bool direct = false;     // one launch straight to f: no scratch, no finish kernel
  long long rows = 0;      // candidates per slice
  size_t per_row = 0;      // scratch bytes per candidate
};

// Groups F's components by precision (cmode[c]) in component order.  With
// x^T at hand (with_xt), an unrotated member whose blocks' kinds keep a
// single sum needs no contraction: the finish kernel evaluates it from x^T.
SplitPlan split_plan(const Function& F, const int* cmode, int N, bool with_xt) {
  SplitPlan sp;
  for (int c = 0; c < F.ncomp; ++c) {
    if (with_xt && (F.xcand >> c & 1)) {
      sp.xmask |= 1u << c;
      continue;
    }
    const int g = (sp.ngroups == 0 || sp.mode[0] == cmode[c]) ? 0 : 1;
    if (g + 1 > sp.ngroups) sp.ngroups = g + 1;
    sp.mode[g] = cmode[c];
    sp.list[g][sp.nlist[g]++] = c;
  }
  sp.direct = sp.ngroups == 1 && F.hcols == 0 && sp.xmask == 0;
  sp.per_row = sizeof(float) * (size_t)F.hcols + 2 * sizeof(double) * kMaxComponents;
  long long rows = (long long)(kScratchCap / sp.per_row) / kTileM * kTileM;
  sp.rows = std::min<long long>(std::max<long long>(rows, kTileM), std::max(N, 1));
  return sp;
}

// Evaluates F with component c at precision cmode[c] (at most two distinct
// precisions).  Unless one launch can write f itself, every group writes its
// components' G_c, ||x - o_c||^2 and heavy-kind z into a stream-ordered
// scratch and finish_kernel closes the heavy kinds and composes.
cudaError_t launch_split(const MmaPlan& p, const Tables& tb, const Function& F, const int* cmode,
                         const float* x, int N, float* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  SplitPlan sp = split_plan(F, cmode, N, true);
  const int D = tb.D;
  // Each slice of x is first transposed (x^T, D rows of ld candidates), so
  // that the producers fetch a K stage's variables as TMA row gathers; the
  // copy shares the stream-ordered scratch.  Without room for it the
  // producers gather from x itself.
  const int ld = xt_ld((int)sp.rows);
  bool use_xt = (ld + 31) / 32 <= 65535 && (N + kTileM - 1) / kTileM >= 1;
  const size_t scratch = sp.direct ? 0 : sp.per_row * (size_t)sp.rows;
  const size_t off_xt = (scratch + 255) / 256 * 256;
  void* buf = nullptr;
  cudaError_t e = cudaErrorMemoryAllocation;
  auto alloc = [&](size_t bytes) {
    e = p.pool ? cudaMallocFromPoolAsync(&buf, bytes, p.pool, st) : cudaMallocAsync(&buf, bytes, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      buf = nullptr;
    }
  };
  // Scaled-mode members (EXACT, FP16X3) need each row's max_j |x_j - o_j|
  // before their first stage; the transpose forms it in partials of 64
  // variables while it reads x, instead of the producers reading the rows
  // once more.
  bool scaled = false;
  for (int gi = 0; gi < sp.ngroups; ++gi)
    scaled |= sp.mode[gi] == CUROB_PRECISION_EXACT || sp.mode[gi] == CUROB_PRECISION_FP16X3;
  const int ntx = (D + 63) / 64;
  const size_t off_pm = off_xt + ((size_t)D * ld * sizeof(float) + 255) / 256 * 256;
  const size_t pm_bytes = scaled ? (size_t)F.ncomp * ntx * ld * sizeof(float) : 0;
  if (use_xt) alloc(off_pm + pm_bytes);
  if (!buf) {
    use_xt = false;
    sp = split_plan(F, cmode, N, false);  // every member through the contraction
    if (sp.direct)
      return launch_any(sp.mode[0], p, tb, F, x, N, out, st, nullptr, 0, nullptr, nullptr, nullptr);
    alloc(scratch);
    if (!buf) {
      if (sp.ngroups == 1)  // no room: the epilogue evaluates the heavy kinds itself
        return launch_any(sp.mode[0], p, tb, F, x, N, out, st, nullptr, 0, nullptr, nullptr,
                          nullptr);
      return e;
    }
  }
  e = cudaSuccess;
  float* xtp = use_xt ? reinterpret_cast<float*>(static_cast<char*>(buf) + off_xt) : nullptr;
  for (long long r0 = 0; r0 < N && e == cudaSuccess; r0 += sp.rows) {
    const int n = (int)std::min<long long>(sp.rows, N - r0);
    const float* xs = x + (size_t)r0 * D;
    XtView xv;
    CUtensorMap map;
    if (use_xt) {
      RowMaxJob job;
      float* pm = reinterpret_cast<float*>(static_cast<char*>(buf) + off_pm);
      const bool with_pm = scaled && transpose_vec(xs, D, ld);
      if (with_pm)
        for (int gi = 0; gi < sp.ngroups; ++gi) {
          if (sp.mode[gi] != CUROB_PRECISION_EXACT && sp.mode[gi] != CUROB_PRECISION_FP16X3)
            continue;
          for (int k = 0; k < sp.nlist[gi]; ++k) {
            const int c = sp.list[gi][k];
            // component c's vectors start at (F.comp0 + c) D in the instance
            job.o[job.nc] = p.onat + (size_t)(F.comp0 + c) * D;
            job.pm[job.nc] = pm + (size_t)c * ntx * ld;
            ++job.nc;
          }
        }
      e = launch_transpose_x(xs, n, D, xtp, ld, st, job);
      if (e == cudaSuccess &&
          encode_2d(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, xtp, (uint64_t)n, (uint64_t)D,
                    (uint64_t)ld * sizeof(float), kTileM, 1, CU_TENSOR_MAP_SWIZZLE_NONE)) {
        xv.xt = xtp;
        xv.map = &map;
      }
      if (e == cudaSuccess && with_pm) {
        xv.pm = pm;
        xv.ntx = ntx;
        xv.pm_ld = ld;
      }
    }
    if (sp.direct) {
      if (e == cudaSuccess)
        e = launch_any(sp.mode[0], p, tb, F, xs, n, out + r0, st, nullptr, 0, nullptr, nullptr,
                       nullptr, xv);
      continue;
    }
    double* g = static_cast<double*>(buf);
    double* d2 = g + (size_t)kMaxComponents * n;
    float* z = F.hcols > 0 ? reinterpret_cast<float*>(d2 + (size_t)kMaxComponents * n) : nullptr;
    for (int gi = 0; gi < sp.ngroups && e == cudaSuccess; ++gi)
      e = launch_any(sp.mode[gi], p, tb, F, xs, n, out + r0, st, sp.list[gi], sp.nlist[gi], g,
                     d2, z, xv);
    if (e == cudaSuccess) {
      finish_kernel<<<(unsigned)((n + kFinX - 1) / kFinX), dim3(kFinX, kFinSlices), 0, st>>>(
          tb, F, z, g, d2, n, out + r0, xtp, (long long)ld, p.ohi, p.olo,
          use_xt ? sp.xmask : 0u);
      e = cudaGetLastError();
    }
  }
  cudaFreeAsync(buf, st);
  return e;
}

void component_modes(const Function& F, int mode, int* cmode) {
  for (int c = 0; c < F.ncomp; ++c)
    cmode[c] = mode != CUROB_PRECISION_MIXED
                   ? mode
                   : ((F.sens_mask >> c & 1) ? CUROB_PRECISION_EXACT : CUROB_PRECISION_TF32X3);
}
}  // namespace

int mma_launch_count(const Function& F, int mode, int N) {
  if (N <= 0) return 0;
  int cmode[kMaxComponents];
  component_modes(F, mode, cmode);
  const SplitPlan sp = split_plan(F, cmode, N, true);
  const long long slices = (N + sp.rows - 1) / sp.rows;
  // per slice: the transpose of x, one launch per precision group, and the
  // finish kernel unless one launch writes f itself
  return (int)(slices * (1 + sp.ngroups + (sp.direct ? 0 : 1)));
}

cudaError_t launch_mma_fused(const MmaPlan& p, const Tables& tb, const Function& F, int mode,
                             const float* x, int N, float* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  return launch_any(mode, p, tb, F, x, N, out, st, nullptr, 0, nullptr, nullptr, nullptr);
}

cudaError_t launch_mma_mixed(const MmaPlan& p, const Tables& tb, const Function& F,
                             const float* x, int N, float* out, cudaStream_t st) {
  int cmode[kMaxComponents];
  component_modes(F, CUROB_PRECISION_MIXED, cmode);
  return launch_split(p, tb, F, cmode, x, N, out, st);
}

cudaError_t launch_mma(const MmaPlan& p, const Tables& tb, const Function& F, int mode,
                       const float* x, int N, float* out, cudaStream_t st) {
  if (mode != CUROB_PRECISION_TF32X3 && mode != CUROB_PRECISION_BF16X3 &&
      mode != CUROB_PRECISION_EXACT && mode != CUROB_PRECISION_FP16X3)
    return cudaErrorInvalidValue;
  int cmode[kMaxComponents];
  component_modes(F, mode, cmode);
  return launch_split(p, tb, F, cmode, x, N, out, st);
}

}  // namespace curob

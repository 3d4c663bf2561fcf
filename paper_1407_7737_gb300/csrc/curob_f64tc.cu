// curob_f64tc.cu -- tensor-core evaluator of curob_evaluate (FP64 in/out).
//
// The block rotation z_b = R_b y_b of the General Setup, with y = s (x - o)
// in FP64, as an error-free split product on the BF16 tensor cores (the
// splitting of matrix products of Ozaki, Ogita, Oishi and Rump, with BF16
// integer slices):
//   * each candidate's y over a block and each row of R_b are scaled by a
//     power of two (sigma_m >= max_j |y_mj|, tau_i >= max_j |R_ij|) and
//     rounded to an integer V of 56 bits, |V| <= 2^55 (a rounding of at most
//     2^-56 of the scale), which is cut into seven balanced base-256 digits
//     d_1 .. d_7, |d_a| <= 128.  Digits are exact in BF16; digit a is stored
//     pre-scaled by 2^-8(a-1), so that every product d_a r_b lands with its
//     weight 2^-8(a+b-2);
//   * the products of weight class k = a + b - 2 <= 6 (28 of the 49) are
//     accumulated on the tensor cores in FP32: classes 0..4 each in their own
//     accumulator, classes 5 and 6 together in a sixth.  Over K chunks of at
//     most 192 columns every partial sum of classes 0..4 is an integer
//     multiple of 2^-8k below 2^24 of it (at most 5 products of magnitude
//     <= 2^14 per column), so the FP32 accumulation is exact whatever the
//     tensor core's rounding; the epilogue converts each class to an integer
//     and adds it into an int64 per output;
//   * the sixth accumulator carries classes 5 and 6 (weight <= 2^-40 of the
//     leading one) to the end; its FP32 rounding lies far below an FP64 ulp
//     of z.  The dropped classes (k >= 7) weigh <= 2^-56.
// z = (W 2^16 + round(T 2^48)) 2^(e_m + t_i - 62) is then rounded once to
// FP64 from the exact 128-bit integer, and c is added as the FP64 path does.
//
// Three launches per slice of candidates:
//   f64_prep_kernel    one thread per candidate and block: y, sigma, the
//                      digit image of the candidates' tile (the exact shared-
//                      memory layout of the MMA's A operand), ||x - o||^2 of
//                      the block; unrotated blocks write z = y + c directly;
//   f64_mma_kernel     persistent, one CTA per SM over the units (tile of 128
//                      candidates, chunk of <= 80 output columns of a block):
//                      warp 0 loads the A and B digit images of each K step
//                      with bulk copies, warp 1 issues the 28 MMAs per step,
//                      warps 2..9 drain the exact classes after every K chunk
//                      and write z;
//   f64_finish_kernel  the FP64 terms of every variable (the expressions of
//                      the FP64 path), the sums of each basic function, its
//                      closing map and the composition (Sec. 6).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "curob_f64tc.hpp"
#include "curob_tc.cuh"

namespace curob {
namespace {

using namespace tc;

constexpr int kDigits = 7;             // base-256 digits per operand
constexpr int kExactClasses = 5;       // classes 0..4 accumulated exactly
constexpr int kKChunkSteps = 12;       // K steps (of 16) per exact accumulation: 192 columns
constexpr int kTile = 128;             // candidates per tile (MMA M)
constexpr int kASlice = kTile * 32;    // bytes of one digit slice of a tile's K step
constexpr int kABytes = kDigits * kASlice;  // 28672: A operand of one K step
constexpr int kBMaxBytes = kDigits * kF64Nw * 32;
constexpr int kStageStride = (kABytes + kBMaxBytes + 1023) / 1024 * 1024;
constexpr int kStages = 4;
constexpr int kMmaThreads = 320;       // loader, MMA issuer, 8 epilogue warps
constexpr int kTmemCols = 512;
constexpr size_t kF64ScratchCap = size_t(2) << 30;  // scratch bytes per slice of candidates

// Balanced base-256 digits of V = round(v 2^(55 - e)) for |v| < 2^e:
// V = sum_a d_a 2^(8 (7 - a)), |d_a| <= 128; out[a-1] = d_a 2^(-8 (a-1)) as
// FP32 (exact).  Zero and subnormal v (far below 2^(e - 55) wherever e comes
// from the row's maximum) give V = 0.
__device__ __forceinline__ void f64_digits(double v, int e, float* out) {
  const long long b = __double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7ff);
  long long V = 0;
  if (be != 0) {
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);  // |v| = m 2^(be - 1075)
    const int s = be - 1020 - e;                                // V = m 2^s, s <= 2
    if (s >= 0) {
      V = m << s;
    } else if (s > -62) {
      V = (m + (1LL << (-s - 1))) >> (-s);  // nearest, ties up
    }
    if (b < 0) V = -V;
  }
  float scale = 0x1p-48f;  // digit 7 weighs 2^-48 of digit 1
#pragma unroll
  for (int a = kDigits - 1; a >= 1; --a) {
    const long long d = ((V + 128) & 255) - 128;
    V = (V - d) >> 8;
    out[a] = (float)(int)d * scale;
    scale *= 256.f;
  }
  out[0] = (float)(int)V;  // |V| <= 128 here
}

// Exponent e with max < 2^e for a non-negative finite max (e = -1022 for 0).
__device__ __forceinline__ int f64_scale_exp(double mx) {
  const int be = (int)((__double_as_longlong(mx) >> 52) & 0x7ff);
  return be == 0 ? -1022 : be - 1022;
}

__device__ __forceinline__ uint32_t bf16_bits(float f) {  // exact for the digits
  return __float_as_uint(f) >> 16;
}

// ----------------------------------------------------------- R digit images
struct RImgJob {
  long long r_off;   // block in the FP64 rotation pool (row-major n x n)
  long long img_off; // its chunks' images in the digit pool (bytes)
  int rexp_off;      // its rows' exponents
  int n;
};

// Row exponents t_i: max_j |R_ij| < 2^t_i.
__global__ void f64_rexp_kernel(const RImgJob* jobs, const double* R, int* rexp) {
  const RImgJob J = jobs[blockIdx.x];
  for (int i = threadIdx.x; i < J.n; i += blockDim.x) {
    const double* Ri = R + J.r_off + (long long)i * J.n;
    double mx = 0.0;
    for (int j = 0; j < J.n; ++j) mx = fmax(mx, fabs(Ri[j]));
    rexp[J.rexp_off + i] = f64_scale_exp(mx);
  }
}

// Digit images of one block: chunk c (rows [80c, 80c + nwc)), K step t:
// seven slices of nwc rows x 32 bytes (32-byte swizzle), slice b holding
// r_b 2^(-8(b-1)) of R_ij / 2^t_i; rows and columns past n are zero.
// blockIdx.y = K step, threads over the rows of all chunks.
__global__ void f64_rimg_kernel(const RImgJob* jobs, const double* R, const int* rexp,
                                uint8_t* img) {
  const RImgJob J = jobs[blockIdx.x];
  const int t = blockIdx.y;
  const int nk = (J.n + 15) / 16;
  if (t >= nk) return;
  const int nch = (J.n + kF64Nw - 1) / kF64Nw;
  for (int row = threadIdx.x; row < nch * kF64Nw; row += blockDim.x) {
    const int c = row / kF64Nw, rr = row - c * kF64Nw;
    const int nvalid = min(kF64Nw, J.n - c * kF64Nw);
    const int nwc = (nvalid + 15) / 16 * 16;
    if (rr >= nwc) continue;
    // the chunks before c are full (80 rows): nk K steps of 80 x 224 bytes each
    const long long cbase = (long long)c * nk * kF64Nw * kDigits * 32;
    uint8_t* st = img + J.img_off + cbase + (long long)t * nwc * kDigits * 32;
    const int i = c * kF64Nw + rr;
    const int e = i < J.n ? rexp[J.rexp_off + i] : 0;
    uint32_t w[kDigits][8];
#pragma unroll
    for (int a = 0; a < kDigits; ++a)
#pragma unroll
      for (int q = 0; q < 8; ++q) w[a][q] = 0;
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int j = t * 16 + jj;
      const double v = (i < J.n && j < J.n) ? R[J.r_off + (long long)i * J.n + j] : 0.0;
      float d[kDigits];
      f64_digits(v, e, d);
#pragma unroll
      for (int a = 0; a < kDigits; ++a) w[a][jj >> 1] |= bf16_bits(d[a]) << (16 * (jj & 1));
    }
#pragma unroll
    for (int a = 0; a < kDigits; ++a) {
      uint8_t* sl = st + (long long)a * nwc * 32;
      *reinterpret_cast<uint4*>(sl + swz32((uint32_t)rr, 0)) =
          make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
      *reinterpret_cast<uint4*>(sl + swz32((uint32_t)rr, 16)) =
          make_uint4(w[a][4], w[a][5], w[a][6], w[a][7]);
    }
  }
}

// ------------------------------------------------------------ prep kernel
// Marks a candidate whose y over a block holds a non-finite value: its z
// becomes NaN (non-finite inputs give NaN outputs).
constexpr int kExpNonFinite = 0x7fffffff;

// A block takes 32 candidates (the lanes; a quarter of a 128-row tile) and
// one segment of F (blockIdx.y); warp g of 4 takes every fourth variable of
// the block (pass 1, unrotated blocks) and every fourth K step (pass 2), so
// each candidate has four threads.  Rotated blocks: pass 1 finds max_j |y_j|
// through max_j |x_j - o_j| (the rounded product s d is monotone in |d|),
// pass 2 writes the seven digit slices of each K step of 16 variables in the
// 32-byte-swizzled K-major layout of the MMA's A operand (a warp writes 32
// consecutive rows).  Unrotated blocks write z = s (x - o) + c straight into
// the z scratch ([component][variable][N], candidates inner).  Both leave the
// block's share of ||x - o||^2 (compositions) in d2p[segment][N], the four
// warps' parts added in warp order.
constexpr int kPrepRows = 32;
constexpr int kPrepWarps = 4;

__global__ void __launch_bounds__(kPrepRows * kPrepWarps) f64_prep_kernel(
    Tables tb, Function F, const int2* __restrict__ seginfo, const double* __restrict__ x, int N,
    int KS, uint8_t* __restrict__ aimg, int* __restrict__ sexp, double* __restrict__ z,
    double* __restrict__ d2p) {
  __shared__ long long mxs[kPrepWarps][kPrepRows];
  __shared__ double d2s[kPrepWarps][kPrepRows];
  const int seg0 = tb.comp[F.comp0].seg0;
  const int si = blockIdx.y;
  const Segment sg = tb.seg[seg0 + si];
  const int c = sg.comp - F.comp0;
  const Component C = tb.comp[sg.comp];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int tile = blockIdx.x / (kTile / kPrepRows);
  const int m = (blockIdx.x % (kTile / kPrepRows)) * kPrepRows + lane;  // row in the tile
  const long long row = (long long)tile * kTile + m;
  const bool valid = row < N;
  const int D = tb.D;
  const int* __restrict__ S = tb.S + C.base + sg.zoff;
  const double* __restrict__ op = tb.operm + C.base + sg.zoff;
  const double* __restrict__ xr = x + (valid ? row : 0) * (long long)D;
  const int n = sg.n;
  const int2 info = seginfo[seg0 + si];
  const bool want_d2 = F.composition != 0;
  double d2 = 0.0;
  if (info.x < 0) {
    if (valid) {
      double* zc = z + ((long long)c * D + sg.zoff) * N + row;
      for (int j = g; j < n; j += kPrepWarps) {
        const double d = xr[S[j]] - op[j];
        if (want_d2) d2 += d * d;
        const double y = sg.scale * d;
        zc[(long long)j * N] = y + sg.offset;
      }
    }
  } else {
    long long mb = 0;  // bits of max_j |x_j - o_j| (non-negative doubles order as integers)
    if (valid)
      for (int j = g; j < n; j += kPrepWarps) {
        const double d = xr[S[j]] - op[j];
        if (want_d2) d2 += d * d;
        mb = max(mb, __double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFLL);
      }
    mxs[g][lane] = mb;
    __syncthreads();
    mb = max(max(mxs[0][lane], mxs[1][lane]), max(mxs[2][lane], mxs[3][lane]));
    const bool finite = mb < 0x7FF0000000000000LL;
    const int e = finite ? f64_scale_exp(fabs(sg.scale) * __longlong_as_double(mb)) : 0;
    if (valid && g == 0) sexp[(long long)info.x * N + row] = finite ? e : kExpNonFinite;
    const int nk = (n + 15) / 16;
    uint8_t* at = aimg + ((long long)tile * KS + info.y) * kABytes;
    const bool live = valid && finite;
    for (int t = g; t < nk; t += kPrepWarps) {
      uint32_t w[kDigits][8];
#pragma unroll
      for (int a = 0; a < kDigits; ++a)
#pragma unroll
        for (int q = 0; q < 8; ++q) w[a][q] = 0;
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = t * 16 + jj;
        double y = 0.0;
        if (live && j < n) y = sg.scale * (xr[S[j]] - op[j]);
        float dg[kDigits];
        f64_digits(y, e, dg);
#pragma unroll
        for (int a = 0; a < kDigits; ++a) w[a][jj >> 1] |= bf16_bits(dg[a]) << (16 * (jj & 1));
      }
      uint8_t* stp = at + (long long)t * kABytes;
#pragma unroll
      for (int a = 0; a < kDigits; ++a) {
        uint8_t* sl = stp + a * kASlice;
        *reinterpret_cast<uint4*>(sl + swz32((uint32_t)m, 0)) =
            make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
        *reinterpret_cast<uint4*>(sl + swz32((uint32_t)m, 16)) =
            make_uint4(w[a][4], w[a][5], w[a][6], w[a][7]);
      }
    }
  }
  if (want_d2) {
    d2s[g][lane] = d2;
    __syncthreads();
    if (valid && g == 0)
      d2p[(long long)si * N + row] = ((d2s[0][lane] + d2s[1][lane]) + d2s[2][lane]) + d2s[3][lane];
  }
}

// ------------------------------------------------------------- MMA kernel
// 32 lanes x 8 consecutive FP32 columns (no wait: see tmem_wait_ld).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The double nearest (ties to even) to X 2^sc for a 128-bit integer X: the
// magnitude is cut to its top 63 bits with the bits below OR-ed into the
// last one (ten guard bits and a sticky bit decide the rounding to 53 bits
// as the full value would), converted once, and scaled by its exponent.
__device__ __forceinline__ double i128_to_double(__int128 X, int sc) {
  if (X == 0) return 0.0;
  const bool neg = X < 0;
  const unsigned __int128 M = neg ? (unsigned __int128)(-X) : (unsigned __int128)X;
  const unsigned long long hi = (unsigned long long)(M >> 64), lo = (unsigned long long)M;
  const int nb = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  unsigned long long v = lo;
  int sh = 0;
  if (nb > 63) {
    sh = nb - 63;
    const unsigned __int128 rest = M & ((((unsigned __int128)1) << sh) - 1);
    v = (unsigned long long)(M >> sh) | (rest != 0 ? 1ull : 0ull);
  }
  double d = __ull2double_rn(v);
  const int adj = sh + sc;
  const long long bits = __double_as_longlong(d);
  const int be = (int)(bits >> 52) + adj;
  d = (be > 0 && be < 2047) ? __longlong_as_double(bits + ((long long)adj << 52)) : ldexp(d, adj);
  return neg ? -d : d;
}

struct MmaArgs64 {
  const uint8_t* aimg;      // y digit images: [tile][K step of the function][7][128][32 B]
  const uint8_t* bimg;      // R digit pool
  const int* sexp;          // [rotated slot][N] exponents of the candidates' scales
  const int* rexp;          // row exponent pool
  const F64Chunk* chunks;   // the function's chunks
  double* z;                // [component][D][N]
  int* status;
  int nchunks, KS, N, D;
  int nunits;               // tiles x chunks
};

// Persistent: CTA b takes the units (tile, chunk) b, b + gridDim.x, ... in
// order (unit u = tile * nchunks + chunk, so the CTAs working at one time
// share their tiles' A images in L2).  The operand ring and the accumulator
// hand-off run on across units: the loader fetches the next unit's K steps
// while the epilogue drains the last one.  TMEM columns: class k (0..4) at
// k * 80, classes 5 and 6 at 400.  Every wait is bounded: past ~2 s it
// raises DEV_TIMEOUT, the roles stop, copies and MMAs in flight are waited
// for (again bounded) and TMEM is freed before the CTA exits.
__global__ void __launch_bounds__(kMmaThreads, 1) f64_mma_kernel(const MmaArgs64 a) {
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageStride);
  uint64_t* full = bars;                 // [kStages]
  uint64_t* empty = bars + kStages;      // [kStages]
  uint64_t* tfull = bars + 2 * kStages;  // accumulators of a K chunk complete
  uint64_t* tempty = tfull + 1;          // epilogue has read them
  uint64_t* done = tfull + 2;            // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 8);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // loader
      uint32_t g = 0;  // K steps issued
      bool ok = true;
      for (int unit = blockIdx.x; unit < a.nunits && ok; unit += gridDim.x) {
        const int tile = unit / a.nchunks;
        const F64Chunk ch = a.chunks[unit - tile * a.nchunks];
        const uint8_t* A = a.aimg + ((long long)tile * a.KS + ch.ksg) * kABytes;
        const uint8_t* B = a.bimg + ch.b_off;
        const uint32_t bbytes = (uint32_t)ch.nwc * kDigits * 32;
        for (int t = 0; t < ch.nk; ++t, ++g) {
          const int s = g % kStages;
          if (g >= kStages && !mbar_wait(&empty[s], ((g / kStages) - 1) & 1, abort_flag, a.status)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * kStageStride;
          mbar_arrive_expect_tx(&full[s], kABytes + bbytes);
          bulk_g2s(st, A + (long long)t * kABytes, kABytes, &full[s]);
          bulk_g2s(st + kABytes, B + (long long)t * bbytes, bbytes, &full[s]);
        }
      }
      // no copy may still be landing when the CTA exits
      const unsigned long long deadline = globaltimer() + kTimeoutNs;
      for (uint32_t v = g > (uint32_t)kStages ? g - kStages : 0; v < g; ++v)
        mbar_drain(&full[v % kStages], (v / kStages) & 1u, deadline);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t g = 0, c = 0;  // K steps consumed, K chunks handed to the epilogue
      bool ok = true;
      for (int unit = blockIdx.x; unit < a.nunits && ok; unit += gridDim.x) {
        const int tile = unit / a.nchunks;
        const F64Chunk ch = a.chunks[unit - tile * a.nchunks];
        const uint32_t idesc = idesc_make(1u, 128u, (uint32_t)ch.nwc);
        for (int t = 0; t < ch.nk; ++t, ++g) {
          const int s = g % kStages;
          const bool first = (t % kKChunkSteps) == 0;
          // the previous K chunk (of this unit or the last) has been drained
          if (first && c > 0 && !mbar_wait(tempty, (c - 1) & 1u, abort_flag, a.status)) {
            ok = false;
            break;
          }
          if (!mbar_wait(&full[s], (g / kStages) & 1u, abort_flag, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t abase = smem_u32(smem + s * kStageStride);
          const uint32_t bbase = abase + kABytes;
#pragma unroll
          for (int k = 0; k < kDigits; ++k) {  // classes 0..6: digit pairs (ai, k - ai)
            const uint32_t dcol =
                tmem + (uint32_t)(k < kExactClasses ? k : kExactClasses) * kF64Nw;
#pragma unroll
            for (int ai = 0; ai <= k; ++ai) {
              const int bi = k - ai;
              const uint64_t ad = sdesc_sw32(abase + ai * kASlice);
              const uint64_t bd = sdesc_sw32(bbase + bi * ch.nwc * 32);
              // the first product of an exact class in a K chunk, and of the
              // tail in the unit, overwrites its accumulator
              const bool fresh = (k < kExactClasses) ? (first && ai == 0)
                                                     : (t == 0 && k == kExactClasses && ai == 0);
              tc_mma<false>(dcol, ad, bd, idesc, fresh ? 0u : 1u);
            }
          }
          tc_commit(&empty[s]);
          if ((t % kKChunkSteps) == kKChunkSteps - 1 || t == ch.nk - 1) {
            tc_commit(tfull);
            ++c;
          }
        }
      }
      tc_commit(done);
      mbar_drain(done, 0, globaltimer() + kTimeoutNs);
    }
  } else {  // epilogue: warps 2..9
    const int ew = warp - 2;
    const int quarter = warp & 3;  // a warp reads TMEM lanes 32 (warp % 4) .. + 31
    const int half = ew >> 2;      // columns [40 half, 40 half + 40)
    const int m = quarter * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t c = 0;  // K chunks drained
    bool ok = true;
    for (int unit = blockIdx.x; unit < a.nunits && ok; unit += gridDim.x) {
      const int tile = unit / a.nchunks;
      const F64Chunk ch = a.chunks[unit - tile * a.nchunks];
      const int nkc = (ch.nk + kKChunkSteps - 1) / kKChunkSteps;
      const long long row = (long long)tile * kTile + m;
      const bool valid = row < a.N;
      const int em = valid ? a.sexp[(long long)ch.sslot * a.N + row] : 0;
      long long W[40];
      float T[40];  // classes 5 and 6, read at the unit's last K chunk
#pragma unroll
      for (int i = 0; i < 40; ++i) W[i] = 0;
      for (int kc = 0; kc < nkc; ++kc, ++c) {
        const bool got = mbar_wait(tfull, c & 1u, abort_flag, a.status);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool last = kc == nkc - 1;
#pragma unroll
        for (int gq = 0; gq < 5; ++gq) {
          const int col0 = half * 40 + gq * 8;
          if (col0 < ch.nwc) {  // warp-uniform; nwc is a multiple of 16
            uint32_t r[kExactClasses + 1][8];
#pragma unroll
            for (int k = 0; k < kExactClasses; ++k) tmem_ld8(taddr + k * kF64Nw + col0, r[k]);
            if (last) tmem_ld8(taddr + kExactClasses * kF64Nw + col0, r[kExactClasses]);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              // class k holds C_k 2^-8k, |C_k| <= 2^24: exact integers once scaled
              long long w = (long long)__float2int_rn(__uint_as_float(r[0][i])) << 32;
              w += (long long)__float2int_rn(__uint_as_float(r[1][i]) * 256.f) << 24;
              w += (long long)__float2int_rn(__uint_as_float(r[2][i]) * 65536.f) << 16;
              w += (long long)__float2int_rn(__uint_as_float(r[3][i]) * 16777216.f) << 8;
              w += (long long)__float2int_rn(__uint_as_float(r[4][i]) * 4294967296.f);
              W[gq * 8 + i] += w;
              if (last) T[gq * 8 + i] = __uint_as_float(r[kExactClasses][i]);
            }
          }
        }
        // TMEM is read: hand it back, so the next K chunk (or unit) runs
        // under the conversions below
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty);
        if (last && valid) {
#pragma unroll
          for (int gq = 0; gq < 5; ++gq) {
            const int col0 = half * 40 + gq * 8;
            if (col0 < ch.nwc) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int col = col0 + i;
                if (col < ch.nvalid) {
                  const long long tf = __float2ll_rn(T[gq * 8 + i] * 281474976710656.f);
                  const __int128 X = ((__int128)W[gq * 8 + i] << 16) + tf;
                  double zv;
                  if (em == kExpNonFinite) {
                    zv = __longlong_as_double(0x7FF8000000000000LL);
                  } else {
                    zv = i128_to_double(X, em + a.rexp[ch.rexp_off + col] - 62);
                    if (ch.offset != 0.0) zv = zv + ch.offset;
                  }
                  a.z[((long long)ch.comp * a.D + ch.zcol + col) * a.N + row] = zv;
                }
              }
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_free(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------- finish kernel
// A block takes 32 candidates (the lanes) and walks every block of every
// component in chunks of 32 variables.  The eight warps form a chunk's terms
// -- term_f64, the FP64 path's expression of each variable's term -- four
// variables each, into a shared-memory tile (two tiles alternate); warp 0
// then adds them in index order into its candidate's running sums, closes
// each basic function at its last block (finalize) and, for a composition,
// mixes the members with ||x - o_i||^2 summed block after block (Sec. 6).
// The sums therefore round like a sequential evaluation of the formula, as
// on the FP64 CUDA-core path: near an optimum, where f is a small difference
// of large sums (Modified Schwefel: 418.9829 D - sum g1), the order of the
// additions decides the last digits.
constexpr int kFinCols = 32;  // variables per chunk
constexpr int kFinWarps = 8;
constexpr int kFinArr = 3;    // term arrays of a kind (f64_num_terms <= 3)
constexpr int kFinTile = kFinArr * kFinCols * 32;  // doubles of one tile
constexpr size_t kFinSmem = 2 * kFinTile * sizeof(double);  // 48 KB

// Katsuura's inner sum (Sec. 4.11) sum_{j=1}^{32} |2^j z - [2^j z]| / 2^j,
// exact: with z = +-m 2^q (m the 53-bit significand), 2^j |z| has t = -(q + j)
// fraction bits, its distance to the nearest integer is min(r, 2^t - r) 2^-t
// (r its low t bits of m), and divided by 2^j every term is an integer
// multiple of 2^q.  The sum is therefore S 2^q with S < 2^58, formed in
// integer arithmetic and rounded once -- the same value as the series added
// term by term, up to the additions' roundings (a few ulps).
__device__ __forceinline__ double katsuura_inner_exact(double z) {
  const long long b = __double_as_longlong(z);
  const int be = (int)((b >> 52) & 0x7ff);
  if (be == 0x7ff) return z - z;          // non-finite: NaN, as the series gives
  if (be == 0) return 32.0 * fabs(z);     // zero or subnormal: every term is |z|
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const int q = be - 1075;
  unsigned long long S = 0;
#pragma unroll 4
  for (int j = 1; j <= 32; ++j) {
    const int t = -(q + j);
    if (t <= 0) break;                    // 2^j |z| and every later one are integers
    if (t >= 54) {
      S += (unsigned long long)m;         // 2^j |z| < 1/2
    } else {
      const unsigned long long one = 1ull << t;
      const unsigned long long r = (unsigned long long)m & (one - 1ull);
      S += r < one - r ? r : one - r;
    }
  }
  return ldexp((double)S, q);
}

// Weierstrass inner sum of the FP64 path (Sec. 4.2), the value of
// weierstrass_inner(double): sum_{k=0}^{20} 2^-k cos(x_k) with
// x_k = fl(c_k w), c_k = fl(P 3^k), P = 2 fl(pi) and w = fl(z + 1/2) -- the
// rounded arguments of the printed expression -- but with each cosine from an
// exact reduction instead of the library's:
//   c_k w = x_k + d_k exactly (d_k by one fma), and P 3^k = c_k + e_k exactly,
//   P = 2 pi - eta, so x_k = 2 pi 3^k w - (eta 3^k + e_k) w - d_k: modulo 2 pi
//   it is 2 pi F_k - G_k w - d_k, F_k = frac(3^k w) formed exactly from w's
//   significand in 128-bit integer arithmetic, G_k = eta 3^k + e_k (a
//   constant, |G_k w + d_k| < 2e-5).  F_k is centred on the nearest quarter
//   turn Q/4, leaving |theta| <= pi/4 + 2e-5 (theta to ~1e-17 in double), and
//   cos(x_k) = +-cos(theta) or +-sin(theta) by Q from Taylor series to
//   theta^16 / theta^17 (truncation below 2e-17).
constexpr double kEta = 2.4492935982947064e-16;  // 2 pi - 2 fl(pi), to double precision
struct WeierK {
  double c, g;  // c_k = fl(P 3^k); G_k = eta 3^k + e_k
};
__constant__ WeierK c_weier[21];

// cos(theta) (odd = 0) or sin(theta) (odd = 1), |theta| <= ~0.8, without a
// branch (the parity differs from lane to lane): cos = 1 + u Pc(u) and
// sin = theta + theta u Ps(u), u = theta^2, Pc and Ps the Taylor series to
// theta^16 and theta^17 (coefficients 1/n! by correctly rounded division),
// one Horner chain on per-lane selected coefficients.
__device__ __forceinline__ double cos_or_sin_small(double th, bool odd) {
  const double u = th * th;
  double p = odd ? 1.0 / 355687428096000.0 : 1.0 / 20922789888000.0;  // 1/17!, 1/16!
  p = fma(p, u, odd ? -1.0 / 1307674368000.0 : -1.0 / 87178291200.0);  // 1/15!, 1/14!
  p = fma(p, u, odd ? 1.0 / 6227020800.0 : 1.0 / 479001600.0);         // 1/13!, 1/12!
  p = fma(p, u, odd ? -1.0 / 39916800.0 : -1.0 / 3628800.0);           // 1/11!, 1/10!
  p = fma(p, u, odd ? 1.0 / 362880.0 : 1.0 / 40320.0);                 // 1/9!, 1/8!
  p = fma(p, u, odd ? -1.0 / 5040.0 : -1.0 / 720.0);                   // 1/7!, 1/6!
  p = fma(p, u, odd ? 1.0 / 120.0 : 1.0 / 24.0);                       // 1/5!, 1/4!
  p = fma(p, u, odd ? -1.0 / 6.0 : -0.5);                              // 1/3!, 1/2!
  const double base = odd ? th : 1.0;
  return fma(p * u, base, base);
}

// -v for flip, v otherwise (the sign bit, no arithmetic).
__device__ __forceinline__ double flip_sign(double v, bool flip) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)flip << 63));
}

__device__ __forceinline__ double weierstrass_inner_exact(double z) {
  const double w = z + 0.5;
  const long long b = __double_as_longlong(w);
  const int be = (int)((b >> 52) & 0x7ff);
  const int s = 1075 - be;  // fraction bits of w's significand
  // |w| in [2^-9, 2^50): s in [3, 62], where 3^k m mod 2^s is the low s bits
  // of the 64-bit product; other w (far outside the box) take the series
  if (be == 0 || s < 3 || s > 62) return weierstrass_inner(z);
  const unsigned long long m = (unsigned long long)((b & 0xFFFFFFFFFFFFFLL) | (1LL << 52));
  const bool neg = b < 0;
  const unsigned long long mask = (1ull << s) - 1ull;
  const unsigned long long half_q = 1ull << (s - 3);   // an eighth turn
  const unsigned long long quart = (1ull << (s - 2)) - 1ull;
  const double scale = __longlong_as_double((long long)(1023 - s) << 52);  // 2^-s
  double acc = 0.0, ak = 1.0;
  unsigned long long p3 = 1;  // 3^k
#pragma unroll 3
  for (int k = 0; k <= 20; ++k) {
    const WeierK K = c_weier[k];
    const double x = K.c * w;                            // the printed expression's argument
    const double corr = fma(K.g, w, fma(K.c, w, -x));    // G_k w + d_k
    // F = frac(3^k |w|) (the low s bits of 3^k m), centred on the nearest quarter turn
    const unsigned long long u = ((m * p3) & mask) + half_q;
    int Q = (int)(u >> (s - 2)) & 3;
    // frac(-v) = -frac(v)
    const double F = flip_sign((double)((long long)(u & quart) - (long long)half_q) * scale, neg);
    if (neg) Q = (4 - Q) & 3;
    // theta = 2 pi F - corr, 2 pi = P + eta
    const double hi = (2.0 * kPi) * F;
    const double th = hi + (fma(kEta, F, fma(2.0 * kPi, F, -hi)) - corr);
    const double v = cos_or_sin_small(th, Q & 1);       // cos(theta + Q pi/2), up to sign
    acc += ak * flip_sign(v, Q == 1 || Q == 2);
    ak *= 0.5;
    p3 *= 3ull;
  }
  return acc;
}

// The terms of one warp's columns of a chunk, with the kind fixed at compile
// time (a kind known only at run time inside the loop lets the compiler
// form other kinds' transcendentals for every variable).
template <int KIND>
__device__ __forceinline__ void fin64_terms(double* T, const double* zb, long long N, int j0,
                                            int ncol, int warp, int lane, int gpos, double gnd,
                                            const double* aux, double kat_e) {
  constexpr int kPer = kFinCols / kFinWarps;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int jc = warp * kPer + q;
    if (jc < ncol) {
      const int j = j0 + jc;
      if constexpr (kind_has_pairs(KIND)) {
        T[jc * 32 + lane] =
            (gpos + j > 0)
                ? pair_term<double>(KIND, zb[(long long)(j - 1) * N], zb[(long long)j * N])
                : 0.0;
      } else if constexpr (KIND == K_WEIERSTRASS) {
        T[jc * 32 + lane] = weierstrass_inner_exact(zb[(long long)j * N]);
      } else if constexpr (KIND == K_KATSUURA) {
        // log of the factor 1 + (i+1) s_i: the function's product of the
        // factors' powers is formed as exp(e * sum log) at its last block
        const double zj = zb[(long long)j * N];
        T[jc * 32 + lane] = log(1.0 + (double)(gpos + j + 1) * katsuura_inner_exact(zj));
      } else {
        const double zj = zb[(long long)j * N];
        const double av = aux ? aux[j] : 0.0;
#pragma unroll
        for (int q2 = 0; q2 < f64_num_terms(KIND); ++q2)
          T[(q2 * kFinCols + jc) * 32 + lane] = term_f64(KIND, q2, zj, 0.0, gpos + j, gnd, av, kat_e);
      }
    }
  }
}

__device__ __forceinline__ void fin64_dispatch(int kind, double* T, const double* zb, long long N,
                                               int j0, int ncol, int warp, int lane, int gpos,
                                               double gnd, const double* aux, double kat_e) {
  switch (kind) {
#define CUROB_FIN64_CASE(K) \
  case K: fin64_terms<K>(T, zb, N, j0, ncol, warp, lane, gpos, gnd, aux, kat_e); break;
    CUROB_FIN64_CASE(K_SPHERE) CUROB_FIN64_CASE(K_ELLIPSOID) CUROB_FIN64_CASE(K_ELLIPTIC)
    CUROB_FIN64_CASE(K_DISCUS) CUROB_FIN64_CASE(K_CIGAR) CUROB_FIN64_CASE(K_POWERS)
    CUROB_FIN64_CASE(K_SHARPV) CUROB_FIN64_CASE(K_STEP) CUROB_FIN64_CASE(K_WEIERSTRASS)
    CUROB_FIN64_CASE(K_GRIEWANK) CUROB_FIN64_CASE(K_RASTRIGIN) CUROB_FIN64_CASE(K_SCHAFFER7)
    CUROB_FIN64_CASE(K_EGR) CUROB_FIN64_CASE(K_ROSENBROCK) CUROB_FIN64_CASE(K_SCHWEFEL)
    CUROB_FIN64_CASE(K_KATSUURA) CUROB_FIN64_CASE(K_LUNACEK) CUROB_FIN64_CASE(K_ACKLEY)
    CUROB_FIN64_CASE(K_HAPPYCAT) CUROB_FIN64_CASE(K_HGBAT) CUROB_FIN64_CASE(K_SCHAFFER6)
#undef CUROB_FIN64_CASE
    default: break;
  }
}

__global__ void __launch_bounds__(kFinWarps * 32, 2) f64_finish_kernel(Tables tb, Function F,
                                                                    const double* __restrict__ z,
                                                                    const double* __restrict__ d2p,
                                                                    int N, double* __restrict__ out) {
  extern __shared__ double fin_tiles[];  // [2][kFinArr][kFinCols][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * 32 + lane;
  const bool valid = i < N;
  const long long ic = valid ? i : 0;  // rows past N read row 0 and write nothing
  const int D = tb.D;
  const int fseg0 = tb.comp[F.comp0].seg0;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, p = 1.0;  // warp 0: the open function's sums
  double G[kMaxComponents];
  int buf = 0;
  for (int c = 0; c < F.ncomp; ++c) {
    const Component C = tb.comp[F.comp0 + c];
    const double* zc = z + (long long)c * D * N + ic;
    double gsum = 0.0;
    for (int si = 0; si < C.nseg; ++si) {
      const Segment sg = tb.seg[C.seg0 + si];
      const int n = sg.n, kind = sg.kind;
      const bool pairs = kind_has_pairs(kind);
      const bool first_special = (kind == K_DISCUS || kind == K_CIGAR || kind == K_SHARPV);
      const double gnd = (double)sg.gn;
      const double kat_e = (kind == K_KATSUURA) ? 10.0 / pow(gnd, 1.2) : 0.0;
      const double* aux = sg.aux_off >= 0 ? tb.aux + sg.aux_off : nullptr;
      const int na = pairs ? 1 : f64_num_terms(kind);
      const double* zb = zc + (long long)sg.zoff * N;
      for (int j0 = 0; j0 < n; j0 += kFinCols) {
        double* T = fin_tiles + buf * kFinTile;
        const int ncol = min(kFinCols, n - j0);
        // the terms of columns j0 + 4 warp .. + 3; a pair kind's column j
        // holds the pair (z_{j-1}, z_j) of function positions >= 1 (z_{-1}
        // is the previous block's last variable: a function's blocks are
        // consecutive in z)
        fin64_dispatch(kind, T, zb, N, j0, ncol, warp, lane, sg.gpos, gnd, aux, kat_e);
        __syncthreads();
        if (warp == 0) {
          if (j0 == 0 && sg.gfirst) {
            a0 = a1 = a2 = 0.0;
            p = 1.0;
          }
          if (pairs) {
            for (int jc = 0; jc < ncol; ++jc)
              if (sg.gpos + j0 + jc > 0) a0 += T[jc * 32 + lane];
          } else {
            for (int q2 = 0; q2 < na; ++q2) {
              const double* t = T + q2 * kFinCols * 32 + lane;
              if (f64_term_is_product(kind, q2) && kind != K_KATSUURA) {
                for (int jc = 0; jc < ncol; ++jc) p *= t[jc * 32];
              } else if (q2 == 0) {
                for (int jc = 0; jc < ncol; ++jc) {
                  if (first_special && sg.gpos + j0 + jc == 0) a1 = t[jc * 32];  // z_1 apart
                  else a0 += t[jc * 32];
                }
              } else if (q2 == 1) {
                for (int jc = 0; jc < ncol; ++jc) a1 += t[jc * 32];
              } else {
                for (int jc = 0; jc < ncol; ++jc) a2 += t[jc * 32];
              }
            }
          }
          if (j0 + kFinCols >= n && sg.glast) {
            if (kind_is_cyclic(kind)) {  // (z_gn, z_1) closes the cycle
              const double* zf = zc + (long long)(sg.zoff - sg.gpos) * N;
              a0 += pair_term<double>(kind, zf[(long long)(sg.gn - 1) * N], zf[0]);
            }
            if (kind == K_KATSUURA) {  // prod_i (1 + (i+1) s_i)^e = exp(e sum log)
              p = exp(kat_e * a0);
              a0 = 0.0;
            }
            gsum += finalize(kind, a0, a1, a2, p, sg.gn);
          }
        }
        buf ^= 1;
      }
    }
    G[c] = gsum;
  }
  if (warp != 0 || !valid) return;
  double f;
  if (F.composition) {
    double d2v[kMaxComponents];
    for (int c = 0; c < F.ncomp; ++c) {
      const Component C = tb.comp[F.comp0 + c];
      double dd = 0.0;
      for (int si = 0; si < C.nseg; ++si) dd += d2p[(long long)(C.seg0 - fseg0 + si) * N + i];
      d2v[c] = dd;
    }
    f = compose(tb.comp + F.comp0, F.ncomp, G, d2v, D);
  } else {
    f = G[0];
  }
  out[i] = f + kFopt;
}

size_t mma_smem_bytes() { return (size_t)kStages * kStageStride + 256 + 1024; }

// Bytes of one slice's scratch at ns candidates, each part 256-byte aligned.
struct SliceLayout {
  size_t a, z, sexp, d2p, total;
};
SliceLayout slice_layout(const F64Plan& p, const Function& F, int fid, int D, long long ns) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  SliceLayout L;
  const long long ntiles = (ns + kTile - 1) / kTile;
  L.a = 0;
  L.z = up((size_t)ntiles * p.ks_total[fid] * kABytes);
  L.sexp = L.z + up((size_t)F.ncomp * D * ns * sizeof(double));
  L.d2p = L.sexp + up((size_t)std::max(p.nrot[fid], 1) * ns * sizeof(int));
  L.total = L.d2p + up((size_t)(F.composition ? F.nseg : 1) * ns * sizeof(double));
  return L;
}

// Candidates per slice: whole tiles, scratch within kF64ScratchCap.
long long slice_size(const F64Plan& p, const Function& F, int fid, int D, int N) {
  long long ns = ((long long)N + kTile - 1) / kTile * kTile;
  while (ns > kTile && slice_layout(p, F, fid, D, ns).total > kF64ScratchCap)
    ns = std::max<long long>(kTile, (ns / 2 + kTile - 1) / kTile * kTile);
  return std::min<long long>(ns, N);
}

}  // namespace

// ------------------------------------------------------------- host side
namespace {

// Digit images and row exponents of the given segments (rotated ones).
curob_status build_rimg(const F64Plan& p, const std::vector<Segment>& segs,
                        const std::vector<int>& ids, const Tables& tb) {
  std::vector<RImgJob> jobs;
  int maxk = 1;
  for (int s : ids) {
    if (p.seg_img[s] < 0) continue;
    const Segment& sg = segs[s];
    jobs.push_back(RImgJob{sg.r_off, p.seg_img[s], (int)p.seg_rexp[s], sg.n});
    maxk = std::max(maxk, (sg.n + 15) / 16);
  }
  if (jobs.empty()) return CUROB_OK;
  RImgJob* d = nullptr;
  if (cudaMalloc(&d, sizeof(RImgJob) * jobs.size()) != cudaSuccess) return CUROB_ERR_OUT_OF_MEMORY;
  cudaError_t e = cudaMemcpy(d, jobs.data(), sizeof(RImgJob) * jobs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    f64_rexp_kernel<<<(unsigned)jobs.size(), 128>>>(d, tb.R, p.rexp);
    f64_rimg_kernel<<<dim3((unsigned)jobs.size(), (unsigned)maxk), 128>>>(d, tb.R, p.rexp,
                                                                          p.rimg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d);
  return e == cudaSuccess ? CUROB_OK : CUROB_ERR_CUDA;
}

}  // namespace

void f64_release(F64Plan& p) {
  cudaFree(p.rimg);
  cudaFree(p.rexp);
  cudaFree(p.chunks);
  cudaFree(p.seginfo);
  p.rimg = nullptr;
  p.rexp = nullptr;
  p.chunks = nullptr;
  p.seginfo = nullptr;
  p.seg_img.clear();
  p.seg_rexp.clear();
  p.ready = false;
}

curob_status f64_prepare(F64Plan& p, const std::vector<Segment>& segs,
                         const std::vector<Component>& comps, const Function* funcs,
                         const bool* func_ok, const Tables& tb) {
  f64_release(p);
  int dev = 0, cc_major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
  const size_t nseg = segs.size();
  p.seg_img.assign(nseg, -1);
  p.seg_rexp.assign(nseg, 0);
  std::vector<int2> info(nseg, make_int2(-1, 0));
  long long img = 0, rx = 0;
  for (size_t s = 0; s < nseg; ++s) {
    const Segment& sg = segs[s];
    if (sg.identity) continue;
    const int nk = (sg.n + 15) / 16;
    const int nch = (sg.n + kF64Nw - 1) / kF64Nw;
    const int last = ((sg.n - (nch - 1) * kF64Nw) + 15) / 16 * 16;
    p.seg_img[s] = img;
    img += (long long)nk * ((nch - 1) * kF64Nw + last) * kDigits * 32;
    p.seg_rexp[s] = rx;
    rx += sg.n;
  }
  std::vector<F64Chunk> chunks;
  for (int f = 0; f < kNumFunctions; ++f) {
    p.chunk0[f] = (int)chunks.size();
    p.nchunk[f] = p.nrot[f] = p.ks_total[f] = 0;
    if (!func_ok[f]) continue;
    const Function& F = funcs[f];
    for (int c = 0; c < F.ncomp; ++c) {
      const Component& C = comps[F.comp0 + c];
      for (int k = 0; k < C.nseg; ++k) {
        const int s = C.seg0 + k;
        const Segment& sg = segs[s];
        if (sg.identity) continue;
        const int nk = (sg.n + 15) / 16;
        const int slot = p.nrot[f]++;
        info[s] = make_int2(slot, p.ks_total[f]);
        const int nch = (sg.n + kF64Nw - 1) / kF64Nw;
        for (int q = 0; q < nch; ++q) {
          F64Chunk ch;
          memset(&ch, 0, sizeof(ch));
          ch.nvalid = std::min(kF64Nw, sg.n - q * kF64Nw);
          ch.nwc = (ch.nvalid + 15) / 16 * 16;
          ch.b_off = p.seg_img[s] + (long long)q * nk * kF64Nw * kDigits * 32;
          ch.comp = c;
          ch.zcol = sg.zoff + q * kF64Nw;
          ch.nk = nk;
          ch.ksg = p.ks_total[f];
          ch.sslot = slot;
          ch.rexp_off = (int)(p.seg_rexp[s] + q * kF64Nw);
          ch.offset = sg.offset;
          chunks.push_back(ch);
        }
        p.ks_total[f] += nk;
      }
    }
    p.nchunk[f] = (int)chunks.size() - p.chunk0[f];
  }
  const size_t cb = sizeof(F64Chunk) * std::max<size_t>(chunks.size(), 1);
  if (cudaMalloc(&p.rimg, std::max<long long>(img, 16)) != cudaSuccess ||
      cudaMalloc(&p.rexp, sizeof(int) * std::max<long long>(rx, 1)) != cudaSuccess ||
      cudaMalloc(&p.chunks, cb) != cudaSuccess ||
      cudaMalloc(&p.seginfo, sizeof(int2) * std::max<size_t>(nseg, 1)) != cudaSuccess) {
    f64_release(p);
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  if ((!chunks.empty() && cudaMemcpy(p.chunks, chunks.data(), sizeof(F64Chunk) * chunks.size(),
                                     cudaMemcpyHostToDevice) != cudaSuccess) ||
      (nseg && cudaMemcpy(p.seginfo, info.data(), sizeof(int2) * nseg, cudaMemcpyHostToDevice) !=
                   cudaSuccess)) {
    f64_release(p);
    return CUROB_ERR_CUDA;
  }
  std::vector<int> all(nseg);
  for (size_t s = 0; s < nseg; ++s) all[s] = (int)s;
  cudaDeviceGetAttribute(&p.nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cc_major == 10) {  // the digit images feed tcgen05: built where it runs
    const curob_status rc = build_rimg(p, segs, all, tb);
    if (rc != CUROB_OK) {
      f64_release(p);
      return rc;
    }
    WeierK wk[21];
    double bk = 1.0;
    for (int k = 0; k <= 20; ++k, bk *= 3.0) {
      wk[k].c = (2.0 * kPi) * bk;                           // as the FP64 path rounds it
      const double e = std::fma(2.0 * kPi, bk, -wk[k].c);    // P 3^k - c_k, exact
      wk[k].g = std::fma(kEta, bk, e);
    }
    if (cudaMemcpyToSymbol(c_weier, wk, sizeof(wk)) != cudaSuccess ||
        cudaFuncSetAttribute(f64_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mma_smem_bytes()) != cudaSuccess) {
      f64_release(p);
      return CUROB_ERR_CUDA;
    }
    p.ready = true;
  }
  return CUROB_OK;
}

curob_status f64_refresh(F64Plan& p, const std::vector<Segment>& segs, const std::vector<int>& ids,
                         const Tables& tb) {
  if (!p.ready) return CUROB_OK;
  return build_rimg(p, segs, ids, tb);
}

bool f64_supports(const F64Plan& p, int fid) {
  return p.ready && fid >= 0 && fid < kNumFunctions;
}

int f64_launch_count(const F64Plan& p, const Function& F, int fid, int D, int N) {
  if (N <= 0) return 0;
  const long long ns = slice_size(p, F, fid, D, N);
  const long long slices = (N + ns - 1) / ns;
  return (int)(slices * (p.nchunk[fid] > 0 ? 3 : 2));
}

cudaError_t launch_f64tc(const F64Plan& p, cudaMemPool_t pool, const Tables& tb,
                         const Function& F, int fid, const double* x, int N, double* out,
                         cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const int D = tb.D;
  const long long ns_max = slice_size(p, F, fid, D, N);
  for (long long s0 = 0; s0 < N; s0 += ns_max) {
    const int ns = (int)std::min<long long>(ns_max, N - s0);
    const SliceLayout L = slice_layout(p, F, fid, D, ns);
    void* buf = nullptr;
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&buf, L.total, pool, st)
                         : cudaMallocAsync(&buf, L.total, st);
    if (e != cudaSuccess) return e;
    uint8_t* b = static_cast<uint8_t*>(buf);
    uint8_t* aimg = b + L.a;
    double* zs = reinterpret_cast<double*>(b + L.z);
    int* sexp = reinterpret_cast<int*>(b + L.sexp);
    double* d2p = reinterpret_cast<double*>(b + L.d2p);
    const double* xs = x + s0 * D;
    const unsigned ntiles = (unsigned)((ns + kTile - 1) / kTile);
    f64_prep_kernel<<<dim3(ntiles * (kTile / kPrepRows), (unsigned)F.nseg), kPrepRows * kPrepWarps,
                      0, st>>>(
        tb, F, p.seginfo, xs, ns, p.ks_total[fid], aimg, sexp, zs, d2p);
    e = cudaGetLastError();
    if (e == cudaSuccess && p.nchunk[fid] > 0) {
      MmaArgs64 a;
      a.aimg = aimg;
      a.bimg = p.rimg;
      a.sexp = sexp;
      a.rexp = p.rexp;
      a.chunks = p.chunks + p.chunk0[fid];
      a.z = zs;
      a.status = tb.status;
      a.nchunks = p.nchunk[fid];
      a.KS = p.ks_total[fid];
      a.N = ns;
      a.D = D;
      a.nunits = (int)ntiles * p.nchunk[fid];
      const unsigned grid = (unsigned)std::min(a.nunits, std::max(p.nsm, 1));
      f64_mma_kernel<<<grid, kMmaThreads, mma_smem_bytes(), st>>>(a);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      f64_finish_kernel<<<(unsigned)((ns + 31) / 32), kFinWarps * 32, kFinSmem, st>>>(
          tb, F, zs, d2p, ns, out + s0);
      e = cudaGetLastError();
    }
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace curob

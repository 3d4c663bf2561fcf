// curob_small.cuh -- evaluators for small populations (the paper's own
// timing setting, Sec. 2: a few tens of candidates per call).
//
// At N ~ 50 a call is latency-bound: the batched kernels give each candidate
// a share of a CTA and walk every component and block of the function in
// sequence between CTA-wide barriers.  Here one CTA evaluates one candidate
// and one warp one block (segment) of it: every block of every member of a
// composition is worked on at the same time.  A warp
//   1. gathers y = s (x - o) at its block's variables S_b (lanes over the
//      block's variables) and sums that block's share of ||x - o||^2,
//   2. forms z_b = R_b y + c, lane i taking outputs i, i + 32, ... with the
//      dot product in index order,
//   3. forms the block's per-variable terms (General Setup, Sec. 3-5);
// then, after one CTA barrier, one thread per component walks its blocks in
// order, adds the terms into the running sums of the open basic function and
// closes each function at its last block, and thread 0 composes the members
// (Sec. 6, Eq. composition, Eq. weight).
//
// FP64 (curob_evaluate): the arithmetic of the batched FP64 kernel, term for
// term -- one fma per term of each dot product in index order, each term
// with the formula's expression, the sums in index order, the squared
// distance summed per block across the lanes and then block after block --
// so both give the same bits.  Weierstrass's inner series runs its 21
// cosines across the lanes and is added in k order per variable.
// FP32 (curob_evaluatef): y and R as FP32 hi/lo pairs and a compensated dot
// product (TwoProd + TwoSum: z within about one FP32 rounding), FP32 terms
// summed per lane and then across the lanes in FP64, as the batched CUDA-core
// FP32 kernel.
#pragma once

#include "curob_internal.hpp"

namespace curob {

constexpr int kSmallMaxN = 128;     // widest block the small kernels take
constexpr int kSmallMaxWarps = 16;  // segments of a function (15 at most in the suite)
constexpr int kWeierK = 21;         // Weierstrass terms k = 0..20 (Sec. 4.2)
constexpr int kWeierChunk = 32;     // variables per pass of the spread series

__device__ inline double small_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double small_warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Running state of the open basic function of a component (one thread).
struct SmallAccum {
  double a0 = 0, a1 = 0, a2 = 0, p = 1;
  double zfirst = 0, zlast = 0;
  double gsum = 0;
};

// Shared-memory layout of one CTA (offsets in bytes, all 8-byte aligned).
struct SmallSmem {
  size_t x, z, t, y, yl, p, d2, w, total;
};

// What a small-population launch reads of the instance, passed by value: the
// function's segments and components sit in the kernel's parameter space,
// so no warp waits on global memory for its block's descriptor.
struct SmallArgs {
  Tables tb;
  Function F;
  int seg_base;                     // the function's first segment in the table
  Segment seg[kSmallMaxWarps];      // its segments, in table order
  Component comp[kMaxComponents];   // its components
};

// T: element type of x; D the dimension.  FP64: z, y (ncomp x D doubles),
// three term arrays per component, the spread Weierstrass series.  FP32: u =
// z before its offset, y as hi/lo words (ncomp x D floats each), four FP64
// partial sums per segment.  Both: per-segment ||x - o||^2 shares.
template <typename T>
__host__ __device__ inline SmallSmem small_smem_layout(const Function& F, int D) {
  SmallSmem L;
  const size_t zd = (size_t)F.ncomp * D;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 15) / 16 * 16;
    return o;
  };
  L.x = take(sizeof(T) * D);
  L.z = take(sizeof(T) * zd);
  L.y = take(sizeof(T) * zd);
  L.yl = take(sizeof(T) == 4 ? sizeof(float) * zd : 0);
  L.t = take(sizeof(T) == 8 ? sizeof(double) * 3 * zd : 0);
  L.p = take(sizeof(T) == 4 ? sizeof(double) * 4 * F.nseg : 0);
  L.d2 = take(sizeof(double) * F.nseg);
  L.w = take(sizeof(T) == 8 ? sizeof(double) * kWeierK * kWeierChunk * F.nweier : 0);
  L.total = off;
  return L;
}

#ifdef CUROB_SMALL_F64
// Steps 1-3 of one block in FP64 (warp-wide).
__device__ inline void small_block_f64(const Tables& tb, const Segment& sg, const Component& C,
                                       const double* xs, double* Zc, double* Yc, double* Tc,
                                       double* W, double* d2p_out) {
  const int lane = threadIdx.x & 31;
  const int D = tb.D;
  const int n = sg.n;
  const int* __restrict__ S = tb.S + C.base;
  const double* __restrict__ op = tb.operm + C.base;
  // 1. y = s (x - o)
  double d2p = 0.0;
  for (int j = lane; j < n; j += 32) {
    const double ov = op[sg.zoff + j];
    const double d = xs[S[sg.zoff + j]] - ov;
    Yc[sg.zoff + j] = sg.scale * d;
    d2p += d * d;
  }
  d2p = small_warp_sum(d2p);
  if (lane == 0) *d2p_out = d2p;
  __syncwarp();
  // 2. z = R_b y + c
  if (sg.identity) {
    for (int i = lane; i < n; i += 32) Zc[sg.zoff + i] = Yc[sg.zoff + i] + sg.offset;
  } else {
    const double* __restrict__ Rt = tb.Rt + sg.r_off;  // column-major: (i, j) at j n + i
    const double* Yb = Yc + sg.zoff;
    for (int i = lane; i < n; i += 32) {
      double acc = 0.0;
#pragma unroll 8
      for (int j = 0; j < n; ++j) acc = fma(Rt[(long long)j * n + i], Yb[j], acc);
      Zc[sg.zoff + i] = acc + sg.offset;
    }
  }
  __syncwarp();
  // 3. terms
  const int kind = sg.kind;
  const double* Zb = Zc + sg.zoff;
  if (kind == K_WEIERSTRASS) {
    // a^k cos(2 pi b^k (z + 1/2)) for (variable, k) pairs across the lanes,
    // then each variable's series added in k order, as weierstrass_inner
    for (int i0 = 0; i0 < n; i0 += kWeierChunk) {
      const int m = min(kWeierChunk, n - i0);
      for (int q = lane; q < m * kWeierK; q += 32) {
        const int i = q / kWeierK, k = q - i * kWeierK;
        const double ak = ldexp(1.0, -k);
        double bk = 1.0;
        for (int r = 0; r < k; ++r) bk *= 3.0;  // 3^k, exact
        W[q] = ak * cos(2.0 * kPi * bk * (Zb[i0 + i] + 0.5));
      }
      __syncwarp();
      if (lane < m) {
        double s = 0.0;
        for (int k = 0; k < kWeierK; ++k) s += W[lane * kWeierK + k];
        Tc[sg.zoff + i0 + lane] = s;
      }
      __syncwarp();
    }
    return;
  }
  const bool pairs = kind_has_pairs(kind);
  const double gnd = (double)sg.gn;
  const double kat_e = (kind == K_KATSUURA) ? 10.0 / pow(gnd, 1.2) : 0.0;
  const double* aux = tb.aux + (sg.aux_off >= 0 ? sg.aux_off : 0);
  const bool has_aux = sg.aux_off >= 0;
  const int nterm = pairs ? n - 1 : n;
  const int na = f64_num_terms(kind);
  for (int a = 0; a < na; ++a)
    for (int i = lane; i < nterm; i += 32)
      Tc[(size_t)a * D + sg.zoff + i] =
          term_f64(kind, a, Zb[i], pairs ? Zb[i + 1] : 0.0, sg.gpos + i, gnd,
                   has_aux ? aux[i] : 0.0, kat_e);
}

// The component's sums in index order over its blocks (one thread), as the
// batched FP64 kernel: returns G_c; *d2 = ||x - o_c||^2 block after block.
__device__ inline double small_close_f64(const SmallArgs& a, const Component& C,
                                         const double* Zc, const double* Tc, const double* d2s,
                                         double* d2) {
  const int D = a.tb.D;
  const int seg_base = a.seg_base;
  SmallAccum st;
  double dd = 0.0;
  for (int si = 0; si < C.nseg; ++si) {
    const Segment& sg = a.seg[C.seg0 - seg_base + si];
    dd += d2s[C.seg0 - seg_base + si];
    const int n = sg.n, kind = sg.kind;
    const bool pairs = kind_has_pairs(kind);
    const bool first_special = (kind == K_DISCUS || kind == K_CIGAR || kind == K_SHARPV);
    const int nterm = pairs ? n - 1 : n;
    const double* Zb = Zc + sg.zoff;
    if (sg.gfirst) {
      st.a0 = st.a1 = st.a2 = 0.0;
      st.p = 1.0;
      st.zfirst = Zb[0];
    } else if (pairs) {
      st.a0 += pair_term<double>(kind, st.zlast, Zb[0]);
    }
    const int na = f64_num_terms(kind);
    for (int a = 0; a < na; ++a) {
      const double* t = Tc + (size_t)a * D + sg.zoff;
      if (f64_term_is_product(kind, a)) {
        double pr = st.p;
        for (int i = 0; i < nterm; ++i) pr *= t[i];
        st.p = pr;
      } else {
        double acc = (a == 0) ? st.a0 : (a == 1 ? st.a1 : st.a2);
        int i0 = 0;
        if (first_special && sg.gpos == 0) {  // z_1 enters separately
          st.a1 = t[0];
          i0 = 1;
        }
        for (int i = i0; i < nterm; ++i) acc += t[i];
        if (a == 0) st.a0 = acc; else if (a == 1) st.a1 = acc; else st.a2 = acc;
      }
    }
    st.zlast = Zb[n - 1];
    if (sg.glast) {
      if (kind_is_cyclic(kind)) st.a0 += pair_term<double>(kind, st.zlast, st.zfirst);
      st.gsum += finalize(kind, st.a0, st.a1, st.a2, st.p, sg.gn);
    }
  }
  *d2 = dd;
  return st.gsum;
}
#endif  // CUROB_SMALL_F64

#ifdef CUROB_SMALL_F32
// Steps 1-3 of one block on the FP32 path (warp-wide); the block's four FP64
// partial sums go to P[0..3].
__device__ inline void small_block_f32(const Tables& tb, const Segment& sg, const Component& C,
                                       const float* xs, float* Uc, float* Yh, float* Yl,
                                       double* P, double* d2p_out) {
  const int lane = threadIdx.x & 31;
  const int n = sg.n;
  const int* __restrict__ S = tb.S + C.base;
  const double* __restrict__ op = tb.operm + C.base;
  // 1. y = s (x - o) in FP64, kept as an FP32 hi/lo pair
  double d2p = 0.0;
  for (int j = lane; j < n; j += 32) {
    const double ov = op[sg.zoff + j];
    const double d = (double)xs[S[sg.zoff + j]] - ov;
    const double y = sg.scale * d;
    const float yh = (float)y;
    Yh[sg.zoff + j] = yh;
    Yl[sg.zoff + j] = (float)(y - (double)yh);
    d2p += d * d;
  }
  d2p = small_warp_sum(d2p);
  if (lane == 0) *d2p_out = d2p;
  __syncwarp();
  // 2. u = R_b y, compensated
  const float* yh = Yh + sg.zoff;
  const float* yl = Yl + sg.zoff;
  float* Ub = Uc + sg.zoff;
  if (sg.identity) {
    for (int i = lane; i < n; i += 32) Ub[i] = yh[i] + yl[i];
  } else {
    const float* __restrict__ Rh = tb.R32t + sg.r_off;   // column-major: (i, j) at j n + i
    const float* __restrict__ Rl = tb.R32lot + sg.r_off;
    for (int i = lane; i < n; i += 32) {
      float s = 0.f, c = 0.f;
#pragma unroll 8
      for (int j = 0; j < n; ++j) {
        const float a = Rh[(long long)j * n + i], b = yh[j];
        const float p = a * b;
        const float e = fmaf(a, b, -p);                // a*b = p + e exactly
        const float t = s + p;
        const float bb = t - s;
        const float err = (s - (t - bb)) + (p - bb);   // s + p = t + err exactly
        s = t;
        c += err + e + fmaf(a, yl[j], Rl[(long long)j * n + i] * b);
      }
      Ub[i] = s + c;
    }
  }
  __syncwarp();
  // 3. terms, summed per lane in FP32 and across the lanes in FP64
  const int kind = sg.kind;
  const bool pairs = kind_has_pairs(kind);
  const float gnT = (float)sg.gn, off = (float)sg.offset;
  const float* aux = tb.aux32 + (sg.aux_off >= 0 ? sg.aux_off : 0);
  const bool has_aux = sg.aux_off >= 0;
  Acc<float> a = acc_zero<float>();
  for (int i = lane; i < n; i += 32) {
    const float ui = Ub[i], zi = ui + off;
    elem_term_f32(kind, zi, ui, sg.gpos + i, gnT, has_aux ? aux[i] : 0.f, sg.kat_e, a);
    if (pairs && i + 1 < n) a.a0 += pair_term<float>(kind, zi, Ub[i + 1] + off);
  }
  // FP64 across the lanes only for the sums the kind uses (each FP64 warp
  // instruction costs the same as 32 lanes' worth)
  const double r0 = small_warp_sum((double)a.a0);
  const double r1 = kind_uses_a1(kind) ? small_warp_sum((double)a.a1) : 0.0;
  const double r2 = kind_uses_a2(kind) ? small_warp_sum((double)a.a2) : 0.0;
  const double rp = kind_uses_p(kind) ? small_warp_prod((double)a.p) : 1.0;
  if (lane == 0) {
    P[0] = r0;
    P[1] = r1;
    P[2] = r2;
    P[3] = rp;
  }
}

// The component's blocks in order (one thread), as the batched CUDA-core
// FP32 kernel: returns G_c; *d2 = ||x - o_c||^2 block after block.
__device__ inline double small_close_f32(const SmallArgs& a, const Component& C,
                                         const float* Uc, const double* P, const double* d2s,
                                         double* d2) {
  const int seg_base = a.seg_base;
  SmallAccum st;
  double dd = 0.0;
  for (int si = 0; si < C.nseg; ++si) {
    const Segment& sg = a.seg[C.seg0 - seg_base + si];
    const int g = C.seg0 - seg_base + si;
    dd += d2s[g];
    const int kind = sg.kind;
    const bool pairs = kind_has_pairs(kind);
    const float off = (float)sg.offset;
    const float z0 = Uc[sg.zoff] + off;
    if (sg.gfirst) {
      st.a0 = st.a1 = st.a2 = 0.0;
      st.p = 1.0;
      st.zfirst = (double)z0;
    } else if (pairs) {
      st.a0 += (double)pair_term<float>(kind, (float)st.zlast, z0);
    }
    st.a0 += P[4 * g];
    st.a1 += P[4 * g + 1];
    st.a2 += P[4 * g + 2];
    st.p *= P[4 * g + 3];
    st.zlast = (double)(Uc[sg.zoff + sg.n - 1] + off);
    if (sg.glast) {
      if (kind_is_cyclic(kind))
        st.a0 += (double)pair_term<float>(kind, (float)st.zlast, (float)st.zfirst);
      st.gsum += finalize_f32(kind, st.a0, st.a1, st.a2, st.p, sg.gn);
    }
  }
  *d2 = dd;
  return st.gsum;
}
#endif  // CUROB_SMALL_F32

}  // namespace curob

// curob_simt.cuh -- the CUDA-core evaluators of the cuROB functions.
//
// One CTA owns BM candidates (BM = 32 while the largest block fits: then the
// 32 lanes of a warp are the 32 candidates, so every rotation element R[i][j]
// is one broadcast load shared by the warp).  For each component and each of
// its blocks (segments) the CTA
//   1. gathers y = s (x - o) at the block's variables S_b into shared memory
//      (shift in FP64; a warp reads one candidate's row, lanes walk the
//      sorted index list),
//   2. rotates z_b = R_b y (+ c), one dot product per (candidate, output),
//   3. applies the per-variable transform and reduces,
// and closes each basic function when its last block is done.  A composition
// keeps each member's value and ||x - o_i||^2 and mixes them (Sec. 6,
// Eq. weight) in FP64.
//
// FP64 kernel (curob_evaluate): the dot products take one fma per term in
// index order; the terms of step 3 are computed in parallel and then summed
// by one thread per candidate in index order (products likewise), so the
// value rounds like the sequential statement of the formula.
// FP32 kernel (CUDA-core FP32 path): y and R are carried as FP32 hi/lo pairs
// and the dot product is compensated (TwoProd + TwoSum), which keeps z within
// about one FP32 rounding; step 3 runs warp-parallel with FP64 reductions
// across lanes.
#pragma once

#include "curob_internal.hpp"

namespace curob {

struct CandState {
  double a0, a1, a2, p;   // running sums / product of the open function
  double zfirst, zlast;   // first z of the open function, last z seen
  double gsum;            // sum of closed functions of the current component
  double G[kMaxComponents];
  double d2[kMaxComponents];
};

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kSimtThreads = 256;

__device__ inline void init_state(CandState* st, int BM) {
  for (int m = threadIdx.x; m < BM; m += blockDim.x) {
    CandState& s = st[m];
    s.a0 = s.a1 = s.a2 = 0.0;
    s.p = 1.0;
    s.zfirst = s.zlast = 0.0;
    s.gsum = 0.0;
    for (int c = 0; c < kMaxComponents; ++c) s.G[c] = s.d2[c] = 0.0;
  }
}

template <typename Tout>
__device__ inline void write_out(const Tables& tb, const Function& F, CandState* st, int BM,
                                 long long row0, int N, Tout* out) {
  for (int m = threadIdx.x; m < BM; m += blockDim.x) {
    const long long row = row0 + m;
    if (row >= N) continue;
    double f = F.composition ? compose(tb.comp + F.comp0, F.ncomp, st[m].G, st[m].d2, tb.D)
                             : st[m].G[0];
    out[row] = (Tout)(f + kFopt);
  }
}

// ------------------------------------------------------------------ FP64
#ifdef CUROB_SIMT_F64
__global__ void __launch_bounds__(kSimtThreads)
eval_simt_f64_kernel(Tables tb, Function F, const double* __restrict__ x, int N,
                     double* __restrict__ out, int BM, int ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CandState* st = reinterpret_cast<CandState*>(smem_raw);
  double* Ys = reinterpret_cast<double*>(smem_raw + sizeof(CandState) * BM);
  double* Zs = Ys + (size_t)BM * ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const long long row0 = (long long)blockIdx.x * BM;
  const int D = tb.D;
  init_state(st, BM);
  __syncthreads();

  for (int ci = 0; ci < F.ncomp; ++ci) {
    const Component C = tb.comp[F.comp0 + ci];
    const int* __restrict__ S = tb.S + C.base;
    const double* __restrict__ op = tb.operm + C.base;
    for (int si = 0; si < C.nseg; ++si) {
      const Segment sg = tb.seg[C.seg0 + si];
      const int n = sg.n;
      // 1. y = s (x - o) at the block's variables
      for (int m = warp; m < BM; m += nwarps) {
        const long long row = row0 + m;
        const bool valid = row < N;
        const double* xr = x + (valid ? row : 0) * (long long)D;
        double d2p = 0.0;
        for (int j = lane; j < n; j += 32) {
          const double ov = op[sg.zoff + j];
          const double d = (valid ? xr[S[sg.zoff + j]] : ov) - ov;
          Ys[m * ld + j] = sg.scale * d;
          d2p += d * d;
        }
        if (F.composition) {
          d2p = warp_sum(d2p);
          if (lane == 0) st[m].d2[ci] += d2p;
        }
      }
      __syncthreads();
      // 2. z = R_b y + c
      if (sg.identity) {
        for (int idx = tid; idx < BM * n; idx += blockDim.x) {
          const int m = idx / n, i = idx - m * n;
          Zs[m * ld + i] = Ys[m * ld + i] + sg.offset;
        }
      } else {
        const double* __restrict__ Rb = tb.R + sg.r_off;
        const int per = blockDim.x / BM;
        const int m = tid % BM;
        const double* Ym = Ys + m * ld;
        for (int i = tid / BM; i < n; i += per) {
          const double* Ri = Rb + (long long)i * n;
          double acc = 0.0;
          for (int j = 0; j < n; ++j) acc = fma(Ri[j], Ym[j], acc);
          Zs[m * ld + i] = acc + sg.offset;
        }
      }
      __syncthreads();
      // 3. terms in parallel (into Ys), sums per candidate in index order
      const int kind = sg.kind;
      const bool pairs = kind_has_pairs(kind);
      const bool first_special = (kind == K_DISCUS || kind == K_CIGAR || kind == K_SHARPV);
      const double gnd = (double)sg.gn;
      const double kat_e = (kind == K_KATSUURA) ? 10.0 / pow(gnd, 1.2) : 0.0;
      const double* aux = tb.aux + (sg.aux_off >= 0 ? sg.aux_off : 0);
      const bool has_aux = sg.aux_off >= 0;
      const int nterm = pairs ? n - 1 : n;
      const int na = f64_num_terms(kind);
      for (int a = 0; a < na; ++a) {
        for (int idx = tid; idx < BM * nterm; idx += blockDim.x) {
          const int m = idx / nterm, i = idx - m * nterm;
          const double z = Zs[m * ld + i];
          const double zn = pairs ? Zs[m * ld + i + 1] : 0.0;
          Ys[m * ld + i] = term_f64(kind, a, z, zn, sg.gpos + i, gnd, has_aux ? aux[i] : 0.0, kat_e);
        }
        __syncthreads();
        for (int m = tid; m < BM; m += blockDim.x) {
          CandState& s = st[m];
          const double* t = Ys + m * ld;
          if (a == 0) {
            if (sg.gfirst) {
              s.a0 = s.a1 = s.a2 = 0.0;
              s.p = 1.0;
              s.zfirst = Zs[m * ld];
            } else if (pairs) {
              s.a0 += pair_term<double>(kind, s.zlast, Zs[m * ld]);
            }
          }
          if (f64_term_is_product(kind, a)) {
            double pr = s.p;
            for (int i = 0; i < nterm; ++i) pr *= t[i];
            s.p = pr;
          } else {
            double acc = (a == 0) ? s.a0 : (a == 1 ? s.a1 : s.a2);
            int i0 = 0;
            if (first_special && sg.gpos == 0) {  // z_1 enters separately
              s.a1 = t[0];
              i0 = 1;
            }
            for (int i = i0; i < nterm; ++i) acc += t[i];
            if (a == 0) s.a0 = acc; else if (a == 1) s.a1 = acc; else s.a2 = acc;
          }
        }
        __syncthreads();
      }
      for (int m = tid; m < BM; m += blockDim.x) {
        CandState& s = st[m];
        s.zlast = Zs[m * ld + n - 1];
        if (sg.glast) {
          if (kind_is_cyclic(kind)) s.a0 += pair_term<double>(kind, s.zlast, s.zfirst);
          s.gsum += finalize(kind, s.a0, s.a1, s.a2, s.p, sg.gn);
        }
      }
      __syncthreads();
    }
    for (int m = tid; m < BM; m += blockDim.x) {
      st[m].G[ci] = st[m].gsum;
      st[m].gsum = 0.0;
    }
    __syncthreads();
  }
  write_out(tb, F, st, BM, row0, N, out);
}

#endif  // CUROB_SIMT_F64

// ------------------------------------------------------------------ FP32
#ifdef CUROB_SIMT_F32
__global__ void __launch_bounds__(kSimtThreads)
eval_simt_f32_kernel(Tables tb, Function F, const float* __restrict__ x, int N,
                     float* __restrict__ out, int BM, int ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CandState* st = reinterpret_cast<CandState*>(smem_raw);
  float* Yh = reinterpret_cast<float*>(smem_raw + sizeof(CandState) * BM);
  float* Yl = Yh + (size_t)BM * ld;
  float* Zs = Yl + (size_t)BM * ld;  // z before the offset (u)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const long long row0 = (long long)blockIdx.x * BM;
  const int D = tb.D;
  init_state(st, BM);
  __syncthreads();

  for (int ci = 0; ci < F.ncomp; ++ci) {
    const Component C = tb.comp[F.comp0 + ci];
    const int* __restrict__ S = tb.S + C.base;
    const double* __restrict__ op = tb.operm + C.base;
    for (int si = 0; si < C.nseg; ++si) {
      const Segment sg = tb.seg[C.seg0 + si];
      const int n = sg.n;
      // 1. y = s (x - o) in FP64, kept as an FP32 hi/lo pair
      for (int m = warp; m < BM; m += nwarps) {
        const long long row = row0 + m;
        const bool valid = row < N;
        const float* xr = x + (valid ? row : 0) * (long long)D;
        double d2p = 0.0;
        for (int j = lane; j < n; j += 32) {
          const double ov = op[sg.zoff + j];
          const double d = (valid ? (double)xr[S[sg.zoff + j]] : ov) - ov;
          const double y = sg.scale * d;
          const float yh = (float)y;
          Yh[m * ld + j] = yh;
          Yl[m * ld + j] = (float)(y - (double)yh);
          d2p += d * d;
        }
        if (F.composition) {
          d2p = warp_sum(d2p);
          if (lane == 0) st[m].d2[ci] += d2p;
        }
      }
      __syncthreads();
      // 2. u = R_b y, compensated
      if (sg.identity) {
        for (int idx = tid; idx < BM * n; idx += blockDim.x) {
          const int m = idx / n, i = idx - m * n;
          Zs[m * ld + i] = Yh[m * ld + i] + Yl[m * ld + i];
        }
      } else {
        const float* __restrict__ Rh = tb.R32 + sg.r_off;
        const float* __restrict__ Rl = tb.R32lo + sg.r_off;
        const int per = blockDim.x / BM;
        const int m = tid % BM;
        const float* yh = Yh + m * ld;
        const float* yl = Yl + m * ld;
        for (int i = tid / BM; i < n; i += per) {
          const float* rh = Rh + (long long)i * n;
          const float* rl = Rl + (long long)i * n;
          float s = 0.f, c = 0.f;
          for (int j = 0; j < n; ++j) {
            const float a = rh[j], b = yh[j];
            const float p = a * b;
            const float e = fmaf(a, b, -p);          // a*b = p + e exactly
            const float t = s + p;
            const float bb = t - s;
            const float err = (s - (t - bb)) + (p - bb);  // s + p = t + err exactly
            s = t;
            c += err + e + fmaf(a, yl[j], rl[j] * b);
          }
          Zs[m * ld + i] = s + c;
        }
      }
      __syncthreads();
      // 3. transform + warp reduction (FP64 across lanes)
      const int kind = sg.kind;
      const bool pairs = kind_has_pairs(kind);
      const float gnT = (float)sg.gn, off = (float)sg.offset;
      const float kat_e = sg.kat_e;
      const float* aux = tb.aux32 + (sg.aux_off >= 0 ? sg.aux_off : 0);
      const bool has_aux = sg.aux_off >= 0;
      for (int m = warp; m < BM; m += nwarps) {
        const float* u = Zs + m * ld;
        Acc<float> a = acc_zero<float>();
        for (int i = lane; i < n; i += 32) {
          const float ui = u[i], zi = ui + off;
          elem_term_f32(kind, zi, ui, sg.gpos + i, gnT, has_aux ? aux[i] : 0.f, kat_e, a);
          if (pairs && i + 1 < n) a.a0 += pair_term<float>(kind, zi, u[i + 1] + off);
        }
        const double r0 = warp_sum((double)a.a0), r1 = warp_sum((double)a.a1);
        const double r2 = warp_sum((double)a.a2), rp = warp_prod((double)a.p);
        if (lane == 0) {
          CandState& s = st[m];
          const float z0 = u[0] + off;
          if (sg.gfirst) {
            s.a0 = s.a1 = s.a2 = 0.0;
            s.p = 1.0;
            s.zfirst = (double)z0;
          } else if (pairs) {
            s.a0 += (double)pair_term<float>(kind, (float)s.zlast, z0);
          }
          s.a0 += r0;
          s.a1 += r1;
          s.a2 += r2;
          s.p *= rp;
          s.zlast = (double)(u[n - 1] + off);
          if (sg.glast) {
            if (kind_is_cyclic(kind))
              s.a0 += (double)pair_term<float>(kind, (float)s.zlast, (float)s.zfirst);
            s.gsum += finalize_f32(kind, s.a0, s.a1, s.a2, s.p, sg.gn);
          }
        }
      }
      __syncthreads();
    }
    for (int m = tid; m < BM; m += blockDim.x) {
      st[m].G[ci] = st[m].gsum;
      st[m].gsum = 0.0;
    }
    __syncthreads();
  }
  write_out(tb, F, st, BM, row0, N, out);
}

#endif  // CUROB_SIMT_F32

// Picks BM (candidates per CTA) so that the tiles and the per-candidate state
// fit in shared memory, and launches.
template <typename Tin, int kTiles, typename Kern>
cudaError_t launch_simt(Kern kern, const Tables& tb, const Function& F, const Tin* x, int N,
                        Tin* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  int ld = F.max_n + 1;
  if ((ld & 1) == 0) ++ld;  // odd row stride: lanes over candidates hit distinct banks
  const size_t limit = 200 * 1024;
  int BM = 32;
  auto bytes = [&](int bm) {
    return sizeof(CandState) * bm + kTiles * sizeof(Tin) * (size_t)bm * ld;
  };
  while (BM > 1 && bytes(BM) > limit) BM >>= 1;
  if (bytes(BM) > limit) return cudaErrorInvalidValue;
  const size_t smem = bytes(BM);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const long long grid = ((long long)N + BM - 1) / BM;
  kern<<<(unsigned)grid, kSimtThreads, smem, st>>>(tb, F, x, N, out, BM, ld);
  return cudaGetLastError();
}

}  // namespace curob

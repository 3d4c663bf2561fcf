// curob_simt.cuh -- the CUDA-core evaluator of the cuROB functions.
//
// One CTA owns BM candidates (BM = 32 while the largest block fits: then the
// 32 lanes of a warp are the 32 candidates, so every rotation element R[i][j]
// is one broadcast load shared by the warp).  For each component and each of
// its blocks (segments) the CTA
//   1. gathers y = s (x - o) at the block's variables S_b into shared memory
//      (the shift is taken in FP64; warp = candidate, lanes walk the sorted
//      index list, so a warp reads one row of x nearly contiguously),
//   2. rotates z_b = R_b y (+ c) -- one dot product per (candidate, output),
//      in index order with one fused multiply-add per term,
//   3. applies the block's per-variable transform and reduces it (warp =
//      candidate, lanes walk z, warp-shuffle sums; neighbour pairs inside the
//      block read z_{i+1} from shared memory, the pair across a block boundary
//      and the cyclic pair (z_D, z_1) are carried in per-candidate state),
// and closes each basic function when its last block is done.  A composition
// keeps each member's value and ||x - o_i||^2 and mixes them at the end
// (Sec. 6, Eq. weight) in FP64.
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

template <typename T> __device__ inline const T* rot_pool(const Tables& tb);
template <> __device__ inline const double* rot_pool<double>(const Tables& tb) { return tb.R; }
template <> __device__ inline const float* rot_pool<float>(const Tables& tb) { return tb.R32; }
template <typename T> __device__ inline const T* aux_pool(const Tables& tb);
template <> __device__ inline const double* aux_pool<double>(const Tables& tb) { return tb.aux; }
template <> __device__ inline const float* aux_pool<float>(const Tables& tb) { return tb.aux32; }

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

template <typename T, typename Tin>
__global__ void __launch_bounds__(kSimtThreads)
eval_simt_kernel(Tables tb, Function F, const Tin* __restrict__ x, int N, Tin* __restrict__ out,
                 int BM, int ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CandState* st = reinterpret_cast<CandState*>(smem_raw);
  T* Ys = reinterpret_cast<T*>(smem_raw + sizeof(CandState) * BM);
  T* Zs = Ys + (size_t)BM * ld;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const long long row0 = (long long)blockIdx.x * BM;
  const int D = tb.D;

  for (int m = tid; m < BM; m += blockDim.x) {
    CandState& s = st[m];
    s.a0 = s.a1 = s.a2 = 0.0;
    s.p = 1.0;
    s.zfirst = s.zlast = 0.0;
    s.gsum = 0.0;
    for (int c = 0; c < kMaxComponents; ++c) s.G[c] = s.d2[c] = 0.0;
  }
  __syncthreads();

  for (int ci = 0; ci < F.ncomp; ++ci) {
    const Component C = tb.comp[F.comp0 + ci];
    const int* __restrict__ S = tb.S + C.base;
    const double* __restrict__ op = tb.operm + C.base;
    for (int si = 0; si < C.nseg; ++si) {
      const Segment sg = tb.seg[C.seg0 + si];
      const int n = sg.n;

      // 1. gather y = s (x - o) over the block's variables (FP64 shift)
      for (int m = warp; m < BM; m += nwarps) {
        const long long row = row0 + m;
        const bool valid = row < N;
        const Tin* xr = x + (valid ? row : 0) * (long long)D;
        double d2p = 0.0;
        for (int j = lane; j < n; j += 32) {
          const int col = S[sg.zoff + j];
          const double ov = op[sg.zoff + j];
          const double xv = valid ? (double)xr[col] : ov;
          const double d = xv - ov;
          Ys[m * ld + j] = (T)(sg.scale * d);
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
          Zs[m * ld + i] = Ys[m * ld + i] + (T)sg.offset;
        }
      } else {
        const T* __restrict__ Rb = rot_pool<T>(tb) + sg.r_off;
        const int per = blockDim.x / BM;
        const int m = tid % BM;
        const T* Ym = Ys + m * ld;
        for (int i = tid / BM; i < n; i += per) {
          const T* Ri = Rb + (long long)i * n;
          T acc = T(0);
          for (int j = 0; j < n; ++j) acc = fma(Ri[j], Ym[j], acc);
          Zs[m * ld + i] = acc + (T)sg.offset;
        }
      }
      __syncthreads();

      // 3. per-variable transform and reduction
      {
        const int kind = sg.kind;
        const bool pairs = kind_has_pairs(kind);
        const T gnT = T(sg.gn);
        const T kat_e = (kind == K_KATSUURA) ? T(10.0 / pow((double)sg.gn, 1.2)) : T(0);
        const T* aux = aux_pool<T>(tb) + (sg.aux_off >= 0 ? sg.aux_off : 0);
        const bool has_aux = sg.aux_off >= 0;
        for (int m = warp; m < BM; m += nwarps) {
          const T* z = Zs + m * ld;
          Acc<T> a = acc_zero<T>();
          for (int i = lane; i < n; i += 32) {
            const T zi = z[i];
            elem_term<T>(kind, zi, sg.gpos + i, gnT, has_aux ? aux[i] : T(0), kat_e, a);
            if (pairs && i + 1 < n) a.a0 += pair_term<T>(kind, zi, z[i + 1]);
          }
          const double r0 = warp_sum((double)a.a0), r1 = warp_sum((double)a.a1);
          const double r2 = warp_sum((double)a.a2), rp = warp_prod((double)a.p);
          if (lane == 0) {
            CandState& s = st[m];
            if (sg.gfirst) {
              s.a0 = s.a1 = s.a2 = 0.0;
              s.p = 1.0;
              s.zfirst = (double)z[0];
            } else if (pairs) {
              s.a0 += (double)pair_term<T>(kind, (T)s.zlast, z[0]);
            }
            s.a0 += r0;
            s.a1 += r1;
            s.a2 += r2;
            s.p *= rp;
            s.zlast = (double)z[n - 1];
            if (sg.glast) {
              if (kind_is_cyclic(kind))
                s.a0 += (double)pair_term<T>(kind, (T)s.zlast, (T)s.zfirst);
              s.gsum += finalize(kind, s.a0, s.a1, s.a2, s.p, sg.gn);
            }
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

  for (int m = tid; m < BM; m += blockDim.x) {
    const long long row = row0 + m;
    if (row >= N) continue;
    double f = F.composition ? compose(tb.comp + F.comp0, F.ncomp, st[m].G, st[m].d2, D)
                             : st[m].G[0];
    out[row] = (Tin)(f + kFopt);
  }
}

// Picks BM (candidates per CTA) so that two BM x (max_n + 1) tiles and the
// per-candidate state fit in shared memory, and launches.
template <typename T, typename Tin>
cudaError_t launch_simt(const Tables& tb, const Function& F, const Tin* x, int N, Tin* out,
                        cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  int ld = F.max_n + 1;
  if ((ld & 1) == 0) ++ld;  // odd row stride: lanes over candidates hit distinct banks
  const size_t limit = 200 * 1024;
  int BM = 32;
  auto bytes = [&](int bm) {
    return sizeof(CandState) * bm + 2 * sizeof(T) * (size_t)bm * ld;
  };
  while (BM > 1 && bytes(BM) > limit) BM >>= 1;
  if (bytes(BM) > limit) return cudaErrorInvalidValue;
  const size_t smem = bytes(BM);
  auto kern = eval_simt_kernel<T, Tin>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const long long grid = ((long long)N + BM - 1) / BM;
  kern<<<(unsigned)grid, kSimtThreads, smem, st>>>(tb, F, x, N, out, BM, ld);
  return cudaGetLastError();
}

}  // namespace curob

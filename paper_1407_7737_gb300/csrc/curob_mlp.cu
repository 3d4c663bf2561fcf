// curob_mlp.cu -- the learned pre-screen (include/curob.h, curob_surrogate_*,
// curob_select_smallest, curob_gather_rows): MLP surrogate training and
// inference on tcgen05, AdamW, top-k selection and the screen that hands the
// selected candidates to the exact evaluator.
//
// Layers (B rows of a batch, all operands K-major, C = A B^T):
//   forward 1  A = U   (B x 128)     B = W1   (256 x 128)  -> a1
//   forward 2  A = H1  (B x 256)     B = W2   (256 x 256)  -> a2, then y, the
//              loss, dL/dy and dL/da2 in the same epilogue
//   backward 1 A = D2  (B x 256)     B = W2^T (256 x 256)  -> dL/da1
//   backward 2 A = D2^T (256 x B)    B = H1^T (256 x B)    -> dL/dW2 (split-K)
//   backward 3 A = D1^T (256 x B)    B = U^T  (128 x B)    -> dL/dW1 (split-K)
// The epilogues write the transposed copies the weight-gradient contractions
// read, so every contraction is K-major on both sides.  Column sums over a
// tile (bias gradients, dL/dw3, the loss) and the split-K partials are
// reduced in a fixed order by the AdamW kernel: a training step is
// bit-for-bit reproducible.
//
// Warp roles of mlp_gemm_kernel (192 threads, one 128-row tile):
//   warp 0     TMA producer: per 32-column K stage one tensor copy of the A
//              tile (128 x 32) and one of the B tile (N x 32), 64-byte
//              swizzle, into a 3-stage ring under full/empty mbarriers;
//   warp 1     allocates TMEM (N columns) and issues the MMAs (M = 128,
//              N = 128 or 256, K = 16 per instruction);
//   warps 2-5  epilogue: thread = row = TMEM lane, 32 columns per tcgen05.ld.
// Every wait is bounded (2 s, then DEV_TIMEOUT in the status word).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/curob.h"
#include "curob_mlp.cuh"
#include "curob_tc.cuh"
#include "curob_tmap.hpp"

namespace curob {
bool device_accessible(const void* p);
}

using namespace curob;
using namespace curob::tc;

namespace {

constexpr int kGemmThreads = 192;
constexpr int kStages = 3;
constexpr int kTile = 128;
constexpr int kATileBytes = kTile * kRowBytes;  // 8 KB
constexpr int kRedStride = 33;                  // padded row of the column-sum scratch

enum Epi : int { EPI_L1_TRAIN, EPI_L1_INFER, EPI_L2_TRAIN, EPI_L2_INFER, EPI_BWD1, EPI_PARTIAL };

constexpr bool epi_reduces(int e) { return e == EPI_L2_TRAIN || e == EPI_BWD1; }

struct GemmArgs {
  int M;                // valid rows of A (rows >= M are zero-filled by TMA and not stored)
  int N;                // accumulator columns: 128 or 256
  int kstages;          // 32-column K stages per CTA
  int ksplit;           // K columns per blockIdx.y
  const float* bias;    // b1 / b2 (FP32)
  const float* w3;      // w3 rounded to BF16, held as FP32
  const float* b3;      // scalar
  const float* T;       // standardised targets (forward 2, training)
  float inv_half_b;     // 2 / B: dL/dy = (y - t) 2 / B
  float out_scale;      // inference: out = out_scale * y + out_shift
  float out_shift;
  __nv_bfloat16* H;     // row-major B x 256 output (h1, or dL/da2)
  __nv_bfloat16* HT;    // transposed 256 x ldt output (h1^T, dL/da2^T, dL/da1^T)
  int ldt;
  float* G;             // gelu'(a1), row-major B x 256
  float* out;           // predictions (M) or split-K partials [splits][M][N]
  float* pvec;          // per-tile column sums
  float* pscal;         // per-tile scalars (loss sum, dL/db3)
  int* status;
};

struct SmemMap {
  uint8_t* stages;
  float* red;   // [128][33]
  float* red4;  // [4][32]
  uint64_t* full;
  uint64_t* empty;
  uint64_t* tmem_full;
  uint64_t* grp;
  int* abort_flag;
  uint32_t* tmem_slot;
};

__host__ __device__ constexpr int stage_bytes(int N) { return kATileBytes + N * kRowBytes; }

__host__ __device__ constexpr size_t gemm_smem_bytes(int N, bool reduces) {
  return 1024 + (size_t)kStages * stage_bytes(N) +
         (reduces ? (size_t)(kTile * kRedStride + 4 * 32) * sizeof(float) : 0) + 256;
}

__device__ inline SmemMap smem_map(uint8_t* raw, int N, bool reduces) {
  SmemMap m;
  uint8_t* p = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  m.stages = p;
  p += (size_t)kStages * stage_bytes(N);
  m.red = reinterpret_cast<float*>(p);
  m.red4 = m.red + kTile * kRedStride;
  if (reduces) p += (size_t)(kTile * kRedStride + 4 * 32) * sizeof(float);
  p = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 7) & ~uintptr_t(7));
  m.full = reinterpret_cast<uint64_t*>(p);
  m.empty = m.full + kStages;
  m.tmem_full = m.empty + kStages;
  m.grp = m.tmem_full + 1;
  m.abort_flag = reinterpret_cast<int*>(m.grp + 1);
  m.tmem_slot = reinterpret_cast<uint32_t*>(m.abort_flag + 1);
  return m;
}

// ---------------------------------------------------------------- GELU
__device__ __forceinline__ float phi_cdf(float a) { return 0.5f * erfcf(-a * 0.70710678118654752f); }
__device__ __forceinline__ float gelu_f(float a) { return a * phi_cdf(a); }
__device__ __forceinline__ float gelu_grad_f(float a) {
  return phi_cdf(a) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Bounded barrier of the 4 epilogue warps (an mbarrier of count 4).
__device__ __forceinline__ bool epi_sync(const SmemMap& m, uint32_t& phase, int* status) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(m.grp);
  const bool ok = mbar_wait(m.grp, phase & 1u, m.abort_flag, status);
  ++phase;
  return ok;
}

// Sum over the tile's 128 rows of 32 column values per thread (row = the
// thread's TMEM lane), in a fixed order (rows in 4 quarters, quarters added
// in order); the thread of row e < 32 receives column e's sum.
__device__ __forceinline__ bool column_sums(const SmemMap& m, int row, const float* v,
                                            uint32_t& phase, int* status, float& total) {
#pragma unroll
  for (int j = 0; j < 32; ++j) m.red[row * kRedStride + j] = v[j];
  if (!epi_sync(m, phase, status)) return false;
  {
    const int j = row & 31, q = row >> 5;
    float s = 0.f;
    for (int r = 32 * q; r < 32 * q + 32; ++r) s += m.red[r * kRedStride + j];
    m.red4[q * 32 + j] = s;
  }
  if (!epi_sync(m, phase, status)) return false;
  total = 0.f;
  if (row < 32) total = ((m.red4[row] + m.red4[32 + row]) + m.red4[64 + row]) + m.red4[96 + row];
  return epi_sync(m, phase, status);
}

template <int kEpi>
__global__ void __launch_bounds__(kGemmThreads, 1)
    mlp_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    const GemmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  const int N = a.N;
  const SmemMap m = smem_map(smem_raw, N, epi_reduces(kEpi));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTile;
  const int k0 = blockIdx.y * a.ksplit;
  const int sbytes = stage_bytes(N);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&m.full[s], 1);   // the producer's arrive.expect_tx
      mbar_init(&m.empty[s], 1);  // one tcgen05.commit
    }
    mbar_init(m.tmem_full, 1);
    mbar_init(m.grp, 4);
    *m.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(m.tmem_slot, (uint32_t)N);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *m.tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------- TMA loads
    if (lane == 0) {
      tma_prefetch_desc(&mapA);
      tma_prefetch_desc(&mapB);
      uint32_t issued = 0, last_par = 0;  // bit st: stage st used / parity of its last use
      for (int s = 0; s < a.kstages; ++s) {
        const int st = s % kStages;
        const uint32_t round = (uint32_t)(s / kStages);
        if (round > 0 && !mbar_wait(&m.empty[st], (round - 1) & 1u, m.abort_flag, a.status)) break;
        uint8_t* dst = m.stages + (size_t)st * sbytes;
        mbar_arrive_expect_tx(&m.full[st], (uint32_t)sbytes);
        tma_load_2d(dst, &mapA, k0 + 32 * s, m0, &m.full[st]);
        tma_load_2d(dst + kATileBytes, &mapB, k0 + 32 * s, 0, &m.full[st]);
        issued |= 1u << st;
        last_par = (last_par & ~(1u << st)) | ((round & 1u) << st);
      }
      // every copy issued has landed before the CTA may exit
      for (int st = 0; st < kStages; ++st)
        if (issued >> st & 1u) mbar_wait(&m.full[st], last_par >> st & 1u, m.abort_flag, a.status);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = idesc_make(1u, kTile, (uint32_t)N);
      for (int s = 0; s < a.kstages; ++s) {
        const int st = s % kStages;
        const uint32_t round = (uint32_t)(s / kStages);
        if (!mbar_wait(&m.full[st], round & 1u, m.abort_flag, a.status)) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(m.stages + (size_t)st * sbytes);
        const uint32_t sb = sa + kATileBytes;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          tc_mma<false>(tmem, sdesc_sw64(sa + 32 * kk), sdesc_sw64(sb + 32 * kk), idesc,
                        (s | kk) ? 1u : 0u);
        tc_commit(&m.empty[st]);
      }
      tc_commit(m.tmem_full);
      // the MMAs have retired before TMEM is freed
      mbar_wait(m.tmem_full, 0, m.abort_flag, a.status);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    const int grow = m0 + row;
    const bool valid = grow < a.M;
    uint32_t phase = 0;
    bool ok = mbar_wait(m.tmem_full, 0, m.abort_flag, a.status);
    tc_fence_after();
    ok = ok && !*m.abort_flag;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    float v[32];
    if (ok) {
      if constexpr (kEpi == EPI_L1_TRAIN || kEpi == EPI_L1_INFER) {
        for (int c = 0; c < N; c += 32) {
          tmem_ld32(tl + (uint32_t)c, v);
          if (valid) {
            uint32_t pk[16];
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              const float a0 = v[j] + a.bias[c + j], a1 = v[j + 1] + a.bias[c + j + 1];
              const float h0 = gelu_f(a0), h1 = gelu_f(a1);
              pk[j / 2] = bf16x2(h0, h1);
              if constexpr (kEpi == EPI_L1_TRAIN) {
                v[j] = gelu_grad_f(a0);
                v[j + 1] = gelu_grad_f(a1);
                const __nv_bfloat162 hh = *reinterpret_cast<__nv_bfloat162*>(&pk[j / 2]);
                a.HT[(size_t)(c + j) * a.ldt + grow] = hh.x;
                a.HT[(size_t)(c + j + 1) * a.ldt + grow] = hh.y;
              }
            }
            uint4* dst = reinterpret_cast<uint4*>(a.H + (size_t)grow * kSurH + c);
#pragma unroll
            for (int i = 0; i < 4; ++i)
              dst[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
            if constexpr (kEpi == EPI_L1_TRAIN) {
              float4* gd = reinterpret_cast<float4*>(a.G + (size_t)grow * kSurH + c);
#pragma unroll
              for (int i = 0; i < 8; ++i)
                gd[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
          }
        }
      } else if constexpr (kEpi == EPI_L2_INFER) {
        float y = 0.f;
        for (int c = 0; c < N; c += 32) {
          tmem_ld32(tl + (uint32_t)c, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) y += a.w3[c + j] * gelu_f(v[j] + a.bias[c + j]);
        }
        if (valid) a.out[grow] = a.out_scale * (y + *a.b3) + a.out_shift;
      } else if constexpr (kEpi == EPI_L2_TRAIN) {
        float y = 0.f;
        for (int c = 0; c < N && ok; c += 32) {
          tmem_ld32(tl + (uint32_t)c, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) y += a.w3[c + j] * gelu_f(v[j] + a.bias[c + j]);
        }
        y += *a.b3;
        const float r = valid ? y - a.T[grow] : 0.f;
        const float d3 = r * a.inv_half_b;
        float hv[32];
        for (int c = 0; c < N && ok; c += 32) {
          tmem_ld32(tl + (uint32_t)c, v);
          uint32_t pk[16];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float a2 = v[j] + a.bias[c + j];
            hv[j] = d3 * gelu_f(a2);                       // row's share of dL/dw3
            v[j] = d3 * a.w3[c + j] * gelu_grad_f(a2);     // dL/da2
          }
#pragma unroll
          for (int j = 0; j < 32; j += 2) pk[j / 2] = bf16x2(v[j], v[j + 1]);
          if (valid) {
            uint4* dst = reinterpret_cast<uint4*>(a.H + (size_t)grow * kSurH + c);
#pragma unroll
            for (int i = 0; i < 4; ++i)
              dst[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              const __nv_bfloat162 hh = *reinterpret_cast<__nv_bfloat162*>(&pk[j / 2]);
              a.HT[(size_t)(c + j) * a.ldt + grow] = hh.x;
              a.HT[(size_t)(c + j + 1) * a.ldt + grow] = hh.y;
            }
          }
          float tot;
          ok = column_sums(m, row, v, phase, a.status, tot);
          if (ok && row < 32) a.pvec[((size_t)blockIdx.x * 2 + 0) * kSurH + c + row] = tot;
          ok = ok && column_sums(m, row, hv, phase, a.status, tot);
          if (ok && row < 32) a.pvec[((size_t)blockIdx.x * 2 + 1) * kSurH + c + row] = tot;
        }
        // tile scalars: sum of squared residuals and dL/db3
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
        v[0] = r * r;
        v[1] = d3;
        float tot;
        ok = ok && column_sums(m, row, v, phase, a.status, tot);
        if (ok && row < 2) a.pscal[(size_t)blockIdx.x * 2 + row] = tot;
      } else if constexpr (kEpi == EPI_BWD1) {
        for (int c = 0; c < N && ok; c += 32) {
          tmem_ld32(tl + (uint32_t)c, v);
          if (valid) {
            const float4* gd = reinterpret_cast<const float4*>(a.G + (size_t)grow * kSurH + c);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float4 g4 = gd[i];
              v[4 * i] *= g4.x;
              v[4 * i + 1] *= g4.y;
              v[4 * i + 2] *= g4.z;
              v[4 * i + 3] *= g4.w;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j)
              a.HT[(size_t)(c + j) * a.ldt + grow] = __float2bfloat16_rn(v[j]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0.f;
          }
          float tot;
          ok = column_sums(m, row, v, phase, a.status, tot);
          if (ok && row < 32) a.pvec[(size_t)blockIdx.x * kSurH + c + row] = tot;
        }
      } else {  // EPI_PARTIAL
        for (int c = 0; c < N; c += 32) {
          tmem_ld32(tl + (uint32_t)c, v);
          if (valid) {
            float4* dst = reinterpret_cast<float4*>(
                a.out + ((size_t)blockIdx.y * a.M + grow) * (size_t)N + c);
#pragma unroll
            for (int i = 0; i < 8; ++i)
              dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_free(tmem, (uint32_t)N);
  }
}

// ------------------------------------------------------------------ prep
// x (n x 100 FP32) -> U = bf16(x / 128) zero-padded to 128 columns, its
// transpose U^T (128 x ldut, optional), and the standardised targets
// T = (log(max(f - f_opt, 0) + 1) - mu) / sd (optional).  32 rows per block.
__global__ void mlp_prep_kernel(const float* __restrict__ x, int n, const float* __restrict__ f,
                                float f_opt, float mu, float inv_sd, __nv_bfloat16* U,
                                __nv_bfloat16* UT, long long ldut, float* T) {
  __shared__ float s[32][kSurIn + 1];
  const long long r0 = (long long)blockIdx.x * 32;
  for (int e = threadIdx.x; e < 32 * kSurIn; e += blockDim.x) {
    const int r = e / kSurIn, c = e % kSurIn;
    s[r][c] = (r0 + r < n) ? x[(r0 + r) * kSurIn + c] * 0.0078125f : 0.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * (kSurInPad / 2); e += blockDim.x) {
    const int r = e / (kSurInPad / 2), c = 2 * (e % (kSurInPad / 2));
    if (r0 + r < n) {
      const float lo = c < kSurIn ? s[r][c] : 0.f, hi = c + 1 < kSurIn ? s[r][c + 1] : 0.f;
      reinterpret_cast<uint32_t*>(U + (r0 + r) * kSurInPad)[c / 2] = bf16x2(lo, hi);
    }
  }
  if (UT) {
    for (int e = threadIdx.x; e < kSurInPad * 32; e += blockDim.x) {
      const int c = e / 32, r = e % 32;
      if (r0 + r < n) UT[(long long)c * ldut + r0 + r] = __float2bfloat16_rn(c < kSurIn ? s[r][c] : 0.f);
    }
  }
  if (T && threadIdx.x < 32 && r0 + threadIdx.x < n) {
    const float fv = f[r0 + threadIdx.x];
    T[r0 + threadIdx.x] = (log1pf(fmaxf(fv - f_opt, 0.f)) - mu) * inv_sd;
  }
}

// Mean and standard deviation of t = log(max(f - f_opt, 0) + 1) over n
// values, in FP64, in a fixed summation order: a fixed grid of kStatBlocks
// blocks writes one partial sum each (thread-strided sums, then a tree), and
// one block adds the partials in block order.  Pass 0 sums t, pass 1 sums
// (t - mu)^2 with mu from pass 0.
constexpr int kStatBlocks = 256, kStatThreads = 256;

__global__ void __launch_bounds__(kStatThreads) mlp_stats_partial_kernel(
    const float* __restrict__ f, long long n, double f_opt, const double* __restrict__ stats,
    int pass, double* __restrict__ partial) {
  __shared__ double sh[kStatThreads];
  const double mu = pass ? stats[0] : 0.0;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * kStatThreads + threadIdx.x; i < n;
       i += (long long)kStatBlocks * kStatThreads) {
    const double t = log1p(fmax((double)f[i] - f_opt, 0.0));
    s += pass ? (t - mu) * (t - mu) : t;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kStatThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kStatBlocks) mlp_stats_final_kernel(
    const double* __restrict__ partial, long long n, int pass, double* __restrict__ stats) {
  __shared__ double sh[kStatBlocks];
  sh[threadIdx.x] = partial[threadIdx.x];
  __syncthreads();
  for (int w = kStatBlocks / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (pass == 0) stats[0] = sh[0] / (double)n;
    else stats[1] = sqrt(sh[0] / (double)n);
  }
}

// ----------------------------------------------------------------- AdamW
struct AdamArgs {
  float* master;
  float* mom1;
  float* mom2;
  float* grad;
  const float* pW1;   // [splits][256][128]
  const float* pW2;   // [splits][256][256]
  const float* pb1;   // [tiles][256]
  const float* pv2;   // [tiles][2][256]: dL/db2, dL/dw3
  const float* ps2;   // [tiles][2]: loss sum, dL/db3
  int splits, tiles, batch;
  __nv_bfloat16* W1b;   // [256][128]
  __nv_bfloat16* W2b;   // [256][256]
  __nv_bfloat16* W2tb;  // [256][256]
  float* w3b;
  float* loss_out;      // mean loss of the batch (may be null)
  int update;
  float lr, beta1, beta2, eps, wd, bc1, bc2;
};

__global__ void mlp_adamw_kernel(const AdamArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kSurParams) return;
  float g = 0.f;
  if (p < kOffB1) {
    const int i = p / kSurIn, k = p % kSurIn;
    for (int s = 0; s < a.splits; ++s) g += a.pW1[((size_t)s * kSurH + i) * kSurInPad + k];
  } else if (p < kOffW2) {
    const int i = p - kOffB1;
    for (int t = 0; t < a.tiles; ++t) g += a.pb1[(size_t)t * kSurH + i];
  } else if (p < kOffB2) {
    const int e = p - kOffW2;
    for (int s = 0; s < a.splits; ++s) g += a.pW2[(size_t)s * kSurH * kSurH + e];
  } else if (p < kOffW3) {
    const int j = p - kOffB2;
    for (int t = 0; t < a.tiles; ++t) g += a.pv2[((size_t)t * 2 + 0) * kSurH + j];
  } else if (p < kOffB3) {
    const int j = p - kOffW3;
    for (int t = 0; t < a.tiles; ++t) g += a.pv2[((size_t)t * 2 + 1) * kSurH + j];
  } else {
    float l = 0.f;
    for (int t = 0; t < a.tiles; ++t) {
      l += a.ps2[(size_t)t * 2 + 0];
      g += a.ps2[(size_t)t * 2 + 1];
    }
    if (a.loss_out) *a.loss_out = l / (float)a.batch;
  }
  a.grad[p] = g;
  float w = a.master[p];
  if (a.update) {
    const float m1 = a.beta1 * a.mom1[p] + (1.f - a.beta1) * g;
    const float m2 = a.beta2 * a.mom2[p] + (1.f - a.beta2) * g * g;
    a.mom1[p] = m1;
    a.mom2[p] = m2;
    const float mhat = m1 / a.bc1, vhat = m2 / a.bc2;
    w = w * (1.f - a.lr * a.wd);
    w = w - a.lr * mhat / (sqrtf(vhat) + a.eps);
    a.master[p] = w;
  }
  const __nv_bfloat16 wb = __float2bfloat16_rn(w);
  if (p < kOffB1) {
    a.W1b[(p / kSurIn) * kSurInPad + p % kSurIn] = wb;
  } else if (p >= kOffW2 && p < kOffB2) {
    const int e = p - kOffW2, j = e / kSurH, i = e % kSurH;
    a.W2b[j * kSurH + i] = wb;
    a.W2tb[i * kSurH + j] = wb;
  } else if (p >= kOffW3 && p < kOffB3) {
    a.w3b[p - kOffW3] = __bfloat162float(wb);
  }
}

// ------------------------------------------------------------- selection
// Order-preserving key of a float (NaN above +inf, -0 equal to +0).
__device__ __forceinline__ uint32_t fkey(float v) {
  uint32_t b = __float_as_uint(v);
  if (v != v) return 0xFFFFFFFFu;
  if (b == 0x80000000u) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// state: [0] prefix of the k-th key, [1] mask of the decided bits, [2] how
// many of the keys equal to the final prefix are still to take.
__global__ void select_hist_kernel(const float* __restrict__ v, long long n, const uint32_t* state,
                                   int shift, int bits, unsigned* hist) {
  __shared__ unsigned sh[2048];
  for (int b = threadIdx.x; b < 2048; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const uint32_t prefix = state[0], mask = state[1];
  const uint32_t digit = (1u << bits) - 1u;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint32_t k = fkey(v[i]);
    if ((k & mask) == prefix) atomicAdd(&sh[(k >> shift) & digit], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 2048; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

// One block of 1024 threads: finds the digit of the k-th key, zeroes the
// histogram for the next pass.
__global__ void select_find_kernel(unsigned* hist, int bits, int shift, uint32_t* state) {
  __shared__ unsigned cs[1024];
  const int nb = 1 << bits;
  const int per = (nb + 1023) / 1024;
  const int t = threadIdx.x;
  unsigned s = 0;
  for (int b = t * per; b < min(nb, (t + 1) * per); ++b) s += hist[b];
  cs[t] = s;
  __syncthreads();
  if (t == 0) {
    unsigned krem = state[2], cum = 0;
    int tsel = 0;
    for (; tsel < 1024; ++tsel) {
      if (cum + cs[tsel] >= krem) break;
      cum += cs[tsel];
    }
    int b = tsel * per;
    for (; b < nb; ++b) {
      if (cum + hist[b] >= krem) break;
      cum += hist[b];
    }
    b = min(b, nb - 1);  // (k <= N: the k-th key's digit is always found)
    state[0] |= (uint32_t)b << shift;
    state[1] |= (uint32_t)(nb - 1) << shift;
    state[2] = krem - cum;
  }
  __syncthreads();
  for (int b = t; b < nb; b += 1024) hist[b] = 0;
}

constexpr int kSelPer = 16;                       // keys per thread
constexpr int kSelBlock = 256;
constexpr int kSelChunk = kSelPer * kSelBlock;    // keys per block

// Per-block counts of keys below and equal to the k-th key.
__global__ void select_count_kernel(const float* __restrict__ v, long long n, const uint32_t* state,
                                    int* cnt) {
  __shared__ int sl[kSelBlock], se[kSelBlock];
  const uint32_t T = state[0];
  const long long base = (long long)blockIdx.x * kSelChunk + (long long)threadIdx.x * kSelPer;
  int lt = 0, eq = 0;
  for (int i = 0; i < kSelPer; ++i) {
    if (base + i < n) {
      const uint32_t k = fkey(v[base + i]);
      lt += k < T;
      eq += k == T;
    }
  }
  sl[threadIdx.x] = lt;
  se[threadIdx.x] = eq;
  __syncthreads();
  for (int w = kSelBlock / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sl[threadIdx.x] += sl[threadIdx.x + w];
      se[threadIdx.x] += se[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    cnt[2 * blockIdx.x] = sl[0];
    cnt[2 * blockIdx.x + 1] = se[0];
  }
}

// Exclusive prefix sums of the per-block counts, one block.
__global__ void select_scan_kernel(int* cnt, int nblk) {
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int i = 0; i < nblk; ++i) {
      const int l = cnt[2 * i], e = cnt[2 * i + 1];
      cnt[2 * i] = a;
      cnt[2 * i + 1] = b;
      a += l;
      b += e;
    }
  }
}

// Writes the selected indices in ascending order: a key below the k-th goes
// to (keys below before it) + min(equal keys before it, k_eq); an equal key
// is taken while fewer than k_eq equal keys precede it.
__global__ void select_write_kernel(const float* __restrict__ v, long long n, const uint32_t* state,
                                    const int* off, int k, int* idx) {
  __shared__ int sl[kSelBlock], se[kSelBlock];
  const uint32_t T = state[0];
  const int keq = (int)state[2];
  const long long base = (long long)blockIdx.x * kSelChunk + (long long)threadIdx.x * kSelPer;
  uint32_t keys[kSelPer];
  int lt = 0, eq = 0;
  for (int i = 0; i < kSelPer; ++i) {
    keys[i] = base + i < n ? fkey(v[base + i]) : 0xFFFFFFFFu;
    const bool in = base + i < n;
    lt += in && keys[i] < T;
    eq += in && keys[i] == T;
  }
  sl[threadIdx.x] = lt;
  se[threadIdx.x] = eq;
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive scan over the block's threads, in order
    int a = 0, b = 0;
    for (int t = 0; t < kSelBlock; ++t) {
      const int l = sl[t], e = se[t];
      sl[t] = a;
      se[t] = b;
      a += l;
      b += e;
    }
  }
  __syncthreads();
  int lb = off[2 * blockIdx.x] + sl[threadIdx.x];
  int eb = off[2 * blockIdx.x + 1] + se[threadIdx.x];
  for (int i = 0; i < kSelPer; ++i) {
    if (base + i >= n) break;
    if (keys[i] < T) {
      const int pos = lb + min(eb, keq);
      if (pos < k) idx[pos] = (int)(base + i);
      ++lb;
    } else if (keys[i] == T) {
      if (eb < keq && lb + eb < k) idx[lb + eb] = (int)(base + i);
      ++eb;
    }
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ x, int D, const int* __restrict__ idx,
                                   int k, float* __restrict__ out) {
  for (int r = blockIdx.x; r < k; r += gridDim.x) {
    const float* src = x + (size_t)idx[r] * D;
    for (int d = threadIdx.x; d < D; d += blockDim.x) out[(size_t)r * D + d] = src[d];
  }
}

// ----------------------------------------------------------- host helpers
thread_local char g_last_error[256] = "";

// Records the failing step and returns CUROB_ERR_CUDA.
curob_status fail(const char* where, cudaError_t e = cudaSuccess) {
  snprintf(g_last_error, sizeof(g_last_error), "%s%s%s", where, e != cudaSuccess ? ": " : "",
           e != cudaSuccess ? cudaGetErrorString(e) : "");
  return CUROB_ERR_CUDA;
}
// 2-D BF16 tensor map, 32-element (64-byte) inner box, 64-byte swizzle,
// zero fill outside the tensor.
bool make_map(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t rows, uint64_t row_bytes,
              uint32_t box_rows) {
  return encode_2d(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, ptr, inner, rows, row_bytes, 32, box_rows,
                   CU_TENSOR_MAP_SWIZZLE_64B);
}

template <int kEpi>
cudaError_t launch_gemm(const CUtensorMap& A, const CUtensorMap& B, const GemmArgs& a, int mtiles,
                        int splits, cudaStream_t st) {
  // At most two 256-column (or four 128-column) CTAs per SM, so that TMEM
  // (512 columns) never runs out.
  const size_t need = gemm_smem_bytes(a.N, epi_reduces(kEpi));
  const size_t smem = std::max(need, (size_t)(a.N == 256 ? 80 * 1024 : 48 * 1024));
  // the attribute is per kernel: raise it to the largest size launched
  static size_t attr_max = 0;
  if (attr_max < smem) {
    cudaError_t e = cudaFuncSetAttribute(mlp_gemm_kernel<kEpi>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_max = smem;
  }
  mlp_gemm_kernel<kEpi><<<dim3(mtiles, splits), kGemmThreads, smem, st>>>(A, B, a);
  return cudaGetLastError();
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

// ------------------------------------------------------------ the object
struct curob_surrogate_st {
  int max_batch = 0;
  int chunk = 0;
  float* master = nullptr;  // FP32 parameters (flat, kSurParams)
  float* mom1 = nullptr;
  float* mom2 = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* W1b = nullptr;
  __nv_bfloat16* W2b = nullptr;
  __nv_bfloat16* W2tb = nullptr;
  float* w3b = nullptr;
  // training scratch (max_batch rows)
  __nv_bfloat16 *U = nullptr, *UT = nullptr, *H1 = nullptr, *H1T = nullptr, *D2 = nullptr,
                *D2T = nullptr, *D1T = nullptr;
  float* G1D = nullptr;
  float* T = nullptr;
  float* pW1 = nullptr;
  float* pW2 = nullptr;
  float* pb1 = nullptr;
  float* pv2 = nullptr;
  float* ps2 = nullptr;
  double* stats = nullptr;
  int* d_status = nullptr;  // device-side error word of this object's kernels
  // inference scratch (chunk rows)
  __nv_bfloat16 *Uc = nullptr, *H1c = nullptr;
  // selection scratch
  unsigned* hist = nullptr;
  uint32_t* sel_state = nullptr;
  int* sel_cnt = nullptr;
  long long sel_cap = 0;
  float* pred = nullptr;
  long long pred_cap = 0;
  CUtensorMap mW1, mW2, mW2t;
  int t = 0;  // AdamW step count
  float lr = 1e-3f, beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f, wd = 1e-4f;
  float mu = 0.f, sd = 1.f;
  std::mutex mtx;
};

namespace {

void free_surrogate(curob_surrogate s) {
  if (!s) return;
  void* ptrs[] = {s->master, s->mom1, s->mom2, s->grad, s->W1b, s->W2b, s->W2tb, s->w3b,
                  s->d_status, s->U, s->UT, s->H1, s->H1T, s->D2, s->D2T, s->D1T, s->G1D, s->T, s->pW1,
                  s->pW2, s->pb1, s->pv2, s->ps2, s->stats, s->Uc, s->H1c, s->hist,
                  s->sel_state, s->sel_cnt, s->pred};
  for (void* p : ptrs) cudaFree(p);
  delete s;
}

template <class T>
bool dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(count, 1)) ==
         cudaSuccess;
}

// Rewrites the BF16 copies from the masters (AdamW kernel with update = 0
// and zero gradient partials is not needed: a plain pass with splits = 0).
cudaError_t refresh_copies(curob_surrogate s, cudaStream_t st) {
  AdamArgs a{};
  a.master = s->master;
  a.mom1 = s->mom1;
  a.mom2 = s->mom2;
  a.grad = s->grad;
  a.pW1 = s->pW1;
  a.pW2 = s->pW2;
  a.pb1 = s->pb1;
  a.pv2 = s->pv2;
  a.ps2 = s->ps2;
  a.splits = 0;
  a.tiles = 0;
  a.batch = 1;
  a.W1b = s->W1b;
  a.W2b = s->W2b;
  a.W2tb = s->W2tb;
  a.w3b = s->w3b;
  a.update = 0;
  mlp_adamw_kernel<<<(kSurParams + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// One training (or gradient-only) step on a prepared batch: U (B x 128),
// U^T (128 x ldut, columns of this batch), T (B).
curob_status run_step(curob_surrogate s, const __nv_bfloat16* U, const __nv_bfloat16* UT,
                      long long ldut, const float* T, int B, float lr, int update, float* loss_out,
                      int* status, cudaStream_t st) {
  const int tiles = B / kTile, splits = B / kTile;
  const long long ldt = s->max_batch;
  CUtensorMap mA1, mA2, mA3, mA4, mB4, mA5, mB5;
  bool ok = make_map(&mA1, U, kSurInPad, B, kSurInPad * 2, kTile) &&
            make_map(&mA2, s->H1, kSurH, B, kSurH * 2, kTile) &&
            make_map(&mA3, s->D2, kSurH, B, kSurH * 2, kTile) &&
            make_map(&mA4, s->D2T, B, kSurH, ldt * 2, kTile) &&
            make_map(&mB4, s->H1T, B, kSurH, ldt * 2, kSurH) &&
            make_map(&mA5, s->D1T, B, kSurH, ldt * 2, kTile) &&
            make_map(&mB5, UT, B, kSurInPad, ldut * 2, kSurInPad);
  if (!ok) return fail("tensor map encoding (training step)");
  GemmArgs g{};
  g.status = status;
  g.ldt = (int)ldt;
  // forward 1
  g.M = B;
  g.N = kSurH;
  g.kstages = kSurInPad / 32;
  g.ksplit = 0;
  g.bias = s->master + kOffB1;
  g.H = s->H1;
  g.HT = s->H1T;
  g.G = s->G1D;
  cudaError_t e;
  if ((e = launch_gemm<EPI_L1_TRAIN>(mA1, s->mW1, g, tiles, 1, st)) != cudaSuccess)
    return fail("forward 1", e);
  // forward 2 + loss + dL/da2
  g.kstages = kSurH / 32;
  g.bias = s->master + kOffB2;
  g.w3 = s->w3b;
  g.b3 = s->master + kOffB3;
  g.T = T;
  g.inv_half_b = 2.0f / (float)B;
  g.H = s->D2;
  g.HT = s->D2T;
  g.pvec = s->pv2;
  g.pscal = s->ps2;
  if ((e = launch_gemm<EPI_L2_TRAIN>(mA2, s->mW2, g, tiles, 1, st)) != cudaSuccess)
    return fail("forward 2", e);
  // backward 1: dL/da1 = (D2 W2) * gelu'(a1)
  g.HT = s->D1T;
  g.pvec = s->pb1;
  if ((e = launch_gemm<EPI_BWD1>(mA3, s->mW2t, g, tiles, 1, st)) != cudaSuccess)
    return fail("backward 1", e);
  // backward 2 and 3: weight gradients, split over the batch
  GemmArgs w{};
  w.status = status;
  w.M = kSurH;
  w.N = kSurH;
  w.kstages = kTile / 32;
  w.ksplit = kTile;
  w.out = s->pW2;
  if ((e = launch_gemm<EPI_PARTIAL>(mA4, mB4, w, kSurH / kTile, splits, st)) != cudaSuccess)
    return fail("backward 2", e);
  w.N = kSurInPad;
  w.out = s->pW1;
  if ((e = launch_gemm<EPI_PARTIAL>(mA5, mB5, w, kSurH / kTile, splits, st)) != cudaSuccess)
    return fail("backward 3", e);
  // AdamW
  AdamArgs a{};
  a.master = s->master;
  a.mom1 = s->mom1;
  a.mom2 = s->mom2;
  a.grad = s->grad;
  a.pW1 = s->pW1;
  a.pW2 = s->pW2;
  a.pb1 = s->pb1;
  a.pv2 = s->pv2;
  a.ps2 = s->ps2;
  a.splits = splits;
  a.tiles = tiles;
  a.batch = B;
  a.W1b = s->W1b;
  a.W2b = s->W2b;
  a.W2tb = s->W2tb;
  a.w3b = s->w3b;
  a.loss_out = loss_out;
  a.update = update;
  if (update) {
    s->t += 1;
    a.lr = lr;
    a.beta1 = s->beta1;
    a.beta2 = s->beta2;
    a.eps = s->eps;
    a.wd = s->wd;
    a.bc1 = (float)(1.0 - std::pow((double)s->beta1, (double)s->t));
    a.bc2 = (float)(1.0 - std::pow((double)s->beta2, (double)s->t));
  }
  mlp_adamw_kernel<<<(kSurParams + 255) / 256, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("adamw", e);
  return CUROB_OK;
}

curob_status ensure_select_scratch(curob_surrogate s, long long n) {
  if (s->sel_cap >= n && s->hist) return CUROB_OK;
  cudaFree(s->sel_cnt);
  s->sel_cnt = nullptr;
  const long long nblk = (n + kSelChunk - 1) / kSelChunk;
  if (!dalloc(&s->sel_cnt, 2 * nblk)) return CUROB_ERR_OUT_OF_MEMORY;
  if (!s->hist && !dalloc(&s->hist, 2048)) return CUROB_ERR_OUT_OF_MEMORY;
  if (!s->sel_state && !dalloc(&s->sel_state, 4)) return CUROB_ERR_OUT_OF_MEMORY;
  s->sel_cap = n;
  return CUROB_OK;
}

// Radix selection (11 + 11 + 10 bits of the key) and the ordered write.
cudaError_t select_launch(const float* v, long long n, int k, int* idx, unsigned* hist,
                          uint32_t* state, int* cnt, cudaStream_t st) {
  const uint32_t init[4] = {0u, 0u, (uint32_t)k, 0u};
  cudaError_t e = cudaMemcpyAsync(state, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(hist, 0, 2048 * sizeof(unsigned), st)) != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (n + 255) / 256;
  const int hgrid = (int)std::max<long long>(1, std::min<long long>(want, (long long)nsm * 4));
  const int shifts[3] = {21, 10, 0}, bits[3] = {11, 11, 10};
  for (int p = 0; p < 3; ++p) {
    select_hist_kernel<<<hgrid, 256, 0, st>>>(v, n, state, shifts[p], bits[p], hist);
    select_find_kernel<<<1, 1024, 0, st>>>(hist, bits[p], shifts[p], state);
  }
  const int nblk = (int)((n + kSelChunk - 1) / kSelChunk);
  select_count_kernel<<<nblk, kSelBlock, 0, st>>>(v, n, state, cnt);
  select_scan_kernel<<<1, 32, 0, st>>>(cnt, nblk);
  select_write_kernel<<<nblk, kSelBlock, 0, st>>>(v, n, state, cnt, k, idx);
  return cudaGetLastError();
}

curob_status predict_impl(curob_surrogate s, const float* x, long long N, float* out,
                          cudaStream_t st) {
  CUtensorMap mA1, mA2;
  for (long long off = 0; off < N; off += s->chunk) {
    const int rows = (int)std::min<long long>(s->chunk, N - off);
    mlp_prep_kernel<<<(rows + 31) / 32, 256, 0, st>>>(x + off * kSurIn, rows, nullptr, 0.f, 0.f,
                                                       1.f, s->Uc, nullptr, 0, nullptr);
    if (!make_map(&mA1, s->Uc, kSurInPad, rows, kSurInPad * 2, kTile) ||
        !make_map(&mA2, s->H1c, kSurH, rows, kSurH * 2, kTile))
      return fail("tensor map encoding (predict)");
    GemmArgs g{};
    g.status = s->d_status;
    g.M = rows;
    g.N = kSurH;
    g.kstages = kSurInPad / 32;
    g.bias = s->master + kOffB1;
    g.H = s->H1c;
    const int tiles = (rows + kTile - 1) / kTile;
    cudaError_t e;
    if ((e = launch_gemm<EPI_L1_INFER>(mA1, s->mW1, g, tiles, 1, st)) != cudaSuccess)
      return fail("predict layer 1", e);
    g.kstages = kSurH / 32;
    g.bias = s->master + kOffB2;
    g.w3 = s->w3b;
    g.b3 = s->master + kOffB3;
    g.out = out + off;
    g.out_scale = s->sd;
    g.out_shift = s->mu;
    if ((e = launch_gemm<EPI_L2_INFER>(mA2, s->mW2, g, tiles, 1, st)) != cudaSuccess)
      return fail("predict layer 2", e);
  }
  return CUROB_OK;
}

bool sm10x() {
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  return major == 10;
}

}  // namespace

extern "C" {

const char* curob_last_error(void) { return g_last_error; }

curob_status curob_surrogate_create(int max_batch, uint64_t seed, curob_surrogate* out) {
  if (!out) return CUROB_ERR_NULL_POINTER;
  *out = nullptr;
  if (max_batch < kTile || max_batch % kTile != 0 || max_batch > (1 << 20))
    return CUROB_ERR_INVALID_ARGUMENT;
  if (!sm10x()) return CUROB_ERR_UNSUPPORTED;
  curob_surrogate s = new curob_surrogate_st();
  s->max_batch = max_batch;
  s->chunk = 65536;
  const size_t B = (size_t)max_batch, tiles = B / kTile;
  bool ok = dalloc(&s->master, kSurParams) && dalloc(&s->mom1, kSurParams) &&
            dalloc(&s->mom2, kSurParams) && dalloc(&s->grad, kSurParams) &&
            dalloc(&s->W1b, kSurH * kSurInPad) && dalloc(&s->W2b, kSurH * kSurH) &&
            dalloc(&s->W2tb, kSurH * kSurH) && dalloc(&s->w3b, kSurH) &&
            dalloc(&s->U, B * kSurInPad) && dalloc(&s->UT, B * kSurInPad) &&
            dalloc(&s->H1, B * kSurH) && dalloc(&s->H1T, B * kSurH) && dalloc(&s->D2, B * kSurH) &&
            dalloc(&s->D2T, B * kSurH) && dalloc(&s->D1T, B * kSurH) &&
            dalloc(&s->G1D, B * kSurH) && dalloc(&s->T, B) &&
            dalloc(&s->pW1, tiles * kSurH * kSurInPad) && dalloc(&s->pW2, tiles * kSurH * kSurH) &&
            dalloc(&s->pb1, tiles * kSurH) && dalloc(&s->pv2, tiles * 2 * kSurH) &&
            dalloc(&s->ps2, tiles * 2) && dalloc(&s->stats, 2 + kStatBlocks) && dalloc(&s->d_status, 1) &&
            dalloc(&s->Uc, (size_t)s->chunk * kSurInPad) && dalloc(&s->H1c, (size_t)s->chunk * kSurH) &&
            ensure_select_scratch(s, 1 << 20) == CUROB_OK;
  ok = ok && cudaMemset(s->W1b, 0, sizeof(__nv_bfloat16) * kSurH * kSurInPad) == cudaSuccess &&
       cudaMemset(s->mom1, 0, sizeof(float) * kSurParams) == cudaSuccess &&
       cudaMemset(s->mom2, 0, sizeof(float) * kSurParams) == cudaSuccess &&
       cudaMemset(s->d_status, 0, sizeof(int)) == cudaSuccess;
  ok = ok && make_map(&s->mW1, s->W1b, kSurInPad, kSurH, kSurInPad * 2, kSurH) &&
       make_map(&s->mW2, s->W2b, kSurH, kSurH, kSurH * 2, kSurH) &&
       make_map(&s->mW2t, s->W2tb, kSurH, kSurH, kSurH * 2, kSurH);
  if (!ok) {
    cudaGetLastError();
    free_surrogate(s);
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  // PyTorch's default initialisation of a linear layer: weights and biases
  // uniform in +-1/sqrt(fan_in).
  std::vector<float> p(kSurParams);
  uint64_t rs = seed ^ 0x5u;
  auto fill = [&](int off, int count, int fan_in) {
    const double b = 1.0 / std::sqrt((double)fan_in);
    for (int i = 0; i < count; ++i) p[off + i] = (float)((2.0 * uniform01(rs) - 1.0) * b);
  };
  fill(kOffW1, kSurH * kSurIn, kSurIn);
  fill(kOffB1, kSurH, kSurIn);
  fill(kOffW2, kSurH * kSurH, kSurH);
  fill(kOffB2, kSurH, kSurH);
  fill(kOffW3, kSurH, kSurH);
  fill(kOffB3, 1, kSurH);
  if (cudaMemcpy(s->master, p.data(), sizeof(float) * kSurParams, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      refresh_copies(s, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    free_surrogate(s);
    return CUROB_ERR_CUDA;
  }
  *out = s;
  return CUROB_OK;
}

curob_status curob_surrogate_destroy(curob_surrogate s) {
  if (!s) return CUROB_ERR_NULL_POINTER;
  cudaDeviceSynchronize();
  free_surrogate(s);
  return CUROB_OK;
}

curob_status curob_surrogate_set_hyper(curob_surrogate s, float lr, float beta1, float beta2,
                                       float eps, float weight_decay) {
  if (!s) return CUROB_ERR_NULL_POINTER;
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f) || !(weight_decay >= 0.f))
    return CUROB_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mtx);
  s->lr = lr;
  s->beta1 = beta1;
  s->beta2 = beta2;
  s->eps = eps;
  s->wd = weight_decay;
  return CUROB_OK;
}

curob_status curob_surrogate_get_params(curob_surrogate s, float* host) {
  if (!s || !host) return CUROB_ERR_NULL_POINTER;
  std::lock_guard<std::mutex> lk(s->mtx);
  return cudaMemcpy(host, s->master, sizeof(float) * kSurParams, cudaMemcpyDeviceToHost) ==
                 cudaSuccess
             ? CUROB_OK
             : CUROB_ERR_CUDA;
}

curob_status curob_surrogate_set_params(curob_surrogate s, const float* host) {
  if (!s || !host) return CUROB_ERR_NULL_POINTER;
  std::lock_guard<std::mutex> lk(s->mtx);
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(s->master, host, sizeof(float) * kSurParams, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(s->mom1, 0, sizeof(float) * kSurParams) != cudaSuccess ||
      cudaMemset(s->mom2, 0, sizeof(float) * kSurParams) != cudaSuccess ||
      refresh_copies(s, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return CUROB_ERR_CUDA;
  s->t = 0;
  return CUROB_OK;
}

curob_status curob_surrogate_get_grads(curob_surrogate s, float* host) {
  if (!s || !host) return CUROB_ERR_NULL_POINTER;
  std::lock_guard<std::mutex> lk(s->mtx);
  if (cudaDeviceSynchronize() != cudaSuccess) return CUROB_ERR_CUDA;
  return cudaMemcpy(host, s->grad, sizeof(float) * kSurParams, cudaMemcpyDeviceToHost) ==
                 cudaSuccess
             ? CUROB_OK
             : CUROB_ERR_CUDA;
}

curob_status curob_surrogate_set_standardisation(curob_surrogate s, float mu, float sd) {
  if (!s) return CUROB_ERR_NULL_POINTER;
  if (!(sd > 0.f) || !std::isfinite(mu) || !std::isfinite(sd)) return CUROB_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mtx);
  s->mu = mu;
  s->sd = sd;
  return CUROB_OK;
}

curob_status curob_surrogate_get_standardisation(curob_surrogate s, float* mu, float* sd) {
  if (!s || !mu || !sd) return CUROB_ERR_NULL_POINTER;
  std::lock_guard<std::mutex> lk(s->mtx);
  *mu = s->mu;
  *sd = s->sd;
  return CUROB_OK;
}

curob_status curob_surrogate_standardise(curob_surrogate s, const float* f, long long n, float f_opt,
                                         curob_stream_t stream) {
  if (!s || !f) return CUROB_ERR_NULL_POINTER;
  if (n < 1) return CUROB_ERR_INVALID_ARGUMENT;
  if (!device_accessible(f)) return CUROB_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mtx);
  cudaStream_t st = (cudaStream_t)stream;
  double h[2];
  for (int pass = 0; pass < 2; ++pass) {
    mlp_stats_partial_kernel<<<kStatBlocks, kStatThreads, 0, st>>>(f, n, (double)f_opt,
                                                                    s->stats, pass,
                                                                    s->stats + 2);
    mlp_stats_final_kernel<<<1, kStatBlocks, 0, st>>>(s->stats + 2, n, pass, s->stats);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail("standardise", e);
  if (cudaMemcpyAsync(h, s->stats, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CUROB_ERR_CUDA;
  s->mu = (float)h[0];
  s->sd = h[1] > 0.0 ? (float)h[1] : 1.f;
  return CUROB_OK;
}

curob_status curob_surrogate_step(curob_surrogate s, const float* x, const float* f, int B,
                                  float f_opt, float lr, int update, float* loss_out,
                                  curob_stream_t stream) {
  if (!s || !x || !f) return CUROB_ERR_NULL_POINTER;
  if (B < kTile || B % kTile != 0) return CUROB_ERR_INVALID_ARGUMENT;
  if (B > s->max_batch) return CUROB_ERR_CAPACITY;
  if (update && !(lr > 0.f)) return CUROB_ERR_INVALID_ARGUMENT;
  if (!device_accessible(x) || !device_accessible(f) || (loss_out && !device_accessible(loss_out)))
    return CUROB_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mtx);
  cudaStream_t st = (cudaStream_t)stream;
  mlp_prep_kernel<<<B / 32, 256, 0, st>>>(x, B, f, f_opt, s->mu, 1.f / s->sd, s->U, s->UT,
                                          s->max_batch, s->T);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail("prep", e);
  return run_step(s, s->U, s->UT, s->max_batch, s->T, B, lr, update, loss_out, s->d_status, st);
}

curob_status curob_surrogate_fit(curob_surrogate s, const float* x, const float* f, long long n,
                                 float f_opt, int epochs, int batch, float lr_max,
                                 uint64_t shuffle_seed, float* loss_hist, curob_stream_t stream) {
  if (!s || !x || !f) return CUROB_ERR_NULL_POINTER;
  if (batch < kTile || batch % kTile != 0 || epochs < 1 || !(lr_max > 0.f) || n < batch)
    return CUROB_ERR_INVALID_ARGUMENT;
  if (batch > s->max_batch) return CUROB_ERR_CAPACITY;
  if (!device_accessible(x) || !device_accessible(f) || (loss_hist && !device_accessible(loss_hist)))
    return CUROB_ERR_INVALID_ARGUMENT;
  curob_status rc = curob_surrogate_standardise(s, f, n, f_opt, stream);
  if (rc != CUROB_OK) return rc;
  std::lock_guard<std::mutex> lk(s->mtx);
  cudaStream_t st = (cudaStream_t)stream;
  const long long nb = n / batch, npad = nb * batch;
  __nv_bfloat16 *U = nullptr, *UT = nullptr;
  float* T = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&U), sizeof(__nv_bfloat16) * npad * kSurInPad, st) !=
          cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&UT), sizeof(__nv_bfloat16) * npad * kSurInPad, st) !=
          cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&T), sizeof(float) * npad, st) != cudaSuccess) {
    cudaGetLastError();
    if (U) cudaFreeAsync(U, st);
    if (UT) cudaFreeAsync(UT, st);
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  mlp_prep_kernel<<<(unsigned)(npad / 32), 256, 0, st>>>(x, (int)npad, f, f_opt, s->mu,
                                                         1.f / s->sd, U, UT, npad, T);
  std::vector<long long> order(nb);
  uint64_t rs = shuffle_seed ^ 0xA5A5A5A5ull;
  const long long total = (long long)epochs * nb;
  const double lr_min = lr_max / 20.0;
  long long step = 0;
  int* status = s->d_status;
  for (int e = 0; e < epochs && rc == CUROB_OK; ++e) {
    for (long long i = 0; i < nb; ++i) order[i] = i;
    for (long long i = nb - 1; i > 0; --i) {  // Fisher-Yates
      const long long j = (long long)(uniform01(rs) * (double)(i + 1));
      std::swap(order[i], order[std::min(j, i)]);
    }
    for (long long i = 0; i < nb && rc == CUROB_OK; ++i, ++step) {
      const long long b = order[i];
      const double lr = lr_min + 0.5 * (lr_max - lr_min) *
                                     (1.0 + std::cos(3.14159265358979323846 * (double)step / (double)total));
      rc = run_step(s, U + b * batch * kSurInPad, UT + b * batch, npad, T + b * batch, batch,
                    (float)lr, 1, loss_hist ? loss_hist + step : nullptr, status, st);
    }
  }
  cudaFreeAsync(U, st);
  cudaFreeAsync(UT, st);
  cudaFreeAsync(T, st);
  return rc;
}

curob_status curob_surrogate_predict(curob_surrogate s, const float* x, long long N, float* out,
                                     curob_stream_t stream) {
  if (!s) return CUROB_ERR_NULL_POINTER;
  if (N < 0) return CUROB_ERR_INVALID_ARGUMENT;
  if (N == 0) return CUROB_OK;
  if (!x || !out) return CUROB_ERR_NULL_POINTER;
  if (!device_accessible(x) || !device_accessible(out)) return CUROB_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mtx);
  return predict_impl(s, x, N, out, (cudaStream_t)stream);
}

curob_status curob_surrogate_device_status(curob_surrogate s, curob_stream_t stream) {
  if (!s) return CUROB_ERR_NULL_POINTER;
  std::lock_guard<std::mutex> lk(s->mtx);
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CUROB_ERR_CUDA;
  int st = 0;
  int* p = s->d_status;
  if (cudaMemcpy(&st, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CUROB_ERR_CUDA;
  if (st != DEV_OK) {
    cudaMemset(p, 0, sizeof(int));
    return st == DEV_TIMEOUT ? CUROB_ERR_DEVICE_TIMEOUT : CUROB_ERR_CUDA;
  }
  return CUROB_OK;
}

curob_status curob_select_smallest(const float* v, long long N, int k, int* idx,
                                   curob_stream_t stream) {
  if (N < 0 || k < 0 || k > N) return CUROB_ERR_INVALID_ARGUMENT;
  if (k == 0) return CUROB_OK;
  if (!v || !idx) return CUROB_ERR_NULL_POINTER;
  if (!device_accessible(v) || !device_accessible(idx)) return CUROB_ERR_INVALID_ARGUMENT;
  if (N > (1LL << 31) - 1) return CUROB_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const long long nblk = (N + kSelChunk - 1) / kSelChunk;
  void* scratch = nullptr;
  const size_t bytes = 2048 * sizeof(unsigned) + 4 * sizeof(uint32_t) + 2 * nblk * sizeof(int);
  if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  unsigned* hist = static_cast<unsigned*>(scratch);
  uint32_t* state = reinterpret_cast<uint32_t*>(hist + 2048);
  int* cnt = reinterpret_cast<int*>(state + 4);
  cudaError_t e = select_launch(v, N, k, idx, hist, state, cnt, st);
  cudaFreeAsync(scratch, st);
  return e == cudaSuccess ? CUROB_OK : CUROB_ERR_CUDA;
}

curob_status curob_gather_rows(const float* x, int D, const int* idx, int k, float* out,
                               curob_stream_t stream) {
  if (D < 1 || k < 0) return CUROB_ERR_INVALID_ARGUMENT;
  if (k == 0) return CUROB_OK;
  if (!x || !idx || !out) return CUROB_ERR_NULL_POINTER;
  if (!device_accessible(x) || !device_accessible(idx) || !device_accessible(out))
    return CUROB_ERR_INVALID_ARGUMENT;
  gather_rows_kernel<<<std::min(k, 65535), 128, 0, (cudaStream_t)stream>>>(x, D, idx, k, out);
  return cudaGetLastError() == cudaSuccess ? CUROB_OK : CUROB_ERR_CUDA;
}

curob_status curob_surrogate_screen(curob_surrogate s, int fid, const float* pool, long long N,
                                    int k, float* pred, int* idx, float* x_sel, float* f_sel,
                                    curob_stream_t stream) {
  if (!s) return CUROB_ERR_NULL_POINTER;
  if (N < 1 || k < 1 || k > N) return CUROB_ERR_INVALID_ARGUMENT;
  if (!pool || !pred || !idx || !x_sel || !f_sel) return CUROB_ERR_NULL_POINTER;
  int D = 0;
  int maxc = 0;
  curob_status rc = curob_get_config(&D, &maxc);
  if (rc != CUROB_OK) return rc;
  if (D != kSurIn) return CUROB_ERR_INVALID_DIM;
  if (k > maxc) return CUROB_ERR_CAPACITY;
  if (!device_accessible(pool) || !device_accessible(pred) || !device_accessible(idx) ||
      !device_accessible(x_sel) || !device_accessible(f_sel))
    return CUROB_ERR_INVALID_ARGUMENT;
  if (N > (1LL << 31) - 1) return CUROB_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  {
    std::lock_guard<std::mutex> lk(s->mtx);
    rc = predict_impl(s, pool, N, pred, st);
    if (rc != CUROB_OK) return rc;
    rc = ensure_select_scratch(s, N);
    if (rc != CUROB_OK) return rc;
    if (select_launch(pred, N, k, idx, s->hist, s->sel_state, s->sel_cnt, st) != cudaSuccess)
      return CUROB_ERR_CUDA;
  }
  rc = curob_gather_rows(pool, kSurIn, idx, k, x_sel, stream);
  if (rc != CUROB_OK) return rc;
  return curob_evaluatef(fid, x_sel, k, f_sel, stream);
}

}  // extern "C"

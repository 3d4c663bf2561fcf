// curob_mma.cu -- tensor-core evaluator of curob_evaluatef (sm_103a).
//
// The block rotation z_b = R_b y_b of the General Setup is a dense
// contraction per block: for a tile of 128 candidates, Z_b (128 x n_b) =
// Y_b (128 x n_b) R_b^T.  It runs on tcgen05 in split precision:
//   TF32X3: y = yh + yl, R = Rh + Rl (TF32 halves), Z = Yh Rh + Yh Rl + Yl Rh
//   BF16X3: the same with BF16 halves,
// accumulated in FP32 in tensor memory (TMEM), then transformed and reduced
// by the epilogue warps straight out of TMEM.
//
// Warp roles of one CTA (one tile of 128 candidates, 1 CTA per SM):
//   warps 0-3  producers: gather x at the block's variables (S_b), take the
//              shift y = x - o in double-float (exact TwoSum, then the low
//              word of o), split y into hi/lo and store the A operand in the
//              64-byte-swizzled K-major layout the tensor core reads;
//   warps 4-7  epilogue: thread t owns candidate row t (TMEM lane t), loads
//              its z row 32 columns at a time (tcgen05.ld), applies
//              z = s z + c, the per-variable transform and the running sums
//              (FP32 per 32 columns, FP64 across), closes functions, mixes
//              composition members (FP64) and writes f;
//   warp 8     allocates TMEM and issues the MMAs (one elected lane);
//   warp 9     loads the B operand (R_b hi/lo, pre-laid-out in global memory
//              in exactly the shared-memory image) with one bulk copy per
//              stage (cp.async.bulk, the TMA engine).
// Stages of K (16 TF32 or 32 BF16 columns = 64 bytes per row) rotate through
// shared memory under full/empty mbarriers; the accumulator is handed from
// the MMA warp to the epilogue and back under tmem_full/tmem_empty.  Every
// wait is bounded: past ~2 s it raises DEV_TIMEOUT in the status word, the
// CTA stops, and TMEM is freed before exit.
#include <cuda_bf16.h>

#include <algorithm>

#include "curob_mma.hpp"

namespace curob {
namespace {

constexpr int kTileM = 128;
constexpr int kThreads = 320;
constexpr int kRowBytes = 64;                 // one K-stage row: 64 B (SW64)
constexpr int kATileBytes = kTileM * kRowBytes;  // 8 KB per hi/lo
constexpr unsigned long long kTimeoutNs = 2000000000ull;
constexpr int kMaxNpad = 512;                 // TMEM columns

// -------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on the phase of `parity`; false when the CTA aborts or the
// wait exceeds kTimeoutNs (then the status word gets DEV_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kTimeoutNs) {
      *abort_flag = 1;
      atomicExch(status, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
template <bool kBf16>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  if constexpr (kBf16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}
// 32 lanes x 32 consecutive FP32 columns: thread i of the warp gets row
// (its TMEM lane) columns [col, col+32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, rows of 64 B,
// 8-row groups 512 B apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                     // LBO (unused for swizzled K-major)
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;  // SBO
  d |= (uint64_t)1u << 46;                     // version
  d |= (uint64_t)4u << 61;                     // SWIZZLE_64B
  return d;
}
// Instruction descriptor: FP32 accumulator, A/B format (TF32 = 2, BF16 = 1),
// both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_make(uint32_t fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Byte offset of element (row, byte-in-row) in the 64-byte-swizzled image:
// the 16-byte chunk index (bits 4-5) XOR bits 7-8 of the linear offset.
__host__ __device__ __forceinline__ uint32_t swz64(uint32_t row, uint32_t byte_in_row) {
  uint32_t off = row * kRowBytes + byte_in_row;
  return off ^ (((off >> 7) & 3u) << 4);
}

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// x - o with o = ohi + olo: TwoSum(x, -ohi) is exact, the low word follows.
__device__ __forceinline__ float shift_ff(float x, float ohi, float olo) {
  float s = __fsub_rn(x, ohi);
  float bb = __fsub_rn(s, x);
  float err = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(-ohi, bb));
  return __fadd_rn(s, __fsub_rn(err, olo));
}

struct MmaArgs {
  Tables tb;
  Function F;
  const float* x;
  float* out;
  int N;
  const float* ohi;      // o[S[k]] high words per component
  const float* olo;      // low words
  const uint8_t* img;    // B images (TF32 or BF16 pool)
  int nstage;
  int stage_bytes;       // A hi + A lo + B hi + B lo
  int b_bytes_max;
};

// -------------------------------------------------------------- the kernel
template <bool kBf16>
__global__ void __launch_bounds__(kThreads, 1) mma_eval_kernel(MmaArgs args) {
  constexpr int kKs = kBf16 ? 32 : 16;          // K columns per stage
  constexpr int kEl = kBf16 ? 2 : 4;            // bytes per element
  constexpr int kMmaK = kBf16 ? 16 : 8;         // K per MMA instruction
  constexpr int kKsteps = kKs / kMmaK;          // 2
  constexpr uint32_t kFmt = kBf16 ? 1u : 2u;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // stage bases must sit on 1024-byte boundaries (swizzle atoms)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const Tables& tb = args.tb;
  const Function& F = args.F;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // layout: [stages][ctrl]
  uint8_t* stages = smem;
  uint8_t* ctrl = smem + (size_t)args.nstage * args.stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl);
  uint64_t* empty = full + args.nstage;
  uint64_t* tmem_full = empty + args.nstage;
  uint64_t* tmem_empty = tmem_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* rowG = reinterpret_cast<double*>(ctrl + 256);        // [kMaxComponents][128]
  double* rowD2 = rowG + kMaxComponents * kTileM;             // [kMaxComponents][128]

  if (threadIdx.x == 0) {
    for (int s = 0; s < args.nstage; ++s) {
      mbar_init(&full[s], 5);   // 4 producer warps + the B loader's expect_tx
      mbar_init(&empty[s], 1);  // one tcgen05.commit
    }
    mbar_init(tmem_full, 1);
    mbar_init(tmem_empty, 4);  // the 4 epilogue warps
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kMaxNpad));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const long long row0 = (long long)blockIdx.x * kTileM;
  const int D = tb.D;

  if (warp < 4) {
    // ------------------------------------------------------------ producers
    // thread = candidate row r of the tile: per stage it gathers its row's
    // kKs variables, shifts, splits and stores one 64-byte row of A_hi/A_lo;
    // it also sums ||x - o||^2 of its row for the composition weights.
    const int r = warp * 32 + lane;
    const long long grow = row0 + r;
    const bool vrow = grow < args.N;
    const float* xrow = args.x + (vrow ? grow : 0) * (long long)D;
    uint32_t it = 0;
    for (int ci = 0; ci < F.ncomp && !*abort_flag; ++ci) {
      const Component C = tb.comp[F.comp0 + ci];
      const int* S = tb.S + C.base;
      const float* ohi = args.ohi + C.base;
      const float* olo = args.olo + C.base;
      double d2 = 0.0;
      for (int si = 0; si < C.nseg && !*abort_flag; ++si) {
        const Segment sg = tb.seg[C.seg0 + si];
        const int nslab = (sg.npad + kKs - 1) / kKs;
        const int* Sb = S + sg.zoff;
        const float* oh = ohi + sg.zoff;
        const float* ol = olo + sg.zoff;
        for (int t = 0; t < nslab; ++t, ++it) {
          const int stage = it % args.nstage;
          const uint32_t ph = (it / args.nstage) & 1u;
          if (!mbar_wait(&empty[stage], ph ^ 1u, abort_flag, tb.status)) break;
          uint8_t* A_hi = stages + (size_t)stage * args.stage_bytes;
          uint8_t* A_lo = A_hi + kATileBytes;
          float y[kKs];
#pragma unroll
          for (int k = 0; k < kKs; ++k) {
            const int j = t * kKs + k;
            y[k] = 0.f;
            if (j < sg.n && vrow) y[k] = shift_ff(__ldg(xrow + Sb[j]), oh[j], ol[j]);
          }
          float d2p = 0.f;
#pragma unroll
          for (int k = 0; k < kKs; ++k) d2p = fmaf(y[k], y[k], d2p);
          d2 += (double)d2p;
          // one 64-byte row = four 16-byte chunks, each stored whole
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint32_t off = swz64((uint32_t)r, (uint32_t)(c * 16));
            uint4 h, l;
            if constexpr (kBf16) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float a = y[c * 8 + 2 * q], b = y[c * 8 + 2 * q + 1];
                __nv_bfloat162 hh = __floats2bfloat162_rn(a, b);
                const float2 hf = __bfloat1622float2(hh);
                __nv_bfloat162 ll = __floats2bfloat162_rn(a - hf.x, b - hf.y);
                hw[q] = *reinterpret_cast<uint32_t*>(&hh);
                lw[q] = *reinterpret_cast<uint32_t*>(&ll);
              }
              h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            } else {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float a = y[c * 4 + q];
                hw[q] = to_tf32(a);
                lw[q] = to_tf32(a - __uint_as_float(hw[q]));
              }
              h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            *reinterpret_cast<uint4*>(A_hi + off) = h;
            *reinterpret_cast<uint4*>(A_lo + off) = l;
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[stage]);
        }
      }
      rowD2[ci * kTileM + r] = d2;
    }
  } else if (warp < 8) {
    // ------------------------------------------------------------- epilogue
    const int q = warp - 4;                 // TMEM lane quadrant
    const int r = q * 32 + lane;            // candidate row in the tile
    const uint32_t t_lane = tmem_base + ((uint32_t)(q * 32) << 16);
    uint32_t seg_it = 0;
    double a0 = 0, a1 = 0, a2 = 0, p = 1, gsum = 0;
    float zfirst = 0.f, zprev = 0.f;
    for (int ci = 0; ci < F.ncomp && !*abort_flag; ++ci) {
      const Component C = tb.comp[F.comp0 + ci];
      gsum = 0.0;
      for (int si = 0; si < C.nseg; ++si, ++seg_it) {
        const Segment sg = tb.seg[C.seg0 + si];
        if (!mbar_wait(tmem_full, seg_it & 1u, abort_flag, tb.status)) break;
        tc_fence_after();
        const int kind = sg.kind;
        const bool pairs = kind_has_pairs(kind);
        const float s = (float)sg.scale, c0 = (float)sg.offset, gnT = (float)sg.gn;
        const float kat_e = (kind == K_KATSUURA) ? (float)(10.0 / pow((double)sg.gn, 1.2)) : 0.f;
        const float* aux = tb.aux32 + (sg.aux_off >= 0 ? sg.aux_off : 0);
        const bool has_aux = sg.aux_off >= 0;
        if (sg.gfirst) {
          a0 = a1 = a2 = 0.0;
          p = 1.0;
        }
        for (int c = 0; c < sg.n; c += 32) {
          float v[32];
          tmem_ld32(t_lane + (uint32_t)c, v);
          Acc<float> part = acc_zero<float>();
          const int cend = min(32, sg.n - c);
          for (int k = 0; k < cend; ++k) {
            const float acc = v[k];
            const float u = acc * s;       // z before its offset
            const float z = u + c0;
            const int col = c + k;
            elem_term_f32(kind, z, u, sg.gpos + col, gnT, has_aux ? aux[col] : 0.f, kat_e, part);
            if (col == 0 && sg.gfirst) {
              zfirst = z;
            } else if (pairs) {
              part.a0 += pair_term<float>(kind, zprev, z);
            }
            zprev = z;
          }
          a0 += (double)part.a0;
          a1 += (double)part.a1;
          a2 += (double)part.a2;
          p *= (double)part.p;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tmem_empty);
        if (sg.glast) {
          if (kind_is_cyclic(kind)) a0 += (double)pair_term<float>(kind, zprev, zfirst);
          gsum += finalize_f32(kind, a0, a1, a2, p, sg.gn);
        }
      }
      rowG[ci * kTileM + r] = gsum;
    }
  } else if (warp == 8) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      uint32_t it = 0, seg_it = 0;
      for (int ci = 0; ci < F.ncomp && !*abort_flag; ++ci) {
        const Component C = tb.comp[F.comp0 + ci];
        for (int si = 0; si < C.nseg && !*abort_flag; ++si, ++seg_it) {
          const Segment sg = tb.seg[C.seg0 + si];
          const int nslab = (sg.npad + kKs - 1) / kKs;
          const int n0 = sg.npad > 256 ? 256 : sg.npad;  // N split: <= 256 per MMA
          const int n1 = sg.npad - n0;
          const uint32_t id0 = idesc_make(kFmt, kTileM, (uint32_t)n0);
          const uint32_t id1 = idesc_make(kFmt, kTileM, (uint32_t)(n1 > 0 ? n1 : 16));
          if (!mbar_wait(tmem_empty, (seg_it & 1u) ^ 1u, abort_flag, tb.status)) break;
          tc_fence_after();
          bool ok = true;
          for (int t = 0; t < nslab; ++t, ++it) {
            const int stage = it % args.nstage;
            const uint32_t ph = (it / args.nstage) & 1u;
            if (!mbar_wait(&full[stage], ph, abort_flag, tb.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a_hi = smem_u32(stages + (size_t)stage * args.stage_bytes);
            const uint32_t a_lo = a_hi + kATileBytes;
            const uint32_t b_hi = a_hi + 2 * kATileBytes;
            const uint32_t b_lo = b_hi + (uint32_t)(sg.npad * kRowBytes);
#pragma unroll
            for (int kk = 0; kk < kKsteps; ++kk) {
              const uint32_t ko = (uint32_t)(kk * kMmaK * kEl);  // 32 B per K step
              const uint64_t dah = sdesc_sw64(a_hi + ko), dal = sdesc_sw64(a_lo + ko);
              for (int h = 0; h < (n1 > 0 ? 2 : 1); ++h) {
                const uint32_t boff = (uint32_t)(h * n0 * kRowBytes) + ko;
                const uint64_t dbh = sdesc_sw64(b_hi + boff), dbl = sdesc_sw64(b_lo + boff);
                const uint32_t dt = tmem_base + (uint32_t)(h * n0);
                const uint32_t idd = h ? id1 : id0;
                const uint32_t accum = (t > 0 || kk > 0) ? 1u : 0u;
                tc_mma<kBf16>(dt, dah, dbh, idd, accum);
                tc_mma<kBf16>(dt, dah, dbl, idd, 1u);
                tc_mma<kBf16>(dt, dal, dbh, idd, 1u);
              }
            }
            tc_commit(&empty[stage]);  // frees the stage when these MMAs retire
          }
          if (!ok) break;
          tc_commit(tmem_full);  // accumulator of this block complete
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- B loads
    if (lane == 0) {
      uint32_t it = 0;
      for (int ci = 0; ci < F.ncomp && !*abort_flag; ++ci) {
        const Component C = tb.comp[F.comp0 + ci];
        for (int si = 0; si < C.nseg && !*abort_flag; ++si) {
          const Segment sg = tb.seg[C.seg0 + si];
          const int nslab = (sg.npad + kKs - 1) / kKs;
          const uint32_t bytes = (uint32_t)(2 * sg.npad * kRowBytes);
          // img_off counts floats; a block's BF16 image follows its TF32 one
          const long long tf32_floats = (long long)((sg.npad + 15) / 16) * 2 * sg.npad * kRowBytes / 4;
          const uint8_t* src = args.img + ((size_t)sg.img_off + (kBf16 ? tf32_floats : 0)) * 4;
          for (int t = 0; t < nslab; ++t, ++it) {
            const int stage = it % args.nstage;
            const uint32_t ph = (it / args.nstage) & 1u;
            if (!mbar_wait(&empty[stage], ph ^ 1u, abort_flag, tb.status)) break;
            uint8_t* dst = stages + (size_t)stage * args.stage_bytes + 2 * kATileBytes;
            mbar_arrive_expect_tx(&full[stage], bytes);
            bulk_g2s(dst, src + (size_t)t * bytes, bytes, &full[stage]);
          }
        }
      }
    }
    __syncwarp();
  }

  // drain: every issued MMA has been consumed by the epilogue (or the CTA
  // aborted); write f, free TMEM.
  tc_fence_before();
  __syncthreads();
  if (warp >= 4 && warp < 8 && !*abort_flag) {
    const int r = (warp - 4) * 32 + lane;
    const long long grow = row0 + r;
    if (grow < args.N) {
      double f;
      if (F.composition) {
        double G[kMaxComponents], d2v[kMaxComponents];
        for (int ci = 0; ci < F.ncomp; ++ci) {
          G[ci] = rowG[ci * kTileM + r];
          d2v[ci] = rowD2[ci * kTileM + r];
        }
        f = compose(tb.comp + F.comp0, F.ncomp, G, d2v, D);
      } else {
        f = rowG[r];
      }
      args.out[grow] = (float)(f + kFopt);
    }
  }
  if (warp == 8) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kMaxNpad));
  }
}

// ----------------------------------------------------- operand image builder
// For one block (rotated or identity) writes, per K-stage t, the hi image
// (npad rows x 64 B, swizzled) followed by the lo image.  R entries beyond n
// are zero.  Split from FP64: hi = round(R), lo = round(R - hi).
struct ImgJob {
  long long r_off;     // FP64 block (or -1 for identity)
  long long img_off;   // destination, in floats (4-byte units)
  int n, npad;
};

template <bool kBf16>
__global__ void build_image_kernel(const ImgJob* jobs, const double* R, uint8_t* img) {
  constexpr int kKs = kBf16 ? 32 : 16;
  constexpr int kEl = kBf16 ? 2 : 4;
  const ImgJob J = jobs[blockIdx.x];
  const int nslab = (J.npad + kKs - 1) / kKs;
  const long long total = (long long)nslab * J.npad * kKs;
  uint8_t* base = img + (size_t)J.img_off * 4;
  const uint32_t slab_bytes = (uint32_t)(2 * J.npad * kRowBytes);
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int t = (int)(e / ((long long)J.npad * kKs));
    const int rem = (int)(e - (long long)t * J.npad * kKs);
    const int row = rem / kKs, k = rem - row * kKs;
    const int col = t * kKs + k;
    double v = 0.0;
    if (row < J.n && col < J.n) v = (J.r_off >= 0) ? R[J.r_off + (long long)row * J.n + col]
                                                   : (row == col ? 1.0 : 0.0);
    uint8_t* hi = base + (size_t)t * slab_bytes;
    uint8_t* lo = hi + J.npad * kRowBytes;
    const uint32_t off = swz64((uint32_t)row, (uint32_t)(k * kEl));
    if constexpr (kBf16) {
      __nv_bfloat16 h = __double2bfloat16(v);
      __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
      *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
      *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
    } else {
      uint32_t h = to_tf32((float)v);
      uint32_t l = to_tf32((float)(v - (double)__uint_as_float(h)));
      *reinterpret_cast<uint32_t*>(hi + off) = h;
      *reinterpret_cast<uint32_t*>(lo + off) = l;
    }
  }
}

__global__ void split_o_kernel(const double* operm, float* ohi, float* olo, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double o = operm[i];
    const float h = (float)o;
    ohi[i] = h;
    olo[i] = (float)(o - (double)h);
  }
}

int npad_of(int n) { return (n + 31) / 32 * 32; }

// bytes of one block's image (both precisions use the same byte count per
// element pair: TF32 slabs of 16 x 4 B, BF16 slabs of 32 x 2 B)
long long image_floats(int npad) {
  const long long slabs16 = (npad + 15) / 16;
  return slabs16 * 2LL * npad * kRowBytes / 4;
}

size_t stage_bytes_for(int npad_max) { return 2 * kATileBytes + 2 * (size_t)npad_max * kRowBytes; }

}  // namespace

// ------------------------------------------------------------- host side
curob_status mma_prepare(MmaPlan& p, std::vector<Segment>& segs, const Tables& tb, float* prev) {
  (void)prev;
  mma_release(p);
  int dev = 0, cc_major = 0, cc_minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
  p.ready = false;
  // layout: per segment, a TF32 image then a BF16 image of the same size
  long long off = 0;
  for (Segment& s : segs) {
    s.npad = npad_of(s.n);
    if (s.npad > kMaxNpad) {
      s.img_off = -1;
      continue;
    }
    s.img_off = off;
    off += 2 * image_floats(s.npad);
  }
  p.img_floats = off;
  if (off > 0 && cudaMalloc(&p.img, sizeof(float) * (size_t)off) != cudaSuccess) {
    cudaGetLastError();
    return CUROB_ERR_OUT_OF_MEMORY;
  }
  // o[S] split, one entry per (component, variable)
  int max_comp = 0;
  for (const Segment& s : segs) max_comp = std::max(max_comp, s.comp + 1);
  p.o_entries = (long long)max_comp * tb.D;
  if (cudaMalloc(&p.ohi, sizeof(float) * (size_t)std::max<long long>(p.o_entries, 1)) != cudaSuccess ||
      cudaMalloc(&p.olo, sizeof(float) * (size_t)std::max<long long>(p.o_entries, 1)) != cudaSuccess) {
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
  std::vector<ImgJob> jobs16, jobs32;
  for (int id : ids) {
    const Segment& s = segs[id];
    if (s.img_off < 0) continue;
    ImgJob J;
    J.r_off = s.identity ? -1 : s.r_off;
    J.n = s.n;
    J.npad = s.npad;
    J.img_off = s.img_off;
    jobs32.push_back(J);
    J.img_off = s.img_off + image_floats(s.npad);
    jobs16.push_back(J);
  }
  if (!jobs32.empty()) {
    ImgJob* d = nullptr;
    const size_t bytes = sizeof(ImgJob) * jobs32.size();
    if (cudaMalloc(&d, 2 * bytes) != cudaSuccess) return CUROB_ERR_OUT_OF_MEMORY;
    cudaError_t e = cudaMemcpy(d, jobs32.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + jobs32.size(), jobs16.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      build_image_kernel<false><<<(unsigned)jobs32.size(), 256>>>(d, tb.R, (uint8_t*)p.img);
      build_image_kernel<true><<<(unsigned)jobs16.size(), 256>>>(d + jobs32.size(), tb.R,
                                                                 (uint8_t*)p.img);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d);
    if (e != cudaSuccess) return CUROB_ERR_CUDA;
  }
  if (p.o_entries > 0) {
    split_o_kernel<<<256, 256>>>(tb.operm, p.ohi, p.olo, p.o_entries);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      return CUROB_ERR_CUDA;
  }
  return CUROB_OK;
}

void mma_release(MmaPlan& p) {
  cudaFree(p.img);
  cudaFree(p.ohi);
  cudaFree(p.olo);
  p.img = nullptr;
  p.ohi = p.olo = nullptr;
  p.img_floats = 0;
  p.o_entries = 0;
  p.ready = false;
}

bool mma_supports(const MmaPlan& p, const Function& F) {
  return p.ready && F.max_n >= 16 && F.max_n <= kMaxNpad;
}

int mma_auto_mode(const MmaPlan& p, const Function& F) {
  (void)p;
  // FP32 accumulation in TMEM truncates: |z| shrinks by ~2e-6 relative over
  // a 334-long block, too much for the kinds that magnify z errors.
  return F.sensitive ? CUROB_PRECISION_SIMT : CUROB_PRECISION_TF32X3;
}

cudaError_t launch_mma(const MmaPlan& p, const Tables& tb, const Function& F, bool bf16,
                       const float* x, int N, float* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const int npad_max = npad_of(F.max_n);
  const size_t sb = stage_bytes_for(npad_max);
  const size_t ctrl = 256 + 2 * sizeof(double) * kMaxComponents * kTileM;
  int nstage = (int)std::min<size_t>(4, (219 * 1024 - ctrl) / sb);
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
  a.nstage = nstage;
  a.stage_bytes = (int)sb;
  a.b_bytes_max = 2 * npad_max * kRowBytes;
  // the BF16 image of a block sits image_floats(npad) floats after its TF32 one
  cudaError_t e;
  if (bf16) {
    e = cudaFuncSetAttribute(mma_eval_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    mma_eval_kernel<true><<<(unsigned)((N + kTileM - 1) / kTileM), kThreads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(mma_eval_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    mma_eval_kernel<false><<<(unsigned)((N + kTileM - 1) / kTileM), kThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace curob

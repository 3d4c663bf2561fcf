// curob_device.cuh -- device-side descriptors and per-function arithmetic of
// the cuROB benchmark (Ding & Tan, "A CUDA-Based Real Parameter Optimization
// Benchmark").  Shared by every kernel of libcurob.
//
// An instance of function `fid` is a list of components (one, or N for a
// composition, Sec. 6 Eq. composition).  A component is a list of segments:
// a segment is one rotation block b of the General Setup (or one block i of a
// hybrid, Sec. 5 Eq. hybrid): z_b = s * R_b * (x - o)[S_b] + c.  Segments are
// grouped into basic functions G: a plain function's G spans all three blocks
// of its component; each hybrid block is a G of its own, of dimension n_i.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace curob {

constexpr int kNumFunctions = 37;
constexpr int kMaxComponents = 5;
constexpr double kFopt = 100.0;  // Table 1: f_opt = 100 for every function
constexpr double kPi = 3.14159265358979323846;

// Basic functions, numbered as the Table 1 rows 0..22 they come from.
enum Kind : int {
  K_SPHERE = 0, K_ELLIPSOID, K_ELLIPTIC, K_DISCUS, K_CIGAR, K_POWERS,
  K_SHARPV, K_STEP, K_WEIERSTRASS, K_GRIEWANK, K_RASTRIGIN, K_SCHAFFER7,
  K_EGR, K_ROSENBROCK, K_SCHWEFEL, K_KATSUURA, K_LUNACEK, K_ACKLEY,
  K_HAPPYCAT, K_HGBAT, K_SCHAFFER6, K_COUNT
};

struct Segment {
  int n;          // variables in the block
  int zoff;       // first position of the block in the component's z and S
  int kind;       // basic function of the block
  int gn;         // dimension of that function (D, or n_i in a hybrid)
  int gpos;       // index of the block's first variable inside the function
  int gfirst;     // the block opens a function
  int glast;      // the block closes a function
  int identity;   // R_b = I (unrotated component)
  double scale;   // s of "z = R(s (x - o)) + c"
  double offset;  // c
  long long r_off;    // rotation block (n x n, row-major) in the rotation pools
  long long aux_off;  // per-variable table of the block (n entries)
  long long img_off;  // tensor-core operand image of R_b (floats)
  long long tau_off;  // row scales of R_b's integer slices (tensor-core EXACT)
  int npad;           // n rounded up to the tensor-core tile
  int comp;           // owning component (index into the component table)
  int hoff;           // heavy kinds: first column of the block among its function's
                      // heavy columns (tensor-core z scratch); -1 otherwise
  float kat_e;        // Katsuura: the exponent 10 / gn^1.2 (FP32 paths); 0 otherwise
};

struct Component {
  int seg0, nseg;     // its segments in the segment table
  long long base;     // offset of its o, S, o[S] vectors (D entries each)
  double sigma, lambda, bias;  // composition parameters (Sec. 6)
};

struct Function {
  int comp0, ncomp;
  int composition;
  int max_n;          // largest block of any component (sizes shared memory)
  int sensitive;      // has a kind whose value magnifies contraction error:
                      // Discus (10^6 z_1^2), Weierstrass (3^k phases),
                      // expanded Griewank-Rosenbrock (cos of g2 ~ 1e4),
                      // Katsuura (2^j phases)
  int sens_mask;      // bit c: component c has such a kind
  int hcols;          // variables of the function's heavy-kind blocks (kind_is_heavy)
  int nseg;           // segments of all its components (consecutive in the table)
  int nweier;         // of them, Weierstrass blocks
  int xcand;          // bit c: member c is unrotated and its kinds keep one sum
                      // (kind_from_x): it can be evaluated straight from x
};

// Device view of an initialised instance.
struct Tables {
  const Segment* seg;
  const Component* comp;
  const double* o;      // shift x^opt per component
  const int* S;         // variable indices in block order per component
  const double* operm;  // o[S[k]] per component
  const double* R;      // FP64 rotation blocks
  const float* R32;     // FP32 rounding of the rotation blocks (hi word)
  const float* R32lo;   // R - R32 rounded to FP32 (lo word)
  const double* Rt;     // the same three, each block column-major (small-population
  const float* R32t;    // kernels: lane i reads entry (i, j) at step j)
  const float* R32lot;
  const double* aux;    // per-variable tables (FP64)
  const float* aux32;   // per-variable tables (FP32)
  const float* img;     // tensor-core operand images
  int D;
  int* status;          // device-side error word (0 = ok)
};

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) -- counter-based RNG that
// the instance generator draws o, the permutation and the Gaussian entries
// from.  Counter = (word/4, purpose | block << 8, fid, component), key =
// (seed, 0), word `index % 4` of the block.
// ---------------------------------------------------------------------------
enum Purpose : int { P_SHIFT = 0, P_PERM = 1, P_GAUSS = 2 };

__host__ __device__ inline void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
    uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
#else
    unsigned __int128 p0 = (unsigned __int128)M0 * c[0];
    unsigned __int128 p1 = (unsigned __int128)M1 * c[2];
    uint64_t lo0 = (uint64_t)p0, hi0 = (uint64_t)(p0 >> 64);
    uint64_t lo1 = (uint64_t)p1, hi1 = (uint64_t)(p1 >> 64);
#endif
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += W0; k1 += W1;
  }
}

__host__ __device__ inline uint64_t rng_word(uint64_t seed, int purpose, int block, int fid,
                                             int comp, uint64_t index) {
  uint64_t c[4] = {index >> 2, (uint64_t)purpose | ((uint64_t)block << 8), (uint64_t)fid,
                   (uint64_t)comp};
  philox4x64_10(c, seed, 0);
  return c[index & 3];
}

// ---------------------------------------------------------------------------
// Per-function arithmetic.  Every basic function is "sum/product of per-
// variable terms, then a closing map", so a kernel walks z once and keeps four
// running values (a0, a1, a2: sums; p: product).  The neighbour-coupled
// functions (Schaffer F7, expanded Griewank-Rosenbrock, Rosenbrock, expanded
// Schaffer F6) add one term per consecutive pair (z_i, z_{i+1}); the two
// "expanded" ones close the cycle with (z_D, z_1).
// ---------------------------------------------------------------------------
template <typename T>
struct Acc {
  T a0, a1, a2, p;
};

template <typename T>
__host__ __device__ inline Acc<T> acc_zero() {
  return Acc<T>{T(0), T(0), T(0), T(1)};
}

__host__ __device__ constexpr bool kind_has_pairs(int k) {
  return k == K_SCHAFFER7 || k == K_EGR || k == K_ROSENBROCK || k == K_SCHAFFER6;
}
__host__ __device__ inline bool kind_is_cyclic(int k) { return k == K_EGR || k == K_SCHAFFER6; }
// Which of a1, a2 and p a kind's FP32 terms touch (a0 is always a sum);
// the others stay 0 or 1, so their FP64 accumulation can be skipped.
__host__ __device__ constexpr bool kind_uses_a1(int k) {
  return k == K_DISCUS || k == K_CIGAR || k == K_SHARPV || k == K_LUNACEK || k == K_ACKLEY ||
         k == K_HAPPYCAT || k == K_HGBAT;
}
__host__ __device__ constexpr bool kind_uses_a2(int k) { return k == K_LUNACEK || k == K_HGBAT; }
__host__ __device__ constexpr bool kind_uses_p(int k) { return k == K_GRIEWANK || k == K_KATSUURA; }
// Kinds whose terms feed one running sum only (no second sum, product or
// neighbour pair): an unrotated block of such a kind needs no contraction.
__host__ __device__ constexpr bool kind_from_x(int k) {
  return !kind_uses_a1(k) && !kind_uses_a2(k) && !kind_uses_p(k) && !kind_has_pairs(k);
}
__host__ __device__ inline bool kind_is_sensitive(int k) {
  return k == K_DISCUS || k == K_WEIERSTRASS || k == K_EGR || k == K_KATSUURA;
}
// Kinds whose per-variable term calls transcendentals with slow paths (large
// arguments, long series): many instructions per variable, so the
// tensor-core path evaluates them with more threads than its epilogue has.
__host__ __device__ constexpr bool kind_is_heavy(int k) {
  return k == K_POWERS || k == K_WEIERSTRASS || k == K_GRIEWANK || k == K_SCHAFFER7 ||
         k == K_EGR || k == K_SCHWEFEL || k == K_KATSUURA || k == K_SCHAFFER6;
}

// Math wrappers so one statement of each formula serves FP64 and FP32.
__device__ inline double m_cos(double v) { return cos(v); }
__device__ inline float m_cos(float v) { return cosf(v); }
__device__ inline double m_sin(double v) { return sin(v); }
__device__ inline float m_sin(float v) { return sinf(v); }
__device__ inline double m_exp(double v) { return exp(v); }
__device__ inline float m_exp(float v) { return expf(v); }
__device__ inline double m_pow(double a, double b) { return pow(a, b); }
__device__ inline float m_pow(float a, float b) { return powf(a, b); }
__device__ inline double m_sqrt(double v) { return sqrt(v); }
__device__ inline float m_sqrt(float v) { return sqrtf(v); }
__device__ inline double m_floor(double v) { return floor(v); }
__device__ inline float m_floor(float v) { return floorf(v); }
__device__ inline double m_rint(double v) { return rint(v); }
__device__ inline float m_rint(float v) { return rintf(v); }
__device__ inline double m_fmod(double a, double b) { return fmod(a, b); }
__device__ inline float m_fmod(float a, float b) { return fmodf(a, b); }
__device__ inline double m_fabs(double v) { return fabs(v); }
__device__ inline float m_fabs(float v) { return fabsf(v); }
__device__ inline double m_cospi(double v) { return cospi(v); }
__device__ inline float m_cospi(float v) { return cospif(v); }

// Sec. 4.9, Eq. basic_schwefel: g1(w) with the two out-of-range branches.
template <typename T>
__device__ inline T schwefel_g1(T w, T gn) {
  if (m_fabs(w) <= T(500)) return w * m_sin(m_sqrt(m_fabs(w)));
  if (w > T(500)) {
    T m = m_fmod(w, T(500));
    T t = w - T(500);
    return (T(500) - m) * m_sin(m_sqrt(T(500) - m)) - t * t / (T(10000) * gn);
  }
  T m = m_fmod(-w, T(500));
  T t = w + T(500);
  return (m - T(500)) * m_sin(m_sqrt(T(500) - m)) - t * t / (T(10000) * gn);
}

// Term of the pair (u, v) = (z_i, z_{i+1}) for the neighbour-coupled kinds.
template <typename T>
__device__ inline T pair_term(int kind, T u, T v) {
  switch (kind) {
    case K_SCHAFFER7: {  // Sec. 4.6: (1 + sin^2(50 w^0.2)) sqrt(w), w = |(u,v)|
      T w = m_sqrt(u * u + v * v);
      T t = m_sin(T(50) * m_pow(w, T(0.2)));
      return (T(1) + t * t) * m_sqrt(w);
    }
    case K_EGR: {  // Sec. 4.7: g3(g2(u, v))
      T a = u * u - v, b = u - T(1);
      T g2 = T(100) * (a * a) + b * b;
      return g2 * g2 / T(4000) - m_cos(g2) + T(1);
    }
    case K_ROSENBROCK: {  // Sec. 4.8: 100 (u^2 - v)^2 + (u - 1)^2
      T a = u * u - v, b = u - T(1);
      return T(100) * (a * a) + b * b;
    }
    case K_SCHAFFER6: {  // Sec. 4.16: g4(u, v)
      T r2 = u * u + v * v;
      T t = m_sin(m_sqrt(r2));
      T d = T(1) + T(0.001) * r2;
      return (t * t - T(0.5)) / (d * d) + T(0.5);
    }
    default:
      return T(0);
  }
}

// Weierstrass inner sum for one variable (Sec. 4.2): sum_{k=0}^{20}
// a^k cos(2 pi b^k (z + 1/2)), a = 1/2, b = 3.  FP64 evaluates the printed
// expression; FP32 carries the phase as frac(3^k (z + 1/2)) so that the
// argument of the cosine stays in [0, 1).
__device__ inline double weierstrass_inner(double z) {
  double s = 0.0, ak = 1.0, bk = 1.0;
  for (int k = 0; k <= 20; ++k) {
    s += ak * cos(2.0 * kPi * bk * (z + 0.5));
    ak *= 0.5;
    bk *= 3.0;
  }
  return s;
}
// FP32: the phase frac(3^k (z + 1/2)) is carried exactly as a 40-bit binary
// fraction (z is exact in it for |z| >= 2^-17), multiplied by 3 modulo 1 in
// integer arithmetic, so rounding adds no phase error however large 3^k is.
// Each term rounds the phase to 23 bits (error <= 2^-24 of a turn), which is
// the mantissa of a float in [2^23, 2^24): OR-ing it into 2^23 and
// subtracting 2^23 gives it exactly without an integer-to-float conversion;
// cos(2 pi t) = -cos(2 pi (t - 1/2)) with the argument in [-pi, pi].
__device__ inline float weierstrass_inner(float z) {
  const float az = fabsf(z);
  if (az >= 0x1p-9f && az <= 0x1p30f) {
    // Here z 2^32 is an integer (z's last bit weighs at least 2^-32), so the
    // fraction of (z + 1/2) is exact in 32 bits: the same phases and the same
    // 23-bit rounding as the 40-bit form below (whose low 8 bits are then
    // zero), with one 32-bit multiply per term.
    uint32_t P = (uint32_t)__float2ll_rn(z * 4294967296.0f) + 0x80000000u;  // (z + 1/2) 2^32
    float s = 0.f, ak = 1.f;
#pragma unroll
    for (int k = 0; k <= 20; ++k) {
      // the fraction's top 23 bits, rounded (a carry out of 32 bits wraps to 0)
      const unsigned b = (P + 256u) >> 9;
      const float t = __uint_as_float(0x4B000000u | b) - 8388608.0f;
      s = fmaf(-ak, __cosf(fmaf(t, 7.490140565847157e-07f, -3.14159265358979323846f)), s);
      ak *= 0.5f;
      P *= 3u;
    }
    return s;
  }
  const long long Z = __float2ll_rn(z * 1099511627776.0f);          // z 2^40
  unsigned long long P = (unsigned long long)(Z + 549755813888LL);   // (z + 1/2) 2^40
  float s = 0.f, ak = 1.f;
#pragma unroll
  for (int k = 0; k <= 20; ++k) {
    // bits 16..39 of P (the fraction's top 24), rounded to 23 (a carry out
    // of the field wraps to 0: the same point of the circle)
    const unsigned b = ((((unsigned)(P >> 16)) + 1u) >> 1) & 0x7FFFFFu;
    const float t = __uint_as_float(0x4B000000u | b) - 8388608.0f;   // b, exactly
    // 2 pi 2^-23 t - pi, one rounding
    s = fmaf(-ak, __cosf(fmaf(t, 7.490140565847157e-07f, -3.14159265358979323846f)), s);
    ak *= 0.5f;
    P *= 3ull;  // the low 40 bits hold frac(3^{k+1} (z + 1/2))
  }
  return s;
}

// Weierstrass constant sum_k a^k cos(2 pi b^k / 2), in the working precision.
template <typename T>
__device__ inline T weierstrass_const() {
  double c = 0.0, ak = 1.0, bk = 1.0;
  for (int k = 0; k <= 20; ++k) {
    c += ak * cos(2.0 * kPi * bk * 0.5);
    ak *= 0.5;
    bk *= 3.0;
  }
  return T(c);
}

// Katsuura inner sum (Sec. 4.11): sum_{j=1}^{32} |2^j z - [2^j z]| / 2^j.
template <typename T>
__device__ inline T katsuura_inner(T z) {
  // 2^j z and the division by 2^j are exact scalings: the reciprocal power
  // of two gives the same value as the division.
  T s = T(0), tj = T(1), itj = T(1);
#pragma unroll 8
  for (int j = 1; j <= 32; ++j) {
    tj = tj * T(2);
    itj = itj * T(0.5);
    T v = tj * z;
    s += m_fabs(v - m_rint(v)) * itj;
  }
  return s;
}
// FP32: the same terms from the signed fractional part f_j = 2^j z -
// rint(2^j z), carried as f_j = w - rint(w), w = 2 f_{j-1} (2^j z differs
// from w by an even integer): |w| <= 1, so w, its rounding (the 1.5 * 2^23
// addition rounds to the nearest integer, ties to even as rint) and w -
// rint(w) are all exact, and every term equals the direct one, without a
// round-to-integer instruction per term.
__device__ inline float katsuura_inner(float z) {
  constexpr float kRnd = 12582912.0f;  // 1.5 * 2^23
  float f = z - rintf(z);
  float s = 0.f, itj = 1.f;
#pragma unroll 8
  for (int j = 1; j <= 32; ++j) {
    const float w = f + f;
    const float r = (w + kRnd) - kRnd;
    f = w - r;
    itj = itj * 0.5f;
    s += fabsf(f) * itj;
  }
  return s;
}

// ---------------------------------------------------------------------------
// FP64 terms.  The FP64 path evaluates each variable's term(s) with exactly
// the expression of the formula, then sums them per candidate in index
// order, so that its sums round like a sequential evaluation of the printed
// formula.  Array a of a kind is a sum, except Griewank's a = 1 and
// Katsuura's a = 0, which are products.
// ---------------------------------------------------------------------------
__host__ __device__ inline int f64_num_terms(int kind) {
  switch (kind) {
    case K_GRIEWANK: case K_ACKLEY: case K_HAPPYCAT: case K_HGBAT: return 2;
    case K_LUNACEK: return 3;
    default: return 1;
  }
}
__host__ __device__ inline bool f64_term_is_product(int kind, int a) {
  return (kind == K_GRIEWANK && a == 1) || (kind == K_KATSUURA && a == 0);
}

// Term a of variable z (index gi in its function of dimension gn).  For the
// neighbour-coupled kinds the term is the pair (z, znext).
__device__ inline double term_f64(int kind, int a, double z, double znext, int gi, double gn,
                                  double aux, double kat_e) {
  switch (kind) {
    case K_SPHERE: case K_DISCUS: case K_CIGAR: case K_SHARPV: return z * z;
    case K_ELLIPSOID: return (double)(gi + 1) * (z * z);      // Sec. 3.2
    case K_ELLIPTIC: return aux * (z * z);                     // Sec. 3.3
    case K_POWERS: return pow(fabs(z), aux);                   // Sec. 3.6
    case K_STEP: { double t = floor(z + 0.5); return t * t; }  // Sec. 4.1
    case K_WEIERSTRASS: return weierstrass_inner(z);           // Sec. 4.2
    case K_GRIEWANK: return a == 0 ? z * z / 4000.0 : cos(z / aux);  // Sec. 4.3
    case K_RASTRIGIN: return z * z - 10.0 * cos(2.0 * kPi * z) + 10.0;  // Sec. 4.4
    case K_SCHWEFEL: return schwefel_g1(z + 420.9687462275036, gn);     // Sec. 4.9
    case K_KATSUURA: return pow(1.0 + (double)(gi + 1) * katsuura_inner(z), kat_e);  // 4.11
    case K_LUNACEK: {                                          // Sec. 4.12
      if (a == 0) { double u = z - 2.5; return u * u; }
      if (a == 1) { double v = z - (-2.5); return v * v; }
      return cos(2.0 * kPi * (z - 2.5));
    }
    case K_ACKLEY: return a == 0 ? z * z : cos(2.0 * kPi * z);  // Sec. 4.13
    case K_HAPPYCAT: case K_HGBAT: return a == 0 ? z * z : z;   // Sec. 4.14, 4.15
    default: return pair_term<double>(kind, z, znext);
  }
}

// ---------------------------------------------------------------------------
// FP32 terms (tensor-core and CUDA-core FP32 paths).  z is the transformed
// variable, u = z - c its value before the offset c (exact, no rounding of
// c), so that forms that cancel near the optimum can be rewritten in u:
//   HappyCat  sum z^2 - D           = sum u (u - 2)          (c = -1)
//             (sum z^2/2 + sum z)/D + 1/2 = sum u^2 / (2 D)
//   HGBat     (sum z^2)^2 - (sum z)^2 = sum z(z-1) * sum z(z+1)
//                                     = sum (u-1)(u-2) * sum (u-1) u
//   Lunacek   z - mu_1 = u,  z - mu_2 = u + 5                (c = 2.5)
// Cosines of 2 pi v reduce v exactly to [-1/2, 1/2] first (cos2pi_sfu).
// ---------------------------------------------------------------------------
// Modified Schwefel term 418.9829 - g1(z + c), c = 420.9687462275036, in
// FP32 without the cancellation that makes the sum over D such terms lose
// digits near the optimum: for |z| < 1 (so 0 < w = z + c <= 500),
//   g1(w) - g1(c) = 2 w cos((sqrt w + sqrt c)/2) sin(z / (2 (sqrt w + sqrt c)))
//                   + z sin(sqrt c),
// and 418.9829 - g1(c) = 1.27275662959398e-5 (constants to 40 digits).
// Elsewhere the plain expression with the SFU sine: its absolute error, a
// few 1e-4 per term at w ~ 500, is random from term to term and stays far
// below the tolerance of f, whose floor 1e-6 f_scale is about 0.4 for this
// function at D = 1000 (hybrids and compositions weight the term by their
// own lambda).  The careful form only where it matters keeps the warps of
// uniform candidates, nearly none of whose terms have |z| < 1, on one path.
__device__ inline float schwefel_term_f32(float z, float gn) {
  const float w = z + 420.96875f;  // sqrt and prefactor only: z enters exactly below
  if (fabsf(z) < 1.0f) {
    const float sc = 20.51752290671326630f;      // sqrt(c)
    const float ssc = 0.99528264515390726719f;   // sin(sqrt(c))
    const float sum = sqrtf(w) + sc;
    const float dg = 2.f * w * cosf(0.5f * sum) * sinf(0.5f * z * __frcp_rn(sum)) + z * ssc;
    return 1.2727566295939802e-5f - dg;
  }
  // |w| > 500 (or w <= 0): g1 of Eq. basic_schwefel with the remainder
  // m = |w| mod 500 taken exactly (|w| - 500 q is representable, q corrected
  // by one step) instead of by fmodf, and the penalty scaled by a reciprocal.
  // Far from the optimum the term is not a near-cancelling difference, so
  // the sine's argument (at most sqrt(500)) goes through the SFU: its
  // absolute error of a few 1e-6 stays far below the FP32 tolerance of f.
  const float wv = z + 420.9687462275036f;
  const float a = fabsf(wv);
  if (a <= 500.f) return 418.9829f - wv * __sinf(sqrtf(a));
  const float q = floorf(a * 0.002f);
  float m = fmaf(-500.f, q, a);
  if (m < 0.f) m += 500.f;
  else if (m >= 500.f) m -= 500.f;
  const float t = a - 500.f;
  const float g = (500.f - m) * __sinf(sqrtf(500.f - m));
  return 418.9829f - ((wv > 0.f ? g : -g) - t * t * __frcp_rn(10000.f * gn));
}

// cos(2 pi v) in FP32 for the cosine terms of Rastrigin, Lunacek and Ackley:
// v - rint(v) is exact (|r| <= 1/2; an integral v, e.g. every |v| >= 2^23,
// gives r = 0), and the SFU cosine of 2 pi r in [-pi, pi] has an absolute
// error of about 2^-21.4.  Over 1000 variables that stays more than ten
// times below the FP32 tolerance of f (an absolute floor of 1e-6 f_scale,
// with f_scale in the thousands for these functions at the box's scale),
// and it is a handful of instructions where cospif's reduction and
// polynomials are a few dozen on the epilogue's critical path.
__device__ __forceinline__ float cos2pi_sfu(float v) {
  const float r = v - rintf(v);
  return __cosf(6.2831853071795865f * r);
}

__device__ inline void elem_term_f32(int kind, float z, float u, int gi, float gn, float aux,
                                     float kat_e, Acc<float>& a) {
  switch (kind) {
    case K_SPHERE: a.a0 = fmaf(z, z, a.a0); break;
    case K_ELLIPSOID: a.a0 = fmaf((float)(gi + 1), z * z, a.a0); break;
    case K_ELLIPTIC: a.a0 = fmaf(aux, z * z, a.a0); break;
    case K_DISCUS: case K_CIGAR: case K_SHARPV:
      if (gi == 0) a.a1 = fmaf(z, z, a.a1); else a.a0 = fmaf(z, z, a.a0);
      break;
    case K_POWERS: a.a0 += powf(fabsf(z), aux); break;
    case K_STEP: { float t = floorf(z + 0.5f); a.a0 = fmaf(t, t, a.a0); } break;
    case K_WEIERSTRASS: a.a0 += weierstrass_inner(z); break;
    case K_GRIEWANK:
      a.a0 = fmaf(z, z * (1.0f / 4000.0f), a.a0);
      a.p *= cosf(z / aux);
      break;
    case K_RASTRIGIN: a.a0 += fmaf(z, z, 10.0f - 10.0f * cos2pi_sfu(z)); break;
    case K_SCHWEFEL: a.a0 += schwefel_term_f32(z, gn); break;
    case K_KATSUURA: a.p *= powf(fmaf((float)(gi + 1), katsuura_inner(z), 1.0f), kat_e); break;
    case K_LUNACEK: {
      float v = u + 5.0f;
      a.a0 = fmaf(u, u, a.a0);
      a.a1 = fmaf(v, v, a.a1);
      a.a2 += cos2pi_sfu(u);
    } break;
    case K_ACKLEY:
      a.a0 = fmaf(z, z, a.a0);
      a.a1 += cos2pi_sfu(z);
      break;
    case K_HAPPYCAT:
      a.a0 = fmaf(u, u - 2.0f, a.a0);
      a.a1 = fmaf(u, u, a.a1);
      break;
    case K_HGBAT:
      a.a0 = fmaf(u - 1.0f, u - 2.0f, a.a0);
      a.a1 = fmaf(u, u, a.a1);
      a.a2 = fmaf(u - 1.0f, u, a.a2);
      break;
    default: break;  // pair kinds: only pair terms
  }
}

// Closing map of each basic function; gn = its dimension.  Returns the value
// without f_opt.  Works in FP64 whatever the working precision.
__device__ inline double finalize(int kind, double a0, double a1, double a2, double p, int gn_i) {
  if (gn_i == 0) return 0.0;
  const double gn = (double)gn_i;
  switch (kind) {
    case K_DISCUS: return 1.0e6 * a1 + a0;                 // Sec. 3.4
    case K_CIGAR: return a1 + 1.0e6 * a0;                  // Sec. 3.5
    case K_SHARPV: return a1 + 100.0 * sqrt(a0);           // Sec. 3.7
    case K_POWERS: return sqrt(a0);                        // Sec. 3.6
    case K_WEIERSTRASS: return a0 - gn * weierstrass_const<double>();  // Sec. 4.2
    case K_GRIEWANK: return a0 - p + 1.0;                  // Sec. 4.3
    case K_SCHAFFER7: {                                    // Sec. 4.6
      if (gn_i < 2) return 0.0;
      double m = a0 / (gn - 1.0);
      return m * m;
    }
    case K_SCHWEFEL: return 418.9829 * gn - a0;            // Sec. 4.9
    case K_KATSUURA: {                                     // Sec. 4.11
      double c = 10.0 / (gn * gn);
      return c * p - c;
    }
    case K_LUNACEK: {                                      // Sec. 4.12
      double t2 = 1.0 * gn + 0.9 * a1;
      return (a0 < t2 ? a0 : t2) + 10.0 * (gn - a2);
    }
    case K_ACKLEY:                                         // Sec. 4.13
      return -20.0 * exp(-0.2 * sqrt(a0 / gn)) - exp(a1 / gn) + 20.0 + exp(1.0);
    case K_HAPPYCAT:                                       // Sec. 4.14
      return pow(fabs(a0 - gn), 0.25) + (0.5 * a0 + a1) / gn + 0.5;
    case K_HGBAT:                                          // Sec. 4.15
      return pow(fabs(a0 * a0 - a1 * a1), 0.5) + (0.5 * a0 + a1) / gn + 0.5;
    default:  // sphere, ellipsoid, elliptic, step, rastrigin, EGR, rosenbrock, F6
      return a0;
  }
}

// Closing map of the FP32 forms: HappyCat, HGBat and Modified Schwefel use
// the sums of elem_term_f32; every other kind closes as in finalize.
__device__ inline double finalize_f32(int kind, double a0, double a1, double a2, double p,
                                      int gn_i) {
  if (gn_i == 0) return 0.0;
  const double gn = (double)gn_i;
  if (kind == K_HAPPYCAT) return pow(fabs(a0), 0.25) + 0.5 * a1 / gn;
  if (kind == K_HGBAT) return sqrt(fabs(a0 * a2)) + 0.5 * a1 / gn;
  if (kind == K_SCHWEFEL) return a0;  // the terms already hold 418.9829 - g1
  // Weierstrass constant in closed form: cos(2 pi 3^k / 2) = cos(pi 3^k) = -1
  // (3^k is odd), so sum_{k=0}^{20} 2^-k cos(...) = -(2 - 2^-20); the FP64
  // path evaluates the printed series (21 FP64 cosines per candidate).
  if (kind == K_WEIERSTRASS) return a0 + gn * (2.0 - 0x1p-20);
  return finalize(kind, a0, a1, a2, p, gn_i);
}

// Composition (Sec. 6, Eq. composition and Eq. weight): sum_i omega_i
// (lambda_i G_i + bias_i), omega = w / sum w, w_i = exp(-d_i^2/(2 D sigma_i^2))
// / d_i; one-hot at the first i with d_i = 0.  FP64.
__device__ inline double compose(const Component* comps, int nc, const double* G, const double* d2,
                                 int D) {
  int hit = -1;
  for (int c = 0; c < nc; ++c)
    if (d2[c] == 0.0 && hit < 0) hit = c;
  if (hit >= 0) return comps[hit].lambda * G[hit] + comps[hit].bias;
  double w[kMaxComponents], W = 0.0;
  for (int c = 0; c < nc; ++c) {
    double s = comps[c].sigma;
    w[c] = (1.0 / sqrt(d2[c])) * exp(-d2[c] / (2.0 * (double)D * s * s));
    W += w[c];
  }
  double F = 0.0;
  if (W > 0.0) {
    for (int c = 0; c < nc; ++c) F += (w[c] / W) * (comps[c].lambda * G[c] + comps[c].bias);
    return F;
  }
  // all weights underflowed (far outside the box): the same ratio in logs
  double lw[kMaxComponents], mx = -1e300;
  for (int c = 0; c < nc; ++c) {
    double s = comps[c].sigma;
    lw[c] = -0.5 * log(d2[c]) - d2[c] / (2.0 * (double)D * s * s);
    mx = lw[c] > mx ? lw[c] : mx;
  }
  double Z = 0.0;
  for (int c = 0; c < nc; ++c) Z += exp(lw[c] - mx);
  for (int c = 0; c < nc; ++c) F += (exp(lw[c] - mx) / Z) * (comps[c].lambda * G[c] + comps[c].bias);
  return F;
}

// compose() by one warp: lane c < nc forms member c's weight (FP64 costs the
// same per warp instruction whatever the number of active lanes, so nc
// weights take the time of one); lane 0 adds them and the members' values in
// member order, as compose() does, so the value is the same.  Every lane of
// the warp calls it; the result is lane 0's.
__device__ inline double compose_warp(const Component* comps, int nc, const double* G,
                                      const double* d2, int D) {
  const int lane = threadIdx.x & 31;
  int hit = -1;
  for (int c = 0; c < nc; ++c)
    if (d2[c] == 0.0 && hit < 0) hit = c;
  if (hit >= 0) return comps[hit].lambda * G[hit] + comps[hit].bias;
  double w = 0.0;
  if (lane < nc) {
    const double s = comps[lane].sigma;
    w = (1.0 / sqrt(d2[lane])) * exp(-d2[lane] / (2.0 * (double)D * s * s));
  }
  double wc[kMaxComponents];
#pragma unroll
  for (int c = 0; c < kMaxComponents; ++c) wc[c] = __shfl_sync(0xffffffffu, w, c);
  double W = 0.0;
  for (int c = 0; c < nc; ++c) W += wc[c];
  if (!(W > 0.0)) return compose(comps, nc, G, d2, D);  // log-domain branch (far outside)
  double F = 0.0;
  for (int c = 0; c < nc; ++c) F += (wc[c] / W) * (comps[c].lambda * G[c] + comps[c].bias);
  return F;
}

// Device error codes written to Tables::status.
enum DeviceError : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD_ARG = 2 };

}  // namespace curob

/*
 * curob_oracle.c -- plain FP64 CPU oracle for the cuROB benchmark
 * (Ding & Tan, "A CUDA-Based Real Parameter Optimization Benchmark").
 *
 * TEST INFRASTRUCTURE ONLY: the independent reference the GPU library is
 * checked against.  Loaded by the tests, the smoke check and the CPU-baseline
 * leg of the benchmark script; never by the product path.  Shares no code
 * with the CUDA library.  Compile with -ffp-contract=off so that every
 * formula below is evaluated exactly as written, one rounding per operation.
 *
 * Every function is written straight from the paper's formula, in index
 * order, in FP64, with libm.  The rotation's dot products take one fused
 * multiply-add per term (C99 fma, exactly rounded on every platform), in
 * index order.  Readings of silent or garbled points:
 *   - functions are numbered by their Table 1 ID (the equation labels in the
 *     paper are left over from other suites);
 *   - f_opt = 100 for every function (Table 1 footer);
 *   - Sharp Valley's first term is z_1^2 (Sec. "Sharp Valley" prints z_i^2);
 *   - Ackley's sums run over z (the equation prints x, the text defines z);
 *   - Lunacek: z = R(0.1 (x - o)) + 2.5, so that f(o) = f_opt and the two
 *     funnels sit at mu_1*1 and mu_2*1 (the paper puts the 2.5 inside R);
 *   - Hybrid Function 2 has N = 3 (it lists three p's and three G's);
 *   - Composition Function 5 takes its G's in the printed list order;
 *   - a composition member not called "Rotated" is unrotated (R = I),
 *     "Expanded Schwefel" is the unrotated Modified Schwefel;
 *   - inside a hybrid, G_i uses its own scale and offset, and "D" inside
 *     G_i is n_i; an empty block (n_i = 0) contributes 0;
 *   - composition weights at x = o_i are the one-hot limit (first such i).
 * Parity unpinned: these readings, and the instance-generation choices
 * (Philox keying and counter layout, Fisher-Yates draw, Box-Muller branch,
 * Gram-Schmidt order), are choices the paper does not fix; they are checked
 * for self-consistency only.  Every formula itself is pinned by the CPU
 * tests (closed forms, f(x_opt) = f_opt, invariances, brute-force grids).
 */
#include "curob_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define F_OPT 100.0
#define PI_D 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 5).          */
/* ------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                          uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, &hi0, &lo0);
    mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { PURPOSE_SHIFT = 0, PURPOSE_PERM = 1, PURPOSE_GAUSS = 2 };

/* word number `index` of the stream (purpose, block, fid, comp). */
static uint64_t stream_word(uint64_t seed, int purpose, int block, int fid,
                            int comp, uint64_t index) {
  uint64_t ctr[4] = {index / 4, (uint64_t)purpose | ((uint64_t)block << 8),
                     (uint64_t)fid, (uint64_t)comp};
  uint64_t key[2] = {seed, 0};
  uint64_t out[4];
  oracle_philox4x64_10(ctr, key, out);
  return out[index % 4];
}

static double u01(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

/* ------------------------------------------------------------------ */
/* Function table (Table 1 and the per-function sections).             */
/* ------------------------------------------------------------------ */
/* scale s and offset c of each basic kind: z = R(s (x - o)) + c        */
static const double KIND_SCALE[OG_NUM_KINDS] = {
    1.0,     /* sphere: z = R(x-o) */
    1.0,     /* ellipsoid */
    1.0,     /* elliptic */
    1.0,     /* discus */
    1.0,     /* bent cigar */
    0.01,    /* different powers: R(0.01(x-o)) */
    1.0,     /* sharp valley */
    1.0,     /* step */
    0.005,   /* weierstrass: R(0.005(x-o)) */
    6.0,     /* griewank: R(6(x-o)) */
    0.0512,  /* rastrigin: 0.0512(x-o) */
    1.0,     /* schaffer F7 */
    0.05,    /* expanded griewank+rosenbrock: R(0.05(x-o)) + 1 */
    0.02048, /* rosenbrock: R(0.02048(x-o)) + 1 */
    10.0,    /* modified schwefel: 10(x-o) */
    0.05,    /* katsuura: R(0.05(x-o)) */
    0.1,     /* lunacek: R(0.1(x-o)) + 2.5 */
    1.0,     /* ackley */
    0.05,    /* happycat: R(0.05(x-o)) - 1 */
    0.05,    /* hgbat: R(0.05(x-o)) - 1 */
    1.0,     /* expanded schaffer F6 */
};
static const double KIND_OFFSET[OG_NUM_KINDS] = {
    0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,
    1.0,  /* EGR */
    1.0,  /* rosenbrock */
    0,    /* schwefel (its 420.97 shift lives inside w_i) */
    0,
    2.5,  /* lunacek (mu_1) */
    0,
    -1.0, /* happycat */
    -1.0, /* hgbat */
    0,
};

enum { T_BASIC = 0, T_HYBRID = 1, T_COMPOSITION = 2 };

typedef struct {
  int type;
  /* basic */
  int gkind, rotated;
  /* hybrid */
  int nh, hk[5], pct[5];
  /* composition: member m is a hybrid (member_fid >= 23) or a basic kind */
  int nc, member_kind[5], member_rot[5], member_fid[5];
  double sigma[5], lambda[5], bias[5];
} fdesc_t;

#define B(k, r) {T_BASIC, k, r, 0, {0}, {0}, 0, {0}, {0}, {0}, {0}, {0}, {0}}
#define H(n, k0, k1, k2, k3, k4, p0, p1, p2, p3, p4)                      \
  {T_HYBRID, 0, 1, n, {k0, k1, k2, k3, k4}, {p0, p1, p2, p3, p4}, 0, {0}, \
   {0}, {0}, {0}, {0}, {0}}

static const fdesc_t FTAB[ORACLE_NUM_FUNCTIONS] = {
    /* Unimodal functions, Sec. 3 */
    B(OG_SPHERE, 1), B(OG_ELLIPSOID, 1), B(OG_ELLIPTIC, 1), B(OG_DISCUS, 1),
    B(OG_CIGAR, 1), B(OG_POWERS, 1), B(OG_SHARPV, 1),
    /* Basic multi-modal functions, Sec. 4 */
    B(OG_STEP, 1), B(OG_WEIERSTRASS, 1), B(OG_GRIEWANK, 1),
    B(OG_RASTRIGIN, 0), B(OG_RASTRIGIN, 1), B(OG_SCHAFFERF7, 1),
    B(OG_EGR, 1), B(OG_ROSENBROCK, 1), B(OG_SCHWEFEL, 0), B(OG_SCHWEFEL, 1),
    B(OG_KATSUURA, 1), B(OG_LUNACEK, 1), B(OG_ACKLEY, 1), B(OG_HAPPYCAT, 1),
    B(OG_HGBAT, 1), B(OG_SCHAFFERF6, 1),
    /* Hybrid functions, Sec. 5 (Eq. hybrid, Eq. numbers) */
    H(3, OG_SCHWEFEL, OG_RASTRIGIN, OG_ELLIPTIC, 0, 0, 30, 30, 40, 0, 0),
    H(3, OG_CIGAR, OG_HGBAT, OG_RASTRIGIN, 0, 0, 30, 30, 40, 0, 0),
    H(4, OG_GRIEWANK, OG_WEIERSTRASS, OG_ROSENBROCK, OG_SCHAFFERF6, 0, 20, 20,
      30, 30, 0),
    H(4, OG_HGBAT, OG_DISCUS, OG_EGR, OG_RASTRIGIN, 0, 20, 20, 30, 30, 0),
    H(5, OG_SCHAFFERF6, OG_HGBAT, OG_ROSENBROCK, OG_SCHWEFEL, OG_ELLIPTIC, 10,
      20, 20, 20, 30),
    H(5, OG_KATSUURA, OG_HAPPYCAT, OG_EGR, OG_SCHWEFEL, OG_ACKLEY, 10, 20, 20,
      20, 30),
    /* Composition functions, Sec. 6 (Eq. composition, Eq. weight) */
    {T_COMPOSITION, 0, 0, 0, {0}, {0}, 5,
     {OG_ROSENBROCK, OG_ELLIPTIC, OG_CIGAR, OG_DISCUS, OG_ELLIPTIC},
     {1, 0, 1, 1, 0}, {-1, -1, -1, -1, -1},
     {10, 20, 30, 40, 50}, {1e-10, 1e-6, 1e-26, 1e-6, 1e-6},
     {0, 100, 200, 300, 400}},
    {T_COMPOSITION, 0, 0, 0, {0}, {0}, 3,
     {OG_SCHWEFEL, OG_RASTRIGIN, OG_HGBAT}, {0, 1, 1}, {-1, -1, -1},
     {15, 15, 15}, {1, 1, 1}, {0, 100, 200}},
    {T_COMPOSITION, 0, 0, 0, {0}, {0}, 3,
     {OG_SCHWEFEL, OG_RASTRIGIN, OG_ELLIPTIC}, {1, 1, 1}, {-1, -1, -1},
     {20, 50, 40}, {0.25, 1, 1e-7}, {0, 100, 200}},
    {T_COMPOSITION, 0, 0, 0, {0}, {0}, 5,
     {OG_SCHWEFEL, OG_HAPPYCAT, OG_ELLIPTIC, OG_WEIERSTRASS, OG_GRIEWANK},
     {1, 1, 1, 1, 1}, {-1, -1, -1, -1, -1},
     {20, 15, 10, 10, 40}, {2.5e-2, 0.1, 1e-8, 0.25, 1},
     {0, 100, 200, 300, 400}},
    {T_COMPOSITION, 0, 0, 0, {0}, {0}, 5,
     {OG_HGBAT, OG_RASTRIGIN, OG_SCHWEFEL, OG_WEIERSTRASS, OG_ELLIPTIC},
     {1, 1, 1, 1, 1}, {-1, -1, -1, -1, -1},
     {15, 15, 15, 15, 15}, {10, 10, 2.5, 2.5, 1e-6},
     {0, 100, 200, 300, 400}},
    {T_COMPOSITION, 0, 0, 0, {0}, {0}, 5,
     {OG_EGR, OG_HAPPYCAT, OG_SCHWEFEL, OG_SCHAFFERF6, OG_ELLIPTIC},
     {1, 1, 1, 1, 0}, {-1, -1, -1, -1, -1},
     {10, 20, 30, 40, 50}, {2.5, 10, 2.5, 5e-4, 1e-6},
     {0, 100, 200, 300, 400}},
    {T_COMPOSITION, 0, 0, 0, {0}, {0}, 3, {0, 0, 0}, {1, 1, 1},
     {23, 24, 25}, {10, 30, 50}, {1, 1, 1}, {0, 100, 200}},
    {T_COMPOSITION, 0, 0, 0, {0}, {0}, 3, {0, 0, 0}, {1, 1, 1},
     {26, 27, 28}, {10, 30, 50}, {1, 1, 1}, {0, 100, 200}},
};

/* ------------------------------------------------------------------ */
/* Basic functions G(z), z already scaled, rotated and offset.          */
/* Each returns the formula's value without f_opt; n = 0 gives 0.       */
/* ------------------------------------------------------------------ */

/* Sec. 3.1, Eq. sphere: sum z_i^2 */
static double g_sphere(const double* z, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += z[i] * z[i];
  return s;
}

/* Sec. 3.2, Eq. ellipsoid: sum i * z_i^2 (i from 1) */
static double g_ellipsoid(const double* z, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += (double)(i + 1) * (z[i] * z[i]);
  return s;
}

/* Sec. 3.3, Eq. elliptic: sum (10^6)^((i-1)/(D-1)) z_i^2 */
static double g_elliptic(const double* z, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double w = (n > 1) ? pow(1.0e6, (double)i / (double)(n - 1)) : 1.0;
    s += w * (z[i] * z[i]);
  }
  return s;
}

/* Sec. 3.4, Eq. discus: 10^6 z_1^2 + sum_{i>=2} z_i^2 */
static double g_discus(const double* z, int n) {
  if (n == 0) return 0.0;
  double s = 0.0;
  for (int i = 1; i < n; ++i) s += z[i] * z[i];
  return 1.0e6 * (z[0] * z[0]) + s;
}

/* Sec. 3.5, Eq. cigar: z_1^2 + 10^6 sum_{i>=2} z_i^2 */
static double g_cigar(const double* z, int n) {
  if (n == 0) return 0.0;
  double s = 0.0;
  for (int i = 1; i < n; ++i) s += z[i] * z[i];
  return z[0] * z[0] + 1.0e6 * s;
}

/* Sec. 3.6, Eq. powers: sqrt(sum |z_i|^(2 + 4 (i-1)/(D-1))) */
static double g_powers(const double* z, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double e = 2.0 + ((n > 1) ? 4.0 * ((double)i / (double)(n - 1)) : 0.0);
    s += pow(fabs(z[i]), e);
  }
  return sqrt(s);
}

/* Sec. 3.7, Eq. sharp_valley: z_1^2 + 100 sqrt(sum_{i>=2} z_i^2) */
static double g_sharpv(const double* z, int n) {
  if (n == 0) return 0.0;
  double s = 0.0;
  for (int i = 1; i < n; ++i) s += z[i] * z[i];
  return z[0] * z[0] + 100.0 * sqrt(s);
}

/* Sec. 4.1, Eq. step: sum floor(z_i + 0.5)^2 */
static double g_step(const double* z, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double t = floor(z[i] + 0.5);
    s += t * t;
  }
  return s;
}

/* Sec. 4.2, Eq. weierstrass, a = 0.5, b = 3, k_max = 20:
 * sum_i sum_k a^k cos(2 pi b^k (z_i + 0.5)) - D sum_k a^k cos(2 pi b^k 0.5) */
static double g_weierstrass(const double* z, int n) {
  const double a = 0.5, b = 3.0;
  const int kmax = 20;
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double inner = 0.0; /* the bracketed sum over k of Eq. weierstrass */
    for (int k = 0; k <= kmax; ++k) {
      double ak = pow(a, (double)k), bk = pow(b, (double)k);
      inner += ak * cos(2.0 * PI_D * bk * (z[i] + 0.5));
    }
    s += inner;
  }
  double c = 0.0;
  for (int k = 0; k <= kmax; ++k) {
    double ak = pow(a, (double)k), bk = pow(b, (double)k);
    c += ak * cos(2.0 * PI_D * bk * 0.5);
  }
  return s - (double)n * c;
}

/* Sec. 4.3, Eq. griewank: sum z_i^2/4000 - prod cos(z_i/sqrt(i)) + 1 */
static double g_griewank(const double* z, int n) {
  if (n == 0) return 0.0;
  double s = 0.0, p = 1.0;
  for (int i = 0; i < n; ++i) {
    s += z[i] * z[i] / 4000.0;
    p *= cos(z[i] / sqrt((double)(i + 1)));
  }
  return s - p + 1.0;
}

/* Sec. 4.4/4.5, Eq. rastrigin: sum (z_i^2 - 10 cos(2 pi z_i) + 10) */
static double g_rastrigin(const double* z, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i)
    s += z[i] * z[i] - 10.0 * cos(2.0 * PI_D * z[i]) + 10.0;
  return s;
}

/* Sec. 4.6, Eq. schaffersf7:
 * (1/(D-1) sum_{i<D} (1 + sin^2(50 w_i^0.2)) sqrt(w_i))^2,
 * w_i = sqrt(z_i^2 + z_{i+1}^2) */
static double g_schafferf7(const double* z, int n) {
  if (n < 2) return 0.0;
  double s = 0.0;
  for (int i = 0; i < n - 1; ++i) {
    double w = sqrt(z[i] * z[i] + z[i + 1] * z[i + 1]);
    double t = sin(50.0 * pow(w, 0.2));
    s += (1.0 + t * t) * sqrt(w);
  }
  double m = s / (double)(n - 1);
  return m * m;
}

/* Sec. 4.7: g2 (2-D Rosenbrock) and g3 (1-D Griewank) */
static double g2_rosen(double x, double y) {
  double a = x * x - y, b = x - 1.0;
  return 100.0 * (a * a) + b * b;
}
static double g3_griewank(double x) { return x * x / 4000.0 - cos(x) + 1.0; }

/* Sec. 4.7, Eq. expanded_griewank_rosenbrock (cyclic) */
static double g_egr(const double* z, int n) {
  if (n == 0) return 0.0;
  double s = 0.0;
  for (int i = 0; i < n - 1; ++i) s += g3_griewank(g2_rosen(z[i], z[i + 1]));
  s += g3_griewank(g2_rosen(z[n - 1], z[0]));
  return s;
}

/* Sec. 4.8, Eq. rosenbrok: sum_{i<D} 100(z_i^2 - z_{i+1})^2 + (z_i - 1)^2 */
static double g_rosenbrock(const double* z, int n) {
  double s = 0.0;
  for (int i = 0; i < n - 1; ++i) {
    double a = z[i] * z[i] - z[i + 1], b = z[i] - 1.0;
    s += 100.0 * (a * a) + b * b;
  }
  return s;
}

/* Sec. 4.9, Eq. basic_schwefel: the three-branch g_1 */
static double g1_schwefel(double w, int n) {
  if (fabs(w) <= 500.0) return w * sin(sqrt(fabs(w)));
  if (w > 500.0) {
    double m = fmod(w, 500.0);
    double t = w - 500.0;
    return (500.0 - m) * sin(sqrt(500.0 - m)) - t * t / (10000.0 * n);
  }
  double m = fmod(-w, 500.0);
  double t = w + 500.0;
  return (m - 500.0) * sin(sqrt(500.0 - m)) - t * t / (10000.0 * n);
}

/* Sec. 4.9/4.10, Eq. schwefel: 418.9829 D - sum g1(z_i + 420.9687462275036) */
static double g_schwefel(const double* z, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += g1_schwefel(z[i] + 420.9687462275036, n);
  return 418.9829 * (double)n - s;
}

/* Sec. 4.11, Eq. katsuura:
 * 10/D^2 prod (1 + i sum_{j=1}^{32} |2^j z_i - [2^j z_i]| / 2^j)^(10/D^1.2)
 *   - 10/D^2 */
static double g_katsuura(const double* z, int n) {
  if (n == 0) return 0.0;
  double e = 10.0 / pow((double)n, 1.2);
  double p = 1.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 1; j <= 32; ++j) {
      double tj = ldexp(1.0, j);
      double v = tj * z[i];
      s += fabs(v - rint(v)) / tj;
    }
    p *= pow(1.0 + (double)(i + 1) * s, e);
  }
  double c = 10.0 / ((double)n * (double)n);
  return c * p - c;
}

/* Sec. 4.12, Eq. (Lunacek) with mu_1 = 2.5, mu_2 = -2.5, d = 1, s = 0.9:
 * min(sum (z-mu1)^2, d D + s sum (z-mu2)^2) + 10 (D - sum cos(2 pi (z-mu1))) */
static double g_lunacek(const double* z, int n) {
  const double mu1 = 2.5, mu2 = -2.5, d = 1.0, sv = 0.9;
  double s1 = 0.0, s2 = 0.0, c = 0.0;
  for (int i = 0; i < n; ++i) {
    double a = z[i] - mu1, b = z[i] - mu2;
    s1 += a * a;
    s2 += b * b;
    c += cos(2.0 * PI_D * a);
  }
  double t2 = d * (double)n + sv * s2;
  double m = (s1 < t2) ? s1 : t2;
  return m + 10.0 * ((double)n - c);
}

/* Sec. 4.13, Eq. ackley:
 * -20 exp(-0.2 sqrt(sum z^2 / D)) - exp(sum cos(2 pi z) / D) + 20 + e */
static double g_ackley(const double* z, int n) {
  if (n == 0) return 0.0;
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < n; ++i) {
    s1 += z[i] * z[i];
    s2 += cos(2.0 * PI_D * z[i]);
  }
  return -20.0 * exp(-0.2 * sqrt(s1 / (double)n)) - exp(s2 / (double)n) +
         20.0 + exp(1.0);
}

/* Sec. 4.14, Eq. happycat:
 * |sum z^2 - D|^0.25 + (0.5 sum z^2 + sum z)/D + 0.5 */
static double g_happycat(const double* z, int n) {
  if (n == 0) return 0.0;
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < n; ++i) {
    s1 += z[i] * z[i];
    s2 += z[i];
  }
  return pow(fabs(s1 - (double)n), 0.25) + (0.5 * s1 + s2) / (double)n + 0.5;
}

/* Sec. 4.15, Eq. hgbat:
 * |(sum z^2)^2 - (sum z)^2|^0.5 + (0.5 sum z^2 + sum z)/D + 0.5 */
static double g_hgbat(const double* z, int n) {
  if (n == 0) return 0.0;
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < n; ++i) {
    s1 += z[i] * z[i];
    s2 += z[i];
  }
  return pow(fabs(s1 * s1 - s2 * s2), 0.5) + (0.5 * s1 + s2) / (double)n +
         0.5;
}

/* Sec. 4.16: Schaffer's F6 pair function g4 */
static double g4_schaffer(double x, double y) {
  double r2 = x * x + y * y;
  double t = sin(sqrt(r2));
  double d = 1.0 + 0.001 * r2;
  return (t * t - 0.5) / (d * d) + 0.5;
}

/* Sec. 4.16, Eq. expanded_schaffersf6 (cyclic) */
static double g_schafferf6(const double* z, int n) {
  if (n == 0) return 0.0;
  double s = 0.0;
  for (int i = 0; i < n - 1; ++i) s += g4_schaffer(z[i], z[i + 1]);
  s += g4_schaffer(z[n - 1], z[0]);
  return s;
}

double oracle_G(int gkind, const double* z, int n) {
  switch (gkind) {
    case OG_SPHERE: return g_sphere(z, n);
    case OG_ELLIPSOID: return g_ellipsoid(z, n);
    case OG_ELLIPTIC: return g_elliptic(z, n);
    case OG_DISCUS: return g_discus(z, n);
    case OG_CIGAR: return g_cigar(z, n);
    case OG_POWERS: return g_powers(z, n);
    case OG_SHARPV: return g_sharpv(z, n);
    case OG_STEP: return g_step(z, n);
    case OG_WEIERSTRASS: return g_weierstrass(z, n);
    case OG_GRIEWANK: return g_griewank(z, n);
    case OG_RASTRIGIN: return g_rastrigin(z, n);
    case OG_SCHAFFERF7: return g_schafferf7(z, n);
    case OG_EGR: return g_egr(z, n);
    case OG_ROSENBROCK: return g_rosenbrock(z, n);
    case OG_SCHWEFEL: return g_schwefel(z, n);
    case OG_KATSUURA: return g_katsuura(z, n);
    case OG_LUNACEK: return g_lunacek(z, n);
    case OG_ACKLEY: return g_ackley(z, n);
    case OG_HAPPYCAT: return g_happycat(z, n);
    case OG_HGBAT: return g_hgbat(z, n);
    case OG_SCHAFFERF6: return g_schafferf6(z, n);
    default: return NAN;
  }
}

/* ------------------------------------------------------------------ */
/* Component layout (General Setup: three subcomponents; Eq. numbers).  */
/* ------------------------------------------------------------------ */
typedef struct {
  int hybrid_fid;  /* >= 0: component is this hybrid function */
  int gkind;       /* basic kind when hybrid_fid < 0 */
  int rotated;
  int nb;
  int sizes[5];
} layout_t;

static int valid_fid(int fid) { return fid >= 0 && fid < ORACLE_NUM_FUNCTIONS; }

static int needs_d10(int fid) {
  return (fid >= 23 && fid <= 28) || fid == 35 || fid == 36;
}

static int make_layout(int fid, int D, int comp, layout_t* L) {
  if (!valid_fid(fid)) return -1;
  if (D < 2 || (needs_d10(fid) && D < 10)) return -2;
  const fdesc_t* f = &FTAB[fid];
  int member_fid = -1, kind = 0, rot = 0;
  if (f->type == T_COMPOSITION) {
    if (comp < 0 || comp >= f->nc) return -1;
    member_fid = f->member_fid[comp];
    kind = f->member_kind[comp];
    rot = f->member_rot[comp];
  } else {
    if (comp != 0) return -1;
    if (f->type == T_HYBRID) {
      member_fid = fid;
    } else {
      kind = f->gkind;
      rot = f->rotated;
    }
  }
  memset(L, 0, sizeof(*L));
  if (member_fid >= 0) {
    const fdesc_t* h = &FTAB[member_fid];
    L->hybrid_fid = member_fid;
    L->rotated = 1;
    L->nb = h->nh;
    int used = 0;
    for (int i = 0; i < h->nh - 1; ++i) {
      /* n_i = ceil(p_i D), p_i in integer percent (Eq. numbers) */
      L->sizes[i] = (h->pct[i] * D + 99) / 100;
      used += L->sizes[i];
    }
    L->sizes[h->nh - 1] = D - used;
    if (L->sizes[h->nh - 1] < 0) return -2;
  } else {
    L->hybrid_fid = -1;
    L->gkind = kind;
    L->rotated = rot;
    if (rot) {
      L->nb = 3;
      L->sizes[0] = D / 3;
      L->sizes[1] = D / 3;
      L->sizes[2] = D - 2 * (D / 3);
    } else {
      L->nb = 1;
      L->sizes[0] = D;
    }
  }
  return 0;
}

int oracle_num_components(int fid) {
  if (!valid_fid(fid)) return -1;
  return FTAB[fid].type == T_COMPOSITION ? FTAB[fid].nc : 1;
}

int oracle_component_layout(int fid, int D, int comp, int* n_blocks,
                            int block_sizes[5], int* rotated) {
  layout_t L;
  int rc = make_layout(fid, D, comp, &L);
  if (rc) return rc;
  *n_blocks = L.nb;
  for (int i = 0; i < 5; ++i) block_sizes[i] = (i < L.nb) ? L.sizes[i] : 0;
  *rotated = L.rotated;
  return 0;
}

static long layout_rsize(const layout_t* L) {
  if (!L->rotated) return 0;
  long s = 0;
  for (int b = 0; b < L->nb; ++b) s += (long)L->sizes[b] * L->sizes[b];
  return s;
}

long oracle_component_rsize(int fid, int D, int comp) {
  layout_t L;
  if (make_layout(fid, D, comp, &L)) return -1;
  return layout_rsize(&L);
}

/* ------------------------------------------------------------------ */
/* Instance generation (General Setup).                                 */
/* ------------------------------------------------------------------ */
static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

int oracle_generate_component(int fid, int D, uint64_t seed, int comp,
                              double* o, int* S, double* R) {
  layout_t L;
  int rc = make_layout(fid, D, comp, &L);
  if (rc) return rc;

  /* x^opt uniform in [-70,70]^D; the third composition member sits at
   * the origin (Composition Functions section). */
  int at_origin = (FTAB[fid].type == T_COMPOSITION && comp == 2);
  for (int k = 0; k < D; ++k) {
    if (at_origin) {
      o[k] = 0.0;
    } else {
      double u = u01(stream_word(seed, PURPOSE_SHIFT, 0, fid, comp, (uint64_t)k));
      double t = 140.0 * u;
      o[k] = t - 70.0;
    }
  }

  for (int k = 0; k < D; ++k) S[k] = k;
  if (!L.rotated) return 0;

  /* random split of the variables: a random permutation (Fisher-Yates)
   * cut into consecutive blocks, each block's indices sorted. */
  for (int i = D - 1; i >= 1; --i) {
    uint64_t w = stream_word(seed, PURPOSE_PERM, 0, fid, comp, (uint64_t)i);
    uint64_t hi, lo;
    mulhilo64(w, (uint64_t)(i + 1), &hi, &lo);
    int j = (int)hi;
    int t = S[i];
    S[i] = S[j];
    S[j] = t;
  }
  int off = 0;
  for (int b = 0; b < L.nb; ++b) {
    qsort(S + off, (size_t)L.sizes[b], sizeof(int), cmp_int);
    off += L.sizes[b];
  }

  /* rotation of each subcomponent: standard normal entries (Box-Muller),
   * then Gram-Schmidt orthonormalisation of the rows, done twice. */
  long roff = 0;
  for (int b = 0; b < L.nb; ++b) {
    int n = L.sizes[b];
    double* Rb = R + roff;
    for (long t = 0; t < (long)n * n; ++t) {
      uint64_t w1 = stream_word(seed, PURPOSE_GAUSS, b, fid, comp, (uint64_t)(2 * t));
      uint64_t w2 = stream_word(seed, PURPOSE_GAUSS, b, fid, comp, (uint64_t)(2 * t + 1));
      double u1 = (double)((w1 >> 11) + 1) * 0x1.0p-53;
      double u2 = (double)(w2 >> 11) * 0x1.0p-53;
      double r = sqrt(-2.0 * log(u1));
      Rb[t] = r * cos(2.0 * PI_D * u2);
    }
    for (int r = 0; r < n; ++r) {
      double* v = Rb + (long)r * n;
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = 0; q < r; ++q) {
          const double* e = Rb + (long)q * n;
          double d = 0.0;
          for (int c = 0; c < n; ++c) d += v[c] * e[c];
          for (int c = 0; c < n; ++c) v[c] -= d * e[c];
        }
      }
      double nrm = 0.0;
      for (int c = 0; c < n; ++c) nrm += v[c] * v[c];
      nrm = sqrt(nrm);
      if (!(nrm > 1e-10)) return -3; /* degenerate draw (probability 0) */
      for (int c = 0; c < n; ++c) v[c] = v[c] / nrm;
    }
    roff += (long)n * n;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Evaluation.                                                          */
/* ------------------------------------------------------------------ */

/* z of one component, in block order (General Setup, "z = R(s(x - o)) + c"):
 * y = x - o; each block takes y at its variables S_b, scaled by the s of its
 * basic kind, rotated by R_b and offset by the kind's c (a hybrid's block i
 * by the s and c of its own G_i, Eq. hybrid).  An unrotated component is
 * z = s y + c.  plain = 0: each dot product takes one fma per term in index
 * order (the oracle's evaluation); plain = 1: each product is rounded, then
 * added, in index order.  work holds 2 D doubles. */
static void component_z(const layout_t* L, int D, const double* o,
                        const int* S, const double* R, const double* x,
                        int plain, double* work, double* z) {
  double* y = work;
  double* v = work + D;
  for (int j = 0; j < D; ++j) y[j] = x[j] - o[j];
  if (!L->rotated) {
    int k = L->gkind;
    for (int j = 0; j < D; ++j) z[j] = KIND_SCALE[k] * y[j] + KIND_OFFSET[k];
    return;
  }
  const fdesc_t* h = (L->hybrid_fid >= 0) ? &FTAB[L->hybrid_fid] : NULL;
  int off = 0;
  long roff = 0;
  for (int b = 0; b < L->nb; ++b) {
    int n = L->sizes[b];
    int k = h ? h->hk[b] : L->gkind;
    for (int c = 0; c < n; ++c) v[c] = KIND_SCALE[k] * y[S[off + c]];
    const double* Rb = R + roff;
    for (int r = 0; r < n; ++r) {
      double acc = 0.0;
      if (plain) {
        for (int c = 0; c < n; ++c) acc += Rb[(long)r * n + c] * v[c];
      } else {
        for (int c = 0; c < n; ++c) acc = fma(Rb[(long)r * n + c], v[c], acc);
      }
      z[off + r] = acc + KIND_OFFSET[k];
    }
    off += n;
    roff += (long)n * n;
  }
}

/* One component's value (no f_opt) from its z: the basic function on the
 * whole of z, or a hybrid's sum of G_i over its blocks in block order, with
 * "D" inside G_i equal to n_i (Eq. hybrid). */
static double component_value(const layout_t* L, int D, const double* z) {
  if (L->hybrid_fid >= 0) {
    const fdesc_t* h = &FTAB[L->hybrid_fid];
    double total = 0.0;
    int off = 0;
    for (int b = 0; b < L->nb; ++b) {
      total += oracle_G(h->hk[b], z + off, L->sizes[b]);
      off += L->sizes[b];
    }
    return total;
  }
  return oracle_G(L->gkind, z, D);
}

/* ||x - o||^2 in index order (Eq. weight's d_i^2). */
static double sq_distance(int D, const double* x, const double* o) {
  double s = 0.0;
  for (int j = 0; j < D; ++j) {
    double t = x[j] - o[j];
    s += t * t;
  }
  return s;
}

/* Eq. composition with the weights of Eq. weight (no f_opt):
 * sum_i omega_i (lambda_i G_i + bias_i), omega_i = w_i / sum_j w_j,
 * w_i = (1 / sqrt(d_i^2)) exp(-d_i^2 / (2 D sigma_i^2)). */
static double compose_value(const fdesc_t* f, int nc, int D, const double* G,
                            const double* d2) {
  int hit = -1;
  for (int c = 0; c < nc; ++c)
    if (d2[c] == 0.0 && hit < 0) hit = c;
  if (hit >= 0) {
    /* x = x^{opt,i}: omega is one-hot at i (stated limit) */
    return f->lambda[hit] * G[hit] + f->bias[hit];
  }
  double w[5], W = 0.0;
  for (int c = 0; c < nc; ++c) {
    w[c] = (1.0 / sqrt(d2[c])) *
           exp(-d2[c] / (2.0 * (double)D * f->sigma[c] * f->sigma[c]));
    W += w[c];
  }
  double F = 0.0;
  if (W > 0.0) {
    for (int c = 0; c < nc; ++c)
      F += (w[c] / W) * (f->lambda[c] * G[c] + f->bias[c]);
    return F;
  }
  /* every w_i underflowed (far outside the search box): the same
   * normalisation taken in the log domain */
  double lw[5], mx = -INFINITY;
  for (int c = 0; c < nc; ++c) {
    lw[c] = -0.5 * log(d2[c]) -
            d2[c] / (2.0 * (double)D * f->sigma[c] * f->sigma[c]);
    if (lw[c] > mx) mx = lw[c];
  }
  double Z = 0.0;
  for (int c = 0; c < nc; ++c) Z += exp(lw[c] - mx);
  for (int c = 0; c < nc; ++c)
    F += (exp(lw[c] - mx) / Z) * (f->lambda[c] * G[c] + f->bias[c]);
  return F;
}

static int make_layouts(int fid, int D, layout_t L[5], long roffs[5]) {
  int nc = oracle_num_components(fid);
  long rtot = 0;
  for (int c = 0; c < nc; ++c) {
    int rc = make_layout(fid, D, c, &L[c]);
    if (rc) return rc;
    if (roffs) roffs[c] = rtot;
    rtot += layout_rsize(&L[c]);
  }
  return 0;
}

int oracle_evaluate_given(int fid, int D, const double* o, const int* S,
                          const double* R, const double* x, long N,
                          double* out, int nthreads) {
  if (!valid_fid(fid)) return -1;
  const fdesc_t* f = &FTAB[fid];
  int nc = oracle_num_components(fid);
  layout_t L[5];
  long roffs[5];
  int rc0 = make_layouts(fid, D, L, roffs);
  if (rc0) return rc0;
  if (nthreads < 1) nthreads = 1;
  int err = 0;

#pragma omp parallel num_threads(nthreads)
  {
    double* work = (double*)malloc(sizeof(double) * 3 * (size_t)D);
    if (!work) {
#pragma omp atomic write
      err = -4;
    }
#pragma omp for schedule(dynamic, 4)
    for (long n = 0; n < N; ++n) {
      if (!work) continue;
      const double* xn = x + n * (long)D;
      double* z = work + 2 * D;
      if (f->type != T_COMPOSITION) {
        component_z(&L[0], D, o, S, R, xn, 0, work, z);
        out[n] = component_value(&L[0], D, z) + F_OPT;
        continue;
      }
      double G[5], d2[5];
      for (int c = 0; c < nc; ++c) {
        const double* oc = o + (long)c * D;
        component_z(&L[c], D, oc, S + (long)c * D, R + roffs[c], xn, 0, work, z);
        G[c] = component_value(&L[c], D, z);
        d2[c] = sq_distance(D, xn, oc);
      }
      out[n] = compose_value(f, nc, D, G, d2) + F_OPT;
    }
    free(work);
  }
  return err;
}

int oracle_component_z(int fid, int D, int comp, const double* o,
                       const int* S, const double* R, const double* x,
                       int plain, double* z) {
  layout_t L;
  int rc = make_layout(fid, D, comp, &L);
  if (rc) return rc;
  double* work = (double*)malloc(sizeof(double) * 2 * (size_t)D);
  if (!work) return -4;
  component_z(&L, D, o, S, R, x, plain, work, z);
  free(work);
  return 0;
}

int oracle_block_affine(int fid, int D, int comp, double scale[5],
                        double offset[5]) {
  layout_t L;
  int rc = make_layout(fid, D, comp, &L);
  if (rc) return rc;
  const fdesc_t* h = (L.hybrid_fid >= 0) ? &FTAB[L.hybrid_fid] : NULL;
  for (int b = 0; b < 5; ++b) {
    int k = (h && b < L.nb) ? h->hk[b] : L.gkind;
    scale[b] = (b < L.nb) ? KIND_SCALE[k] : 0.0;
    offset[b] = (b < L.nb) ? KIND_OFFSET[k] : 0.0;
  }
  return 0;
}

int oracle_evaluate_from_z(int fid, int D, const double* z, const double* d2,
                           double* out) {
  if (!valid_fid(fid)) return -1;
  const fdesc_t* f = &FTAB[fid];
  int nc = oracle_num_components(fid);
  layout_t L[5];
  int rc = make_layouts(fid, D, L, NULL);
  if (rc) return rc;
  if (f->type != T_COMPOSITION) {
    *out = component_value(&L[0], D, z) + F_OPT;
    return 0;
  }
  double G[5];
  for (int c = 0; c < nc; ++c) G[c] = component_value(&L[c], D, z + (long)c * D);
  *out = compose_value(f, nc, D, G, d2) + F_OPT;
  return 0;
}

int oracle_compose(int fid, int D, const double* G, const double* d2,
                   double* out) {
  if (!valid_fid(fid) || FTAB[fid].type != T_COMPOSITION) return -1;
  *out = compose_value(&FTAB[fid], FTAB[fid].nc, D, G, d2) + F_OPT;
  return 0;
}

int oracle_evaluate(int fid, int D, uint64_t seed, const double* x, long N,
                    double* out, int nthreads) {
  if (!valid_fid(fid)) return -1;
  int nc = oracle_num_components(fid);
  long rtot = 0;
  for (int c = 0; c < nc; ++c) {
    long r = oracle_component_rsize(fid, D, c);
    if (r < 0) return -2;
    rtot += r;
  }
  double* o = (double*)malloc(sizeof(double) * (size_t)nc * D);
  int* S = (int*)malloc(sizeof(int) * (size_t)nc * D);
  double* R = (double*)malloc(sizeof(double) * (size_t)(rtot > 0 ? rtot : 1));
  int rc = (o && S && R) ? 0 : -4;
  long roff = 0;
  for (int c = 0; c < nc && rc == 0; ++c) {
    rc = oracle_generate_component(fid, D, seed, c, o + (long)c * D,
                                   S + (long)c * D, R + roff);
    roff += oracle_component_rsize(fid, D, c);
  }
  if (rc == 0) rc = oracle_evaluate_given(fid, D, o, S, R, x, N, out, nthreads);
  free(o);
  free(S);
  free(R);
  return rc;
}

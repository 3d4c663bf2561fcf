/*
 * curob_oracle.h -- plain FP64 CPU oracle for the cuROB benchmark functions
 * (Ding & Tan, "A CUDA-Based Real Parameter Optimization Benchmark").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that
 * the GPU library is checked against.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark script may load it; the product
 * path never does.  It shares no code, header, table or generator with the
 * CUDA library.
 *
 * Everything is FP64, evaluated in index order, with the C library's libm.
 * Instance data (shift o, permutation S, rotation blocks R) is generated
 * from a seed by the procedure of the "General Setup" section:
 *   o ~ U[-70,70]^D                                  (General Setup, x^opt)
 *   variables split at random into 3 near-equal parts, each rotated by a
 *   Gram-Schmidt orthonormalised standard-normal matrix  (General Setup, R)
 * The random draws come from Philox4x64-10 (Salmon et al., SC'11); the
 * layout of the draws is fixed by the library's instance-generation spec,
 * which both implementations follow independently:
 *   key     = (seed, 0)
 *   counter = (word_index / 4, purpose | block << 8, fid, component)
 *   purpose: 0 = shift, 1 = permutation, 2 = Gaussian rotation entries
 *   u       = (word >> 11) * 2^-53                     in [0,1)
 *   o_k     = 140*u_k - 70 (two roundings); component 3 of a composition
 *             has o = 0 (Composition Functions section).
 *   pi      = Fisher-Yates, i = D-1..1, j = floor(word_i * (i+1) / 2^64)
 *   blocks  = basic: (D/3, D/3, D-2*(D/3)); hybrid: n_i = ceil(P_i*D/100)
 *             in integer percent, last takes the rest (Eq. numbers);
 *             each block's index set is sorted ascending.
 *   G_b     = Box-Muller (cos branch) on words 2t, 2t+1, t = r*n_b + c,
 *             u1 = ((w>>11)+1)*2^-53 in (0,1]
 *   R_b     = rows of G_b orthonormalised in row order by modified
 *             Gram-Schmidt applied twice.
 * z is laid out in block order: z = [R_1 y_{S_1}, R_2 y_{S_2}, R_3 y_{S_3}].
 */
#ifndef CUROB_ORACLE_H
#define CUROB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of Table-1 functions (IDs 0..36). */
#define ORACLE_NUM_FUNCTIONS 37

/* Basic-function kinds (the G_i of the hybrid and composition sections). */
enum oracle_gkind {
  OG_SPHERE = 0, OG_ELLIPSOID, OG_ELLIPTIC, OG_DISCUS, OG_CIGAR, OG_POWERS,
  OG_SHARPV, OG_STEP, OG_WEIERSTRASS, OG_GRIEWANK, OG_RASTRIGIN,
  OG_SCHAFFERF7, OG_EGR, OG_ROSENBROCK, OG_SCHWEFEL, OG_KATSUURA,
  OG_LUNACEK, OG_ACKLEY, OG_HAPPYCAT, OG_HGBAT, OG_SCHAFFERF6,
  OG_NUM_KINDS
};

/* Philox4x64-10 block function: out = philox(counter, key). */
void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                          uint64_t out[4]);

/* G(z) for a basic kind on an n-vector z that already includes the
 * function's scale and offset (the value of the formula without f_opt). */
double oracle_G(int gkind, const double* z, int n);

/* Number of components of function fid (1 unless a composition). */
int oracle_num_components(int fid);

/* Layout of component comp of fid at dimension D.
 * rotated: 1 if R is a random rotation, 0 if the component is unrotated
 * (then n_blocks = 1, S = identity, R unused).  Returns 0 on success,
 * -1 for an invalid fid/comp, -2 for an invalid D. */
int oracle_component_layout(int fid, int D, int comp, int* n_blocks,
                            int block_sizes[5], int* rotated);

/* Total rotation storage (sum of n_b^2) for component comp. */
long oracle_component_rsize(int fid, int D, int comp);

/* Generate component comp's instance data: o[D], S[D] (block order),
 * R (blocks packed row-major, block after block).  Returns 0 on success. */
int oracle_generate_component(int fid, int D, uint64_t seed, int comp,
                              double* o, int* S, double* R);

/* Evaluate fid on N candidates x (N x D row-major) with explicitly given
 * instance data: o and S are n_comp x D, R is the concatenation of each
 * component's packed blocks.  Uses up to nthreads OpenMP threads.
 * out[n] = f(x_n) including f_opt = 100. */
int oracle_evaluate_given(int fid, int D, const double* o, const int* S,
                          const double* R, const double* x, long N,
                          double* out, int nthreads);

/* z of component comp (block order, D values) for one candidate x, with that
 * component's own o[D], S[D] and packed R: z = R(s (x - o)) + c.  plain = 0:
 * each dot product one fma per term in index order, as oracle_evaluate_given;
 * plain = 1: each product rounded, then added. */
int oracle_component_z(int fid, int D, int comp, const double* o,
                       const int* S, const double* R, const double* x,
                       int plain, double* z);

/* The scale s and offset c of each block of component comp (z_b =
 * R_b (s_b y_b) + c_b; an unrotated component reports its one block). */
int oracle_block_affine(int fid, int D, int comp, double scale[5],
                        double offset[5]);

/* f (f_opt included) of one candidate from its components' z (n_comp x D,
 * block order) and, for a composition, d2[c] = ||x - o_c||^2 (Eq. weight);
 * d2 is not read otherwise.  The same assembly as oracle_evaluate_given. */
int oracle_evaluate_from_z(int fid, int D, const double* z, const double* d2,
                           double* out);

/* A composition's value (f_opt included) from its members' G_c and d2_c
 * (Eq. composition, Eq. weight).  -1 if fid is not a composition. */
int oracle_compose(int fid, int D, const double* G, const double* d2,
                   double* out);

/* Generate the instance from seed and evaluate. */
int oracle_evaluate(int fid, int D, uint64_t seed, const double* x, long N,
                    double* out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif

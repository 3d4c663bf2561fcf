/*
 * curob.h -- C ABI of libcurob, a GB300 (sm_103a) implementation of the cuROB
 * real-parameter optimisation benchmark (Ding & Tan, "A CUDA-Based Real
 * Parameter Optimization Benchmark").
 *
 * The library evaluates populations of N candidate vectors on the 37 test
 * functions of the paper's Table 1 (IDs 0..36): shifted and block-rotated
 * unimodal, multimodal, hybrid and composition functions, f_opt = 100.
 *
 * Conventions for every entry point:
 *  - x is N x D, row-major (candidate n occupies x[n*D .. n*D+D-1]); out has N
 *    entries.  Pointers passed to curob_evaluate / curob_evaluatef are DEVICE
 *    pointers owned by the caller (Sec. 1.3 "Interface": device pointers are
 *    passed to func_evaluate/func_evaluatef); the call is asynchronous on
 *    `stream` (NULL = legacy default stream) and writes out[0..N-1] only.
 *  - Argument errors are reported synchronously and launch nothing.  Errors
 *    raised inside a kernel (a bounded wait that timed out) are latched in the
 *    library and reported by curob_get_device_status().
 *  - Non-finite inputs give NaN outputs, not an error.
 *  - The library holds one instance (one D) between curob_initialize and
 *    curob_dispose, like the paper's compile-time DIM (Sec. 1.3).  Calls are
 *    thread-safe with respect to one another; evaluations may overlap on
 *    different streams.
 *  - The instance lives on the device that was current at curob_initialize.
 *    Every evaluation must be made with that device current and with x and
 *    out in its memory (or managed memory); otherwise it returns
 *    CUROB_ERR_INVALID_ARGUMENT and launches nothing.
 */
#ifndef CUROB_H
#define CUROB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* curob_stream_t; /* same type as cudaStream_t */

typedef enum {
  CUROB_OK = 0,
  CUROB_ERR_NOT_INITIALIZED = 1,     /* no curob_initialize yet */
  CUROB_ERR_ALREADY_INITIALIZED = 2, /* curob_initialize twice */
  CUROB_ERR_INVALID_FID = 3,         /* fid outside 0..36 */
  CUROB_ERR_INVALID_DIM = 4,         /* D < 2, or D < 10 for IDs 23..28, 35, 36 */
  CUROB_ERR_CAPACITY = 5,            /* N > max_concurrency */
  CUROB_ERR_NULL_POINTER = 6,        /* NULL where data is required */
  CUROB_ERR_CUDA = 7,                /* a CUDA runtime call failed */
  CUROB_ERR_DEVICE_TIMEOUT = 8,      /* a bounded device-side wait expired */
  CUROB_ERR_OUT_OF_MEMORY = 9,       /* device allocation failed */
  CUROB_ERR_INVALID_ARGUMENT = 10,   /* e.g. N < 0, host pointer where a device one is needed */
  CUROB_ERR_UNSUPPORTED = 11         /* size outside what the chosen kernel handles */
} curob_status;

/* Rotation-contraction precision of curob_evaluatef (the paper evaluates FP32
 * plainly; these are this library's choices).  TF32X3: three TF32
 * tensor-core products per term (hi*hi + hi*lo + lo*hi), FP32 accumulation.
 * BF16X3: the same with BF16 halves.  EXACT: both operands cut into four
 * integer slices held exactly in BF16; the leading slice product is
 * accumulated exactly (every partial sum an integer below 2^23), the nine
 * lower-weight products in a second FP32 accumulator 2^-8 below it; z to
 * about 2^-26 of each candidate's |x - o|_max.
 * FP16X3: y scaled by a power of two above each candidate's max |x - o|
 * over the component and R by a power of two per row, both cut into FP16
 * hi + lo (22 significant bits, as TF32 hi + lo), three products with FP32
 * accumulation at the FP16 tensor rate (half the operand bytes of TF32X3).
 * SIMT: FP32 CUDA cores with a compensated dot product.  AUTO (default):
 * EXACT for functions containing Discus, Weierstrass, expanded
 * Griewank-Rosenbrock or Katsuura (they magnify z errors), TF32X3 for the
 * rest; for a composition only some of whose members contain such a kind,
 * MIXED: those members on EXACT, the others on TF32X3 (reported by
 * curob_query_precision, not selectable); SIMT where a block is narrower
 * than 16 or wider than 512. */
typedef enum {
  CUROB_PRECISION_AUTO = 0,
  CUROB_PRECISION_TF32X3 = 1,
  CUROB_PRECISION_BF16X3 = 2,
  CUROB_PRECISION_SIMT = 3,
  CUROB_PRECISION_EXACT = 4,
  CUROB_PRECISION_MIXED = 5,
  CUROB_PRECISION_FP16X3 = 6
} curob_precision;

/* Number of functions (Table 1). */
#define CUROB_NUM_FUNCTIONS 37
/* f_opt of every function (Table 1 footer). */
#define CUROB_FOPT 100.0

/* Sec. 1.3 "Interface", initialize(): builds every function's instance on the
 * current CUDA device: shifts x^opt ~ U[-70,70]^D, a random split of the
 * variables into blocks, one Gram-Schmidt-orthonormalised Gaussian rotation
 * per block (General Setup), drawn from Philox4x64-10 keyed by `seed`.
 * max_concurrency bounds N of every later evaluation (the paper's
 * MAX_CONCURRENCY); device buffers for the host wrappers are sized by it.
 * Errors: ALREADY_INITIALIZED, INVALID_DIM (D < 2), INVALID_ARGUMENT
 * (max_concurrency < 1), OUT_OF_MEMORY, CUDA.  Synchronous. */
curob_status curob_initialize(int D, int max_concurrency, uint64_t seed);

/* Sec. 1.3, dispose(): releases everything curob_initialize allocated.
 * Synchronises the device first.  Errors: NOT_INITIALIZED. */
curob_status curob_dispose(void);

/* Sec. 1.3, func_evaluate(): out[n] = f_fid(x_n) in FP64 for n < N.  x, out:
 * device pointers (x: N*D doubles, out: N doubles).  0 <= N <= max_concurrency.
 * The path is set by curob_set_precision64: on the tensor cores (default
 * where the device has them) the block rotation is an error-free split
 * product of BF16 integer digits (z rounded once to FP64 from an exact
 * integer sum of all products above 2^-56 of the scale), with scratch (about
 * 230 bytes per candidate and K step of 16 variables of the rotated blocks,
 * plus 8 bytes per candidate and variable of every component; at most 2 GB
 * per slice of candidates) taken stream-ordered from the library's pool;
 * terms, sums and the composition are evaluated in FP64 as on the CUDA
 * cores.  Calls with N at most the small-population limit (see
 * curob_set_small_batch) run on the small kernels.  Errors: NOT_INITIALIZED,
 * INVALID_FID, INVALID_DIM, CAPACITY, NULL_POINTER, INVALID_ARGUMENT,
 * UNSUPPORTED (tensor cores forced where the device has none), CUDA.
 * Asynchronous on `stream`. */
curob_status curob_evaluate(int fid, const double* x, int N, double* out, curob_stream_t stream);

/* Sec. 1.3, func_evaluatef(): the same with FP32 x and out.  The shift x - o
 * is taken in FP64 (o is FP64), the block rotation runs on the tensor cores
 * in the precision set by curob_set_precision, reductions are carried in
 * FP64 across lanes.  A function with a block of a heavy kind (see
 * curob_query_launches), or a MIXED composition, takes a second kernel on
 * the same stream.  Scratch, taken stream-ordered from a pool the library
 * keeps, per slice of candidates (the heavy-kind part at most 256 MB,
 * candidates in slices beyond that): the transposed copy of the slice's x
 * (4 D bytes per candidate), 4 bytes per heavy variable and 80 bytes per
 * candidate for the second kernel, and, when a member runs on EXACT or
 * FP16X3, 4 bytes per candidate and 64 variables of each component for the
 * row maxima those precisions scale by; calls on different streams may run
 * concurrently.  If that scratch cannot be had, a function with one
 * precision group falls back to the single fused launch, and a MIXED
 * composition returns CUDA.  Same errors as curob_evaluate, plus
 * UNSUPPORTED if a forced precision cannot handle the instance's block
 * sizes. */
curob_status curob_evaluatef(int fid, const float* x, int N, float* out, curob_stream_t stream);

/* Sec. 1.3, h_func_evaluate / h_func_evaluatef: host-pointer wrappers (x:
 * N x D host array, out: N host values).  The call is cut into up to four
 * chunks of whole 128-candidate tiles (one chunk below 2048 candidates), each
 * copied in, evaluated and copied out on its own library stream, so that a
 * chunk's copy-in overlaps the kernels of the chunks before it; the values
 * are those of curob_evaluate / curob_evaluatef.  Returns once out is
 * written (synchronous).  Copies run at full speed from page-locked host
 * memory; pageable memory works but the copies then stage through the
 * driver.  The staging buffers are the library's: concurrent host-wrapper
 * calls from several threads are serialised.  Errors: those of
 * curob_evaluate / curob_evaluatef. */
curob_status curob_h_evaluate(int fid, const double* x, int N, double* out);
curob_status curob_h_evaluatef(int fid, const float* x, int N, float* out);

/* Select the precision of curob_evaluatef (see curob_precision; every value
 * but MIXED; INVALID_ARGUMENT otherwise). */
curob_status curob_set_precision(int mode);

/* Paths of curob_evaluate (FP64) for calls beyond the small-population
 * kernels. */
typedef enum {
  CUROB_PRECISION64_AUTO = 0,   /* TENSOR where the device runs tcgen05, else SIMT */
  CUROB_PRECISION64_SIMT = 1,   /* FP64 pipe: each dot product one fma per term in index order */
  CUROB_PRECISION64_TENSOR = 2  /* seven BF16 digits per operand, 28 products on the tensor
                                   cores, classes summed exactly, z rounded once */
} curob_precision64;

/* Select the path of curob_evaluate (a curob_precision64 value;
 * INVALID_ARGUMENT otherwise).  curob_initialize restores AUTO. */
curob_status curob_set_precision64(int mode);

/* The path curob_evaluate takes for fid beyond the small kernels
 * (CUROB_PRECISION64_TENSOR or _SIMT, AUTO resolved).  Errors:
 * NOT_INITIALIZED, INVALID_FID, INVALID_DIM, NULL_POINTER, UNSUPPORTED
 * (TENSOR forced where the device has no tcgen05). */
curob_status curob_query_precision64(int fid, int* mode);

/* Kernel launches curob_evaluate(fid, ., N, ., .) makes: 1 on the small and
 * SIMT kernels; on the tensor cores, per slice of candidates, the digit
 * launch, a tensor-core launch when the function has a rotated block, and the
 * finish launch.  Errors: as curob_query_precision64, and INVALID_ARGUMENT
 * for N < 0. */
curob_status curob_query_launches64(int fid, int N, int* launches);

/* Small populations (the paper's timing setting, Sec. 2: 50 candidates per
 * call).  A call with N <= max_n candidates -- curob_evaluate, and
 * curob_evaluatef under CUROB_PRECISION_AUTO -- runs on the small-population
 * kernels when every block of the function is at most 128 wide: one warp per
 * candidate and component, one CTA per candidate.  Their arithmetic is that
 * of the FP64 path (curob_evaluate) and of the compensated CUDA-core FP32
 * path (curob_evaluatef, CUROB_PRECISION_SIMT).  max_n = 0 turns them off;
 * the default is 512, and curob_initialize restores it.  Errors:
 * INVALID_ARGUMENT for max_n < 0. */
curob_status curob_set_small_batch(int max_n);

/* *small = 1 when a call of fid on N candidates takes the small-population
 * kernels (see curob_set_small_batch), else 0.  Errors: NOT_INITIALIZED,
 * INVALID_FID, INVALID_DIM, NULL_POINTER, INVALID_ARGUMENT (N < 0). */
curob_status curob_query_small(int fid, int N, int* small);

/* The precision curob_evaluatef will use for fid under the current setting
 * (AUTO resolved): CUROB_PRECISION_TF32X3, _BF16X3, _EXACT, _MIXED or _SIMT.
 * Errors: NOT_INITIALIZED, INVALID_FID, INVALID_DIM, NULL_POINTER,
 * UNSUPPORTED (a forced tensor-core precision the instance cannot use). */
curob_status curob_query_precision(int fid, int* mode);

/* Number of kernel launches curob_evaluatef(fid, ., N, ., .) makes under the
 * current precision.  On the tensor cores, per slice of candidates (the
 * heavy-kind scratch is bounded to 256 MB per slice): one that transposes
 * the slice of x (the tensor-core kernels fetch each stage's variables as
 * rows of x^T), one per precision group, and a finish kernel when a block
 * has a heavy kind (Powers, Weierstrass, Griewank, Schaffer F7, expanded
 * Griewank-Rosenbrock, Modified Schwefel, Katsuura, expanded Schaffer F6:
 * their terms run in a separate kernel over z) or the function is a MIXED
 * composition.  1 on the CUDA-core and small-population kernels.  (If the
 * stream-ordered scratch cannot be had, a call makes fewer: no transpose, or
 * one fused launch.)  Errors: as curob_query_precision, and INVALID_ARGUMENT
 * for N < 0. */
curob_status curob_query_launches(int fid, int N, int* launches);

/* The precision component `comp` of fid runs at (the same as
 * curob_query_precision except for MIXED compositions, where it is EXACT or
 * TF32X3 per member).  INVALID_ARGUMENT for comp outside the function. */
curob_status curob_query_component_precision(int fid, int comp, int* mode);

/* Synchronise `stream` and report (then clear) a latched device-side error. */
curob_status curob_get_device_status(curob_stream_t stream);

/* Self-test of the bounded device-side waits every kernel of the library
 * uses: one CTA waits on an mbarrier that nothing completes; the wait gives
 * up after 2 s and the kernel reports it through a status word instead of
 * hanging or trapping.  Returns CUROB_ERR_DEVICE_TIMEOUT when that works;
 * the context stays usable.  Synchronous; needs no curob_initialize. */
curob_status curob_selftest_bounded_wait(curob_stream_t stream);

/* Human-readable name of a status code (static string). */
const char* curob_status_string(curob_status s);

/* D and max_concurrency of the current instance (host pointers). */
curob_status curob_get_config(int* D, int* max_concurrency);

/* Number of components of fid: N for a composition (Sec. 6), else 1. */
curob_status curob_num_components(int fid, int* ncomp);

/* Block layout of component comp of fid: n_blocks (<= 5) block sizes in
 * z order, and whether the component is rotated.  Unrotated components
 * report one block of size D.  Block sizes: (D/3, D/3, D - 2(D/3)) (General
 * Setup), or ceil(p_i D) with the last taking the rest (Sec. 5, Eq. numbers).
 * Host pointers. */
curob_status curob_component_layout(int fid, int comp, int* n_blocks, int sizes[5], int* rotated);

/* Basic function of each non-empty block of component comp, in z order
 * (host pointers): the Table 1 row 0..22 it is taken from (0 Sphere,
 * 1 Ellipsoid, 2 Elliptic, 3 Discus, 4 Bent Cigar, 5 Different Powers,
 * 6 Sharp Valley, 7 Step, 8 Weierstrass, 9 Griewank, 10 Rastrigin,
 * 11 Schaffer F7, 12 expanded Griewank-Rosenbrock, 13 Rosenbrock,
 * 14 Modified Schwefel, 15 Katsuura, 16 Lunacek bi-Rastrigin, 17 Ackley,
 * 18 HappyCat, 19 HGBat, 20 expanded Schaffer F6); a hybrid's blocks carry
 * their G_i (Sec. 5), a composition member its G (Sec. 6).  Unused entries
 * are -1.  Errors as curob_component_layout. */
curob_status curob_component_kinds(int fid, int comp, int* n_blocks, int kinds[5]);

/* Copy component comp's instance data to host memory: o[D] (x^{opt,comp}),
 * S[D] (variable indices in block order; block b takes S[off_b..off_b+n_b)),
 * R (each rotation block n_b x n_b row-major, blocks back to back; nothing for
 * unrotated components).  Any pointer may be NULL to skip it. */
curob_status curob_get_component(int fid, int comp, double* o, int* S, double* R);

/* Replace component comp's instance data with caller data (host pointers,
 * layout as in curob_get_component), e.g. to evaluate published shift and
 * rotation data.  S must be a permutation of 0..D-1; R's blocks should be
 * orthogonal (not checked).  Synchronous.  Errors: INVALID_ARGUMENT for a
 * bad permutation, NULL_POINTER. */
curob_status curob_set_component(int fid, int comp, const double* o, const int* S, const double* R);

/* x^opt of fid (component 0's shift; for a composition the global optimum,
 * Sec. 6: the member with the smallest bias).  Host pointer, D doubles. */
curob_status curob_get_optimum(int fid, double* xopt);

/* Evaluates n_items functions of the current instance (curob_initialize) on
 * FP32 candidates in one persistent tensor-core launch, WITHOUT ALLOCATING
 * anything: for callers that may not allocate device memory once they are
 * running, e.g. an optimizer that reserves its whole GPU budget at start-up,
 * or a plugin whose host framework owns every device allocation.  The paper
 * has no counterpart; this is a variant of the ragged-batch launch whose
 * work list, argument blocks and work counter live in a 160 KB static device
 * array that every GPU loading the library holds until the process exits.
 * fids[i], x[i] (device, N[i] x D), N[i], out[i] (device, N[i]) describe item
 * i; all host arrays.  Every item uses the EXACT contraction, and every kind
 * is closed in the kernel's epilogue: the values of curob_evaluatef with
 * CUROB_PRECISION_EXACT bit for bit where that call makes one launch
 * (curob_query_launches); where it evaluates heavy kinds in a second kernel,
 * the same within the FP32 tolerance (the partial sums round differently).
 * Limits: at most 64 items and
 * 16384 tiles of 128 candidates per call (CUROB_ERR_CAPACITY beyond), each
 * N[i] <= max_concurrency, block widths <= 512 (else UNSUPPORTED).  The
 * first call on a device looks the array's address up.  All calls share the
 * array and each call overwrites it: calls that overlap on the GPU (two
 * streams, two threads) race; order them on one stream.  The kernel runs
 * asynchronously on `stream`, but the call copies its work list and argument
 * blocks from static (pageable) host arrays, so it may block the host until
 * earlier work on `stream` has finished.  The device current at the call
 * must be the instance's (else INVALID_ARGUMENT). */
curob_status curob_evaluatef_multi_noalloc(const int* fids, const float* const* x, const int* N,
                                           float* const* out, int n_items, curob_stream_t stream);

/* ---------------------------------------------------------------------------
 * Ragged batches (this library's extension; the paper evaluates one function
 * at one D at a time).  A batch is a list of (function, D, seed, population)
 * items evaluated together by persistent tensor-core kernels: each CTA of a
 * grid of at most one CTA per SM takes 128-candidate tiles of any item from a
 * work counter until none is left.  Each item runs at the precision
 * curob_evaluatef's AUTO rule gives its function (TF32X3 where no kind
 * magnifies contraction error, else EXACT; a MIXED composition, and a function
 * AUTO leaves to the CUDA cores, on EXACT), so every item meets the FP32
 * tolerance; the items of each precision form one persistent launch.  The
 * first curob_batch_run times a few schedules (work order per launch, the two
 * launches in sequence or side by side on a split of the SMs, or every item
 * on EXACT in one launch), keeps the fastest, and captures it in a CUDA graph
 * that later runs replay.  A batch
 * owns its instances (one per distinct D, seed); it is independent of
 * curob_initialize.
 * ------------------------------------------------------------------------- */
typedef struct {
  int fid;          /* Table 1 ID */
  int D;            /* dimension: >= 2, >= 10 for IDs 23..28, 35, 36, blocks <= 512 */
  uint64_t seed;    /* instance seed (as curob_initialize) */
  int N;            /* candidates, >= 0 */
  const float* x;   /* device pointer, N x D row-major, read at every run */
  float* out;       /* device pointer, N values, written at every run */
} curob_batch_item;

typedef struct curob_batch_st* curob_batch;

/* Builds the instances and the work list of n_items items (host array).
 * Pointers inside items must stay valid for the life of the batch.  Errors:
 * NULL_POINTER, INVALID_ARGUMENT (n_items < 1, N < 0, host pointers),
 * INVALID_FID, INVALID_DIM, UNSUPPORTED (a block wider than 512, or a device
 * without tcgen05), OUT_OF_MEMORY, CUDA.  Synchronous. */
curob_status curob_batch_create(const curob_batch_item* items, int n_items, curob_batch* batch);

/* Evaluates every item on `stream` (asynchronous): the first call autotunes
 * and captures the CUDA graph (it synchronises the stream while timing and
 * must not be made during a stream capture); later calls launch the graph. */
curob_status curob_batch_run(curob_batch batch, curob_stream_t stream);

/* The same tile arithmetic as one fused launch of the tensor-core kernel per
 * item, in item order, each at the precision the tuner gave its item (values
 * equal to curob_batch_run's bit for bit; call it after the first
 * curob_batch_run). */
curob_status curob_batch_run_separate(curob_batch batch, curob_stream_t stream);

/* Every item as curob_evaluatef under CUROB_PRECISION_AUTO would evaluate it
 * (small-population kernels for N <= 512, else the tensor-core launches with a
 * finish kernel for heavy kinds and MIXED compositions, or the CUDA-core
 * kernel), one item after another on `stream`: the per-call baseline the
 * persistent launches are measured against.  Scratch as curob_evaluatef. */
curob_status curob_batch_run_auto(curob_batch batch, curob_stream_t stream);

/* Schedule chosen by the autotuner (host pointers, any may be NULL): number
 * of work items, grid size (the sum of the two launches' grids when they run
 * side by side), order of the costlier launch (0 = longest first, 1 = round
 * robin over items, 2 = item order).  NOT_INITIALIZED before the first run. */
curob_status curob_batch_schedule(curob_batch batch, int* n_work, int* grid, int* order);

/* The autotuner's choices per precision (host pointers, any may be NULL):
 * items and work items on EXACT and on TF32X3, each launch's grid (0 when it
 * has no work) and work order, and whether the two launches run side by side
 * (1) or one after the other (0).  NOT_INITIALIZED before the first run. */
curob_status curob_batch_plan(curob_batch batch, int* items_exact, int* items_tf32,
                              int* work_exact, int* work_tf32, int* grid_exact, int* grid_tf32,
                              int* order_exact, int* order_tf32, int* concurrent);

/* Synchronises `stream` and reports (then clears) a device-side error of any
 * of the batch's instances. */
curob_status curob_batch_status(curob_batch batch, curob_stream_t stream);

/* Releases the batch (synchronises the device first). */
curob_status curob_batch_destroy(curob_batch batch);

/* ---------------------------------------------------------------------------
 * Learned pre-screen (this library's extension; the paper has no learned
 * part).  A surrogate is an MLP 100 -> 256 -> 256 -> 1 of one function at
 * D = 100: u = x / 128, a1 = W1 u + b1, h1 = gelu(a1), a2 = W2 h1 + b2,
 * h2 = gelu(a2), y = w3 . h2 + b3, gelu(a) = a Phi(a) with Phi the standard
 * normal CDF (Hendrycks and Gimpel 2016).  It predicts t = log(f - f_opt + 1)
 * as mu + sd * y, mu and sd the mean and standard deviation of t over its
 * training set.  Training minimises the mean squared error of y against
 * (t - mu) / sd with AdamW (Loshchilov and Hutter 2019: w <- w (1 - lr wd),
 * then the bias-corrected Adam step, eps added to sqrt(v_hat)).  Weights are
 * FP32 masters with BF16 copies; every contraction (forward and backward)
 * runs on the tensor cores with BF16 operands (u, h1, dL/da2, dL/da1 rounded
 * to nearest-even BF16 where they enter one) and FP32 accumulation; biases,
 * activations outside contractions and reductions are FP32.
 *
 * Flat parameter vector (CUROB_SURROGATE_PARAMS floats): W1 (256 x 100,
 * row = output unit), b1 (256), W2 (256 x 256), b2 (256), w3 (256), b3.
 * All x, f, out, idx pointers below are DEVICE pointers unless stated;
 * calls are asynchronous on `stream` unless stated.  Kernel-side errors
 * (bounded waits) are reported by curob_surrogate_device_status.
 * ------------------------------------------------------------------------- */
#define CUROB_SURROGATE_INPUT 100
#define CUROB_SURROGATE_HIDDEN 256
#define CUROB_SURROGATE_PARAMS 91905

typedef struct curob_surrogate_st* curob_surrogate;

/* Text of the last CUDA failure recorded on the calling thread by the
 * surrogate and selection entry points (the failing step and CUDA's error
 * string), or "" when none.  Owned by the library. */
const char* curob_last_error(void);

/* Allocates a surrogate on the current device for training batches of up to
 * max_batch rows (a multiple of 128, <= 2^20), initialised like PyTorch's
 * linear layers (weights and biases uniform in +-1/sqrt(fan_in)) from a
 * generator seeded by `seed`; mu = 0, sd = 1; AdamW lr 1e-3, betas (0.9,
 * 0.999), eps 1e-8, weight decay 1e-4.  Errors: NULL_POINTER,
 * INVALID_ARGUMENT, UNSUPPORTED (no tcgen05), OUT_OF_MEMORY.  Synchronous. */
curob_status curob_surrogate_create(int max_batch, uint64_t seed, curob_surrogate* s);
curob_status curob_surrogate_destroy(curob_surrogate s);

/* AdamW hyper-parameters (lr is the default of curob_surrogate_step's
 * callers; curob_surrogate_fit takes its own schedule). */
curob_status curob_surrogate_set_hyper(curob_surrogate s, float lr, float beta1, float beta2,
                                       float eps, float weight_decay);

/* FP32 master parameters to / from a HOST array of CUROB_SURROGATE_PARAMS
 * floats (synchronous).  set_params also zeroes the AdamW moments and step. */
curob_status curob_surrogate_get_params(curob_surrogate s, float* host_params);
curob_status curob_surrogate_set_params(curob_surrogate s, const float* host_params);

/* Gradient of the loss of the last curob_surrogate_step / fit step, as a
 * HOST array laid out like the parameters (synchronous). */
curob_status curob_surrogate_get_grads(curob_surrogate s, float* host_grads);

/* Target standardisation: set directly, read back, or computed (FP64, one
 * kernel) as the mean and standard deviation of log(max(f - f_opt, 0) + 1)
 * over n device values f (synchronises the stream; sd = 1 when it is 0). */
curob_status curob_surrogate_set_standardisation(curob_surrogate s, float mu, float sd);
curob_status curob_surrogate_get_standardisation(curob_surrogate s, float* mu, float* sd);
curob_status curob_surrogate_standardise(curob_surrogate s, const float* f, long long n,
                                         float f_opt, curob_stream_t stream);

/* One step on a batch of B candidates x (B x 100) with exact values f (B):
 * forward, loss, back-propagation; with update != 0 also the AdamW update at
 * learning rate lr.  loss_out (device, may be NULL) receives the batch's
 * mean loss.  B a multiple of 128, <= max_batch (else CAPACITY). */
curob_status curob_surrogate_step(curob_surrogate s, const float* x, const float* f, int B,
                                  float f_opt, float lr, int update, float* loss_out,
                                  curob_stream_t stream);

/* Trains on n samples (x: n x 100, f: n): standardises the targets (as
 * curob_surrogate_standardise), then `epochs` passes over floor(n / batch)
 * batches of consecutive rows, the batch order reshuffled every epoch
 * (Fisher-Yates, seeded by shuffle_seed), learning rate on a cosine from
 * lr_max down to lr_max / 20.  loss_hist (device, may be NULL) receives
 * epochs * floor(n / batch) batch losses.  Uses ~512 bytes of device memory
 * per sample for the duration of the call. */
curob_status curob_surrogate_fit(curob_surrogate s, const float* x, const float* f, long long n,
                                 float f_opt, int epochs, int batch, float lr_max,
                                 uint64_t shuffle_seed, float* loss_hist, curob_stream_t stream);

/* Predicted t = mu + sd * y for N candidates x (N x 100) into out (N). */
curob_status curob_surrogate_predict(curob_surrogate s, const float* x, long long N, float* out,
                                     curob_stream_t stream);

/* Synchronises `stream` and reports (then clears) a device-side error of the
 * surrogate's kernels (DEVICE_TIMEOUT). */
curob_status curob_surrogate_device_status(curob_surrogate s, curob_stream_t stream);

/* Indices of the k smallest of v[0..N-1] (0 <= k <= N < 2^31), equal values
 * taken in index order, written to idx[0..k-1] in ascending index order; NaN
 * ranks above +inf.  Radix selection on the order-preserving integer keys,
 * exact (bit-identical to a full sort).  Uses a small stream-ordered
 * allocation.  INVALID_ARGUMENT for k outside [0, N]. */
curob_status curob_select_smallest(const float* v, long long N, int k, int* idx,
                                   curob_stream_t stream);

/* out[r][:] = x[idx[r]][:] for r < k (rows of D floats). */
curob_status curob_gather_rows(const float* x, int D, const int* idx, int k, float* out,
                               curob_stream_t stream);

/* One generation of surrogate pre-screening on the current instance (D must
 * be 100): predicts all N pool candidates (pred, N), keeps the k with the
 * smallest prediction (idx, ascending), gathers them (x_sel, k x 100) and
 * evaluates them exactly with curob_evaluatef (f_sel, k; k <= the
 * instance's max_concurrency).  Errors: INVALID_DIM (D != 100), CAPACITY,
 * INVALID_ARGUMENT, and those of curob_evaluatef. */
curob_status curob_surrogate_screen(curob_surrogate s, int fid, const float* pool, long long N,
                                    int k, float* pred, int* idx, float* x_sel, float* f_sel,
                                    curob_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CUROB_H */

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
 * 7-bit integer slices held in BF16, accumulated exactly (every partial sum
 * an integer below 2^24), z to about 2^-28 of each candidate's |x - o|_max.
 * SIMT: FP32 CUDA cores with a compensated dot product.  AUTO (default):
 * EXACT for functions containing Discus, Weierstrass, expanded
 * Griewank-Rosenbrock or Katsuura (they magnify z errors), TF32X3 for the
 * rest; SIMT where a block is narrower than 16 or wider than 512. */
typedef enum {
  CUROB_PRECISION_AUTO = 0,
  CUROB_PRECISION_TF32X3 = 1,
  CUROB_PRECISION_BF16X3 = 2,
  CUROB_PRECISION_SIMT = 3,
  CUROB_PRECISION_EXACT = 4
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
 * Errors: NOT_INITIALIZED, INVALID_FID, INVALID_DIM, CAPACITY, NULL_POINTER,
 * INVALID_ARGUMENT, CUDA.  Asynchronous on `stream`. */
curob_status curob_evaluate(int fid, const double* x, int N, double* out, curob_stream_t stream);

/* Sec. 1.3, func_evaluatef(): the same with FP32 x and out.  The shift x - o
 * is taken in FP64 (o is FP64), the block rotation runs on the tensor cores
 * in the precision set by curob_set_precision, reductions are carried in
 * FP64 across lanes.  Same errors as curob_evaluate, plus UNSUPPORTED if a
 * forced precision cannot handle the instance's block sizes. */
curob_status curob_evaluatef(int fid, const float* x, int N, float* out, curob_stream_t stream);

/* Sec. 1.3, h_func_evaluate / h_func_evaluatef: host-pointer wrappers.
 * Copy x in, evaluate on the library's own stream, copy out, synchronise. */
curob_status curob_h_evaluate(int fid, const double* x, int N, double* out);
curob_status curob_h_evaluatef(int fid, const float* x, int N, float* out);

/* Select the precision of curob_evaluatef (see curob_precision). */
curob_status curob_set_precision(int mode);

/* The precision curob_evaluatef will use for fid under the current setting
 * (AUTO resolved): CUROB_PRECISION_TF32X3, _BF16X3, _EXACT or _SIMT.
 * Errors: NOT_INITIALIZED, INVALID_FID, INVALID_DIM, NULL_POINTER,
 * UNSUPPORTED (a forced tensor-core precision the instance cannot use). */
curob_status curob_query_precision(int fid, int* mode);

/* Synchronise `stream` and report (then clear) a latched device-side error. */
curob_status curob_get_device_status(curob_stream_t stream);

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
 * i; all host arrays.  Every item uses the EXACT contraction (same values as
 * curob_evaluatef with CUROB_PRECISION_EXACT).  Limits: at most 64 items and
 * 16384 tiles of 128 candidates per call (CUROB_ERR_CAPACITY beyond), each
 * N[i] <= max_concurrency, block widths <= 512 (else UNSUPPORTED).  The
 * first call on a device looks the array's address up.  All calls share the
 * array and each call overwrites it: calls that overlap on the GPU (two
 * streams, two threads) race; order them on one stream.  Asynchronous on
 * `stream`. */
curob_status curob_evaluatef_multi_noalloc(const int* fids, const float* const* x, const int* N,
                                           float* const* out, int n_items, curob_stream_t stream);

/* ---------------------------------------------------------------------------
 * Ragged batches (this library's extension; the paper evaluates one function
 * at one D at a time).  A batch is a list of (function, D, seed, population)
 * items evaluated together by one persistent tensor-core kernel: each CTA of
 * a grid of at most one CTA per SM takes 128-candidate tiles of any item from
 * a work counter until none is left.  Every item uses the EXACT contraction
 * (curob_precision), so any function at any block width up to 512 meets the
 * FP32 tolerance.  The first curob_batch_run times a few schedules (work
 * order, grid size), keeps the fastest, and captures it in a CUDA graph that
 * later runs replay.  A batch owns its instances (one per distinct D, seed);
 * it is independent of curob_initialize.
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

/* The same work as one launch of the tensor-core kernel per item, in item
 * order (the baseline the persistent launch is measured against). */
curob_status curob_batch_run_separate(curob_batch batch, curob_stream_t stream);

/* Schedule chosen by the autotuner (host pointers, any may be NULL): number
 * of work items, grid size, order (0 = longest first, 1 = round robin over
 * items, 2 = item order).  NOT_INITIALIZED before the first run. */
curob_status curob_batch_schedule(curob_batch batch, int* n_work, int* grid, int* order);

/* Synchronises `stream` and reports (then clears) a device-side error of any
 * of the batch's instances. */
curob_status curob_batch_status(curob_batch batch, curob_stream_t stream);

/* Releases the batch (synchronises the device first). */
curob_status curob_batch_destroy(curob_batch batch);

#ifdef __cplusplus
}
#endif
#endif /* CUROB_H */

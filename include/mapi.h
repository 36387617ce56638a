/*
 * mapi.h -- C ABI of the GB300 (sm_103a) library for multiplication-avoiding
 * power iteration (MAPI), after H. Pan, D. Badawi, R. Miao, E. Koyuncu and
 * A. E. Cetin, "Multiplication-Avoiding Variant of Power Iteration with
 * Applications" (arXiv 2110.12065).
 *
 * Vocabulary (paper notation)
 *   (+)   an MAVP "vector product": min1 (.) of Eq. (3),
 *         w^T (.) x = sum_i sign(w_i x_i) min(|w_i|, |x_i|), or min2 (.)_m of
 *         Eq. (4), sum_i 1(sign w_i = sign x_i) min(|w_i|, |x_i|).
 *   A (+) w   the row-wise product: (A (+) w)_i = a_i^T (+) w, a_i = row i.
 *   MAPI  Eq. (6) / Alg. 1: w <- (A (+) w) / ||A (+) w||_1.
 *   RPI   Eq. (1): b <- A b / ||A b||_2 (op MAPI_OP_DOT).
 *
 * Conventions for every entry point
 *   - Every call returns a mapi_status; nothing throws across the ABI.
 *   - Device pointers are plain CUDA device addresses on the context's
 *     device (for example torch tensors' data_ptr()); they stay owned by the
 *     caller.  Work is ordered on the context's stream (mapi_config
 *     .cuda_stream); calls that return host results synchronise that stream
 *     before returning.
 *   - Matrices are dense, row-major, with a leading dimension ld >= cols (in
 *     elements).  Vectors are contiguous; several vectors are column-major
 *     with a leading dimension.
 *   - Matrices uploaded with mapi_matrix_upload are copied into a packed,
 *     library-owned device copy (mapi_mat); free them with mapi_matrix_free or
 *     mapi_destroy.
 *   - One context is used by one host thread at a time.
 *   - Arithmetic on the device is FP32 (float storage) or exact INT32/INT64
 *     (integer storage); no step uses FP64 on the GPU.
 *   - On any error the outputs are unspecified and the detail text is
 *     available from mapi_last_error(ctx).
 */
#ifndef MAPI_H
#define MAPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mapi_ctx mapi_ctx; /* opaque; one per device */
typedef struct mapi_mat mapi_mat; /* opaque; a packed device matrix */

typedef enum {
  MAPI_OK = 0,
  MAPI_EINVAL = 1,     /* bad argument: null pointer, size, op/storage pair */
  MAPI_ENOMEM = 2,     /* a device or pinned allocation failed */
  MAPI_EBUDGET = 3,    /* a request can never fit the HBM admission budget */
  MAPI_EZERONORM = 4,  /* ||A (+) w|| = 0 (e.g. A = 0, or min2 with all signs
                          opposed); the last good iterate is returned */
  MAPI_ENONFINITE = 5, /* NaN/Inf in an input or a norm */
  MAPI_EAGAIN = 6,     /* mapi_poll: the request is still running */
  MAPI_ETIMEOUT = 7,   /* a bounded device wait gave up */
  MAPI_ECANCELLED = 8, /* the request was cancelled */
  MAPI_ECUDA = 9,      /* a CUDA runtime call failed */
  MAPI_ENOTSUP = 10    /* valid but not supported in this build */
} mapi_status;

/* The vector product used in A (+) w.
 *   MIN1    Eq. (3)
 *   MIN2    Eq. (4)
 *   DIAMOND Eq. (7), read as sum_i sign(w_i) x_i + w_i sign(x_i) (the
 *           printed formula mixes the letters; the proof of Proposition 1
 *           fixes this reading).  Test mode: Proposition 1 pins it.
 *   DOT     the ordinary product: regular power iteration, Eq. (1), which
 *           also switches the per-step normalisation to the l2 norm. */
typedef enum {
  MAPI_OP_MIN1 = 0,
  MAPI_OP_MIN2 = 1,
  MAPI_OP_DIAMOND = 2,
  MAPI_OP_DOT = 3
} mapi_op;

/* Storage of a packed matrix (the paper fixes none).  Reduced-precision
 * copies round to nearest even.  Since (c A) (+) w != c (A (+) w), every
 * scale is an exact power of two and is undone exactly inside the kernels.
 *   F32             4 B/element
 *   BF16            2 B/element
 *   FP8E4M3_ROWPOW2 1 B/element plus one scale 2^k_i per row, k_i the
 *                   smallest integer with max_j |a_ij| <= 448 * 2^k_i
 *   I16 / I8        fixed point with one shared exponent q: A_q =
 *                   RNE(A 2^q), q the largest in [0, 24] with max|A| 2^q <=
 *                   32767 (I16) or 127 (I8); the whole iteration then runs in
 *                   exact integers (MIN1/MIN2 only) */
typedef enum {
  MAPI_ST_F32 = 0,
  MAPI_ST_BF16 = 1,
  MAPI_ST_FP8E4M3_ROWPOW2 = 2,
  MAPI_ST_I16 = 3,
  MAPI_ST_I8 = 4
} mapi_storage;

/* Element type of an upload source. */
typedef enum { MAPI_SRC_F32 = 0 } mapi_src_dtype;

/* int_scale_log2 value that asks mapi_matrix_upload to pick q itself. */
#define MAPI_SCALE_AUTO ((int)0x80000000)

/* flags of mapi_iterate */
#define MAPI_FLAG_FINAL_L2 1u  /* Alg. 1 optional last step: w_T / ||w_T||_2 */
#define MAPI_FLAG_RAW_START 2u /* use w0 as given; by default w0 is first
                                  scaled to ||w0||_2 = 1 (Alg. 1 step 1) */

typedef struct {
  int device;              /* CUDA device ordinal */
  size_t hbm_budget_bytes; /* admission budget for served requests (0: none) */
  void* cuda_stream;       /* cudaStream_t for all work; NULL: a stream the
                              context creates and owns */
  int max_slots;           /* served requests resident at once (0: 64) */
  const char* tune_cache_path; /* autotuner cache file, NULL: in memory only */
} mapi_config;

/* Create a context on cfg->device.  *out receives the handle.
 * Errors: MAPI_EINVAL (null pointers, bad device), MAPI_ECUDA. */
mapi_status mapi_create(const mapi_config* cfg, mapi_ctx** out);

/* Release the context, every matrix it owns and its device buffers.
 * Synchronises the context's stream first. */
mapi_status mapi_destroy(mapi_ctx* ctx);

/* Static English text for a status code. */
const char* mapi_status_str(mapi_status s);

/* Detail text of the last failing call on ctx (owned by ctx; "" if none). */
const char* mapi_last_error(const mapi_ctx* ctx);

/*
 * Pack a rows x cols matrix into the chosen storage (library-owned device
 * copy).  src: rows x cols row-major FP32 values with leading dimension ld
 * (elements), in device memory if src_is_device else in host memory.
 * int_scale_log2: q for I16/I8 storage, or MAPI_SCALE_AUTO; ignored for the
 * float storages.  The packed copy pads every row to a multiple of 16 bytes
 * (and the row count to a multiple of 64) with zeros; zero entries add
 * nothing to any product.
 * A host source is copied into a device staging buffer that the context
 * keeps (grown to the largest host upload so far, released by
 * mapi_destroy); the call returns once the copy is done, so the host buffer
 * may then be reused.
 * Errors: MAPI_EINVAL (sizes, ld < cols, storage, q out of [0, 24] or
 * entries too large for the integer range), MAPI_ENONFINITE (NaN/Inf
 * entry), MAPI_ENOMEM, MAPI_ECUDA.
 */
mapi_status mapi_matrix_upload(mapi_ctx* ctx, const void* src, int src_is_device,
                               int src_dtype, int rows, int cols, int64_t ld,
                               mapi_storage storage, int int_scale_log2,
                               mapi_mat** out);

/* Free a packed matrix (synchronises the context's stream first).  The
 * device storage of up to two freed matrices is kept by the context and
 * reused by the next matrix of exactly the same size; mapi_destroy, or an
 * allocation that would otherwise fail, releases it. */
mapi_status mapi_matrix_free(mapi_ctx* ctx, mapi_mat* m);

/* Shape and storage of a packed matrix; any output pointer may be NULL.
 * int_scale_log2 receives q for integer storage, 0 otherwise; ld_elems the
 * padded row length in elements. */
mapi_status mapi_matrix_info(const mapi_mat* m, int* rows, int* cols,
                             int64_t* ld_elems, int* storage,
                             int* int_scale_log2);

/* Read back the values the packed copy represents, dequantised exactly, as
 * doubles: host_out is a caller-owned host array of rows x cols (row-major,
 * leading dimension cols).  For FP8 storage row_exp (host, rows ints, may be
 * NULL) receives the exponents k_i.  Synchronous. */
mapi_status mapi_matrix_download(mapi_ctx* ctx, const mapi_mat* m,
                                 double* host_out, int* row_exp);

/*
 * Algorithm 1 (MAPI), or regular power iteration with MAPI_OP_DOT, on a
 * square packed matrix A (n x n), for nvec independent start vectors that
 * share every read of A (nvec in 1..8).
 *   w0     device, n x nvec column-major FP32 with leading dimension ldw
 *          (>= n): the start vectors, scaled to unit l2 norm first unless
 *          MAPI_FLAG_RAW_START (Alg. 1 step 1).
 *   Each step: y = A (+) w (Alg. 1 step 3), w = y / ||y||_1 (step 4; the l2
 *   norm for MAPI_OP_DOT), delta = ||w_new - w_old||_1.  A vector stops
 *   after max_iters steps or once delta < tol_l1 (tol_l1 <= 0: never).
 *   w_out  device, n x nvec column-major (leading dimension ldw): the last
 *          iterate, l2-normalised if MAPI_FLAG_FINAL_L2 (Alg. 1 step 6).
 *   iters_done, last_delta: host arrays of nvec entries (may be NULL).
 * Integer storage: w0 is quantised to RNE(w0 2^q), l1-normalised by the
 * integer rule w_i = sign(y_i) floor((|y_i| 2^q + floor(L/2)) / L), and
 * every step runs in exact integers with the same rule (the n divisions of
 * §2.2); w_out holds w_q 2^-q exactly.  Only MIN1/MIN2 are allowed there.
 * Errors: MAPI_EINVAL (shape, op/storage pair, nvec), MAPI_EZERONORM (some
 * vector hit a zero norm; its last good iterate is returned), MAPI_ENONFINITE,
 * MAPI_ECUDA.  Synchronous.
 */
mapi_status mapi_iterate(mapi_ctx* ctx, const mapi_mat* A, mapi_op op,
                         int nvec, const float* w0, int64_t ldw, int max_iters,
                         double tol_l1, unsigned flags, float* w_out,
                         int* iters_done, double* last_delta);

/*
 * MAPI, then regular power iteration (the switch §3.2 suggests when the
 * eigenvector itself is wanted): Alg. 1 with op (MIN1, MIN2 or DIAMOND) from
 * w0 for up to mapi_iters steps or until its delta < mapi_tol; its last
 * iterate is the start vector (scaled to unit l2 norm, Alg. 1 step 1) of
 * Eq. (1)'s iteration for up to rpi_iters steps or until delta < rpi_tol.
 *   A: square float storage.  w0, w_out: device n FP32 (caller-owned).
 *   flags: MAPI_FLAG_RAW_START applies to the first phase, MAPI_FLAG_FINAL_L2
 *     to the result (the second phase already ends l2-normalised).
 *   iters_done, last_delta: host arrays of 2 (phase 1, phase 2), may be NULL.
 * Errors: MAPI_EINVAL; a status of the first phase (then w_out holds its last
 * good iterate) or of the second; MAPI_ECUDA.  Synchronous.
 */
mapi_status mapi_iterate_switch(mapi_ctx* ctx, const mapi_mat* A, mapi_op op, const float* w0,
                                int mapi_iters, double mapi_tol, int rpi_iters, double rpi_tol,
                                unsigned flags, float* w_out, int* iters_done,
                                double* last_delta);

/*
 * Mini-batch MAPI with momentum, Alg. 3 (and, with MAPI_OP_DOT, the
 * momentum power method it is set against in §3.2), one CTA for all steps.
 *   X      device, N x D row-major FP32 (rows are samples), 1 <= D <= 128.
 *   batch  device, T x s row-major int32 (NULL when T = 0): the s sample
 *          indices of step t
 *          (Alg. 3 step 3 draws them; the caller passes the draws).
 *   Step 1: w_0 = w0 / ||w0||_2, w_{-1} = 0.  Step t: A_t = (1/s) sum over
 *   the batch of x (+) x^T, v = A_t (+) w_t - beta w_{t-1}, then
 *   w_{t+1} = v / L and w_t / L for the momentum term, L = ||v||_1
 *   (||v||_2 for DOT).  After T steps w_T goes to w_out, scaled to unit l2
 *   norm if MAPI_FLAG_FINAL_L2.
 *   op: MIN1, MIN2 or DOT.  w0, w_out: device D FP32 (caller-owned).
 * Errors: MAPI_EINVAL (shape, op, an index outside [0, N)), MAPI_EZERONORM,
 * MAPI_ENONFINITE (the step's norm), MAPI_ECUDA.  Synchronous.
 */
mapi_status mapi_minibatch_momentum(mapi_ctx* ctx, const float* X, int N, int D,
                                    const int* batch, int T, int s, double beta, mapi_op op,
                                    const float* w0, unsigned flags, float* w_out);

/*
 * Min-covariance matrix, Eq. (5): C = (1/denom) X (+) X^T for a packed
 * X (D x N, columns are samples); op MIN1, MIN2 or DOT (then C is the
 * ordinary covariance of Eq. (2)).  Eq. (5) uses denom = N, Alg. 2 step 4
 * uses N - 1.  C_out: device, D x D row-major FP32, caller-owned.
 * Errors: MAPI_EINVAL, MAPI_ECUDA.  Asynchronous on the context stream.
 */
mapi_status mapi_mincov(mapi_ctx* ctx, const mapi_mat* X, mapi_op op,
                        double denom, float* C_out);

/*
 * Outer-product projection, Alg. 2 step 8 (and the operator of step 6):
 * out_r = (W (+) W^T) in_r + add for `rows` input rows, with
 * (W (+) W^T)_pq = sum_c term(wt_pc, wt_qc) (the matrix extension of the
 * operator) and an ordinary product with in_r.  wt_c is column c of W at the
 * unit norm of its iteration: W_c / ||W_c||_1 for MIN1 / MIN2 (Eq. (8)), W_c
 * as given for DOT (then the product is W W^T in_r).  The D x D matrix is
 * never formed: each component is ranked by |wt| once and every row takes
 * two prefix sums over that order.
 *   W: device D x k column-major (leading dimension ldw >= D), k in 1..64.
 *   in, out: device rows x D row-major (ld_in, ld_out >= D); add: device D
 *   or NULL.  1 <= D <= 16384.
 * Errors: MAPI_EINVAL, MAPI_ECUDA.  Asynchronous on the context stream.
 */
mapi_status mapi_mavp_project(mapi_ctx* ctx, mapi_op op, const float* W, int64_t ldw, int D,
                              int k, const float* in, int64_t ld_in, int rows, const float* add,
                              float* out, int64_t ld_out);

/*
 * Image reconstruction by MAPI, Alg. 2 end to end.  images: device N x P
 * row-major FP32, row i the pixels of image i (steps 1-2: v_i, V = [v_1 ..
 * v_N]).  Step 3: m = the mean image, V - m.  Step 4: C = (V - m) (+)
 * (V - m)^T / (N - 1) (P x P).  Steps 5-6: k components by MAPI (op MIN1 or
 * MIN2; DOT gives the RPI baseline), each on C_c = C - sum_{m<c} P_m C, for
 * iters steps (or until delta < tol_l1), ended at unit l2 norm.  Step 8, for
 * every image: recon_i = (W (+) W^T)(v_i - m) + m as in mapi_mavp_project.
 *   w0: device P x k column-major raw start vectors.  W_out: device P x k
 *   column-major, the components.  recon_out: device N x P row-major.
 *   iters_done: host k ints (may be NULL).  N >= 2, 1 <= P <= 16384,
 *   1 <= k <= min(P, 64).
 * Errors: MAPI_EINVAL, MAPI_EZERONORM / MAPI_ENONFINITE (a component; then
 * recon_out is not written), MAPI_ENOMEM, MAPI_ECUDA.  Synchronous.
 */
mapi_status mapi_image_reconstruct(mapi_ctx* ctx, const float* images, int N, int P, int k,
                                   mapi_op op, int iters, double tol_l1, const float* w0,
                                   float* W_out, float* recon_out, int* iters_done);

#define MAPI_PCA_MINCOV 0 /* Alg. 2: C = X (+) X^T / denom, deflate, MAPI */
#define MAPI_PCA_PAIR 1   /* matrix-free: t = X^T (+) w, y = X (+) t / denom */

/*
 * Top-k principal vectors by MAPI (Alg. 2 steps 4-7, k components).
 *   MINCOV: C = (1/cov_denom) X (+) X^T once; component c runs Alg. 1 on
 *     C_c = (I - sum_{m<c} P_m) C, P_m = wt_m (+) wt_m^T built from the
 *     earlier components at the unit norm of their iteration (l1 for MIN1 /
 *     MIN2, l2 for DOT), the product P_m C being ordinary (Alg. 2 step 6 with
 *     the sum form that follows Eq. (2)); k > 1 needs D <= 16384.
 *   PAIR: component c iterates y = X (+) (X^T (+) w) / cov_denom on X
 *     directly (t_n = x_n^T (+) w for every sample n, then y_d = sum_n
 *     X_dn (+) t_n / cov_denom), deflates y <- y - sum_{m<c} P_m y, and
 *     normalises (l1; l2 for DOT).  The paper has no such step; it is the
 *     matrix-free counterpart of C w = X (X^T w) / N.
 *   Both end every component with the l2 normalisation (§2.2).
 *   w0: device, D x k column-major raw start vectors (each scaled to unit l2
 *   norm first).  P_out: device, D x k column-major.  iters_done: host, k
 *   ints (may be NULL).  tol_l1 <= 0 runs exactly iters_per_vec steps.
 * Errors: MAPI_EINVAL (k outside 1..min(D, 64), op), MAPI_ENOTSUP (MINCOV
 * with k > 1 and D > 16384), MAPI_EZERONORM, MAPI_ENOMEM, MAPI_ECUDA.
 * Synchronous.
 */
mapi_status mapi_pca_topk(mapi_ctx* ctx, const mapi_mat* X, int k, int mode,
                          mapi_op op, int iters_per_vec, double tol_l1,
                          double cov_denom, const float* w0, float* P_out,
                          int* iters_done);

/*
 * Google matrix of §3.3, Eq. (11), packed in the chosen storage:
 * G = alpha H + (1 - alpha)/n 1, H column-stochastic with H_ij =
 * (#links j -> i)/outdeg(j), dangling columns uniform (1/n).  The graph is
 * out-link CSR in device memory: the targets of node j are
 * indices[indptr[j] .. indptr[j+1]) (int32, n+1 and nnz entries).
 * Errors: MAPI_EINVAL (n, alpha outside [0, 1], index out of range is not
 * checked on the device: the caller guarantees 0 <= indices < n),
 * MAPI_ENOMEM, MAPI_ECUDA.
 */
mapi_status mapi_google_matrix(mapi_ctx* ctx, const int* indptr,
                               const int* indices, int n, double alpha,
                               mapi_storage storage, mapi_mat** out);

/*
 * MAPI-PageRank (§3.3): builds G as mapi_google_matrix does, runs Alg. 1
 * with op from w0 (device, n FP32) and ends with one l2 normalisation, as
 * the paper does "for easier comparison".  rank_out: device, n FP32.
 * iters_done / last_delta: host scalars (may be NULL).  Synchronous.
 */
mapi_status mapi_pagerank(mapi_ctx* ctx, const int* indptr, const int* indices,
                          int n, double alpha, mapi_storage storage,
                          mapi_op op, const float* w0, int max_iters,
                          double tol_l1, float* rank_out, int* iters_done,
                          double* last_delta);

/*
 * MAPI-PageRank (§3.3) without forming G: each step costs O(E + n) instead
 * of O(n^2).  Every entry of G (Eq. (11)) is one of three values: the
 * teleport value (1 - alpha)/n, that value plus alpha * (#links j -> i)/d_j
 * on a link, or alpha/n plus it in a dangling column, each formed in FP64
 * and rounded to FP32 exactly as mapi_google_matrix stores them.  Row i of
 * G (+) w is then one base sum over all columns plus a correction for each
 * in-link of i.  Same iteration, stop rule and final l2 step as
 * mapi_pagerank; only the FP32 summation order differs.
 *   indptr, indices: device out-link CSR (n + 1 and indptr[n] int32; indices
 *     may be NULL when indptr[n] = 0), checked on the device: an entry out of
 *     range returns MAPI_EINVAL.
 *   op: MIN1, MIN2 or DOT.  w0: device n FP32.  rank_out: device n FP32.
 *   iters_done / last_delta: host scalars (may be NULL).
 * Errors: MAPI_EINVAL, MAPI_ENOTSUP (a node with more than 16384 in-links),
 * MAPI_ENOMEM, MAPI_EZERONORM, MAPI_ENONFINITE, MAPI_ECUDA.  Synchronous.
 */
mapi_status mapi_pagerank_sparse(mapi_ctx* ctx, const int* indptr, const int* indices, int n,
                                 double alpha, mapi_op op, const float* w0, int max_iters,
                                 double tol_l1, float* rank_out, int* iters_done,
                                 double* last_delta);


/* ------------------------------------------------------------------ */
/* Pieces of a partitioned solve.  When the data is split over processes */
/* (one GPU each), each rank computes the unnormalised product of its    */
/* shard, the ranks combine them (a gather of row blocks, or a sum of    */
/* column-shard partials), and the normalisation of Eq. (6) (and, for    */
/* PCA, the deflation of Alg. 2 step 6) is applied to the whole vector.  */
/* ------------------------------------------------------------------ */

/*
 * y_out[r] = a_i^T (+) w for the rows i = row_begin + r < row_end of A: the
 * matrix-vector product of Alg. 1 step 3 (matrix extension of §2.1) for a
 * block of rows, before the l1 normalisation.  Row-partitioned MAPI: rank k
 * holds all of w and its rows' results; gathering the blocks gives A (+) w.
 *   A: packed matrix in F32, BF16 or FP8 storage (integer storage has the
 *      exact path of mapi_iterate only: MAPI_EINVAL).
 *   op: MIN1, MIN2 or DOT.  w: device, A->cols FP32 (used as given).
 *   y_out: device, row_end - row_begin FP32 (caller-owned).
 * FP32 accumulation (one warp per row).  MAPI_EINVAL for rows outside A.
 * Synchronous on the context's stream.
 */
mapi_status mapi_rows_product(mapi_ctx* ctx, const mapi_mat* A, int row_begin, int row_end,
                              mapi_op op, const float* w, float* y_out);

/*
 * The pair product of the PCA pair mode on X (D x N) without its
 * denominator, deflation or normalisation:
 *   t_n = x_n^T (+) w,  y_out[d] = sum_n X_dn (+) t_n.
 * Column-partitioned PCA: rank k holds the columns (samples) of its shard as
 * its own X; the sum of the ranks' y_out is the product over all of X, since
 * t_n depends only on column n.  w: device, D FP32, used as given.  y_out:
 * device, D FP32.  Same kernel as the pair mode of mapi_pca_topk (one step;
 * row sums added exactly in 64-bit fixed point).  X in F32 or BF16 storage,
 * D <= 1024; op MIN1, MIN2 or DOT.  Synchronous.
 */
mapi_status mapi_pair_partial(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, const float* w,
                              float* y_out);

/* ------------------------------------------------------------------ */
/* Diagnostics: kernel timing and launch counting.  Not part of the    */
/* paper's method; they let a caller measure the kernels against their */
/* rooflines without an external profiler.                             */
/* ------------------------------------------------------------------ */

/* Kernel classes timed by mapi_profile. */
typedef enum {
  MAPI_KC_GEMV = 0,        /* K1 MAVP-GEMV step (Alg. 1 steps 3-4) */
  MAPI_KC_PAIR = 1,        /* pair steps over X, their reduction, deflation and
                              normalisation included: one persistent launch
                              per component, counted as max_iters steps */
  MAPI_KC_PAIR_FINISH = 2, /* reserved: the pair step has no separate finish
                              kernel, so this class stays empty */
  MAPI_KC_MINCOV = 3,      /* min-covariance build, Eq. (5) */
  MAPI_KC_BATCHED = 4,     /* persistent batched solve (whole launch) */
  MAPI_KC_COUNT = 5
} mapi_kernel_class;

typedef struct {
  uint64_t launches;             /* kernels launched by the library (each node
                                    of a replayed CUDA graph counts once) */
  uint64_t timed[MAPI_KC_COUNT]; /* launches timed, per class */
  double ms[MAPI_KC_COUNT];      /* summed device durations of those launches */
  double bytes[MAPI_KC_COUNT];   /* algorithmic bytes they had to read: the
                                    stored matrix once per launch */
  double terms[MAPI_KC_COUNT];   /* algorithmic vector-product terms evaluated */
} mapi_stats;

/* enable != 0: bracket every launch of the classes above with CUDA events
 * recorded on the stream the kernel is launched on (inside CUDA graphs as
 * event nodes); durations are collected when the synchronous call that
 * launched them returns.  Adds a few microseconds per timed launch. */
mapi_status mapi_profile(mapi_ctx* ctx, int enable);

/* Copy the counters to *out (may be NULL) and, if reset != 0, zero them. */
mapi_status mapi_get_stats(mapi_ctx* ctx, mapi_stats* out, int reset);

/* Phase time stamps of the pair step (the PCA pair mode of mapi_pca_topk).
 * Synchronises ctx's stream, then writes to out_us (8 doubles, may be NULL)
 * what was stamped since stamping was last switched on: [0] the steps
 * stamped, then per step, in microseconds of %globaltimer: [1] from the
 * publication of the previous step's iterate to the earliest start of this
 * step's streaming CTAs, [2] from that start to the first streaming CTA's
 * end of its tiles, [3] to the last one's, [4] from that last arrival until
 * the epilogue cluster sees it, [5] the reduction of the accumulated row
 * sums, [6] the deflation, [7] norm, normalisation, stop test and
 * publication.  enable != 0 then clears the stamps and stamps later pair steps;
 * enable == 0 stops.  A few global atomics per CTA and step while on.
 * Not part of the method: it shows where a step's time goes. */
mapi_status mapi_pair_phases(mapi_ctx* ctx, int enable, double* out_us);

/* Each streaming cluster's loop time per pair step (from its CTAs' own
 * start of the step to their arrival, averaged over its CTAs and the steps
 * stamped since mapi_pair_phases last switched stamping on), in
 * microseconds.  Synchronises ctx's stream.  *n <- the streaming clusters of
 * the last pair launch (0 before any stamps); us[0 .. *n) is written when
 * capacity >= *n, else MAPI_EINVAL.  A diagnostic of how evenly the tile
 * loop's work and speed are spread over the clusters. */
mapi_status mapi_pair_cluster_times(mapi_ctx* ctx, double* us, int capacity, int* n);

/* Issue-rate probe of the MAVP term (the ALU roofline of the batched and
 * min-covariance kernels).  One full wave of blocks runs a register-resident
 * loop of independent chains; the slowest block's SM cycles (clock64) give
 * what one SM completes per clock, written to *per_clock_per_sm:
 *   mix 0: FP32 min1 terms, sign(w) clamp(a, -|w|, |w|) accumulated by a
 *          fused multiply-add by +-1 (2 min/max + 1 FMA);
 *   mix 1: FMA instructions;  mix 2: min/max instructions;
 *   mix 3: min1 terms on a BF16 operand widened to FP32 (1 shift + the term);
 *   mix 4: min1 terms on BF16 operands each widened once for four vectors
 *          (the batched kernel's mix with four start vectors).
 * Per thread-lane counts; clock-independent.  Synchronous. */
mapi_status mapi_alu_probe(mapi_ctx* ctx, int mix, double* per_clock_per_sm);

/* Failure-detection test hook.  limit_ns > 0: in every later pair step each
 * CTA also waits, through the same bounded wait as its tile copies and
 * cluster exchanges, on a barrier that nothing ever arrives at, with this
 * limit (at most 2 s).  No copy or store is pending on that barrier, so the
 * wait just runs out; the step then completes as usual and reports the
 * expiry like any other bounded wait, so the solve stops with
 * MAPI_ETIMEOUT and the context stays usable.  0 (the default) turns it
 * off.  MAPI_EINVAL for a negative or larger limit. */
mapi_status mapi_debug_stall(mapi_ctx* ctx, int64_t limit_ns);



/*
 * Batched MAPI: `count` independent instances, each a square packed matrix
 * with nvec start vectors, solved by Alg. 1 in one persistent launch of
 * 8-CTA clusters (replayed from a cached CUDA graph while the batch keeps its
 * shape): instances with n >= 1024 take a whole cluster each (each CTA holds
 * 1/8 of the rows and the whole iterate, norms and deltas combined over the
 * cluster in a fixed order); once those are claimed, every CTA claims the
 * smaller instances alone.  Claims go largest first and run all their steps;
 * the nvec vectors of an instance share every read of its matrix.  Same step,
 * stop rule, flags and statuses as mapi_iterate, per vector.
 *   items     host array of count entries; every A is F32 (or every A is
 *             BF16), square, n <= 8192 / nvec (8192 for one vector, 2048
 *             for four); w0 / w_out are device n x nvec
 *             column-major (ld = n), caller-owned.
 *   nvec      1 or 4.
 *   iters_done, last_delta, statuses: host arrays of count * nvec entries
 *             (item-major; any may be NULL).
 * Errors: MAPI_EINVAL (item pointers, sizes, mixed storage, op), MAPI_ENOMEM,
 * MAPI_ECUDA; otherwise the first non-OK vector status.  Synchronous.
 */
typedef struct {
  const mapi_mat* A;
  const float* w0;
  float* w_out;
} mapi_batch_item;

mapi_status mapi_iterate_batched(mapi_ctx* ctx, const mapi_batch_item* items, int count,
                                 mapi_op op, int nvec, int max_iters, double tol_l1,
                                 unsigned flags, int* iters_done, double* last_delta,
                                 int* statuses);

/*
 * Autotuner of the batched solve: times `iters` steps of the given batch
 * for each candidate rows-per-warp (1, 2, 4, 8) and keeps the fastest for this
 * context, storage and vector count (*chosen receives it; may be NULL).
 * The outputs of the batch are overwritten.
 */
mapi_status mapi_autotune_batched(mapi_ctx* ctx, const mapi_batch_item* items, int count,
                                  mapi_op op, int nvec, int iters, int* chosen);

/*
 * Set the batched solve's rows per warp (1, 2, 4 or 8) for this context,
 * storage (MAPI_ST_F32 or MAPI_ST_BF16) and vector count, as the autotuner
 * would: a way to pin a tuning found earlier, or to run a chosen variant.
 * The results of a solve agree within FP32 rounding whatever the value (the
 * order of the additions differs).  MAPI_EINVAL for other values.
 */
mapi_status mapi_set_batched_rows(mapi_ctx* ctx, mapi_storage storage, int nvec,
                                  int rows_per_warp);

/* ------------------------------------------------------------------ */
/* Serving: PCA and PageRank requests admitted as they arrive.          */
/* ------------------------------------------------------------------ */

typedef enum { MAPI_REQ_PCA = 0, MAPI_REQ_PAGERANK = 1 } mapi_req_kind;

/*
 * One served solve.  Every host pointer stays the caller's and must stay
 * valid until mapi_poll has reported the request finished.
 *   kind       MAPI_REQ_PCA: top-k components of X by the min-covariance
 *              route of Alg. 2 (C = X (+) X^T / cov_denom, Eq. (5); then per
 *              component Alg. 1 on the deflated C_c, as mapi_pca_topk with
 *              MAPI_PCA_MINCOV).  MAPI_REQ_PAGERANK: MAPI-PageRank of §3.3 on
 *              the Google matrix of Eq. (11), as mapi_pagerank.
 *   op         MIN1, MIN2 or DOT.
 *   storage    F32 or BF16: of X (PCA; C itself stays FP32) or of G.
 *   max_iters  steps per component (PCA) or of the solve (PageRank), >= 1.
 *   tol_l1     stop rule on ||w_{t+1} - w_t||_1 (<= 0: none).
 *   X, D, N, k, cov_denom   PCA: X host D x N row-major FP32, columns are
 *              samples; 1 <= k <= min(8, D); D <= 8192; cov_denom > 0.
 *   indptr, indices, n, alpha   PageRank: host out-link CSR as
 *              mapi_google_matrix takes it (n + 1 and indptr[n] int32
 *              entries, 0 <= index < n), n <= 8192, alpha in [0, 1].
 *   w0         host start vectors: D x k column-major (PCA) or n (PageRank),
 *              each scaled to unit l2 norm first (Alg. 1 step 1).
 *   out        host result, written before the request is reported done:
 *              P (D x k column-major, l2-normalised components) or the
 *              l2-normalised rank vector (n).
 *   user       echoed in the result.
 */
typedef struct {
  int kind;
  mapi_op op;
  mapi_storage storage;
  int max_iters;
  double tol_l1;
  const float* X;
  int D, N, k;
  double cov_denom;
  const int* indptr;
  const int* indices;
  int n;
  double alpha;
  const float* w0;
  float* out;
  void* user;
} mapi_request;

/* Outcome of a served request (filled by mapi_poll). */
typedef struct {
  mapi_status status;  /* OK, or why the request stopped (EZERONORM, ...,
                          ECANCELLED, ENOMEM, ECUDA) */
  int iters[8];        /* steps per component (PageRank: iters[0]) */
  double last_delta;   /* last l1 change of the last component */
  double queue_ms;     /* submit -> admission */
  double build_ms;     /* admission -> matrix built on the device (upload,
                          Eq. (5) or Eq. (11), packing) */
  double run_ms;       /* admission -> result in `out` */
  double latency_ms;   /* submit -> result in `out` */
  void* user;
} mapi_result;

/*
 * Queue a request.  A serving loop (a host thread with its own stream and
 * device buffers, started by the first submit on ctx) admits queued requests
 * in arrival order while the device bytes of the resident ones stay within
 * the budget (mapi_config.hbm_budget_bytes; 0: 80 % of the device memory free
 * when the loop starts) and at most max_slots are resident.  It builds each
 * admitted request's matrix on the device (C, or G), keeps every iterate
 * resident, and advances all resident solves together: each round runs up
 * to 25 steps of every solve, those with n < 2048 in one persistent batched
 * launch per (storage, op) (as mapi_iterate_batched), larger ones through
 * the GEMV of mapi_iterate on another stream at the same time; after it,
 * finished components are deflated or results copied out.
 *   ticket   receives the request's handle (> 0).
 * Errors: MAPI_EINVAL (a field out of range, null pointer), MAPI_EBUDGET
 * (the request alone needs more device bytes than the budget: it could never
 * be admitted), MAPI_ECUDA, MAPI_ENOMEM.  Returns at once.
 */
mapi_status mapi_submit(mapi_ctx* ctx, const mapi_request* req, uint64_t* ticket);

/*
 * MAPI_EAGAIN while the request is queued or running.  Once it has finished,
 * fills *out (may be NULL), forgets the ticket and returns the request's
 * status.  MAPI_EINVAL for a ticket that is unknown or already reported.
 */
mapi_status mapi_poll(mapi_ctx* ctx, uint64_t ticket, mapi_result* out);

/*
 * Ask the loop to drop a request: a queued one finishes at once, a running
 * one at the end of the current round; either reports MAPI_ECANCELLED
 * (`out` is then undefined).  A request that has already finished keeps its
 * result.  MAPI_EINVAL for an unknown ticket.
 */
mapi_status mapi_cancel(mapi_ctx* ctx, uint64_t ticket);

/*
 * Allocation-free solve.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory, and it calls no
 * cudaMalloc, cudaFree or any allocating library routine.  Typical callers:
 * a process whose device memory is already owned by another allocator (a
 * framework's caching allocator or a pool reserved at start-up, where a raw
 * cudaMalloc would fail or fragment it), and latency-critical loops that
 * cannot afford the implicit device synchronisation of cudaMalloc/cudaFree.
 *
 * Runs Algorithm 1 like mapi_iterate (one start vector; op MIN1, MIN2,
 * DIAMOND or DOT; same flags, stop rule and statuses) on the calling thread's
 * current device, on `cuda_stream` (NULL: the legacy default stream), and
 * returns after the stream has finished the solve.
 *   A      device, n x n row-major FP32 with leading dimension lda (elements);
 *          lda % 4 == 0 and A 16-byte aligned.  Entries between column n and
 *          lda are never used.  Caller-owned, read only.
 *   w0     device, n FP32 (caller-owned).
 *   w_out  device, n FP32 (caller-owned): the last iterate.
 *   iters_done, last_delta: host scalars (may be NULL).
 * Limit: n <= 8192; a larger n (or a bad pointer, lda or op) returns
 * MAPI_EINVAL before anything runs.  The library cannot see the lengths of
 * w0 and w_out: they must hold n floats (the Python binding checks this).
 * Cost: the call enqueues all max_iters step kernels up front, whatever step
 * the stop rule fires at; the steps after it return at once but are still
 * launched, so a large max_iters with an early stop pays for those launches.
 * Scratch: one static device array of about 320 KiB inside the library,
 * present on every GPU that loads it until the process exits.  The first
 * call on a device looks the array's address up (cudaGetSymbolAddress), so
 * make that first call before any stream capture begins.  Every call
 * reuses the same array and rewrites what it needs, so calls that overlap on
 * the GPU (other threads, other streams) race with each other: serialise
 * them.
 */
mapi_status mapi_iterate_noalloc(const float* A, int n, int64_t lda, mapi_op op,
                                 const float* w0, int max_iters, double tol_l1,
                                 unsigned flags, float* w_out, int* iters_done,
                                 double* last_delta, void* cuda_stream);

#ifdef __cplusplus
} /* extern "C" */
#endif

#endif /* MAPI_H */

/*
 * Plain FP64 CPU oracle for multiplication-avoiding power iteration (MAPI),
 * from H. Pan, D. Badawi, R. Miao, E. Koyuncu, A. E. Cetin,
 * "Multiplication-Avoiding Variant of Power Iteration with Applications"
 * (arXiv 2110.12065).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no code, header, table
 * or helper with the CUDA library; neither side includes or calls the other.
 *
 * Conventions
 *   - every value is an IEEE double; every sum runs sequentially in index
 *     order, exactly as the definitions are written;
 *   - matrices are row-major with an explicit leading dimension;
 *   - the only parallelism is an OpenMP split over independent outputs
 *     (rows, columns), which leaves every individual sum's order unchanged,
 *     so results do not depend on the thread count;
 *   - compiled with -ffp-contract=off: no fused multiply-add may change the
 *     rounding of a*b + c.
 *
 * Readings of points the paper leaves open (sign(0), the start-vector norm,
 * deflation, pair mode, integer storage) are stated at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_EZERONORM 4
#define OR_ENONFINITE 5

enum { OP_MIN1 = 0, OP_MIN2 = 1, OP_DIAMOND = 2, OP_DOT = 3 };

/* flags of or_mapi / or_pca_topk */
#define OR_FINAL_L2 1   /* Alg. 1, optional last step: w_T / ||w_T||_2 */
#define OR_RAW_START 2  /* take w0 as given instead of scaling it to ||w0||_2 = 1 */

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_get_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* sign(x) in {-1, 0, +1} */
static double sgn(double x) { return (double)((x > 0.0) - (x < 0.0)); }

/*
 * One term of a vector product between scalars a and b.
 *   min1   Eq. (3):  sign(a b) min(|a|, |b|)      (sign(ab) = sign(a) sign(b))
 *   min2   Eq. (4):  1(sign a = sign b) min(|a|, |b|)
 *   diamond Eq. (7): sign(a) b + a sign(b)        (the printed formula mixes
 *                    the letters w, x, y; the proof of Proposition 1 fixes
 *                    this symmetric reading)
 *   dot    Eq. (1):  a b                          (regular power iteration)
 */
double or_term(int op, double a, double b) {
  switch (op) {
    case OP_MIN1: return sgn(a) * sgn(b) * fmin(fabs(a), fabs(b));
    case OP_MIN2: return (sgn(a) == sgn(b)) ? fmin(fabs(a), fabs(b)) : 0.0;
    case OP_DIAMOND: return sgn(a) * b + a * sgn(b);
    case OP_DOT: return a * b;
    default: return NAN;
  }
}

/* w^T (+) x = sum_i term(w_i, x_i), Eq. (3) / (4) / (7) / dot. */
double or_vecprod(int op, const double* w, const double* x, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += or_term(op, w[i], x[i]);
  return s;
}

/*
 * Matrix-vector product y = A (+) w, row by row: y_i = a_i^T (+) w with a_i
 * the i-th row of A (§2.2, "A = [a_1^T ... a_n^T]" before Proposition 1;
 * Alg. 1 step 3).
 */
void or_matvec(int op, const double* A, long rows, long cols, long ld,
               const double* w, double* y) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < rows; ++i) y[i] = or_vecprod(op, A + i * ld, w, cols);
}

double or_norm1(const double* v, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += fabs(v[i]);
  return s;
}

double or_norm2(const double* v, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += v[i] * v[i];
  return sqrt(s);
}

static int all_finite(const double* v, long n) {
  for (long i = 0; i < n; ++i)
    if (!isfinite(v[i])) return 0;
  return 1;
}

/*
 * Algorithm 1 (MAPI) and, with op = dot, regular power iteration Eq. (1).
 *   step 1: w_0 = w0 / ||w0||_2 (the unmarked norm of Alg. 1 is read as the
 *           Euclidean norm, as in Eq. (1)); skipped with OR_RAW_START;
 *   step 3: y = A (+) w_t;
 *   step 4: w_{t+1} = y / ||y||_1 (Eq. (6)); for op = dot the Euclidean norm
 *           of Eq. (1) is used instead;
 *   the loop stops after max_iters products, or as soon as
 *   delta_t = ||w_t - w_{t-1}||_1 < tol (tol <= 0 disables the test);
 *   step 6 (optional, OR_FINAL_L2): w_T / ||w_T||_2.
 * A zero norm returns OR_EZERONORM and leaves w_out at the last iterate.
 */
int or_mapi(int op, const double* A, long n, long ld, const double* w0,
            int flags, int max_iters, double tol, double* w_out,
            int* iters_done, double* last_delta) {
  if (n <= 0 || ld < n || max_iters < 0) return OR_EINVAL;
  double* w = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * n);
  int status = OR_OK, t = 0;
  double delta = NAN;
  memcpy(w, w0, sizeof(double) * n);
  if (!(flags & OR_RAW_START)) {
    double s = or_norm2(w, n);
    if (s == 0.0) { status = OR_EZERONORM; goto done; }
    for (long i = 0; i < n; ++i) w[i] = w[i] / s;
  }
  for (t = 0; t < max_iters;) {
    or_matvec(op, A, n, n, ld, w, y);
    double s = (op == OP_DOT) ? or_norm2(y, n) : or_norm1(y, n);
    if (!isfinite(s)) { status = OR_ENONFINITE; break; }
    if (s == 0.0) { status = OR_EZERONORM; break; }
    delta = 0.0;
    for (long i = 0; i < n; ++i) {
      double v = y[i] / s;
      delta += fabs(v - w[i]);
      w[i] = v;
    }
    ++t;
    if (tol > 0.0 && delta < tol) break;
  }
  if (status == OR_OK && (flags & OR_FINAL_L2)) {
    double s = or_norm2(w, n);
    if (s == 0.0) status = OR_EZERONORM;
    else for (long i = 0; i < n; ++i) w[i] = w[i] / s;
  }
done:
  memcpy(w_out, w, sizeof(double) * n);
  if (iters_done) *iters_done = t;
  if (last_delta) *last_delta = delta;
  free(w);
  free(y);
  return status;
}

/*
 * Min-covariance matrix, Eq. (5): C = (1/denom) X (+) X^T for X in R^{D x N}
 * (columns are samples), i.e. C_pq = (sum_n term(X_pn, X_qn)) / denom.
 * Eq. (5) uses denom = N, Alg. 2 step 4 uses N - 1; the caller chooses.  With
 * op = dot this is the ordinary sample covariance of Eq. (2).  The full D x D
 * matrix is computed; its symmetry is checked, not assumed.
 */
void or_mincov(int op, const double* X, long D, long N, long ldx,
               double denom, double* C) {
#pragma omp parallel for schedule(dynamic, 1)
  for (long p = 0; p < D; ++p)
    for (long q = 0; q < D; ++q)
      C[p * D + q] = or_vecprod(op, X + p * ldx, X + q * ldx, N) / denom;
}

/* P = w (+) w^T: the D x D matrix with P_ij = term(w_i, w_j) (Alg. 2 steps 6
 * and 8, where the outer product of vectors uses the same operator). */
void or_mavp_outer(int op, const double* w, long D, double* P) {
  for (long i = 0; i < D; ++i)
    for (long j = 0; j < D; ++j) P[i * D + j] = or_term(op, w[i], w[j]);
}

/*
 * The vector an outer product w (+) w^T of Alg. 2 (steps 6 and 8) is formed
 * from.  The components are kept at unit l2 norm (§2.2); the outer product
 * takes each at the unit norm of its own iteration: the l1 norm for the
 * MAVP operators (the normalisation of Eq. (8)), the l2 norm for the
 * ordinary product (w w^T, the projector of §1).  A vector of equal
 * magnitudes at unit l1 norm gives exactly the projector u u^T, u = w/||w||_2,
 * under min1; at unit l2 norm it would give sqrt(D) u u^T.
 */
static void outer_vector(int op, const double* w, long D, double* out) {
  double s = (op == OP_DOT) ? 1.0 : or_norm1(w, D);
  for (long i = 0; i < D; ++i) out[i] = (s > 0.0) ? w[i] / s : w[i];
}

/* Q = sum_{m<k} wt_m (+) wt_m^T with wt_m = outer_vector(w_m). */
static double* outer_sum(int op, long D, const double* W, long k, long ldw) {
  double* Q = (double*)calloc((size_t)D * D, sizeof(double));
  double* wt = (double*)malloc(sizeof(double) * (D > 0 ? D : 1));
  for (long m = 0; m < k; ++m) {
    outer_vector(op, W + m * ldw, D, wt);
    for (long i = 0; i < D; ++i)
      for (long j = 0; j < D; ++j) Q[i * D + j] += or_term(op, wt[i], wt[j]);
  }
  free(wt);
  return Q;
}

/*
 * Deflation of a covariance for the k-th component (Alg. 2 step 6 generalised
 * with the sum form that follows Eq. (2)):
 *     C_k = (I - sum_{m<k} P_m) C,   P_m = wt_m (+) wt_m^T,
 * where wt_m is the earlier component w_m (kept at unit l2 norm, §2.2) taken
 * at the unit norm of its iteration (outer_vector: l1 for the MAVP
 * operators, l2 for dot) and the juxtaposition P_m C is the ordinary matrix
 * product.  With op = dot this is the projection deflation
 * (I - sum p_m p_m^T) C of §1.
 * W holds the k earlier components as columns: W[i + m*ldw].
 */
void or_deflate(int op, const double* C, long D, const double* W, long k,
                long ldw, double* Ck) {
  double* Q = outer_sum(op, D, W, k, ldw);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < D; ++i)
    for (long j = 0; j < D; ++j) {
      double s = 0.0;  /* (Q C)_ij */
      for (long l = 0; l < D; ++l) s += Q[i * D + l] * C[l * D + j];
      Ck[i * D + j] = C[i * D + j] - s;
    }
  free(Q);
}

/* y <- y - sum_{m<k} P_m y, the same deflation applied to an iterate. */
void or_deflate_vec(int op, double* y, long D, const double* W, long k,
                    long ldw) {
  if (k <= 0) return;
  double* Q = outer_sum(op, D, W, k, ldw);
  double* z = (double*)malloc(sizeof(double) * D);
  for (long i = 0; i < D; ++i) {
    double s = 0.0;
    for (long j = 0; j < D; ++j) s += Q[i * D + j] * y[j];
    z[i] = y[i] - s;
  }
  memcpy(y, z, sizeof(double) * D);
  free(z);
  free(Q);
}

/*
 * Image reconstruction, Alg. 2 step 8: out_i = (W (+) W^T)(v_i - m) + m for
 * the N columns v_i of V (D x N, leading dimension ldv).  W holds the k
 * components as columns (W[p + c*ldw]), each taken at the unit norm of its
 * iteration (outer_vector) as in step 6; R = W (+) W^T is the D x D matrix
 * of the operator's matrix extension, rows of W against the columns of W^T:
 * R_pq = sum_c term(Wt_pc, Wt_qc).  Its product with v_i - m is the ordinary
 * one, as in the deflation of step 6.  Row p of R is formed when needed, so D
 * may be large; out is D x N with leading dimension ldo.
 */
void or_reconstruct(int op, const double* W, long D, long k, long ldw,
                    const double* V, long N, long ldv, const double* m,
                    double* out, long ldo) {
  double* Z = (double*)malloc(sizeof(double) * D * N);  /* v_i - m, row-major */
  for (long q = 0; q < D; ++q)
    for (long i = 0; i < N; ++i) Z[q * N + i] = V[q * ldv + i] - m[q];
  double* Wt = (double*)malloc(sizeof(double) * (D * k > 0 ? D * k : 1));
  for (long c = 0; c < k; ++c) outer_vector(op, W + c * ldw, D, Wt + c * D);
#pragma omp parallel for schedule(dynamic, 16)
  for (long p = 0; p < D; ++p) {
    double* acc = (double*)calloc((size_t)N, sizeof(double));
    for (long q = 0; q < D; ++q) {
      double r = 0.0;
      for (long c = 0; c < k; ++c) r += or_term(op, Wt[p + c * D], Wt[q + c * D]);
      for (long i = 0; i < N; ++i) acc[i] += r * Z[q * N + i];
    }
    for (long i = 0; i < N; ++i) out[p * ldo + i] = acc[i] + m[p];
    free(acc);
  }
  free(Wt);
  free(Z);
}

/*
 * Matrix-free "pair" step for PCA, the MAVP analogue of C w = X (X^T w) / N.
 * The paper has no such step; it is defined here as
 *     t_n = x_n^T (+) w            (x_n = column n of X),
 *     y_d = (sum_n term(X_dn, t_n)) / denom.
 * It is not equal to C (+) w for the min-covariance C of Eq. (5).
 */
void or_pair_step(int op, const double* X, long D, long N, long ldx,
                  const double* w, double denom, double* y) {
  double* t = (double*)calloc((size_t)N, sizeof(double));
  /* t_n accumulates over d in increasing order; the loop over n is split
   * into column blocks only so that rows of X are read contiguously. */
  const long B = 512;
#pragma omp parallel for schedule(static)
  for (long n0 = 0; n0 < N; n0 += B) {
    long n1 = n0 + B < N ? n0 + B : N;
    for (long d = 0; d < D; ++d)
      for (long n = n0; n < n1; ++n) t[n] += or_term(op, X[d * ldx + n], w[d]);
  }
#pragma omp parallel for schedule(static)
  for (long d = 0; d < D; ++d) {
    double s = 0.0;
    for (long n = 0; n < N; ++n) s += or_term(op, X[d * ldx + n], t[n]);
    y[d] = s / denom;
  }
  free(t);
}

/*
 * Top-k principal vectors by MAPI (Alg. 2 steps 4-7 generalised to k
 * components; op = dot gives the RPI-PCA of §1).
 *   mode 0 (min-covariance): C = (1/denom) X (+) X^T once; component k runs
 *     Alg. 1 on C_k = (I - sum_{m<k} P_m) C with OR_FINAL_L2.
 *   mode 1 (pair): component k runs the pair step on X directly, deflates the
 *     iterate, y <- y - sum_{m<k} P_m y, then normalises (l1; l2 for dot),
 *     and ends with the l2 normalisation.
 * W0 (D x k, column-major, ldw0) holds raw start vectors, each scaled to unit
 * l2 norm first (Alg. 1 step 1).  P (D x k, column-major, ldp) receives the
 * l2-normalised components; iters_done[k] the products run per component.
 */
int or_pca_topk(int mode, int op, const double* X, long D, long N, long ldx,
                long k, int iters, double tol, double denom, const double* W0,
                long ldw0, double* P, long ldp, int* iters_done) {
  if (D <= 0 || N <= 0 || k <= 0 || k > D || iters < 0) return OR_EINVAL;
  int status = OR_OK;
  if (mode == 0) {
    double* C = (double*)malloc(sizeof(double) * D * D);
    double* Ck = (double*)malloc(sizeof(double) * D * D);
    or_mincov(op, X, D, N, ldx, denom, C);
    for (long c = 0; c < k && status == OR_OK; ++c) {
      or_deflate(op, C, D, P, c, ldp, Ck);
      double dl;
      status = or_mapi(op, Ck, D, D, W0 + c * ldw0, OR_FINAL_L2, iters, tol,
                       P + c * ldp, &iters_done[c], &dl);
    }
    free(C);
    free(Ck);
    return status;
  }
  if (mode != 1) return OR_EINVAL;
  double* w = (double*)malloc(sizeof(double) * D);
  double* y = (double*)malloc(sizeof(double) * D);
  for (long c = 0; c < k && status == OR_OK; ++c) {
    memcpy(w, W0 + c * ldw0, sizeof(double) * D);
    double s = or_norm2(w, D);
    if (s == 0.0) { status = OR_EZERONORM; break; }
    for (long i = 0; i < D; ++i) w[i] = w[i] / s;
    int t = 0;
    for (t = 0; t < iters;) {
      or_pair_step(op, X, D, N, ldx, w, denom, y);
      or_deflate_vec(op, y, D, P, c, ldp);
      double nrm = (op == OP_DOT) ? or_norm2(y, D) : or_norm1(y, D);
      if (!isfinite(nrm)) { status = OR_ENONFINITE; break; }
      if (nrm == 0.0) { status = OR_EZERONORM; break; }
      double delta = 0.0;
      for (long i = 0; i < D; ++i) {
        double v = y[i] / nrm;
        delta += fabs(v - w[i]);
        w[i] = v;
      }
      ++t;
      if (tol > 0.0 && delta < tol) break;
    }
    iters_done[c] = t;
    if (status != OR_OK) break;
    s = or_norm2(w, D);
    if (s == 0.0) { status = OR_EZERONORM; break; }
    for (long i = 0; i < D; ++i) P[i + c * ldp] = w[i] / s;
  }
  free(w);
  free(y);
  return status;
}

/*
 * Google matrix of §3.3, Eq. (11): G = alpha H + (1 - alpha)/n * 1 (all ones).
 * H is column-stochastic: column j spreads node j's weight over its
 * out-links, H_ij = (#links j -> i) / outdeg(j).  A node without out-links
 * (dangling) gets the uniform column H_ij = 1/n.  The graph arrives as
 * out-link CSR: the targets of j are indices[indptr[j] .. indptr[j+1]).
 * G is written row-major (n x n); row i then holds the in-links of i, so
 * MAPI's row-wise product G (+) w follows the orientation of Eq. (1).
 */
void or_google_matrix(long n, const int* indptr, const int* indices,
                      double alpha, double* G) {
  double tele = (1.0 - alpha) / (double)n;
  for (long i = 0; i < n * n; ++i) G[i] = 0.0;
  for (long j = 0; j < n; ++j) {
    long d = indptr[j + 1] - indptr[j];
    if (d == 0) {
      for (long i = 0; i < n; ++i) G[i * n + j] = 1.0 / (double)n;
    } else {
      for (long e = indptr[j]; e < indptr[j + 1]; ++e)
        G[(long)indices[e] * n + j] += 1.0 / (double)d;
    }
  }
  for (long i = 0; i < n * n; ++i) G[i] = alpha * G[i] + tele;
}

/*
 * MAPI-PageRank on the Google matrix of Eq. (11) without forming it (§3.3).
 * Every entry of column j is one of a few values: the teleport value
 * tele = alpha * 0 + (1 - alpha)/n where j has no link to i, alpha * acc + tele
 * where j links to i (acc = 1/d_j added once per link, as or_google_matrix
 * adds it), and alpha * (1/n) + tele in a dangling column.  So row i of
 * G (+) w is the same base sum S = sum_j term(b_j, w_j) for every row (b_j:
 * the teleport value, or the dangling value), plus, over the in-links of i,
 * term(g_ij, w_j) - term(tele, w_j).  Exact algebra, not an approximation: the
 * dense oracle (or_google_matrix, or_mapi) pins it.  With round32 != 0 every
 * entry value is first rounded to FP32, the values an FP32 copy of G holds.
 * Steps, stop rule and final l2 step as or_mapi with OR_FINAL_L2.
 */
static double pr_value(double v, int round32) { return round32 ? (double)(float)v : v; }

static int cmp_int(const void* a, const void* b) {
  const int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

int or_pagerank_sparse(int op, long n, const int* indptr, const int* indices,
                       double alpha, int round32, const double* w0, int max_iters,
                       double tol, double* w_out, int* iters_done, double* last_delta) {
  if (n <= 0 || max_iters < 0) return OR_EINVAL;
  const double tele = (1.0 - alpha) / (double)n;
  const double g0 = pr_value(alpha * 0.0 + tele, round32);
  const double gd = pr_value(alpha * (1.0 / (double)n) + tele, round32);
  /* per column: its distinct targets and their entry values */
  long nnz = indptr[n];
  int* tgt = (int*)malloc(sizeof(int) * (nnz > 0 ? nnz : 1));
  double* val = (double*)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
  long* cnt = (long*)malloc(sizeof(long) * (n + 1));
  double* w = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * n);
  long k = 0;
  for (long j = 0; j < n; ++j) {
    long b = indptr[j], e = indptr[j + 1], d = e - b;
    int* t = (int*)malloc(sizeof(int) * (d > 0 ? d : 1));
    for (long q = 0; q < d; ++q) t[q] = indices[b + q];
    qsort(t, (size_t)d, sizeof(int), cmp_int);
    cnt[j] = k;
    for (long q = 0; q < d;) {
      long r = q;
      double acc = 0.0;
      while (r < d && t[r] == t[q]) { acc += 1.0 / (double)d; ++r; }
      tgt[k] = t[q];
      val[k] = pr_value(alpha * acc + tele, round32);
      ++k;
      q = r;
    }
    free(t);
  }
  cnt[n] = k;
  int status = OR_OK, t = 0;
  double delta = NAN;
  for (long i = 0; i < n; ++i) w[i] = w0[i];
  {
    double s = or_norm2(w, n);
    if (s == 0.0) status = OR_EZERONORM;
    else for (long i = 0; i < n; ++i) w[i] = w[i] / s;
  }
  while (status == OR_OK && t < max_iters) {
    double S = 0.0;
    for (long j = 0; j < n; ++j)
      S += or_term(op, (indptr[j + 1] == indptr[j]) ? gd : g0, w[j]);
    for (long i = 0; i < n; ++i) y[i] = S;
    for (long j = 0; j < n; ++j) {
      if (indptr[j + 1] == indptr[j]) continue;
      for (long q = cnt[j]; q < cnt[j + 1]; ++q)
        y[tgt[q]] += or_term(op, val[q], w[j]) - or_term(op, g0, w[j]);
    }
    double s = (op == OP_DOT) ? or_norm2(y, n) : or_norm1(y, n);
    if (!isfinite(s)) { status = OR_ENONFINITE; break; }
    if (s == 0.0) { status = OR_EZERONORM; break; }
    delta = 0.0;
    for (long i = 0; i < n; ++i) {
      double v = y[i] / s;
      delta += fabs(v - w[i]);
      w[i] = v;
    }
    ++t;
    if (tol > 0.0 && delta < tol) break;
  }
  if (status == OR_OK) {
    double s = or_norm2(w, n);
    if (s == 0.0) status = OR_EZERONORM;
    else for (long i = 0; i < n; ++i) w[i] = w[i] / s;
  }
  for (long i = 0; i < n; ++i) w_out[i] = w[i];
  if (iters_done) *iters_done = t;
  if (last_delta) *last_delta = delta;
  free(tgt); free(val); free(cnt); free(w); free(y);
  return status;
}

/*
 * Mini-batch MAPI with momentum (Alg. 3), on data X (N x D, row-major: one
 * sample per row).  The mini-batches are given: batch[t * s + i] is the i-th
 * sample of step t (Alg. 3 step 3 draws them; the caller passes the draws).
 *   step 1: w_0 = w0 / ||w0||_2 (reading of the unnamed norm, as in Alg. 1),
 *           w_{-1} = 0;
 *   step 4: A_t = (1/s) sum_i x_{t_i} (+) x_{t_i}^T (entries term(x_p, x_q),
 *           summed over the batch in order, then divided by s);
 *           v = A_t (+) w_t - beta w_{t-1}  (rows of A_t against w_t);
 *   step 5: w_{t+1} = v / ||v||_1, w_t = w_t / ||v||_1 (the l2 norm for
 *           op = dot: the momentum power method of the comparison);
 *   step 7 (OR_FINAL_L2): w_T / ||w_T||_2.
 */
int or_minibatch_momentum(int op, const double* X, long N, long D, const int* batch, int T,
                          int s, double beta, const double* w0, int flags, double* w_out) {
  if (N <= 0 || D <= 0 || T < 0 || s <= 0) return OR_EINVAL;
  double* w = (double*)malloc(sizeof(double) * D);
  double* wp = (double*)malloc(sizeof(double) * D);
  double* v = (double*)malloc(sizeof(double) * D);
  double* A = (double*)malloc(sizeof(double) * D * D);
  int status = OR_OK;
  for (long p = 0; p < D; ++p) { w[p] = w0[p]; wp[p] = 0.0; }
  {
    double n2 = or_norm2(w, D);
    if (n2 == 0.0) status = OR_EZERONORM;
    else for (long p = 0; p < D; ++p) w[p] = w[p] / n2;
  }
  for (int t = 0; t < T && status == OR_OK; ++t) {
    for (long p = 0; p < D; ++p)
      for (long q = 0; q < D; ++q) {
        double a = 0.0;
        for (int i = 0; i < s; ++i) {
          long k = batch[(long)t * s + i];
          if (k < 0 || k >= N) { status = OR_EINVAL; break; }
          a += or_term(op, X[k * D + p], X[k * D + q]);
        }
        A[p * D + q] = a / (double)s;
      }
    if (status != OR_OK) break;
    for (long p = 0; p < D; ++p) v[p] = or_vecprod(op, A + p * D, w, D) - beta * wp[p];
    double L = (op == OP_DOT) ? or_norm2(v, D) : or_norm1(v, D);
    if (!isfinite(L)) { status = OR_ENONFINITE; break; }
    if (L == 0.0) { status = OR_EZERONORM; break; }
    for (long p = 0; p < D; ++p) {
      wp[p] = w[p] / L;
      w[p] = v[p] / L;
    }
  }
  if (status == OR_OK && (flags & OR_FINAL_L2)) {
    double n2 = or_norm2(w, D);
    if (n2 == 0.0) status = OR_EZERONORM;
    else for (long p = 0; p < D; ++p) w[p] = w[p] / n2;
  }
  for (long p = 0; p < D; ++p) w_out[p] = w[p];
  free(w); free(wp); free(v); free(A);
  return status;
}

/* ---------------------------------------------------------------------- */
/* Storage formats.  The paper fixes no storage; these follow the format    */
/* definitions (IEEE-754 round-to-nearest-even) so that the oracle can run  */
/* on exactly the values a reduced-precision copy holds.                     */
/* ---------------------------------------------------------------------- */

/* Round a finite value to the nearest number with `bits` significant bits
 * (ties to even), never below the spacing 2^min_exp_spacing (subnormals). */
static double round_sig(double x, int bits, int min_spacing_exp) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  frexp(x, &e);                 /* x = m 2^e, 0.5 <= |m| < 1 */
  int sp = e - bits;            /* spacing of `bits`-bit significands at this binade */
  if (sp < min_spacing_exp) sp = min_spacing_exp;
  double r = nearbyint(ldexp(x, -sp));   /* exact scaling, RNE rounding */
  return ldexp(r, sp);
}

/* bfloat16: 8 significant bits, fp32 exponent range (subnormal spacing 2^-133). */
double or_round_bf16(double x) { return round_sig(x, 8, -133); }

/* FP8 E4M3 (OCP "fn" variant): 4 significant bits, exponent bias 7, largest
 * finite 448, smallest normal 2^-6, subnormal spacing 2^-9.  Values beyond
 * the largest finite saturate to +-448. */
double or_round_e4m3(double x) {
  double r = round_sig(x, 4, -9);
  if (r > 448.0) r = 448.0;
  if (r < -448.0) r = -448.0;
  return r;
}

/* Smallest integer k with max_j |row_j| <= 448 * 2^k (0 for an all-zero row):
 * the power-of-two row scale of the FP8 storage. */
int or_fp8_row_exponent(const float* row, long cols) {
  double mx = 0.0;
  for (long j = 0; j < cols; ++j) mx = fmax(mx, fabs((double)row[j]));
  if (mx == 0.0) return 0;
  int k = -160;
  while (mx > ldexp(448.0, k)) ++k;
  return k;
}

/* Quantise rows of A (fp32) to E4M3 with per-row scale 2^k_i and write the
 * dequantised values (exact doubles) and the exponents. */
void or_quant_fp8_rows(const float* A, long rows, long cols, long lda,
                       double* out, long ldo, int* row_exp) {
  for (long i = 0; i < rows; ++i) {
    int k = or_fp8_row_exponent(A + i * lda, cols);
    row_exp[i] = k;
    for (long j = 0; j < cols; ++j)
      out[i * ldo + j] = ldexp(or_round_e4m3(ldexp((double)A[i * lda + j], -k)), k);
  }
}

void or_quant_bf16(const float* A, long rows, long cols, long lda, double* out,
                   long ldo) {
  for (long i = 0; i < rows; ++i)
    for (long j = 0; j < cols; ++j)
      out[i * ldo + j] = or_round_bf16((double)A[i * lda + j]);
}

/* Shared fixed-point exponent q of the integer storage: the largest q in
 * [0, 24] with max|A| * 2^q <= qmax (qmax = 32767 for int16, 127 for int8).
 * Returns OR_EINVAL if even q = 0 does not fit. */
int or_int_scale(const float* A, long rows, long cols, long lda, int qmax,
                 int* q_out) {
  double mx = 0.0;
  for (long i = 0; i < rows; ++i)
    for (long j = 0; j < cols; ++j) mx = fmax(mx, fabs((double)A[i * lda + j]));
  int q = 24;
  while (q >= 0 && mx * ldexp(1.0, q) > (double)qmax) --q;
  if (q < 0) return OR_EINVAL;
  *q_out = q;
  return OR_OK;
}

/* A_q = RNE(A * 2^q) as exact integers. */
void or_quant_int(const float* A, long rows, long cols, long lda, int q,
                  long long* out, long ldo) {
  for (long i = 0; i < rows; ++i)
    for (long j = 0; j < cols; ++j)
      out[i * ldo + j] = (long long)nearbyint(ldexp((double)A[i * lda + j], q));
}

/* integer term of min1 / min2 */
static long long iterm(int op, long long a, long long b) {
  long long sa = (a > 0) - (a < 0), sb = (b > 0) - (b < 0);
  long long m = llabs(a) < llabs(b) ? llabs(a) : llabs(b);
  if (op == OP_MIN1) return sa * sb * m;
  return (sa == sb) ? m : 0;
}

/* Integer l1 normalisation to units of 2^-q: w_i = sign(y_i) *
 * floor((|y_i| 2^q + floor(L/2)) / L) with L = sum |y_i| (n divisions). */
static void inormalise(const long long* y, long n, long long L, int q,
                       long long* w) {
  for (long i = 0; i < n; ++i) {
    long long a = llabs(y[i]);
    long long v = ((a << q) + L / 2) / L;
    w[i] = (y[i] < 0) ? -v : v;
  }
}

/*
 * Alg. 1 on integer storage, exactly: A_q (units 2^-q), start vector
 * x_i = RNE(w0_i 2^q) normalised in the same integer way (Euclidean
 * normalisation has no exact integer form, so the integer path starts from
 * the l1-normalised vector), then per step y = A_q (+) w in exact integers,
 * w <- integer l1 normalisation of y, delta = sum |w_new - w_old| (units
 * 2^-q); stop after max_iters or when delta * 2^-q < tol.  Only min1 and
 * min2 are defined here (their terms stay within |a|).
 */
int or_mapi_int(int op, const long long* Aq, long n, long ld, int q,
                const float* w0, int max_iters, double tol, long long* w_out,
                int* iters_done, long long* last_delta) {
  if ((op != OP_MIN1 && op != OP_MIN2) || n <= 0 || q < 0 || q > 30)
    return OR_EINVAL;
  long long* w = (long long*)malloc(sizeof(long long) * n);
  long long* y = (long long*)malloc(sizeof(long long) * n);
  long long* wn = (long long*)malloc(sizeof(long long) * n);
  int status = OR_OK, t = 0;
  long long delta = -1, L = 0;
  for (long i = 0; i < n; ++i) y[i] = (long long)nearbyint(ldexp((double)w0[i], q));
  for (long i = 0; i < n; ++i) L += llabs(y[i]);
  if (L == 0) { status = OR_EZERONORM; memcpy(w, y, sizeof(long long) * n); goto done; }
  inormalise(y, n, L, q, w);
  for (t = 0; t < max_iters;) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
      long long s = 0;
      for (long j = 0; j < n; ++j) s += iterm(op, Aq[i * ld + j], w[j]);
      y[i] = s;
    }
    L = 0;
    for (long i = 0; i < n; ++i) L += llabs(y[i]);
    if (L == 0) { status = OR_EZERONORM; break; }
    inormalise(y, n, L, q, wn);
    delta = 0;
    for (long i = 0; i < n; ++i) delta += llabs(wn[i] - w[i]);
    memcpy(w, wn, sizeof(long long) * n);
    ++t;
    if (tol > 0.0 && (double)delta < tol * ldexp(1.0, q)) break;
  }
done:
  memcpy(w_out, w, sizeof(long long) * n);
  if (iters_done) *iters_done = t;
  if (last_delta) *last_delta = delta;
  free(w);
  free(y);
  free(wn);
  return status;
}

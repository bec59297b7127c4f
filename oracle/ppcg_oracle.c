/*
 * Oracle for pipelined PCG -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential FP64 restatement of the two algorithms of Tiwari & Vadhiyar,
 * "Efficient executions of Pipelined Conjugate Gradient Method on Heterogeneous
 * Architectures" (arXiv 2105.06176), Sec. III:
 *   - Algorithm 1: preconditioned CG (Hestenes-Stiefel form), used as a cross-check;
 *   - Algorithm 2: pipelined PCG (Ghysels-Vanroose form), the method the GPU path runs.
 * The preconditioner is Jacobi, M = diag(A) (Sec. V-A); the matrix is CSR (Sec. V-A).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark load this
 * file.  It shares no code, header or constant with the CUDA library.  Build with
 * -O2 -ffp-contract=off so every product and sum is rounded separately, in the order
 * written here.
 *
 * Loops whose rows are independent (SpMV rows, Jacobi application, vector updates) carry
 * OpenMP pragmas.  A plain build ignores them; a build with -fopenmp spreads those rows over
 * the host cores with each row's arithmetic unchanged, and the dot products stay sequential
 * in index order, so both builds return bitwise-identical results.  The OpenMP build exists
 * only to time the same source on all host cores.
 *
 * Readings where the paper is silent or loose (each is repeated in the design notes):
 *   - alpha_{i-1} in the alpha update of Algorithm 2 is the previous iteration's alpha;
 *     the un-subscripted delta is the value of the latest (w, u) dot product.
 *   - Default stop test: ||r_i||_2 <= tol * ||b||_2 on the recursively updated r, checked
 *     at the top of each iteration with "<=".  The paper's own test (Sec. VI) is the
 *     absolute preconditioned norm sqrt((u, u)) <= tol, kept as norm_mode 1.
 *   - In norm_mode 0, when the recursive residual passes, the true residual b - A x is
 *     formed; if it fails, the recurrence vectors are replaced by their true values
 *     (residual replacement, not in the paper) and the iteration continues.
 *   - rr_period > 0 additionally replaces residuals every rr_period iterations.
 *   - gap_theta > 0 (not in the paper; the accuracy criterion of the residual-replacement
 *     literature for pipelined CG: van der Vorst & Ye 2000, Cools et al., SIMAX 2018):
 *     whenever gamma has fallen by the factor gap_fall since the residuals were last
 *     measured or replaced, the deviation of the recursive residual from the true one,
 *     ||(b - A x) - r||, is measured, and the residuals are replaced when it exceeds
 *     gap_theta * ||r||.  Replacing while that deviation is still small keeps the alpha
 *     and beta recurrences consistent with the vectors; a replacement made only once the
 *     recursive residual has passed the stopping test can change r by a percent or more
 *     and derail the iteration (it can then grow until the alpha denominator breaks down).
 *   - jacobi_elim (a variant, not the paper's literal algorithm): with a diagonal M the
 *     recurrences of q and u in the update block reproduce q = M^-1 s and u = M^-1 r in exact
 *     arithmetic, so the variant computes q and u from s and r after their updates instead.
 *   - Restart on breakdown (not in the paper): when the alpha denominator is not positive
 *     after the first iteration -- which pipelined PCG meets near its attainable accuracy --
 *     and fewer than max_restarts restarts were made, the residuals are replaced by their
 *     true values, the direction recurrences p, s, q, z are reset to zero, and the next
 *     step takes beta = 0, alpha = gamma / delta as at i = 0.  max_restarts = 0 reports the
 *     breakdown instead.
 *   - b == 0 returns x = 0 with 0 iterations; a non-positive diagonal is "not SPD";
 *     gamma <= 0 or a non-positive alpha denominator is a breakdown.
 *   - The iteration count is the number of times the vector-update block runs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NOT_SPD (-2)
#define OR_ERR_BREAKDOWN (-3)
#define OR_ERR_NOT_CONVERGED (-4)
#define OR_ERR_NONFINITE (-5)

typedef struct {
  int32_t status;
  int32_t iters;
  int32_t rr_count;
  int32_t pad;
  double bnorm;
  double res_recursive;   /* ||r|| (norm_mode 0) or sqrt((u,u)) (norm_mode 1) at exit */
  double res_true;        /* ||b - A x|| at exit */
  double gamma, delta;
} oracle_result;

/* Host threads the row loops use: 1 for the plain build. */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---- building blocks ---------------------------------------------------------------- */

/* y = A x, one row at a time, terms added in CSR order. */
void oracle_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                 const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    double acc = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; k++) acc += v[k] * x[ci[k]];
    y[i] = acc;
  }
}

static double dot_seq(int64_t n, const double* a, const double* b) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; i++) acc += a[i] * b[i];
  return acc;
}

static double dot_pairwise(int64_t n, const double* a, const double* b) {
  if (n <= 8) return dot_seq(n, a, b);
  int64_t h = n / 2;
  return dot_pairwise(h, a, b) + dot_pairwise(n - h, a + h, b + h);
}

/* sum_mode 0: left-to-right in index order; 1: pairwise (for rounding-sensitivity checks). */
static double dot(int sum_mode, int64_t n, const double* a, const double* b) {
  return sum_mode ? dot_pairwise(n, a, b) : dot_seq(n, a, b);
}

/* Jacobi: d[i] = a_ii.  Returns 0, or OR_ERR_NOT_SPD if a diagonal entry is missing or <= 0. */
static int jacobi_diag(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double* d) {
  for (int64_t i = 0; i < n; i++) {
    double di = 0.0;
    int found = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; k++)
      if (ci[k] == i) { di += v[k]; found = 1; }
    if (!found || !(di > 0.0)) return OR_ERR_NOT_SPD;
    d[i] = di;
  }
  return OR_OK;
}

/* y = M^-1 x with M = diag(A): y_i = x_i / a_ii. */
static void apply_jacobi(int64_t n, const double* d, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) y[i] = x[i] / d[i];
}

static double true_residual(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                            const double* b, const double* x, double* tmp, int sum_mode) {
  oracle_spmv(n, rp, ci, v, x, tmp);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) tmp[i] = b[i] - tmp[i];
  return sqrt(dot(sum_mode, n, tmp, tmp));
}

/* ---- Algorithm 2: pipelined PCG -------------------------------------------------------- */

/*
 * x0 may be NULL (zero initial guess).  x receives the final iterate.
 * alpha_hist/beta_hist (length maxit) and res_hist (length maxit + 1) may be NULL.
 * state_out may be NULL or hold 10*n doubles: x r u w p q s z m n at exit (p q s z are
 * those of the last executed update block; zero if none ran).
 * Returns the status (also stored in res->status).
 */
int oracle_pipecg(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                  const double* b, const double* x0, double* x, double tol, int32_t maxit,
                  int32_t norm_mode, int32_t rr_period, int32_t max_restarts, int32_t jacobi_elim,
                  int32_t sum_mode, double gap_theta, double gap_fall,
                  double* alpha_hist, double* beta_hist, double* res_hist,
                  double* state_out, oracle_result* res) {
  memset(res, 0, sizeof(*res));
  if (n < 0 || maxit < 0 || !(tol >= 0.0)) { res->status = OR_ERR_ARG; return res->status; }
  if (n == 0) { res->status = OR_OK; return OR_OK; }

  double* d = calloc(n, sizeof(double));
  double* r = calloc(n, sizeof(double));
  double* u = calloc(n, sizeof(double));
  double* w = calloc(n, sizeof(double));
  double* m = calloc(n, sizeof(double));
  double* nv = calloc(n, sizeof(double));
  double* z = calloc(n, sizeof(double));
  double* q = calloc(n, sizeof(double));
  double* s = calloc(n, sizeof(double));
  double* p = calloc(n, sizeof(double));
  double* tmp = calloc(n, sizeof(double));
  int status = jacobi_diag(n, rp, ci, v, d);
  double gamma = 0.0, gamma_prev = 0.0, delta = 0.0, alpha = 0.0, alpha_prev = 0.0, beta = 0.0;
  double norm = 0.0;
  int32_t it = 0;
  int restart = 0;        /* the next step starts the recurrences afresh (beta = 0) */
  int32_t restarts = 0;
  int32_t last_rr_it = -1; /* iteration of the latest residual replacement */
  double gamma_ref = 0.0;  /* gamma when the residuals were last measured or replaced */

  for (int64_t i = 0; i < n; i++) x[i] = x0 ? x0[i] : 0.0;
  res->bnorm = sqrt(dot(sum_mode, n, b, b));
  if (status != OR_OK) goto done;
  if (norm_mode == 0 && res->bnorm == 0.0) {     /* A x = 0 has the solution x = 0 */
    for (int64_t i = 0; i < n; i++) x[i] = 0.0;
    status = OR_OK;
    goto done;
  }

  /* setup: r0 = b - A x0; u0 = M^-1 r0; w0 = A u0 */
  oracle_spmv(n, rp, ci, v, x, tmp);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) r[i] = b[i] - tmp[i];
  apply_jacobi(n, d, r, u);
  oracle_spmv(n, rp, ci, v, u, w);
  /* setup: gamma0 = (r0, u0); delta = (w0, u0); norm0 */
  gamma = dot(sum_mode, n, r, u);
  delta = dot(sum_mode, n, w, u);
  norm = norm_mode ? sqrt(dot(sum_mode, n, u, u)) : sqrt(dot(sum_mode, n, r, r));
  gamma_ref = gamma;
  /* setup: m0 = M^-1 w0; n0 = A m0 */
  apply_jacobi(n, d, w, m);
  oracle_spmv(n, rp, ci, v, m, nv);

  status = OR_ERR_NOT_CONVERGED;
  for (it = 0;; it++) {
    if (res_hist) res_hist[it] = norm;
    /* optional periodic residual replacement (not in the paper) */
    int replace = (rr_period > 0 && it > 0 && it % rr_period == 0 && last_rr_it != it);
    /* optional measured-gap replacement (not in the paper) */
    if (!replace && gap_theta > 0.0 && it > 0 && gamma > 0.0 && gamma * gap_fall <= gamma_ref) {
      oracle_spmv(n, rp, ci, v, x, tmp);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; i++) tmp[i] = (b[i] - tmp[i]) - r[i];
      double gap = sqrt(dot(sum_mode, n, tmp, tmp));
      double rnorm = sqrt(dot(sum_mode, n, r, r));
      gamma_ref = gamma;
      if (gap > gap_theta * rnorm) replace = 1;
    }
    /* stop test at the top of iteration i on norm_i */
    if (!replace) {
      int passed = norm_mode ? (norm <= tol) : (norm <= tol * res->bnorm);
      if (passed) {
        if (norm_mode) { status = OR_OK; break; }
        double t = true_residual(n, rp, ci, v, b, x, tmp, sum_mode);
        if (t <= tol * res->bnorm) { status = OR_OK; break; }
        replace = 1;
      }
    }
    if (replace) {
      /* r = b - A x, u = M^-1 r, w = A u, s = A p, q = M^-1 s, z = A q, m = M^-1 w, n = A m */
      oracle_spmv(n, rp, ci, v, x, tmp);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; i++) r[i] = b[i] - tmp[i];
      apply_jacobi(n, d, r, u);
      oracle_spmv(n, rp, ci, v, u, w);
      oracle_spmv(n, rp, ci, v, p, s);
      apply_jacobi(n, d, s, q);
      oracle_spmv(n, rp, ci, v, q, z);
      apply_jacobi(n, d, w, m);
      oracle_spmv(n, rp, ci, v, m, nv);
      gamma = dot(sum_mode, n, r, u);
      delta = dot(sum_mode, n, w, u);
      norm = norm_mode ? sqrt(dot(sum_mode, n, u, u)) : sqrt(dot(sum_mode, n, r, r));
      res->rr_count++;
      last_rr_it = it;
      gamma_ref = gamma;
      if (norm_mode ? (norm <= tol) : (norm <= tol * res->bnorm)) { status = OR_OK; break; }
    }
    if (it >= maxit) { status = OR_ERR_NOT_CONVERGED; break; }
    if (!isfinite(gamma) || !isfinite(delta)) { status = OR_ERR_NONFINITE; break; }
    /* scalars: beta, alpha */
    if (it > 0 && !restart) {
      beta = gamma / gamma_prev;
      double den = delta - beta * gamma / alpha_prev;
      if (!(gamma > 0.0) || !(den > 0.0)) {
        if (restarts >= max_restarts) { status = OR_ERR_BREAKDOWN; break; }
        /* restart: true residuals, direction recurrences reset, then beta = 0 */
        restarts++;
        for (int64_t i = 0; i < n; i++) { p[i] = 0.0; s[i] = 0.0; q[i] = 0.0; z[i] = 0.0; }
        oracle_spmv(n, rp, ci, v, x, tmp);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) r[i] = b[i] - tmp[i];
        apply_jacobi(n, d, r, u);
        oracle_spmv(n, rp, ci, v, u, w);
        apply_jacobi(n, d, w, m);
        oracle_spmv(n, rp, ci, v, m, nv);
        gamma = dot(sum_mode, n, r, u);
        delta = dot(sum_mode, n, w, u);
        norm = norm_mode ? sqrt(dot(sum_mode, n, u, u)) : sqrt(dot(sum_mode, n, r, r));
        res->rr_count++;
        last_rr_it = it;
        gamma_ref = gamma;
        restart = 1;
        it--;              /* re-enter the top of this iteration with the new values */
        continue;
      }
      alpha = gamma / den;
    } else {
      beta = 0.0;
      if (!(gamma > 0.0) || !(delta > 0.0)) { status = OR_ERR_BREAKDOWN; break; }
      alpha = gamma / delta;
    }
    restart = 0;
    if (alpha_hist) alpha_hist[it] = alpha;
    if (beta_hist) beta_hist[it] = beta;
    /* vector updates: z, q, s, p, then x, r, u, w */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
      z[i] = nv[i] + beta * z[i];
      s[i] = w[i] + beta * s[i];
      q[i] = jacobi_elim ? s[i] / d[i] : m[i] + beta * q[i];
      p[i] = u[i] + beta * p[i];
      x[i] = x[i] + alpha * p[i];
      r[i] = r[i] - alpha * s[i];
      u[i] = jacobi_elim ? r[i] / d[i] : u[i] - alpha * q[i];
      w[i] = w[i] - alpha * z[i];
    }
    /* dot products: gamma_{i+1}, delta, norm_{i+1} */
    gamma_prev = gamma;
    alpha_prev = alpha;
    gamma = dot(sum_mode, n, r, u);
    delta = dot(sum_mode, n, w, u);
    norm = norm_mode ? sqrt(dot(sum_mode, n, u, u)) : sqrt(dot(sum_mode, n, r, r));
    /* preconditioner and SpMV: m = M^-1 w; n = A m */
    apply_jacobi(n, d, w, m);
    oracle_spmv(n, rp, ci, v, m, nv);
  }

done:
  res->status = status;
  res->iters = it;
  res->res_recursive = norm;
  res->res_true = true_residual(n, rp, ci, v, b, x, tmp, sum_mode);
  res->gamma = gamma;
  res->delta = delta;
  if (state_out) {
    const double* vecs[10] = {x, r, u, w, p, q, s, z, m, nv};
    for (int k = 0; k < 10; k++) memcpy(state_out + (int64_t)k * n, vecs[k], n * sizeof(double));
  }
  free(d); free(r); free(u); free(w); free(m); free(nv);
  free(z); free(q); free(s); free(p); free(tmp);
  return status;
}

/* ---- Algorithm 1: classic PCG -------------------------------------------------------- */

/* Same conventions as oracle_pipecg (norm_mode 0: ||r|| <= tol ||b||; 1: sqrt((u,u)) <= tol),
 * without residual replacement.  state_out may hold 4*n doubles: x r u p. */
int oracle_pcg(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
               const double* b, const double* x0, double* x, double tol, int32_t maxit,
               int32_t norm_mode, int32_t sum_mode,
               double* alpha_hist, double* beta_hist, double* res_hist,
               double* state_out, oracle_result* res) {
  memset(res, 0, sizeof(*res));
  if (n < 0 || maxit < 0 || !(tol >= 0.0)) { res->status = OR_ERR_ARG; return res->status; }
  if (n == 0) { res->status = OR_OK; return OR_OK; }
  double* d = calloc(n, sizeof(double));
  double* r = calloc(n, sizeof(double));
  double* u = calloc(n, sizeof(double));
  double* p = calloc(n, sizeof(double));
  double* s = calloc(n, sizeof(double));
  double* tmp = calloc(n, sizeof(double));
  int status = jacobi_diag(n, rp, ci, v, d);
  double gamma = 0.0, gamma_prev = 0.0, delta = 0.0, alpha = 0.0, beta = 0.0, norm = 0.0;
  int32_t it = 0;
  for (int64_t i = 0; i < n; i++) x[i] = x0 ? x0[i] : 0.0;
  res->bnorm = sqrt(dot(sum_mode, n, b, b));
  if (status != OR_OK) goto done;
  if (norm_mode == 0 && res->bnorm == 0.0) {
    for (int64_t i = 0; i < n; i++) x[i] = 0.0;
    status = OR_OK;
    goto done;
  }
  /* setup: r0 = b - A x0; u0 = M^-1 r0 */
  oracle_spmv(n, rp, ci, v, x, tmp);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) r[i] = b[i] - tmp[i];
  apply_jacobi(n, d, r, u);
  /* setup: gamma0 = (u0, r0); norm0 */
  gamma = dot(sum_mode, n, u, r);
  norm = norm_mode ? sqrt(dot(sum_mode, n, u, u)) : sqrt(dot(sum_mode, n, r, r));
  status = OR_ERR_NOT_CONVERGED;
  for (it = 0;; it++) {
    if (res_hist) res_hist[it] = norm;
    if (norm_mode ? (norm <= tol) : (norm <= tol * res->bnorm)) { status = OR_OK; break; }
    if (it >= maxit) break;
    if (!isfinite(gamma)) { status = OR_ERR_NONFINITE; break; }
    if (!(gamma > 0.0)) { status = OR_ERR_BREAKDOWN; break; }
    /* beta */
    beta = it > 0 ? gamma / gamma_prev : 0.0;
    /* search direction: p_i = u_i + beta p_{i-1} */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) p[i] = u[i] + beta * p[i];
    /* s = A p; delta = (s, p); alpha = gamma / delta */
    oracle_spmv(n, rp, ci, v, p, s);
    delta = dot(sum_mode, n, s, p);
    if (!isfinite(delta)) { status = OR_ERR_NONFINITE; break; }
    if (!(delta > 0.0)) { status = OR_ERR_BREAKDOWN; break; }
    alpha = gamma / delta;
    if (alpha_hist) alpha_hist[it] = alpha;
    if (beta_hist) beta_hist[it] = beta;
    /* x, r and u = M^-1 r */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
      x[i] = x[i] + alpha * p[i];
      r[i] = r[i] - alpha * s[i];
    }
    apply_jacobi(n, d, r, u);
    /* gamma_{i+1} = (u, r), stopping norm */
    gamma_prev = gamma;
    gamma = dot(sum_mode, n, u, r);
    norm = norm_mode ? sqrt(dot(sum_mode, n, u, u)) : sqrt(dot(sum_mode, n, r, r));
  }
done:
  res->status = status;
  res->iters = it;
  res->res_recursive = norm;
  res->res_true = true_residual(n, rp, ci, v, b, x, tmp, sum_mode);
  res->gamma = gamma;
  res->delta = delta;
  if (state_out) {
    const double* vecs[4] = {x, r, u, p};
    for (int k = 0; k < 4; k++) memcpy(state_out + (int64_t)k * n, vecs[k], n * sizeof(double));
  }
  free(d); free(r); free(u); free(p); free(s); free(tmp);
  return status;
}

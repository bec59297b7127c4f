/*
 * Test driver: runs the oracle (oracle/ppcg_oracle.c, Alg. 1 and Alg. 2 of arXiv 2105.06176)
 * under AddressSanitizer and UndefinedBehaviorSanitizer on small systems that reach every
 * branch the tests use: both algorithms, both norms, residual replacement, the
 * Jacobi-elimination mode, both summation orders, a non-zero x0, history and state export,
 * maxit, and breakdown with and without restarts (an indefinite matrix).  It prints one
 * line per run, "<name> <status> <iters> <rr_count>", for the test to compare with the
 * uninstrumented library.  Built and run by tests/test_oracle_sanitize.py only.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

typedef struct {
  int32_t status, iters, rr_count, pad;
  double bnorm, res_recursive, res_true, gamma, delta;
} oracle_result;

int oracle_pipecg(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* b,
                  const double* x0, double* x, double tol, int32_t maxit, int32_t norm_mode,
                  int32_t rr_period, int32_t max_restarts, int32_t jacobi_elim, int32_t sum_mode,
                  double gap_theta, double gap_fall, double* alpha_hist, double* beta_hist,
                  double* res_hist, double* state_out, oracle_result* res);
int oracle_pcg(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* b,
               const double* x0, double* x, double tol, int32_t maxit, int32_t norm_mode, int32_t sum_mode,
               double* alpha_hist, double* beta_hist, double* res_hist, double* state_out, oracle_result* res);

/* 2-D 5-point stencil on an m x m grid with diagonal `diag` (4 for Poisson). */
static int64_t poisson(int m, double diag, int64_t** rp, int32_t** ci, double** v) {
  const int64_t n = (int64_t)m * m;
  *rp = malloc((n + 1) * sizeof(int64_t));
  *ci = malloc(5 * n * sizeof(int32_t));
  *v = malloc(5 * n * sizeof(double));
  int64_t k = 0;
  for (int64_t i = 0; i < n; i++) {
    const int y = (int)(i / m), x = (int)(i % m);
    (*rp)[i] = k;
    if (y > 0) { (*ci)[k] = (int32_t)(i - m); (*v)[k++] = -1.0; }
    if (x > 0) { (*ci)[k] = (int32_t)(i - 1); (*v)[k++] = -1.0; }
    (*ci)[k] = (int32_t)i; (*v)[k++] = diag;
    if (x < m - 1) { (*ci)[k] = (int32_t)(i + 1); (*v)[k++] = -1.0; }
    if (y < m - 1) { (*ci)[k] = (int32_t)(i + m); (*v)[k++] = -1.0; }
  }
  (*rp)[n] = k;
  return n;
}

int main(void) {
  int64_t *rp; int32_t *ci; double *v;
  const int m = 24;
  const int64_t n = poisson(m, 4.0, &rp, &ci, &v);
  double* b = malloc(n * sizeof(double));
  double* x0 = malloc(n * sizeof(double));
  double* x = malloc(n * sizeof(double));
  for (int64_t i = 0; i < n; i++) { b[i] = (double)((i * 7919) % 97) / 97.0 - 0.5; x0[i] = 0.01 * (double)(i % 13); }
  const int maxit = 2000;
  double* ah = malloc(maxit * sizeof(double));
  double* bh = malloc(maxit * sizeof(double));
  double* rh = malloc((maxit + 1) * sizeof(double));
  double* st = malloc(10 * n * sizeof(double));
  oracle_result r;
  struct { const char* name; int alg, norm, rr, restarts, elim, sum, use_x0, hist, it; double tol, gap; } runs[] = {
    {"pipecg", 2, 0, 0, 8, 0, 0, 0, 1, maxit, 1e-8, 1e-6},
    {"pipecg_nogap", 2, 0, 0, 8, 0, 0, 0, 1, maxit, 1e-8, 0.0},
    {"pipecg_gap_every", 2, 0, 0, 8, 0, 0, 0, 1, maxit, 1e-8, 1e-300},
    {"pipecg_paper", 2, 1, 0, 8, 0, 0, 0, 0, maxit, 1e-5, 1e-6},
    {"pipecg_rr", 2, 0, 7, 8, 0, 0, 1, 1, maxit, 1e-8, 1e-6},
    {"pipecg_elim", 2, 0, 0, 8, 1, 0, 0, 1, maxit, 1e-8, 1e-6},
    {"pipecg_pairwise", 2, 0, 0, 8, 0, 1, 0, 0, maxit, 1e-8, 1e-6},
    {"pipecg_maxit", 2, 0, 0, 8, 0, 0, 0, 1, 5, 1e-8, 1e-6},
    {"pcg", 1, 0, 0, 0, 0, 0, 0, 1, maxit, 1e-8, 0.0},
    {"pcg_paper_x0", 1, 1, 0, 0, 0, 1, 1, 1, maxit, 1e-5, 0.0},
  };
  for (size_t k = 0; k < sizeof(runs) / sizeof(runs[0]); k++) {
    const double* x0p = runs[k].use_x0 ? x0 : NULL;
    double *a1 = runs[k].hist ? ah : NULL, *b1 = runs[k].hist ? bh : NULL, *r1 = runs[k].hist ? rh : NULL;
    double* s1 = runs[k].hist ? st : NULL;
    if (runs[k].alg == 2)
      oracle_pipecg(n, rp, ci, v, b, x0p, x, runs[k].tol, runs[k].it, runs[k].norm, runs[k].rr, runs[k].restarts,
                    runs[k].elim, runs[k].sum, runs[k].gap, runs[k].gap > 1e-100 ? 100.0 : 1.0, a1, b1, r1, s1, &r);
    else
      oracle_pcg(n, rp, ci, v, b, x0p, x, runs[k].tol, runs[k].it, runs[k].norm, runs[k].sum, a1, b1, r1, s1, &r);
    printf("%s %d %d %d\n", runs[k].name, r.status, r.iters, r.rr_count);
  }
  /* indefinite 3 x 3 (breakdown), with and without restarts */
  const int64_t rp3[4] = {0, 2, 4, 5};
  const int32_t ci3[5] = {0, 1, 0, 1, 2};
  const double v3[5] = {1.0, 2.0, 2.0, 1.0, 1.0};
  const double b3[3] = {1.0, -1.0, 1.0};
  double x3[3];
  oracle_pipecg(3, rp3, ci3, v3, b3, NULL, x3, 1e-8, 100, 0, 0, 8, 0, 0, 1e-6, 100.0, NULL, NULL, NULL, NULL, &r);
  printf("indefinite %d %d %d\n", r.status, r.iters, r.rr_count);
  oracle_pipecg(3, rp3, ci3, v3, b3, NULL, x3, 1e-8, 100, 0, 0, 0, 0, 0, 1e-6, 100.0, NULL, NULL, NULL, NULL, &r);
  printf("indefinite_norestart %d %d %d\n", r.status, r.iters, r.rr_count);
  free(rp); free(ci); free(v); free(b); free(x0); free(x); free(ah); free(bh); free(rh); free(st);
  return 0;
}

/* The C ABI used from plain C99 (no C++, no Python): defaults, the host
 * checks of pdhg_create, NULL safety and, where a GPU is present, a short
 * solve of a 2x3 LP with its KKT measures. Prints one line per check and
 * "ok" at the end; exits non-zero if any check fails.
 *
 * LP (Section 2's standard form): A = [[1, 2, 0], [0, 1, 1]], b = (3, 2),
 * c = (1, 1, 1). With x1 = 3 - 2 x2 and x3 = 2 - x2 the objective is 5 - 2 x2,
 * so the unique optimum is x = (0, 1.5, 0.5) with value 2 (dual y = (0, 1),
 * b^T y = 2). */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "pdhg.h"

static int fails = 0;

static void check(int cond, const char* what) {
  printf("%s %s\n", cond ? "pass" : "FAIL", what);
  if (!cond) fails += 1;
}

int main(void) {
  pdhg_options o;
  memset(&o, 0, sizeof(o));
  pdhg_default_options(&o);
  check(o.precision == PDHG_FP64 && o.eval_every == 64 && o.ruiz_iters == 10 && o.step_factor == 0.9,
        "defaults");

  const int64_t m = 2, n = 3, nnz = 4;
  const int64_t rp[3] = {0, 2, 4};
  const int32_t ci[4] = {0, 1, 1, 2};
  const double v[4] = {1.0, 2.0, 1.0, 1.0};
  const double b[2] = {3.0, 2.0};
  const double c[3] = {1.0, 1.0, 1.0};

  pdhg_ctx* ctx = (pdhg_ctx*)0x1;
  const int64_t bad_rp[3] = {0, 3, 4}; /* row 0 would hold columns 0, 1, 1: not increasing */
  pdhg_status st = pdhg_create(m, n, nnz, bad_rp, ci, v, b, c, NULL, NULL, &o, NULL, &ctx);
  check(st == PDHG_ERR_INVALID && ctx == NULL, "malformed CSR rejected, *out set to NULL");
  check(strlen(pdhg_last_error(NULL)) > 0, "pdhg_last_error(NULL) describes it");

  const double nan_b[2] = {3.0, NAN};
  st = pdhg_create(m, n, nnz, rp, ci, v, nan_b, c, NULL, NULL, &o, NULL, &ctx);
  check(st == PDHG_ERR_NUMERIC, "NaN in b rejected");

  check(pdhg_iterate(NULL, 10, 0.0, NULL) == PDHG_ERR_INVALID, "NULL context rejected");
  pdhg_destroy(NULL);

  st = pdhg_create(m, n, nnz, rp, ci, v, b, c, NULL, NULL, &o, NULL, &ctx);
  if (st == PDHG_ERR_CUDA) {
    printf("skip solve: no usable GPU (%s)\n", pdhg_last_error(NULL));
  } else {
    check(st == PDHG_OK && ctx != NULL, "well-formed LP accepted");
    if (st == PDHG_OK) {
      int64_t done = 0;
      st = pdhg_iterate(ctx, 20000, 1e-8, &done);
      pdhg_kkt_info k;
      pdhg_status sk = pdhg_kkt(ctx, PDHG_CURRENT, &k);
      check(st == PDHG_OK && sk == PDHG_OK && k.rel_kkt <= 1e-8 && fabs(k.primal_obj - 2.0) <= 1e-6,
            "solve to 1e-8 reaches the optimal value 2");
      pdhg_destroy(ctx);
    }
  }
  printf(fails ? "FAILED\n" : "ok\n");
  return fails ? 1 : 0;
}

/* A plain C99 user of libajf: include/ajf.h and the shared library, no Python.
 *
 * On a host-only context (device -1) it loads a 2-qubit circuit (H on qubit 0, then CX with
 * control 0), adds one single-qubit depolarising noise after the H (Kraus operators
 * sqrt(1 - 3p/4) I and sqrt(p/4) X, Y, Z, p = 0.01), plans Alg. I and Alg. II, replays both
 * programs with ajf_check_plan, and drives the error paths the header documents. It prints one
 * "key value" line per figure for the test that runs it, and exits non-zero at the first
 * unexpected status. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "ajf.h"

static int expect(const char *what, ajf_status got, ajf_status want) {
  if (got != want) {
    fprintf(stderr, "%s: status %d, expected %d\n", what, (int)got, (int)want);
    return 1;
  }
  return 0;
}

int main(void) {
  ajf_ctx *ctx = NULL;
  if (expect("create", ajf_create(&ctx, -1, NULL), AJF_OK)) return 1;

  const double r = 1.0 / sqrt(2.0);
  /* complex128 interleaved, row-major: H (2 x 2), then CX (4 x 4, first listed qubit = control) */
  double mats[2 * 4 + 2 * 16];
  memset(mats, 0, sizeof(mats));
  mats[0] = r; mats[2] = r; mats[4] = r; mats[6] = -r;
  double *cx = mats + 8;
  cx[2 * 0] = 1; cx[2 * 5] = 1; cx[2 * 11] = 1; cx[2 * 14] = 1;
  const int32_t arity[2] = {1, 2};
  const int32_t qubits[3] = {0, 0, 1};
  if (expect("load", ajf_load_circuit(ctx, AJF_IDEAL, 2, 2, arity, qubits, mats), AJF_OK)) return 1;

  const double p = 0.01, a = sqrt(1.0 - 0.75 * p), b = sqrt(p / 4.0);
  double kraus[4 * 8];
  memset(kraus, 0, sizeof(kraus));
  kraus[0] = a; kraus[6] = a;            /* sqrt(1 - 3p/4) I */
  kraus[8 + 2] = b; kraus[8 + 4] = b;    /* sqrt(p/4) X */
  kraus[16 + 3] = -b; kraus[16 + 5] = b; /* sqrt(p/4) Y = [[0, -i], [i, 0]] */
  kraus[24 + 0] = b; kraus[24 + 6] = -b; /* sqrt(p/4) Z */
  const int32_t nq[1] = {0};
  if (expect("noise", ajf_add_noise(ctx, 0, 1, nq, 4, kraus), AJF_OK)) return 1;

  for (int alg = 1; alg <= 2; ++alg) {
    ajf_plan_opts o;
    memset(&o, 0, sizeof(o));
    o.planner = AJF_PLANNER_AUTO;
    o.precision = AJF_PREC_F64;
    o.trials = 4;
    ajf_plan_info info;
    if (expect("plan", ajf_plan(ctx, alg, &o, &info), AJF_OK)) return 1;
    if (expect("check", ajf_check_plan(ctx), AJF_OK)) return 1;
    int64_t units = 0;
    if (expect("slice count", ajf_slice_count(ctx, &units), AJF_OK)) return 1;
    printf("alg%d_leaves %d\n", alg, (int)info.n_leaves);
    printf("alg%d_open_bits %d\n", alg, (int)info.n_open_bits);
    printf("alg%d_width %d\n", alg, (int)info.width);
    printf("alg%d_cmacs %.17g\n", alg, info.cmacs);
    printf("alg%d_units %lld\n", alg, (long long)units);
    ajf_result res;
    if (expect("fidelity on a host-only context", ajf_fidelity(ctx, -1.0, &res), AJF_E_STATE)) return 1;
  }

  /* documented errors */
  ajf_plan_opts bad;
  memset(&bad, 0, sizeof(bad));
  bad.reserved[0] = 1;
  if (expect("reserved field", ajf_plan(ctx, 2, &bad, NULL), AJF_E_ARG)) return 1;
  if (expect("bad alg", ajf_plan(ctx, 7, NULL, NULL), AJF_E_ARG)) return 1;
  mats[0] = 2.0; /* H no longer unitary */
  if (expect("non-unitary gate", ajf_load_circuit(ctx, AJF_IDEAL, 2, 2, arity, qubits, mats), AJF_E_NOT_UNITARY))
    return 1;
  mats[0] = r;
  if (expect("reload", ajf_load_circuit(ctx, AJF_IDEAL, 2, 2, arity, qubits, mats), AJF_OK)) return 1;
  kraus[0] = 1.5; /* no longer trace preserving */
  if (expect("non-TP noise", ajf_add_noise(ctx, 0, 1, nq, 4, kraus), AJF_E_NOT_TP)) return 1;
  if (strlen(ajf_last_error(ctx)) == 0) {
    fprintf(stderr, "no error message\n");
    return 1;
  }
  printf("last_error %s\n", ajf_last_error(ctx));
  ajf_destroy(ctx);
  printf("done 1\n");
  return 0;
}

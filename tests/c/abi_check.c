/* A plain C11 consumer of libcoffee.so: the three headers compile as C, every declared entry
 * point links, and the host-only calls behave as documented (no CUDA device is needed).
 * Prints "ok" and exits 0 on success; prints the failed check and exits 1 otherwise. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "coffee.h"
#include "coffee_diag.h"
#include "coffee_peaks.h"

static int failures = 0;
#define CHECK(cond)                                                        \
  do {                                                                     \
    if (!(cond)) {                                                         \
      printf("FAILED %s:%d: %s (%s)\n", __FILE__, __LINE__, #cond,         \
             coffee_last_error());                                         \
      ++failures;                                                          \
    }                                                                      \
  } while (0)

/* Every entry point's address is taken, so the link fails if one is missing. */
typedef void (*entry_fn)(void);
static const entry_fn entry_points[] = {
    (entry_fn)coffee_ndof, (entry_fn)coffee_tabulate, (entry_fn)coffee_reference_tensor,
    (entry_fn)coffee_supported, (entry_fn)coffee_assemble, (entry_fn)coffee_assemble_ex,
    (entry_fn)coffee_split_coords, (entry_fn)coffee_round_coef, (entry_fn)coffee_assemble_path,
    (entry_fn)coffee_assemble_host, (entry_fn)coffee_host_pool_trim,
    (entry_fn)coffee_assemble_backward, (entry_fn)coffee_assemble_backward_noalloc,
    (entry_fn)coffee_batch_plan, (entry_fn)coffee_batch_plan_costs, (entry_fn)coffee_batch_launch,
    (entry_fn)coffee_batch_free, (entry_fn)coffee_batch_split, (entry_fn)coffee_sparsity,
    (entry_fn)coffee_csr_map,
    (entry_fn)coffee_assemble_csr, (entry_fn)coffee_csr_supported, (entry_fn)coffee_check_errors,
    (entry_fn)coffee_last_error, (entry_fn)coffee_peak_fp64, (entry_fn)coffee_peak_mma,
    (entry_fn)coffee_diag_wait_timeout, (entry_fn)coffee_table_image};

int main(void) {
  for (size_t i = 0; i < sizeof entry_points / sizeof entry_points[0]; ++i) CHECK(entry_points[i] != NULL);

  /* ndof: triangle/tetrahedron/prism Lagrange counts, times d for the vector forms */
  CHECK(coffee_ndof(COFFEE_MASS, 3, COFFEE_TRIANGLE) == 10);
  CHECK(coffee_ndof(COFFEE_HELMHOLTZ, 4, COFFEE_TETRAHEDRON) == 35);
  CHECK(coffee_ndof(COFFEE_MASS, 2, COFFEE_PRISM) == 18);
  CHECK(coffee_ndof(COFFEE_BURGERS_JAC, 2, COFFEE_TETRAHEDRON) == 30);
  CHECK(coffee_ndof(COFFEE_MASS, 9, COFFEE_TRIANGLE) == COFFEE_ERR_INVALID_ARG);

  /* tabulate: size query, then a rule that integrates x^2 y exactly on the reference
   * triangle (2! 1! / 5! = 1/60) and a basis that sums to one at every point */
  int nq = 0, nd = 0;
  CHECK(coffee_tabulate(COFFEE_TRIANGLE, 2, 3, &nq, &nd, NULL, NULL, NULL, NULL) == COFFEE_OK);
  CHECK(nq > 0 && nd == 6);
  double* pts = malloc(sizeof(double) * nq * 2);
  double* wts = malloc(sizeof(double) * nq);
  double* phi = malloc(sizeof(double) * nq * nd);
  CHECK(coffee_tabulate(COFFEE_TRIANGLE, 2, 3, NULL, NULL, pts, wts, phi, NULL) == COFFEE_OK);
  double m = 0.0, worst = 0.0;
  for (int q = 0; q < nq; ++q) {
    m += wts[q] * pts[2 * q] * pts[2 * q] * pts[2 * q + 1];
    double s = 0.0;
    for (int i = 0; i < nd; ++i) s += phi[q * nd + i];
    if (fabs(s - 1.0) > worst) worst = fabs(s - 1.0);
  }
  CHECK(fabs(m - 1.0 / 60.0) < 1e-15);
  CHECK(worst < 1e-13);
  free(pts);
  free(wts);
  free(phi);

  /* reference tensors: P1 triangle mass, T[0][i*3+j] = (1 + [i==j]) / 24 on the reference cell */
  int K = 0, N = 0;
  CHECK(coffee_reference_tensor(COFFEE_MASS, 1, COFFEE_TRIANGLE, &K, &N, NULL) == COFFEE_OK);
  CHECK(K == 1 && N == 9);
  double T[9];
  CHECK(coffee_reference_tensor(COFFEE_MASS, 1, COFFEE_TRIANGLE, NULL, NULL, T) == COFFEE_OK);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) CHECK(fabs(T[i * 3 + j] - (i == j ? 2.0 : 1.0) / 24.0) < 1e-16);
  CHECK(coffee_reference_tensor(COFFEE_HELMHOLTZ, 2, COFFEE_PRISM, &K, &N, NULL) == COFFEE_ERR_UNSUPPORTED);

  /* support queries */
  CHECK(coffee_supported(COFFEE_HELMHOLTZ, 3, COFFEE_TETRAHEDRON, COFFEE_TF32X3) == 1);
  CHECK(coffee_supported(COFFEE_HELMHOLTZ, 4, COFFEE_PRISM, COFFEE_TF32X3) == 1);
  CHECK(coffee_assemble_path(COFFEE_HELMHOLTZ, 1, COFFEE_TETRAHEDRON, COFFEE_TF32X3, 0) == 2);
  CHECK(coffee_assemble_path(COFFEE_HELMHOLTZ, 1, COFFEE_TETRAHEDRON, COFFEE_TF32X3, COFFEE_FLAG_TENSOR_CORES) == 1);
  CHECK(coffee_assemble_path(COFFEE_HELMHOLTZ, 3, COFFEE_TETRAHEDRON, COFFEE_TF32X3, 0) == 1);
  CHECK(coffee_assemble_path(COFFEE_HELMHOLTZ, 3, COFFEE_TETRAHEDRON, COFFEE_FP64, 0) == 0);
  CHECK(coffee_assemble_path(COFFEE_BURGERS_JAC, 1, COFFEE_TRIANGLE, COFFEE_TF32X3, 0) == 2);
  CHECK(coffee_assemble_path(COFFEE_BURGERS_JAC, 2, COFFEE_TETRAHEDRON, COFFEE_TF32X3, COFFEE_FLAG_CUDA_CORES) == 1);
  CHECK(coffee_csr_supported(COFFEE_BURGERS_RESIDUAL, 2, COFFEE_TETRAHEDRON, COFFEE_FP64) == 0);

  /* argument errors are reported on the host, before any CUDA call */
  coffee_assemble_args a = {0};
  a.form = COFFEE_HELMHOLTZ;
  a.degree = 7;
  a.cell = COFFEE_TETRAHEDRON;
  a.ncells = 4;
  CHECK(coffee_assemble_ex(&a, NULL) == COFFEE_ERR_INVALID_ARG);
  a.degree = 2;
  CHECK(coffee_assemble_ex(&a, NULL) == COFFEE_ERR_INVALID_ARG); /* NULL pointers */
  CHECK(coffee_split_coords(NULL, 0, NULL, NULL) == COFFEE_OK);   /* nothing to split */
  CHECK(coffee_split_coords(NULL, -1, NULL, NULL) == COFFEE_ERR_INVALID_ARG);
  CHECK(coffee_round_coef(NULL, 0, NULL, NULL) == COFFEE_OK);     /* nothing to round */
  CHECK(coffee_round_coef(NULL, -1, NULL, NULL) == COFFEE_ERR_INVALID_ARG);
  a.ncells = 0;
  CHECK(coffee_assemble_ex(&a, NULL) == COFFEE_OK); /* empty input: no launch */
  CHECK(coffee_assemble_host(&a, 0, NULL) == COFFEE_ERR_INVALID_ARG);
  CHECK(coffee_peak_fp64(NULL) == COFFEE_ERR_INVALID_ARG);

  if (failures) return 1;
  printf("ok\n");
  return 0;
}

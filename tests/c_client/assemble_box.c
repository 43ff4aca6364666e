/* A client of the C ABI alone (no Python): the cross-lattice tile on an affine 2 x 2 x 2 box of tiles,
 * assembled in the FP64 and the FP64-accurate forms; checks their agreement, that translations lie in
 * the null space of the assembled matrix (a property of eq. 58's tile blocks for any macro map), and
 * that tables stored with msasm_tables_save and read back assemble the same values bit for bit.
 * Prints one line per check and exits 0 when all pass. */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "msasm.h"

#define CHECK(call)                                                            \
  do {                                                                         \
    msasm_status st_ = (call);                                                 \
    if (st_ != MSASM_OK) {                                                     \
      fprintf(stderr, "%s -> %d: %s\n", #call, (int)st_, msasm_last_error()); \
      return 1;                                                                \
    }                                                                          \
  } while (0)
#define CUDA(call)                                                                   \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      fprintf(stderr, "%s -> %s\n", #call, cudaGetErrorString(e_));                  \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

static int assemble(msasm_plan* plan, const double* d_ctrl, msasm_precision prec, double* h_vals, int64_t nnz) {
  void* d_vals = NULL;
  CUDA(cudaMalloc(&d_vals, (size_t)nnz * sizeof(double)));
  CHECK(msasm_assemble(plan, d_ctrl, 1.0, 0.3, prec, d_vals, MSASM_FLAG_CHECK_DEGENERATE, NULL));
  CUDA(cudaMemcpy(h_vals, d_vals, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToHost));
  CUDA(cudaFree(d_vals));
  return 0;
}

int main(int argc, char** argv) {
  const char* path = argc > 1 ? argv[1] : "cross_q2.msasm";
  /* the cross cell: a centre cube and six struts, strut width 0.3, degree 2, 2 elements per direction */
  const double c0 = 0.35, c1 = 0.65;
  const double lo[7][3] = {{c0, c0, c0}, {0, c0, c0}, {c1, c0, c0}, {c0, 0, c0}, {c0, c1, c0}, {c0, c0, 0}, {c0, c0, c1}};
  const double hi[7][3] = {{c1, c1, c1}, {c0, c1, c1}, {1, c1, c1}, {c1, c0, c1}, {c1, 1, c1}, {c1, c1, c0}, {c1, c1, 1}};
  int32_t degree[21], n_elem[21];
  for (int i = 0; i < 21; ++i) degree[i] = 2, n_elem[i] = 2;
  msasm_micro_desc micro = {7, degree, n_elem, &lo[0][0], &hi[0][0]};
  msasm_tables* tab = NULL;
  CHECK(msasm_build_tables(&micro, 2, 0, NULL, &tab));

  /* the affine map of [0,1]^3 onto [0,2]^3: degree 2, two elements per direction, control points at
     the Greville abscissae of the open knot vector */
  const double knots[7] = {0, 0, 0, 0.5, 1, 1, 1};
  const double grev[4] = {0.0, 0.25, 0.75, 1.0};
  msasm_macro_desc macro;
  for (int d = 0; d < 3; ++d) macro.degree[d] = 2, macro.n_knots[d] = 7, macro.knots[d] = knots;
  double h_ctrl[64 * 3];
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < 4; ++j)
      for (int i = 0; i < 4; ++i) {
        double* p = h_ctrl + 3 * (i + 4 * (j + 4 * k));
        p[0] = 2.0 * grev[i], p[1] = 2.0 * grev[j], p[2] = 2.0 * grev[k];
      }
  msasm_plan* plan = NULL;
  int64_t n_rows = 0, nnz = 0;
  CHECK(msasm_plan_create(tab, &macro, 0, NULL, &plan, &n_rows, &nnz));
  double* d_ctrl = NULL;
  CUDA(cudaMalloc((void**)&d_ctrl, sizeof(h_ctrl)));
  CUDA(cudaMemcpy(d_ctrl, h_ctrl, sizeof(h_ctrl), cudaMemcpyHostToDevice));

  double* v64 = (double*)malloc((size_t)nnz * sizeof(double));
  double* vemu = (double*)malloc((size_t)nnz * sizeof(double));
  double* vload = (double*)malloc((size_t)nnz * sizeof(double));
  if (!v64 || !vemu || !vload) return 1;
  if (assemble(plan, d_ctrl, MSASM_F64, v64, nnz) || assemble(plan, d_ctrl, MSASM_F64_EMU, vemu, nnz)) return 1;
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < nnz; ++i) num += (vemu[i] - v64[i]) * (vemu[i] - v64[i]), den += v64[i] * v64[i];
  const double rel = sqrt(num / den);
  printf("rows %lld nnz %lld: FP64-accurate vs FP64 relative Frobenius %.3e\n", (long long)n_rows, (long long)nnz, rel);
  if (!(rel <= 1e-12)) return 1;

  /* K t = 0 for the three translations t (CSR pattern from the plan) */
  int64_t* d_rowptr = NULL;
  int32_t* d_col = NULL;
  CUDA(cudaMalloc((void**)&d_rowptr, (size_t)(n_rows + 1) * sizeof(int64_t)));
  CUDA(cudaMalloc((void**)&d_col, (size_t)nnz * sizeof(int32_t)));
  CHECK(msasm_plan_csr(plan, d_rowptr, d_col, NULL));
  int64_t* rowptr = (int64_t*)malloc((size_t)(n_rows + 1) * sizeof(int64_t));
  int32_t* col = (int32_t*)malloc((size_t)nnz * sizeof(int32_t));
  if (!rowptr || !col) return 1;
  CUDA(cudaMemcpy(rowptr, d_rowptr, (size_t)(n_rows + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(col, d_col, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
  double worst = 0.0;
  for (int a = 0; a < 3; ++a) {
    double r2 = 0.0, k2 = 0.0;
    for (int64_t r = 0; r < n_rows; ++r) {
      double s = 0.0;
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        if (col[e] % 3 == a) s += v64[e];
        k2 += v64[e] * v64[e];
      }
      r2 += s * s;
    }
    const double res = sqrt(r2 / k2);
    worst = res > worst ? res : worst;
  }
  printf("translations: |K t| / |K| at most %.3e\n", worst);
  if (!(worst <= 1e-13)) return 1;

  /* stored tables read back: the same values bit for bit */
  CHECK(msasm_tables_save(tab, path, NULL));
  msasm_tables* tab2 = NULL;
  CHECK(msasm_tables_load(path, NULL, &tab2));
  msasm_plan* plan2 = NULL;
  int64_t n_rows2 = 0, nnz2 = 0;
  CHECK(msasm_plan_create(tab2, &macro, 0, NULL, &plan2, &n_rows2, &nnz2));
  if (nnz2 != nnz || assemble(plan2, d_ctrl, MSASM_F64, vload, nnz)) return 1;
  const int same = memcmp(vload, v64, (size_t)nnz * sizeof(double)) == 0;
  printf("tables stored and read back: %s\n", same ? "identical values" : "values differ");
  if (!same) return 1;

  msasm_plan_destroy(plan2);
  msasm_plan_destroy(plan);
  msasm_tables_destroy(tab2);
  msasm_tables_destroy(tab);
  cudaFree(d_ctrl);
  cudaFree(d_rowptr);
  cudaFree(d_col);
  free(v64), free(vemu), free(vload), free(rowptr), free(col);
  printf("ok\n");
  return 0;
}

// Smoothed-aggregation multigrid preconditioner (host setup, device cycle).
#pragma once
#include <vector>

#include "common.cuh"

namespace pdfgb {

struct AmgLevel {
  int32_t n = 0, nc = 0;  // rows of this level, of the next one
  int64_t nnz_a = 0, nnz_q = 0;
  int32_t *a_rp = nullptr, *a_ci = nullptr;  // the level's matrix A
  double* a_v = nullptr;
  double* w = nullptr;                       // damped Jacobi weights w_s / a_ii
  int32_t *q_rp = nullptr, *q_ci = nullptr;  // Q = (I - W A) P, n x nc
  double* q_v = nullptr;
  int32_t *s_rp = nullptr, *s_ci = nullptr;  // Q^T, nc x n
  double* s_v = nullptr;
  double *b = nullptr, *x = nullptr, *z = nullptr;  // right-hand side (l > 0), pre-smoothed, result (l > 0)
};

struct Amg {
  std::vector<AmgLevel> lv;
  int32_t nc = 0;           // coarsest size
  double* cinv = nullptr;   // [nc][nc] regularised inverse of the coarsest matrix
  double *cb = nullptr, *cz = nullptr;
};

// Builds the hierarchy of the symmetric CSR matrix (n rows, columns
// sorted; positive definite, or with singular = true positive semi-definite
// with the constants as null space) and uploads it.
pdf_status amg_setup(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                     const std::vector<double>& v, bool singular, Amg& G);
void amg_free(Amg& G);
// z = M^-1 r (one V-cycle); part receives the block partials of r . z
// (blocks of 256 rows) when the hierarchy has a level, else nothing.  Every
// kernel returns at once when *done is set.
pdf_status amg_apply(const Amg& G, const double* r, double* z, double* part, const int32_t* done, cudaStream_t st);

}  // namespace pdfgb

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
// z = M^-1 r (one V-cycle).  When the hierarchy has a level, the finest
// up-sweep also forms r . z (block partials in part, finished by the last
// block through *counter, which it resets): *rz_old = *rz, *rz = r . z;
// else the caller forms it.  Every kernel returns at once when *done is set.
pdf_status amg_apply(const Amg& G, const double* r, double* z, double* part, int32_t* counter, double* rz,
                     double* rz_old, const int32_t* done, cudaStream_t st);

// The whole preconditioned conjugate-gradient iteration for the CSR matrix
// (n rows; rp, ci, val) in one persistent cooperative kernel, the phases
// separated by grid-wide barriers.  Entry state (as left by the caller's
// initialisation): x, r = b - A x, p = q = 0, scal[kPcgRz] = scal[kPcgRzOld] = 1,
// scal[kPcgTol2] = the stopping threshold on r.r, ctl[kPcgDone/Iters/MaxIt].
// On return x, r, scal[kPcgRr], ctl[kPcgIters] and ctl[kPcgDone] = 1 (the
// caller tells convergence from r.r <= tol2).  part: 3 x grid doubles.
// Returns PDF_EINVAL when the device cannot launch it cooperatively (the
// caller then runs the separate kernels).
enum { kPcgDone = 0, kPcgIters = 1, kPcgMaxIt = 2 };
enum { kPcgPq = 0, kPcgRz = 1, kPcgRr = 2, kPcgRzOld = 6, kPcgTol2 = 7 };
pdf_status amg_pcg(const Amg& G, int32_t n, const int32_t* rp, const int32_t* ci, const double* val, double* x,
                   double* r, double* z, double* p, double* q, double* scal, int32_t* ctl, double* part,
                   int32_t part_cap, cudaStream_t st);

}  // namespace pdfgb

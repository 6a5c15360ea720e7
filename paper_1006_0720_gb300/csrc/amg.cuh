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

// ---------------------------------------------------------------------------
// The relaxation's multigrid: the prolongations of the smoothed-aggregation
// hierarchy of the stiffness matrix K (fixed per mesh), applied to the
// relaxation matrices M + K_{L^2} of the current statistics, whose Galerkin
// coarse matrices, smoothers and Q = (I - W A) P are recomputed on the
// device at every solve through precomputed plans.  Four operators
// ("variants"): the C_xi classes of wp_11, wp_22, wp_33 with their Dirichlet
// rows (no-slip nodes) and the off-diagonal components (walls and no-slip
// nodes).  Fixed unknowns carry identity rows and columns.
constexpr int kRxVar = 4;
constexpr int kRxMaxLv = 12;

struct RxLevel {
  int32_t n = 0, nc = 0;
  int64_t nnz_a = 0, nnz_ap = 0;
  int32_t *a_rp = nullptr, *a_ci = nullptr, *a_dpos = nullptr;  // A_l and its diagonal positions
  int32_t *q_rp = nullptr, *q_ci = nullptr;                      // pattern of A_l P_l = pattern of Q_l
  int32_t *s_rp = nullptr, *s_ci = nullptr, *s_perm = nullptr;   // Q_l^T: S[t] = Q[s_perm[t]]
  int32_t *ap_off = nullptr, *ap_qa = nullptr;                   // (A P)[t] = sum a[ap_qa] * ap_pv
  double* ap_pv = nullptr;
  int32_t *c_off = nullptr, *c_tap = nullptr;                    // A_{l+1}[c] = sum c_pv * (A P)[c_tap]
  double* c_pv = nullptr;
  double* q_pin = nullptr;                                       // P at each (A P) position, else 0
  int32_t* q_row = nullptr;
  double *a_v[kRxVar] = {}, *ap_v[kRxVar] = {}, *q_v[kRxVar] = {}, *s_v[kRxVar] = {};
  double* w_v[kRxVar] = {};  // smoother weights W = omega / a_ii
  // FP32 copies for the cycle: A, Q, S and W
  float *a_f[kRxVar] = {}, *q_f[kRxVar] = {}, *s_f[kRxVar] = {}, *w_f[kRxVar] = {};
  float *b = nullptr, *x = nullptr, *z = nullptr;                // [9][n] (b, z for l > 0)
};

struct RelaxAmg {
  std::vector<RxLevel> lv;
  int32_t nc = 0;
  int64_t nnz_c = 0;
  int32_t *c_rp = nullptr, *c_ci = nullptr;  // the coarsest matrix
  double* c_v[kRxVar] = {};
  double* cmat = nullptr;                    // [kRxVar][nc][2 nc] Gauss-Jordan work
  float* cinv = nullptr;                     // [kRxVar][nc][nc]
  float *cb = nullptr, *cz = nullptr;        // [9][nc]
  double *omega = nullptr, *gpart = nullptr; // [kRxVar][kRxMaxLv], Gershgorin partial maxima
  int32_t gblocks = 0;
  double* upart = nullptr;                   // [9][blocks of the finest up-sweep], r . z partials
};

// The end of a preconditioner application: z = 0 on the fixed unknowns
// (wall[i] == 2 for every component; wall[i] == 1 also for the off-diagonal
// components c != 0, 4, 8) and r . z per component, whose last block sets
// beta[c] = (first ? 0 : r.z / rz[c]), rz[c] = r.z and returns counter[c]
// to 0.
struct RxDot {
  const uint8_t* wall = nullptr;
  double* rz = nullptr;       // [9]
  double* beta = nullptr;     // [9]
  int32_t* counter = nullptr; // [9]
  int first = 0;
};

// Plans from the hierarchy of K (n unknowns, CSR rp / ci / kv), coarsest
// level at most 64 unknowns.
pdf_status relax_amg_setup(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                           const std::vector<double>& kv, RelaxAmg& G);
void relax_amg_free(RelaxAmg& G);
// The finest matrix values of variant v, on the relaxation pattern: filled
// by the caller before relax_amg_update.
inline double* relax_amg_level0(RelaxAmg& G, int v) { return G.lv.empty() ? G.c_v[v] : G.lv[0].a_v[v]; }
// The Galerkin matrices, smoother weights, Q and S of every level and the
// inverses of the coarsest matrices of the four variants, from the finest
// values (fixed unknowns with their diagonal only).
pdf_status relax_amg_update(RelaxAmg& G, cudaStream_t st);
// z = M^-1 r for the nine components ([9][n] each; component c uses
// variant 0, 1, 2 for c = 0, 4, 8 and 3 otherwise); components with
// active[c] = 0 and everything after *done are skipped.  The cycle runs in
// FP32 (the level matrices and vectors), r and z are FP64.
pdf_status relax_amg_apply(const RelaxAmg& G, const double* r, double* z, const int32_t* active,
                           const int32_t* done, const RxDot& dot, cudaStream_t st);

}  // namespace pdfgb

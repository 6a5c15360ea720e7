// Smoothed-aggregation algebraic multigrid for the pressure projection's
// Poisson matrix and for the elliptic relaxation (sec. 3.2 solves both by
// Jacobi-preconditioned conjugate gradients; a multigrid V-cycle as the
// preconditioner cuts the iterations from hundreds or thousands to tens
// while the solution stays that of the same linear system).  The Poisson
// matrix depends on the mesh only: its hierarchy is built once.  The
// relaxation matrices change with the statistics: the prolongations come
// once from the stiffness matrix, the level matrices are recomputed on the
// device at every solve (the second half of this file).
//
// Hierarchy (host, FP64, once): plain aggregation of the strongly connected
// unknowns (|a_ij| >= theta sqrt(a_ii a_jj)), tentative prolongation by the
// constant vector (the null space of the pure-Neumann matrix), smoothed
// prolongation P = (I - w_p D^-1 A) P_tent with w_p = 4 / (3 rho(D^-1 A)),
// Galerkin coarse matrices A_c = P^T A P, down to a dense coarsest matrix
// whose inverse (for a singular matrix with constant null space the
// regularised (A_c + mean(diag) 1 1^T / n_c)^-1, which solves every
// compatible right-hand side exactly) is applied directly.
//
// One V-cycle with one damped-Jacobi sweep (W = w_s D^-1) before and after
// the coarse correction is, per level,
//   M^-1 b = (2 W - W A W) b + Q M_c^-1 Q^T b,   Q = (I - W A) P,
// so the device runs two kernels per level: "down" (x = W b and
// b_c = Q^T b) and "up" (z = x + W (b - A x) + Q e_c), and one dense
// matrix-vector product on the coarsest level.  The cycle is symmetric, as
// the conjugate-gradient method needs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "amg.cuh"

namespace pdfgb {

namespace {

struct HCsr {
  int32_t n = 0, m = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
};

HCsr transpose(const HCsr& A) {
  HCsr T;
  T.n = A.m;
  T.m = A.n;
  T.rp.assign(T.n + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int32_t i = 0; i < T.n; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int32_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int32_t i = 0; i < A.n; ++i)
    for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      const int32_t d = fill[A.ci[q]]++;
      T.ci[d] = i;
      T.v[d] = A.v[q];
    }
  return T;  // columns ascending within each row
}

// C = A B (Gustavson), columns sorted within each row.
HCsr multiply(const HCsr& A, const HCsr& B) {
  HCsr C;
  C.n = A.n;
  C.m = B.m;
  C.rp.assign(C.n + 1, 0);
  std::vector<int32_t> mark(B.m, -1);
  std::vector<double> acc(B.m, 0.0);
  std::vector<int32_t> cols;
  for (int32_t i = 0; i < A.n; ++i) {
    cols.clear();
    for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      const int32_t k = A.ci[q];
      const double a = A.v[q];
      for (int32_t t = B.rp[k]; t < B.rp[k + 1]; ++t) {
        const int32_t j = B.ci[t];
        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols.push_back(j); }
        acc[j] += a * B.v[t];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t j : cols) { C.ci.push_back(j); C.v.push_back(acc[j]); }
    C.rp[i + 1] = (int32_t)C.ci.size();
  }
  return C;
}

std::vector<double> diagonal(const HCsr& A) {
  std::vector<double> d(A.n, 0.0);
  for (int32_t i = 0; i < A.n; ++i)
    for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (A.ci[q] == i) d[i] = A.v[q];
  return d;
}

// Spectral radius of D^-1 A: power iteration from a fixed non-constant
// start, times a safety factor, capped by Gershgorin's bound.
double spectral_radius(const HCsr& A, const std::vector<double>& d) {
  double gersh = 0.0;
  for (int32_t i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q) s += std::fabs(A.v[q]);
    gersh = std::max(gersh, s / d[i]);
  }
  std::vector<double> x(A.n), y(A.n);
  for (int32_t i = 0; i < A.n; ++i) x[i] = 1.0 + (double)((i * 7919) % 101) / 101.0;
  double lam = 0.0;
  for (int it = 0; it < 60; ++it) {
    double nx = 0.0;
    for (int32_t i = 0; i < A.n; ++i) {
      double s = 0.0;
      for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q) s += A.v[q] * x[A.ci[q]];
      y[i] = s / d[i];
      nx += y[i] * y[i];
    }
    nx = std::sqrt(nx);
    if (!(nx > 0.0)) break;
    double xn = 0.0;
    for (int32_t i = 0; i < A.n; ++i) xn += x[i] * x[i];
    lam = nx / std::sqrt(xn);
    for (int32_t i = 0; i < A.n; ++i) x[i] = y[i] / nx;
  }
  return std::min(gersh, 1.1 * lam > 0.0 ? 1.1 * lam : gersh);
}

// Aggregates of strongly connected unknowns: seeds whose strong
// neighbourhood is free take it whole; leftovers join the aggregate they
// are most strongly connected to; what remains forms new aggregates.
std::vector<int32_t> aggregate(const HCsr& A, const std::vector<double>& d, double theta, int32_t* n_agg) {
  const int32_t n = A.n;
  auto strong = [&](int32_t i, int32_t q) {
    const int32_t j = A.ci[q];
    return j != i && std::fabs(A.v[q]) >= theta * std::sqrt(std::fabs(d[i] * d[j]));
  };
  std::vector<int32_t> agg(n, -1);
  int32_t na = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free_nb = true;
    for (int32_t q = A.rp[i]; q < A.rp[i + 1] && free_nb; ++q)
      if (strong(i, q) && agg[A.ci[q]] >= 0) free_nb = false;
    if (!free_nb) continue;
    agg[i] = na;
    for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (strong(i, q)) agg[A.ci[q]] = na;
    ++na;
  }
  std::vector<int32_t> agg2 = agg;
  for (int32_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    double best = 0.0;
    for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (strong(i, q) && agg[A.ci[q]] >= 0 && std::fabs(A.v[q]) > best) {
        best = std::fabs(A.v[q]);
        agg2[i] = agg[A.ci[q]];
      }
  }
  for (int32_t i = 0; i < n; ++i) {
    if (agg2[i] >= 0) continue;
    agg2[i] = na;
    for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (strong(i, q) && agg2[A.ci[q]] < 0) agg2[A.ci[q]] = na;
    ++na;
  }
  *n_agg = na;
  return agg2;
}

template <typename T>
pdf_status up(T** dst, const std::vector<T>& src) {
  if (src.empty()) { *dst = nullptr; return PDF_OK; }
  cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? PDF_OK : cuda_fail(e, "amg: upload");
}

pdf_status dev_vec(double** p, int64_t n) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(double) * std::max<int64_t>(n, 1));
  return e == cudaSuccess ? PDF_OK : cuda_fail(e, "amg: allocation");
}

}  // namespace

void amg_free(Amg& G) {
  for (AmgLevel& L : G.lv) {
    cudaFree(L.a_rp); cudaFree(L.a_ci); cudaFree(L.a_v); cudaFree(L.w);
    cudaFree(L.q_rp); cudaFree(L.q_ci); cudaFree(L.q_v);
    cudaFree(L.s_rp); cudaFree(L.s_ci); cudaFree(L.s_v);
    cudaFree(L.b); cudaFree(L.x); cudaFree(L.z);
  }
  cudaFree(G.cinv); cudaFree(G.cb); cudaFree(G.cz);
  G = Amg();
}

// The smoothed-aggregation hierarchy of A0 down to at most kCoarse
// unknowns: the level matrices As, prolongations Ps, Q = (I - W A) P and
// the smoother weights W of every level, and the coarsest matrix.
static pdf_status build_levels(HCsr A, int32_t kCoarse, std::vector<HCsr>& As, std::vector<HCsr>& Ps,
                               std::vector<HCsr>& Qs, std::vector<std::vector<double>>& Ws, HCsr& Afinal) {
  constexpr int32_t kMaxLevels = 12;
  double theta = 0.08;
  while (A.n > kCoarse && (int32_t)As.size() < kMaxLevels) {
    const std::vector<double> d = diagonal(A);
    for (double x : d)
      if (!(x > 0.0)) return fail(PDF_EINVAL, "amg: non-positive diagonal");
    int32_t na = 0;
    const std::vector<int32_t> agg = aggregate(A, d, theta, &na);
    if (na >= A.n || na < 1) break;
    const double rho = spectral_radius(A, d);
    const double wp = 4.0 / (3.0 * rho);
    // P = (I - wp D^-1 A) P_tent
    HCsr P;
    P.n = A.n;
    P.m = na;
    P.rp.assign(A.n + 1, 0);
    {
      std::vector<int32_t> mark(na, -1), cols;
      std::vector<double> acc(na, 0.0);
      for (int32_t i = 0; i < A.n; ++i) {
        cols.clear();
        auto add = [&](int32_t c, double x) {
          if (mark[c] != i) { mark[c] = i; acc[c] = 0.0; cols.push_back(c); }
          acc[c] += x;
        };
        add(agg[i], 1.0);
        for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q) add(agg[A.ci[q]], -wp * A.v[q] / d[i]);
        std::sort(cols.begin(), cols.end());
        for (int32_t c : cols) { P.ci.push_back(c); P.v.push_back(acc[c]); }
        P.rp[i + 1] = (int32_t)P.ci.size();
      }
    }
    const HCsr AP = multiply(A, P);
    HCsr Ac = multiply(transpose(P), AP);
    // smoother W = ws D^-1 and Q = P - W A P
    const double ws = 4.0 / (3.0 * rho);
    std::vector<double> W(A.n);
    for (int32_t i = 0; i < A.n; ++i) W[i] = ws / d[i];
    HCsr Q;
    Q.n = A.n;
    Q.m = na;
    Q.rp.assign(A.n + 1, 0);
    {
      std::vector<int32_t> mark(na, -1), cols;
      std::vector<double> acc(na, 0.0);
      for (int32_t i = 0; i < A.n; ++i) {
        cols.clear();
        auto add = [&](int32_t c, double x) {
          if (mark[c] != i) { mark[c] = i; acc[c] = 0.0; cols.push_back(c); }
          acc[c] += x;
        };
        for (int32_t q = P.rp[i]; q < P.rp[i + 1]; ++q) add(P.ci[q], P.v[q]);
        for (int32_t q = AP.rp[i]; q < AP.rp[i + 1]; ++q) add(AP.ci[q], -W[i] * AP.v[q]);
        std::sort(cols.begin(), cols.end());
        for (int32_t c : cols) { Q.ci.push_back(c); Q.v.push_back(acc[c]); }
        Q.rp[i + 1] = (int32_t)Q.ci.size();
      }
    }
    As.push_back(A);
    Ps.push_back(P);
    Qs.push_back(Q);
    Ws.push_back(W);
    A = std::move(Ac);
    theta *= 0.5;
  }
  Afinal = std::move(A);
  return PDF_OK;
}

pdf_status amg_setup(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                     const std::vector<double>& v, bool singular, Amg& G) {
  constexpr int32_t kCoarse = 256;
  HCsr A0;
  A0.n = A0.m = n;
  A0.rp = rp;
  A0.ci = ci;
  A0.v = v;
  std::vector<HCsr> As, Ps, Qs;
  std::vector<std::vector<double>> Ws;
  HCsr A;
  pdf_status bs = build_levels(A0, kCoarse, As, Ps, Qs, Ws, A);
  if (bs != PDF_OK) return bs;
  // coarsest: regularised dense inverse (Gauss-Jordan with partial pivoting)
  const int32_t nc = A.n;
  std::vector<double> B((size_t)nc * nc, 0.0), Inv((size_t)nc * nc, 0.0);
  double dmean = 0.0;
  for (int32_t i = 0; i < nc; ++i)
    for (int32_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      B[(size_t)i * nc + A.ci[q]] += A.v[q];
      if (A.ci[q] == i) dmean += A.v[q];
    }
  dmean = nc > 0 ? dmean / nc : 1.0;
  if (!(dmean > 0.0)) dmean = 1.0;
  if (singular)
    for (size_t k = 0; k < B.size(); ++k) B[k] += dmean / nc;
  for (int32_t i = 0; i < nc; ++i) Inv[(size_t)i * nc + i] = 1.0;
  for (int32_t c = 0; c < nc; ++c) {
    int32_t piv = c;
    for (int32_t r = c + 1; r < nc; ++r)
      if (std::fabs(B[(size_t)r * nc + c]) > std::fabs(B[(size_t)piv * nc + c])) piv = r;
    if (!(std::fabs(B[(size_t)piv * nc + c]) > 0.0)) return fail(PDF_EINVAL, "amg: singular coarse matrix");
    if (piv != c)
      for (int32_t k = 0; k < nc; ++k) {
        std::swap(B[(size_t)c * nc + k], B[(size_t)piv * nc + k]);
        std::swap(Inv[(size_t)c * nc + k], Inv[(size_t)piv * nc + k]);
      }
    const double s = 1.0 / B[(size_t)c * nc + c];
    for (int32_t k = 0; k < nc; ++k) { B[(size_t)c * nc + k] *= s; Inv[(size_t)c * nc + k] *= s; }
    for (int32_t r = 0; r < nc; ++r) {
      if (r == c) continue;
      const double f = B[(size_t)r * nc + c];
      if (f == 0.0) continue;
      for (int32_t k = 0; k < nc; ++k) {
        B[(size_t)r * nc + k] -= f * B[(size_t)c * nc + k];
        Inv[(size_t)r * nc + k] -= f * Inv[(size_t)c * nc + k];
      }
    }
  }
  // upload
  amg_free(G);
  pdf_status s = PDF_OK;
  for (size_t l = 0; l < As.size() && s == PDF_OK; ++l) {
    G.lv.emplace_back();
    AmgLevel& L = G.lv.back();
    L.n = As[l].n;
    L.nc = Qs[l].m;
    const HCsr S = transpose(Qs[l]);
    L.nnz_a = (int64_t)As[l].ci.size();
    L.nnz_q = (int64_t)Qs[l].ci.size();
    if ((s = up(&L.a_rp, As[l].rp)) != PDF_OK || (s = up(&L.a_ci, As[l].ci)) != PDF_OK ||
        (s = up(&L.a_v, As[l].v)) != PDF_OK || (s = up(&L.w, Ws[l])) != PDF_OK ||
        (s = up(&L.q_rp, Qs[l].rp)) != PDF_OK || (s = up(&L.q_ci, Qs[l].ci)) != PDF_OK ||
        (s = up(&L.q_v, Qs[l].v)) != PDF_OK || (s = up(&L.s_rp, S.rp)) != PDF_OK ||
        (s = up(&L.s_ci, S.ci)) != PDF_OK || (s = up(&L.s_v, S.v)) != PDF_OK)
      break;
    if (l > 0 && ((s = dev_vec(&L.b, L.n)) != PDF_OK || (s = dev_vec(&L.z, L.n)) != PDF_OK)) break;
    s = dev_vec(&L.x, L.n);
  }
  G.nc = nc;
  if (s == PDF_OK) s = up(&G.cinv, Inv);
  if (s == PDF_OK) s = dev_vec(&G.cb, nc);
  if (s == PDF_OK) s = dev_vec(&G.cz, nc);
  if (s != PDF_OK) amg_free(G);
  return s;
}

// ------------------------------------------------------------------ device

// Rows of the coarse levels hold tens to hundreds of entries: a group of
// kG lanes shares a row (strided over its entries, then a shuffle sum).
constexpr int kG = 8;

__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = kG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, kG);
  return v;
}

// x = W b on the level's rows (one thread per row); b_c = Q^T b on the
// coarse rows (kG lanes per row; blocks past the first nbx).  Skipped when
// *done is set.
__global__ void __launch_bounds__(256) k_amg_down(int32_t n, int32_t nc, int32_t nbx, const double* __restrict__ w,
                                                  const int32_t* __restrict__ s_rp, const int32_t* __restrict__ s_ci,
                                                  const double* __restrict__ s_v, const double* __restrict__ b,
                                                  double* __restrict__ x, double* __restrict__ bc,
                                                  const int32_t* __restrict__ done) {
  if (*done) return;
  if ((int32_t)blockIdx.x < nbx) {
    const int32_t i = blockIdx.x * 256 + threadIdx.x;
    if (i < n) x[i] = w[i] * b[i];
  } else {
    const int32_t J = ((blockIdx.x - nbx) * 256 + threadIdx.x) / kG, g = threadIdx.x % kG;
    double s = 0.0;
    if (J < nc)
      for (int32_t q = s_rp[J] + g; q < s_rp[J + 1]; q += kG) s += s_v[q] * b[s_ci[q]];
    s = group_sum(s);
    if (J < nc && g == 0) bc[J] = s;
  }
}

// Coarsest level: z = Inv b, one warp per row.
__global__ void __launch_bounds__(256) k_amg_coarse(int32_t nc, const double* __restrict__ inv,
                                                    const double* __restrict__ b, double* __restrict__ z,
                                                    const int32_t* __restrict__ done) {
  if (*done) return;
  const int32_t row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= nc) return;
  double s = 0.0;
  for (int32_t k = lane; k < nc; k += 32) s += inv[(int64_t)row * nc + k] * b[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) z[row] = s;
}

// z = x + W (b - A x) + Q e_c on the finest level (kF lanes per row), the
// block partials of b . z to part, and in the last block to finish their
// sum: *rz_old = *rz, *rz = sum (counter returns to 0).  More lanes per row
// shorten the gather chains but multiply the blocks, which costs more on
// this level's 10^5 rows than it saves, so one.
constexpr int kF = 1;

__global__ void __launch_bounds__(256) k_amg_up(int32_t n, const int32_t* __restrict__ a_rp,
                                                const int32_t* __restrict__ a_ci, const double* __restrict__ a_v,
                                                const double* __restrict__ w, const int32_t* __restrict__ q_rp,
                                                const int32_t* __restrict__ q_ci, const double* __restrict__ q_v,
                                                const double* __restrict__ b, const double* __restrict__ x,
                                                const double* __restrict__ ec, double* __restrict__ z,
                                                double* __restrict__ part, int32_t* __restrict__ counter,
                                                double* __restrict__ rz, double* __restrict__ rz_old,
                                                const int32_t* __restrict__ done) {
  if (*done) return;
  const int32_t i = (blockIdx.x * 256 + threadIdx.x) / kF, g = threadIdx.x % kF;
  double ax = 0.0, qe = 0.0;
  if (i < n) {
    for (int32_t q = a_rp[i] + g; q < a_rp[i + 1]; q += kF) ax += a_v[q] * x[a_ci[q]];
    for (int32_t q = q_rp[i] + g; q < q_rp[i + 1]; q += kF) qe += q_v[q] * ec[q_ci[q]];
  }
#pragma unroll
  for (int o = kF / 2; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o, kF);
    qe += __shfl_xor_sync(0xffffffffu, qe, o, kF);
  }
  double bz = 0.0;
  if (i < n && g == 0) {
    const double bi = b[i];
    const double zi = x[i] + w[i] * (bi - ax) + qe;
    z[i] = zi;
    bz = bi * zi;
  }
  __shared__ double sh[8];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bz += __shfl_xor_sync(0xffffffffu, bz, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = bz;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += sh[k];
    part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(counter, 1) == (int32_t)gridDim.x - 1;
    if (last) *counter = 0;
  }
  __syncthreads();
  if (!last) return;
  double t = 0.0;
  for (int32_t k = threadIdx.x; k < (int32_t)gridDim.x; k += 256) t += __ldcg(part + k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < 8; ++k) v += sh[k];
    *rz_old = *rz;
    *rz = v;
  }
}

// The same with kG lanes per row (coarse levels, no partials).
__global__ void __launch_bounds__(256) k_amg_up_g(int32_t n, const int32_t* __restrict__ a_rp,
                                                  const int32_t* __restrict__ a_ci, const double* __restrict__ a_v,
                                                  const double* __restrict__ w, const int32_t* __restrict__ q_rp,
                                                  const int32_t* __restrict__ q_ci, const double* __restrict__ q_v,
                                                  const double* __restrict__ b, const double* __restrict__ x,
                                                  const double* __restrict__ ec, double* __restrict__ z,
                                                  const int32_t* __restrict__ done) {
  if (*done) return;
  const int32_t i = (blockIdx.x * 256 + threadIdx.x) / kG, g = threadIdx.x % kG;
  double ax = 0.0, qe = 0.0;
  if (i < n) {
    for (int32_t q = a_rp[i] + g; q < a_rp[i + 1]; q += kG) ax += a_v[q] * x[a_ci[q]];
    for (int32_t q = q_rp[i] + g; q < q_rp[i + 1]; q += kG) qe += q_v[q] * ec[q_ci[q]];
  }
  ax = group_sum(ax);
  qe = group_sum(qe);
  if (i < n && g == 0) z[i] = x[i] + w[i] * (b[i] - ax) + qe;
}

pdf_status amg_apply(const Amg& G, const double* r, double* z, double* part, int32_t* counter, double* rz,
                     double* rz_old, const int32_t* done, cudaStream_t st) {
  const int32_t L = (int32_t)G.lv.size();
  // down: level l's right-hand side is r (l = 0) or lv[l].b
  for (int32_t l = 0; l < L; ++l) {
    const AmgLevel& V = G.lv[l];
    const double* b = l == 0 ? r : V.b;
    double* bc = l + 1 < L ? G.lv[l + 1].b : G.cb;
    const int32_t nbx = (V.n + 255) / 256, nbc = (int32_t)(((int64_t)V.nc * kG + 255) / 256);
    PDF_KERNEL("k_amg_down", st, k_amg_down<<<nbx + nbc, 256, 0, st>>>(V.n, V.nc, nbx, V.w, V.s_rp, V.s_ci, V.s_v, b,
                                                                        V.x, bc, done));
  }
  if (L == 0) {
    PDF_KERNEL("k_amg_coarse", st, k_amg_coarse<<<(G.nc + 7) / 8, 256, 0, st>>>(G.nc, G.cinv, r, z, done));
    return PDF_OK;
  }
  PDF_KERNEL("k_amg_coarse", st, k_amg_coarse<<<(G.nc + 7) / 8, 256, 0, st>>>(G.nc, G.cinv, G.cb, G.cz, done));
  for (int32_t l = L - 1; l >= 0; --l) {
    const AmgLevel& V = G.lv[l];
    const double* b = l == 0 ? r : V.b;
    const double* ec = l + 1 < L ? G.lv[l + 1].z : G.cz;
    double* out = l == 0 ? z : V.z;
    if (l == 0)
      PDF_KERNEL("k_amg_up", st, k_amg_up<<<(int32_t)(((int64_t)V.n * kF + 255) / 256), 256, 0, st>>>(
                                     V.n, V.a_rp, V.a_ci, V.a_v, V.w, V.q_rp, V.q_ci, V.q_v, b, V.x, ec, out, part,
                                     counter, rz, rz_old, done));
    else
      PDF_KERNEL("k_amg_up", st, k_amg_up_g<<<(int32_t)(((int64_t)V.n * kG + 255) / 256), 256, 0, st>>>(
                                     V.n, V.a_rp, V.a_ci, V.a_v, V.w, V.q_rp, V.q_ci, V.q_v, b, V.x, ec, out, done));
  }
  return PDF_OK;
}

// ------------------------------------------------------------- persistent PCG

constexpr int kMaxLv = 12;

struct PcgLevel {
  int32_t n, nc;
  const int32_t *a_rp, *a_ci, *q_rp, *q_ci, *s_rp, *s_ci;
  const double *a_v, *w, *q_v, *s_v;
  double *b, *x, *z;
};

struct PcgArgs {
  int32_t n, L, nc;
  const int32_t *rp, *ci;
  const double* val;
  double *x, *r, *z, *p, *q, *scal, *part;
  int32_t* ctl;
  const double* cinv;
  double *cb, *cz;
  PcgLevel lv[kMaxLv];
};

// Sum over the block of v; the result in every thread.
__device__ __forceinline__ double block_sum_all(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += sh[i];
  __syncthreads();
  return t;
}

// Sum of the grid's block partials, in block order: identical in every block.
__device__ __forceinline__ double grid_total(const double* part, double* sh) {
  double t = 0.0;
  for (int32_t i = threadIdx.x; i < (int32_t)gridDim.x; i += 256) t += __ldcg(part + i);
  return block_sum_all(t, sh);
}

__global__ void __launch_bounds__(256) k_amg_pcg(PcgArgs A) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[8];
  const int32_t tid = blockIdx.x * 256 + threadIdx.x, nthr = gridDim.x * 256;
  const int32_t gl = tid / kG, lane_g = threadIdx.x % kG, ngrp = nthr / kG;
  double* part0 = A.part;
  double* part1 = A.part + gridDim.x;
  double* part2 = A.part + 2 * gridDim.x;
  int32_t it = A.ctl[kPcgIters];
  const int32_t max_it = A.ctl[kPcgMaxIt];
  bool done = A.ctl[kPcgDone] != 0;
  double rz = A.scal[kPcgRz], rz_old = A.scal[kPcgRzOld], rr = A.scal[kPcgRr], pq = 0.0;
  const double tol2 = A.scal[kPcgTol2];
  while (!done) {
    // z = M^-1 r: down the levels
    for (int l = 0; l < A.L; ++l) {
      const PcgLevel& V = A.lv[l];
      const double* b = l == 0 ? A.r : V.b;
      double* bc = l + 1 < A.L ? A.lv[l + 1].b : A.cb;
      for (int32_t i = tid; i < V.n; i += nthr) V.x[i] = V.w[i] * b[i];
      for (int32_t J0 = 0; J0 < V.nc; J0 += ngrp) {
        const int32_t J = J0 + gl;
        double s = 0.0;
        if (J < V.nc)
          for (int32_t k = V.s_rp[J] + lane_g; k < V.s_rp[J + 1]; k += kG) s += V.s_v[k] * b[V.s_ci[k]];
#pragma unroll
        for (int o = kG / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, kG);
        if (J < V.nc && lane_g == 0) bc[J] = s;
      }
      grid.sync();
    }
    // coarsest level, one warp per row
    {
      const double* b = A.L > 0 ? A.cb : A.r;
      double* zc = A.L > 0 ? A.cz : A.z;
      const int32_t w = tid >> 5, lane = threadIdx.x & 31, nw = nthr >> 5;
      for (int32_t row0 = 0; row0 < A.nc; row0 += nw) {
        const int32_t row = row0 + w;
        double s = 0.0;
        if (row < A.nc)
          for (int32_t k = lane; k < A.nc; k += 32) s += A.cinv[(int64_t)row * A.nc + k] * b[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (row < A.nc && lane == 0) zc[row] = s;
      }
      grid.sync();
    }
    // up the levels; the finest one also gives r . z
    double bz = 0.0;
    for (int l = A.L - 1; l >= 0; --l) {
      const PcgLevel& V = A.lv[l];
      const double* b = l == 0 ? A.r : V.b;
      const double* ec = l + 1 < A.L ? A.lv[l + 1].z : A.cz;
      double* out = l == 0 ? A.z : V.z;
      if (l == 0) {
        for (int32_t i = tid; i < V.n; i += nthr) {
          double ax = 0.0, qe = 0.0;
          for (int32_t k = V.a_rp[i]; k < V.a_rp[i + 1]; ++k) ax += V.a_v[k] * V.x[V.a_ci[k]];
          for (int32_t k = V.q_rp[i]; k < V.q_rp[i + 1]; ++k) qe += V.q_v[k] * ec[V.q_ci[k]];
          const double zi = V.x[i] + V.w[i] * (b[i] - ax) + qe;
          out[i] = zi;
          bz += b[i] * zi;
        }
      } else {
        for (int32_t i0 = 0; i0 < V.n; i0 += ngrp) {
          const int32_t i = i0 + gl;
          double ax = 0.0, qe = 0.0;
          if (i < V.n) {
            for (int32_t k = V.a_rp[i] + lane_g; k < V.a_rp[i + 1]; k += kG) ax += V.a_v[k] * V.x[V.a_ci[k]];
            for (int32_t k = V.q_rp[i] + lane_g; k < V.q_rp[i + 1]; k += kG) qe += V.q_v[k] * ec[V.q_ci[k]];
          }
#pragma unroll
          for (int o = kG / 2; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o, kG);
            qe += __shfl_xor_sync(0xffffffffu, qe, o, kG);
          }
          if (i < V.n && lane_g == 0) out[i] = V.x[i] + V.w[i] * (b[i] - ax) + qe;
        }
      }
      if (l > 0) grid.sync();
    }
    if (A.L == 0)
      for (int32_t i = tid; i < A.n; i += nthr) bz += A.r[i] * A.z[i];
    {
      const double t = block_sum_all(bz, sh);
      if (threadIdx.x == 0) part0[blockIdx.x] = t;
    }
    grid.sync();
    // beta; p = z + beta p and q = K z + beta q (= K p by the recurrence,
    // so no barrier between them); p . q
    rz_old = rz;
    rz = grid_total(part0, sh);
    const double beta = rz_old != 0.0 ? rz / rz_old : 0.0;
    double s_pq = 0.0;
    for (int32_t i = tid; i < A.n; i += nthr) {
      double kz = 0.0;
      for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) kz += A.val[k] * A.z[A.ci[k]];
      const double pv = A.z[i] + beta * A.p[i];
      const double qv = kz + beta * A.q[i];
      A.p[i] = pv;
      A.q[i] = qv;
      s_pq += pv * qv;
    }
    {
      const double t = block_sum_all(s_pq, sh);
      if (threadIdx.x == 0) part1[blockIdx.x] = t;
    }
    grid.sync();
    pq = grid_total(part1, sh);
    const double alpha = pq > 0.0 ? rz / pq : 0.0;
    double s_rr = 0.0;
    for (int32_t i = tid; i < A.n; i += nthr) {
      A.x[i] += alpha * A.p[i];
      const double rv = A.r[i] - alpha * A.q[i];
      A.r[i] = rv;
      s_rr += rv * rv;
    }
    {
      const double t = block_sum_all(s_rr, sh);
      if (threadIdx.x == 0) part2[blockIdx.x] = t;
    }
    grid.sync();
    rr = grid_total(part2, sh);
    ++it;
    done = rr <= tol2 || it >= max_it || !(pq > 0.0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.scal[kPcgRr] = rr;
    A.scal[kPcgRz] = rz;
    A.scal[kPcgRzOld] = rz_old;
    A.scal[kPcgPq] = pq;
    A.ctl[kPcgIters] = it;
    A.ctl[kPcgDone] = 1;
  }
}

pdf_status amg_pcg(const Amg& G, int32_t n, const int32_t* rp, const int32_t* ci, const double* val, double* x,
                   double* r, double* z, double* p, double* q, double* scal, int32_t* ctl, double* part,
                   int32_t part_cap, cudaStream_t st) {
  if ((int)G.lv.size() > kMaxLv) return fail(PDF_EINVAL, "amg_pcg: too many levels");
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  PDF_CUDA(cudaGetDevice(&dev));
  PDF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  PDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_amg_pcg, 256, 0));
  if (!coop || per_sm < 1) return fail(PDF_EINVAL, "amg_pcg: no cooperative launch");
  // at most one row per thread on the finest level, at most the resident grid
  int blocks = std::min<int64_t>((int64_t)sms * per_sm, ((int64_t)n + 255) / 256);
  blocks = std::max(1, std::min(blocks, part_cap / 3));
  PcgArgs A;
  std::memset(&A, 0, sizeof(A));
  A.n = n;
  A.L = (int32_t)G.lv.size();
  A.nc = G.nc;
  A.rp = rp; A.ci = ci; A.val = val;
  A.x = x; A.r = r; A.z = z; A.p = p; A.q = q; A.scal = scal; A.part = part; A.ctl = ctl;
  A.cinv = G.cinv; A.cb = G.cb; A.cz = G.cz;
  for (int l = 0; l < A.L; ++l) {
    const AmgLevel& V = G.lv[l];
    A.lv[l] = PcgLevel{V.n, V.nc, V.a_rp, V.a_ci, V.q_rp, V.q_ci, V.s_rp, V.s_ci,
                       V.a_v, V.w, V.q_v, V.s_v, V.b, V.x, V.z};
  }
  void* args[] = {&A};
  cudaError_t le = cudaSuccess;
  PDF_KERNEL("k_amg_pcg", st,
             le = cudaLaunchCooperativeKernel((const void*)k_amg_pcg, dim3(blocks), dim3(256), args, 0, st));
  if (le != cudaSuccess) return cuda_fail(le, "amg_pcg: cooperative launch");
  return PDF_OK;
}

// ------------------------------------------------------- relaxation multigrid

namespace {

template <typename T>
pdf_status up_vec(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(src.size(), 1) * sizeof(T));
  if (e == cudaSuccess && !src.empty())
    e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? PDF_OK : cuda_fail(e, "relax multigrid: upload");
}

template <typename T>
pdf_status zeros(T** p, int64_t n) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<int64_t>(n, 1));
  if (e == cudaSuccess) e = cudaMemset(*p, 0, sizeof(T) * std::max<int64_t>(n, 1));
  return e == cudaSuccess ? PDF_OK : cuda_fail(e, "relax multigrid: allocation");
}

}  // namespace

void relax_amg_free(RelaxAmg& G) {
  for (RxLevel& L : G.lv) {
    cudaFree(L.a_rp); cudaFree(L.a_ci); cudaFree(L.a_dpos); cudaFree(L.q_rp); cudaFree(L.q_ci);
    cudaFree(L.s_rp); cudaFree(L.s_ci); cudaFree(L.s_perm); cudaFree(L.ap_off); cudaFree(L.ap_qa);
    cudaFree(L.ap_pv); cudaFree(L.c_off); cudaFree(L.c_tap); cudaFree(L.c_pv); cudaFree(L.q_pin);
    cudaFree(L.q_row); cudaFree(L.b); cudaFree(L.x); cudaFree(L.z);
    for (int v = 0; v < kRxVar; ++v) {
      cudaFree(L.a_v[v]); cudaFree(L.ap_v[v]); cudaFree(L.q_v[v]); cudaFree(L.s_v[v]);
      cudaFree(L.a_f[v]); cudaFree(L.q_f[v]); cudaFree(L.s_f[v]); cudaFree(L.w_f[v]); cudaFree(L.w_v[v]);
    }
  }
  cudaFree(G.c_rp); cudaFree(G.c_ci);
  for (int v = 0; v < kRxVar; ++v) cudaFree(G.c_v[v]);
  cudaFree(G.cmat); cudaFree(G.cinv); cudaFree(G.cb); cudaFree(G.cz); cudaFree(G.omega); cudaFree(G.gpart);
  cudaFree(G.upart);
  G = RelaxAmg();
}

pdf_status relax_amg_setup(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                           const std::vector<double>& kv, RelaxAmg& G) {
  HCsr K;
  K.n = K.m = n;
  K.rp = rp;
  K.ci = ci;
  K.v = kv;
  std::vector<HCsr> As, Ps, Qs;
  std::vector<std::vector<double>> Ws;
  HCsr Afinal;
  pdf_status s = build_levels(K, 64, As, Ps, Qs, Ws, Afinal);
  if (s != PDF_OK) return s;
  if ((int)As.size() > kRxMaxLv) return fail(PDF_EINVAL, "relax multigrid: too many levels");
  relax_amg_free(G);
  // the pattern of every level's matrix follows from the plans: level 0 is
  // the relaxation pattern, level l + 1 that of P_l^T (A_l P_l)
  std::vector<int32_t> a_rp = rp, a_ci = ci;
  int32_t na = n;
  for (size_t l = 0; l < As.size() && s == PDF_OK; ++l) {
    const HCsr& P = Ps[l];
    G.lv.emplace_back();
    RxLevel& L = G.lv.back();
    L.n = na;
    L.nc = P.m;
    L.nnz_a = (int64_t)a_ci.size();
    // diagonal positions
    std::vector<int32_t> dpos(na, -1);
    for (int32_t i = 0; i < na; ++i)
      for (int32_t q = a_rp[i]; q < a_rp[i + 1]; ++q)
        if (a_ci[q] == i) dpos[i] = q;
    for (int32_t i = 0; i < na; ++i)
      if (dpos[i] < 0) return fail(PDF_EINVAL, "relax multigrid: missing diagonal");
    // plan of A P: per row, the (A entry, P value) pairs of each column
    std::vector<int32_t> q_rp(na + 1, 0), q_ci, ap_off(1, 0), ap_qa, q_row;
    std::vector<double> ap_pv, q_pin;
    {
      std::vector<int32_t> mark(P.m, -1), cols;
      std::vector<std::vector<std::pair<int32_t, double>>> lists(P.m);
      for (int32_t i = 0; i < na; ++i) {
        cols.clear();
        for (int32_t q = a_rp[i]; q < a_rp[i + 1]; ++q) {
          const int32_t j = a_ci[q];
          for (int32_t t = P.rp[j]; t < P.rp[j + 1]; ++t) {
            const int32_t J = P.ci[t];
            if (mark[J] != i) { mark[J] = i; lists[J].clear(); cols.push_back(J); }
            lists[J].push_back({q, P.v[t]});
          }
        }
        std::sort(cols.begin(), cols.end());
        for (int32_t J : cols) {
          q_ci.push_back(J);
          q_row.push_back(i);
          for (auto& pr : lists[J]) { ap_qa.push_back(pr.first); ap_pv.push_back(pr.second); }
          ap_off.push_back((int32_t)ap_qa.size());
          double pin = 0.0;
          for (int32_t t = P.rp[i]; t < P.rp[i + 1]; ++t)
            if (P.ci[t] == J) pin = P.v[t];
          q_pin.push_back(pin);
        }
        q_rp[i + 1] = (int32_t)q_ci.size();
      }
    }
    const int64_t nap = (int64_t)q_ci.size();
    L.nnz_ap = nap;
    // S = Q^T with the permutation of the entries
    std::vector<int32_t> s_rp(P.m + 1, 0), s_ci(nap), s_perm(nap);
    for (int64_t t = 0; t < nap; ++t) s_rp[q_ci[t] + 1]++;
    for (int32_t J = 0; J < P.m; ++J) s_rp[J + 1] += s_rp[J];
    {
      std::vector<int32_t> fill(s_rp.begin(), s_rp.end() - 1);
      for (int32_t i = 0; i < na; ++i)
        for (int32_t t = q_rp[i]; t < q_rp[i + 1]; ++t) {
          const int32_t d = fill[q_ci[t]]++;
          s_ci[d] = i;
          s_perm[d] = t;
        }
    }
    // plan of the next matrix, P^T (A P): coarse entry (I, J) sums P_iI (A P)_iJ
    std::vector<int32_t> n_rp(P.m + 1, 0), n_ci, c_off(1, 0), c_tap;
    std::vector<double> c_pv;
    {
      // transpose of P for the rows of the coarse matrix
      std::vector<int32_t> pt_rp(P.m + 1, 0), pt_i(P.ci.size());
      std::vector<double> pt_v(P.ci.size());
      for (int32_t c : P.ci) pt_rp[c + 1]++;
      for (int32_t I = 0; I < P.m; ++I) pt_rp[I + 1] += pt_rp[I];
      std::vector<int32_t> fill(pt_rp.begin(), pt_rp.end() - 1);
      for (int32_t i = 0; i < na; ++i)
        for (int32_t t = P.rp[i]; t < P.rp[i + 1]; ++t) {
          const int32_t d = fill[P.ci[t]]++;
          pt_i[d] = i;
          pt_v[d] = P.v[t];
        }
      std::vector<int32_t> mark(P.m, -1), cols;
      std::vector<std::vector<std::pair<int32_t, double>>> lists(P.m);
      for (int32_t I = 0; I < P.m; ++I) {
        cols.clear();
        for (int32_t k = pt_rp[I]; k < pt_rp[I + 1]; ++k) {
          const int32_t i = pt_i[k];
          for (int32_t t = q_rp[i]; t < q_rp[i + 1]; ++t) {
            const int32_t J = q_ci[t];
            if (mark[J] != I) { mark[J] = I; lists[J].clear(); cols.push_back(J); }
            lists[J].push_back({t, pt_v[k]});
          }
        }
        std::sort(cols.begin(), cols.end());
        for (int32_t J : cols) {
          n_ci.push_back(J);
          for (auto& pr : lists[J]) { c_tap.push_back(pr.first); c_pv.push_back(pr.second); }
          c_off.push_back((int32_t)c_tap.size());
        }
        n_rp[I + 1] = (int32_t)n_ci.size();
      }
    }
    if ((s = up_vec(&L.a_rp, a_rp)) != PDF_OK || (s = up_vec(&L.a_ci, a_ci)) != PDF_OK ||
        (s = up_vec(&L.a_dpos, dpos)) != PDF_OK || (s = up_vec(&L.q_rp, q_rp)) != PDF_OK ||
        (s = up_vec(&L.q_ci, q_ci)) != PDF_OK || (s = up_vec(&L.s_rp, s_rp)) != PDF_OK ||
        (s = up_vec(&L.s_ci, s_ci)) != PDF_OK || (s = up_vec(&L.s_perm, s_perm)) != PDF_OK ||
        (s = up_vec(&L.ap_off, ap_off)) != PDF_OK || (s = up_vec(&L.ap_qa, ap_qa)) != PDF_OK ||
        (s = up_vec(&L.ap_pv, ap_pv)) != PDF_OK || (s = up_vec(&L.c_off, c_off)) != PDF_OK ||
        (s = up_vec(&L.c_tap, c_tap)) != PDF_OK || (s = up_vec(&L.c_pv, c_pv)) != PDF_OK ||
        (s = up_vec(&L.q_pin, q_pin)) != PDF_OK || (s = up_vec(&L.q_row, q_row)) != PDF_OK)
      break;
    for (int v = 0; v < kRxVar && s == PDF_OK; ++v)
      if ((s = zeros(&L.a_v[v], L.nnz_a)) != PDF_OK || (s = zeros(&L.ap_v[v], nap)) != PDF_OK ||
          (s = zeros(&L.q_v[v], nap)) != PDF_OK || (s = zeros(&L.s_v[v], nap)) != PDF_OK ||
          (s = zeros(&L.a_f[v], L.nnz_a)) != PDF_OK || (s = zeros(&L.q_f[v], nap)) != PDF_OK ||
          (s = zeros(&L.s_f[v], nap)) != PDF_OK || (s = zeros(&L.w_f[v], (int64_t)na)) != PDF_OK ||
          (s = zeros(&L.w_v[v], (int64_t)na)) != PDF_OK)
        break;
    if (s != PDF_OK) break;
    if ((s = zeros(&L.x, 9 * (int64_t)na)) != PDF_OK) break;
    if (l > 0 && ((s = zeros(&L.b, 9 * (int64_t)na)) != PDF_OK || (s = zeros(&L.z, 9 * (int64_t)na)) != PDF_OK))
      break;
    a_rp = n_rp;
    a_ci = n_ci;
    na = P.m;
  }
  if (s == PDF_OK && na > 64) s = fail(PDF_EINVAL, "relax multigrid: coarsest level above 64 unknowns");
  if (s == PDF_OK) {
    G.nc = na;
    G.nnz_c = (int64_t)a_ci.size();
    s = up_vec(&G.c_rp, a_rp);
    if (s == PDF_OK) s = up_vec(&G.c_ci, a_ci);
    for (int v = 0; v < kRxVar && s == PDF_OK; ++v) s = zeros(&G.c_v[v], G.nnz_c);
    if (s == PDF_OK) s = zeros(&G.cmat, (int64_t)kRxVar * na * 2 * na);
    if (s == PDF_OK) s = zeros(&G.cinv, (int64_t)kRxVar * na * na);
    if (s == PDF_OK) s = zeros(&G.cb, 9 * (int64_t)na);
    if (s == PDF_OK) s = zeros(&G.cz, 9 * (int64_t)na);
    if (s == PDF_OK) s = zeros(&G.omega, kRxVar * kRxMaxLv);
    G.gblocks = (int32_t)std::min<int64_t>(1024, ((int64_t)n + 255) / 256);
    if (s == PDF_OK) s = zeros(&G.gpart, (int64_t)kRxVar * G.gblocks);
    if (s == PDF_OK) s = zeros(&G.upart, 9 * (((int64_t)n + 255) / 256));
  }
  if (s != PDF_OK) relax_amg_free(G);
  return s;
}

// Per-variant pointers of one level, for the kernels.
struct RxVals {
  const double* a[kRxVar];
  double* ap[kRxVar];
  double* q[kRxVar];
  double* s[kRxVar];
  double* an[kRxVar];  // the next level's matrix values
  float *af[kRxVar], *qf[kRxVar], *sf[kRxVar], *wf[kRxVar];
  double* w[kRxVar];
};

// (A P)[t] for the four variants (each thread all four: the plan's indices
// are loaded once).
__global__ void k_rx_ap(int64_t nnz_ap, const int32_t* __restrict__ off, const int32_t* __restrict__ qa,
                        const double* __restrict__ pv, RxVals V) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz_ap; t += (int64_t)gridDim.x * blockDim.x) {
    double s[kRxVar] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t k = off[t]; k < off[t + 1]; ++k) {
      const int32_t q = qa[k];
      const double w = pv[k];
#pragma unroll
      for (int v = 0; v < kRxVar; ++v) s[v] += V.a[v][q] * w;
    }
#pragma unroll
    for (int v = 0; v < kRxVar; ++v) V.ap[v][t] = s[v];
  }
}

// Gershgorin bound of D^-1 A per variant: block partial maxima.
__global__ void __launch_bounds__(256) k_rx_gersh(int32_t n, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ dpos, RxVals V,
                                                  double* __restrict__ part) {
  const int v = blockIdx.y;
  const double* a = V.a[v];
  double m = 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) s += fabs(a[q]);
    m = fmax(m, s / a[dpos[i]]);
  }
  __shared__ double sh[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t = fmax(t, sh[k]);
    part[(int64_t)v * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_rx_omega(const double* __restrict__ part, int32_t nb, int level, double* __restrict__ omega) {
  const int v = threadIdx.x;
  if (v >= kRxVar) return;
  double m = 0.0;
  for (int32_t b = 0; b < nb; ++b) m = fmax(m, part[(int64_t)v * nb + b]);
  omega[v * kRxMaxLv + level] = m > 0.0 ? 4.0 / (3.0 * m) : 0.0;
}

// The smoother weights W = omega / a_ii (FP64 and FP32) and the FP32 copy
// of the level matrix.
__global__ void k_rx_cast(int32_t n, int64_t nnz_a, const int32_t* __restrict__ dpos,
                          const double* __restrict__ omega, int level, RxVals V) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz_a; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = t < n ? dpos[t] : 0;
#pragma unroll
    for (int v = 0; v < kRxVar; ++v) {
      V.af[v][t] = (float)V.a[v][t];
      if (t < n) {
        const double w = omega[v * kRxMaxLv + level] / V.a[v][d];
        V.w[v][t] = w;
        V.wf[v][t] = (float)w;
      }
    }
  }
}

// Q = P - W (A P); S = Q^T; the next level's matrix.
__global__ void k_rx_q(int64_t nnz_ap, const double* __restrict__ pin, const int32_t* __restrict__ row, RxVals V) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz_ap; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = row[t];
    const double p = pin[t];
#pragma unroll
    for (int v = 0; v < kRxVar; ++v) {
      const double q = p - V.w[v][i] * V.ap[v][t];
      V.q[v][t] = q;
      V.qf[v][t] = (float)q;
    }
  }
}

__global__ void k_rx_s(int64_t nnz_ap, const int32_t* __restrict__ perm, RxVals V) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz_ap; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = perm[t];
#pragma unroll
    for (int v = 0; v < kRxVar; ++v) {
      const double q = V.q[v][k];
      V.s[v][t] = q;
      V.sf[v][t] = (float)q;
    }
  }
}

__global__ void k_rx_next(int64_t nnz_n, const int32_t* __restrict__ off, const int32_t* __restrict__ tap,
                          const double* __restrict__ pv, RxVals V) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nnz_n; c += (int64_t)gridDim.x * blockDim.x) {
    double s[kRxVar] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t k = off[c]; k < off[c + 1]; ++k) {
      const int32_t q = tap[k];
      const double w = pv[k];
#pragma unroll
      for (int v = 0; v < kRxVar; ++v) s[v] += V.ap[v][q] * w;
    }
#pragma unroll
    for (int v = 0; v < kRxVar; ++v) V.an[v][c] = s[v];
  }
}

// Inverse of the coarsest matrix per variant (blockIdx.x): Gauss-Jordan on
// [A | I] without pivoting (the matrices are symmetric positive definite).
__global__ void __launch_bounds__(256) k_rx_coarse_inv(int32_t nc, const int32_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, RxVals V,
                                                       double* __restrict__ cmat, float* __restrict__ cinv) {
  const int v = blockIdx.x;
  const int w2 = 2 * nc;
  double* M = cmat + (int64_t)v * nc * w2;
  for (int32_t k = threadIdx.x; k < nc * w2; k += blockDim.x) M[k] = 0.0;
  __syncthreads();
  for (int32_t i = threadIdx.x; i < nc; i += blockDim.x) {
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) M[(int64_t)i * w2 + ci[q]] = V.an[v][q];
    M[(int64_t)i * w2 + nc + i] = 1.0;
  }
  __syncthreads();
  __shared__ double f[64];
  for (int32_t c = 0; c < nc; ++c) {
    const double piv = M[(int64_t)c * w2 + c];
    __syncthreads();
    for (int32_t k = threadIdx.x; k < w2; k += blockDim.x) M[(int64_t)c * w2 + k] /= piv;
    for (int32_t r = threadIdx.x; r < nc; r += blockDim.x) f[r] = r == c ? 0.0 : M[(int64_t)r * w2 + c];
    __syncthreads();
    for (int32_t k = threadIdx.x; k < nc * w2; k += blockDim.x) {
      const int32_t r = k / w2, col = k - r * w2;
      if (r != c) M[k] -= f[r] * M[(int64_t)c * w2 + col];
    }
    __syncthreads();
  }
  for (int32_t k = threadIdx.x; k < nc * nc; k += blockDim.x) {
    const int32_t i = k / nc, j = k - i * nc;
    // symmetric part (the exact inverse is symmetric)
    cinv[(int64_t)v * nc * nc + k] = (float)(0.5 * (M[(int64_t)i * w2 + nc + j] + M[(int64_t)j * w2 + nc + i]));
  }
}

static int rx_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

pdf_status relax_amg_update(RelaxAmg& G, cudaStream_t st) {
  const int L = (int)G.lv.size();
  for (int l = 0; l < L; ++l) {
    RxLevel& V = G.lv[l];
    RxVals R;
    for (int v = 0; v < kRxVar; ++v) {
      R.a[v] = V.a_v[v];
      R.ap[v] = V.ap_v[v];
      R.q[v] = V.q_v[v];
      R.s[v] = V.s_v[v];
      R.an[v] = l + 1 < L ? G.lv[l + 1].a_v[v] : G.c_v[v];
      R.af[v] = V.a_f[v];
      R.qf[v] = V.q_f[v];
      R.sf[v] = V.s_f[v];
      R.wf[v] = V.w_f[v];
      R.w[v] = V.w_v[v];
    }
    const int64_t nnz_n = l + 1 < L ? G.lv[l + 1].nnz_a : G.nnz_c;
    PDF_KERNEL("k_rx_ap", st, k_rx_ap<<<rx_blocks(V.nnz_ap), 256, 0, st>>>(V.nnz_ap, V.ap_off, V.ap_qa, V.ap_pv, R));
    const int gb = std::min<int>(G.gblocks, rx_blocks(V.n));
    PDF_KERNEL("k_rx_gersh", st, k_rx_gersh<<<dim3(gb, kRxVar), 256, 0, st>>>(V.n, V.a_rp, V.a_dpos, R, G.gpart));
    PDF_KERNEL("k_rx_omega", st, k_rx_omega<<<1, 32, 0, st>>>(G.gpart, gb, l, G.omega));
    PDF_KERNEL("k_rx_cast", st, k_rx_cast<<<rx_blocks(V.nnz_a), 256, 0, st>>>(V.n, V.nnz_a, V.a_dpos, G.omega, l, R));
    PDF_KERNEL("k_rx_q", st, k_rx_q<<<rx_blocks(V.nnz_ap), 256, 0, st>>>(V.nnz_ap, V.q_pin, V.q_row, R));
    PDF_KERNEL("k_rx_s", st, k_rx_s<<<rx_blocks(V.nnz_ap), 256, 0, st>>>(V.nnz_ap, V.s_perm, R));
    PDF_KERNEL("k_rx_next", st, k_rx_next<<<rx_blocks(nnz_n), 256, 0, st>>>(nnz_n, V.c_off, V.c_tap, V.c_pv, R));
  }
  RxVals R;
  for (int v = 0; v < kRxVar; ++v) {
    R.a[v] = nullptr; R.ap[v] = nullptr; R.q[v] = nullptr; R.s[v] = nullptr;
    R.af[v] = R.qf[v] = R.sf[v] = R.wf[v] = nullptr;
    R.w[v] = nullptr;
    R.an[v] = G.c_v[v];
  }
  PDF_KERNEL("k_rx_coarse_inv", st, k_rx_coarse_inv<<<kRxVar, 256, 0, st>>>(G.nc, G.c_rp, G.c_ci, R, G.cmat, G.cinv));
  return PDF_OK;
}

__device__ __forceinline__ int rx_variant(int c) { return c == 0 ? 0 : (c == 4 ? 1 : (c == 8 ? 2 : 3)); }

struct RxLevelDev {
  int32_t n, nc;
  const int32_t *a_rp, *a_ci, *q_rp, *q_ci, *s_rp, *s_ci;
  const float *a_f[kRxVar], *q_f[kRxVar], *s_f[kRxVar], *w_f[kRxVar];
};

template <int G>
__device__ __forceinline__ float group_sum_f(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// x_c = W b_c on the level's rows; b_{c, next} = S b_c on the coarse rows
// (G lanes per row: 32 where the rows of S are long), component c =
// blockIdx.y.  FP32 arithmetic; TB the type of b (FP64 at the finest level).
template <typename TB, int G>
__global__ void __launch_bounds__(256) k_rx_down(RxLevelDev V, int32_t nbx, const TB* __restrict__ b,
                                                 float* __restrict__ x, float* __restrict__ bc,
                                                 const int32_t* __restrict__ active, const int32_t* __restrict__ done) {
  const int c = blockIdx.y;
  if (*done || !active[c]) return;
  const int v = rx_variant(c);
  const TB* bb = b + (int64_t)c * V.n;
  if ((int32_t)blockIdx.x < nbx) {
    const int32_t i = blockIdx.x * 256 + threadIdx.x;
    if (i < V.n) x[(int64_t)c * V.n + i] = V.w_f[v][i] * (float)bb[i];
  } else {
    const int32_t J = ((blockIdx.x - nbx) * 256 + threadIdx.x) / G, g = threadIdx.x % G;
    float s = 0.0f;
    if (J < V.nc) {
      const float* sv = V.s_f[v];
      for (int32_t q = V.s_rp[J] + g; q < V.s_rp[J + 1]; q += G) s += sv[q] * (float)bb[V.s_ci[q]];
    }
    s = group_sum_f<G>(s);
    if (J < V.nc && g == 0) bc[(int64_t)c * V.nc + J] = s;
  }
}

template <typename TB, typename TZ>
__global__ void __launch_bounds__(256) k_rx_coarse(int32_t nc, const float* __restrict__ cinv,
                                                   const TB* __restrict__ b, TZ* __restrict__ z,
                                                   const int32_t* __restrict__ active,
                                                   const int32_t* __restrict__ done) {
  const int c = blockIdx.y;
  if (*done || !active[c]) return;
  const int v = rx_variant(c);
  const int32_t row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= nc) return;
  const float* Ci = cinv + (int64_t)v * nc * nc + (int64_t)row * nc;
  const TB* bb = b + (int64_t)c * nc;
  float s = 0.0f;
  for (int32_t k = lane; k < nc; k += 32) s += Ci[k] * (float)bb[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) z[(int64_t)c * nc + row] = (TZ)s;
}

// z_c = x_c + W (b_c - A x_c) + Q e_c on a coarse level, kG lanes per row.
__global__ void __launch_bounds__(256) k_rx_up(RxLevelDev V, const float* __restrict__ b, const float* __restrict__ x,
                                               const float* __restrict__ ec, float* __restrict__ z,
                                               const int32_t* __restrict__ active, const int32_t* __restrict__ done) {
  const int c = blockIdx.y;
  if (*done || !active[c]) return;
  const int v = rx_variant(c);
  const int32_t i = (blockIdx.x * 256 + threadIdx.x) / kG, g = threadIdx.x % kG;
  const float* xx = x + (int64_t)c * V.n;
  const float* ee = ec + (int64_t)c * V.nc;
  float ax = 0.0f, qe = 0.0f;
  if (i < V.n) {
    const float *av = V.a_f[v], *qv = V.q_f[v];
    for (int32_t q = V.a_rp[i] + g; q < V.a_rp[i + 1]; q += kG) ax += av[q] * xx[V.a_ci[q]];
    for (int32_t q = V.q_rp[i] + g; q < V.q_rp[i + 1]; q += kG) qe += qv[q] * ee[V.q_ci[q]];
  }
  ax = group_sum_f<kG>(ax);
  qe = group_sum_f<kG>(qe);
  if (i < V.n && g == 0) {
    const int64_t o = (int64_t)c * V.n + i;
    z[o] = xx[i] + V.w_f[v][i] * (b[o] - ax) + qe;
  }
}

__device__ __forceinline__ bool rx_fixed(int c, uint8_t w) { return w == 2 || (w == 1 && c != 0 && c != 4 && c != 8); }

// The finest up-sweep (one thread per row) with the application's end
// (RxDot): z = 0 on fixed unknowns, r . z and beta.
__device__ void rx_dot_finish(int c, double rz, double* __restrict__ part, const RxDot& D) {
  __shared__ double sh[8];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rz += __shfl_xor_sync(0xffffffffu, rz, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = rz;
  __syncthreads();
  double* pc = part + (int64_t)c * gridDim.x;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += sh[k];
    pc[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(D.counter + c, 1) == (int32_t)gridDim.x - 1;
    if (last) D.counter[c] = 0;
  }
  __syncthreads();
  if (!last) return;
  double t = 0.0;
  for (int32_t k = threadIdx.x; k < (int32_t)gridDim.x; k += 256) t += __ldcg(pc + k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < 8; ++k) v += sh[k];
    const double old = D.rz[c];
    D.beta[c] = D.first || old == 0.0 ? 0.0 : v / old;
    D.rz[c] = v;
  }
}

__global__ void __launch_bounds__(256) k_rx_up0(RxLevelDev V, const double* __restrict__ r,
                                                const float* __restrict__ x, const float* __restrict__ ec,
                                                double* __restrict__ z, double* __restrict__ part, RxDot D,
                                                const int32_t* __restrict__ active,
                                                const int32_t* __restrict__ done) {
  const int c = blockIdx.y;
  if (*done || !active[c]) return;
  const int v = rx_variant(c);
  const int32_t i = blockIdx.x * 256 + threadIdx.x;
  double rz = 0.0;
  if (i < V.n) {
    const int64_t o = (int64_t)c * V.n + i;
    double zi = 0.0;
    if (!rx_fixed(c, D.wall[i])) {
      const float* xx = x + (int64_t)c * V.n;
      const float* ee = ec + (int64_t)c * V.nc;
      const float *av = V.a_f[v], *qv = V.q_f[v];
      float ax = 0.0f, qe = 0.0f;
      for (int32_t q = V.a_rp[i]; q < V.a_rp[i + 1]; ++q) ax += av[q] * xx[V.a_ci[q]];
      for (int32_t q = V.q_rp[i]; q < V.q_rp[i + 1]; ++q) qe += qv[q] * ee[V.q_ci[q]];
      const double ri = r[o];
      zi = (double)(xx[i] + V.w_f[v][i] * ((float)ri - ax) + qe);
      rz = ri * zi;
    }
    z[o] = zi;
  }
  rx_dot_finish(c, rz, part, D);
}

// Without levels: z = Inv r in FP32, then the same end.
__global__ void __launch_bounds__(256) k_rx_dot(int32_t n, const double* __restrict__ r, double* __restrict__ z,
                                                double* __restrict__ part, RxDot D, const int32_t* __restrict__ active,
                                                const int32_t* __restrict__ done) {
  const int c = blockIdx.y;
  if (*done || !active[c]) return;
  const int32_t i = blockIdx.x * 256 + threadIdx.x;
  double rz = 0.0;
  if (i < n) {
    const int64_t o = (int64_t)c * n + i;
    if (rx_fixed(c, D.wall[i])) z[o] = 0.0;
    else rz = r[o] * z[o];
  }
  rx_dot_finish(c, rz, part, D);
}

pdf_status relax_amg_apply(const RelaxAmg& G, const double* r, double* z, const int32_t* active,
                           const int32_t* done, const RxDot& dot, cudaStream_t st) {
  const int L = (int)G.lv.size();
  auto dev = [&](int l) {
    const RxLevel& V = G.lv[l];
    RxLevelDev D;
    D.n = V.n;
    D.nc = V.nc;
    D.a_rp = V.a_rp; D.a_ci = V.a_ci;
    D.q_rp = V.q_rp; D.q_ci = V.q_ci; D.s_rp = V.s_rp; D.s_ci = V.s_ci;
    for (int v = 0; v < kRxVar; ++v) { D.a_f[v] = V.a_f[v]; D.q_f[v] = V.q_f[v]; D.s_f[v] = V.s_f[v]; D.w_f[v] = V.w_f[v]; }
    return D;
  };
  if (L == 0) {
    PDF_KERNEL("k_rx_coarse", st, (k_rx_coarse<double, double><<<dim3((G.nc + 7) / 8, 9), 256, 0, st>>>(
                                      G.nc, G.cinv, r, z, active, done)));
    PDF_KERNEL("k_rx_dot", st, k_rx_dot<<<dim3((G.nc + 255) / 256, 9), 256, 0, st>>>(G.nc, r, z, G.upart, dot,
                                                                                       active, done));
    return PDF_OK;
  }
  for (int l = 0; l < L; ++l) {
    const RxLevel& V = G.lv[l];
    float* bc = l + 1 < L ? G.lv[l + 1].b : G.cb;
    // a warp per coarse row where the rows of S are long
    const bool wide = V.nnz_ap > 48 * (int64_t)V.nc;
    const int lanes = wide ? 32 : kG;
    const int32_t nbx = (V.n + 255) / 256, nbc = (int32_t)(((int64_t)V.nc * lanes + 255) / 256);
    const dim3 grid(nbx + nbc, 9);
    if (l == 0 && wide)
      PDF_KERNEL("k_rx_down", st, (k_rx_down<double, 32><<<grid, 256, 0, st>>>(dev(l), nbx, r, V.x, bc, active, done)));
    else if (l == 0)
      PDF_KERNEL("k_rx_down", st, (k_rx_down<double, kG><<<grid, 256, 0, st>>>(dev(l), nbx, r, V.x, bc, active, done)));
    else if (wide)
      PDF_KERNEL("k_rx_down", st, (k_rx_down<float, 32><<<grid, 256, 0, st>>>(dev(l), nbx, V.b, V.x, bc, active, done)));
    else
      PDF_KERNEL("k_rx_down", st, (k_rx_down<float, kG><<<grid, 256, 0, st>>>(dev(l), nbx, V.b, V.x, bc, active, done)));
  }
  PDF_KERNEL("k_rx_coarse", st, (k_rx_coarse<float, float><<<dim3((G.nc + 7) / 8, 9), 256, 0, st>>>(
                                    G.nc, G.cinv, G.cb, G.cz, active, done)));
  for (int l = L - 1; l >= 0; --l) {
    const RxLevel& V = G.lv[l];
    const float* ec = l + 1 < L ? G.lv[l + 1].z : G.cz;
    if (l == 0)
      PDF_KERNEL("k_rx_up0", st, k_rx_up0<<<dim3((V.n + 255) / 256, 9), 256, 0, st>>>(dev(l), r, V.x, ec, z, G.upart,
                                                                                       dot, active, done));
    else
      PDF_KERNEL("k_rx_up", st, k_rx_up<<<dim3((int32_t)(((int64_t)V.n * kG + 255) / 256), 9), 256, 0, st>>>(
                                    dev(l), V.b, V.x, ec, V.z, active, done));
  }
  return PDF_OK;
}

}  // namespace pdfgb


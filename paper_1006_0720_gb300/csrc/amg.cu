// Smoothed-aggregation algebraic multigrid for the pressure projection's
// Poisson matrix (sec. 3.2 solves it by Jacobi-preconditioned conjugate
// gradients; the matrix depends on the mesh only, so a multigrid hierarchy
// built once per mesh cuts the iterations from thousands to tens while the
// solution stays that of the same linear system).
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

pdf_status amg_setup(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                     const std::vector<double>& v, bool singular, Amg& G) {
  constexpr int32_t kCoarse = 256, kMaxLevels = 12;
  HCsr A;
  A.n = A.m = n;
  A.rp = rp;
  A.ci = ci;
  A.v = v;
  double theta = 0.08;
  std::vector<HCsr> As, Qs;
  std::vector<std::vector<double>> Ws;
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
    HCsr Q = P;  // same pattern as AP's union with P: rebuild row by row
    {
      Q.ci.clear();
      Q.v.clear();
      Q.rp.assign(A.n + 1, 0);
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
    Qs.push_back(Q);
    Ws.push_back(W);
    A = std::move(Ac);
    theta *= 0.5;
  }
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

}  // namespace pdfgb

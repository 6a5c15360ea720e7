// Elliptic relaxation for the tensor wp_ij (eq. elliptic-relaxation-
// Lagrangian): (M + K_L) wp = M rhs with linear triangles (sec. 3.2: P1 FEM,
// Jacobi-preconditioned conjugate gradients, warm start), solved by
// conjugate gradients in FP64 for the nine components at once, with the
// paper's Jacobi preconditioner or (the default) the multigrid V-cycle of
// amg.cu.
//   M_ab   = sum_e A_e (1 + delta_ab) / 12
//   K_L,ab = sum_e L2_e A_e grad N_a . grad N_b,  L2_e = mean of nodal L^2
//   L = C_L max(C_xi k^1.5 / eps, C_eta (nu^3 / eps)^1/4) (eq. L), with
//   C_xi = 1 + 1.3 n_i n_i for wp_ii and 1 otherwise (eq. Cxi), n the unit
//   outward normal of the nearest wall edge.
// Reflecting (free-slip) walls are symmetry planes: off-diagonal components
// are held at 0 on wall nodes, diagonal components take the natural
// condition.  No-slip walls hold every component at wp_ij = -4.5 eps n_i n_j
// (the section on no-slip wall-boundary conditions).  Periodic twin nodes
// are one unknown.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "amg.cuh"
#include "common.cuh"

namespace pdfgb {

struct RelaxParams {
  double nu, C1, C2, CT, CL, Ceta, Cv, gamma5;
};

constexpr double kRKFloor = 1e-12, kREFloor = 1e-12;

// Per node: the nine right-hand sides and the three L^2 fields (C_xi of
// wp_11, of wp_22, and 1).
__global__ void k_relax_nodes(int32_t n_nodes, const double* __restrict__ ns, const double* __restrict__ nd,
                              const double* __restrict__ wall_n, RelaxParams P, double* __restrict__ rhs,
                              double* __restrict__ L2, double* __restrict__ gdir) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    const double* S = ns + (int64_t)n * PDF_NNS;
    const double* D = nd + (int64_t)n * PDF_NND;
    const double k = fmax(0.5 * (S[5] + S[6] + S[7]), kRKFloor);
    const double om = S[3];
    const double eps = fmax(om * (k + P.nu * P.CT * P.CT * om), kREFloor);
    // right-hand side (eq. elliptic-relaxation-Lagrangian with eqs. H, A_v, bij)
    const double R[3][3] = {{S[5], S[8], S[9]}, {S[8], S[6], S[10]}, {S[9], S[10], S[7]}};
    const double g[3][3] = {{D[0], D[1], 0.0}, {D[2], D[3], 0.0}, {D[4], D[5], 0.0}};
    const double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                       R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                       R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
    const double tk = 2.0 * k / 3.0;
    const double Av = fmin(1.0, P.Cv * det / (tk * tk * tk));
    double b[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) b[i][j] = R[i][j] / (2.0 * k) - (i == j ? 1.0 / 3.0 : 0.0);
    const double g3 = P.gamma5 / 3.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double bk = 0.0, bl = 0.0;
        for (int q = 0; q < 3; ++q) {
          bk += b[i][q] * g[q][j];
          bl += b[i][q] * g[j][q];
        }
        const double h = (P.C2 * Av + g3) * g[i][j] - g3 * g[j][i] + P.gamma5 * (bk - bl);
        rhs[(int64_t)(3 * i + j) * n_nodes + n] = (i == j ? 0.5 * (1.0 - P.C1) * k * om : 0.0) + k * h;
      }
    const double nx = wall_n[2 * n], ny = wall_n[2 * n + 1];
    // the no-slip Dirichlet values -4.5 eps n_i n_j (n_z = 0)
    const double n3[3] = {nx, ny, 0.0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gdir[(int64_t)(3 * i + j) * n_nodes + n] = -4.5 * eps * n3[i] * n3[j];
    const double lt = k * sqrt(k) / eps, lk = P.Ceta * sqrt(sqrt(P.nu * P.nu * P.nu / eps));
    const double cxi[3] = {1.0 + 1.3 * nx * nx, 1.0 + 1.3 * ny * ny, 1.0};
    for (int c = 0; c < 3; ++c) {
      const double L = P.CL * fmax(cxi[c] * lt, lk);
      L2[(int64_t)c * n_nodes + n] = L * L;
    }
  }
}

// Element means of the nodal L^2 of the three classes, [n_tri][3].
__global__ void k_relax_elem_l2(int32_t n_tri, const int32_t* __restrict__ tri, int32_t n_nodes,
                                const double* __restrict__ L2, double* __restrict__ eL2) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    const int32_t a = tri[3 * e], b = tri[3 * e + 1], c = tri[3 * e + 2];
#pragma unroll
    for (int cl = 0; cl < 3; ++cl) {
      const double* L = L2 + (int64_t)cl * n_nodes;
      eL2[3 * (int64_t)e + cl] = (L[a] + L[b] + L[c]) / 3.0;
    }
  }
}

// Matrix values of the three classes for every stored entry: the constant
// mass part plus sum over contributing elements of L2_e * (stiffness entry).
__global__ void k_relax_assemble(int64_t nnz, const double* __restrict__ mval, const int32_t* __restrict__ ctb_off,
                                 const int32_t* __restrict__ ctb_e, const double* __restrict__ ctb_k,
                                 const double* __restrict__ eL2, double* __restrict__ aval) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
    double s[3] = {mval[q], mval[q], mval[q]};
    for (int32_t t = ctb_off[q]; t < ctb_off[q + 1]; ++t) {
      const double* L = eL2 + 3 * (int64_t)ctb_e[t];
      const double kab = ctb_k[t];
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) s[cl] += L[cl] * kab;
    }
#pragma unroll
    for (int cl = 0; cl < 3; ++cl) aval[(int64_t)cl * nnz + q] = s[cl];
  }
}

__device__ __forceinline__ int comp_class(int ij) { return ij == 0 ? 0 : (ij == 4 ? 1 : 2); }
__device__ __forceinline__ bool comp_dirichlet(int ij) { return ij != 0 && ij != 4 && ij != 8; }
// component ij of unknown r is held fixed: off-diagonal on any wall, every
// component on a no-slip wall
__device__ __forceinline__ bool fixed_at(int ij, uint8_t w) { return w == 2 || (w == 1 && comp_dirichlet(ij)); }

// y = A x for component ij over the unknowns (masked rows/cols for Dirichlet).
__device__ __forceinline__ double spmv_row(int32_t r, int ij, int32_t n_rep, int64_t nnz,
                                           const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                           const double* __restrict__ aval, const uint8_t* __restrict__ wall,
                                           const double* __restrict__ x) {
  if (fixed_at(ij, wall[r])) return 0.0;
  const double* A = aval + (int64_t)comp_class(ij) * nnz;
  const double* X = x + (int64_t)ij * n_rep;
  double s = 0.0;
  for (int32_t q = rp[r]; q < rp[r + 1]; ++q) {
    const int32_t c = ci[q];
    if (fixed_at(ij, wall[c])) continue;
    s += A[q] * X[c];
  }
  return s;
}

constexpr int kRBlock = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kRBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  v = __shfl_sync(0xffffffffu, v, 0);  // every lane takes part in the broadcast
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kRBlock / 32; ++i) t += sh[i];
  __syncthreads();
  return t;  // valid in thread 0
}

// Set-up: b = M f (masked), x = initial guess (masked), r = b - A x,
// z = r / diag, p = z; partials of r.z, r.r and b.b.  grid (blocks, 9).
__global__ void __launch_bounds__(kRBlock) k_cg_init(
    int32_t n_rep, int64_t nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const double* __restrict__ mval, const double* __restrict__ aval, const double* __restrict__ diag,
    const uint8_t* __restrict__ wall, const int32_t* __restrict__ rep_node, int32_t n_nodes,
    const double* __restrict__ f, const double* __restrict__ gdir, const double* __restrict__ wp,
    double* __restrict__ x, double* __restrict__ r, double* __restrict__ z, double* __restrict__ p,
    double* __restrict__ q, double* __restrict__ part) {
  const int ij = blockIdx.y;
  const int32_t row = blockIdx.x * kRBlock + threadIdx.x;
  double rz = 0.0, rr = 0.0, bb = 0.0;
  // the starting value of an unknown: its fixed value (0, or the no-slip
  // Dirichlet value), else the initial guess
  auto start = [&](int32_t u) {
    const uint8_t w = wall[u];
    const int64_t o = (int64_t)ij * n_nodes + rep_node[u];
    return fixed_at(ij, w) ? (w == 2 ? gdir[o] : 0.0) : wp[o];
  };
  if (row < n_rep) x[(int64_t)ij * n_rep + row] = start(row);
  // x of other rows is written by other blocks: the residual below takes the
  // starting values directly; the fixed columns carry their values into the
  // free rows' right-hand side
  const bool fixed_row = row < n_rep && fixed_at(ij, wall[row]);
  if (row < n_rep) {
    double b = 0.0, ax = 0.0;
    if (!fixed_row) {
      const double* A = aval + (int64_t)comp_class(ij) * nnz;
      for (int32_t q = rp[row]; q < rp[row + 1]; ++q) {
        const int32_t c = ci[q];
        b += mval[q] * f[(int64_t)ij * n_nodes + rep_node[c]];
        ax += A[q] * start(c);
      }
    }
    const double res = b - ax;
    const double zz = res / diag[(int64_t)comp_class(ij) * n_rep + row];
    const int64_t o = (int64_t)ij * n_rep + row;
    r[o] = res;
    z[o] = fixed_row ? 0.0 : zz;
    p[o] = z[o];
    q[o] = 0.0;  // the multigrid path's q = A z + beta q starts from 0
    rz = res * z[o];
    rr = res * res;
    bb = b * b;
  }
  const double s1 = block_sum(rz), s2 = block_sum(rr), s3 = block_sum(bb);
  if (threadIdx.x == 0) {
    const int64_t nb = gridDim.x;
    part[(0 * 9 + ij) * nb + blockIdx.x] = s1;
    part[(1 * 9 + ij) * nb + blockIdx.x] = s2;
    part[(2 * 9 + ij) * nb + blockIdx.x] = s3;
  }
}

// Sum the block partials of `nq` quantities for 9 components (fixed order).
__global__ void k_cg_reduce(const double* __restrict__ part, int32_t nb, int32_t nq, double* __restrict__ out) {
  const int q = blockIdx.x;  // quantity * 9 + component
  double s = 0.0;
  for (int32_t i = threadIdx.x; i < nb; i += kRBlock) s += part[(int64_t)q * nb + i];
  s = block_sum(s);
  if (threadIdx.x == 0) out[q] = s;
}

// Device scalars (9 components each) and control words of the iteration.
enum { kRPq = 0, kRRz = 9, kRRr = 18, kRBb = 27, kRTol2 = 36, kRAlpha = 45, kRBeta = 54 };
enum { kRDone = 0, kRIt = 1, kRMaxIt = 2, kRCntSpmv = 8, kRCntUpd = 17, kRActive = 26, kRIters = 35 };

// True in the block of component blockIdx.y that arrives last (its partial
// written before); it resets the counter.
__device__ __forceinline__ bool last_block_of(int32_t* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(counter, 1) == (int32_t)gridDim.x - 1;
    if (last) *counter = 0;
  }
  __syncthreads();
  return last;
}

__device__ __forceinline__ double sum_of(const double* part, int32_t nb) {
  double t = 0.0;
  for (int32_t i = threadIdx.x; i < nb; i += kRBlock) t += __ldcg(part + i);
  return block_sum(t);  // valid in thread 0
}

// After the set-up sums (scal: [0,9) r.z, [9,18) r.r, [18,27) b.b): the
// stopping thresholds, the active components and the control words.
__global__ void k_cg_start(double rtol2, int32_t max_it, double* __restrict__ scal, int32_t* __restrict__ ctl) {
  if (threadIdx.x != 0) return;
  double rz[9], rr[9], bb[9];
  for (int c = 0; c < 9; ++c) { rz[c] = scal[c]; rr[c] = scal[9 + c]; bb[c] = scal[18 + c]; }
  int n_active = 0;
  for (int c = 0; c < 9; ++c) {
    scal[kRRz + c] = rz[c];
    scal[kRRr + c] = rr[c];
    scal[kRBb + c] = bb[c];
    scal[kRTol2 + c] = rtol2 * bb[c];
    const int a = (rr[c] > rtol2 * bb[c] && bb[c] > 0.0) ? 1 : 0;
    ctl[kRActive + c] = a;
    ctl[kRIters + c] = 0;
    ctl[kRCntSpmv + c] = 0;
    ctl[kRCntUpd + c] = 0;
    n_active += a;
  }
  ctl[kRIt] = 0;
  ctl[kRMaxIt] = max_it;
  ctl[kRDone] = (n_active == 0 || max_it <= 0) ? 1 : 0;
}

// q = A p and p.q (last block of a component: alpha = r.z / p.q).
__global__ void __launch_bounds__(kRBlock) k_cg_spmv(int32_t n_rep, int64_t nnz, const int32_t* __restrict__ rp,
                                                      const int32_t* __restrict__ ci, const double* __restrict__ aval,
                                                      const uint8_t* __restrict__ wall, const double* __restrict__ p,
                                                      double* __restrict__ q, double* __restrict__ part,
                                                      double* __restrict__ scal, int32_t* __restrict__ ctl) {
  const int ij = blockIdx.y;
  if (ctl[kRDone] || !ctl[kRActive + ij]) return;
  const int32_t row = blockIdx.x * kRBlock + threadIdx.x;
  double pq = 0.0;
  if (row < n_rep) {
    const double v = spmv_row(row, ij, n_rep, nnz, rp, ci, aval, wall, p);
    q[(int64_t)ij * n_rep + row] = v;
    pq = v * p[(int64_t)ij * n_rep + row];
  }
  double* pp = part + (int64_t)ij * gridDim.x;
  const double s = block_sum(pq);
  if (threadIdx.x == 0) pp[blockIdx.x] = s;
  if (!last_block_of(ctl + kRCntSpmv + ij)) return;
  const double t = sum_of(pp, gridDim.x);
  if (threadIdx.x == 0) {
    scal[kRPq + ij] = t;
    scal[kRAlpha + ij] = t != 0.0 ? scal[kRRz + ij] / t : 0.0;
  }
}

// x += alpha p; r -= alpha q; z = r / diag; r.z, r.r (last block of a
// component: beta = r.z_new / r.z_old, count the iteration, retire the
// component at r.r <= rtol^2 b.b; the last component to finish the
// iteration stops the solve when none is left or at max_it).
__global__ void __launch_bounds__(kRBlock) k_cg_update(int32_t n_rep, const double* __restrict__ diag,
                                                        const uint8_t* __restrict__ wall, double* __restrict__ scal,
                                                        double* __restrict__ x, double* __restrict__ r,
                                                        double* __restrict__ z, const double* __restrict__ p,
                                                        const double* __restrict__ q, double* __restrict__ part,
                                                        int32_t* __restrict__ ctl) {
  const int ij = blockIdx.y;
  if (ctl[kRDone] || !ctl[kRActive + ij]) return;
  const int32_t row = blockIdx.x * kRBlock + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (row < n_rep) {
    const double alpha = scal[kRAlpha + ij];
    const int64_t o = (int64_t)ij * n_rep + row;
    x[o] += alpha * p[o];
    const double res = r[o] - alpha * q[o];
    r[o] = res;
    const bool fixed = fixed_at(ij, wall[row]);
    const double zz = fixed ? 0.0 : res / diag[(int64_t)comp_class(ij) * n_rep + row];
    z[o] = zz;
    rz = res * zz;
    rr = res * res;
  }
  double* p1 = part + (int64_t)(9 + ij) * gridDim.x;
  double* p2 = part + (int64_t)(18 + ij) * gridDim.x;
  const double s1 = block_sum(rz), s2 = block_sum(rr);
  if (threadIdx.x == 0) {
    p1[blockIdx.x] = s1;
    p2[blockIdx.x] = s2;
  }
  if (!last_block_of(ctl + kRCntUpd + ij)) return;
  const double rzn = sum_of(p1, gridDim.x), rrn = sum_of(p2, gridDim.x);
  if (threadIdx.x == 0) {
    const double rzo = scal[kRRz + ij];
    scal[kRBeta + ij] = rzo != 0.0 ? rzn / rzo : 0.0;
    scal[kRRz + ij] = rzn;
    scal[kRRr + ij] = rrn;
    ctl[kRIters + ij] += 1;
    if (rrn <= scal[kRTol2 + ij]) ctl[kRActive + ij] = 0;
  }
}

// p = z + beta p for the active components; one thread closes the
// iteration: it counts it and stops the solve when every component is done
// or at max_it.
__global__ void k_cg_dir(int32_t n_rep, const double* __restrict__ scal, const double* __restrict__ z,
                         double* __restrict__ p, int32_t* __restrict__ ctl) {
  const int ij = blockIdx.y;
  if (ctl[kRDone]) return;
  const int32_t row = blockIdx.x * kRBlock + threadIdx.x;
  if (ctl[kRActive + ij] && row < n_rep) {
    const int64_t o = (int64_t)ij * n_rep + row;
    p[o] = z[o] + scal[kRBeta + ij] * p[o];
  }
}

__global__ void k_cg_close(int32_t* __restrict__ ctl) {
  if (threadIdx.x != 0 || ctl[kRDone]) return;
  const int32_t it = ctl[kRIt] + 1;
  ctl[kRIt] = it;
  int n_active = 0;
  for (int c = 0; c < 9; ++c) n_active += ctl[kRActive + c];
  if (n_active == 0 || it >= ctl[kRMaxIt]) ctl[kRDone] = 1;
}

// Multigrid path.  The finest matrices of the four preconditioner variants
// (components 0, 4, 8 and the off-diagonal ones): the class values with the
// fixed unknowns' rows and columns reduced to their diagonal.
__global__ void k_rx_fill(int32_t n_rep, int64_t nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ aval, const uint8_t* __restrict__ wall, double* __restrict__ a0,
                          double* __restrict__ a1, double* __restrict__ a2, double* __restrict__ a3) {
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rep; r += gridDim.x * blockDim.x) {
    const uint8_t wr = wall[r];
    for (int32_t q = rp[r]; q < rp[r + 1]; ++q) {
      const int32_t c = ci[q];
      const uint8_t wc = wall[c];
      const bool diag = c == r;
      // variants 0-2: every component fixed on no-slip nodes; variant 3:
      // also on free-slip wall nodes
      const bool f012 = wr == 2 || wc == 2, f3 = wr != 0 || wc != 0;
      a0[q] = f012 && !diag ? 0.0 : aval[q];
      a1[q] = f012 && !diag ? 0.0 : aval[nnz + q];
      a2[q] = f012 && !diag ? 0.0 : aval[2 * nnz + q];
      a3[q] = f3 && !diag ? 0.0 : aval[2 * nnz + q];
    }
  }
}

// Multigrid path: p = z + beta p, q = A z + beta q (= A p) and p.q (last
// block of a component: alpha = r.z / p.q).
__global__ void __launch_bounds__(kRBlock) k_cg_spmv_rec(int32_t n_rep, int64_t nnz, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          const double* __restrict__ aval,
                                                          const uint8_t* __restrict__ wall,
                                                          const double* __restrict__ z, double* __restrict__ p,
                                                          double* __restrict__ q, double* __restrict__ part,
                                                          double* __restrict__ scal, int32_t* __restrict__ ctl) {
  const int ij = blockIdx.y;
  if (ctl[kRDone] || !ctl[kRActive + ij]) return;
  const int32_t row = blockIdx.x * kRBlock + threadIdx.x;
  double pq = 0.0;
  if (row < n_rep) {
    const double beta = scal[kRBeta + ij];
    const int64_t o = (int64_t)ij * n_rep + row;
    const double qn = spmv_row(row, ij, n_rep, nnz, rp, ci, aval, wall, z) + beta * q[o];
    const double pn = z[o] + beta * p[o];
    q[o] = qn;
    p[o] = pn;
    pq = qn * pn;
  }
  double* pp = part + (int64_t)ij * gridDim.x;
  const double s = block_sum(pq);
  if (threadIdx.x == 0) pp[blockIdx.x] = s;
  if (!last_block_of(ctl + kRCntSpmv + ij)) return;
  const double t = sum_of(pp, gridDim.x);
  if (threadIdx.x == 0) {
    scal[kRPq + ij] = t;
    scal[kRAlpha + ij] = t != 0.0 ? scal[kRRz + ij] / t : 0.0;
  }
}

// x += alpha p; r -= alpha q; r.r (last block of a component: count the
// iteration, retire the component at r.r <= rtol^2 b.b).
__global__ void __launch_bounds__(kRBlock) k_cg_update_mg(int32_t n_rep, double* __restrict__ scal,
                                                           double* __restrict__ x, double* __restrict__ r,
                                                           const double* __restrict__ p, const double* __restrict__ q,
                                                           double* __restrict__ part, int32_t* __restrict__ ctl) {
  const int ij = blockIdx.y;
  if (ctl[kRDone] || !ctl[kRActive + ij]) return;
  const int32_t row = blockIdx.x * kRBlock + threadIdx.x;
  double rr = 0.0;
  if (row < n_rep) {
    const double alpha = scal[kRAlpha + ij];
    const int64_t o = (int64_t)ij * n_rep + row;
    x[o] += alpha * p[o];
    const double res = r[o] - alpha * q[o];
    r[o] = res;
    rr = res * res;
  }
  double* p2 = part + (int64_t)(18 + ij) * gridDim.x;
  const double s2 = block_sum(rr);
  if (threadIdx.x == 0) p2[blockIdx.x] = s2;
  if (!last_block_of(ctl + kRCntUpd + ij)) return;
  const double rrn = sum_of(p2, gridDim.x);
  if (threadIdx.x == 0) {
    scal[kRRr + ij] = rrn;
    ctl[kRIters + ij] += 1;
    if (rrn <= scal[kRTol2 + ij]) ctl[kRActive + ij] = 0;
  }
}

__global__ void k_cg_diag(int32_t n_rep, int64_t nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ aval, double* __restrict__ diag) {
  const int cl = blockIdx.y;
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rep; r += gridDim.x * blockDim.x) {
    double d = 1.0;
    for (int32_t q = rp[r]; q < rp[r + 1]; ++q)
      if (ci[q] == r) d = aval[(int64_t)cl * nnz + q];
    diag[(int64_t)cl * n_rep + r] = d;
  }
}

// Solution back to all nodes (twins get their representative's value).
__global__ void k_cg_scatter(int32_t n_nodes, const int32_t* __restrict__ node_rep, int32_t n_rep,
                             const double* __restrict__ x, double* __restrict__ wp) {
  const int ij = blockIdx.y;
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x)
    wp[(int64_t)ij * n_nodes + n] = x[(int64_t)ij * n_rep + node_rep[n]];
}

}  // namespace pdfgb

// ----------------------------------------------------------------------------
// Host side.
// ----------------------------------------------------------------------------
namespace pdfgb {

// The multigrid hierarchy of the relaxation pattern's stiffness matrix,
// built once; on failure the solve falls back to Jacobi for good.
static pdf_status relax_amg_build(pdf_particles* P) {
  RelaxWork& W = P->rx;
  if (W.amg || !W.multigrid) return PDF_OK;
  const RelaxMesh& R = P->mesh->rx;
  std::vector<int32_t> rp(R.n_rep + 1), ci(R.nnz), off(R.nnz + 1);
  PDF_CUDA(cudaMemcpy(rp.data(), R.rp, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost));
  PDF_CUDA(cudaMemcpy(ci.data(), R.ci, sizeof(int32_t) * ci.size(), cudaMemcpyDeviceToHost));
  PDF_CUDA(cudaMemcpy(off.data(), R.ctb_off, sizeof(int32_t) * off.size(), cudaMemcpyDeviceToHost));
  std::vector<double> kc(off[R.nnz]), kv(R.nnz, 0.0);
  if (!kc.empty()) PDF_CUDA(cudaMemcpy(kc.data(), R.ctb_k, sizeof(double) * kc.size(), cudaMemcpyDeviceToHost));
  for (int64_t q = 0; q < R.nnz; ++q)
    for (int32_t t = off[q]; t < off[q + 1]; ++t) kv[q] += kc[t];
  RelaxAmg* G = new RelaxAmg();
  if (relax_amg_setup(R.n_rep, rp, ci, kv, *G) != PDF_OK) {
    delete G;
    W.multigrid = false;
    return PDF_OK;
  }
  W.amg = G;
  return PDF_OK;
}

static pdf_status relax_alloc(pdf_particles* P) {
  if (P->rx.x) return relax_amg_build(P);
  const RelaxMesh& R = P->mesh->rx;
  const int32_t nn = P->mesh->d.n_nodes;
  const int32_t nb = (R.n_rep + kRBlock - 1) / kRBlock;
  RelaxWork& W = P->rx;
  W.nb = nb;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void**)&W.f, sizeof(double) * 9 * nn);
  A((void**)&W.g, sizeof(double) * 9 * nn);
  A((void**)&W.L2, sizeof(double) * 3 * nn);
  A((void**)&W.eL2, sizeof(double) * 3 * (size_t)P->mesh->d.n_tri);
  A((void**)&W.aval, sizeof(double) * 3 * R.nnz);
  A((void**)&W.diag, sizeof(double) * 3 * R.n_rep);
  A((void**)&W.x, sizeof(double) * 9 * R.n_rep);
  A((void**)&W.r, sizeof(double) * 9 * R.n_rep);
  A((void**)&W.z, sizeof(double) * 9 * R.n_rep);
  A((void**)&W.p, sizeof(double) * 9 * R.n_rep);
  A((void**)&W.q, sizeof(double) * 9 * R.n_rep);
  A((void**)&W.part, sizeof(double) * 3 * 9 * nb);
  A((void**)&W.scal, sizeof(double) * 64);
  A((void**)&W.ctl, sizeof(int32_t) * 64);
  if (e == cudaSuccess) e = cudaMemset(W.ctl, 0, sizeof(int32_t) * 64);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&W.host, sizeof(double) * 64);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&W.host_ctl, sizeof(int32_t) * 64);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&W.cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W.ev0, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W.ev1, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    relax_free(W);
    return cuda_fail(e, "pdf_relax_solve: allocation");
  }
  return relax_amg_build(P);
}

void relax_free(RelaxWork& W) {
  cudaFree(W.f); cudaFree(W.g); cudaFree(W.L2); cudaFree(W.eL2); cudaFree(W.aval); cudaFree(W.diag); cudaFree(W.x); cudaFree(W.r);
  cudaFree(W.z); cudaFree(W.p); cudaFree(W.q); cudaFree(W.part); cudaFree(W.scal); cudaFree(W.ctl);
  if (W.host) cudaFreeHost(W.host);
  if (W.host_ctl) cudaFreeHost(W.host_ctl);
  if (W.gx) cudaGraphExecDestroy(W.gx);
  if (W.ev0) cudaEventDestroy(W.ev0);
  if (W.ev1) cudaEventDestroy(W.ev1);
  if (W.cs) cudaStreamDestroy(W.cs);
  if (W.amg) {
    relax_amg_free(*W.amg);
    delete W.amg;
  }
  W = RelaxWork();
}

// k iterations of the nine components (every kernel returns at once after
// the stop).
// z = M^-1 r (multigrid), z = 0 on fixed unknowns, r.z and beta.
static pdf_status relax_precondition(pdf_particles* P, int first, cudaStream_t st) {
  const RelaxMesh& R = P->mesh->rx;
  RelaxWork& W = P->rx;
  RxDot d;
  d.wall = R.wall;
  d.rz = W.scal + kRRz;
  d.beta = W.scal + kRBeta;
  d.counter = W.ctl + kRCntUpd;
  d.first = first;
  return relax_amg_apply(*W.amg, W.r, W.z, W.ctl + kRActive, W.ctl + kRDone, d, st);
}

static pdf_status relax_iterations(pdf_particles* P, int k, cudaStream_t st) {
  const RelaxMesh& R = P->mesh->rx;
  RelaxWork& W = P->rx;
  const dim3 grid(W.nb, 9);
  if (W.multigrid && W.amg) {
    for (int i = 0; i < k; ++i) {
      PDF_KERNEL("k_cg_spmv_rec", st, k_cg_spmv_rec<<<grid, kRBlock, 0, st>>>(R.n_rep, R.nnz, R.rp, R.ci, W.aval,
                                                                               R.wall, W.z, W.p, W.q, W.part, W.scal,
                                                                               W.ctl));
      PDF_KERNEL("k_cg_update_mg", st, k_cg_update_mg<<<grid, kRBlock, 0, st>>>(R.n_rep, W.scal, W.x, W.r, W.p, W.q,
                                                                                 W.part, W.ctl));
      PDF_KERNEL("k_cg_close", st, k_cg_close<<<1, 32, 0, st>>>(W.ctl));
      const pdf_status s = relax_precondition(P, 0, st);
      if (s != PDF_OK) return s;
    }
    return PDF_OK;
  }
  for (int i = 0; i < k; ++i) {
    PDF_KERNEL("k_cg_spmv", st, k_cg_spmv<<<grid, kRBlock, 0, st>>>(R.n_rep, R.nnz, R.rp, R.ci, W.aval, R.wall, W.p,
                                                                     W.q, W.part, W.scal, W.ctl));
    PDF_KERNEL("k_cg_update", st, k_cg_update<<<grid, kRBlock, 0, st>>>(R.n_rep, W.diag, R.wall, W.scal, W.x, W.r,
                                                                         W.z, W.p, W.q, W.part, W.ctl));
    PDF_KERNEL("k_cg_dir", st, k_cg_dir<<<grid, kRBlock, 0, st>>>(R.n_rep, W.scal, W.z, W.p, W.ctl));
    PDF_KERNEL("k_cg_close", st, k_cg_close<<<1, 32, 0, st>>>(W.ctl));
  }
  return PDF_OK;
}

static pdf_status relax_capture(pdf_particles* P, int k) {
  RelaxWork& W = P->rx;
  const long long n0 = prof_launches();
  PDF_CUDA(cudaStreamBeginCapture(W.cs, cudaStreamCaptureModeThreadLocal));
  pdf_status s = relax_iterations(P, k, W.cs);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(W.cs, &g);
  if (s != PDF_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "pdf_relax_solve: graph capture");
  const cudaError_t e2 = cudaGraphInstantiate(&W.gx, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    W.gx = nullptr;
    return cuda_fail(e2, "pdf_relax_solve: graph instantiation");
  }
  W.graph_launches = prof_launches() - n0;
  prof_count(-W.graph_launches);  // captured, not launched
  return PDF_OK;
}

static RelaxParams relax_params(const pdf_model_params* p) {
  RelaxParams r;
  r.nu = p->nu; r.C1 = p->C1; r.C2 = p->C2; r.CT = p->CT; r.CL = p->CL; r.Ceta = p->Ceta;
  r.Cv = p->Cv; r.gamma5 = p->gamma5;
  return r;
}

static int rblocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

static pdf_status relax_prepare(pdf_particles* P, const pdf_model_params* params, cudaStream_t st) {
  const pdf_mesh* m = P->mesh;
  const RelaxMesh& R = m->rx;
  RelaxWork& W = P->rx;
  const int32_t nn = m->d.n_nodes;
  PDF_KERNEL("k_relax_nodes", st, k_relax_nodes<<<rblocks(nn), 256, 0, st>>>(nn, P->ns, P->nd, R.wall_n, relax_params(params), W.f, W.L2, W.g));
  PDF_KERNEL("k_relax_elem_l2", st, k_relax_elem_l2<<<rblocks(m->d.n_tri), 256, 0, st>>>(m->d.n_tri, m->d.tri, nn, W.L2,
                                                                                         W.eL2));
  PDF_KERNEL("k_relax_assemble", st, k_relax_assemble<<<rblocks(R.nnz), 256, 0, st>>>(R.nnz, R.mval, R.ctb_off, R.ctb_e, R.ctb_k,
                                                                                      W.eL2, W.aval));
  PDF_KERNEL("k_cg_diag", st, k_cg_diag<<<dim3(rblocks(R.n_rep), 3), 256, 0, st>>>(R.n_rep, R.nnz, R.rp, R.ci, W.aval, W.diag));
  return PDF_OK;
}

// The preconditioner's matrices from the current relaxation matrices.
static pdf_status relax_amg_values(pdf_particles* P, cudaStream_t st) {
  const RelaxMesh& R = P->mesh->rx;
  RelaxWork& W = P->rx;
  RelaxAmg& G = *W.amg;
  PDF_KERNEL("k_rx_fill", st, k_rx_fill<<<rblocks(R.n_rep), 256, 0, st>>>(
                                  R.n_rep, R.nnz, R.rp, R.ci, W.aval, R.wall, relax_amg_level0(G, 0),
                                  relax_amg_level0(G, 1), relax_amg_level0(G, 2), relax_amg_level0(G, 3)));
  return relax_amg_update(G, st);
}

// The nodal right-hand side [9][n_nodes] and L^2 [3][n_nodes] of the
// relaxation for the particle set's statistics (the solve's own work space;
// valid until its next call).
pdf_status relax_fields(pdf_particles* P, const pdf_model_params* params, cudaStream_t st, const double** rhs,
                        const double** L2) {
  pdf_status s = relax_alloc(P);
  if (s != PDF_OK) return s;
  s = relax_prepare(P, params, st);
  if (s != PDF_OK) return s;
  *rhs = P->rx.f;
  *L2 = P->rx.L2;
  return PDF_OK;
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_relax_set_solver(pdf_particles* p, int32_t multigrid) {
  if (!p || (multigrid != 0 && multigrid != 1)) return fail(PDF_EINVAL, "pdf_relax_set_solver: bad arguments");
  RelaxWork& W = p->rx;
  if (W.multigrid == (multigrid == 1)) return PDF_OK;
  PDF_CUDA(cudaDeviceSynchronize());
  if (W.gx) {  // the captured iterations belong to the other preconditioner
    cudaGraphExecDestroy(W.gx);
    W.gx = nullptr;
  }
  W.multigrid = multigrid == 1;  // a built hierarchy is kept for a switch back
  return PDF_OK;
}

extern "C" pdf_status pdf_relax_rhs(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                                    double* rhs, double* L2, void* stream) {
  if (!p || !m || p->mesh != m || !params) return fail(PDF_EINVAL, "pdf_relax_rhs: bad arguments");
  if (!p->have_stats) return fail(PDF_ESTATE, "pdf_relax_rhs: call pdf_estimate_stats first");
  cudaStream_t st = (cudaStream_t)stream;
  pdf_status s = relax_alloc(p);
  if (s != PDF_OK) return s;
  s = relax_prepare(p, params, st);
  if (s != PDF_OK) return s;
  const int32_t nn = m->d.n_nodes;
  if (rhs) PDF_CUDA(cudaMemcpyAsync(rhs, p->rx.f, sizeof(double) * 9 * nn, cudaMemcpyDefault, st));
  if (L2) PDF_CUDA(cudaMemcpyAsync(L2, p->rx.L2, sizeof(double) * 3 * nn, cudaMemcpyDefault, st));
  return PDF_OK;
}

namespace pdfgb {

// The solve for the node statistics and derivatives held in p->ns, p->nd.
static pdf_status relax_solve(pdf_particles* p, const pdf_model_params* params, double* wp, double rtol,
                              int32_t max_it, int32_t* iters, double* rel_res, cudaStream_t st) {
  const pdf_mesh* m = p->mesh;
  pdf_status s = relax_alloc(p);
  if (s != PDF_OK) return s;
  s = relax_prepare(p, params, st);
  if (s != PDF_OK) return s;
  const RelaxMesh& R = m->rx;
  RelaxWork& W = p->rx;
  const int32_t nn = m->d.n_nodes, nb = W.nb;
  const dim3 grid(nb, 9);
  PDF_KERNEL("k_cg_init", st, k_cg_init<<<grid, kRBlock, 0, st>>>(R.n_rep, R.nnz, R.rp, R.ci, R.mval, W.aval, W.diag,
                                                                   R.wall, R.rep_node, nn, W.f, W.g, wp, W.x, W.r, W.z,
                                                                   W.p, W.q, W.part));
  PDF_KERNEL("k_cg_reduce", st, k_cg_reduce<<<27, kRBlock, 0, st>>>(W.part, nb, 3, W.scal));
  PDF_KERNEL("k_cg_start", st, k_cg_start<<<1, 32, 0, st>>>(rtol * rtol, max_it, W.scal, W.ctl));
  if (W.multigrid && W.amg) {
    // the first direction from the multigrid (k_cg_init's Jacobi values
    // replaced)
    s = relax_amg_values(p, st);
    if (s == PDF_OK) s = relax_precondition(p, 1, st);
    if (s != PDF_OK) return s;
  }
  // iterations in chunks of 8 (CUDA-graph replays while kernel timing is
  // off); the host reads the control words once per chunk
  constexpr int kChunk = 8;
  if (prof_timing()) {
    for (int launched = 0; launched < max_it; launched += kChunk) {
      s = relax_iterations(p, kChunk, st);
      if (s != PDF_OK) return s;
      PDF_CUDA(cudaMemcpyAsync(W.host_ctl, W.ctl, sizeof(int32_t) * 64, cudaMemcpyDeviceToHost, st));
      PDF_CUDA(cudaStreamSynchronize(st));
      if (W.host_ctl[kRDone]) break;
    }
  } else if (max_it > 0) {
    if (!W.gx) {
      s = relax_capture(p, kChunk);
      if (s != PDF_OK) return s;
    }
    PDF_CUDA(cudaEventRecord(W.ev0, st));
    PDF_CUDA(cudaStreamWaitEvent(W.cs, W.ev0, 0));
    for (int launched = 0; launched < max_it; launched += kChunk) {
      PDF_CUDA(cudaGraphLaunch(W.gx, W.cs));
      prof_count(W.graph_launches);
      PDF_CUDA(cudaMemcpyAsync(W.host_ctl, W.ctl, sizeof(int32_t) * 64, cudaMemcpyDeviceToHost, W.cs));
      PDF_CUDA(cudaStreamSynchronize(W.cs));
      if (W.host_ctl[kRDone]) break;
    }
    PDF_CUDA(cudaEventRecord(W.ev1, W.cs));
    PDF_CUDA(cudaStreamWaitEvent(st, W.ev1, 0));
  }
  PDF_CUDA(cudaMemcpyAsync(W.host, W.scal, sizeof(double) * 64, cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaMemcpyAsync(W.host_ctl, W.ctl, sizeof(int32_t) * 64, cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaStreamSynchronize(st));
  int n_active = 0;
  double rn[9], bn[9];
  for (int c = 0; c < 9; ++c) {
    rn[c] = std::sqrt(W.host[kRRr + c]);
    bn[c] = std::sqrt(W.host[kRBb + c]);
    n_active += W.host_ctl[kRActive + c];
  }
  PDF_KERNEL("k_cg_scatter", st, k_cg_scatter<<<dim3(rblocks(nn), 9), 256, 0, st>>>(nn, R.node_rep, R.n_rep, W.x, wp));
  for (int c = 0; c < 9; ++c) {
    if (iters) iters[c] = W.host_ctl[kRIters + c];
    if (rel_res) rel_res[c] = bn[c] > 0.0 ? rn[c] / bn[c] : 0.0;
  }
  if (n_active > 0) return fail(PDF_ENOTCONV, "pdf_relax_solve: iteration cap reached");
  return PDF_OK;
}

}  // namespace pdfgb

extern "C" pdf_status pdf_relax_solve_particles(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                                                double* wp, double rtol, int32_t max_it, int32_t* iters,
                                                double* rel_res, void* stream) {
  if (!p || !m || p->mesh != m || !params || !wp)
    return fail(PDF_EINVAL, "pdf_relax_solve_particles: bad arguments");
  if (!(rtol > 0.0) || max_it < 0)
    return fail(PDF_EINVAL, "pdf_relax_solve_particles: rtol must be > 0 and max_it >= 0");
  if (!p->have_stats) return fail(PDF_ESTATE, "pdf_relax_solve_particles: call pdf_estimate_stats first");
  return relax_solve(p, params, wp, rtol, max_it, iters, rel_res, (cudaStream_t)stream);
}

extern "C" pdf_status pdf_relax_solve(const pdf_mesh* m, const pdf_model_params* params, const double* node_stats,
                                      double* wp, double rtol, int32_t max_it, int32_t* iters, double* rel_res,
                                      void* stream) {
  if (!m || !params || !node_stats || !wp) return fail(PDF_EINVAL, "pdf_relax_solve: bad arguments");
  if (!(rtol > 0.0) || max_it < 0) return fail(PDF_EINVAL, "pdf_relax_solve: rtol must be > 0 and max_it >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (!m->solver) {
    pdf_particles* h = nullptr;
    const pdf_status s = stats_only_handle(m, &h);
    if (s != PDF_OK) return s;
    m->solver = h;
  }
  pdf_particles* S = m->solver;
  PDF_CUDA(cudaMemcpyAsync(S->ns, node_stats, sizeof(double) * (size_t)m->d.n_nodes * PDF_NNS, cudaMemcpyDefault, st));
  const pdf_status s = node_derivs_from_node_stats(S, st);
  if (s != PDF_OK) return s;
  S->have_stats = true;
  return relax_solve(S, params, wp, rtol, max_it, iters, rel_res, st);
}

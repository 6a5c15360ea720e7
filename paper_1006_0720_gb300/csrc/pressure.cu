// The stabilised pressure projection (sec. 3.2: eqs. velocity-prediction,
// pressure-projection-smooth, velocity-correction):
//   grad^2 dP = (div <U*> - C_p grad^2 <P'>^n) / dt
// with linear triangles over the relaxation mesh's unknowns (periodic twins
// merged): K dP = -(d + C_p (K <P'>^n - G^n)) / dt + G^{n+1} - G^n,
// K_ab = sum_e A_e grad N_a . grad N_b, d_a = sum_e A_e / 3 div_e, G the load
// of the Neumann condition at solid walls (eq. wall-pressure-condition) from
// the statistics at the projection that made <P'>^n (G^0 = 0) and from the
// present ones; zero flux at inflow and outflow edges.  The pure-Neumann
// system is made compatible by removing the mean of the right-hand side and
// solved by preconditioned conjugate gradients in FP64 from zero; dP is
// normalised to zero mean.  The particles' velocities are corrected by
// -dt grad dP of their element, and the statistics follow the correction.
//
// The conjugate-gradient iteration runs under device control: alpha, beta
// and the stopping test live in device memory (the last block of each
// reduction finishes it), every kernel returns at once after the stop, and
// the host looks at the state once per chunk of iterations.  The
// preconditioner is one V-cycle of the smoothed-aggregation multigrid of
// amg.cu (the paper's Jacobi preconditioner needs thousands of iterations on
// meshes of 10^5 nodes).
#include <algorithm>
#include <cmath>

#include "amg.cuh"
#include "common.cuh"

namespace pdfgb {

pdf_status node_stats_from_elements(pdf_particles* P, cudaStream_t st);

constexpr int kPBlock = 256;

__device__ __forceinline__ double pblock_sum(double v) {
  __shared__ double sh[kPBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kPBlock / 32; ++i) t += sh[i];
  __syncthreads();
  return t;  // valid in thread 0
}

// Neumann data at solid walls (eq. wall-pressure-condition; with wall
// functions, SLM, the advection term of the following equation as well) on
// one wall edge of element e:
//   h = nu lap<U_i> n_i - d<u_i u_j>/dx_j n_i [- <U_j> d<U_i>/dx_j n_i],
// the stress and velocity gradients those of element e, lap<U_i> and <U_j>
// the means of the edge's two nodes; the edge's load on each of its two
// nodes is h |edge| / 2.
__device__ __forceinline__ double wall_load(const int32_t* __restrict__ ed, const double* __restrict__ en,
                                            const int32_t* __restrict__ tri, const double* __restrict__ dN,
                                            const double* __restrict__ ns, const double* __restrict__ nd, double nu,
                                            bool slm) {
  const int32_t e = ed[0], a = ed[1], b = ed[2];
  const double* g = dN + (int64_t)e * 6;
  double duu_x = 0.0, duv_y = 0.0, duv_x = 0.0, dvv_y = 0.0, du_x = 0.0, du_y = 0.0, dv_x = 0.0, dv_y = 0.0;
  for (int j = 0; j < 3; ++j) {
    const double* S = ns + (int64_t)tri[3 * e + j] * PDF_NNS;
    duu_x += g[j] * S[5];
    duv_y += g[3 + j] * S[8];
    duv_x += g[j] * S[8];
    dvv_y += g[3 + j] * S[6];
    du_x += g[j] * S[0];
    du_y += g[3 + j] * S[0];
    dv_x += g[j] * S[1];
    dv_y += g[3 + j] * S[1];
  }
  const double* Sa = ns + (int64_t)a * PDF_NNS;
  const double* Sb = ns + (int64_t)b * PDF_NNS;
  const double* Da = nd + (int64_t)a * PDF_NND;
  const double* Db = nd + (int64_t)b * PDF_NND;
  const double nx = en[0], ny = en[1];
  double hx = nu * 0.5 * (Da[6] + Db[6]) - (duu_x + duv_y);
  double hy = nu * 0.5 * (Da[7] + Db[7]) - (duv_x + dvv_y);
  if (slm) {
    const double U = 0.5 * (Sa[0] + Sb[0]), V = 0.5 * (Sa[1] + Sb[1]);
    hx -= U * du_x + V * du_y;
    hy -= U * dv_x + V * dv_y;
  }
  return (hx * nx + hy * ny) * en[2] * 0.5;
}

// The device view of one pressure system.
struct PSys {
  int32_t n;
  const int32_t *rp, *ci, *rep_node, *pw_off, *pw_e;
  const double *kval, *pw_n;
  const int8_t* dir;  // nullptr: no Dirichlet unknowns
};

// Dirichlet value of dP at a node of the inflow (1) or outflow (2) (the
// street canyon's inflow/outflow condition): the target <P> there, Pi L_x
// at the inflow, 0 at the outflow, minus <vv> of the node (the cross-stream
// balance of an undisturbed channel), minus the current <P'>.
__device__ __forceinline__ double dirichlet_dP(int kind, int32_t node, const double* __restrict__ ns,
                                               const double* __restrict__ pres, double PiLx) {
  return (kind == 1 ? PiLx : 0.0) - ns[(int64_t)node * PDF_NNS + 6] - pres[node];
}

// Free unknowns: b_u = -(d_u + C_p ((K <P'>)_u - G_u^n)) / dt + G_u^{n+1}
// - G_u^n - sum over Dirichlet columns v of K_uv g_v, d_u = sum over the
// elements around the unknown's node(s) of A_e / 3 times the element
// divergence of the nodal <U>, <V>; G the wall load above (G^n the one the
// current <P'> satisfies, G^{n+1} from the present statistics, written to
// gw).  Dirichlet unknowns: b_u = 0 (the iteration solves for the free
// part; the values are set afterwards).  Block partials of sum b.
__global__ void __launch_bounds__(kPBlock) k_press_rhs(
    PSys S, const int32_t* __restrict__ nse_off, const int32_t* __restrict__ nse, const int32_t* __restrict__ tri,
    const double* __restrict__ dN, const ElemGeo* __restrict__ geo, const double* __restrict__ ns,
    const double* __restrict__ nd, double nu, int slm, const double* __restrict__ pres,
    const double* __restrict__ gw_prev, double Cp, double inv_dt, double PiLx, double* __restrict__ gw,
    double* __restrict__ b, double* __restrict__ part) {
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  double bv = 0.0;
  if (u < S.n && (S.dir == nullptr || S.dir[u] == 0)) {
    const int32_t n = S.rep_node[u];
    double d = 0.0;
    for (int32_t i = nse_off[n]; i < nse_off[n + 1]; ++i) {
      const int32_t e = nse[i];
      const double* g = dN + (int64_t)e * 6;
      double div = 0.0;
      for (int j = 0; j < 3; ++j) {
        const double* Sn = ns + (int64_t)tri[3 * e + j] * PDF_NNS;
        div += g[j] * Sn[0] + g[3 + j] * Sn[1];
      }
      d += 0.5 * geo[e].two_area / 3.0 * div;
    }
    double kp = 0.0, lift = 0.0;
    for (int32_t q = S.rp[u]; q < S.rp[u + 1]; ++q) {
      const int32_t v = S.ci[q], node = S.rep_node[v];
      kp += S.kval[q] * pres[node];
      if (S.dir != nullptr && S.dir[v] != 0) lift += S.kval[q] * dirichlet_dP(S.dir[v], node, ns, pres, PiLx);
    }
    double gn = 0.0;
    for (int32_t i = S.pw_off[u]; i < S.pw_off[u + 1]; ++i)
      gn += wall_load(S.pw_e + 3 * (int64_t)i, S.pw_n + 3 * (int64_t)i, tri, dN, ns, nd, nu, slm != 0);
    const double gp = gw_prev[u];
    gw[u] = gn;
    bv = -(d + Cp * (kp - gp)) * inv_dt + (gn - gp) - lift;
  } else if (u < S.n) {
    gw[u] = 0.0;
  }
  if (u < S.n) b[u] = bv;
  const double s = pblock_sum(bv);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_press_sum(const double* __restrict__ part, int32_t nb, double* __restrict__ out) {
  double s = 0.0;
  for (int32_t i = threadIdx.x; i < nb; i += kPBlock) s += part[i];
  s = pblock_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// Device control words of the iteration.
enum { kCtlDone = 0, kCtlIters = 1, kCtlMaxIt = 2, kCtlCount0 = 4, kCtlCount1 = 5 };
// Device scalars.
enum { kSPq = 0, kSRz = 1, kSRr = 2, kSXsum = 3, kSBsum = 4, kSAlpha = 5, kSRzOld = 6, kSTol2 = 7, kSRr0 = 8 };

// True in the one block that arrives last at this reduction (its partial
// written before); it resets the counter for the next use.
__device__ __forceinline__ bool last_block(int32_t* counter) {
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

// Sum of the block partials by the whole (last) block, in a fixed order;
// the result is valid in thread 0.
__device__ __forceinline__ double sum_parts(const double* part, int32_t nb) {
  double t = 0.0;
  for (int32_t i = threadIdx.x; i < nb; i += kPBlock) t += __ldcg(part + i);
  return pblock_sum(t);
}

// b -= mean(b) (the singular system only); x = 0; r = b; p = 0; r.r (last
// block: the stopping threshold rtol^2 r.r, done when r = 0).
__global__ void __launch_bounds__(kPBlock) k_press_init(int32_t n_rep, int singular, double rtol2, int32_t max_it,
                                                        double* __restrict__ scal,
                                                        int32_t* __restrict__ ctl, double* __restrict__ b,
                                                        double* __restrict__ x, double* __restrict__ r,
                                                        double* __restrict__ p, double* __restrict__ q,
                                                        double* __restrict__ part) {
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  double rr = 0.0;
  if (u < n_rep) {
    const double bv = singular ? b[u] - scal[kSBsum] / (double)n_rep : b[u];
    b[u] = bv;
    x[u] = 0.0;
    r[u] = bv;
    p[u] = 0.0;
    q[u] = 0.0;
    rr = bv * bv;
  }
  const double s = pblock_sum(rr);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(ctl + kCtlCount0)) return;
  const double t = sum_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    scal[kSRr] = t;
    scal[kSRr0] = t;
    scal[kSTol2] = rtol2 * t;
    scal[kSRz] = 1.0;
    scal[kSRzOld] = 1.0;
    ctl[kCtlIters] = 0;
    ctl[kCtlMaxIt] = max_it;
    ctl[kCtlDone] = (t > 0.0 && max_it > 0) ? 0 : 1;
  }
}

// The direction and its image in one pass (q = K p by the recurrence
// K p_new = K z + beta K p_old, so no barrier between p and q): beta =
// rz / rz_old, p = z + beta p, q = K z + beta q, p . q (last block: alpha =
// rz / p.q).  p = q = 0 before the first iteration.
__global__ void __launch_bounds__(kPBlock) k_press_dirspmv(int32_t n_rep, const int32_t* __restrict__ rp,
                                                           const int32_t* __restrict__ ci,
                                                           const double* __restrict__ kval,
                                                           const double* __restrict__ z, double* __restrict__ p,
                                                           double* __restrict__ q, double* __restrict__ scal,
                                                           int32_t* __restrict__ ctl, double* __restrict__ part) {
  if (ctl[kCtlDone]) return;
  const double rz = scal[kSRz], rz_old = scal[kSRzOld];
  const double beta = rz_old != 0.0 ? rz / rz_old : 0.0;
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  double pq = 0.0;
  if (u < n_rep) {
    double kz = 0.0;
    for (int32_t k = rp[u]; k < rp[u + 1]; ++k) kz += kval[k] * z[ci[k]];
    const double pv = z[u] + beta * p[u];
    const double qv = kz + beta * q[u];
    p[u] = pv;
    q[u] = qv;
    pq = pv * qv;
  }
  const double t = pblock_sum(pq);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (!last_block(ctl + kCtlCount0)) return;
  const double v = sum_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    scal[kSPq] = v;
    scal[kSAlpha] = v > 0.0 ? rz / v : 0.0;
  }
}

// x += alpha p, r -= alpha q, r . r (last block: count the iteration and
// stop at r.r <= rtol^2 r0.r0, at max_it, or when p.q <= 0).
__global__ void __launch_bounds__(kPBlock) k_press_update(int32_t n_rep, double* __restrict__ scal,
                                                          int32_t* __restrict__ ctl, double* __restrict__ x,
                                                          double* __restrict__ r, const double* __restrict__ p,
                                                          const double* __restrict__ q, double* __restrict__ part) {
  if (ctl[kCtlDone]) return;
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  const double a = scal[kSAlpha];
  double rr = 0.0;
  if (u < n_rep) {
    x[u] += a * p[u];
    const double rv = r[u] - a * q[u];
    r[u] = rv;
    rr = rv * rv;
  }
  const double t = pblock_sum(rr);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (!last_block(ctl + kCtlCount1)) return;
  const double v = sum_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    scal[kSRr] = v;
    const int32_t it = ctl[kCtlIters] + 1;
    ctl[kCtlIters] = it;
    if (v <= scal[kSTol2] || it >= ctl[kCtlMaxIt] || !(scal[kSPq] > 0.0)) ctl[kCtlDone] = 1;
  }
}

// r . z from its partials when the hierarchy has no level: rz_old = rz,
// rz = sum.
__global__ void k_press_rz(const double* __restrict__ part, int32_t nb, double* __restrict__ scal,
                           const int32_t* __restrict__ done) {
  if (*done) return;
  double s = 0.0;
  for (int32_t i = threadIdx.x; i < nb; i += kPBlock) s += part[i];
  s = pblock_sum(s);
  if (threadIdx.x == 0) {
    scal[kSRzOld] = scal[kSRz];
    scal[kSRz] = s;
  }
}

// r . z partials when the hierarchy has no level (z = the coarse solve).
__global__ void __launch_bounds__(kPBlock) k_press_dot(int32_t n_rep, const double* __restrict__ r,
                                                       const double* __restrict__ z, double* __restrict__ part,
                                                       const int32_t* __restrict__ done) {
  if (*done) return;
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  const double s = pblock_sum(u < n_rep ? r[u] * z[u] : 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// partials of sum x (for the zero-mean normalisation)
__global__ void __launch_bounds__(kPBlock) k_press_xsum(int32_t n_rep, const double* __restrict__ x,
                                                        double* __restrict__ part) {
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  const double s = pblock_sum(u < n_rep ? x[u] : 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// dP at the nodes and <P'> += dP: the Dirichlet value at inflow/outflow
// nodes, else the solution (less its mean over the unknowns for the
// singular system).
__global__ void k_press_scatter(int32_t n_nodes, int32_t n_rep, const int32_t* __restrict__ node_rep,
                                const int8_t* __restrict__ dir, const double* __restrict__ x,
                                const double* __restrict__ xsum, const double* __restrict__ ns, double PiLx,
                                double* __restrict__ dP, double* __restrict__ pres) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    const int32_t u = node_rep[n];
    double v;
    if (dir != nullptr && dir[u] != 0)
      v = dirichlet_dP(dir[u], n, ns, pres, PiLx);
    else
      v = x[u] - (xsum ? *xsum / (double)n_rep : 0.0);
    dP[n] = v;
    pres[n] += v;
  }
}

// Element gradient of a nodal field: g[e] = (d/dx, d/dy).
__global__ void k_press_egrad(int32_t n_tri, const int32_t* __restrict__ tri, const double* __restrict__ dN,
                              const double* __restrict__ f, double* __restrict__ g) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    const double* d = dN + (int64_t)e * 6;
    double gx = 0.0, gy = 0.0;
    for (int j = 0; j < 3; ++j) {
      const double v = f[tri[3 * e + j]];
      gx += d[j] * v;
      gy += d[3 + j] * v;
    }
    g[2 * (int64_t)e] = gx;
    g[2 * (int64_t)e + 1] = gy;
  }
}

// Nodal gradient: the mean of the surrounding elements' gradients (twins merged).
__global__ void k_press_ngrad(int32_t n_nodes, const int32_t* __restrict__ nse_off, const int32_t* __restrict__ nse,
                              const double* __restrict__ ge, double* __restrict__ gn) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    double gx = 0.0, gy = 0.0;
    const int32_t b = nse_off[n], c = nse_off[n + 1] - b;
    for (int32_t i = b; i < b + c; ++i) {
      gx += ge[2 * (int64_t)nse[i]];
      gy += ge[2 * (int64_t)nse[i] + 1];
    }
    const double inv = 1.0 / (c > 0 ? (double)c : 1.0);
    gn[2 * (int64_t)n] = gx * inv;
    gn[2 * (int64_t)n + 1] = gy * inv;
  }
}

// The correction shifts every particle of an element by the same vector, so
// the element means <U>, <V> shift by it and the central moments (and the
// velocity ranks the conditional means bin by) stay as they are.
__global__ void k_press_shift_stats(int32_t n_tri, const double* __restrict__ gdp, double dt, double* __restrict__ es) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    double* s = es + (int64_t)e * PDF_NES;
    if (s[0] <= 0.0) continue;
    s[1] -= dt * gdp[2 * (int64_t)e];
    s[2] -= dt * gdp[2 * (int64_t)e + 1];
  }
}

// The correction of an element, -dt grad dP, as double-float pairs
// (x.h, x.l, y.h, y.l), so that the particle pass needs no FP64.
__global__ void k_press_corr_coef(int32_t n_tri, const double* __restrict__ gdp, double dt, float4* __restrict__ gc) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    const fx::df cx = fx::from_double(-dt * gdp[2 * (int64_t)e]);
    const fx::df cy = fx::from_double(-dt * gdp[2 * (int64_t)e + 1]);
    gc[e] = make_float4(cx.h, cx.l, cy.h, cy.l);
  }
}

// Velocity correction of every particle: U += -dt grad dP of its element
// (double-float addition; FP32 state: the nearest float of the sum).
template <typename T>
__global__ void k_press_correct(int64_t n, const int32_t* __restrict__ elem, const float4* __restrict__ gc,
                                T* __restrict__ u, T* __restrict__ v);

template <>
__global__ void k_press_correct<fx::df>(int64_t n, const int32_t* __restrict__ elem, const float4* __restrict__ gc,
                                        fx::df* __restrict__ u, fx::df* __restrict__ v) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float4 c = __ldg(gc + elem[p]);
  u[p] = fx::add(u[p], fx::df{c.x, c.y});
  v[p] = fx::add(v[p], fx::df{c.z, c.w});
}

template <>
__global__ void k_press_correct<float>(int64_t n, const int32_t* __restrict__ elem, const float4* __restrict__ gc,
                                       float* __restrict__ u, float* __restrict__ v) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float4 c = __ldg(gc + elem[p]);
  u[p] = fx::add(fx::df{u[p], 0.f}, fx::df{c.x, c.y}).h;
  v[p] = fx::add(fx::df{v[p], 0.f}, fx::df{c.z, c.w}).h;
}

static int pblocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

static int32_t nblocks(int32_t n) { return (n + kPBlock - 1) / kPBlock; }

// Work vectors for up to n_nodes unknowns, control words, the library's
// stream and events.
static pdf_status press_alloc(pdf_particles* P) {
  PressWork& W = P->pw;
  if (W.x) return PDF_OK;
  const pdf_mesh* m = P->mesh;
  const int32_t nn = m->d.n_nodes, nt = m->d.n_tri;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void**)&W.b, sizeof(double) * nn);
  A((void**)&W.x, sizeof(double) * nn);
  A((void**)&W.r, sizeof(double) * nn);
  A((void**)&W.z, sizeof(double) * nn);
  A((void**)&W.p, sizeof(double) * nn);
  A((void**)&W.q, sizeof(double) * nn);
  A((void**)&W.part, sizeof(double) * 4 * nblocks(nn));
  A((void**)&W.scal, sizeof(double) * 16);
  A((void**)&W.dP, sizeof(double) * nn);
  A((void**)&W.ge, sizeof(double) * 2 * nt);
  A((void**)&W.gc, sizeof(float4) * nt);
  A((void**)&W.ctl, sizeof(int32_t) * 8);
  if (e == cudaSuccess) e = cudaMemset(W.ctl, 0, sizeof(int32_t) * 8);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&W.host, sizeof(double) * 16);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&W.host_ctl, sizeof(int32_t) * 8);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&W.cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W.ev0, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W.ev1, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    press_free(W);
    return cuda_fail(e, "pdf_pressure_project: allocation");
  }
  return PDF_OK;
}

static void sys_free(PressSys& S) {
  if (S.own) {
    cudaFree(S.rp); cudaFree(S.ci); cudaFree(S.rep_node); cudaFree(S.node_rep);
    cudaFree(S.pw_off); cudaFree(S.pw_e); cudaFree(S.pw_n); cudaFree(S.dir); cudaFree(S.kmask);
  }
  cudaFree(S.kval); cudaFree(S.gw); cudaFree(S.gw_prev);
  if (S.amg) {
    amg_free(*S.amg);
    delete S.amg;
  }
  if (S.gx) cudaGraphExecDestroy(S.gx);
  S = PressSys();
}

void press_free(PressWork& W) {
  for (PressSys& S : W.sys) sys_free(S);
  cudaFree(W.b); cudaFree(W.x); cudaFree(W.r); cudaFree(W.z);
  cudaFree(W.p); cudaFree(W.q); cudaFree(W.part); cudaFree(W.scal); cudaFree(W.dP); cudaFree(W.ge);
  cudaFree(W.ctl); cudaFree(W.gc);
  if (W.host) cudaFreeHost(W.host);
  if (W.host_ctl) cudaFreeHost(W.host_ctl);
  if (W.ev0) cudaEventDestroy(W.ev0);
  if (W.ev1) cudaEventDestroy(W.ev1);
  if (W.cs) cudaStreamDestroy(W.cs);
  W = PressWork();
}

template <typename T>
static pdf_status up(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(src.size(), 1) * sizeof(T));
  if (e == cudaSuccess && !src.empty())
    e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? PDF_OK : cuda_fail(e, "pdf_pressure_project: upload");
}

// System 0: the relaxation's unknowns (every twin pair merged), K with the
// natural conditions, singular (constants).
static pdf_status build_periodic(const pdf_mesh* m, PressSys& S) {
  const RelaxMesh& R = m->rx;
  S.own = false;
  S.dirichlet = false;
  S.n = R.n_rep;
  S.nnz = R.nnz;
  S.rp = R.rp; S.ci = R.ci; S.rep_node = R.rep_node; S.node_rep = R.node_rep;
  S.pw_off = R.pw_off; S.pw_e = R.pw_e; S.pw_n = R.pw_n;
  S.dir = nullptr;
  pdf_status s = up(&S.kval, m->k_v);
  if (s != PDF_OK) return s;
  S.kmask = S.kval;
  S.amg = new Amg();
  return amg_setup(S.n, m->k_rp, m->k_ci, m->k_v, true, *S.amg);
}

// System 1: twins merged except the inflow/outflow pairs, whose nodes are
// Dirichlet unknowns (the street canyon's inflow/outflow condition).
static pdf_status build_inout(const pdf_mesh* m, PressSys& S) {
  const int32_t nn = m->d.n_nodes, nt = m->d.n_tri;
  const int32_t* T = m->tri.data();
  const double* X = m->xy.data();
  std::vector<int32_t> rep_of(nn), idx(nn, -1), rep_node, node_rep(nn);
  for (int32_t n = 0; n < nn; ++n) {
    const int32_t t = m->twin[n];
    const bool split = t >= 0 && m->inout[n] != 0 && m->inout[t] != 0;
    rep_of[n] = (t >= 0 && !split) ? std::min(n, t) : n;
  }
  for (int32_t n = 0; n < nn; ++n)
    if (rep_of[n] == n) { idx[n] = (int32_t)rep_node.size(); rep_node.push_back(n); }
  for (int32_t n = 0; n < nn; ++n) node_rep[n] = idx[rep_of[n]];
  const int32_t nr = (int32_t)rep_node.size();
  std::vector<int8_t> dir(nr);
  int32_t n_dir = 0;
  for (int32_t u = 0; u < nr; ++u) {
    dir[u] = m->inout[rep_node[u]];
    n_dir += dir[u] != 0;
  }
  if (n_dir == 0) return fail(PDF_EINVAL, "pdf_pressure_project: the mesh has no inflow/outflow edges");
  // pattern and values, K_ab = sum_e A_e grad N_a . grad N_b
  std::vector<std::vector<std::pair<int32_t, double>>> rows(nr);
  for (int32_t e = 0; e < nt; ++e) {
    const double* d = &m->dN[6 * (size_t)e];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        rows[node_rep[T[3 * e + a]]].push_back(
            {node_rep[T[3 * e + b]], m->area[e] * (d[a] * d[b] + d[3 + a] * d[3 + b])});
  }
  std::vector<int32_t> rp(nr + 1, 0), ci;
  std::vector<double> kv, km;
  for (int32_t u = 0; u < nr; ++u) {
    auto& r = rows[u];
    std::stable_sort(r.begin(), r.end(), [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
      return x.first < y.first;
    });
    for (size_t i = 0; i < r.size();) {
      const int32_t c = r[i].first;
      double v = 0.0;
      for (; i < r.size() && r[i].first == c; ++i) v += r[i].second;
      ci.push_back(c);
      kv.push_back(v);
      km.push_back(dir[u] != 0 ? (c == u ? 1.0 : 0.0) : (dir[c] != 0 ? 0.0 : v));
    }
    rp[u + 1] = (int32_t)ci.size();
    if (rp[u + 1] - rp[u] > 64) return fail(PDF_EINVAL, "pdf_pressure_project: pressure row out of range");
  }
  // wall edges at each unknown
  std::vector<std::vector<int32_t>> pwl(nr);
  std::vector<int32_t> we;
  std::vector<double> wn;
  for (int32_t e = 0; e < nt; ++e)
    for (int k = 0; k < 3; ++k) {
      const int32_t c = m->nbr[3 * e + k];
      if (c != kNbrWall && c != kNbrNoslip) continue;
      const int32_t a = T[3 * e + (k + 1) % 3], b = T[3 * e + (k + 2) % 3];
      const int32_t id = (int32_t)(we.size() / 3);
      we.insert(we.end(), {e, a, b});
      const double tx = X[2 * b] - X[2 * a], ty = X[2 * b + 1] - X[2 * a + 1];
      const double len = std::sqrt(tx * tx + ty * ty);
      wn.insert(wn.end(), {ty / len, -tx / len, len});
      pwl[node_rep[a]].push_back(id);
      pwl[node_rep[b]].push_back(id);
    }
  std::vector<int32_t> pw_off(nr + 1, 0), pw_e;
  std::vector<double> pw_n;
  for (int32_t u = 0; u < nr; ++u) {
    pw_off[u + 1] = pw_off[u] + (int32_t)pwl[u].size();
    for (int32_t id : pwl[u]) {
      pw_e.insert(pw_e.end(), we.begin() + 3 * id, we.begin() + 3 * id + 3);
      pw_n.insert(pw_n.end(), wn.begin() + 3 * id, wn.begin() + 3 * id + 3);
    }
  }
  S.own = true;
  S.dirichlet = true;
  S.n = nr;
  S.nnz = (int64_t)ci.size();
  pdf_status s;
  if ((s = up(&S.rp, rp)) != PDF_OK || (s = up(&S.ci, ci)) != PDF_OK || (s = up(&S.rep_node, rep_node)) != PDF_OK ||
      (s = up(&S.node_rep, node_rep)) != PDF_OK || (s = up(&S.pw_off, pw_off)) != PDF_OK ||
      (s = up(&S.pw_e, pw_e)) != PDF_OK || (s = up(&S.pw_n, pw_n)) != PDF_OK || (s = up(&S.dir, dir)) != PDF_OK ||
      (s = up(&S.kval, kv)) != PDF_OK || (s = up(&S.kmask, km)) != PDF_OK)
    return s;
  S.amg = new Amg();
  return amg_setup(nr, rp, ci, km, false, *S.amg);
}

static pdf_status sys_get(pdf_particles* P, int k, PressSys** out) {
  PressSys& S = P->pw.sys[k];
  if (!S.built) {
    pdf_status s = k == 0 ? build_periodic(P->mesh, S) : build_inout(P->mesh, S);
    if (s == PDF_OK) {
      cudaError_t e = cudaMalloc((void**)&S.gw, sizeof(double) * std::max(S.n, 1));
      if (e == cudaSuccess) e = cudaMalloc((void**)&S.gw_prev, sizeof(double) * std::max(S.n, 1));
      if (e == cudaSuccess) e = cudaMemset(S.gw_prev, 0, sizeof(double) * std::max(S.n, 1));
      if (e != cudaSuccess) s = cuda_fail(e, "pdf_pressure_project: allocation");
    }
    if (s != PDF_OK) {
      sys_free(S);
      return s;
    }
    S.built = true;
  }
  *out = &S;
  return PDF_OK;
}

static PSys dev_view(const PressSys& S) {
  return PSys{S.n, S.rp, S.ci, S.rep_node, S.pw_off, S.pw_e, S.kval, S.pw_n, S.dir};
}

// k preconditioned conjugate-gradient iterations (each kernel returns at
// once after the stop).
static pdf_status press_iterations(PressWork& W, const PressSys& S, int k, cudaStream_t st) {
  const Amg& G = *S.amg;
  const int nb = nblocks(S.n);
  const int32_t* done = W.ctl + kCtlDone;
  for (int i = 0; i < k; ++i) {
    pdf_status s = amg_apply(G, W.r, W.z, W.part, W.ctl + kCtlCount1, W.scal + kSRz, W.scal + kSRzOld, done, st);
    if (s != PDF_OK) return s;
    if (G.lv.empty()) {
      PDF_KERNEL("k_press_dot", st, k_press_dot<<<nb, kPBlock, 0, st>>>(S.n, W.r, W.z, W.part, done));
      PDF_KERNEL("k_press_rz", st, k_press_rz<<<1, kPBlock, 0, st>>>(W.part, nb, W.scal, done));
    }
    PDF_KERNEL("k_press_dirspmv", st, k_press_dirspmv<<<nb, kPBlock, 0, st>>>(S.n, S.rp, S.ci, S.kmask, W.z, W.p, W.q,
                                                                               W.scal, W.ctl, W.part + nb));
    PDF_KERNEL("k_press_update", st, k_press_update<<<nb, kPBlock, 0, st>>>(S.n, W.scal, W.ctl, W.x, W.r, W.p, W.q,
                                                                             W.part + 2 * nb));
  }
  return PDF_OK;
}

// Captures k iterations of system S into S.gx on the library's stream.
static pdf_status press_capture(PressWork& W, PressSys& S, int k) {
  const long long n0 = prof_launches();
  PDF_CUDA(cudaStreamBeginCapture(W.cs, cudaStreamCaptureModeThreadLocal));
  pdf_status s = press_iterations(W, S, k, W.cs);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(W.cs, &g);
  if (s != PDF_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "pdf_pressure_project: graph capture");
  const cudaError_t e2 = cudaGraphInstantiate(&S.gx, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    S.gx = nullptr;
    return cuda_fail(e2, "pdf_pressure_project: graph instantiation");
  }
  S.graph_launches = prof_launches() - n0;
  prof_count(-S.graph_launches);  // captured, not launched
  return PDF_OK;
}

// Nodal gradient of <P'> for the projection modes of the step.
static pdf_status press_gradient(pdf_particles* P, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  PressWork& W = P->pw;
  PDF_KERNEL("k_press_egrad", st, k_press_egrad<<<pblocks(M.n_tri), 256, 0, st>>>(M.n_tri, M.tri, M.dN, P->pres, W.ge));
  PDF_KERNEL("k_press_ngrad", st, k_press_ngrad<<<pblocks(M.n_nodes), 256, 0, st>>>(M.n_nodes, M.nse_off, M.nse, W.ge,
                                                                                      P->gradP));
  return PDF_OK;
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_pressure_project(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                                           double Cp, double rtol, int32_t max_it, int32_t* iters, double* rel_res,
                                           void* stream) {
  if (!p || !m || p->mesh != m || !params) return fail(PDF_EINVAL, "pdf_pressure_project: bad arguments");
  if (!(rtol > 0.0) || max_it < 0 || !(Cp >= 0.0) || !(params->dt > 0.0))
    return fail(PDF_EINVAL, "pdf_pressure_project: rtol > 0, max_it >= 0, Cp >= 0 and dt > 0 required");
  if (params->pressure != PDF_PRESSURE_PROJECTION && params->pressure != PDF_PRESSURE_PROJECTION_INOUT)
    return fail(PDF_EINVAL, "pdf_pressure_project: params->pressure must be a projection mode");
  if (!p->have_stats) return fail(PDF_ESTATE, "pdf_pressure_project: call pdf_estimate_stats first");
  cudaStream_t st = (cudaStream_t)stream;
  pdf_status s = press_alloc(p);
  if (s != PDF_OK) return s;
  PressWork& W = p->pw;
  const int k = params->pressure == PDF_PRESSURE_PROJECTION_INOUT ? 1 : 0;
  PressSys* Sp = nullptr;
  s = sys_get(p, k, &Sp);
  if (s != PDF_OK) return s;
  PressSys& S = *Sp;
  if (W.last_sys != k) {
    // the stored wall load belongs to the field the other system made
    PDF_CUDA(cudaMemsetAsync(S.gw_prev, 0, sizeof(double) * std::max(S.n, 1), st));
    W.last_sys = k;
  }
  const MeshDev& M = m->d;
  const int nb = nblocks(S.n);
  const double PiLx = params->Pi * m->period;
  PDF_KERNEL("k_press_rhs", st, k_press_rhs<<<nb, kPBlock, 0, st>>>(dev_view(S), M.nse_off, M.nse, M.tri, M.dN, M.geo,
                                                                     p->ns, p->nd, params->nu,
                                                                     params->closure == PDF_CLOSURE_SLM, p->pres,
                                                                     S.gw_prev, Cp, 1.0 / params->dt, PiLx, S.gw, W.b,
                                                                     W.part));
  PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part, nb, W.scal + kSBsum));
  PDF_KERNEL("k_press_init", st, k_press_init<<<nb, kPBlock, 0, st>>>(S.n, S.dirichlet ? 0 : 1, rtol * rtol, max_it,
                                                                       W.scal, W.ctl, W.b, W.x, W.r, W.p, W.q, W.part));
  // the iteration: chunks of separate kernels (the host reads the control
  // words once per chunk), or one persistent cooperative kernel when asked
  // for and the device can launch it
  constexpr int kChunk = 8;
  bool coop = false;
  if (W.persistent) {
    s = amg_pcg(*S.amg, S.n, S.rp, S.ci, S.kmask, W.x, W.r, W.z, W.p, W.q, W.scal, W.ctl, W.part,
                4 * nblocks(m->d.n_nodes), st);
    coop = s == PDF_OK;
    if (!coop) W.persistent = false;
  }
  if (coop) {
    // nothing else to launch
  } else if (prof_timing()) {
    for (int launched = 0; launched < max_it; launched += kChunk) {
      s = press_iterations(W, S, kChunk, st);
      if (s != PDF_OK) return s;
      PDF_CUDA(cudaMemcpyAsync(W.host_ctl, W.ctl, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
      PDF_CUDA(cudaStreamSynchronize(st));
      if (W.host_ctl[kCtlDone]) break;
    }
  } else {
    if (!S.gx) {
      s = press_capture(W, S, kChunk);
      if (s != PDF_OK) return s;
    }
    PDF_CUDA(cudaEventRecord(W.ev0, st));
    PDF_CUDA(cudaStreamWaitEvent(W.cs, W.ev0, 0));
    for (int launched = 0; launched < max_it; launched += kChunk) {
      PDF_CUDA(cudaGraphLaunch(S.gx, W.cs));
      prof_count(S.graph_launches);
      PDF_CUDA(cudaMemcpyAsync(W.host_ctl, W.ctl, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, W.cs));
      PDF_CUDA(cudaStreamSynchronize(W.cs));
      if (W.host_ctl[kCtlDone]) break;
    }
    PDF_CUDA(cudaEventRecord(W.ev1, W.cs));
    PDF_CUDA(cudaStreamWaitEvent(st, W.ev1, 0));
  }
  PDF_CUDA(cudaMemcpyAsync(W.host, W.scal, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaMemcpyAsync(W.host_ctl, W.ctl, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaStreamSynchronize(st));
  const int it = W.host_ctl[kCtlIters];
  const double bn = std::sqrt(W.host[kSRr0]);
  const double rn = std::sqrt(W.host[kSRr]);
  const bool converged = W.host[kSRr] <= W.host[kSTol2];
  if (iters) *iters = it;
  if (rel_res) *rel_res = bn > 0.0 ? rn / bn : 0.0;
  if (!S.dirichlet) {
    PDF_KERNEL("k_press_xsum", st, k_press_xsum<<<nb, kPBlock, 0, st>>>(S.n, W.x, W.part));
    PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part, nb, W.scal + kSXsum));
  }
  PDF_KERNEL("k_press_scatter", st, k_press_scatter<<<pblocks(M.n_nodes), 256, 0, st>>>(
                                        M.n_nodes, S.n, S.node_rep, S.dir, W.x, S.dirichlet ? nullptr : W.scal + kSXsum,
                                        p->ns, PiLx, W.dP, p->pres));
  std::swap(S.gw, S.gw_prev);  // <P'>^{n+1} satisfies the new wall load
  // velocity correction with the element gradients of dP
  PDF_KERNEL("k_press_egrad", st, k_press_egrad<<<pblocks(M.n_tri), 256, 0, st>>>(M.n_tri, M.tri, M.dN, W.dP, W.ge));
  PDF_KERNEL("k_press_corr_coef", st, k_press_corr_coef<<<pblocks(M.n_tri), 256, 0, st>>>(M.n_tri, W.ge, params->dt,
                                                                                            W.gc));
  const unsigned pb = (unsigned)std::max<int64_t>(1, (p->n + 255) / 256);
  if (p->precision == PDF_FP64)
    PDF_KERNEL("k_press_correct", st, k_press_correct<fx::df><<<pb, 256, 0, st>>>(p->n, p->elem, W.gc, p->u, p->v));
  else
    PDF_KERNEL("k_press_correct", st, k_press_correct<float><<<pb, 256, 0, st>>>(p->n, p->elem, W.gc, p->uf, p->vf));
  // the statistics follow the correction (W.ge still holds grad dP)
  PDF_KERNEL("k_press_shift_stats", st, k_press_shift_stats<<<pblocks(M.n_tri), 256, 0, st>>>(M.n_tri, W.ge, params->dt,
                                                                                                p->es));
  s = press_gradient(p, st);
  if (s != PDF_OK) return s;
  s = node_stats_from_elements(p, st);
  if (s != PDF_OK) return s;
  if (!converged) return fail(PDF_ENOTCONV, "pdf_pressure_project: not converged");
  return PDF_OK;
}

extern "C" pdf_status pdf_pressure_set_solver(pdf_particles* p, int32_t persistent) {
  if (!p || (persistent != 0 && persistent != 1)) return fail(PDF_EINVAL, "pdf_pressure_set_solver: bad arguments");
  p->pw.persistent = persistent != 0;
  return PDF_OK;
}

extern "C" pdf_status pdf_pressure_field(pdf_particles* p, const double* set, double* get, void* stream) {
  if (!p) return fail(PDF_EINVAL, "pdf_pressure_field: NULL handle");
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t nn = p->mesh->d.n_nodes;
  if (set) {
    pdf_status s = press_alloc(p);
    if (s != PDF_OK) return s;
    PDF_CUDA(cudaMemcpyAsync(p->pres, set, sizeof(double) * nn, cudaMemcpyDefault, st));
    for (PressSys& S : p->pw.sys)
      if (S.built) PDF_CUDA(cudaMemsetAsync(S.gw_prev, 0, sizeof(double) * std::max(S.n, 1), st));
    s = press_gradient(p, st);
    if (s != PDF_OK) return s;
  }
  if (get) PDF_CUDA(cudaMemcpyAsync(get, p->pres, sizeof(double) * nn, cudaMemcpyDefault, st));
  return PDF_OK;
}

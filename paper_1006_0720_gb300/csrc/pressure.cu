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
// solved by Jacobi-preconditioned conjugate gradients in FP64 from zero; dP
// is normalised to zero mean.  The particles' velocities are corrected by
// -dt grad dP of their element.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace pdfgb {

pdf_status estimate_stats(pdf_particles* P, cudaStream_t st);

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

// K values (the relaxation pattern's stiffness contributions without L^2)
// and the diagonal.
__global__ void k_press_kval(int64_t nnz, const int32_t* __restrict__ ctb_off, const double* __restrict__ ctb_k,
                             double* __restrict__ kval) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t t = ctb_off[q]; t < ctb_off[q + 1]; ++t) s += ctb_k[t];
    kval[q] = s;
  }
}

__global__ void k_press_diag(int32_t n_rep, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ kval, double* __restrict__ diag) {
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rep; r += gridDim.x * blockDim.x) {
    double d = 1.0;
    for (int32_t q = rp[r]; q < rp[r + 1]; ++q)
      if (ci[q] == r) d = kval[q];
    diag[r] = d > 0.0 ? d : 1.0;
  }
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

// b_u = -(d_u + C_p ((K <P'>)_u - G_u^n)) / dt + G_u^{n+1} - G_u^n:
// d_u = sum over the elements around the unknown's node(s) of A_e / 3 times
// the element divergence of the nodal <U>, <V>; G the wall load above (G^n
// the one the current <P'> satisfies, G^{n+1} from the present statistics,
// written to gw).  Block partials of sum b.
__global__ void __launch_bounds__(kPBlock) k_press_rhs(
    int32_t n_rep, const int32_t* __restrict__ rep_node, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const double* __restrict__ kval, const int32_t* __restrict__ nse_off,
    const int32_t* __restrict__ nse, const int32_t* __restrict__ tri, const double* __restrict__ dN,
    const ElemGeo* __restrict__ geo, const double* __restrict__ ns, const double* __restrict__ nd,
    const int32_t* __restrict__ pw_off, const int32_t* __restrict__ pw_e, const double* __restrict__ pw_n, double nu,
    int slm, const double* __restrict__ pres, const double* __restrict__ gw_prev, double Cp, double inv_dt,
    double* __restrict__ gw, double* __restrict__ b, double* __restrict__ part) {
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  double bv = 0.0;
  if (u < n_rep) {
    const int32_t n = rep_node[u];
    double d = 0.0;
    for (int32_t i = nse_off[n]; i < nse_off[n + 1]; ++i) {
      const int32_t e = nse[i];
      const double* g = dN + (int64_t)e * 6;
      double div = 0.0;
      for (int j = 0; j < 3; ++j) {
        const double* S = ns + (int64_t)tri[3 * e + j] * PDF_NNS;
        div += g[j] * S[0] + g[3 + j] * S[1];
      }
      d += 0.5 * geo[e].two_area / 3.0 * div;
    }
    double kp = 0.0;
    for (int32_t q = rp[u]; q < rp[u + 1]; ++q) kp += kval[q] * pres[rep_node[ci[q]]];
    double gn = 0.0;
    for (int32_t i = pw_off[u]; i < pw_off[u + 1]; ++i)
      gn += wall_load(pw_e + 3 * (int64_t)i, pw_n + 3 * (int64_t)i, tri, dN, ns, nd, nu, slm != 0);
    const double gp = gw_prev[u];
    gw[u] = gn;
    bv = -(d + Cp * (kp - gp)) * inv_dt + (gn - gp);
    b[u] = bv;
  }
  const double s = pblock_sum(bv);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_press_sum(const double* __restrict__ part, int32_t nb, double* __restrict__ out) {
  double s = 0.0;
  for (int32_t i = threadIdx.x; i < nb; i += kPBlock) s += part[i];
  s = pblock_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// b -= mean(b); x = 0; r = b; z = r / diag; p = z; partials of r.z, r.r.
__global__ void __launch_bounds__(kPBlock) k_press_init(int32_t n_rep, const double* __restrict__ bsum,
                                                        const double* __restrict__ diag, double* __restrict__ b,
                                                        double* __restrict__ x, double* __restrict__ r,
                                                        double* __restrict__ z, double* __restrict__ p,
                                                        double* __restrict__ part) {
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (u < n_rep) {
    const double bv = b[u] - *bsum / (double)n_rep;
    b[u] = bv;
    x[u] = 0.0;
    r[u] = bv;
    const double zz = bv / diag[u];
    z[u] = zz;
    p[u] = zz;
    rz = bv * zz;
    rr = bv * bv;
  }
  const double s1 = pblock_sum(rz), s2 = pblock_sum(rr);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[gridDim.x + blockIdx.x] = s2;
  }
}

__global__ void __launch_bounds__(kPBlock) k_press_spmv(int32_t n_rep, const int32_t* __restrict__ rp,
                                                        const int32_t* __restrict__ ci, const double* __restrict__ kval,
                                                        const double* __restrict__ p, double* __restrict__ q,
                                                        double* __restrict__ part) {
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  double pq = 0.0;
  if (u < n_rep) {
    double s = 0.0;
    for (int32_t k = rp[u]; k < rp[u + 1]; ++k) s += kval[k] * p[ci[k]];
    q[u] = s;
    pq = s * p[u];
  }
  const double t = pblock_sum(pq);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// scal[0] = p.q, scal[1] = r.z (old): x += a p, r -= a q, z = r / diag.
__global__ void __launch_bounds__(kPBlock) k_press_update(int32_t n_rep, const double* __restrict__ scal,
                                                          const double* __restrict__ diag, double* __restrict__ x,
                                                          double* __restrict__ r, double* __restrict__ z,
                                                          const double* __restrict__ p, const double* __restrict__ q,
                                                          double* __restrict__ part) {
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (u < n_rep) {
    const double a = scal[0] != 0.0 ? scal[1] / scal[0] : 0.0;
    x[u] += a * p[u];
    const double rv = r[u] - a * q[u];
    r[u] = rv;
    const double zz = rv / diag[u];
    z[u] = zz;
    rz = rv * zz;
    rr = rv * rv;
  }
  const double s1 = pblock_sum(rz), s2 = pblock_sum(rr);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[gridDim.x + blockIdx.x] = s2;
  }
}

__global__ void k_press_dir(int32_t n_rep, double beta, const double* __restrict__ z, double* __restrict__ p) {
  for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n_rep; u += gridDim.x * blockDim.x)
    p[u] = z[u] + beta * p[u];
}

// partials of sum x (for the zero-mean normalisation)
__global__ void __launch_bounds__(kPBlock) k_press_xsum(int32_t n_rep, const double* __restrict__ x,
                                                        double* __restrict__ part) {
  const int32_t u = blockIdx.x * kPBlock + threadIdx.x;
  const double s = pblock_sum(u < n_rep ? x[u] : 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// dP at the nodes (zero mean over the unknowns) and <P'> += dP.
__global__ void k_press_scatter(int32_t n_nodes, int32_t n_rep, const int32_t* __restrict__ node_rep,
                                const double* __restrict__ x, const double* __restrict__ xsum,
                                double* __restrict__ dP, double* __restrict__ pres) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    const double v = x[node_rep[n]] - *xsum / (double)n_rep;
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

// Velocity correction of every particle: U -= dt grad dP of its element.
template <typename T>
__global__ void k_press_correct(int64_t n, const int32_t* __restrict__ elem, const double* __restrict__ gdp,
                                double dt, T* __restrict__ u, T* __restrict__ v);

template <>
__global__ void k_press_correct<fx::df>(int64_t n, const int32_t* __restrict__ elem, const double* __restrict__ gdp,
                                        double dt, fx::df* __restrict__ u, fx::df* __restrict__ v) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = elem[p];
    u[p] = fx::from_double(fx::to_double(u[p]) - dt * gdp[2 * e]);
    v[p] = fx::from_double(fx::to_double(v[p]) - dt * gdp[2 * e + 1]);
  }
}

template <>
__global__ void k_press_correct<float>(int64_t n, const int32_t* __restrict__ elem, const double* __restrict__ gdp,
                                       double dt, float* __restrict__ u, float* __restrict__ v) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = elem[p];
    u[p] = (float)((double)u[p] - dt * gdp[2 * e]);
    v[p] = (float)((double)v[p] - dt * gdp[2 * e + 1]);
  }
}

static int pblocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

static pdf_status press_alloc(pdf_particles* P) {
  PressWork& W = P->pw;
  if (W.x) return PDF_OK;
  const RelaxMesh& R = P->mesh->rx;
  const int32_t nn = P->mesh->d.n_nodes, nt = P->mesh->d.n_tri;
  W.nb = (R.n_rep + kPBlock - 1) / kPBlock;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void**)&W.kval, sizeof(double) * R.nnz);
  A((void**)&W.diag, sizeof(double) * R.n_rep);
  A((void**)&W.b, sizeof(double) * R.n_rep);
  A((void**)&W.x, sizeof(double) * R.n_rep);
  A((void**)&W.r, sizeof(double) * R.n_rep);
  A((void**)&W.z, sizeof(double) * R.n_rep);
  A((void**)&W.p, sizeof(double) * R.n_rep);
  A((void**)&W.q, sizeof(double) * R.n_rep);
  A((void**)&W.part, sizeof(double) * 2 * W.nb);
  A((void**)&W.scal, sizeof(double) * 8);
  A((void**)&W.dP, sizeof(double) * nn);
  A((void**)&W.ge, sizeof(double) * 2 * nt);
  A((void**)&W.gw, sizeof(double) * R.n_rep);
  A((void**)&W.gw_prev, sizeof(double) * R.n_rep);
  if (e == cudaSuccess) e = cudaMemset(W.gw_prev, 0, sizeof(double) * R.n_rep);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&W.host, sizeof(double) * 8);
  if (e != cudaSuccess) return cuda_fail(e, "pdf_pressure_project: allocation");
  return PDF_OK;
}

void press_free(PressWork& W) {
  cudaFree(W.kval); cudaFree(W.diag); cudaFree(W.b); cudaFree(W.x); cudaFree(W.r); cudaFree(W.z);
  cudaFree(W.p); cudaFree(W.q); cudaFree(W.part); cudaFree(W.scal); cudaFree(W.dP); cudaFree(W.ge);
  cudaFree(W.gw); cudaFree(W.gw_prev);
  if (W.host) cudaFreeHost(W.host);
  W = PressWork();
}

// Nodal gradient of <P'> for PDF_PRESSURE_PROJECTION steps.
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
  if (!p->have_stats) return fail(PDF_ESTATE, "pdf_pressure_project: call pdf_estimate_stats first");
  cudaStream_t st = (cudaStream_t)stream;
  pdf_status s = press_alloc(p);
  if (s != PDF_OK) return s;
  const MeshDev& M = m->d;
  const RelaxMesh& R = m->rx;
  PressWork& W = p->pw;
  const int nb = W.nb;
  if (!W.have_k) {
    PDF_KERNEL("k_press_kval", st, k_press_kval<<<pblocks(R.nnz), 256, 0, st>>>(R.nnz, R.ctb_off, R.ctb_k, W.kval));
    PDF_KERNEL("k_press_diag", st, k_press_diag<<<pblocks(R.n_rep), 256, 0, st>>>(R.n_rep, R.rp, R.ci, W.kval, W.diag));
    W.have_k = true;
  }
  PDF_KERNEL("k_press_rhs", st, k_press_rhs<<<nb, kPBlock, 0, st>>>(R.n_rep, R.rep_node, R.rp, R.ci, W.kval, M.nse_off,
                                                                     M.nse, M.tri, M.dN, M.geo, p->ns, p->nd, R.pw_off,
                                                                     R.pw_e, R.pw_n, params->nu,
                                                                     params->closure == PDF_CLOSURE_SLM, p->pres,
                                                                     W.gw_prev, Cp, 1.0 / params->dt, W.gw, W.b,
                                                                     W.part));
  PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part, nb, W.scal + 4));
  PDF_KERNEL("k_press_init", st, k_press_init<<<nb, kPBlock, 0, st>>>(R.n_rep, W.scal + 4, W.diag, W.b, W.x, W.r, W.z,
                                                                       W.p, W.part));
  PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part, nb, W.scal + 1));
  PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part + nb, nb, W.scal + 2));
  PDF_CUDA(cudaMemcpyAsync(W.host, W.scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaStreamSynchronize(st));
  double rz = W.host[1];
  const double bn = std::sqrt(W.host[2]);
  double rn = bn;
  int it = 0;
  while (rn > rtol * bn && bn > 0.0 && it < max_it) {
    PDF_KERNEL("k_press_spmv", st, k_press_spmv<<<nb, kPBlock, 0, st>>>(R.n_rep, R.rp, R.ci, W.kval, W.p, W.q, W.part));
    PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part, nb, W.scal));
    PDF_KERNEL("k_press_update", st, k_press_update<<<nb, kPBlock, 0, st>>>(R.n_rep, W.scal, W.diag, W.x, W.r, W.z, W.p,
                                                                             W.q, W.part));
    PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part, nb, W.scal + 1));
    PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part + nb, nb, W.scal + 2));
    PDF_CUDA(cudaMemcpyAsync(W.host, W.scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    PDF_CUDA(cudaStreamSynchronize(st));
    ++it;
    const double rzn = W.host[1];
    rn = std::sqrt(W.host[2]);
    const double beta = rz != 0.0 ? rzn / rz : 0.0;
    rz = rzn;
    if (rn > rtol * bn)
      PDF_KERNEL("k_press_dir", st, k_press_dir<<<pblocks(R.n_rep), 256, 0, st>>>(R.n_rep, beta, W.z, W.p));
  }
  if (iters) *iters = it;
  if (rel_res) *rel_res = bn > 0.0 ? rn / bn : 0.0;
  PDF_KERNEL("k_press_xsum", st, k_press_xsum<<<nb, kPBlock, 0, st>>>(R.n_rep, W.x, W.part));
  PDF_KERNEL("k_press_sum", st, k_press_sum<<<1, kPBlock, 0, st>>>(W.part, nb, W.scal + 3));
  PDF_KERNEL("k_press_scatter", st, k_press_scatter<<<pblocks(M.n_nodes), 256, 0, st>>>(M.n_nodes, R.n_rep, R.node_rep,
                                                                                          W.x, W.scal + 3, W.dP, p->pres));
  std::swap(W.gw, W.gw_prev);  // <P'>^{n+1} satisfies the new wall load
  // velocity correction with the element gradients of dP
  PDF_KERNEL("k_press_egrad", st, k_press_egrad<<<pblocks(M.n_tri), 256, 0, st>>>(M.n_tri, M.tri, M.dN, W.dP, W.ge));
  if (p->precision == PDF_FP64)
    PDF_KERNEL("k_press_correct", st, k_press_correct<fx::df><<<pblocks(p->n), 256, 0, st>>>(p->n, p->elem, W.ge,
                                                                                           params->dt, p->u, p->v));
  else
    PDF_KERNEL("k_press_correct", st, k_press_correct<float><<<pblocks(p->n), 256, 0, st>>>(p->n, p->elem, W.ge,
                                                                                          params->dt, p->uf, p->vf));
  s = press_gradient(p, st);
  if (s != PDF_OK) return s;
  s = estimate_stats(p, st);
  if (s != PDF_OK) return s;
  if (rn > rtol * bn && bn > 0.0) return fail(PDF_ENOTCONV, "pdf_pressure_project: not converged");
  return PDF_OK;
}

static int32_t m_rep(const pdf_particles* p) { return p->mesh->rx.n_rep; }

extern "C" pdf_status pdf_pressure_field(pdf_particles* p, const double* set, double* get, void* stream) {
  if (!p) return fail(PDF_EINVAL, "pdf_pressure_field: NULL handle");
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t nn = p->mesh->d.n_nodes;
  if (set) {
    pdf_status s = press_alloc(p);
    if (s != PDF_OK) return s;
    PDF_CUDA(cudaMemcpyAsync(p->pres, set, sizeof(double) * nn, cudaMemcpyDefault, st));
    PDF_CUDA(cudaMemsetAsync(p->pw.gw_prev, 0, sizeof(double) * m_rep(p), st));
    s = press_gradient(p, st);
    if (s != PDF_OK) return s;
  }
  if (get) PDF_CUDA(cudaMemcpyAsync(get, p->pres, sizeof(double) * nn, cudaMemcpyDefault, st));
  return PDF_OK;
}

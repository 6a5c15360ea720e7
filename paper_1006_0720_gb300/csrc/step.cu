// The particle time step: element coefficient rows (loop (ii) of the table
// of loop designs: nodal statistics -> element averages, precomputed once
// per element) and the fused per-particle kernel (draws, Euler-Maruyama
// updates, boundary conditions, neighbour walk).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "rng.cuh"

namespace pdfgb {

struct CoeffParams {
  double dt, nu, Pi, c_phi;
  int closure, tm_mode, pressure;
  double C1, C2, C3, C4, CT, Cv, gamma5, Comega1, Comega2, C0_slm;
};

static CoeffParams coeff_params(const pdf_model_params* p) {
  CoeffParams c;
  c.dt = p->dt; c.nu = p->nu; c.Pi = p->Pi; c.c_phi = p->c_phi;
  c.closure = p->closure; c.tm_mode = p->tm_mode; c.pressure = p->pressure;
  c.C1 = p->C1; c.C2 = p->C2; c.C3 = p->C3; c.C4 = p->C4; c.CT = p->CT; c.Cv = p->Cv;
  c.gamma5 = p->gamma5; c.Comega1 = p->Comega1; c.Comega2 = p->Comega2; c.C0_slm = p->C0_slm;
  return c;
}

constexpr double kKFloor = 1e-12;  // floor of k in G, C0, b_ij, A_v
constexpr double kEFloor = 1e-12;  // floor of eps

// Right-hand side of eq. elliptic-relaxation-Lagrangian at one node:
// (1 - C1)/2 k <omega> delta_ij + k H_ijkl d<U_k>/dx_l, with H from eq. H,
// A_v = min(1, C_v det<uu> / (2k/3)^3) and b_ij of eq. bij.  Contracting H
// with the gradient gives
//   (C2 A_v + g5/3) dU_i/dx_j - (g5/3) dU_j/dx_i + g5 b_ik dU_k/dx_j - g5 b_il dU_j/dx_l.
__device__ void relax_rhs(const double* S, const double* D, const CoeffParams& P, double rhs[9]) {
  const double R[3][3] = {{S[5], S[8], S[9]}, {S[8], S[6], S[10]}, {S[9], S[10], S[7]}};
  const double k = fmax(0.5 * (S[5] + S[6] + S[7]), kKFloor);
  const double grad[3][3] = {{D[0], D[1], 0.0}, {D[2], D[3], 0.0}, {D[4], D[5], 0.0}};  // dU_i/dx_j
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
        bk += b[i][q] * grad[q][j];
        bl += b[i][q] * grad[j][q];
      }
      const double h = (P.C2 * Av + g3) * grad[i][j] - g3 * grad[j][i] + P.gamma5 * (bk - bl);
      rhs[3 * i + j] = (i == j ? 0.5 * (1.0 - P.C1) * k * S[3] : 0.0) + k * h;
    }
}

// The 26 nodal coefficients a particle sees (element-averaged afterwards):
// <U_i>; d<U_i>/dx_j; a_i = -d<P>/dx_i + 2 nu lap<U_i> (GLM) or -d<P>/dx_i
// (SLM); G_ij (eq. GandC or eq. wall-GandC); sqrt(C0 eps); <omega>; S_omega
// (eq. frequency-source); <phi>; 1/t_m.
__global__ void k_node_coeff(int32_t n_nodes, const double* __restrict__ ns, const double* __restrict__ nd,
                             const double* __restrict__ wp, CoeffParams P, double* __restrict__ nc) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    double S[PDF_NNS], D[PDF_NND];
    for (int q = 0; q < PDF_NNS; ++q) S[q] = ns[(int64_t)n * PDF_NNS + q];
    for (int q = 0; q < PDF_NND; ++q) D[q] = nd[(int64_t)n * PDF_NND + q];
    double* c = nc + (int64_t)n * PDF_NCOEF;
    const double k = 0.5 * (S[5] + S[6] + S[7]);
    const double kg = fmax(k, kKFloor);
    const double om = S[3];
    const double eps = (P.closure == PDF_CLOSURE_SLM) ? k * om : om * (k + P.nu * P.CT * P.CT * om);
    const double eg = fmax(eps, kEFloor);
    c[0] = S[0]; c[1] = S[1]; c[2] = S[2];
    for (int q = 0; q < 6; ++q) c[3 + q] = D[q];
    double dpx = 0.0, dpy = 0.0;
    if (P.pressure == PDF_PRESSURE_CHANNEL) { dpx = P.Pi; dpy = D[9]; }
    if (P.closure == PDF_CLOSURE_SLM) {
      c[9] = dpx; c[10] = dpy; c[11] = 0.0;
      const double g = -(0.5 + 0.75 * P.C0_slm) * om;
      for (int q = 0; q < 9; ++q) c[12 + q] = (q % 4 == 0) ? g : 0.0;
      c[21] = sqrt(P.C0_slm * fmax(eps, 0.0));
    } else {
      c[9] = dpx + 2.0 * P.nu * D[6];
      c[10] = dpy + 2.0 * P.nu * D[7];
      c[11] = 2.0 * P.nu * D[8];
      double w9[9];
      if (wp) {
        for (int q = 0; q < 9; ++q) w9[q] = wp[(int64_t)q * n_nodes + n];
      } else {
        relax_rhs(S, D, P, w9);
      }
      const double R9[9] = {S[5], S[8], S[9], S[8], S[6], S[10], S[9], S[10], S[7]};
      double wr = 0.0;
      for (int q = 0; q < 9; ++q) wr += w9[q] * R9[q];
      for (int q = 0; q < 9; ++q) c[12 + q] = (w9[q] - ((q % 4 == 0) ? 0.5 * eg : 0.0)) / kg;
      const double C0 = fmax(-2.0 * wr / (3.0 * kg * eg), 0.0);
      c[21] = sqrt(C0 * eg);
    }
    c[22] = om;
    const double prod = -(S[5] * D[0] + S[8] * D[1] + S[8] * D[2] + S[6] * D[3] + S[9] * D[4] + S[10] * D[5]);
    c[23] = P.Comega2 - P.Comega1 * prod / eg;
    c[24] = S[4];
    if (P.tm_mode == PDF_TM_CPHI) {
      c[25] = 0.5 * P.c_phi * om;
    } else {
      c[25] = 1.0 / fmax(kg / eg, P.CT * sqrt(P.nu / eg));
    }
  }
}

// Internal row (32 doubles) from the 26 element-average coefficients: the
// time-step factors of the Euler-Maruyama updates folded in once per element.
__device__ __forceinline__ void scale_row(const double a[PDF_NCOEF], const CoeffParams& P, double* r) {
  const double dt = P.dt, sdt = sqrt(P.dt);
  const double sgrad = (P.closure == PDF_CLOSURE_SLM) ? 0.0 : sqrt(2.0 * P.nu) * sdt;
  for (int i = 0; i < 3; ++i) r[i] = a[i];
  for (int q = 0; q < 6; ++q) r[3 + q] = sgrad * a[3 + q];
  for (int i = 0; i < 3; ++i) r[9 + i] = a[9 + i] * dt;
  for (int q = 0; q < 9; ++q) r[12 + q] = a[12 + q] * dt;
  r[21] = a[21] * sdt;
  const double mo = a[22];
  r[22] = mo;
  r[23] = (P.C3 + a[23]) * mo * dt;
  r[24] = P.C3 * mo * mo * dt;
  r[25] = mo * sqrt(2.0 * P.C3 * P.C4 * dt);
  r[26] = a[24];
  r[27] = dt * a[25];
  r[28] = r[29] = r[30] = r[31] = 0.0;
}

__global__ void k_elem_rows(const int32_t* __restrict__ tri, int32_t n_tri, const double* __restrict__ nc,
                            CoeffParams P, double* __restrict__ rows, double* __restrict__ avg_out) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    const double* c0 = nc + (int64_t)tri[3 * e] * PDF_NCOEF;
    const double* c1 = nc + (int64_t)tri[3 * e + 1] * PDF_NCOEF;
    const double* c2 = nc + (int64_t)tri[3 * e + 2] * PDF_NCOEF;
    double a[PDF_NCOEF];
    for (int q = 0; q < PDF_NCOEF; ++q) a[q] = (c0[q] + c1[q] + c2[q]) / 3.0;
    if (avg_out)
      for (int q = 0; q < PDF_NCOEF; ++q) avg_out[(int64_t)e * PDF_NCOEF + q] = a[q];
    if (rows) scale_row(a, P, rows + (int64_t)e * PDFGB_ROW);
  }
}

__global__ void k_frozen_rows(int32_t n_tri, const double* __restrict__ coeff, CoeffParams P,
                              double* __restrict__ rows) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    double a[PDF_NCOEF];
    for (int q = 0; q < PDF_NCOEF; ++q) a[q] = coeff[(int64_t)e * PDF_NCOEF + q];
    scale_row(a, P, rows + (int64_t)e * PDFGB_ROW);
  }
}

// ----------------------------------------------------------------------------
// The fused particle kernel.
// ----------------------------------------------------------------------------
struct StepArgs {
  int64_t n;
  double *x, *y, *u, *v, *w, *om, *ps;
  int32_t* elem;
  const double* rows;
  const ElemGeo* geo;
  const int32_t* tri;
  const double* xy;
  const int32_t* esup_off;
  const int32_t* esup;
  int32_t n_tri;
  double period;
  double dt;      // position advection
  double sdiff;   // sqrt(2 nu dt): position diffusion (0 for SLM)
  uint64_t seed;
  uint32_t step;
  long long* counters;
};

enum { kCntWalk = 0, kCntRefl, kCntPeriodic, kCntFallback, kCntBrute, kCntLost, kCntOmega, kCntNear };

// Twice the signed sub-areas N^A, N^B, N^C of sec. 3.5 (eq. element-test and
// the cross products below it; N^B = A_e - N^A - N^C).
__device__ __forceinline__ void sub_areas(const ElemGeo& g, double x, double y, double& na, double& nb,
                                          double& nc) {
  const double dx = x - g.xb, dy = y - g.yb;
  na = g.cbx * dy - g.cby * dx;
  nc = dx * g.aby - dy * g.abx;
  nb = g.two_area - na - nc;
}

__device__ __forceinline__ ElemGeo load_geo(const ElemGeo* geo, int32_t e) {
  const double2* p = reinterpret_cast<const double2*>(geo + e);
  ElemGeo g;
  const double2 a0 = __ldg(p), a1 = __ldg(p + 1), b0 = __ldg(p + 2);
  const int4 c = __ldg(reinterpret_cast<const int4*>(p + 3));
  const int4 d = __ldg(reinterpret_cast<const int4*>(p + 4));
  g.xb = a0.x; g.yb = a0.y; g.cbx = a1.x; g.cby = a1.y;
  g.abx = b0.x; g.aby = b0.y;
  g.two_area = __hiloint2double(c.y, c.x);
  g.nbr[0] = c.z;
  g.nbr[1] = c.w;
  g.nbr[2] = d.x;
  const int32_t sh = d.y;
  g.shift[0] = (int8_t)(sh & 0xff);
  g.shift[1] = (int8_t)((sh >> 8) & 0xff);
  g.shift[2] = (int8_t)((sh >> 16) & 0xff);
  return g;
}

// Neighbour walk from the old element (sec. 3.5).  Returns the host element
// (or -1 if lost); updates x, y (periodic shifts, wall mirror) and u, v
// (wall-normal component reversed on reflection).
__device__ int32_t walk(const StepArgs& A, int32_t e, double& x, double& y, double& u, double& v,
                        int& c_walk, int& c_refl, int& c_per, int& c_fb, int& c_brute, int& c_near) {
  int steps = 0, refl = 0;
  for (;;) {
    ElemGeo g = load_geo(A.geo, e);
    double na, nb, nc;
    sub_areas(g, x, y, na, nb, nc);
    if (na >= 0.0 && nb >= 0.0 && nc >= 0.0) {
      const double mn = fmin(na, fmin(nb, nc));
      if (mn < 1e-12 * g.two_area) ++c_near;
      break;
    }
    if (steps >= 64) {
      ++c_brute;
      int32_t hit = -1;
      for (int32_t f = 0; f < A.n_tri; ++f) {
        const ElemGeo h = load_geo(A.geo, f);
        double a, b, c;
        sub_areas(h, x, y, a, b, c);
        if (a >= 0.0 && b >= 0.0 && c >= 0.0) { hit = f; break; }
      }
      if (hit < 0) { c_walk += steps; return -1; }
      e = hit;
      steps = 0;  // the next test succeeds
      continue;
    }
    int k = 0;
    double mn = na;
    if (nb < mn) { k = 1; mn = nb; }
    if (nc < mn) { k = 2; }
    const int32_t nbr = g.nbr[k];
    ++steps;
    if (nbr >= 0) {
      if (g.shift[k] != 0) {
        x += (double)g.shift[k] * A.period;
        ++c_per;
      }
      e = nbr;
      continue;
    }
    if (nbr == kNbrInflow || nbr == kNbrOutflow) {  // open boundaries: not in these workloads
      c_walk += steps;
      return -1;
    }
    // wall: fall-back search among the elements around the current nodes
    int32_t hit = -1;
    for (int j = 0; j < 3 && hit < 0; ++j) {
      const int32_t nn = A.tri[3 * e + j];
      for (int32_t i = A.esup_off[nn]; i < A.esup_off[nn + 1] && hit < 0; ++i) {
        const int32_t f = A.esup[i];
        const ElemGeo h = load_geo(A.geo, f);
        double a, b, c;
        sub_areas(h, x, y, a, b, c);
        if (a >= 0.0 && b >= 0.0 && c >= 0.0) hit = f;
      }
    }
    if (hit >= 0) {
      ++c_fb;
      e = hit;
      continue;
    }
    if (refl >= 4) { c_walk += steps; return -1; }
    // mirror across the wall-edge line; outward normal of edge a->b of a
    // counter-clockwise triangle is (t_y, -t_x)/|t|
    const int32_t a = A.tri[3 * e + (k + 1) % 3], b = A.tri[3 * e + (k + 2) % 3];
    const double xa = A.xy[2 * a], ya = A.xy[2 * a + 1];
    const double tx = A.xy[2 * b] - xa, ty = A.xy[2 * b + 1] - ya;
    const double len = sqrt(tx * tx + ty * ty);
    const double nx = ty / len, ny = -tx / len;
    const double d = (x - xa) * nx + (y - ya) * ny;
    x = x - 2.0 * d * nx;
    y = y - 2.0 * d * ny;
    const double un = u * nx + v * ny;
    u = u - 2.0 * un * nx;
    v = v - 2.0 * un * ny;
    ++refl;
    ++c_refl;
  }
  c_walk += steps;
  return e;
}

__device__ __forceinline__ void add_counter(long long* c, int v) {
  // one atomic per warp for each counter that is non-zero somewhere in the warp
  int s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s != 0) atomicAdd(reinterpret_cast<unsigned long long*>(c), (unsigned long long)(long long)s);
}

__global__ void __launch_bounds__(256) k_step(StepArgs A) {
  int c_walk = 0, c_refl = 0, c_per = 0, c_fb = 0, c_brute = 0, c_lost = 0, c_om = 0, c_near = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every lane runs the same number of iterations so the warp reductions below see all lanes
  const int64_t iters = (A.n + stride - 1) / stride;
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < iters; ++it, p += stride) {
    if (p >= A.n) continue;
    const int32_t e = A.elem[p];
    float g[8];
    gauss4(A.seed, (uint32_t)p, A.step, 0u, kPurposeStep, &g[0]);
    gauss4(A.seed, (uint32_t)p, A.step, 1u, kPurposeStep, &g[4]);
    const double* R = A.rows + (int64_t)e * PDFGB_ROW;
    const double U0 = A.u[p], U1 = A.v[p], U2 = A.w[p];
    const double gx = (double)g[0], gy = (double)g[1];
    const double d0 = U0 - __ldg(R + 0), d1 = U1 - __ldg(R + 1), d2 = U2 - __ldg(R + 2);
    const double G0 = (double)g[2], G1 = (double)g[3], G2 = (double)g[4];
    const double b = __ldg(R + 21);
    // velocity prediction (eq. velocity-prediction), time-n values throughout
    double un = U0 + __ldg(R + 9) + __ldg(R + 3) * gx + __ldg(R + 4) * gy +
                __ldg(R + 12) * d0 + __ldg(R + 13) * d1 + __ldg(R + 14) * d2 + b * G0;
    double vn = U1 + __ldg(R + 10) + __ldg(R + 5) * gx + __ldg(R + 6) * gy +
                __ldg(R + 15) * d0 + __ldg(R + 16) * d1 + __ldg(R + 17) * d2 + b * G1;
    const double wn = U2 + __ldg(R + 11) + __ldg(R + 7) * gx + __ldg(R + 8) * gy +
                      __ldg(R + 18) * d0 + __ldg(R + 19) * d1 + __ldg(R + 20) * d2 + b * G2;
    // position (eq. Lagrangian-position-exact) with the same dW_x, dW_y
    double xn = A.x[p] + U0 * A.dt + A.sdiff * gx;
    double yn = A.y[p] + U1 * A.dt + A.sdiff * gy;
    // frequency (eq. frequency-model); a negative result is reflected
    const double o = A.om[p];
    double on = o - __ldg(R + 23) * o + __ldg(R + 24) + __ldg(R + 25) * sqrt(fmax(o, 0.0)) * (double)g[5];
    if (on < 0.0) { on = -on; ++c_om; }
    // scalar (eq. IEM)
    const double s = A.ps[p];
    const double sn = s - (s - __ldg(R + 26)) * __ldg(R + 27);
    const int32_t en = walk(A, e, xn, yn, un, vn, c_walk, c_refl, c_per, c_fb, c_brute, c_near);
    A.x[p] = xn; A.y[p] = yn; A.u[p] = un; A.v[p] = vn; A.w[p] = wn; A.om[p] = on; A.ps[p] = sn;
    if (en >= 0) A.elem[p] = en; else ++c_lost;
  }
  add_counter(A.counters + kCntWalk, c_walk);
  add_counter(A.counters + kCntRefl, c_refl);
  add_counter(A.counters + kCntPeriodic, c_per);
  add_counter(A.counters + kCntFallback, c_fb);
  add_counter(A.counters + kCntBrute, c_brute);
  add_counter(A.counters + kCntLost, c_lost);
  add_counter(A.counters + kCntOmega, c_om);
  add_counter(A.counters + kCntNear, c_near);
}

static int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

static int blocks_for(int64_t n, int threads, int per_sm) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * per_sm));
}

static pdf_status check_params(const pdf_model_params* p) {
  if (!p) return fail(PDF_EINVAL, "NULL params");
  if (!(p->dt > 0.0) || !(p->nu >= 0.0)) return fail(PDF_EINVAL, "params: dt must be > 0 and nu >= 0");
  if (p->closure < 0 || p->closure > 2 || p->tm_mode < 0 || p->tm_mode > 1 || p->pressure < 0 || p->pressure > 1)
    return fail(PDF_EINVAL, "params: closure, tm_mode or pressure out of range");
  return PDF_OK;
}

// Coefficient rows from the stored statistics (GLM/SLM).
static pdf_status build_rows(pdf_particles* P, const pdf_model_params* params, const double* wp,
                             double* avg_out, bool internal, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  const CoeffParams C = coeff_params(params);
  PDF_KERNEL("k_node_coeff", st, k_node_coeff<<<blocks_for(M.n_nodes, 128, 32), 128, 0, st>>>(M.n_nodes, P->ns, P->nd,
                                                                params->closure == PDF_CLOSURE_GLM ? wp : nullptr,
                                                                C, P->nc););
  PDF_KERNEL("k_elem_rows", st, k_elem_rows<<<blocks_for(M.n_tri, 128, 32), 128, 0, st>>>(M.tri, M.n_tri, P->nc, C,
                                                             internal ? P->rows : nullptr, avg_out););
  return PDF_OK;
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_elem_coeff(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                                     const double* wp, double* rows, void* stream) {
  if (!p || !m || p->mesh != m || !rows) return fail(PDF_EINVAL, "pdf_elem_coeff: bad arguments");
  pdf_status s = check_params(params);
  if (s != PDF_OK) return s;
  if (params->closure == PDF_CLOSURE_FROZEN) return fail(PDF_EINVAL, "pdf_elem_coeff: FROZEN has no computed rows");
  if (!p->have_stats) return fail(PDF_ESTATE, "pdf_elem_coeff: call pdf_estimate_stats first");
  return build_rows(p, params, wp, rows, false, (cudaStream_t)stream);
}

extern "C" pdf_status pdf_step(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                               const double* wp, const double* elem_coeff, uint32_t step, void* stream,
                               pdf_step_info* info) {
  if (!p || !m || p->mesh != m) return fail(PDF_EINVAL, "pdf_step: NULL or mismatched handles");
  pdf_status s = check_params(params);
  if (s != PDF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const MeshDev& M = m->d;
  if (params->closure == PDF_CLOSURE_FROZEN) {
    if (!elem_coeff) return fail(PDF_EINVAL, "pdf_step: FROZEN needs elem_coeff");
    PDF_KERNEL("k_frozen_rows", st, k_frozen_rows<<<blocks_for(M.n_tri, 128, 32), 128, 0, st>>>(M.n_tri, elem_coeff, coeff_params(params), p->rows););
  } else {
    if (!p->have_stats) return fail(PDF_ESTATE, "pdf_step: call pdf_estimate_stats before a GLM/SLM step");
    s = build_rows(p, params, wp, nullptr, true, st);
    if (s != PDF_OK) return s;
  }
  if (info) PDF_CUDA(cudaMemsetAsync(p->counters, 0, sizeof(long long) * 8, st));
  StepArgs A;
  A.n = p->n;
  A.x = p->x; A.y = p->y; A.u = p->u; A.v = p->v; A.w = p->w; A.om = p->om; A.ps = p->ps;
  A.elem = p->elem;
  A.rows = p->rows;
  A.geo = M.geo; A.tri = M.tri; A.xy = M.xy; A.esup_off = M.esup_off; A.esup = M.esup;
  A.n_tri = M.n_tri;
  A.period = M.period;
  A.dt = params->dt;
  A.sdiff = (params->closure == PDF_CLOSURE_SLM) ? 0.0 : sqrt(2.0 * params->nu) * sqrt(params->dt);
  A.seed = p->seed;
  A.step = step;
  A.counters = p->counters;
  PDF_KERNEL("k_step", st, k_step<<<blocks_for(p->n, 256, 8), 256, 0, st>>>(A););
  if (info) {
    long long c[8];
    PDF_CUDA(cudaMemcpyAsync(c, p->counters, sizeof(c), cudaMemcpyDeviceToHost, st));
    PDF_CUDA(cudaStreamSynchronize(st));
    info->walk_steps = c[kCntWalk];
    info->reflections = c[kCntRefl];
    info->crossings_periodic = c[kCntPeriodic];
    info->fallbacks = c[kCntFallback];
    info->brute = c[kCntBrute];
    info->lost = c[kCntLost];
    info->omega_reflections = c[kCntOmega];
    info->near_face = c[kCntNear];
    if (info->lost > 0) return fail(PDF_ELOST, "pdf_step: particles lost");
  }
  return PDF_OK;
}

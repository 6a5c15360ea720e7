// The particle time step: element coefficient rows (loop (ii) of the table
// of loop designs: nodal statistics -> element averages, precomputed once
// per element) and the fused per-particle kernel (draws, Euler-Maruyama
// updates, boundary conditions, neighbour walk).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "fx.cuh"
#include "rng.cuh"

namespace pdfgb {

struct CoeffParams {
  double dt, nu, Pi, c_phi;
  int closure, tm_mode, pressure, arith;
  double src_x, src_y, src_r, Cs, Ct;
  double C1, C2, C3, C4, CT, Cv, gamma5, Comega1, Comega2, C0_slm;
  double sdt, s2nu, s2c3c4dt;  // sqrt(dt), sqrt(2 nu), sqrt(2 C3 C4 dt): once per call, not per element
  // products and quotients of the constants, formed once per call on the host
  // with the same operations as before (GB300's FP64 pipe bounds the node pass)
  double g5_3;     // gamma5 / 3
  double half_1mC1;  // 0.5 (1 - C1)
  double nuCT2;    // nu CT CT
  double two_nu;   // 2 nu
};

static CoeffParams coeff_params(const pdf_model_params* p) {
  CoeffParams c;
  c.dt = p->dt; c.nu = p->nu; c.Pi = p->Pi; c.c_phi = p->c_phi;
  c.closure = p->closure; c.tm_mode = p->tm_mode; c.pressure = p->pressure; c.arith = p->arith;
  c.C1 = p->C1; c.C2 = p->C2; c.C3 = p->C3; c.C4 = p->C4; c.CT = p->CT; c.Cv = p->Cv;
  c.gamma5 = p->gamma5; c.Comega1 = p->Comega1; c.Comega2 = p->Comega2; c.C0_slm = p->C0_slm;
  c.src_x = p->src_x; c.src_y = p->src_y; c.src_r = p->src_r; c.Cs = p->Cs; c.Ct = p->Ct;
  c.sdt = std::sqrt(p->dt);
  c.s2nu = std::sqrt(2.0 * p->nu);
  c.s2c3c4dt = std::sqrt(2.0 * p->C3 * p->C4 * p->dt);
  c.g5_3 = p->gamma5 / 3.0;
  c.half_1mC1 = 0.5 * (1.0 - p->C1);
  c.nuCT2 = p->nu * p->CT * p->CT;
  c.two_nu = 2.0 * p->nu;
  return c;
}

constexpr double kKFloor = 1e-12;  // floor of k in G, C0, b_ij, A_v
constexpr double kEFloor = 1e-12;  // floor of eps

// Right-hand side of eq. elliptic-relaxation-Lagrangian at one node:
// (1 - C1)/2 k <omega> delta_ij + k H_ijkl d<U_k>/dx_l, with H from eq. H,
// A_v = min(1, C_v det<uu> / (2k/3)^3) and b_ij of eq. bij.  Contracting H
// with the gradient gives
//   (C2 A_v + g5/3) dU_i/dx_j - (g5/3) dU_j/dx_i + g5 b_ik dU_k/dx_j - g5 b_il dU_j/dx_l.
// k is the floored turbulent energy and inv_k its reciprocal (the caller's);
// the gradient's third column (d/dz) is zero and its terms are left out.
// The FP64 pipe bounds this kernel, so the divisions are reciprocals taken
// once and multiplied.
__device__ void relax_rhs(const double* S, const double* D, const CoeffParams& P, double k, double inv_k,
                          double rhs[9]) {
  const double R[3][3] = {{S[5], S[8], S[9]}, {S[8], S[6], S[10]}, {S[9], S[10], S[7]}};
  const double grad[3][2] = {{D[0], D[1]}, {D[2], D[3]}, {D[4], D[5]}};  // dU_i/dx_j, j < 2
  const double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                     R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                     R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
  // (2k/3)^-3 = (27/8) k^-3
  const double Av = fmin(1.0, P.Cv * det * (3.375 * inv_k * inv_k * inv_k));
  double b[3][3];
  const double inv_2k = 0.5 * inv_k;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) b[i][j] = R[i][j] * inv_2k - (i == j ? 1.0 / 3.0 : 0.0);
  const double g3 = P.g5_3;
  const double cg = P.C2 * Av + g3;
  const double diag = P.half_1mC1 * k * S[3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      // b_ik dU_k/dx_j (zero for j = 2) and b_il dU_j/dx_l (l < 2)
      double bk = 0.0;
      if (j < 2) bk = b[i][0] * grad[0][j] + b[i][1] * grad[1][j] + b[i][2] * grad[2][j];
      const double bl = b[i][0] * grad[j][0] + b[i][1] * grad[j][1];
      double h = P.gamma5 * (bk - bl);
      if (j < 2) h += cg * grad[i][j];
      if (i < 2) h -= g3 * grad[j][i];
      rhs[3 * i + j] = (i == j ? diag : 0.0) + k * h;
    }
}

// The 26 nodal coefficients a particle sees (element-averaged afterwards):
// <U_i>; d<U_i>/dx_j; a_i = -d<P>/dx_i + 2 nu lap<U_i> (GLM) or -d<P>/dx_i
// (SLM); G_ij (eq. GandC or eq. wall-GandC); sqrt(C0 eps); <omega>; S_omega
// (eq. frequency-source); <phi>; 1/t_m.
__global__ void k_node_coeff(int32_t n_nodes, const double* __restrict__ ns, const double* __restrict__ nd,
                             const double* __restrict__ wp, const double* __restrict__ xy, CoeffParams P,
                             const double* __restrict__ gradP, double* __restrict__ nc) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    double S[PDF_NNS], D[PDF_NND];
    for (int q = 0; q < PDF_NNS; ++q) S[q] = ns[(int64_t)n * PDF_NNS + q];
    for (int q = 0; q < PDF_NND; ++q) D[q] = nd[(int64_t)n * PDF_NND + q];
    double* c = nc + (int64_t)n * PDF_NCOEF;
    const double k = 0.5 * (S[5] + S[6] + S[7]);
    const double kg = fmax(k, kKFloor);
    const double om = S[3];
    const double eps = (P.closure == PDF_CLOSURE_SLM) ? k * om : om * (k + P.nuCT2 * om);
    const double eg = fmax(eps, kEFloor);
    const double inv_kg = 1.0 / kg, inv_eg = 1.0 / eg;
    c[0] = S[0]; c[1] = S[1]; c[2] = S[2];
    for (int q = 0; q < 6; ++q) c[3 + q] = D[q];
    double dpx = 0.0, dpy = 0.0;
    if (P.pressure == PDF_PRESSURE_CHANNEL) { dpx = P.Pi; dpy = D[9]; }
    if (P.pressure == PDF_PRESSURE_PROJECTION) { dpx = P.Pi - gradP[2 * n]; dpy = -gradP[2 * n + 1]; }
    if (P.pressure == PDF_PRESSURE_PROJECTION_INOUT) { dpx = -gradP[2 * n]; dpy = -gradP[2 * n + 1]; }
    if (P.closure == PDF_CLOSURE_SLM) {
      c[9] = dpx; c[10] = dpy; c[11] = 0.0;
      const double g = -(0.5 + 0.75 * P.C0_slm) * om;
      for (int q = 0; q < 9; ++q) c[12 + q] = (q % 4 == 0) ? g : 0.0;
      c[21] = sqrt(P.C0_slm * fmax(eps, 0.0));
    } else {
      c[9] = dpx + P.two_nu * D[6];
      c[10] = dpy + P.two_nu * D[7];
      c[11] = P.two_nu * D[8];
      double w9[9];
      if (wp) {
        for (int q = 0; q < 9; ++q) w9[q] = wp[(int64_t)q * n_nodes + n];
      } else {
        relax_rhs(S, D, P, kg, inv_kg, w9);
      }
      const double R9[9] = {S[5], S[8], S[9], S[8], S[6], S[10], S[9], S[10], S[7]};
      double wr = 0.0;
      for (int q = 0; q < 9; ++q) wr += w9[q] * R9[q];
      for (int q = 0; q < 9; ++q) c[12 + q] = (w9[q] - ((q % 4 == 0) ? 0.5 * eg : 0.0)) * inv_kg;
      const double C0 = fmax((-2.0 / 3.0) * wr * inv_kg * inv_eg, 0.0);
      c[21] = sqrt(C0 * eg);
    }
    c[22] = om;
    const double prod = -(S[5] * D[0] + S[8] * D[1] + S[8] * D[2] + S[6] * D[3] + S[9] * D[4] + S[10] * D[5]);
    c[23] = P.Comega2 - P.Comega1 * prod * inv_eg;
    c[24] = S[4];
    if (P.tm_mode == PDF_TM_CPHI) {
      c[25] = 0.5 * P.c_phi * om;
    } else {
      double tm = fmax(kg * inv_eg, P.CT * sqrt(P.nu * inv_eg));
      if (P.tm_mode == PDF_TM_SOURCE) {
        // eq. micromixing-timescale-canyon: the source term, U_c = |<U>| at the node
        const double dx = xy[2 * n] - P.src_x, dy = xy[2 * n + 1] - P.src_y;
        const double d = sqrt(dx * dx + dy * dy);
        const double uc = fmax(sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]), 1e-12);
        tm = fmin(tm, P.Cs * cbrt(P.src_r * P.src_r / eg) + P.Ct * d / uc);
      }
      c[25] = 1.0 / tm;
    }
  }
}

// Internal row (32 doubles) from the 26 element-average coefficients: the
// time-step factors of the Euler-Maruyama updates folded in once per element.
__device__ __forceinline__ void scale_row(const double a[PDF_NCOEF], const CoeffParams& P, double* r) {
  const double dt = P.dt, sdt = P.sdt;
  const double sgrad = (P.closure == PDF_CLOSURE_SLM) ? 0.0 : P.s2nu * sdt;
  for (int i = 0; i < 3; ++i) r[i] = a[i];
  for (int q = 0; q < 6; ++q) r[3 + q] = sgrad * a[3 + q];
  for (int i = 0; i < 3; ++i) r[9 + i] = a[9 + i] * dt;
  for (int q = 0; q < 9; ++q) r[12 + q] = a[12 + q] * dt;
  r[21] = a[21] * sdt;
  const double mo = a[22];
  r[22] = mo;
  r[23] = (P.C3 + a[23]) * mo * dt;
  r[24] = P.C3 * mo * mo * dt;
  r[25] = mo * P.s2c3c4dt;
  r[26] = a[24];
  r[27] = dt * a[25];
  r[28] = r[29] = r[30] = r[31] = 0.0;
}

// The fixed-point kernel's row from the scaled FP64 row.
__device__ __forceinline__ void make_fx_row(const double* r, FxRow* out) {
  FxRow f;
  const int mi[4] = {0, 1, 2, 26};
#pragma unroll
  for (int j = 0; j < 4; ++j) f.mean[j] = fx::d2df((uint64_t)__double_as_longlong(r[mi[j]]));
  const int ci[23] = {3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 23, 24, 25, 27};
#pragma unroll
  for (int q = 0; q < 23; ++q) f.c[q] = fx::d2df((uint64_t)__double_as_longlong(r[ci[q]]));
#pragma unroll
  for (int q = 23; q < 28; ++q) f.c[q] = fx::df{0.f, 0.f};
  *out = f;
}

// Mean of the frequency given to a particle striking a no-slip wall (eq.
// frequency-wallstats): (1/C_T) d sqrt(2k)/dn into the fluid from the
// element gradient of the nodal sqrt(2k) = sqrt(<uu> + <vv> + <ww>); where that
// is not positive, the element average of the nodal <omega>.
__device__ __forceinline__ double noslip_omega(int32_t e, const int32_t* tri, const double* ns, const double* dN,
                                               const double* L, double CT) {
  const double* d = dN + (int64_t)e * 6;
  double g = 0.0, om = 0.0;
  for (int j = 0; j < 3; ++j) {
    const double* S = ns + (int64_t)tri[3 * e + j] * PDF_NNS;
    const double kk = S[5] + S[6] + S[7];
    g += sqrt(kk > 0.0 ? kk : 0.0) * (d[j] * L[2] + d[3 + j] * L[3]);
    om += S[3];
  }
  const double w = g / CT;
  return w > 0.0 ? w : om / 3.0;
}

__global__ void k_elem_rows(const int32_t* __restrict__ tri, int32_t n_tri, const double* __restrict__ nc,
                            CoeffParams P, double* __restrict__ rows, double* __restrict__ avg_out,
                            FxRow* __restrict__ rows_fx, float* __restrict__ rows_f32,
                            const ElemGeo* __restrict__ geo, const double* __restrict__ nsw_line,
                            const double* __restrict__ ns, const double* __restrict__ dN) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    // node rows of 26 doubles (208 B, 16-byte aligned): 16-byte loads, and
    // 16-byte stores of the 256-byte element row (the kernel's loads and
    // stores, not its arithmetic, filled the load-store queue)
    const double2* c0 = reinterpret_cast<const double2*>(nc + (int64_t)tri[3 * e] * PDF_NCOEF);
    const double2* c1 = reinterpret_cast<const double2*>(nc + (int64_t)tri[3 * e + 1] * PDF_NCOEF);
    const double2* c2 = reinterpret_cast<const double2*>(nc + (int64_t)tri[3 * e + 2] * PDF_NCOEF);
    double a[PDF_NCOEF];
#pragma unroll
    for (int q = 0; q < PDF_NCOEF / 2; ++q) {
      const double2 x0 = __ldg(c0 + q), x1 = __ldg(c1 + q), x2 = __ldg(c2 + q);
      a[2 * q] = (x0.x + x1.x + x2.x) * (1.0 / 3.0);
      a[2 * q + 1] = (x0.y + x1.y + x2.y) * (1.0 / 3.0);
    }
    if (avg_out)
      for (int q = 0; q < PDF_NCOEF; ++q) avg_out[(int64_t)e * PDF_NCOEF + q] = a[q];
    if (rows || rows_fx || rows_f32) {
      double r[PDFGB_ROW];
      scale_row(a, P, r);
      // r[28]: the no-slip wall frequency of elements next to a no-slip wall
      if (geo[e].nsw) r[28] = noslip_omega(e, tri, ns, dN, nsw_line + 4 * (int64_t)e, P.CT);
      if (rows) {
        double2* o = reinterpret_cast<double2*>(rows + (int64_t)e * PDFGB_ROW);
#pragma unroll
        for (int q = 0; q < PDFGB_ROW / 2; ++q) o[q] = make_double2(r[2 * q], r[2 * q + 1]);
      }
      if (rows_fx) make_fx_row(r, rows_fx + e);
      if (rows_f32)
        for (int q = 0; q < PDFGB_ROW; ++q) rows_f32[(int64_t)e * PDFGB_ROW + q] = __double2float_rn(r[q]);
    }
  }
}

__global__ void k_frozen_rows(int32_t n_tri, const double* __restrict__ coeff, CoeffParams P,
                              double* __restrict__ rows, FxRow* __restrict__ rows_fx, float* __restrict__ rows_f32) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    double a[PDF_NCOEF];
    for (int q = 0; q < PDF_NCOEF; ++q) a[q] = coeff[(int64_t)e * PDF_NCOEF + q];
    double r[PDFGB_ROW];
    scale_row(a, P, r);
    for (int q = 0; q < PDFGB_ROW; ++q) rows[(int64_t)e * PDFGB_ROW + q] = r[q];
    if (rows_fx) make_fx_row(r, rows_fx + e);
    if (rows_f32)
      for (int q = 0; q < PDFGB_ROW; ++q) rows_f32[(int64_t)e * PDFGB_ROW + q] = __double2float_rn(r[q]);
  }
}

// ----------------------------------------------------------------------------
// The fused particle kernel.
// ----------------------------------------------------------------------------
struct StepArgs {
  int64_t n;
  int64_t *x, *y;                  // fixed point, kPosF fraction bits
  fx::df *u, *v, *w, *om, *ps;     // double-float (PDF_FP64 storage)
  int32_t* elem;
  const int32_t* pid;              // particle id of each slot (the Philox counter)
  const fx::df* cond;              // IECM: the velocity-conditioned scalar mean of each slot, else NULL
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
  double src_x, src_y, src_r;  // concentrated source (src_r > 0)
  const double* nsw_line;      // [n_tri][4] nearest no-slip wall of flagged elements
  double nu;                   // kinematic viscosity (no-slip crossing probability)
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
  g.reinj = (uint8_t)((sh >> 24) & 0xff);
  g.nsw = d.z;
  return g;
}

// Neighbour walk from the old element (sec. 3.5).  Returns the host element
// (or -1 if lost); updates x, y (periodic shifts, wall mirror) and u, v
// (wall-normal component reversed on reflection).
__device__ int32_t walk(const StepArgs& A, int32_t e, double& x, double& y, double& u, double& v,
                        int& c_walk, int& c_refl, int& c_per, int& c_fb, int& c_brute, int& c_near,
                        bool& reinj, bool& noslip) {
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
      // a non-finite position is lost without the search over all elements
      if (!isfinite(x) || !isfinite(y)) { c_walk += steps; return -1; }
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
      if (g.reinj & (1u << k)) reinj = true;
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
    if (nbr == kNbrNoslip) {
      noslip = true;  // the wall condition resets the velocity
    } else {
      const double un = u * nx + v * ny;
      u = u - 2.0 * un * nx;
      v = v - 2.0 * un * ny;
    }
    ++refl;
    ++c_refl;
  }
  c_walk += steps;
  return e;
}

// The scalar after the move: fluid re-entering through the inflow carries
// none, particles inside the concentrated source get 1 (the test is the
// oracle's FP64 expression, rounded the same way).
__device__ __forceinline__ bool in_source(const StepArgs& A, double x, double y) {
  if (!(A.src_r > 0.0)) return false;
  const double dx = __dsub_rn(x, A.src_x), dy = __dsub_rn(y, A.src_y);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= __dmul_rn(A.src_r, A.src_r);
}

__device__ __forceinline__ void add_counter(long long* c, int v) {
  // one atomic per warp for each counter that is non-zero somewhere in the warp
  int s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s != 0) atomicAdd(reinterpret_cast<unsigned long long*>(c), (unsigned long long)(long long)s);
}

struct Counts {
  int walk = 0, refl = 0, per = 0, fb = 0, brute = 0, lost = 0, om = 0, near = 0;
};

struct Draws {
  float g[8];
};

// The step's first Philox block: g0..g3 (dW_x, dW_y, dW'_1, dW'_2).
__device__ __forceinline__ void draw_block0(const StepArgs& A, uint32_t id, Draws& d) {
  gauss4(A.seed, id, A.step, 0u, kPurposeStep, &d.g[0]);
}
// The second block: g4, g5 (dW'_3, dW_omega); g6, g7 are not used.
__device__ __forceinline__ void draw_block1(const StepArgs& A, uint32_t id, Draws& d) {
  uint32_t c[4] = {id, A.step, 1u, kPurposeStep};
  philox4x32_10(c, (uint32_t)A.seed, (uint32_t)(A.seed >> 32));
  box_muller(c[0], c[1], &d.g[4], &d.g[5]);
  d.g[6] = d.g[7] = 0.0f;
}

__device__ __forceinline__ Draws draw_step(const StepArgs& A, int64_t slot) {
  Draws d;
  const uint32_t id = (uint32_t)__ldg(A.pid + slot);
  draw_block0(A, id, d);
  draw_block1(A, id, d);
  return d;
}

// Frequency of a particle striking a no-slip wall (eq. frequency-wallstats):
// Gamma of shape 1/C4 = 4 and mean mw, -mw/4 times the sum of the logarithms
// of the four uniforms of the step's third Philox block (the same FP32
// logarithm as the initial Gamma(4) draw).
__device__ __noinline__ double wall_frequency(uint64_t seed, uint32_t id, uint32_t step, double mw) {
  uint32_t c[4] = {id, step, 2u, kPurposeStep};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  float lsum = __fadd_rn(ln_unit(u01_from_word(c[0])), ln_unit(u01_from_word(c[1])));
  lsum = __fadd_rn(lsum, ln_unit(u01_from_word(c[2])));
  lsum = __fadd_rn(lsum, ln_unit(u01_from_word(c[3])));
  return __dmul_rn(__dmul_rn(-0.25, mw), (double)lsum);
}

// eta of trajectory (b): the third word of the step's second Philox block.
__device__ __forceinline__ double wall_eta(uint64_t seed, uint32_t id, uint32_t step) {
  uint32_t c[4] = {id, step, 1u, kPurposeStep};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return (double)u01_from_word(c[2]);
}

// The stored forms of u, v, w, omega, psi, read as and written from FP64.
struct DfIO {
  fx::df *u, *v, *w, *om, *ps;
  __device__ void load(int64_t p, double& U0, double& U1, double& U2, double& o, double& s) const {
    U0 = fx::to_double(u[p]); U1 = fx::to_double(v[p]); U2 = fx::to_double(w[p]);
    o = fx::to_double(om[p]); s = fx::to_double(ps[p]);
  }
  __device__ void store(int64_t p, double U0, double U1, double U2, double o, double s) const {
    u[p] = fx::from_double(U0); v[p] = fx::from_double(U1); w[p] = fx::from_double(U2);
    om[p] = fx::from_double(o); ps[p] = fx::from_double(s);
  }
};
struct F32IO {
  float *u, *v, *w, *om, *ps;
  __device__ void load(int64_t p, double& U0, double& U1, double& U2, double& o, double& s) const {
    U0 = u[p]; U1 = v[p]; U2 = w[p]; o = om[p]; s = ps[p];
  }
  __device__ void store(int64_t p, double U0, double U1, double U2, double o, double s) const {
    u[p] = (float)U0; v[p] = (float)U1; w[p] = (float)U2; om[p] = (float)o; ps[p] = (float)s;
  }
};

// One particle in native FP64 instructions (PDF_ARITH_FP64, the fall-back
// of the fixed-point kernels for large moves, and every particle next to a
// no-slip wall).  The stored forms are widened to FP64 on load and rounded
// back on store; a particle that is lost, or whose new position leaves
// |x|, |y| < 64, keeps its position and element.
template <typename IO>
__device__ __forceinline__ Counts advance_native(const StepArgs& A, const IO& io, int64_t p, const Draws D) {
  Counts c;
  const float* g = D.g;
  const int32_t e = A.elem[p];
  const double* R = A.rows + (int64_t)e * PDFGB_ROW;
  double U0, U1, U2, o, s;
  io.load(p, U0, U1, U2, o, s);
  const double gx = (double)g[0], gy = (double)g[1];
  const double d0 = U0 - __ldg(R + 0), d1 = U1 - __ldg(R + 1), d2 = U2 - __ldg(R + 2);
  const double G0 = (double)g[2], G1 = (double)g[3], G2 = (double)g[4];
  const double b = __ldg(R + 21);
  // velocity prediction (eq. velocity-prediction), time-n values throughout
  double un = U0 + __ldg(R + 9) + __ldg(R + 3) * gx + __ldg(R + 4) * gy +
              __ldg(R + 12) * d0 + __ldg(R + 13) * d1 + __ldg(R + 14) * d2 + b * G0;
  double vn = U1 + __ldg(R + 10) + __ldg(R + 5) * gx + __ldg(R + 6) * gy +
              __ldg(R + 15) * d0 + __ldg(R + 16) * d1 + __ldg(R + 17) * d2 + b * G1;
  double wn = U2 + __ldg(R + 11) + __ldg(R + 7) * gx + __ldg(R + 8) * gy +
              __ldg(R + 18) * d0 + __ldg(R + 19) * d1 + __ldg(R + 20) * d2 + b * G2;
  // position (eq. Lagrangian-position-exact) with the same dW_x, dW_y
  const double x0 = __longlong_as_double((long long)fx::fix2d(A.x[p], kPosF));
  const double y0 = __longlong_as_double((long long)fx::fix2d(A.y[p], kPosF));
  double xn = x0 + U0 * A.dt + A.sdiff * gx;
  double yn = y0 + U1 * A.dt + A.sdiff * gy;
  // frequency (eq. frequency-model); a negative result is reflected
  double on = o - __ldg(R + 23) * o + __ldg(R + 24) + __ldg(R + 25) * sqrt(fmax(o, 0.0)) * (double)g[5];
  if (on < 0.0) { on = -on; ++c.om; }
  // scalar: eq. IEM (element mean) or eq. IECM (the particle's conditional mean)
  const double tgt = A.cond ? fx::to_double(A.cond[p]) : __ldg(R + 26);
  const double sn = s - (s - tgt) * __ldg(R + 27);
  // distances from the no-slip wall before and after the move
  const bool near = load_geo(A.geo, e).nsw != 0;
  double dn = 0.0, d1w = 0.0;
  if (near) {
    const double* L = A.nsw_line + 4 * (int64_t)e;
    dn = (x0 - L[0]) * L[2] + (y0 - L[1]) * L[3];
    d1w = (xn - L[0]) * L[2] + (yn - L[1]) * L[3];
  }
  bool reinj = false, wall = false;
  const int32_t en = walk(A, e, xn, yn, un, vn, c.walk, c.refl, c.per, c.fb, c.brute, c.near, reinj, wall);
  // no-slip wall condition: trajectory (a) (reflected at a no-slip edge, or
  // behind the wall line) or (b) (eta < f_w, eq. fw): U = 0, omega ~ Gamma
  if (near && !wall) wall = d1w < 0.0 || wall_eta(A.seed, (uint32_t)__ldg(A.pid + p), A.step) <
                                          exp(-dn * d1w / (A.nu * A.dt));
  if (wall) {
    un = vn = wn = 0.0;
    const double mw = __ldg(R + 28) > 0.0 ? __ldg(R + 28) : __ldg(R + 22);
    on = wall_frequency(A.seed, (uint32_t)__ldg(A.pid + p), A.step, mw);
  }
  if (en >= 0 && fabs(xn) < 64.0 && fabs(yn) < 64.0) {
    A.x[p] = fx::d2fix((uint64_t)__double_as_longlong(xn), kPosF);
    A.y[p] = fx::d2fix((uint64_t)__double_as_longlong(yn), kPosF);
    A.elem[p] = en;
  } else {
    ++c.lost;
    xn = x0;
    yn = y0;
  }
  double sf = reinj ? 0.0 : sn;
  if (in_source(A, xn, yn)) sf = 1.0;
  io.store(p, un, vn, wn, on, sf);
  return c;
}

// The same, out of line for the fixed-point kernels' rare fall-backs.  All
// arguments by value, so that no variable of the caller has its address
// taken (which would keep it in local memory for its whole life).
__device__ __noinline__ Counts advance_native_ool(const StepArgs A, int64_t p, const Draws D) {
  return advance_native(A, DfIO{A.u, A.v, A.w, A.om, A.ps}, p, D);
}
__device__ __noinline__ Counts advance_native_f32_ool(const StepArgs A, const F32IO io, int64_t p, const Draws D) {
  return advance_native(A, io, p, D);
}

__device__ __forceinline__ void merge(Counts& a, const Counts& b) {
  a.walk += b.walk; a.refl += b.refl; a.per += b.per; a.fb += b.fb;
  a.brute += b.brute; a.lost += b.lost; a.om += b.om; a.near += b.near;
}

__device__ __forceinline__ void flush_counts(const StepArgs& A, const Counts& c) {
  add_counter(A.counters + kCntWalk, c.walk);
  add_counter(A.counters + kCntRefl, c.refl);
  add_counter(A.counters + kCntPeriodic, c.per);
  add_counter(A.counters + kCntFallback, c.fb);
  add_counter(A.counters + kCntBrute, c.brute);
  add_counter(A.counters + kCntLost, c.lost);
  add_counter(A.counters + kCntOmega, c.om);
  add_counter(A.counters + kCntNear, c.near);
}

__global__ void __launch_bounds__(256) k_step(StepArgs A) {
  Counts c;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every lane runs the same number of iterations so the warp reductions below see all lanes
  const int64_t iters = (A.n + stride - 1) / stride;
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < iters; ++it, p += stride) {
    if (p >= A.n) continue;
    merge(c, advance_native(A, DfIO{A.u, A.v, A.w, A.om, A.ps}, p, draw_step(A, p)));
  }
  flush_counts(A, c);
}

// ----------------------------------------------------------------------------
// The same step without FP64 instructions (PDF_ARITH_FX, the default).
// Positions in their stored fixed point (56 fraction bits): exact
// increments, periodic shifts and element tests; velocity, frequency and
// scalar in their stored double-float form, products by the FMA-exact
// product and sums by TwoSum.  A particle whose position increment
// reaches one length unit, or whose walk meets a wall, an open boundary or
// the step cap, is finished by the native FP64 code above.
// ----------------------------------------------------------------------------
constexpr int kF = kPosF;

struct FxArgs {
  const FxRow* rows;
  const FxGeo* geo;
  int64_t period_fix;
  fx::df dt;      // dt
  fx::df sdiff;   // sqrt(2 nu dt)
  // concentrated source: 0 none, 1 double-float test with the FP64 test in
  // the rounding band, 2 FP64 test only (centre outside the fixed range)
  int src_mode;
  int64_t src_x, src_y;  // centre in fixed point
  fx::df src_r2;         // r^2
};

__device__ __forceinline__ fx::df ldc(const FxRow* r, int q) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(&r->c[q]));
  return fx::df{v.x, v.y};
}

__device__ __forceinline__ fx::df ldmean(const FxRow* r, int j) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(&r->mean[j]));
  return fx::df{v.x, v.y};
}

__device__ __forceinline__ fx::df ld_state(const fx::df* a, int64_t p) {
  const float2 v = reinterpret_cast<const float2*>(a)[p];
  return fx::df{v.x, v.y};
}

__device__ __forceinline__ void st_state(fx::df* a, int64_t p, fx::df v) {
  reinterpret_cast<float2*>(a)[p] = make_float2(v.h, v.l);
}

// a - b with the rounding error of the high parts kept (not renormalized;
// used as a multiplicand).
__device__ __forceinline__ fx::df dsub(fx::df a, fx::df b) {
  fx::acc t;
  t.init(a);
  t.sub(b);
  return fx::df{t.h, t.l};
}

// Twice the sub-areas in double-float (normalized), from fixed-point offsets.
__device__ __forceinline__ void sub_areas_fx(const FxGeo& g, int64_t X, int64_t Y, fx::df& na, fx::df& nb,
                                             fx::df& nc) {
  const fx::df dx = fx::fix2df(X - g.xb, kF), dy = fx::fix2df(Y - g.yb, kF);
  fx::acc a;
  a.init(fx::mul(g.cbx, dy));
  a.sub(fx::mul(g.cby, dx));
  na = a.value();
  fx::acc c;
  c.init(fx::mul(dx, g.aby));
  c.sub(fx::mul(dy, g.abx));
  nc = c.value();
  fx::acc b;
  b.init(g.two_area);
  b.sub(na);
  b.sub(nc);
  nb = b.value();
}

// The three sub-areas in FP32 with error bounds: |n - n_exact| < b for each,
// with a margin of 8 over the accumulated rounding (relative errors of
// 2^-24 from the rounded offsets, 2^-23 from the truncated high parts of the
// coefficients, 2^-24 per operation).  "Certain" decisions below are never
// wrong; the undecided go to the double-float test.
struct Screen {
  float na, nb, nc, ba, bb, bc;
};

__device__ __forceinline__ Screen screen_xy(int64_t xb, int64_t yb, float cbx, float cby, float abx, float aby,
                                            float two_area, int64_t X, int64_t Y) {
  const fx::df dxd = fx::fix2df(X - xb, kF), dyd = fx::fix2df(Y - yb, kF);
  const float dx = dxd.h + dxd.l, dy = dyd.h + dyd.l;
  const float p1 = cbx * dy, p2 = cby * dx;
  const float q1 = dx * aby, q2 = dy * abx;
  Screen S;
  S.na = p1 - p2;
  S.nc = q1 - q2;
  S.ba = (fabsf(p1) + fabsf(p2)) * 0x1p-18f;
  S.bc = (fabsf(q1) + fabsf(q2)) * 0x1p-18f;
  S.nb = two_area - S.na - S.nc;
  S.bb = (fabsf(two_area) + fabsf(S.na) + fabsf(S.nc)) * 0x1p-18f + S.ba + S.bc;
  return S;
}

// All three sub-areas certainly positive: the particle is inside, farther
// than ~4e-6 A_e from every edge (far outside the 1e-12 near-face band).
__device__ __forceinline__ bool certain_inside(const Screen& S) {
  return S.na > S.ba && S.nc > S.bc && S.nb > S.bb;
}

// The edge the walk leaves through when FP32 decides it: the smallest
// sub-area is certainly negative and certainly below the other two, so the
// exact choice (smallest, ties to the lowest local vertex) is the same.
// -1 when undecided.
__device__ __forceinline__ int certain_exit(const Screen& S) {
  int k = 0;
  float mn = S.na, mb = S.ba;
  if (S.nb < mn) { k = 1; mn = S.nb; mb = S.bb; }
  if (S.nc < mn) { k = 2; mn = S.nc; mb = S.bc; }
  const float hi = mn + mb;
  if (!(hi < 0.0f)) return -1;
  if (k != 0 && !(S.na - S.ba > hi)) return -1;
  if (k != 1 && !(S.nb - S.bb > hi)) return -1;
  if (k != 2 && !(S.nc - S.bc > hi)) return -1;
  return k;
}

__device__ __forceinline__ void prefetch_l1(const void* a) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
}
__device__ __forceinline__ void prefetch_l2(const void* a) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// One element of the fixed-point neighbour walk:
// kWalkInside (e holds the point), kWalkSlow (a wall or open-boundary edge,
// or the 64-step cap: the FP64 walk finishes it) or kWalkMoved (e, Xn now
// the neighbour across the edge opposite the smallest sub-area).
enum { kWalkInside = 0, kWalkMoved = 1, kWalkSlow = 2 };

// Crossing edge k of the element whose last 32 bytes are d (2A_e, nbr0,
// nbr1) and f (nbr2, shifts and outflow bits); selects rather than an
// indexed array, so that nothing goes to local memory.
__device__ __forceinline__ int cross_edge(const FxArgs& F, int k, int4 d, int2 f, int32_t& e, int64_t& Xn,
                                          int& steps, int& c_per, bool& reinj) {
  const int32_t nbr = k == 0 ? d.z : (k == 1 ? d.w : f.x);
  if (nbr < 0) return kWalkSlow;
  const int sh = (int)(int8_t)((f.y >> (8 * k)) & 0xff);
  ++steps;
  if (sh != 0) {
    Xn += (int64_t)sh * F.period_fix;
    ++c_per;
  }
  if ((f.y >> (24 + k)) & 1) reinj = true;
  e = nbr;
  return kWalkMoved;
}

// The undecided case: double-float sub-areas (rare; kept out of line so that
// the common path holds few registers; by value in and out).
struct WalkStep {
  int r;              // kWalkInside / kWalkMoved / kWalkSlow
  int32_t e;          // the element after the step
  int64_t Xn;         // x after a periodic shift
  int near, per, reinj, crossed;
};

__device__ __noinline__ WalkStep walk_one_df(const FxGeo* geo, int64_t period_fix, int32_t e, int64_t Xn,
                                             int64_t Yn, int steps) {
  const int4* src = reinterpret_cast<const int4*>(geo + e);
  const int4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2), d = __ldg(src + 3);
  const int2 f = __ldg(reinterpret_cast<const int2*>(src + 4));
  FxGeo G;
  G.xb = ((int64_t)(uint32_t)a.y << 32) | (uint32_t)a.x;
  G.yb = ((int64_t)(uint32_t)a.w << 32) | (uint32_t)a.z;
  G.cbx = fx::df{__int_as_float(b.x), __int_as_float(b.y)};
  G.cby = fx::df{__int_as_float(b.z), __int_as_float(b.w)};
  G.abx = fx::df{__int_as_float(c.x), __int_as_float(c.y)};
  G.aby = fx::df{__int_as_float(c.z), __int_as_float(c.w)};
  G.two_area = fx::df{__int_as_float(d.x), __int_as_float(d.y)};
  WalkStep w{kWalkInside, e, Xn, 0, 0, 0, 0};
  fx::df na, nb, nc;
  sub_areas_fx(G, Xn, Yn, na, nb, nc);
  if (fx::ge0(na) && fx::ge0(nb) && fx::ge0(nc)) {
    const float mn = fminf(na.h, fminf(nb.h, nc.h));
    if (mn < 1e-12f * G.two_area.h) w.near = 1;
    return w;
  }
  w.r = kWalkSlow;
  if (steps >= 64) return w;
  int k = 0;
  fx::df mn = na;
  if (fx::lt(nb, mn)) { k = 1; mn = nb; }
  if (fx::lt(nc, mn)) { k = 2; }
  const int32_t nbr = k == 0 ? d.z : (k == 1 ? d.w : f.x);
  if (nbr < 0) return w;
  const int sh = (int)(int8_t)((f.y >> (8 * k)) & 0xff);
  w.r = kWalkMoved;
  w.crossed = 1;
  if (sh != 0) {
    w.Xn = Xn + (int64_t)sh * period_fix;
    w.per = 1;
  }
  w.reinj = (f.y >> (24 + k)) & 1;
  w.e = nbr;
  return w;
}

__device__ __forceinline__ int walk_one(const FxArgs& F, int32_t& e, int64_t& Xn, int64_t Yn, int& steps,
                                        int& c_per, int& c_near, bool& reinj) {
  const int4* src = reinterpret_cast<const int4*>(F.geo + e);
  const int4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
  const float two_area = __int_as_float(__ldg(reinterpret_cast<const int*>(src + 3)));
  const Screen S = screen_xy(((int64_t)(uint32_t)a.y << 32) | (uint32_t)a.x,
                             ((int64_t)(uint32_t)a.w << 32) | (uint32_t)a.z, __int_as_float(b.x),
                             __int_as_float(b.z), __int_as_float(c.x), __int_as_float(c.z), two_area, Xn, Yn);
  if (certain_inside(S)) return kWalkInside;
  const int k = certain_exit(S);
  if (k < 0) {
    const WalkStep w = walk_one_df(F.geo, F.period_fix, e, Xn, Yn, steps);
    e = w.e;
    Xn = w.Xn;
    steps += w.crossed;
    c_per += w.per;
    c_near += w.near;
    if (w.reinj) reinj = true;
    return w.r;
  }
  if (steps >= 64) return kWalkSlow;
  const int4 d = __ldg(src + 3);
  const int2 f = __ldg(reinterpret_cast<const int2*>(src + 4));
  return cross_edge(F, k, d, f, e, Xn, steps, c_per, reinj);
}

// Fixed-point neighbour walk from element e; returns true when the FP64 walk
// must finish it.
__device__ __forceinline__ bool walk_fx(const FxArgs& F, int32_t& e, int64_t& Xn, int64_t Yn, int& steps, int& c_per,
                                        int& c_near, bool& reinj) {
  for (;;) {
    const int r = walk_one(F, e, Xn, Yn, steps, c_per, c_near, reinj);
    if (r != kWalkMoved) return r == kWalkSlow;
  }
}

// The first element of the walk screened ahead of the velocity update (its
// geometry was prefetched with the row): kWalkInside when the FP32 screen
// certainly places the new position in e, else the certain exit edge (0-2),
// whose neighbour's geometry is then prefetched, or -1 (undecided).
constexpr int kEarlyInside = 3;
__device__ __forceinline__ int early_screen(const FxArgs& F, int32_t e, int64_t Xn, int64_t Yn) {
  const int4* src = reinterpret_cast<const int4*>(F.geo + e);
  const int4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
  const int4 d = __ldg(src + 3);
  const int2 f = __ldg(reinterpret_cast<const int2*>(src + 4));
  const Screen S = screen_xy(((int64_t)(uint32_t)a.y << 32) | (uint32_t)a.x,
                             ((int64_t)(uint32_t)a.w << 32) | (uint32_t)a.z, __int_as_float(b.x),
                             __int_as_float(b.z), __int_as_float(c.x), __int_as_float(c.z), __int_as_float(d.x), Xn, Yn);
  if (certain_inside(S)) return kEarlyInside;
  const int k = certain_exit(S);
  if (k >= 0) {
    const int32_t nbr = k == 0 ? d.z : (k == 1 ? d.w : f.x);
    if (nbr >= 0) prefetch_l1(F.geo + nbr);
  }
  return k;
}

// The walk after early_screen: an "inside" answer ends it at once, a
// certain exit crosses without screening e again.
__device__ __forceinline__ bool walk_fx_from(const FxArgs& F, int first, int32_t& e, int64_t& Xn, int64_t Yn,
                                             int& steps, int& c_per, int& c_near, bool& reinj) {
  if (first == kEarlyInside) return false;
  if (first >= 0) {
    const int4* src = reinterpret_cast<const int4*>(F.geo + e);
    const int4 d = __ldg(src + 3);
    const int2 f = __ldg(reinterpret_cast<const int2*>(src + 4));
    const int r = cross_edge(F, first, d, f, e, Xn, steps, c_per, reinj);
    if (r != kWalkMoved) return r == kWalkSlow;
  }
  return walk_fx(F, e, Xn, Yn, steps, c_per, c_near, reinj);
}

// The FP64 walk (walls, open boundaries, the step cap), out of line and by
// value for the fixed-point kernels.
struct SlowWalk {
  int32_t e;  // host element, -1 if lost
  double x, y, u, v;
  Counts c;
  bool reinj;
  bool noslip;  // reflected at a no-slip wall
};

__device__ __noinline__ SlowWalk walk_slow(const StepArgs A, int32_t e, double x, double y, double u, double v) {
  SlowWalk r;
  r.reinj = false;
  r.noslip = false;
  r.e = walk(A, e, x, y, u, v, r.c.walk, r.c.refl, r.c.per, r.c.fb, r.c.brute, r.c.near, r.reinj, r.noslip);
  r.x = x;
  r.y = y;
  r.u = u;
  r.v = v;
  return r;
}

// Source test on the fixed-point position: d^2 - r^2 in double-float
// (error below 2^-44 of d^2 + r^2); inside a band of 2^-40 of that around
// zero the FP64 expression decides, as in the FP64 kernel.
__device__ __forceinline__ bool in_source_fx(const StepArgs& A, const FxArgs& F, int64_t X, int64_t Y) {
  if (F.src_mode == 0) return false;
  if (F.src_mode == 1) {
    const fx::df dx = fx::fix2df(X - F.src_x, kF), dy = fx::fix2df(Y - F.src_y, kF);
    const fx::df dx2 = fx::mul(dx, dx), dy2 = fx::mul(dy, dy);
    fx::acc a;
    a.init(dx2);
    a.add(dy2);
    a.sub(F.src_r2);
    const float v = a.h + a.l;
    const float band = (dx2.h + dy2.h + F.src_r2.h) * 0x1p-40f;
    if (fabsf(v) > band) return v < 0.0f;
  }
  return in_source(A, __longlong_as_double((long long)fx::fix2d(X, kF)),
                   __longlong_as_double((long long)fx::fix2d(Y, kF)));
}

// Position increment bound of the fixed-point path: |U dt + sqrt(2 nu dt) dW| < 1,
// which keeps every fixed-point offset of the walk below 2^7.
__device__ __forceinline__ bool small_move(const fx::acc& a) { return fabsf(a.h) < 1.0f; }

// FP64 back to the stored forms after the FP64 walk (the wall fall-back).
__device__ __forceinline__ bool pos_fits(double x) { return fabs(x) < 64.0; }


__global__ void __launch_bounds__(256, 4) k_step_fx(StepArgs A, FxArgs F) {
  int c_walk = 0, c_per = 0, c_om = 0, c_near = 0;
  Counts cs;  // counts of the FP64 fall-backs
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (A.n + stride - 1) / stride;
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < iters; ++it, p += stride) {
    if (p >= A.n) continue;
    int32_t e = A.elem[p];
    const FxRow* R = F.rows + e;
    // the element's row and geometry start on their way to L1 while the
    // random numbers are drawn
    prefetch_l1(R);
    prefetch_l1(reinterpret_cast<const char*>(R) + 128);
    prefetch_l1(F.geo + e);
    // the next iteration's state starts on its way from DRAM to L2
    if (p + stride < A.n) {
      const int64_t q = p + stride;
      prefetch_l2(A.x + q);
      prefetch_l2(A.y + q);
      prefetch_l2(A.u + q);
      prefetch_l2(A.v + q);
      prefetch_l2(A.w + q);
      prefetch_l2(A.om + q);
      prefetch_l2(A.ps + q);
      prefetch_l2(A.elem + q);
      prefetch_l2(A.pid + q);
    }
    // the first random block (dW_x, dW_y, dW'_1, dW'_2) gives the position;
    // the second is drawn after the early screen below
    Draws D;
    const uint32_t id = (uint32_t)__ldg(A.pid + p);
    draw_block0(A, id, D);
    const fx::df U[3] = {ld_state(A.u, p), ld_state(A.v, p), ld_state(A.w, p)};
    // position (eq. Lagrangian-position-exact): X + U^n dt + sqrt(2 nu) dW
    fx::acc ax, ay;
    ax.init(fx::mul(U[0], F.dt));
    ax.add(fx::mul_f(F.sdiff, D.g[0]));
    ay.init(fx::mul(U[1], F.dt));
    ay.add(fx::mul_f(F.sdiff, D.g[1]));
    // large moves go to the FP64 path; so do particles next to a no-slip
    // wall (the flag is loaded here and tested after the SDE updates, so
    // that its latency is hidden)
    const int near_noslip = __ldg(reinterpret_cast<const int*>(F.geo + e) + 18);
    if (!(small_move(ax) && small_move(ay))) {
      draw_block1(A, id, D);
      merge(cs, advance_native_ool(A, p, D));
      continue;
    }
    int64_t Xn = A.x[p] + ax.fix(kF);
    const int64_t Yn = A.y[p] + ay.fix(kF);
    // the new position against the old element now, so that the geometry
    // of the neighbour it leaves into arrives during the SDE updates
    const int first = early_screen(F, e, Xn, Yn);
    draw_block1(A, id, D);
    // velocity prediction (eq. velocity-prediction): U + a dt
    // + sqrt(2 nu) dU_i/dx_j dW_j + G_ij (U_j - <U_j>) dt + sqrt(C0 eps) dW'_i
    const fx::df d0 = dsub(U[0], ldmean(R, 0));
    const fx::df d1 = dsub(U[1], ldmean(R, 1));
    const fx::df d2 = dsub(U[2], ldmean(R, 2));
    const fx::df sc = ldc(R, 18);
    fx::df Un[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      fx::acc a;
      a.init(U[i]);
      a.add(ldc(R, 6 + i));
      a.add(fx::mul_f(ldc(R, 2 * i), D.g[0]));
      a.add(fx::mul_f(ldc(R, 2 * i + 1), D.g[1]));
      a.add(fx::mul(ldc(R, 9 + 3 * i), d0));
      a.add(fx::mul(ldc(R, 10 + 3 * i), d1));
      a.add(fx::mul(ldc(R, 11 + 3 * i), d2));
      a.add(fx::mul_f(sc, D.g[2 + i]));
      Un[i] = a.value();
    }
    // frequency (eq. frequency-model): omega - (C3 + S_w) <w> dt omega + C3 <w>^2 dt
    // + <w> sqrt(2 C3 C4 dt) sqrt(max(omega, 0)) dW
    const fx::df O = ld_state(A.om, p);
    fx::df On;
    {
      fx::acc a;
      a.init(O);
      a.sub(fx::mul(ldc(R, 19), O));
      a.add(ldc(R, 20));
      a.add(fx::mul_f(fx::mul(ldc(R, 21), fx::sqrt_df(O)), D.g[5]));
      On = a.value();
      if (On.h < 0.0f) { On = fx::df{-On.h, -On.l}; ++c_om; }
    }
    // scalar: psi - (psi - <phi>) dt / t_m (eq. IEM) or with the particle's
    // velocity-conditioned mean <phi|V> (eq. IECM)
    const fx::df S = ld_state(A.ps, p);
    fx::df Sn;
    {
      fx::acc a;
      a.init(S);
      a.sub(fx::mul(ldc(R, 22), dsub(S, A.cond ? ld_state(A.cond, p) : ldmean(R, 3))));
      Sn = a.value();
    }
    if (near_noslip) {
      merge(cs, advance_native_ool(A, p, D));
      continue;
    }
    // neighbour walk (sec. 3.5) in fixed point; walls, open boundaries and
    // the step cap go to the FP64 walk
    int steps = 0;
    bool reinj = false;
    const bool slow = walk_fx_from(F, first, e, Xn, Yn, steps, c_per, c_near, reinj);
    c_walk += steps;
    int64_t Xs = Xn, Ys = Yn;
    bool slow_noslip = false;
    if (slow) {
      double xn = __longlong_as_double((long long)fx::fix2d(Xn, kF));
      double yn = __longlong_as_double((long long)fx::fix2d(Yn, kF));
      double un = fx::to_double(Un[0]), vn = fx::to_double(Un[1]);
      const SlowWalk sw = walk_slow(A, e, xn, yn, un, vn);
      merge(cs, sw.c);
      if (sw.reinj) reinj = true;
      if (sw.noslip) {  // no-slip wall reached through other elements: the wall condition
        const double* Rd = A.rows + (int64_t)A.elem[p] * PDFGB_ROW;
        const double mw = __ldg(Rd + 28) > 0.0 ? __ldg(Rd + 28) : __ldg(Rd + 22);
        On = fx::from_double(wall_frequency(A.seed, (uint32_t)__ldg(A.pid + p), A.step, mw));
        slow_noslip = true;
      }
      if (sw.e >= 0 && pos_fits(sw.x) && pos_fits(sw.y)) {
        e = sw.e;
        Xs = fx::d2fix((uint64_t)__double_as_longlong(sw.x), kF);
        Ys = fx::d2fix((uint64_t)__double_as_longlong(sw.y), kF);
        Un[0] = fx::from_double(sw.u);
        Un[1] = fx::from_double(sw.v);
      } else {  // lost: keeps its element and position
        ++cs.lost;
        e = A.elem[p];
        Xs = A.x[p];
        Ys = A.y[p];
      }
    }
    if (reinj) Sn = fx::df{0.f, 0.f};
    if (in_source_fx(A, F, Xs, Ys)) Sn = fx::df{1.f, 0.f};
    if (slow_noslip) Un[0] = Un[1] = Un[2] = fx::df{0.f, 0.f};
    A.x[p] = Xs;
    A.y[p] = Ys;
    st_state(A.u, p, Un[0]);
    st_state(A.v, p, Un[1]);
    st_state(A.w, p, Un[2]);
    st_state(A.om, p, On);
    st_state(A.ps, p, Sn);
    A.elem[p] = e;
  }
  cs.walk += c_walk; cs.per += c_per; cs.om += c_om; cs.near += c_near;
  flush_counts(A, cs);
}

// ----------------------------------------------------------------------------
// PDF_FP32_STATE: velocity, frequency and scalar stored and advanced in FP32;
// positions and the walk stay FP64-accurate (fixed point, as above).
// ----------------------------------------------------------------------------
struct F32Args {
  float *u, *v, *w, *om, *ps;
  const float* rows;  // [n_tri][32], the layout of the FP64 rows
};

__global__ void __launch_bounds__(256, 4) k_step_f32(StepArgs A, FxArgs F, F32Args S) {
  int c_walk = 0, c_per = 0, c_om = 0, c_near = 0;
  Counts cs;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (A.n + stride - 1) / stride;
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < iters; ++it, p += stride) {
    if (p >= A.n) continue;
    int32_t e = A.elem[p];
    const float* R = S.rows + (int64_t)e * PDFGB_ROW;
    prefetch_l1(R);  // the 128-byte FP32 row and the geometry, as in k_step_fx
    prefetch_l1(F.geo + e);
    if (p + stride < A.n) {
      const int64_t q = p + stride;
      prefetch_l2(A.x + q);
      prefetch_l2(A.y + q);
      prefetch_l2(S.u + q);
      prefetch_l2(S.v + q);
      prefetch_l2(S.w + q);
      prefetch_l2(S.om + q);
      prefetch_l2(S.ps + q);
      prefetch_l2(A.elem + q);
      prefetch_l2(A.pid + q);
    }
    const Draws D = draw_step(A, p);
    const float U0 = S.u[p], U1 = S.v[p], U2 = S.w[p];
    const float d0 = U0 - __ldg(R + 0), d1 = U1 - __ldg(R + 1), d2 = U2 - __ldg(R + 2);
    const float b = __ldg(R + 21);
    // velocity prediction (eq. velocity-prediction) in FP32
    float un = U0 + __ldg(R + 9) + __ldg(R + 3) * D.g[0] + __ldg(R + 4) * D.g[1] + __ldg(R + 12) * d0 +
               __ldg(R + 13) * d1 + __ldg(R + 14) * d2 + b * D.g[2];
    float vn = U1 + __ldg(R + 10) + __ldg(R + 5) * D.g[0] + __ldg(R + 6) * D.g[1] + __ldg(R + 15) * d0 +
               __ldg(R + 16) * d1 + __ldg(R + 17) * d2 + b * D.g[3];
    float wn = U2 + __ldg(R + 11) + __ldg(R + 7) * D.g[0] + __ldg(R + 8) * D.g[1] + __ldg(R + 18) * d0 +
                     __ldg(R + 19) * d1 + __ldg(R + 20) * d2 + b * D.g[4];
    // frequency (eq. frequency-model) and scalar (eq. IEM) in FP32
    const float o = S.om[p];
    float on = o - __ldg(R + 23) * o + __ldg(R + 24) + __ldg(R + 25) * sqrtf(fmaxf(o, 0.f)) * D.g[5];
    if (on < 0.f) { on = -on; ++c_om; }
    const float s = S.ps[p];
    const float sn = s - (s - (A.cond ? A.cond[p].h : __ldg(R + 26))) * __ldg(R + 27);
    // particles next to a no-slip wall go to the FP64 path
    if (__ldg(reinterpret_cast<const int*>(F.geo + e) + 18) != 0) {
      merge(cs, advance_native_f32_ool(A, F32IO{S.u, S.v, S.w, S.om, S.ps}, p, D));
      continue;
    }
    // position (eq. Lagrangian-position-exact), fixed point
    const int64_t X0 = A.x[p], Y0 = A.y[p];
    fx::acc a;
    a.init(fx::mul_f(F.dt, U0));
    a.add(fx::mul_f(F.sdiff, D.g[0]));
    fx::acc c;
    c.init(fx::mul_f(F.dt, U1));
    c.add(fx::mul_f(F.sdiff, D.g[1]));
    int64_t Xn = X0, Yn = Y0;
    bool slow, reinj = false;
    double xn, yn;
    if (small_move(a) && small_move(c)) {
      Xn = X0 + a.fix(kF);
      Yn = Y0 + c.fix(kF);
      int steps = 0;
      slow = walk_fx(F, e, Xn, Yn, steps, c_per, c_near, reinj);
      c_walk += steps;
      xn = __longlong_as_double((long long)fx::fix2d(Xn, kF));
      yn = __longlong_as_double((long long)fx::fix2d(Yn, kF));
    } else {
      xn = __longlong_as_double((long long)fx::fix2d(X0, kF)) + (double)U0 * A.dt + A.sdiff * (double)D.g[0];
      yn = __longlong_as_double((long long)fx::fix2d(Y0, kF)) + (double)U1 * A.dt + A.sdiff * (double)D.g[1];
      slow = true;
    }
    bool slow_noslip = false;
    if (slow) {
      double ud = (double)un, vd = (double)vn;
      const SlowWalk sw = walk_slow(A, e, xn, yn, ud, vd);
      merge(cs, sw.c);
      if (sw.reinj) reinj = true;
      if (sw.noslip) {  // no-slip wall reached through other elements: the wall condition
        const double* Rd = A.rows + (int64_t)A.elem[p] * PDFGB_ROW;
        const double mw = __ldg(Rd + 28) > 0.0 ? __ldg(Rd + 28) : __ldg(Rd + 22);
        on = (float)wall_frequency(A.seed, (uint32_t)__ldg(A.pid + p), A.step, mw);
        wn = 0.0f;
        slow_noslip = true;
      }
      if (sw.e >= 0 && pos_fits(sw.x) && pos_fits(sw.y)) {
        e = sw.e;
        xn = sw.x;
        yn = sw.y;
        Xn = fx::d2fix((uint64_t)__double_as_longlong(xn), kF);
        Yn = fx::d2fix((uint64_t)__double_as_longlong(yn), kF);
        un = (float)sw.u;
        vn = (float)sw.v;
      } else {  // lost: keeps its element and position
        ++cs.lost;
        e = A.elem[p];
        Xn = X0;
        Yn = Y0;
      }
    }
    if (slow_noslip) un = vn = wn = 0.0f;
    float sf = reinj ? 0.0f : sn;
    if (in_source_fx(A, F, Xn, Yn)) sf = 1.0f;
    A.x[p] = Xn;
    A.y[p] = Yn;
    S.u[p] = un;
    S.v[p] = vn;
    S.w[p] = wn;
    S.om[p] = on;
    S.ps[p] = sf;
    A.elem[p] = e;
  }
  cs.walk += c_walk; cs.per += c_per; cs.om += c_om; cs.near += c_near;
  flush_counts(A, cs);
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
  if (p->closure < 0 || p->closure > 2 || p->tm_mode < 0 || p->tm_mode > 2 || p->pressure < 0 ||
      p->pressure > 3 || p->arith < 0 || p->arith > 1 || p->mix < 0 || p->mix > 1)
    return fail(PDF_EINVAL, "params: closure, tm_mode, pressure, arith or mix out of range");
  return PDF_OK;
}

// Coefficient rows from the stored statistics (GLM/SLM).
static pdf_status build_rows(pdf_particles* P, const pdf_model_params* params, const double* wp,
                             double* avg_out, bool internal, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  const CoeffParams C = coeff_params(params);
  PDF_KERNEL("k_node_coeff", st, k_node_coeff<<<blocks_for(M.n_nodes, 128, 32), 128, 0, st>>>(M.n_nodes, P->ns, P->nd,
                                                                params->closure == PDF_CLOSURE_GLM ? wp : nullptr,
                                                                M.xy, C, P->gradP, P->nc););
  PDF_KERNEL("k_elem_rows", st, k_elem_rows<<<blocks_for(M.n_tri, 128, 32), 128, 0, st>>>(M.tri, M.n_tri, P->nc, C,
                                                             internal ? P->rows : nullptr, avg_out,
                                                             internal && C.arith == PDF_ARITH_FX ? P->rows_fx : nullptr,
                                                             internal ? P->rows_f32 : nullptr, M.geo, M.nsw_line,
                                                             P->ns, M.dN););
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

namespace pdfgb {

// Everything of a step before the particle kernel: checks, the coefficient
// rows, the counters.
static pdf_status step_prepare(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                               const double* wp, const double* elem_coeff, bool count, cudaStream_t st) {
  if (!p || !m || p->mesh != m) return fail(PDF_EINVAL, "pdf_step: NULL or mismatched handles");
  pdf_status s = check_params(params);
  if (s != PDF_OK) return s;
  const MeshDev& M = m->d;
  if (params->closure == PDF_CLOSURE_FROZEN) {
    if (!elem_coeff) return fail(PDF_EINVAL, "pdf_step: FROZEN needs elem_coeff");
    PDF_KERNEL("k_frozen_rows", st, k_frozen_rows<<<blocks_for(M.n_tri, 128, 32), 128, 0, st>>>(
                                         M.n_tri, elem_coeff, coeff_params(params), p->rows,
                                         params->arith == PDF_ARITH_FX ? p->rows_fx : nullptr, p->rows_f32););
  } else {
    if (!p->have_stats) return fail(PDF_ESTATE, "pdf_step: call pdf_estimate_stats before a GLM/SLM step");
    s = build_rows(p, params, wp, nullptr, true, st);
    if (s != PDF_OK) return s;
  }
  if (params->mix == PDF_MIX_IECM && !p->have_cond)
    return fail(PDF_ESTATE, "pdf_step: IECM needs pdf_particles_set_iecm and a pdf_estimate_stats after it");
  if (count) PDF_CUDA(cudaMemsetAsync(p->counters, 0, sizeof(long long) * 8, st));
  return PDF_OK;
}

// The particle kernel's arguments; StepLaunch::run advances the slots
// [beg, beg + cnt) (every per-slot pointer offset by beg) with a grid of at
// most per_sm blocks per SM (4 resident; at 15.9M particles 4, 8, 12, 16
// and 32 blocks per SM took 0.96, 0.94, 0.94, 0.92 and 0.92 ms).
struct StepLaunch {
  StepArgs A;
  FxArgs F;
  F32Args S;
  int kind = 0;  // 0: FP64 kernel, 1: fixed point / double-float, 2: FP32 state

  pdf_status run(int64_t beg, int64_t cnt, cudaStream_t st, int per_sm = 16) const {
    if (cnt <= 0) return PDF_OK;
    const int nb = blocks_for(cnt, 256, per_sm);
    StepArgs a = A;
    a.n = cnt;
    a.x += beg; a.y += beg; a.elem += beg; a.pid += beg;
    if (a.cond) a.cond += beg;
    if (kind == 2) {
      F32Args f = S;
      f.u += beg; f.v += beg; f.w += beg; f.om += beg; f.ps += beg;
      PDF_KERNEL("k_step", st, k_step_f32<<<nb, 256, 0, st>>>(a, F, f));
    } else if (kind == 1) {
      a.u += beg; a.v += beg; a.w += beg; a.om += beg; a.ps += beg;
      PDF_KERNEL("k_step", st, k_step_fx<<<nb, 256, 0, st>>>(a, F));
    } else {
      a.u += beg; a.v += beg; a.w += beg; a.om += beg; a.ps += beg;
      PDF_KERNEL("k_step", st, k_step<<<nb, 256, 0, st>>>(a));
    }
    return PDF_OK;
  }
};

static StepLaunch step_args(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params, uint32_t step) {
  const MeshDev& M = m->d;
  StepLaunch L;
  StepArgs& A = L.A;
  A.n = p->n;
  A.x = p->x; A.y = p->y; A.u = p->u; A.v = p->v; A.w = p->w; A.om = p->om; A.ps = p->ps;
  A.elem = p->elem;
  A.pid = p->pid;
  A.cond = params->mix == PDF_MIX_IECM ? p->cond : nullptr;
  A.rows = p->rows;
  A.geo = M.geo; A.tri = M.tri; A.xy = M.xy; A.esup_off = M.esup_off; A.esup = M.esup;
  A.n_tri = M.n_tri;
  A.period = M.period;
  A.dt = params->dt;
  A.sdiff = (params->closure == PDF_CLOSURE_SLM) ? 0.0 : sqrt(2.0 * params->nu) * sqrt(params->dt);
  A.seed = p->seed;
  A.step = step;
  A.counters = p->counters;
  A.nsw_line = M.nsw_line;
  A.nu = params->nu;
  A.src_x = params->src_x;
  A.src_y = params->src_y;
  A.src_r = params->src_r;
  if (p->precision == PDF_FP32_STATE || params->arith == PDF_ARITH_FX) {
    FxArgs& F = L.F;
    F.rows = p->rows_fx;
    F.geo = M.fgeo;
    uint64_t b;
    std::memcpy(&b, &M.period, 8);
    F.period_fix = fx::d2fix(b, kF);
    std::memcpy(&b, &A.dt, 8);
    F.dt = fx::d2df(b);
    std::memcpy(&b, &A.sdiff, 8);
    F.sdiff = fx::d2df(b);
    F.src_mode = 0;
    F.src_x = F.src_y = 0;
    F.src_r2 = fx::df{0.f, 0.f};
    if (params->src_r > 0.0) {
      const double r2 = params->src_r * params->src_r;
      F.src_mode = (std::fabs(params->src_x) < 64.0 && std::fabs(params->src_y) < 64.0 && r2 < 1e30) ? 1 : 2;
      if (F.src_mode == 1) {
        std::memcpy(&b, &params->src_x, 8);
        F.src_x = fx::d2fix(b, kF);
        std::memcpy(&b, &params->src_y, 8);
        F.src_y = fx::d2fix(b, kF);
        F.src_r2 = fx::from_double(r2);
      }
    }
    if (p->precision == PDF_FP32_STATE) {
      F32Args& S = L.S;
      S.u = p->uf; S.v = p->vf; S.w = p->wf; S.om = p->omf; S.ps = p->psf;
      S.rows = p->rows_f32;
      L.kind = 2;
    } else {
      L.kind = 1;
    }
  }
  return L;
}

// The counters of the step into info (one synchronization).
static pdf_status step_info(pdf_particles* p, pdf_step_info* info, cudaStream_t st) {
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
  return PDF_OK;
}

}  // namespace pdfgb

extern "C" pdf_status pdf_step(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                               const double* wp, const double* elem_coeff, uint32_t step, void* stream,
                               pdf_step_info* info) {
  cudaStream_t st = (cudaStream_t)stream;
  pdf_status s = step_prepare(p, m, params, wp, elem_coeff, info != nullptr, st);
  if (s != PDF_OK) return s;
  s = step_args(p, m, params, step).run(0, p->n, st);
  if (s != PDF_OK) return s;
  return info ? step_info(p, info, st) : PDF_OK;
}

namespace pdfgb {
pdf_status estimate_stats(pdf_particles* P, cudaStream_t st);
}

// pdf_step_host, and with `stats` pdf_step_host_stats: the statistics of the
// stepped state are issued on the compute stream after the last chunk's
// step, so that they run while the copy engines still write the last chunks
// back (es, ns, nd: optional copies of the results, as pdf_estimate_stats).
static pdf_status step_host(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params, const double* wp,
                            const double* elem_coeff, uint32_t step, double* const io_arg[7], int32_t* elem,
                            cudaStream_t st, pdf_step_info* info, bool stats, double* es, double* ns, double* nd) {
  for (int i = 0; i < 7; ++i)
    if (!io_arg[i]) return fail(PDF_EINVAL, "pdf_step_host: NULL argument");
  if (!p || !elem) return fail(PDF_EINVAL, "pdf_step_host: NULL argument");
  if (params && params->mix == PDF_MIX_IECM)
    return fail(PDF_EINVAL, "pdf_step_host: IECM needs the device-resident state (pdf_step)");
  double* io[7];
  for (int i = 0; i < 7; ++i) io[i] = io_arg[i];
  // page-locked host or device memory: the copies then run asynchronously
  for (int i = 0; i < 7; ++i)
    if (!state_kernel_view(io[i]))
      return fail(PDF_EINVAL, "pdf_step_host: the state arrays must be page-locked host or device memory");
  if (!state_kernel_view(elem))
    return fail(PDF_EINVAL, "pdf_step_host: the state arrays must be page-locked host or device memory");
  pdf_status s = host_io_init(p);
  if (s != PDF_OK) return s;
  HostIo& H = p->hio;
  // the state is loaded in particle-id order (slot = id), so that every
  // chunk is a contiguous range of the caller's arrays.  Per chunk: the
  // copy engines bring its 8 arrays into a device staging buffer (stream
  // in), the compute stream converts them into the slots, steps them and
  // converts them back into an outgoing staging buffer, and the copy
  // engines write that back (stream out); two staging buffers per
  // direction, so that chunk k + 1 moves while chunk k is stepped.  Chunks
  // start on 4 KiB boundaries of the arrays: with both directions moving,
  // pieces that start only 8-byte aligned went 12-15 % slower (8 and 16
  // pieces per array of 15.9M doubles: 237 and 233 GB/s together against
  // 271 and 265 aligned).  With the first copies started before the
  // coefficient rows, a call with statistics at 15.9M particles went from
  // 7.54 to 6.89 ms.
  const int64_t n = p->n;
  const int K = (int)std::max<int64_t>(1, std::min<int64_t>(kHostChunks, n / 65536));
  const int64_t chunk = ((n + K - 1) / K + 511) / 512 * 512;
  s = host_io_stage(p, chunk);
  if (s != PDF_OK) return s;
  // the first chunks' copies may start while the coefficient rows are formed
  PDF_CUDA(cudaEventRecord(H.start, st));
  PDF_CUDA(cudaStreamWaitEvent(H.in, H.start, 0));
  PDF_CUDA(cudaStreamWaitEvent(H.out, H.start, 0));
  s = step_prepare(p, m, params, wp, elem_coeff, true, st);
  if (s != PDF_OK) return s;
  unsigned long long* bad = reinterpret_cast<unsigned long long*>(p->counters + 15);
  PDF_CUDA(cudaMemsetAsync(bad, 0, sizeof(long long), st));
  const StepLaunch L = step_args(p, m, params, step);
  const int io_blocks = host_io_blocks();
  for (int k = 0; k < K; ++k) {
    const int64_t beg = k * chunk, cnt = std::min<int64_t>(chunk, n - beg);
    if (cnt <= 0) break;
    const int b = k & 1;
    double* sin[7];
    double* sout[7];
    for (int i = 0; i < 7; ++i) {
      sin[i] = H.stage_in[b] + i * H.cap;
      sout[i] = H.stage_out[b] + i * H.cap;
    }
    // in: the buffer is free once the compute stream has read chunk k - 2
    if (k >= 2) PDF_CUDA(cudaStreamWaitEvent(H.in, H.free_in[b], 0));
    for (int i = 0; i < 7; ++i)
      PDF_CUDA(cudaMemcpyAsync(sin[i], io[i] + beg, sizeof(double) * cnt, cudaMemcpyDefault, H.in));
    PDF_CUDA(cudaMemcpyAsync(H.stage_ie[b], elem + beg, sizeof(int32_t) * cnt, cudaMemcpyDefault, H.in));
    PDF_CUDA(cudaEventRecord(H.loaded[k], H.in));
    // compute: staging -> slots, the step, slots -> staging
    PDF_CUDA(cudaStreamWaitEvent(st, H.loaded[k], 0));
    s = state_in_range(p, sin, H.stage_ie[b], beg, cnt, bad, io_blocks, st, 0);
    if (s != PDF_OK) return s;
    PDF_CUDA(cudaEventRecord(H.free_in[b], st));
    s = L.run(beg, cnt, st);
    if (s != PDF_OK) return s;
    if (k >= 2) PDF_CUDA(cudaStreamWaitEvent(st, H.free_out[b], 0));
    s = state_out_range(p, sout, H.stage_oe[b], beg, cnt, io_blocks, st, 0);
    if (s != PDF_OK) return s;
    PDF_CUDA(cudaEventRecord(H.stepped[k], st));
    // out: the copy engines write the chunk back
    PDF_CUDA(cudaStreamWaitEvent(H.out, H.stepped[k], 0));
    for (int i = 0; i < 7; ++i)
      PDF_CUDA(cudaMemcpyAsync(io[i] + beg, sout[i], sizeof(double) * cnt, cudaMemcpyDefault, H.out));
    PDF_CUDA(cudaMemcpyAsync(elem + beg, H.stage_oe[b], sizeof(int32_t) * cnt, cudaMemcpyDefault, H.out));
    PDF_CUDA(cudaEventRecord(H.free_out[b], H.out));
  }
  p->since_reorder = 0;
  if (stats) {
    s = estimate_stats(p, st);
    if (s != PDF_OK) return s;
    const MeshDev& M = m->d;
    if (es) PDF_CUDA(cudaMemcpyAsync(es, p->es, sizeof(double) * M.n_tri * PDF_NES, cudaMemcpyDefault, st));
    if (ns) PDF_CUDA(cudaMemcpyAsync(ns, p->ns, sizeof(double) * M.n_nodes * PDF_NNS, cudaMemcpyDefault, st));
    if (nd) PDF_CUDA(cudaMemcpyAsync(nd, p->nd, sizeof(double) * M.n_nodes * PDF_NND, cudaMemcpyDefault, st));
  }
  PDF_CUDA(cudaEventRecord(H.done, H.out));
  PDF_CUDA(cudaStreamWaitEvent(st, H.done, 0));
  long long c[16];
  PDF_CUDA(cudaMemcpyAsync(c, p->counters, sizeof(c), cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaStreamSynchronize(st));
  if (c[15]) return fail(PDF_EINVAL, "pdf_step_host: positions must lie within |x|, |y| < 64");
  if (info) {
    info->walk_steps = c[kCntWalk];
    info->reflections = c[kCntRefl];
    info->crossings_periodic = c[kCntPeriodic];
    info->fallbacks = c[kCntFallback];
    info->brute = c[kCntBrute];
    info->lost = c[kCntLost];
    info->omega_reflections = c[kCntOmega];
    info->near_face = c[kCntNear];
  }
  if (c[kCntLost] > 0) return fail(PDF_ELOST, "pdf_step_host: particles lost");
  return PDF_OK;
}

extern "C" pdf_status pdf_step_host(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                                    const double* wp, const double* elem_coeff, uint32_t step, double* x, double* y,
                                    double* u, double* v, double* w, double* om, double* ps, int32_t* elem,
                                    void* stream, pdf_step_info* info) {
  double* const io[7] = {x, y, u, v, w, om, ps};
  return step_host(p, m, params, wp, elem_coeff, step, io, elem, (cudaStream_t)stream, info, false, nullptr,
                   nullptr, nullptr);
}

extern "C" pdf_status pdf_step_host_stats(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                                          const double* wp, const double* elem_coeff, uint32_t step, double* x,
                                          double* y, double* u, double* v, double* w, double* om, double* ps,
                                          int32_t* elem, double* elem_stats, double* node_stats,
                                          double* node_derivs, void* stream, pdf_step_info* info) {
  double* const io[7] = {x, y, u, v, w, om, ps};
  return step_host(p, m, params, wp, elem_coeff, step, io, elem, (cudaStream_t)stream, info, true, elem_stats,
                   node_stats, node_derivs);
}

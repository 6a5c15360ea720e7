// Particle handles: allocation, initialisation (sec. 3.6), state access and
// the exposed Gaussian draw.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "rng.cuh"

namespace pdfgb {

// Radix grouping geometry (see stats.cu).
int64_t radix_tiles(int64_t n);
int32_t radix_bins();
int32_t radix_scan_blocks(int64_t hist_len);

// One thread per particle.  Particle ids run element by element; elem_off is
// the exclusive prefix sum of the per-element counts.
__global__ void k_init(const double* __restrict__ xy, const int32_t* __restrict__ tri,
                       const int64_t* __restrict__ elem_off, int32_t n_tri, int64_t n,
                       uint64_t seed, int32_t u_profile, double u_sigma,
                       const double* __restrict__ elem_psi0, int64_t* __restrict__ x,
                       int64_t* __restrict__ y, fx::df* __restrict__ u, fx::df* __restrict__ v,
                       fx::df* __restrict__ w, fx::df* __restrict__ om, fx::df* __restrict__ ps,
                       int32_t* __restrict__ elem, int32_t* __restrict__ pid, float* __restrict__ uf,
                       float* __restrict__ vf, float* __restrict__ wf, float* __restrict__ omf,
                       float* __restrict__ psf) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    // host element: largest e with elem_off[e] <= p
    int32_t lo = 0, hi = n_tri - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (elem_off[mid] <= p) lo = mid; else hi = mid - 1;
    }
    const int32_t e = lo;
    uint32_t c[4] = {(uint32_t)p, 0u, 0u, kPurposeInit};
    const uint64_t s = seed;
    philox4x32_10(c, (uint32_t)s, (uint32_t)(s >> 32));
    float r1 = u01_from_word(c[0]), r2 = u01_from_word(c[1]);
    if (__fadd_rn(r1, r2) > 1.0f) {
      r1 = __fsub_rn(1.0f, r1);
      r2 = __fsub_rn(1.0f, r2);
    }
    float g[6];
    box_muller(c[2], c[3], &g[0], &g[1]);
    gauss4(seed, (uint32_t)p, 0u, 1u, kPurposeInit, &g[2]);
    uint32_t c2[4] = {(uint32_t)p, 0u, 2u, kPurposeInit};
    philox4x32_10(c2, (uint32_t)s, (uint32_t)(s >> 32));
    float lsum = __fadd_rn(ln_unit(u01_from_word(c2[0])), ln_unit(u01_from_word(c2[1])));
    lsum = __fadd_rn(lsum, ln_unit(u01_from_word(c2[2])));
    lsum = __fadd_rn(lsum, ln_unit(u01_from_word(c2[3])));
    const int32_t na = tri[3 * e], nb = tri[3 * e + 1], nc = tri[3 * e + 2];
    const double xa = xy[2 * na], ya = xy[2 * na + 1];
    const double xb = xy[2 * nb], yb = xy[2 * nb + 1];
    const double xc = xy[2 * nc], yc = xy[2 * nc + 1];
    const double R1 = (double)r1, R2 = (double)r2;
    // uniform point in the triangle, rounded exactly as A + r1 (B-A) + r2 (C-A)
    const double px = __dadd_rn(__dadd_rn(xa, __dmul_rn(R1, __dsub_rn(xb, xa))),
                                __dmul_rn(R2, __dsub_rn(xc, xa)));
    const double py = __dadd_rn(__dadd_rn(ya, __dmul_rn(R1, __dsub_rn(yb, ya))),
                                __dmul_rn(R2, __dsub_rn(yc, ya)));
    const double umean = (u_profile == 1) ? __dsub_rn(1.0, __dmul_rn(py, py)) : (u_profile == 2 ? 1.0 : 0.0);
    x[p] = fx::d2fix((uint64_t)__double_as_longlong(px), kPosF);
    y[p] = fx::d2fix((uint64_t)__double_as_longlong(py), kPosF);
    const double U = __dadd_rn(umean, __dmul_rn(u_sigma, (double)g[0]));
    const double V = __dmul_rn(u_sigma, (double)g[1]);
    const double W = __dmul_rn(u_sigma, (double)g[2]);
    const double O = __dmul_rn(-0.25, (double)lsum);   // Gamma(4, 1/4): -1/4 sum of 4 ln u
    const double S = elem_psi0 ? elem_psi0[e] : 0.0;
    if (u) {
      u[p] = fx::from_double(U); v[p] = fx::from_double(V); w[p] = fx::from_double(W);
      om[p] = fx::from_double(O); ps[p] = fx::from_double(S);
    } else {  // FP32 state: the FP64 values rounded to nearest
      uf[p] = __double2float_rn(U); vf[p] = __double2float_rn(V); wf[p] = __double2float_rn(W);
      omf[p] = __double2float_rn(O); psf[p] = __double2float_rn(S);
    }
    elem[p] = e;
    pid[p] = (int32_t)p;
  }
}

__global__ void k_rng_gauss(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n,
                            float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float g[4];
    gauss4(seed, (uint32_t)i, c1, c2, c3, g);
    out[i] = make_float4(g[0], g[1], g[2], g[3]);
  }
}

// Stored representation in storage order -> FP64 in particle-id order
// (get_state) and back (set_state, which leaves the storage in id order).
__global__ void k_fix_to_f64(const int64_t* __restrict__ a, const int32_t* __restrict__ pid,
                             double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[pid[i]] = __longlong_as_double((long long)fx::fix2d(a[i], kPosF));
}

__global__ void k_df_to_f64(const fx::df* __restrict__ a, const int32_t* __restrict__ pid,
                            double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[pid[i]] = __longlong_as_double((long long)fx::df2d_rn(a[i]));
}

__global__ void k_f32_to_f64(const float* __restrict__ a, const int32_t* __restrict__ pid,
                             double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[pid[i]] = __longlong_as_double((long long)fx::f2d_bits(a[i]));
}

__global__ void k_elem_by_id(const int32_t* __restrict__ a, const int32_t* __restrict__ pid,
                             int32_t* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[pid[i]] = a[i];
}

__global__ void k_iota(int32_t* __restrict__ a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

// Positions outside |x| < 64 are counted in *bad and stored as 0.
__global__ void k_f64_to_fix(const double* __restrict__ a, int64_t* __restrict__ b, int64_t n,
                             unsigned long long* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t bits = (uint64_t)__double_as_longlong(a[i]);
    if (fx::d_exp(bits) <= 1023 + 5) {
      b[i] = fx::d2fix(bits, kPosF);
    } else {
      b[i] = 0;
      atomicAdd(bad, 1ull);
    }
  }
}

__global__ void k_f64_to_df(const double* __restrict__ a, fx::df* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = fx::d2df_rn((uint64_t)__double_as_longlong(a[i]));
}

__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = fx::d2df_rn((uint64_t)__double_as_longlong(a[i])).h;  // the FP64 -> FP32 rounding
}

// Whole-state transfers in one pass, for caller buffers the kernels can
// address (device memory, or page-locked host memory through its mapping:
// the copy then runs as the kernel's own loads and stores over the
// host link, with no staging).  Out: destination q (particle id) reads slot
// inv[q], so that the stores to host memory are consecutive.
struct StateOut {
  int64_t n;
  const int32_t* inv;
  const int64_t *x, *y;
  const fx::df* d[5];
  const float* f[5];
  const int32_t* elem;
  double* o[7];  // x, y, u, v, w, om, ps (nullable)
  int32_t* oe;   // elem (nullable)
};

__global__ void k_inv_pid(const int32_t* __restrict__ pid, int32_t* __restrict__ inv, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    inv[pid[i]] = (int32_t)i;
}

__global__ void k_state_out(StateOut S) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < S.n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = S.inv ? S.inv[q] : q;  // no permutation: slot = particle id
    if (S.o[0]) S.o[0][q] = __longlong_as_double((long long)fx::fix2d(S.x[i], kPosF));
    if (S.o[1]) S.o[1][q] = __longlong_as_double((long long)fx::fix2d(S.y[i], kPosF));
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (S.o[2 + k])
        S.o[2 + k][q] = __longlong_as_double((long long)(S.d[k] ? fx::df2d_rn(S.d[k][i]) : fx::f2d_bits(S.f[k][i])));
    if (S.oe) S.oe[q] = S.elem[i];
  }
}

// In: slot i takes particle pid0 + i; positions outside |x| < 64 are
// counted in *bad and stored as 0.
struct StateIn {
  int64_t n, pid0;
  const double* in[7];  // x, y, u, v, w, om, ps
  const int32_t* ie;
  int64_t *x, *y;
  fx::df* d[5];
  float* f[5];
  int32_t *elem, *pid;
  unsigned long long* bad;
};

__global__ void k_state_in(StateIn S) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint64_t bits = (uint64_t)__double_as_longlong(S.in[k][i]);
      int64_t v = 0;
      if (fx::d_exp(bits) <= 1023 + 5) v = fx::d2fix(bits, kPosF);
      else atomicAdd(S.bad, 1ull);
      (k == 0 ? S.x : S.y)[i] = v;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      // the stored forms without FP64 instructions (bit-identical to
      // from_double and to the FP64 -> FP32 rounding)
      const fx::df v = fx::d2df_rn((uint64_t)__double_as_longlong(S.in[2 + k][i]));
      if (S.d[k]) S.d[k][i] = v;
      else S.f[k][i] = v.h;
    }
    S.elem[i] = S.ie[i];
    S.pid[i] = (int32_t)(S.pid0 + i);
  }
}

static void free_particles(pdf_particles* p) {
  if (!p) return;
  cudaFree(p->uf); cudaFree(p->vf); cudaFree(p->wf); cudaFree(p->omf); cudaFree(p->psf); cudaFree(p->rows_f32);
  cudaFree(p->x); cudaFree(p->y);
  cudaFree(p->u); cudaFree(p->v); cudaFree(p->w); cudaFree(p->om); cudaFree(p->ps);
  cudaFree(p->x2); cudaFree(p->y2);
  cudaFree(p->u2); cudaFree(p->v2); cudaFree(p->w2); cudaFree(p->om2); cudaFree(p->ps2);
  cudaFree(p->uf2); cudaFree(p->vf2); cudaFree(p->wf2); cudaFree(p->omf2); cudaFree(p->psf2);
  cudaFree(p->pid); cudaFree(p->pid2);
  cudaFree(p->cond); cudaFree(p->iecm_scratch_f); cudaFree(p->iecm_scratch_i);
  cudaFree(p->stage);
  double* dbl[] = {p->es, p->ns, p->nd, p->eg, p->nc, p->rows};
  for (double* d : dbl) cudaFree(d);
  cudaFree(p->elem);
  cudaFree(p->rows_fx);
  cudaFree(p->keys[0]); cudaFree(p->keys[1]); cudaFree(p->vals[0]); cudaFree(p->vals[1]);
  cudaFree(p->hist); cudaFree(p->hist_part); cudaFree(p->seg);
  cudaFree(p->counters);
  cudaFree(p->pres); cudaFree(p->gradP);
  {
    HostIo& H = p->hio;
    if (H.in) cudaStreamDestroy(H.in);
    if (H.out) cudaStreamDestroy(H.out);
    if (H.start) cudaEventDestroy(H.start);
    if (H.done) cudaEventDestroy(H.done);
    for (int b = 0; b < 2; ++b) {
      if (H.free_in[b]) cudaEventDestroy(H.free_in[b]);
      if (H.free_out[b]) cudaEventDestroy(H.free_out[b]);
      cudaFree(H.stage_in[b]); cudaFree(H.stage_out[b]); cudaFree(H.stage_ie[b]); cudaFree(H.stage_oe[b]);
    }
    for (int k = 0; k < kHostChunks; ++k) {
      if (H.loaded[k]) cudaEventDestroy(H.loaded[k]);
      if (H.stepped[k]) cudaEventDestroy(H.stepped[k]);
    }
  }
  relax_free(p->rx);
  press_free(p->pw);
  redist_free(p->rd);
  delete p;
}

pdf_status stats_only_handle(const pdf_mesh* m, pdf_particles** out) {
  *out = nullptr;
  pdf_particles* P = new pdf_particles();
  P->mesh = m;
  const size_t nn = (size_t)m->d.n_nodes, nt = (size_t)m->d.n_tri;
  cudaError_t e = cudaMalloc((void**)&P->ns, sizeof(double) * nn * PDF_NNS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&P->nd, sizeof(double) * nn * PDF_NND);
  if (e == cudaSuccess) e = cudaMalloc((void**)&P->eg, sizeof(double) * nt * 8);
  if (e != cudaSuccess) {
    free_particles(P);
    return fail(PDF_ENOMEM, "pdf_relax_solve: cudaMalloc failed");
  }
  *out = P;
  return PDF_OK;
}

void release_particles(pdf_particles* p) { free_particles(p); }

static int grid_for(int64_t n, int threads) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 16;
  return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

}  // namespace pdfgb

using namespace pdfgb;

#define TRY_ALLOC(ptr, count)                                                        \
  do {                                                                               \
    cudaError_t _e = cudaMalloc((void**)&(ptr), (size_t)(count) * sizeof(*(ptr)));  \
    if (_e != cudaSuccess) {                                                         \
      free_particles(P);                                                             \
      return fail(PDF_ENOMEM, "pdf_particles_init: cudaMalloc failed");              \
    }                                                                                \
  } while (0)

#define SA(ptr, count)                                                              \
  do {                                                                              \
    cudaError_t _e = cudaMalloc((void**)&(ptr), (size_t)(count) * sizeof(*(ptr))); \
    if (_e != cudaSuccess) return fail(PDF_ENOMEM, "particle state: cudaMalloc failed"); \
  } while (0)

namespace pdfgb {
// Device arrays of a particle set of P->n particles on P->mesh with
// P->precision; statistics, counters and the pressure field zeroed.  On
// failure the caller releases what was allocated (free_particles).
pdf_status alloc_state(pdf_particles* P, cudaStream_t st) {
  const int64_t n = P->n;
  const int32_t precision = P->precision;
  const int32_t n_tri = P->mesh->d.n_tri, n_nodes = P->mesh->d.n_nodes;
  SA(P->x, n); SA(P->y, n); SA(P->elem, n); SA(P->pid, n);
  SA(P->x2, n); SA(P->y2, n); SA(P->pid2, n);
  if (precision == PDF_FP64) {
    SA(P->u, n); SA(P->v, n); SA(P->w, n); SA(P->om, n); SA(P->ps, n);
    SA(P->u2, n); SA(P->v2, n); SA(P->w2, n); SA(P->om2, n); SA(P->ps2, n);
  } else {
    SA(P->uf, n); SA(P->vf, n); SA(P->wf, n); SA(P->omf, n); SA(P->psf, n);
    SA(P->uf2, n); SA(P->vf2, n); SA(P->wf2, n); SA(P->omf2, n); SA(P->psf2, n);
    SA(P->rows_f32, (int64_t)n_tri * PDFGB_ROW);
  }
  SA(P->es, (int64_t)n_tri * PDF_NES);
  SA(P->ns, (int64_t)n_nodes * PDF_NNS);
  SA(P->nd, (int64_t)n_nodes * PDF_NND);
  SA(P->eg, (int64_t)n_tri * 8);
  SA(P->nc, (int64_t)n_nodes * PDF_NCOEF);
  SA(P->rows, (int64_t)n_tri * PDFGB_ROW);
  SA(P->rows_fx, (int64_t)n_tri);
  SA(P->keys[0], n); SA(P->keys[1], n);
  SA(P->vals[0], n); SA(P->vals[1], n);
  P->n_tiles = radix_tiles(n);
  P->hist_len = P->n_tiles * radix_bins();
  P->n_scan_blocks = radix_scan_blocks(P->hist_len);
  SA(P->hist, P->hist_len);
  SA(P->hist_part, P->n_scan_blocks + 1);
  SA(P->seg, (int64_t)n_tri + 1);
  SA(P->counters, 16);
  SA(P->pres, n_nodes);
  SA(P->gradP, 2 * (int64_t)n_nodes);
  cudaError_t e = cudaMemsetAsync(P->ns, 0, sizeof(double) * n_nodes * PDF_NNS, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->counters, 0, sizeof(long long) * 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->pres, 0, sizeof(double) * n_nodes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->gradP, 0, sizeof(double) * 2 * n_nodes, st);
  if (e != cudaSuccess) return cuda_fail(e, "particle state: initial memsets");
  return PDF_OK;
}
}  // namespace pdfgb
#undef SA

extern "C" pdf_status pdf_particles_init(const pdf_mesh* m, const pdf_init_params* ip,
                                         uint64_t seed, int32_t precision, void* stream,
                                         pdf_particles** out) {
  if (!out) return fail(PDF_EINVAL, "pdf_particles_init: out is NULL");
  *out = nullptr;
  if (!m || !ip) return fail(PDF_EINVAL, "pdf_particles_init: NULL mesh or params");
  if (precision != PDF_FP64 && precision != PDF_FP32_STATE) return fail(PDF_EINVAL, "pdf_particles_init: unknown precision");
  const int32_t n_tri = m->d.n_tri, n_nodes = m->d.n_nodes;
  std::vector<int64_t> off(n_tri + 1, 0);
  for (int32_t e = 0; e < n_tri; ++e) {
    const int64_t c = ip->count ? ip->count[e] : ip->ppe;
    if (c < 0) return fail(PDF_EINVAL, "pdf_particles_init: negative particle count");
    off[e + 1] = off[e] + c;
  }
  const int64_t n = off[n_tri];
  if (n < 1 || n > (int64_t)INT32_MAX) return fail(PDF_EINVAL, "pdf_particles_init: particle count must be in [1, 2^31)");
  cudaStream_t st = (cudaStream_t)stream;
  pdf_particles* P = new (std::nothrow) pdf_particles();
  if (!P) return fail(PDF_ENOMEM, "pdf_particles_init: host allocation");
  P->mesh = m;
  P->n = n;
  P->precision = precision;
  P->seed = seed;
  pdf_status as = alloc_state(P, st);
  if (as != PDF_OK) {
    free_particles(P);
    return as;
  }
  cudaError_t e = cudaSuccess;
  int64_t* d_off = nullptr;
  double* d_psi = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_off, sizeof(int64_t) * (n_tri + 1));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (n_tri + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && ip->elem_psi0) {
    e = cudaMalloc(&d_psi, sizeof(double) * n_tri);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_psi, ip->elem_psi0, sizeof(double) * n_tri, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) {
    prof_launch("k_init", st, nullptr, nullptr);  // counted only
    k_init<<<grid_for(n, 256), 256, 0, st>>>(m->d.xy, m->d.tri, d_off, n_tri, n, seed,
                                              ip->u_profile, ip->u_sigma, d_psi, P->x, P->y, P->u,
                                              P->v, P->w, P->om, P->ps, P->elem, P->pid, P->uf, P->vf,
                                              P->wf, P->omf, P->psf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_off);
  cudaFree(d_psi);
  if (e != cudaSuccess) {
    free_particles(P);
    return cuda_fail(e, "pdf_particles_init");
  }
  *out = P;
  return PDF_OK;
}

extern "C" pdf_status pdf_particles_destroy(pdf_particles* p) {
  free_particles(p);
  return PDF_OK;
}

extern "C" pdf_status pdf_particles_count(const pdf_particles* p, int64_t* n) {
  if (!p || !n) return fail(PDF_EINVAL, "pdf_particles_count: NULL argument");
  *n = p->n;
  return PDF_OK;
}

static bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The address a kernel uses for a caller's buffer: device or managed memory
// as it is, page-locked host memory through its mapping; nullptr for
// pageable host memory (which goes through the staging buffer).
static void* kernel_view(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return const_cast<void*>(ptr);
  if (at.type == cudaMemoryTypeHost && at.devicePointer) return at.devicePointer;
  return nullptr;
}

static pdf_status ensure_stage(const pdf_particles* p) {
  pdf_particles* q = const_cast<pdf_particles*>(p);
  if (!q->stage) PDF_CUDA(cudaMalloc((void**)&q->stage, sizeof(double) * (size_t)p->n));
  return PDF_OK;
}

namespace pdfgb {

void* state_kernel_view(const void* ptr) { return kernel_view(ptr); }

// Grid of the state conversion kernels: four blocks per SM.  For
// get_state / set_state they read and write the caller's page-locked arrays
// through the mapping, and four blocks per SM keep enough loads and stores
// in flight for the host link; pdf_step_host's conversions run between
// device staging buffers and the slots.
int host_io_blocks() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 4 * (sms > 0 ? sms : 148);
}

pdf_status host_io_init(pdf_particles* p) {
  HostIo& H = p->hio;
  if (H.in) return PDF_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&H.in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&H.out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H.start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H.done, cudaEventDisableTiming);
  for (int k = 0; k < kHostChunks && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&H.loaded[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H.stepped[k], cudaEventDisableTiming);
  }
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&H.free_in[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H.free_out[b], cudaEventDisableTiming);
  }
  return e == cudaSuccess ? PDF_OK : cuda_fail(e, "pdf_step_host: streams and events");
}

pdf_status host_io_stage(pdf_particles* p, int64_t cap) {
  HostIo& H = p->hio;
  if (H.cap >= cap) return PDF_OK;
  for (int b = 0; b < 2; ++b) {
    cudaFree(H.stage_in[b]); cudaFree(H.stage_out[b]); cudaFree(H.stage_ie[b]); cudaFree(H.stage_oe[b]);
    H.stage_in[b] = H.stage_out[b] = nullptr;
    H.stage_ie[b] = H.stage_oe[b] = nullptr;
  }
  H.cap = 0;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc((void**)&H.stage_in[b], sizeof(double) * 7 * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&H.stage_out[b], sizeof(double) * 7 * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&H.stage_ie[b], sizeof(int32_t) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&H.stage_oe[b], sizeof(int32_t) * (size_t)cap);
  }
  if (e != cudaSuccess) return fail(PDF_ENOMEM, "pdf_step_host: staging buffers");
  H.cap = cap;
  return PDF_OK;
}

pdf_status state_in_range(pdf_particles* p, double* const in[7], const int32_t* ie, int64_t beg, int64_t cnt,
                          unsigned long long* bad, int blocks, cudaStream_t st, int64_t io_off) {
  p->have_cond = false;  // the conditioned means follow the old slot order
  StateIn S;
  S.n = cnt;
  S.pid0 = beg;
  for (int i = 0; i < 7; ++i) S.in[i] = in[i] + io_off;
  S.ie = ie + io_off;
  S.x = p->x + beg;
  S.y = p->y + beg;
  fx::df* dd[5] = {p->u, p->v, p->w, p->om, p->ps};
  float* ff[5] = {p->uf, p->vf, p->wf, p->omf, p->psf};
  for (int k = 0; k < 5; ++k) {
    S.d[k] = p->precision == PDF_FP64 ? dd[k] + beg : nullptr;
    S.f[k] = p->precision == PDF_FP64 ? nullptr : ff[k] + beg;
  }
  S.elem = p->elem + beg;
  S.pid = p->pid + beg;
  S.bad = bad;
  PDF_KERNEL("k_state_in", st, k_state_in<<<blocks, 256, 0, st>>>(S));
  return PDF_OK;
}

pdf_status state_out_range(const pdf_particles* p, double* const out[7], int32_t* oe, int64_t beg, int64_t cnt,
                           int blocks, cudaStream_t st, int64_t io_off) {
  StateOut S;
  S.n = cnt;
  S.inv = nullptr;
  S.x = p->x + beg;
  S.y = p->y + beg;
  const fx::df* dd[5] = {p->u, p->v, p->w, p->om, p->ps};
  const float* ff[5] = {p->uf, p->vf, p->wf, p->omf, p->psf};
  for (int k = 0; k < 5; ++k) {
    S.d[k] = p->precision == PDF_FP64 ? dd[k] + beg : nullptr;
    S.f[k] = p->precision == PDF_FP64 ? nullptr : ff[k] + beg;
  }
  S.elem = p->elem + beg;
  for (int i = 0; i < 7; ++i) S.o[i] = out[i] + io_off;
  S.oe = oe + io_off;
  PDF_KERNEL("k_state_out", st, k_state_out<<<blocks, 256, 0, st>>>(S));
  return PDF_OK;
}

}  // namespace pdfgb

extern "C" pdf_status pdf_particles_get_state(const pdf_particles* p, double* x, double* y,
                                              double* u, double* v, double* w, double* om,
                                              double* ps, int32_t* elem, void* stream) {
  if (!p) return fail(PDF_EINVAL, "pdf_particles_get_state: NULL handle");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t b = sizeof(double) * p->n;
  double* dst[] = {x, y, u, v, w, om, ps};
  {
    // one pass when every destination is addressable by the kernels
    StateOut S;
    bool all = true;
    for (int i = 0; i < 7; ++i) {
      S.o[i] = dst[i] ? static_cast<double*>(kernel_view(dst[i])) : nullptr;
      if (dst[i] && !S.o[i]) all = false;
    }
    S.oe = elem ? static_cast<int32_t*>(kernel_view(elem)) : nullptr;
    if (elem && !S.oe) all = false;
    if (all && p->n > 0) {
      pdf_status s = ensure_stage(p);
      if (s != PDF_OK) return s;
      int32_t* inv = reinterpret_cast<int32_t*>(p->stage);
      const int g = grid_for(p->n, 256);
      PDF_KERNEL("k_inv_pid", st, k_inv_pid<<<g, 256, 0, st>>>(p->pid, inv, p->n));
      S.n = p->n;
      S.inv = inv;
      S.x = p->x;
      S.y = p->y;
      const fx::df* dd[5] = {p->u, p->v, p->w, p->om, p->ps};
      const float* ff[5] = {p->uf, p->vf, p->wf, p->omf, p->psf};
      for (int k = 0; k < 5; ++k) {
        S.d[k] = p->precision == PDF_FP64 ? dd[k] : nullptr;
        S.f[k] = ff[k];
      }
      S.elem = p->elem;
      PDF_KERNEL("k_state_out", st, k_state_out<<<g, 256, 0, st>>>(S));
      return PDF_OK;
    }
  }
  const fx::df* srcd[] = {nullptr, nullptr, p->u, p->v, p->w, p->om, p->ps};
  const float* srcf[] = {nullptr, nullptr, p->uf, p->vf, p->wf, p->omf, p->psf};
  const int g = grid_for(p->n, 256);
  for (int i = 0; i < 7; ++i) {
    if (!dst[i]) continue;
    // convert on the device, straight into a device destination or through
    // the staging buffer for host memory
    const bool dev = is_device_ptr(dst[i]);
    if (!dev) {
      pdf_status s = ensure_stage(p);
      if (s != PDF_OK) return s;
    }
    double* to = dev ? dst[i] : p->stage;
    if (i < 2) {
      const int64_t* a = i == 0 ? p->x : p->y;
      PDF_KERNEL("k_fix_to_f64", st, k_fix_to_f64<<<g, 256, 0, st>>>(a, p->pid, to, p->n));
    } else if (srcd[i]) {
      PDF_KERNEL("k_df_to_f64", st, k_df_to_f64<<<g, 256, 0, st>>>(srcd[i], p->pid, to, p->n));
    } else {
      PDF_KERNEL("k_f32_to_f64", st, k_f32_to_f64<<<g, 256, 0, st>>>(srcf[i], p->pid, to, p->n));
    }
    if (!dev) PDF_CUDA(cudaMemcpyAsync(dst[i], p->stage, b, cudaMemcpyDeviceToHost, st));
  }
  if (elem) {
    const bool dev = is_device_ptr(elem);
    if (!dev) {
      pdf_status s = ensure_stage(p);
      if (s != PDF_OK) return s;
    }
    int32_t* to = dev ? elem : reinterpret_cast<int32_t*>(p->stage);
    PDF_KERNEL("k_elem_by_id", st, k_elem_by_id<<<g, 256, 0, st>>>(p->elem, p->pid, to, p->n));
    if (!dev) PDF_CUDA(cudaMemcpyAsync(elem, p->stage, sizeof(int32_t) * p->n, cudaMemcpyDeviceToHost, st));
  }
  return PDF_OK;
}

extern "C" pdf_status pdf_particles_set_state(pdf_particles* p, const double* x, const double* y,
                                              const double* u, const double* v, const double* w,
                                              const double* om, const double* ps,
                                              const int32_t* elem, void* stream) {
  if (!p || !x || !y || !u || !v || !w || !om || !ps || !elem)
    return fail(PDF_EINVAL, "pdf_particles_set_state: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t b = sizeof(double) * p->n;
  fx::df* dstd[] = {nullptr, nullptr, p->u, p->v, p->w, p->om, p->ps};
  float* dstf[] = {nullptr, nullptr, p->uf, p->vf, p->wf, p->omf, p->psf};
  const double* src[] = {x, y, u, v, w, om, ps};
  const int g = grid_for(p->n, 256);
  unsigned long long* bad = reinterpret_cast<unsigned long long*>(p->counters + 15);
  PDF_CUDA(cudaMemsetAsync(bad, 0, sizeof(long long), st));
  StateIn S;
  bool all = true;
  for (int i = 0; i < 7; ++i) {
    S.in[i] = static_cast<const double*>(kernel_view(src[i]));
    if (!S.in[i]) all = false;
  }
  S.ie = static_cast<const int32_t*>(kernel_view(elem));
  if (!S.ie) all = false;
  if (all) {  // one pass reading every source where it is
    S.n = p->n;
    S.pid0 = 0;
    S.x = p->x;
    S.y = p->y;
    for (int k = 0; k < 5; ++k) {
      S.d[k] = dstd[2 + k];
      S.f[k] = dstf[2 + k];
    }
    S.elem = p->elem;
    S.pid = p->pid;
    S.bad = bad;
    if (p->n > 0) PDF_KERNEL("k_state_in", st, k_state_in<<<g, 256, 0, st>>>(S));
  }
  for (int i = 0; i < 7 && !all; ++i) {
    const bool dev = is_device_ptr(src[i]);
    if (!dev) {
      pdf_status s = ensure_stage(p);
      if (s != PDF_OK) return s;
      PDF_CUDA(cudaMemcpyAsync(p->stage, src[i], b, cudaMemcpyHostToDevice, st));
    }
    const double* from = dev ? src[i] : p->stage;
    if (i < 2) {
      int64_t* a = i == 0 ? p->x : p->y;
      PDF_KERNEL("k_f64_to_fix", st, k_f64_to_fix<<<g, 256, 0, st>>>(from, a, p->n, bad));
    } else if (dstd[i]) {
      PDF_KERNEL("k_f64_to_df", st, k_f64_to_df<<<g, 256, 0, st>>>(from, dstd[i], p->n));
    } else {
      PDF_KERNEL("k_f64_to_f32", st, k_f64_to_f32<<<g, 256, 0, st>>>(from, dstf[i], p->n));
    }
  }
  if (!all) {
    PDF_CUDA(cudaMemcpyAsync(p->elem, elem, sizeof(int32_t) * p->n, cudaMemcpyDefault, st));
    PDF_KERNEL("k_iota", st, k_iota<<<g, 256, 0, st>>>(p->pid, p->n));
  }
  p->since_reorder = 0;
  p->have_cond = false;
  long long nbad = 0;
  PDF_CUDA(cudaMemcpyAsync(&nbad, bad, sizeof(long long), cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaStreamSynchronize(st));
  if (nbad) return fail(PDF_EINVAL, "pdf_particles_set_state: positions must lie within |x|, |y| < 64");
  return PDF_OK;
}

extern "C" pdf_status pdf_particles_set_reorder(pdf_particles* p, int32_t every) {
  if (!p || every < 0) return fail(PDF_EINVAL, "pdf_particles_set_reorder: NULL handle or negative interval");
  p->reorder_every = every;
  p->since_reorder = 0;
  return PDF_OK;
}

extern "C" pdf_status pdf_rng_gauss(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n,
                                    float* out, void* stream) {
  if (n < 0 || (n > 0 && !out)) return fail(PDF_EINVAL, "pdf_rng_gauss: bad arguments");
  if (n == 0) return PDF_OK;
  if ((reinterpret_cast<uintptr_t>(out) & 15) != 0) return fail(PDF_EINVAL, "pdf_rng_gauss: out must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  PDF_KERNEL("k_rng_gauss", st, k_rng_gauss<<<grid_for(n, 256), 256, 0, st>>>(seed, c1, c2, c3, n, (float4*)out));
  return PDF_OK;
}

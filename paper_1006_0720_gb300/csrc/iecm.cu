// Velocity-conditioned scalar mean for the IECM micromixing model (eq.
// IECM), computed with the sort-and-divide binning of the section on
// conditional statistics and its appendix: the particles of an element are
// sorted by U and divided into parts of equal count (up to one); each part
// is sorted by V and divided, each subpart by W; the conditional mean of a
// particle is the scalar mean of its final part.  A group of n particles is
// divided into k = min(n_c, n / m_min) parts (at least one), part j holding
// the sorted positions i with floor(k i / n) = j; equal velocity components
// are ordered by particle id.
//
// One block per element.  The element's particles are copied into shared
// memory (or, above kIecmCap particles, into a global scratch slice) and
// sorted by rank counting inside each group: O(n^2) comparisons per level,
// fine for the tens to hundreds of particles per element the method uses.
#include "common.cuh"
#include "fx.cuh"

namespace pdfgb {

constexpr int kIecmThreads = 128;
constexpr int kIecmCap = 512;

struct IecmView {  // per-particle working arrays (shared or global)
  float *uh, *ul, *vh, *vl, *wh, *wl;
  float *sh, *sl;  // the scalar
  int32_t *id, *slot, *perm, *perm2, *gs, *ge;
};

__device__ __forceinline__ void load_comp(const fx::df* a, int64_t s, float& h, float& l) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(a) + s);
  h = v.x;
  l = v.y;
}
__device__ __forceinline__ void load_comp(const float* a, int64_t s, float& h, float& l) {
  h = __ldg(a + s);
  l = 0.0f;
}

// (key_i, id_i) < (key_j, id_j) for double-float keys (normalized pairs
// order like their values)
__device__ __forceinline__ bool key_less(float hi, float li, int32_t ii, float hj, float lj, int32_t ij) {
  return hi < hj || (hi == hj && (li < lj || (li == lj && ii < ij)));
}

template <typename T>
__global__ void __launch_bounds__(kIecmThreads) k_iecm_cond(const int32_t* __restrict__ seg,
                                                            const int32_t* __restrict__ order, int32_t n_tri,
                                                            const T* __restrict__ u, const T* __restrict__ v,
                                                            const T* __restrict__ w, const T* __restrict__ ps,
                                                            const int32_t* __restrict__ pid, int nc0, int nc1,
                                                            int nc2, int m_min, IecmView big,
                                                            fx::df* __restrict__ cond) {
  __shared__ float s_f[8][kIecmCap];
  __shared__ int32_t s_i[6][kIecmCap];
  const int tid = threadIdx.x;
  for (int32_t e = blockIdx.x; e < n_tri; e += gridDim.x) {
    const int32_t beg = seg[e], N = seg[e + 1] - beg;
    if (N == 0) continue;
    IecmView V;
    if (N <= kIecmCap) {
      V = IecmView{s_f[0], s_f[1], s_f[2], s_f[3], s_f[4], s_f[5], s_f[6], s_f[7],
                   s_i[0], s_i[1], s_i[2], s_i[3], s_i[4], s_i[5]};
    } else {  // the element's slice of the global scratch
      V = IecmView{big.uh + beg, big.ul + beg, big.vh + beg, big.vl + beg, big.wh + beg, big.wl + beg,
                   big.sh + beg, big.sl + beg, big.id + beg, big.slot + beg, big.perm + beg,
                   big.perm2 + beg, big.gs + beg, big.ge + beg};
    }
    __syncthreads();  // the previous element is done with the arrays
    for (int i = tid; i < N; i += kIecmThreads) {
      const int64_t s = order ? (int64_t)order[beg + i] : (int64_t)(beg + i);
      V.slot[i] = (int32_t)s;
      V.id[i] = pid[s];
      load_comp(u, s, V.uh[i], V.ul[i]);
      load_comp(v, s, V.vh[i], V.vl[i]);
      load_comp(w, s, V.wh[i], V.wl[i]);
      load_comp(ps, s, V.sh[i], V.sl[i]);
      V.perm[i] = i;
      V.gs[i] = 0;
      V.ge[i] = N;
    }
    __syncthreads();
    const int ncs[3] = {nc0, nc1, nc2};
    for (int level = 0; level < 3; ++level) {
      const float* kh = level == 0 ? V.uh : (level == 1 ? V.vh : V.wh);
      const float* kl = level == 0 ? V.ul : (level == 1 ? V.vl : V.wl);
      // sort each group [gs, ge) by rank counting
      for (int pos = tid; pos < N; pos += kIecmThreads) {
        const int32_t i = V.perm[pos];
        const int32_t a = V.gs[pos], b = V.ge[pos];
        const float hi = kh[i], li = kl[i];
        const int32_t ii = V.id[i];
        int32_t r = 0;
        for (int32_t q = a; q < b; ++q) {
          const int32_t j = V.perm[q];
          r += key_less(kh[j], kl[j], V.id[j], hi, li, ii) ? 1 : 0;
        }
        V.perm2[a + r] = i;
      }
      __syncthreads();
      // divide each group into k parts of equal count
      for (int pos = tid; pos < N; pos += kIecmThreads) {
        const int32_t a = V.gs[pos], n = V.ge[pos] - a;
        int32_t k = n / m_min;
        if (k > ncs[level]) k = ncs[level];
        if (k < 1) k = 1;
        const int32_t j = (int32_t)(((int64_t)k * (pos - a)) / n);
        V.gs[pos] = a + (int32_t)(((int64_t)j * n + k - 1) / k);
        V.ge[pos] = a + (int32_t)(((int64_t)(j + 1) * n + k - 1) / k);
        V.perm[pos] = V.perm2[pos];
      }
      __syncthreads();
    }
    // bin means: the first position of each bin adds its bin in sorted order
    // (double-float) and stores the mean at that position
    for (int pos = tid; pos < N; pos += kIecmThreads) {
      const int32_t a = V.gs[pos], b = V.ge[pos];
      if (pos != a) continue;
      fx::acc s;
      s.init(fx::df{V.sh[V.perm[a]], V.sl[V.perm[a]]});
      for (int32_t q = a + 1; q < b; ++q) s.add(fx::df{V.sh[V.perm[q]], V.sl[V.perm[q]]});
      const fx::df mean = fx::df_norm(fx::mul(s.value(), fx::recip_df(b - a)));
      V.uh[a] = mean.h;  // the sort keys are no longer needed
      V.ul[a] = mean.l;
    }
    __syncthreads();
    for (int pos = tid; pos < N; pos += kIecmThreads) {
      const int32_t a = V.gs[pos];
      reinterpret_cast<float2*>(cond)[V.slot[V.perm[pos]]] = make_float2(V.uh[a], V.ul[a]);
    }
  }
}

static int iecm_blocks(int32_t n_tri) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<int64_t>(1, std::min<int64_t>(n_tri, (int64_t)sms * 16));
}

// Conditional means of every particle from the grouping in seg / order
// (order: storage slot of each grouped position, NULL for the identity).
pdf_status iecm_cond(pdf_particles* P, const int32_t* seg, const int32_t* order, cudaStream_t st) {
  if (P->iecm_bins[0] <= 0) return PDF_OK;
  const MeshDev& M = P->mesh->d;
  IecmView big;
  float* f = P->iecm_scratch_f;
  int32_t* g = P->iecm_scratch_i;
  const int64_t n = P->n;
  big = IecmView{f, f + n, f + 2 * n, f + 3 * n, f + 4 * n, f + 5 * n, f + 6 * n, f + 7 * n,
                 g, g + n, g + 2 * n, g + 3 * n, g + 4 * n, g + 5 * n};
  const int nb = iecm_blocks(M.n_tri);
  if (P->precision == PDF_FP64) {
    PDF_KERNEL("k_iecm_cond", st, k_iecm_cond<fx::df><<<nb, kIecmThreads, 0, st>>>(
                                      seg, order, M.n_tri, P->u, P->v, P->w, P->ps, P->pid, P->iecm_bins[0],
                                      P->iecm_bins[1], P->iecm_bins[2], P->iecm_min, big, P->cond));
  } else {
    PDF_KERNEL("k_iecm_cond", st, k_iecm_cond<float><<<nb, kIecmThreads, 0, st>>>(
                                      seg, order, M.n_tri, P->uf, P->vf, P->wf, P->psf, P->pid, P->iecm_bins[0],
                                      P->iecm_bins[1], P->iecm_bins[2], P->iecm_min, big, P->cond));
  }
  P->have_cond = true;
  return PDF_OK;
}

__global__ void k_cond_to_f64(const fx::df* __restrict__ a, const int32_t* __restrict__ pid,
                              double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[pid[i]] = fx::to_double(a[i]);
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_particles_set_iecm(pdf_particles* p, int32_t nu, int32_t nv, int32_t nw,
                                             int32_t m_min) {
  if (!p) return fail(PDF_EINVAL, "pdf_particles_set_iecm: NULL handle");
  if (nu == 0 && nv == 0 && nw == 0) {
    p->iecm_bins[0] = p->iecm_bins[1] = p->iecm_bins[2] = 0;
    p->have_cond = false;
    return PDF_OK;
  }
  if (nu < 1 || nv < 1 || nw < 1 || m_min < 1)
    return fail(PDF_EINVAL, "pdf_particles_set_iecm: bins and m_min must be >= 1 (or all bins 0 to disable)");
  if (!p->cond) {
    const size_t n = (size_t)p->n;
    PDF_CUDA(cudaMalloc((void**)&p->cond, sizeof(fx::df) * n));
    PDF_CUDA(cudaMalloc((void**)&p->iecm_scratch_f, sizeof(float) * 8 * n));
    PDF_CUDA(cudaMalloc((void**)&p->iecm_scratch_i, sizeof(int32_t) * 6 * n));
  }
  p->iecm_bins[0] = nu;
  p->iecm_bins[1] = nv;
  p->iecm_bins[2] = nw;
  p->iecm_min = m_min;
  p->have_cond = false;
  return PDF_OK;
}

extern "C" pdf_status pdf_iecm_cond(const pdf_particles* p, double* cond, void* stream) {
  if (!p || !cond) return fail(PDF_EINVAL, "pdf_iecm_cond: NULL argument");
  if (!p->have_cond) return fail(PDF_ESTATE, "pdf_iecm_cond: enable IECM and call pdf_estimate_stats first");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = p->n;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
  PDF_KERNEL("k_cond_to_f64", st, k_cond_to_f64<<<g, 256, 0, st>>>(p->cond, p->pid, cond, n));
  return PDF_OK;
}

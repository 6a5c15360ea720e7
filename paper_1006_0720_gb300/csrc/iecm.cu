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
// memory (or, above kIecmCap particles, into global scratch slices) and
// sorted by rank counting inside each group: O(n^2) comparisons per level,
// fine for the small groups of the second and third levels.  The first
// level (the whole element) of an element with more than kIecmRunMin
// particles in shared memory is sorted instead in runs of 32 (a bitonic
// network across each warp's lanes) whose entries find their final rank by
// binary searches in the other runs.  Both give the same order: (key, id)
// is a strict total order.
#include "common.cuh"
#include "fx.cuh"

namespace pdfgb {

constexpr int kIecmThreads = 128;
constexpr int kIecmCap = 256;
constexpr int kIecmRunMin = 64;

// One copy of the per-particle data (shared or global): the three velocity
// components and the scalar as (high, low) pairs, the particle id and the
// storage slot.  Two copies alternate: every level sorts by moving the data
// into the other copy at the sorted positions, so that the comparisons read
// consecutive entries (no indirection).
struct IecmBuf {
  float* f[8];  // uh ul vh vl wh wl sh sl
  int32_t* id;
  int32_t* slot;
};

struct IecmView {  // the two copies and the group bounds of each position
  IecmBuf a, b;
  int32_t *gs, *ge;
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

// (key_j, id_j) < (key_i, id_i) for double-float keys (normalized pairs
// order like their values); evaluated without branches
__device__ __forceinline__ int key_less(float hj, float lj, int32_t ij, float hi, float li, int32_t ii) {
  return (int)((hj < hi) | ((hj == hi) & ((lj < li) | ((lj == li) & (ij < ii)))));
}

// Ascending bitonic sort of one (h, l, id, src) entry per lane across the warp.
__device__ __forceinline__ void warp_bitonic(float& h, float& l, int32_t& id, int32_t& src) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const float ph = __shfl_xor_sync(0xffffffffu, h, j);
      const float pl = __shfl_xor_sync(0xffffffffu, l, j);
      const int32_t pid = __shfl_xor_sync(0xffffffffu, id, j);
      const int32_t ps = __shfl_xor_sync(0xffffffffu, src, j);
      const bool partner_less = key_less(ph, pl, pid, h, l, id);
      const bool up = (lane & k) == 0, lower = (lane & j) == 0;
      // the lower lane of a pair keeps the smaller entry in an ascending
      // subsequence, the larger one in a descending one
      if (lower == up ? partner_less : !partner_less) {
        h = ph;
        l = pl;
        id = pid;
        src = ps;
      }
    }
  }
}

// Entries of the sorted run [r0, r0 + len) below (h, l, id).
__device__ __forceinline__ int32_t count_below(const float* rh, const float* rl, const int32_t* rid, int32_t r0,
                                               int32_t len, float h, float l, int32_t id) {
  int32_t lo = 0, hi = len;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (key_less(rh[r0 + mid], rl[r0 + mid], rid[r0 + mid], h, l, id)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// floor(k i / n) and ceil(j n / k) for 0 <= i < n, 0 <= j <= k <= 127: 32-bit
// unsigned arithmetic while the products stay below 2^31 (n < 2^24), 64-bit
// beyond
__device__ __forceinline__ int32_t part_of(int32_t k, int32_t i, int32_t n) {
  if (n < (1 << 24)) return (int32_t)((uint32_t)(k * i) / (uint32_t)n);
  return (int32_t)(((int64_t)k * i) / n);
}
__device__ __forceinline__ int32_t part_start(int32_t j, int32_t n, int32_t k) {
  if (n < (1 << 24)) return (int32_t)(((uint32_t)(j * n) + (uint32_t)(k - 1)) / (uint32_t)k);
  return (int32_t)(((int64_t)j * n + k - 1) / k);
}

template <typename T>
__global__ void __launch_bounds__(kIecmThreads) k_iecm_cond(const int32_t* __restrict__ seg,
                                                            const int32_t* __restrict__ order, int32_t n_tri,
                                                            const T* __restrict__ u, const T* __restrict__ v,
                                                            const T* __restrict__ w, const T* __restrict__ ps,
                                                            const int32_t* __restrict__ pid, int nc0, int nc1,
                                                            int nc2, int m_min, IecmView big,
                                                            fx::df* __restrict__ cond) {
  __shared__ float s_f[2][8][kIecmCap];
  __shared__ int32_t s_i[6][kIecmCap];
  __shared__ float s_rh[kIecmCap], s_rl[kIecmCap];      // sorted runs of the first level
  __shared__ int32_t s_rid[kIecmCap], s_rsrc[kIecmCap];
  const int tid = threadIdx.x;
  for (int32_t e = blockIdx.x; e < n_tri; e += gridDim.x) {
    const int32_t beg = seg[e], N = seg[e + 1] - beg;
    if (N == 0) continue;
    IecmView V;
    if (N <= kIecmCap) {
      for (int c = 0; c < 2; ++c) {
        IecmBuf& B = c == 0 ? V.a : V.b;
        for (int q = 0; q < 8; ++q) B.f[q] = s_f[c][q];
        B.id = s_i[2 * c];
        B.slot = s_i[2 * c + 1];
      }
      V.gs = s_i[4];
      V.ge = s_i[5];
    } else {  // the element's slices of the global scratch
      V = big;
      for (int c = 0; c < 2; ++c) {
        IecmBuf& B = c == 0 ? V.a : V.b;
        for (int q = 0; q < 8; ++q) B.f[q] += beg;
        B.id += beg;
        B.slot += beg;
      }
      V.gs += beg;
      V.ge += beg;
    }
    __syncthreads();  // the previous element is done with the arrays
    {  // the next element's particles on their way to L2 (after the periodic
       // reordering they sit close to their grouped positions)
      const int32_t en = e + gridDim.x;
      if (en < n_tri) {
        const int32_t nb = seg[en], ne = seg[en + 1];
        for (int32_t i = nb + 16 * tid; i < ne; i += 16 * kIecmThreads) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(u + i));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(v + i));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(w + i));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(ps + i));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pid + i));
        }
      }
    }
    for (int i = tid; i < N; i += kIecmThreads) {
      const int64_t s = order ? (int64_t)order[beg + i] : (int64_t)(beg + i);
      V.a.slot[i] = (int32_t)s;
      V.a.id[i] = pid[s];
      load_comp(u, s, V.a.f[0][i], V.a.f[1][i]);
      load_comp(v, s, V.a.f[2][i], V.a.f[3][i]);
      load_comp(w, s, V.a.f[4][i], V.a.f[5][i]);
      load_comp(ps, s, V.a.f[6][i], V.a.f[7][i]);
      V.gs[i] = 0;
      V.ge[i] = N;
    }
    __syncthreads();
    const int ncs[3] = {nc0, nc1, nc2};
#pragma unroll  // static indices into the copies' pointer arrays
    for (int level = 0; level < 3; ++level) {
      const float* kh = V.a.f[2 * level];
      const float* kl = V.a.f[2 * level + 1];
      if (level == 0 && N > kIecmRunMin && N <= kIecmCap) {
        // runs of 32 sorted across each warp's lanes
        const int lane = tid & 31;
        const int32_t R = (N + 31) >> 5;
        for (int32_t r = tid >> 5; r < R; r += kIecmThreads / 32) {
          const int32_t pos = 32 * r + lane;
          const bool real = pos < N;
          float h = real ? kh[pos] : __int_as_float(0x7f800000);
          float l = real ? kl[pos] : 0.0f;
          int32_t id = real ? V.a.id[pos] : 0x7fffffff;
          int32_t src = pos;
          warp_bitonic(h, l, id, src);
          s_rh[pos] = h;
          s_rl[pos] = l;
          s_rid[pos] = id;
          s_rsrc[pos] = src;
        }
        __syncthreads();
        // the final rank of each entry: its place in its run plus the
        // entries below it in the other runs; the entry moves there
        for (int32_t t = tid; t < N; t += kIecmThreads) {
          const int32_t r = t >> 5;
          const float h = s_rh[t], l = s_rl[t];
          const int32_t id = s_rid[t];
          int32_t to = t - 32 * r;
          for (int32_t q = 0; q < R; ++q)
            if (q != r) to += count_below(s_rh, s_rl, s_rid, 32 * q, min(32, N - 32 * q), h, l, id);
          const int32_t pos = s_rsrc[t];
#pragma unroll
          for (int c = 0; c < 8; ++c) V.b.f[c][to] = V.a.f[c][pos];
          V.b.id[to] = id;
          V.b.slot[to] = V.a.slot[pos];
        }
        __syncthreads();
      } else {
      // sort each group [gs, ge) by rank counting; every entry moves to its
      // sorted position in the other copy
      for (int pos = tid; pos < N; pos += kIecmThreads) {
        const int32_t a = V.gs[pos], b = V.ge[pos];
        const float hi = kh[pos], li = kl[pos];
        const int32_t ii = V.a.id[pos];
        int32_t r = 0;
#pragma unroll 4
        for (int32_t q = a; q < b; ++q) r += key_less(kh[q], kl[q], V.a.id[q], hi, li, ii);
        const int32_t to = a + r;
#pragma unroll
        for (int c = 0; c < 8; ++c) V.b.f[c][to] = V.a.f[c][pos];
        V.b.id[to] = ii;
        V.b.slot[to] = V.a.slot[pos];
      }
      __syncthreads();
      }
      // divide each group into k parts of equal count
      for (int pos = tid; pos < N; pos += kIecmThreads) {
        const int32_t a = V.gs[pos], n = V.ge[pos] - a;
        int32_t k = (int32_t)((uint32_t)n / (uint32_t)m_min);
        if (k > ncs[level]) k = ncs[level];
        if (k < 1) k = 1;
        const int32_t j = part_of(k, pos - a, n);
        V.gs[pos] = a + part_start(j, n, k);
        V.ge[pos] = a + part_start(j + 1, n, k);
      }
      const IecmBuf t = V.a;
      V.a = V.b;
      V.b = t;
      __syncthreads();
    }
    // bin means: the first position of each bin adds its bin in sorted order
    // (double-float) and leaves the mean at that position of the spare copy
    for (int pos = tid; pos < N; pos += kIecmThreads) {
      const int32_t a = V.gs[pos], b = V.ge[pos];
      if (pos != a) continue;
      fx::acc s;
      s.init(fx::df{V.a.f[6][a], V.a.f[7][a]});
      for (int32_t q = a + 1; q < b; ++q) s.add(fx::df{V.a.f[6][q], V.a.f[7][q]});
      const fx::df mean = fx::df_norm(fx::mul(s.value(), fx::recip_df(b - a)));
      V.b.f[0][a] = mean.h;
      V.b.f[1][a] = mean.l;
    }
    __syncthreads();
    for (int pos = tid; pos < N; pos += kIecmThreads) {
      const int32_t a = V.gs[pos];
      reinterpret_cast<float2*>(cond)[V.a.slot[pos]] = make_float2(V.b.f[0][a], V.b.f[1][a]);
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
  for (int c = 0; c < 2; ++c) {
    IecmBuf& B = c == 0 ? big.a : big.b;
    for (int q = 0; q < 8; ++q) B.f[q] = f + (8 * c + q) * n;
    B.id = g + (2 * c) * n;
    B.slot = g + (2 * c + 1) * n;
  }
  big.gs = g + 4 * n;
  big.ge = g + 5 * n;
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
    b[pid[i]] = __longlong_as_double((long long)fx::df2d_rn(a[i]));
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
  if (nu < 1 || nv < 1 || nw < 1 || m_min < 1 || nu > 127 || nv > 127 || nw > 127)
    return fail(PDF_EINVAL, "pdf_particles_set_iecm: bins must be in [1, 127] and m_min >= 1 (or all bins 0 to disable)");
  if (!p->cond) {
    const size_t n = (size_t)p->n;
    PDF_CUDA(cudaMalloc((void**)&p->cond, sizeof(fx::df) * n));
    PDF_CUDA(cudaMalloc((void**)&p->iecm_scratch_f, sizeof(float) * 16 * n));
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

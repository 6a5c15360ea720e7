// Particle redistribution: the more efficient algorithm of App. D (its
// idea in App. C and sec. 3.6).  The elements are sorted by their particle
// count (stable radix sort, ties by element index); the k-th critical
// element (fewer than min_npel particles) takes min_npel - n_k particles
// from the k-th element from the top, which copy the critical element's
// own particles in turn (position, U, omega, psi; particle p of the donor
// copies particle p mod n_k); a particle moved into an empty element keeps
// its values and is placed uniformly in it.  "The p-th particle of an
// element" is the one with the p-th smallest particle id; counts and
// element lists are those before any move.  One warp per critical element:
// the donors and the critical elements are disjoint, so the warps write
// disjoint particles and read only unmoved ones.
//
// No grouping of all particles is needed: the counts come from a histogram
// of the element ids (warp-aggregated atomics), and only the particles of
// the critical elements and their donors are collected, unordered, into
// per-element lists (the ordering by particle id happens in the warps).
#include <algorithm>

#include "common.cuh"
#include "rng.cuh"

namespace pdfgb {

pdf_status radix_sort_index(const int32_t* keys, int64_t n, int bits, int32_t* k0, int32_t* v0, int32_t* k1,
                            int32_t* v1, int32_t* hist, int32_t* hist_part, const int32_t** keys_out,
                            const int32_t** vals_out, cudaStream_t st);
int64_t radix_tiles(int64_t n);
int32_t radix_bins();
int32_t radix_scan_blocks(int64_t hist_len);

constexpr int kMaxMin = 64;  // largest min_npel (the critical element's particles fit a warp's scratch)

// cnt[e] += the particles with element e (cnt zeroed before): lanes with
// the same element add once.
__global__ void k_rd_hist(int64_t n, const int32_t* __restrict__ elem, int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; base < n; base += nw * 32) {
    const int64_t p = base + lane;
    const int32_t e = p < n ? elem[p] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, e);
    if (e >= 0 && lane == __ffs(same) - 1) atomicAdd(cnt + e, __popc(same));
  }
}

// dev[0] = the number of critical elements (first sorted count >= min_npel),
// dev[1] = 0 (particles moved).
__global__ void k_rd_nce(int32_t n_tri, const int32_t* __restrict__ sk, int32_t min_npel, int32_t* __restrict__ dev) {
  if (threadIdx.x != 0) return;
  int32_t lo = 0, hi = n_tri;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (sk[mid] < min_npel) lo = mid + 1; else hi = mid;
  }
  dev[0] = lo;
  dev[1] = 0;
}

// role[j] = k + 1 for the k-th critical element j with a donor, role[i] =
// -(k + 1) for its donor i (role zeroed before).
__global__ void k_rd_roles(int32_t n_tri, const int32_t* __restrict__ sv, const int32_t* __restrict__ dev,
                           int32_t* __restrict__ role) {
  const int32_t nce = dev[0];
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nce; k += gridDim.x * blockDim.x) {
    if (n_tri - 1 - k <= k) continue;
    role[sv[k]] = k + 1;
    role[sv[n_tri - 1 - k]] = -(k + 1);
  }
}

// off[k] = sum over k' < k of (n_crit(k') + n_donor(k')): the start of the
// k-th pair's lists (critical first, then the donor's); one block.
__global__ void __launch_bounds__(1024) k_rd_offsets(int32_t n_tri, const int32_t* __restrict__ sk,
                                                     const int32_t* __restrict__ dev, int64_t* __restrict__ off) {
  __shared__ int64_t sh[1024];
  const int32_t nce = dev[0];
  int64_t carry = 0;
  for (int32_t b0 = 0; b0 < nce; b0 += 1024) {
    const int32_t k = b0 + threadIdx.x;
    int64_t v = 0;
    if (k < nce && n_tri - 1 - k > k) v = (int64_t)sk[k] + sk[n_tri - 1 - k];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan
      const int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (k < nce) off[k] = carry + sh[threadIdx.x] - v;
    carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[nce] = carry;
}

// The particles of the critical elements and their donors into the pairs'
// lists (unordered); cur: [n_tri] cursors of the critical lists, then
// [n_tri] of the donor lists (zeroed before).  Lanes with the same role take
// their places with one atomic (the particles are mostly grouped by element).
__global__ void k_rd_collect(int64_t n, int32_t n_tri, const int32_t* __restrict__ elem,
                             const int32_t* __restrict__ role, const int32_t* __restrict__ sk,
                             const int64_t* __restrict__ off, int32_t* __restrict__ cur, int32_t* __restrict__ list) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; base < n; base += nw * 32) {
    const int64_t s = base + lane;
    const int32_t r = s < n ? role[elem[s]] : 0;
    const unsigned same = __match_any_sync(0xffffffffu, r);
    if (r == 0) continue;
    const int leader = __ffs(same) - 1;
    const int32_t k = r > 0 ? r - 1 : -r - 1;
    int32_t* c = r > 0 ? cur + k : cur + n_tri + k;
    int32_t at = 0;
    if (lane == leader) at = atomicAdd(c, __popc(same));
    at = __shfl_sync(same, at, leader) + __popc(same & ((1u << lane) - 1u));
    const int64_t o = off[k] + (r > 0 ? 0 : sk[k]);
    list[o + at] = (int32_t)s;
  }
}

struct RdArgs {
  int32_t n_tri, min_npel;
  uint32_t step;
  uint64_t seed;
  const int32_t *sk, *sv, *list, *pid, *tri;
  const int64_t* off;
  const double* xy;
  int32_t* elem;
  int64_t *x, *y;
  long long* st8[5];  // u, v, w, omega, psi as double-float pairs (FP64 state)
  float* st4[5];      // the same in FP32 (FP32 state)
  bool fp32;
  int32_t* dev;
};

constexpr int kRdWarps = 4;      // warps per block of the move kernel
constexpr int kRdStage = 1024;   // donor particles staged in shared memory per warp

__global__ void __launch_bounds__(kRdWarps * 32) k_rd_move(RdArgs A) {
  __shared__ int32_t s_cslot[kRdWarps][kMaxMin], s_cpid[kRdWarps][kMaxMin], s_dslot[kRdWarps][kMaxMin];
  __shared__ int32_t s_dpid[kRdWarps][kRdStage], s_dsl[kRdWarps][kRdStage];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nce = A.dev[0];
  int32_t* cslot = s_cslot[wi];
  int32_t* cpid = s_cpid[wi];
  int32_t* dslot = s_dslot[wi];
  int32_t* dpid = s_dpid[wi];
  int32_t* dsl = s_dsl[wi];
  const int32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nce; k += nwarps) {
    const int32_t di = A.n_tri - 1 - k;
    if (di <= k) break;  // the donor from the top would be critical itself
    const int32_t j = A.sv[k], nj = A.sk[k];
    const int32_t ni = A.sk[di];
    const int32_t d = min(A.min_npel - nj, ni);
    // the critical element's particles ordered by particle id
    __syncwarp();
    int32_t my_slot[2], my_pid[2];
    const int32_t* clist = A.list + A.off[k];
    const int32_t* dlist = clist + nj;
    for (int r = 0; r < 2; ++r) {
      const int32_t a = lane + 32 * r;
      my_slot[r] = -1;
      my_pid[r] = 0;
      if (a < nj) {
        my_slot[r] = clist[a];
        my_pid[r] = A.pid[my_slot[r]];
        cpid[a] = my_pid[r];
      }
    }
    __syncwarp();
    for (int r = 0; r < 2; ++r) {
      if (my_slot[r] < 0) continue;
      int32_t rank = 0;
      for (int32_t b = 0; b < nj; ++b) rank += cpid[b] < my_pid[r];
      cslot[rank] = my_slot[r];
    }
    // the donor's d particles of smallest id, by repeated minimum search
    // (over a copy in shared memory when the donor's list fits)
    const bool staged = ni <= kRdStage;
    if (staged)
      for (int32_t a = lane; a < ni; a += 32) {
        const int32_t sl = dlist[a];
        dsl[a] = sl;
        dpid[a] = A.pid[sl];
      }
    __syncwarp();
    int32_t last = -1;
    for (int32_t q = 0; q < d; ++q) {
      int32_t best = 0x7fffffff, bslot = -1;
      for (int32_t a = lane; a < ni; a += 32) {
        const int32_t sl = staged ? dsl[a] : dlist[a];
        const int32_t pp = staged ? dpid[a] : A.pid[sl];
        if (pp > last && pp < best) { best = pp; bslot = sl; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const int32_t ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int32_t os = __shfl_xor_sync(0xffffffffu, bslot, o);
        if (ob < best) { best = ob; bslot = os; }
      }
      if (lane == 0) dslot[q] = bslot;
      last = best;
    }
    __syncwarp();
    // the moves
    for (int32_t q = lane; q < d; q += 32) {
      const int32_t dst = dslot[q];
      if (nj > 0) {
        const int32_t src = cslot[q % nj];
        A.x[dst] = A.x[src];
        A.y[dst] = A.y[src];
        if (A.fp32) {
          for (int f = 0; f < 5; ++f) A.st4[f][dst] = A.st4[f][src];
        } else {
          for (int f = 0; f < 5; ++f) A.st8[f][dst] = A.st8[f][src];
        }
      } else {
        uint32_t c[4] = {(uint32_t)A.pid[dst], A.step, 0u, kPurposeRedist};
        philox4x32_10(c, (uint32_t)A.seed, (uint32_t)(A.seed >> 32));
        float r1 = u01_from_word(c[0]), r2 = u01_from_word(c[1]);
        if (__fadd_rn(r1, r2) > 1.0f) {
          r1 = __fsub_rn(1.0f, r1);
          r2 = __fsub_rn(1.0f, r2);
        }
        const int32_t na = A.tri[3 * j], nb = A.tri[3 * j + 1], nc = A.tri[3 * j + 2];
        const double xa = A.xy[2 * na], ya = A.xy[2 * na + 1];
        const double xb = A.xy[2 * nb], yb = A.xy[2 * nb + 1];
        const double xc = A.xy[2 * nc], yc = A.xy[2 * nc + 1];
        const double R1 = (double)r1, R2 = (double)r2;
        const double px = __dadd_rn(__dadd_rn(xa, __dmul_rn(R1, __dsub_rn(xb, xa))), __dmul_rn(R2, __dsub_rn(xc, xa)));
        const double py = __dadd_rn(__dadd_rn(ya, __dmul_rn(R1, __dsub_rn(yb, ya))), __dmul_rn(R2, __dsub_rn(yc, ya)));
        A.x[dst] = fx::d2fix((uint64_t)__double_as_longlong(px), kPosF);
        A.y[dst] = fx::d2fix((uint64_t)__double_as_longlong(py), kPosF);
      }
      A.elem[dst] = j;
    }
    if (lane == 0) atomicAdd(A.dev + 1, d);
  }
}

void redist_free(RedistWork& W) {
  cudaFree(W.cnt); cudaFree(W.k0); cudaFree(W.v0); cudaFree(W.k1); cudaFree(W.v1);
  cudaFree(W.hist); cudaFree(W.hist_part); cudaFree(W.dev); cudaFree(W.role); cudaFree(W.cur); cudaFree(W.off);
  if (W.host) cudaFreeHost(W.host);
  W = RedistWork();
}

static pdf_status redist_alloc(pdf_particles* P) {
  RedistWork& W = P->rd;
  if (W.cnt) return PDF_OK;
  const int64_t nt = P->mesh->d.n_tri;
  const int64_t hist_len = radix_tiles(nt) * radix_bins();
  cudaError_t e = cudaSuccess;
  auto A = [&](int32_t** p, int64_t n) { if (e == cudaSuccess) e = cudaMalloc((void**)p, sizeof(int32_t) * n); };
  A(&W.cnt, nt);
  A(&W.k0, nt);
  A(&W.v0, nt);
  A(&W.k1, nt);
  A(&W.v1, nt);
  A(&W.hist, hist_len);
  A(&W.hist_part, radix_scan_blocks(hist_len) + 1);
  A(&W.dev, 4);
  A(&W.role, nt);
  A(&W.cur, 2 * nt);
  if (e == cudaSuccess) e = cudaMalloc((void**)&W.off, sizeof(int64_t) * (nt + 1));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&W.host, sizeof(int32_t) * 4);
  if (e != cudaSuccess) {
    redist_free(W);
    return cuda_fail(e, "pdf_redistribute: allocation");
  }
  return PDF_OK;
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_redistribute(pdf_particles* p, const pdf_mesh* m, int32_t min_npel, uint64_t seed,
                                       uint32_t step, int32_t* moved, void* stream) {
  if (!p || !m || p->mesh != m) return fail(PDF_EINVAL, "pdf_redistribute: NULL or mismatched handles");
  if (min_npel < 1 || min_npel > kMaxMin) return fail(PDF_EINVAL, "pdf_redistribute: min_npel must be in [1, 64]");
  cudaStream_t st = (cudaStream_t)stream;
  pdf_status s = redist_alloc(p);
  if (s != PDF_OK) return s;
  const MeshDev& M = m->d;
  RedistWork& W = p->rd;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((p->n + 255) / 256, 8192));
  PDF_CUDA(cudaMemsetAsync(W.cnt, 0, sizeof(int32_t) * M.n_tri, st));
  PDF_CUDA(cudaMemsetAsync(W.role, 0, sizeof(int32_t) * M.n_tri, st));
  PDF_CUDA(cudaMemsetAsync(W.cur, 0, sizeof(int32_t) * 2 * M.n_tri, st));
  PDF_KERNEL("k_rd_hist", st, k_rd_hist<<<nb, 256, 0, st>>>(p->n, p->elem, W.cnt));
  int bits = 1;
  while ((1LL << bits) <= p->n) ++bits;
  const int32_t *sk = nullptr, *sv = nullptr;
  s = radix_sort_index(W.cnt, M.n_tri, bits, W.k0, W.v0, W.k1, W.v1, W.hist, W.hist_part, &sk, &sv, st);
  if (s != PDF_OK) return s;
  PDF_KERNEL("k_rd_nce", st, k_rd_nce<<<1, 32, 0, st>>>(M.n_tri, sk, min_npel, W.dev));
  const int eb = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)M.n_tri + 255) / 256, 4096));
  PDF_KERNEL("k_rd_roles", st, k_rd_roles<<<eb, 256, 0, st>>>(M.n_tri, sv, W.dev, W.role));
  PDF_KERNEL("k_rd_offsets", st, k_rd_offsets<<<1, 1024, 0, st>>>(M.n_tri, sk, W.dev, W.off));
  // the lists go to a grouping buffer, free between a step and the statistics
  int32_t* list = p->vals[0];
  PDF_KERNEL("k_rd_collect", st, k_rd_collect<<<nb, 256, 0, st>>>(p->n, M.n_tri, p->elem, W.role, sk, W.off, W.cur,
                                                                   list));
  RdArgs A;
  A.n_tri = M.n_tri;
  A.min_npel = min_npel;
  A.step = step;
  A.seed = seed;
  A.sk = sk;
  A.sv = sv;
  A.list = list;
  A.off = W.off;
  A.pid = p->pid;
  A.tri = M.tri;
  A.xy = M.xy;
  A.elem = p->elem;
  A.x = p->x;
  A.y = p->y;
  A.fp32 = p->precision != PDF_FP64;
  long long* s8[5] = {(long long*)p->u, (long long*)p->v, (long long*)p->w, (long long*)p->om, (long long*)p->ps};
  float* s4[5] = {p->uf, p->vf, p->wf, p->omf, p->psf};
  for (int f = 0; f < 5; ++f) {
    A.st8[f] = s8[f];
    A.st4[f] = s4[f];
  }
  A.dev = W.dev;
  const int mb = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)M.n_tri / 2 + kRdWarps - 1) / kRdWarps, 8192));
  PDF_KERNEL("k_rd_move", st, k_rd_move<<<mb, kRdWarps * 32, 0, st>>>(A));
  PDF_CUDA(cudaMemcpyAsync(W.host, W.dev, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaStreamSynchronize(st));
  if (moved) *moved = W.host[1];
  // the grouping and the statistics no longer describe the particles
  p->have_stats = false;
  return PDF_OK;
}

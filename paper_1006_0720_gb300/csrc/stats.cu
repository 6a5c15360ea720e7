// Particle-in-cell statistics (sec. 3.3) and derivatives (sec. 3.4).
//
// Grouping: a stable least-significant-digit radix sort of (element id,
// particle id) pairs, 9-bit digits, in place of the paper's per-element
// linked lists.  Stability makes the particle order inside every element
// ascending in particle id, so the segmented reductions below always add
// the same numbers in the same order: the statistics are deterministic
// without floating-point atomics.
#include <algorithm>

#include "common.cuh"
#include "fx.cuh"

namespace pdfgb {

constexpr int kRadixBits = 9;
constexpr int kBins = 1 << kRadixBits;      // 512
constexpr int kSortThreads = 256;
constexpr int kItemsPerThread = 16;
constexpr int kTile = kSortThreads * kItemsPerThread;  // 4096 keys per tile
constexpr int kScanChunk = 4096;                       // hist entries per scan block

int64_t radix_tiles(int64_t n) { return (n + kTile - 1) / kTile; }
int32_t radix_bins() { return kBins; }
int32_t radix_scan_blocks(int64_t hist_len) { return (int32_t)((hist_len + kScanChunk - 1) / kScanChunk); }

// Per-tile digit histogram, stored bin-major: hist[bin * n_tiles + tile].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const int32_t* __restrict__ keys, int64_t n,
                                                             int shift, int64_t n_tiles,
                                                             int32_t* __restrict__ hist) {
  __shared__ int32_t h[kBins];
  for (int b = threadIdx.x; b < kBins; b += kSortThreads) h[b] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int r = 0; r < kItemsPerThread; ++r) {
    const int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kBins - 1)], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += kSortThreads) hist[(int64_t)b * n_tiles + blockIdx.x] = h[b];
}

// Exclusive scan of hist in three launches: chunk sums, scan of the sums,
// then each chunk scanned with its base.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* total) {
  __shared__ int32_t warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int32_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  const int32_t warp_base = wid > 0 ? warp_sums[wid - 1] : 0;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  const int32_t r = warp_base + inc - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_scan_reduce(const int32_t* __restrict__ a, int64_t len,
                                                      int32_t* __restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  int32_t s = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x)
    if (base + i < len) s += a[base + i];
  int32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(int32_t* __restrict__ part, int32_t nparts) {
  int32_t carry = 0;
  for (int32_t start = 0; start < nparts; start += blockDim.x) {
    const int32_t i = start + threadIdx.x;
    const int32_t v = i < nparts ? part[i] : 0;
    int32_t total;
    const int32_t ex = block_exclusive_scan(v, &total);
    if (i < nparts) part[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(1024) k_scan_apply(int32_t* __restrict__ a, int64_t len,
                                                     const int32_t* __restrict__ part) {
  // each thread owns 4 consecutive entries of the chunk
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + 4 * threadIdx.x;
  int32_t v[4];
  int32_t s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = (base + j < len) ? a[base + j] : 0;
    s += v[j];
  }
  int32_t ex = block_exclusive_scan(s, nullptr) + part[blockIdx.x];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < len) a[base + j] = ex;
    ex += v[j];
  }
}

// Stable scatter of one tile.  Warp w owns the tile's items
// [512 w, 512 (w + 1)) and ranks them in 16 rounds of 32 in index order,
// counting digits in its own row of shared counters (no block barrier
// between rounds); one block-wide prefix over the warps then gives every
// (warp, digit) its output offset, so items with equal digits keep their
// index order.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, int64_t n, int shift,
    int64_t n_tiles, const int32_t* __restrict__ hist, int32_t* __restrict__ keys_out,
    int32_t* __restrict__ vals_out) {
  constexpr int kWarps = kSortThreads / 32;
  constexpr int kPerWarp = kTile / kWarps;  // 512 items, 16 rounds
  __shared__ int32_t wcnt[kWarps][kBins + 1];  // the extra bin takes the tile's padding
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * (kBins + 1); i += kSortThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t w0 = (int64_t)blockIdx.x * kTile + (int64_t)wid * kPerWarp;
  int32_t key[kItemsPerThread], val[kItemsPerThread], off[kItemsPerThread];
#pragma unroll
  for (int r = 0; r < kItemsPerThread; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    const bool valid = i < n;
    key[r] = valid ? keys_in[i] : 0;
    val[r] = valid ? (vals_in ? vals_in[i] : (int32_t)i) : 0;
  }
#pragma unroll
  for (int r = 0; r < kItemsPerThread; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    const int d = (i < n) ? ((key[r] >> shift) & (kBins - 1)) : kBins;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt_mask);
    const int32_t before = wcnt[wid][d];
    __syncwarp();
    if (rank == 0) wcnt[wid][d] = before + __popc(peers);
    __syncwarp();
    off[r] = before + rank;
  }
  __syncthreads();
  // (warp, digit) offsets: the tile's base of the digit plus the earlier warps' counts
  for (int b = threadIdx.x; b < kBins; b += kSortThreads) {
    int32_t acc = hist[(int64_t)b * n_tiles + blockIdx.x];
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      const int32_t c = wcnt[k][b];
      wcnt[k][b] = acc;
      acc += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItemsPerThread; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    if (i < n) {
      const int d = (key[r] >> shift) & (kBins - 1);
      const int32_t pos = wcnt[wid][d] + off[r];
      keys_out[pos] = key[r];
      vals_out[pos] = val[r];
    }
  }
}

// seg[e] = first sorted position whose key >= e; seg[n_tri] = n.
__global__ void k_seg_offsets(const int32_t* __restrict__ keys, int64_t n, int32_t n_tri,
                              int32_t* __restrict__ seg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t prev = (i == 0) ? -1 : keys[i - 1];
    const int32_t cur = (i == n) ? n_tri : keys[i];
    for (int32_t e = prev + 1; e <= cur; ++e) seg[e] = (int32_t)i;
  }
}

// A state value as FP64, whatever its stored representation.
__device__ __forceinline__ double ld64(const double* a, int64_t i) { return __ldg(a + i); }
__device__ __forceinline__ double ld64(const float* a, int64_t i) { return (double)__ldg(a + i); }
__device__ __forceinline__ double ld64(const fx::df* a, int64_t i) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(a) + i);
  return fx::to_double(fx::df{v.x, v.y});
}

// One warp per element: first pass means, second pass central moments
// (sec. 3.3, 1/N).  Lane j adds sorted positions j, j+32, ...; the lane
// partials are combined by a fixed butterfly and lane 0's result is used.
template <typename T>
__device__ void elem_stats_fp64(int32_t beg, int32_t end, int lane, const int32_t* __restrict__ pid,
                                const T* __restrict__ u, const T* __restrict__ v,
                                const T* __restrict__ w, const T* __restrict__ om,
                                const T* __restrict__ ps, double* __restrict__ out) {
  const int32_t N = end - beg;
  double s[5] = {0, 0, 0, 0, 0};
  for (int32_t i = beg + lane; i < end; i += 32) {
    const int32_t p = pid ? pid[i] : i;
    s[0] += ld64(u, p); s[1] += ld64(v, p); s[2] += ld64(w, p); s[3] += ld64(om, p); s[4] += ld64(ps, p);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    s[q] = __shfl_sync(0xffffffffu, s[q], 0) / (double)N;
  }
  double c[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int32_t i = beg + lane; i < end; i += 32) {
    const int32_t p = pid ? pid[i] : i;
    const double du = ld64(u, p) - s[0], dv = ld64(v, p) - s[1], dw = ld64(w, p) - s[2],
                 dp = ld64(ps, p) - s[4];
    c[0] += du * du; c[1] += dv * dv; c[2] += dw * dw;
    c[3] += du * dv; c[4] += du * dw; c[5] += dv * dw; c[6] += dp * dp;
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c[q] += __shfl_xor_sync(0xffffffffu, c[q], o);
    c[q] = __shfl_sync(0xffffffffu, c[q], 0) / (double)N;
  }
  if (lane == 0) {
    out[0] = (double)N;
    for (int q = 0; q < 5; ++q) out[1 + q] = s[q];
    for (int q = 0; q < 7; ++q) out[6 + q] = c[q];
  }
}

// Element statistics without FP64 arithmetic per particle (the default):
// the same two passes as above, but every particle value is decoded into
// fixed point with 48 fraction bits and the sums are 128-bit integers, so
// they are exact and independent of the order of the particles.
//   pass 1: S_i = sum q_i (q = value 2^48)          -> means S_i / N
//   pass 2: D_i = q_i - M_i with M_i ~ the mean,   -> central moments
//           (sum D_i D_j - sum D_i sum D_j / N) / N
// Only the per-element finishing (a few divisions) runs in FP64.  An element
// with |value| >= 128 (omega >= 2^14) or more than 2^17 particles falls back
// to the FP64 kernel's arithmetic (exact sums need those bounds).
constexpr int kFQ = 48;

// Signed 64 x 64 -> 128-bit product from 32 x 32 -> 64-bit pieces (the
// native 64-bit multiply-high runs on GB300's slow FP64 unit).
__device__ __forceinline__ void mul_s64(long long a, long long b, unsigned long long& lo, long long& hi) {
  const bool neg = (a < 0) != (b < 0);
  const unsigned long long ua = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const unsigned long long ub = b < 0 ? 0ull - (unsigned long long)b : (unsigned long long)b;
  const unsigned int a0 = (unsigned int)ua, a1 = (unsigned int)(ua >> 32);
  const unsigned int b0 = (unsigned int)ub, b1 = (unsigned int)(ub >> 32);
  const unsigned long long p00 = (unsigned long long)a0 * b0;
  const unsigned long long p01 = (unsigned long long)a0 * b1;
  const unsigned long long p10 = (unsigned long long)a1 * b0;
  const unsigned long long p11 = (unsigned long long)a1 * b1;
  const unsigned long long mid = (p00 >> 32) + (unsigned int)p01 + (unsigned int)p10;
  unsigned long long l = (mid << 32) | (unsigned int)p00;
  unsigned long long h = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
  if (neg) {  // two's complement of the 128-bit magnitude
    l = ~l + 1ull;
    h = ~h + (l == 0ull ? 1ull : 0ull);
  }
  lo = l;
  hi = (long long)h;
}

__device__ __forceinline__ void mac128(unsigned long long& lo, long long& hi, long long a, long long b) {
  unsigned long long pl;
  long long ph;
  mul_s64(a, b, pl, ph);
  const unsigned long long nl = lo + pl;
  hi = hi + ph + (nl < lo ? 1 : 0);
  lo = nl;
}

__device__ __forceinline__ void add64(unsigned long long& lo, long long& hi, long long v) {
  const unsigned long long nl = lo + (unsigned long long)v;
  hi = hi + (v < 0 ? -1 : 0) + (nl < lo ? 1 : 0);
  lo = nl;
}

__device__ __forceinline__ void warp_sum128(unsigned long long& lo, long long& hi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ol = __shfl_xor_sync(0xffffffffu, lo, o);
    const long long oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const unsigned long long nl = lo + ol;
    hi = hi + oh + (nl < lo ? 1 : 0);
    lo = nl;
  }
}


// Value -> fixed point with kFQ fraction bits; `ok` cleared outside |v| < 2^lim.
__device__ __forceinline__ long long to_fix(const double* a, int64_t i, int lim, bool& ok) {
  const uint64_t b = (uint64_t)__ldg(reinterpret_cast<const long long*>(a) + i);
  ok = ok && fx::d_exp(b) <= 1023 + lim;
  return fx::d2fix(b, kFQ);
}
__device__ __forceinline__ long long to_fix(const fx::df* a, int64_t i, int lim, bool& ok) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(a) + i);
  ok = ok && (int)((fx::f_bits(v.x) >> 23) & 0xFF) <= 127 + lim;
  return fx::f2fix(v.x, kFQ) + fx::f2fix(v.y, kFQ);
}
__device__ __forceinline__ long long to_fix(const float* a, int64_t i, int lim, bool& ok) {
  const float f = __ldg(a + i);
  ok = ok && (int)((fx::f_bits(f) >> 23) & 0xFF) <= 127 + lim;
  return fx::f2fix(f, kFQ);
}

// Per-warp shared scratch of the statistics kernel.  Lane partials are
// stored column-wise so that one lane can add up one quantity over the 32
// lanes; rows are padded to 33 entries so that the lanes reading different
// quantities at the same column hit different banks.  Pass 1 also keeps the
// fixed-point u, v, w, psi of the element's first kStatCache particles for
// pass 2 (which re-reads only the rest); the double-float partials of pass
// 2 reuse that storage once it has been read.
constexpr int kStatCache = 128;
struct StatScratch {
  unsigned long long lo[5][33];
  long long hi[5][33];
  unsigned long long lo2[5][6];  // second level of the pass-1 sums
  long long hi2[5][6];
  union {
    long long q[4][kStatCache];
    struct {
      float h[11][33], l[11][33];
    } f;
  };
};
constexpr int kStatWarps = 4;  // warps per block (27 KB of shared memory)

__device__ __forceinline__ void prefetch_l2(const void* a) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

template <typename T>
__global__ void __launch_bounds__(kStatWarps * 32, 8) k_elem_stats_fx(const int32_t* __restrict__ seg,
                                                       const int32_t* __restrict__ pid, int32_t n_tri,
                                                       const T* __restrict__ u, const T* __restrict__ v,
                                                       const T* __restrict__ w, const T* __restrict__ om,
                                                       const T* __restrict__ ps, double* __restrict__ es) {
  __shared__ StatScratch scratch[kStatWarps];
  StatScratch& SS = scratch[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < n_tri; e += nwarps) {
    const int32_t beg = seg[e], end = seg[e + 1];
    const int32_t N = end - beg;
    double* out = es + e * PDF_NES;
    if (N == 0) {
      if (lane < PDF_NES) out[lane] = 0.0;
      continue;
    }
    __syncwarp();  // the previous element's readers of the scratch are done
    {  // the next element's state on its way to L2: after the periodic
       // reordering its particles sit close to their grouped positions
      const int64_t en = e + nwarps;
      if (en < n_tri) {
        const int32_t nb = seg[en], ne = seg[en + 1];
        for (int32_t i = nb + 16 * lane; i < ne; i += 16 * 32) {
          prefetch_l2(u + i);
          prefetch_l2(v + i);
          prefetch_l2(w + i);
          prefetch_l2(om + i);
          prefetch_l2(ps + i);
          if (pid) prefetch_l2(pid + i);
        }
      }
    }
    // pass 1: exact sums of the fixed-point values
    unsigned long long lo[5] = {0, 0, 0, 0, 0};
    long long hi[5] = {0, 0, 0, 0, 0};
    bool ok = N <= (1 << 17);
    for (int32_t i = beg + lane; i < end; i += 32) {
      const int32_t p = pid ? pid[i] : i;
      const long long qu = to_fix(u, p, 6, ok), qv = to_fix(v, p, 6, ok), qw = to_fix(w, p, 6, ok);
      const long long qs = to_fix(ps, p, 6, ok);
      add64(lo[0], hi[0], qu);
      add64(lo[1], hi[1], qv);
      add64(lo[2], hi[2], qw);
      add64(lo[3], hi[3], to_fix(om, p, 13, ok));
      add64(lo[4], hi[4], qs);
      const int32_t slot = i - beg;
      if (slot < kStatCache) {
        SS.q[0][slot] = qu;
        SS.q[1][slot] = qv;
        SS.q[2][slot] = qw;
        SS.q[3][slot] = qs;
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
      elem_stats_fp64(beg, end, lane, pid, u, v, w, om, ps, out);
      continue;
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      SS.lo[q][lane] = lo[q];
      SS.hi[q][lane] = hi[q];
    }
    __syncwarp();
    // exact sums over the lanes in two levels: lane 6q + r (r < 6) adds
    // columns r, r + 6, ... of quantity q, then lane q adds its six results
    const fx::df invN = fx::recip_df(N);
    fx::df mean = fx::df{0.f, 0.f};
    if (lane < 30) {
      const int q = lane / 6, r = lane - 6 * (lane / 6);
      unsigned long long sl = 0;
      long long sh = 0;
      for (int j = r; j < 32; j += 6) {
        const unsigned long long nl = sl + SS.lo[q][j];
        sh = sh + SS.hi[q][j] + (nl < sl ? 1 : 0);
        sl = nl;
      }
      SS.lo2[q][r] = sl;
      SS.hi2[q][r] = sh;
    }
    __syncwarp();
    if (lane < 5) {
      unsigned long long sl = 0;
      long long sh = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        const unsigned long long nl = sl + SS.lo2[lane][r];
        sh = sh + SS.hi2[lane][r] + (nl < sl ? 1 : 0);
        sl = nl;
      }
      mean = fx::df_norm(fx::mul(fx::i128_to_df(sl, sh, -kFQ), invN));
    }
    long long M[4];
    const int idx[4] = {0, 1, 2, 4};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float mh = __shfl_sync(0xffffffffu, mean.h, idx[k]);
      const float ml = __shfl_sync(0xffffffffu, mean.l, idx[k]);
      M[k] = fx::f2fix(mh, kFQ) + fx::f2fix(ml, kFQ);
    }
    // pass 2: deviations from M (exact), their products and sums in
    // double-float, each lane's particles in order
    fx::acc c[7], d[4];
#pragma unroll
    for (int q = 0; q < 7; ++q) c[q].init(fx::df{0.f, 0.f});
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k].init(fx::df{0.f, 0.f});
    for (int32_t i = beg + lane; i < end; i += 32) {
      const int32_t slot = i - beg;
      long long qu, qv, qw, qs;
      if (slot < kStatCache) {
        qu = SS.q[0][slot];
        qv = SS.q[1][slot];
        qw = SS.q[2][slot];
        qs = SS.q[3][slot];
      } else {
        const int32_t p = pid ? pid[i] : i;
        bool dummy = true;
        qu = to_fix(u, p, 6, dummy);
        qv = to_fix(v, p, 6, dummy);
        qw = to_fix(w, p, 6, dummy);
        qs = to_fix(ps, p, 6, dummy);
      }
      const fx::df D0 = fx::fix2df(qu - M[0], kFQ);
      const fx::df D1 = fx::fix2df(qv - M[1], kFQ);
      const fx::df D2 = fx::fix2df(qw - M[2], kFQ);
      const fx::df D3 = fx::fix2df(qs - M[3], kFQ);
      d[0].add(D0); d[1].add(D1); d[2].add(D2); d[3].add(D3);
      c[0].add(fx::mul(D0, D0));
      c[1].add(fx::mul(D1, D1));
      c[2].add(fx::mul(D2, D2));
      c[3].add(fx::mul(D0, D1));
      c[4].add(fx::mul(D0, D2));
      c[5].add(fx::mul(D1, D2));
      c[6].add(fx::mul(D3, D3));
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      SS.f.h[q][lane] = c[q].h;
      SS.f.l[q][lane] = c[q].l;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      SS.f.h[7 + k][lane] = d[k].h;
      SS.f.l[7 + k][lane] = d[k].l;
    }
    __syncwarp();
    // lanes 2q and 2q + 1 add the first and second 16 lanes' partials of
    // quantity q in lane order; lane 2q adds the two halves; lane q gets it
    fx::df half = fx::df{0.f, 0.f};
    if (lane < 22) {
      const int q = lane >> 1, j0 = (lane & 1) * 16;
      fx::acc a;
      a.init(fx::df{SS.f.h[q][j0], SS.f.l[q][j0]});
#pragma unroll 5
      for (int j = j0 + 1; j < j0 + 16; ++j) a.add(fx::df{SS.f.h[q][j], SS.f.l[q][j]});
      half = fx::df{a.h, a.l};
    }
    const float oh = __shfl_down_sync(0xffffffffu, half.h, 1), ol = __shfl_down_sync(0xffffffffu, half.l, 1);
    fx::acc a2;
    a2.init(half);
    a2.add(fx::df{oh, ol});
    const fx::df pair = a2.value();
    const float th = __shfl_sync(0xffffffffu, pair.h, (2 * lane) & 31);
    const float tl = __shfl_sync(0xffffffffu, pair.l, (2 * lane) & 31);
    const fx::df tot = lane < 11 ? fx::df{th, tl} : fx::df{0.f, 0.f};
    // output lane: 0 -> N, 1..5 -> means, 6..12 -> central moments
    // (sum D_a D_b - sum D_a sum D_b / N) / N
    const int q = lane - 6;
    const int pa = q == 1 ? 1 : (q == 2 ? 2 : (q == 5 ? 1 : (q == 6 ? 3 : 0)));
    const int pb = q == 0 ? 0 : (q == 1 ? 1 : (q == 2 ? 2 : (q == 3 ? 1 : (q == 6 ? 3 : 2))));
    const float s2h = __shfl_sync(0xffffffffu, tot.h, q < 0 ? 0 : q);
    const float s2l = __shfl_sync(0xffffffffu, tot.l, q < 0 ? 0 : q);
    const float dah = __shfl_sync(0xffffffffu, tot.h, 7 + pa), dal = __shfl_sync(0xffffffffu, tot.l, 7 + pa);
    const float dbh = __shfl_sync(0xffffffffu, tot.h, 7 + pb), dbl = __shfl_sync(0xffffffffu, tot.l, 7 + pb);
    const float mh = __shfl_sync(0xffffffffu, mean.h, (lane + 31) & 31);
    const float ml = __shfl_sync(0xffffffffu, mean.l, (lane + 31) & 31);
    fx::df val = fx::df{mh, ml};
    if (lane >= 6) {
      const fx::df corr = fx::df_norm(fx::mul(fx::df_norm(fx::mul(fx::df{dah, dal}, fx::df{dbh, dbl})), invN));
      val = fx::df_norm(fx::mul(fx::sub(fx::df{s2h, s2l}, corr), invN));
    }
    if (lane == 0) out[0] = (double)N;
    else if (lane < PDF_NES) out[lane] = __longlong_as_double((long long)fx::df2d(val));
  }
}

// Node pass: mean over the non-empty surrounding elements (twins merged);
// a node with none keeps its previous value.
__global__ void k_node_stats(const int32_t* __restrict__ nse_off, const int32_t* __restrict__ nse,
                             int32_t n_nodes, const double* __restrict__ es, double* __restrict__ ns,
                             long long* __restrict__ kept) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    double acc[PDF_NNS];
#pragma unroll
    for (int q = 0; q < PDF_NNS; ++q) acc[q] = 0.0;
    int c = 0;
    for (int32_t i = nse_off[n]; i < nse_off[n + 1]; ++i) {
      const double* s = es + (int64_t)nse[i] * PDF_NES;
      if (s[0] <= 0.0) continue;
#pragma unroll
      for (int q = 0; q < PDF_NNS; ++q) acc[q] += s[1 + q];
      ++c;
    }
    if (c == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(kept), 1ULL);
      continue;
    }
    const double inv = 1.0 / (double)c;
#pragma unroll
    for (int q = 0; q < PDF_NNS; ++q) ns[(int64_t)n * PDF_NNS + q] = acc[q] * inv;
  }
}

// Element gradients of nodal <U>, <V>, <W>, <vv> (eq. gradient with the
// analytic shape-function derivatives): eg[e] = Ux Uy Vx Vy Wx Wy vvx vvy.
__global__ void k_elem_grad1(const int32_t* __restrict__ tri, const double* __restrict__ dN,
                             int32_t n_tri, const double* __restrict__ ns, double* __restrict__ eg) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    const double* d = dN + (int64_t)e * 6;
    double g[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int fld[4] = {0, 1, 2, 6};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double* S = ns + (int64_t)tri[3 * e + j] * PDF_NNS;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        g[2 * f] += d[j] * S[fld[f]];
        g[2 * f + 1] += d[3 + j] * S[fld[f]];
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) eg[(int64_t)e * 8 + q] = g[q];
  }
}

__global__ void k_node_grad1(const int32_t* __restrict__ nse_off, const int32_t* __restrict__ nse,
                             int32_t n_nodes, const double* __restrict__ eg, double* __restrict__ nd) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const int32_t b = nse_off[n], c = nse_off[n + 1] - b;
    for (int32_t i = b; i < b + c; ++i) {
      const double* g = eg + (int64_t)nse[i] * 8;
#pragma unroll
      for (int q = 0; q < 6; ++q) acc[q] += g[q];
      acc[6] += g[7];
    }
    double* D = nd + (int64_t)n * PDF_NND;
    const double inv = 1.0 / (c > 0 ? (double)c : 1.0);
#pragma unroll
    for (int q = 0; q < 6; ++q) D[q] = acc[q] * inv;
    D[9] = acc[6] * inv;
  }
}

// Second pass: d/dx of the node dU_i/dx plus d/dy of the node dU_i/dy.
__global__ void k_elem_grad2(const int32_t* __restrict__ tri, const double* __restrict__ dN,
                             int32_t n_tri, const double* __restrict__ nd, double* __restrict__ eg) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_tri; e += gridDim.x * blockDim.x) {
    const double* d = dN + (int64_t)e * 6;
    double l[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double* D = nd + (int64_t)tri[3 * e + j] * PDF_NND;
#pragma unroll
      for (int i = 0; i < 3; ++i) l[i] += d[j] * D[2 * i] + d[3 + j] * D[2 * i + 1];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) eg[(int64_t)e * 8 + i] = l[i];
  }
}

__global__ void k_node_grad2(const int32_t* __restrict__ nse_off, const int32_t* __restrict__ nse,
                             int32_t n_nodes, const double* __restrict__ eg, double* __restrict__ nd) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    double acc[3] = {0, 0, 0};
    const int32_t b = nse_off[n], c = nse_off[n + 1] - b;
    for (int32_t i = b; i < b + c; ++i) {
      const double* g = eg + (int64_t)nse[i] * 8;
      acc[0] += g[0]; acc[1] += g[1]; acc[2] += g[2];
    }
    const double inv = 1.0 / (c > 0 ? (double)c : 1.0);
    double* D = nd + (int64_t)n * PDF_NND;
    D[6] = acc[0] * inv; D[7] = acc[1] * inv; D[8] = acc[2] * inv;
  }
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

static int blocks_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 32));
}

// Stable grouping of particles by element.  Leaves sorted element ids in
// keys[out], particle ids in vals[out] and segment offsets in seg.
pdf_status group_by_element(pdf_particles* P, cudaStream_t st) {
  const int32_t n_tri = P->mesh->d.n_tri;
  const int64_t n = P->n;
  int bits = 1;
  while ((1LL << bits) < (int64_t)n_tri) ++bits;
  const int passes = (bits + kRadixBits - 1) / kRadixBits;
  const int32_t* kin = P->elem;
  const int32_t* vin = nullptr;  // first pass: particle ids are the indices
  int cur = 0;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kRadixBits;
    PDF_KERNEL("k_radix_hist", st, k_radix_hist<<<(unsigned)P->n_tiles, kSortThreads, 0, st>>>(kin, n, shift, P->n_tiles, P->hist););
    PDF_KERNEL("k_scan_reduce", st, k_scan_reduce<<<P->n_scan_blocks, 1024, 0, st>>>(P->hist, P->hist_len, P->hist_part););
    PDF_KERNEL("k_scan_top", st, k_scan_top<<<1, 1024, 0, st>>>(P->hist_part, P->n_scan_blocks););
    PDF_KERNEL("k_scan_apply", st, k_scan_apply<<<P->n_scan_blocks, 1024, 0, st>>>(P->hist, P->hist_len, P->hist_part););
    PDF_KERNEL("k_radix_scatter", st, k_radix_scatter<<<(unsigned)P->n_tiles, kSortThreads, 0, st>>>(kin, vin, n, shift, P->n_tiles, P->hist,
                                                                   P->keys[cur], P->vals[cur]););
    kin = P->keys[cur];
    vin = P->vals[cur];
    cur ^= 1;
  }
  PDF_KERNEL("k_seg_offsets", st, k_seg_offsets<<<blocks_for(n + 1, 256), 256, 0, st>>>(kin, n, n_tri, P->seg););
  P->sorted_pid = vin;
  P->sorted_key_slot = cur ^ 1;
  return PDF_OK;
}

// Copy of every state array into the grouping's order (slot i <- slot idx[i]).
struct ReorderArgs {
  const int32_t* idx;
  int64_t n;
  const long long* src8[7];
  long long* dst8[7];
  const int32_t* src4[6];
  int32_t* dst4[6];
  int n8, n4;
};

__global__ void k_reorder(ReorderArgs R) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < R.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = R.idx[i];
#pragma unroll
    for (int k = 0; k < 7; ++k)
      if (k < R.n8) R.dst8[k][i] = __ldg(R.src8[k] + j);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < R.n4) R.dst4[k][i] = __ldg(R.src4[k] + j);
  }
}

// Permutes the state into element order after a grouping: afterwards the
// sorted order is the storage order (sorted_pid = NULL) and the element ids
// are the sorted keys.
static pdf_status reorder_state(pdf_particles* P, cudaStream_t st) {
  ReorderArgs R;
  R.idx = P->sorted_pid;
  R.n = P->n;
  R.n8 = R.n4 = 0;
  auto add8 = [&](void* src, void* dst) {
    R.src8[R.n8] = static_cast<const long long*>(src);
    R.dst8[R.n8++] = static_cast<long long*>(dst);
  };
  auto add4 = [&](void* src, void* dst) {
    R.src4[R.n4] = static_cast<const int32_t*>(src);
    R.dst4[R.n4++] = static_cast<int32_t*>(dst);
  };
  add8(P->x, P->x2);
  add8(P->y, P->y2);
  if (P->precision == PDF_FP64) {
    add8(P->u, P->u2); add8(P->v, P->v2); add8(P->w, P->w2); add8(P->om, P->om2); add8(P->ps, P->ps2);
  } else {
    add4(P->uf, P->uf2); add4(P->vf, P->vf2); add4(P->wf, P->wf2); add4(P->omf, P->omf2); add4(P->psf, P->psf2);
  }
  add4(P->pid, P->pid2);
  PDF_KERNEL("k_reorder", st, k_reorder<<<blocks_for(P->n, 256), 256, 0, st>>>(R););
  std::swap(P->x, P->x2);
  std::swap(P->y, P->y2);
  std::swap(P->u, P->u2); std::swap(P->v, P->v2); std::swap(P->w, P->w2);
  std::swap(P->om, P->om2); std::swap(P->ps, P->ps2);
  std::swap(P->uf, P->uf2); std::swap(P->vf, P->vf2); std::swap(P->wf, P->wf2);
  std::swap(P->omf, P->omf2); std::swap(P->psf, P->psf2);
  std::swap(P->pid, P->pid2);
  std::swap(P->elem, P->keys[P->sorted_key_slot]);
  P->sorted_pid = nullptr;
  return PDF_OK;
}

pdf_status iecm_cond(pdf_particles* P, const int32_t* seg, const int32_t* order, cudaStream_t st);

// Node statistics and node derivatives from the element statistics P->es
// (sec. 3.3 second pass, sec. 3.4).
pdf_status node_stats_from_elements(pdf_particles* P, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  PDF_KERNEL("k_node_stats", st, k_node_stats<<<blocks_for(M.n_nodes, 128), 128, 0, st>>>(M.nse_off, M.nse, M.n_nodes, P->es, P->ns,
                                                          P->counters + 8););
  PDF_KERNEL("k_elem_grad1", st, k_elem_grad1<<<blocks_for(M.n_tri, 128), 128, 0, st>>>(M.tri, M.dN, M.n_tri, P->ns, P->eg););
  PDF_KERNEL("k_node_grad1", st, k_node_grad1<<<blocks_for(M.n_nodes, 128), 128, 0, st>>>(M.nse_off, M.nse, M.n_nodes, P->eg, P->nd););
  PDF_KERNEL("k_elem_grad2", st, k_elem_grad2<<<blocks_for(M.n_tri, 128), 128, 0, st>>>(M.tri, M.dN, M.n_tri, P->nd, P->eg););
  PDF_KERNEL("k_node_grad2", st, k_node_grad2<<<blocks_for(M.n_nodes, 128), 128, 0, st>>>(M.nse_off, M.nse, M.n_nodes, P->eg, P->nd););
  return PDF_OK;
}

pdf_status estimate_stats(pdf_particles* P, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  pdf_status s = group_by_element(P, st);
  if (s != PDF_OK) return s;
  if (P->reorder_every > 0 && ++P->since_reorder >= P->reorder_every) {
    s = reorder_state(P, st);
    if (s != PDF_OK) return s;
    P->since_reorder = 0;
  }
  if (P->precision == PDF_FP64)
    PDF_KERNEL("k_elem_stats", st, k_elem_stats_fx<fx::df><<<blocks_for((int64_t)M.n_tri * 32, kStatWarps * 32), kStatWarps * 32, 0, st>>>(
        P->seg, P->sorted_pid, M.n_tri, P->u, P->v, P->w, P->om, P->ps, P->es));
  else
    PDF_KERNEL("k_elem_stats", st, k_elem_stats_fx<float><<<blocks_for((int64_t)M.n_tri * 32, kStatWarps * 32), kStatWarps * 32, 0, st>>>(
        P->seg, P->sorted_pid, M.n_tri, P->uf, P->vf, P->wf, P->omf, P->psf, P->es));
  s = node_stats_from_elements(P, st);
  if (s != PDF_OK) return s;
  P->have_stats = true;
  return iecm_cond(P, P->seg, P->sorted_pid, st);
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_estimate_stats(pdf_particles* p, const pdf_mesh* m, double* elem_stats,
                                         double* node_stats, double* node_derivs, void* stream) {
  if (!p || !m || p->mesh != m) return fail(PDF_EINVAL, "pdf_estimate_stats: NULL or mismatched handles");
  cudaStream_t st = (cudaStream_t)stream;
  pdf_status s = estimate_stats(p, st);
  if (s != PDF_OK) return s;
  const MeshDev& M = m->d;
  if (elem_stats)
    PDF_CUDA(cudaMemcpyAsync(elem_stats, p->es, sizeof(double) * M.n_tri * PDF_NES, cudaMemcpyDefault, st));
  if (node_stats)
    PDF_CUDA(cudaMemcpyAsync(node_stats, p->ns, sizeof(double) * M.n_nodes * PDF_NNS, cudaMemcpyDefault, st));
  if (node_derivs)
    PDF_CUDA(cudaMemcpyAsync(node_derivs, p->nd, sizeof(double) * M.n_nodes * PDF_NND, cudaMemcpyDefault, st));
  return PDF_OK;
}

namespace pdfgb {

// Statistics with caller-chosen grouping buffers (used by the
// allocation-free entry point in noalloc.cu).  keys_a/vals_a receive the
// first radix pass, keys_b/vals_b the second; at most two passes, so
// n_tri <= 2^18.
pdf_status estimate_stats_with_buffers(pdf_particles* P, int32_t* keys_a, int32_t* vals_a,
                                       int32_t* keys_b, int32_t* vals_b, int32_t* hist,
                                       int32_t* hist_part, int32_t* seg, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  const int64_t n = P->n;
  int bits = 1;
  while ((1LL << bits) < (int64_t)M.n_tri) ++bits;
  const int passes = (bits + kRadixBits - 1) / kRadixBits;
  if (passes > 2) return fail(PDF_EINVAL, "estimate_stats_with_buffers: more than 2^18 elements");
  const int64_t n_tiles = radix_tiles(n);
  const int64_t hist_len = n_tiles * kBins;
  const int32_t n_scan = radix_scan_blocks(hist_len);
  const int32_t* kin = P->elem;
  const int32_t* vin = nullptr;
  int32_t* kout[2] = {passes == 2 ? keys_a : keys_b, keys_b};
  int32_t* vout[2] = {passes == 2 ? vals_a : vals_b, vals_b};
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kRadixBits;
    PDF_KERNEL("k_radix_hist", st, k_radix_hist<<<(unsigned)n_tiles, kSortThreads, 0, st>>>(kin, n, shift, n_tiles, hist));
    PDF_KERNEL("k_scan_reduce", st, k_scan_reduce<<<n_scan, 1024, 0, st>>>(hist, hist_len, hist_part));
    PDF_KERNEL("k_scan_top", st, k_scan_top<<<1, 1024, 0, st>>>(hist_part, n_scan));
    PDF_KERNEL("k_scan_apply", st, k_scan_apply<<<n_scan, 1024, 0, st>>>(hist, hist_len, hist_part));
    PDF_KERNEL("k_radix_scatter", st, k_radix_scatter<<<(unsigned)n_tiles, kSortThreads, 0, st>>>(
                                          kin, vin, n, shift, n_tiles, hist, kout[pass], vout[pass]));
    kin = kout[pass];
    vin = vout[pass];
  }
  PDF_KERNEL("k_seg_offsets", st, k_seg_offsets<<<blocks_for(n + 1, 256), 256, 0, st>>>(kin, n, M.n_tri, seg));
  if (P->precision == PDF_FP64)
    PDF_KERNEL("k_elem_stats", st, k_elem_stats_fx<fx::df><<<blocks_for((int64_t)M.n_tri * 32, kStatWarps * 32), kStatWarps * 32, 0, st>>>(
                                       seg, vin, M.n_tri, P->u, P->v, P->w, P->om, P->ps, P->es));
  else
    PDF_KERNEL("k_elem_stats", st, k_elem_stats_fx<float><<<blocks_for((int64_t)M.n_tri * 32, kStatWarps * 32), kStatWarps * 32, 0, st>>>(
                                       seg, vin, M.n_tri, P->uf, P->vf, P->wf, P->omf, P->psf, P->es));
  pdf_status s = node_stats_from_elements(P, st);
  if (s != PDF_OK) return s;
  P->have_stats = true;
  return iecm_cond(P, seg, vin, st);
}

// Stable LSD radix sort of n non-negative int32 keys below 2^bits, the
// values the original indices; ping-pong buffers k0/v0, k1/v1 of n entries,
// hist of radix_tiles(n) * radix_bins() and hist_part of
// radix_scan_blocks(hist_len) + 1 entries.  *keys_out / *vals_out receive
// the sorted buffers.
pdf_status radix_sort_index(const int32_t* keys, int64_t n, int bits, int32_t* k0, int32_t* v0, int32_t* k1,
                            int32_t* v1, int32_t* hist, int32_t* hist_part, const int32_t** keys_out,
                            const int32_t** vals_out, cudaStream_t st) {
  const int64_t n_tiles = radix_tiles(n);
  const int64_t hist_len = n_tiles * kBins;
  const int32_t n_scan = radix_scan_blocks(hist_len);
  const int passes = std::max(1, (bits + kRadixBits - 1) / kRadixBits);
  const int32_t* kin = keys;
  const int32_t* vin = nullptr;
  int32_t* kout[2] = {k0, k1};
  int32_t* vout[2] = {v0, v1};
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kRadixBits;
    int32_t* ko = kout[pass & 1];
    int32_t* vo = vout[pass & 1];
    PDF_KERNEL("k_radix_hist", st, k_radix_hist<<<(unsigned)n_tiles, kSortThreads, 0, st>>>(kin, n, shift, n_tiles, hist));
    PDF_KERNEL("k_scan_reduce", st, k_scan_reduce<<<n_scan, 1024, 0, st>>>(hist, hist_len, hist_part));
    PDF_KERNEL("k_scan_top", st, k_scan_top<<<1, 1024, 0, st>>>(hist_part, n_scan));
    PDF_KERNEL("k_scan_apply", st, k_scan_apply<<<n_scan, 1024, 0, st>>>(hist, hist_len, hist_part));
    PDF_KERNEL("k_radix_scatter", st, k_radix_scatter<<<(unsigned)n_tiles, kSortThreads, 0, st>>>(
                                          kin, vin, n, shift, n_tiles, hist, ko, vo));
    kin = ko;
    vin = vo;
  }
  *keys_out = kin;
  *vals_out = vin;
  return PDF_OK;
}

}  // namespace pdfgb

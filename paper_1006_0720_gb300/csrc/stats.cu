// Particle-in-cell statistics (sec. 3.3) and derivatives (sec. 3.4).
//
// Grouping: a stable least-significant-digit radix sort of (element id,
// storage slot) pairs, 9-bit digits, in place of the paper's per-element
// linked lists.  Stability makes the particle order inside every element
// ascending in storage slot, so the segmented reductions below always add
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

int64_t radix_tiles(int64_t n) { return (n + kTile - 1) / kTile; }
int32_t radix_bins() { return kBins; }
// the digit scan runs one block per digit; callers size the partials
// buffer as radix_scan_blocks(hist_len) + 1
int32_t radix_scan_blocks(int64_t) { return kBins; }

// Per-tile digit histogram, stored bin-major: hist[bin * n_tiles + tile].
// Thread t counts the tile's keys 16t .. 16t + 15 (four 16-byte loads when
// the keys are 16-byte aligned) as runs of equal digits, one shared atomic
// per run: the element ids arrive nearly sorted (the state is reordered
// by element every few steps, and the second pass reads the first pass's
// output), so a thread's sixteen keys are mostly one or two runs.
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const int32_t* __restrict__ keys, int64_t n,
                                                             int shift, int64_t n_tiles,
                                                             int32_t* __restrict__ hist) {
  __shared__ int32_t h[kBins];
  for (int b = threadIdx.x; b < kBins; b += kSortThreads) h[b] = 0;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItemsPerThread;
  int32_t k[kItemsPerThread];
  if (i0 + kItemsPerThread <= n && (reinterpret_cast<uintptr_t>(keys + i0) & 15) == 0) {
    const int4* q = reinterpret_cast<const int4*>(keys + i0);
#pragma unroll
    for (int j = 0; j < kItemsPerThread / 4; ++j) {
      const int4 v = __ldg(q + j);
      k[4 * j] = v.x; k[4 * j + 1] = v.y; k[4 * j + 2] = v.z; k[4 * j + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int r = 0; r < kItemsPerThread; ++r) k[r] = (i0 + r < n) ? __ldg(keys + i0 + r) : 0;
  }
  const int m = (int)max((int64_t)0, min((int64_t)kItemsPerThread, n - i0));  // keys of this thread
  int run_d = -1, run_c = 0;
#pragma unroll
  for (int r = 0; r < kItemsPerThread; ++r) {
    if (r >= m) break;
    const int d = (k[r] >> shift) & (kBins - 1);
    if (d != run_d) {
      if (run_c) atomicAdd(&h[run_d], run_c);
      run_d = d;
      run_c = 0;
    }
    ++run_c;
  }
  if (run_c) atomicAdd(&h[run_d], run_c);
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += kSortThreads) hist[(int64_t)b * n_tiles + blockIdx.x] = h[b];
}

// Exclusive block-wide prefix sum (blockDim a multiple of 32, at most
// 1024); *total receives the block's sum.
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

// Per digit, one block each: the exclusive prefix of the digit's tile
// counts over the tiles (in place; the digit's row of hist is contiguous)
// and the digit's total in part[digit].  The scatter adds the totals of the
// smaller digits.  512 threads (the 512 digit blocks fit on the GPU at once,
// four per SM); each round stages 4,096 entries through shared memory with
// coalesced loads and stores, thread t scanning entries 8t .. 8t + 7 (one
// padding word per 32 keeps those reads free of bank conflicts).
constexpr int kScanThreads = 512;
constexpr int kScanPer = 8;
constexpr int kScanRound = kScanThreads * kScanPer;  // 4096
__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }
__global__ void __launch_bounds__(kScanThreads, 4) k_scan_bins(int32_t* __restrict__ hist, int64_t n_tiles,
                                                            int32_t* __restrict__ part) {
  __shared__ int32_t s[kScanRound + kScanRound / 32];
  int32_t* row = hist + (int64_t)blockIdx.x * n_tiles;
  int32_t carry = 0;
  for (int64_t start = 0; start < n_tiles; start += kScanRound) {
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      const int i = threadIdx.x + j * kScanThreads;
      s[scan_pad(i)] = (start + i < n_tiles) ? row[start + i] : 0;
    }
    __syncthreads();
    int32_t v[kScanPer];
    int32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      v[j] = s[scan_pad(kScanPer * threadIdx.x + j)];
      sum += v[j];
    }
    int32_t total;
    int32_t ex = block_exclusive_scan(sum, &total) + carry;  // (its barriers order the reads above)
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      s[scan_pad(kScanPer * threadIdx.x + j)] = ex;
      ex += v[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      const int i = threadIdx.x + j * kScanThreads;
      if (start + i < n_tiles) row[start + i] = s[scan_pad(i)];
    }
    carry += total;
    __syncthreads();  // the next round overwrites s
  }
  if (threadIdx.x == 0) part[blockIdx.x] = carry;
}

// Stable scatter of one tile, 512 threads of 8 items.  Warp w owns the
// tile's items [256 w, 256 (w + 1)) and ranks them in 8 rounds of 32 in
// index order (match.any groups equal digits, one lane of each group
// advances the warp's own row of shared digit counters, so no block barrier
// between rounds); one pass over the (warp, digit) counts then gives every
// warp and digit its output offset, so items with equal digits keep their
// index order.  Twice the warps per SM of 256 threads with 16 items each
// (64 registers, two blocks per SM): the ranking waits on the MIO queue, and
// more warps cover it.
constexpr int kScatterThreads = 512;
constexpr int kScatterItems = kTile / kScatterThreads;  // 8
__global__ void __launch_bounds__(kScatterThreads, 2) k_radix_scatter(
    const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, int64_t n, int shift,
    int64_t n_tiles, const int32_t* __restrict__ hist, const int32_t* __restrict__ part,
    int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out) {
  constexpr int kWarps = kScatterThreads / 32;  // 16
  constexpr int kPerWarp = kTile / kWarps;      // 256 items, 8 rounds
  static_assert(kBins == kScatterThreads, "one digit per thread in the digit-base scan");
  __shared__ int32_t wcnt[kWarps][kBins + 1];  // the extra bin takes the tile's padding
  __shared__ int32_t dbase[kBins];             // first output position of each digit
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  {
    const int32_t c0 = __ldg(part + threadIdx.x);
    int32_t total;
    dbase[threadIdx.x] = block_exclusive_scan(c0, &total);
  }
  // this tile's count of the thread's digit, loaded before the ranking
  const int32_t th0 = hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
  for (int i = threadIdx.x; i < kWarps * (kBins + 1); i += kScatterThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t w0 = (int64_t)blockIdx.x * kTile + (int64_t)wid * kPerWarp;
  int32_t key[kScatterItems], val[kScatterItems], off[kScatterItems];
#pragma unroll
  for (int r = 0; r < kScatterItems; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    const bool valid = i < n;
    key[r] = valid ? keys_in[i] : 0;
    val[r] = valid ? (vals_in ? vals_in[i] : (int32_t)i) : 0;
  }
#pragma unroll
  for (int r = 0; r < kScatterItems; ++r) {
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
  {  // (warp, digit) offsets: the digit's base, the earlier tiles' counts of
     // the digit and the earlier warps' counts
    const int b = threadIdx.x;
    int32_t acc = dbase[b] + th0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      const int32_t c = wcnt[k][b];
      wcnt[k][b] = acc;
      acc += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kScatterItems; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    if (i < n) {
      const int d = (key[r] >> shift) & (kBins - 1);
      const int32_t pos = wcnt[wid][d] + off[r];
      keys_out[pos] = key[r];
      vals_out[pos] = val[r];
    }
  }
}

// seg[e] = first sorted position whose key >= e; seg[n_tri] = n.  Thread t
// takes positions 16t .. 16t + 15 (four 16-byte loads when the keys are
// 16-byte aligned) and position n counts as key n_tri; the key before the
// thread's first comes from the lane below (lane 0 loads it).  One thread
// per 16 positions, n / 16 + 1 threads in all.
constexpr int kSegPer = 16;
int64_t seg_offsets_threads(int64_t n) { return n / kSegPer + 1; }
__global__ void __launch_bounds__(256) k_seg_offsets(const int32_t* __restrict__ keys, int64_t n, int32_t n_tri,
                                                     int32_t* __restrict__ seg) {
  const int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * kSegPer;
  int32_t k[kSegPer];
  if (i0 + kSegPer <= n && (reinterpret_cast<uintptr_t>(keys + i0) & 15) == 0) {
    const int4* q = reinterpret_cast<const int4*>(keys + i0);
#pragma unroll
    for (int j = 0; j < kSegPer / 4; ++j) {
      const int4 v = __ldg(q + j);
      k[4 * j] = v.x; k[4 * j + 1] = v.y; k[4 * j + 2] = v.z; k[4 * j + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < kSegPer; ++j) k[j] = (i0 + j < n) ? __ldg(keys + i0 + j) : n_tri;
  }
  int32_t prev = __shfl_up_sync(0xffffffffu, k[kSegPer - 1], 1);
  if ((threadIdx.x & 31) == 0) prev = (i0 == 0) ? -1 : ((i0 - 1 < n) ? __ldg(keys + i0 - 1) : n_tri);
  if (i0 > n) return;
#pragma unroll
  for (int j = 0; j < kSegPer; ++j) {
    const int64_t i = i0 + j;
    if (i > n) break;
    const int32_t cur = k[j];  // n_tri at i == n
    for (int32_t e = prev + 1; e <= cur; ++e) seg[e] = (int32_t)i;
    prev = cur;
  }
}

// A stored state value as a double-float (exact for both storage forms).
__device__ __forceinline__ fx::df ld_df(const fx::df* a, int64_t i) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(a) + i);
  return fx::df{v.x, v.y};
}
__device__ __forceinline__ fx::df ld_df(const float* a, int64_t i) { return fx::df{__ldg(a + i), 0.f}; }

// Eight lanes per element (four elements per warp), one pass over the
// element's particles in the grouping's order (sec. 3.3: N, means, central
// moments with 1/N).  Lane j of a group takes sorted positions j, j + 8, ...
// (eight consecutive positions per load across the group).  Every value
// enters as its deviation d = x - x_0 from the element's first particle, a
// double-float with an absolute error of about 2^-48 |x| (the resolution of
// the stored forms); each lane sums the deviations and their pairwise
// products in double-float in its order, the eight lane sums are combined
// by a fixed butterfly, and
//   mean = x_0 + S_a / N,   moment_ab = (S_ab - S_a S_b / N) / N.
// The shift keeps the cancellation in the moments to a factor of about two
// (the deviations are of the size of the fluctuations).  The order of every
// addition is fixed by the stable grouping, so the results are
// deterministic; a reordering of the storage changes them by rounding only.
// Only FP32 additions and fused multiply-adds per particle (no conversions).
constexpr int kStatLanes = 8;

__device__ __forceinline__ void prefetch_l2(const void* a) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

__device__ __forceinline__ void acc_xor(fx::acc& a, int o) {
  const float h = __shfl_xor_sync(0xffffffffu, a.h, o);
  const float l = __shfl_xor_sync(0xffffffffu, a.l, o);
  a.add(fx::df{h, l});
}

// x - k for stored double-floats, normalized: fx::sub with the final
// renormalization by Fast2Sum instead of TwoSum.  Stored values satisfy
// |l| <= ulp(h)/2, so after the exact TwoSum of the high parts (s, e) the
// low part t = x.l + (e - k.l) never has a larger exponent than s (equal
// exponents: x.h - k.h is exact and a nonzero multiple of the ulp, and
// |t| <= one ulp; across a power of two |t| <= 1.5 ulps of the smaller;
// otherwise |t| is far below |s|; s = 0 gives (t, 0)): under that condition
// Fast2Sum returns the same pair as TwoSum, three instructions fewer.
__device__ __forceinline__ fx::df deviation(fx::df x, fx::df k) {
  const fx::df s = fx::two_sum(x.h, -k.h);
  const float t = __fadd_rn(x.l, __fadd_rn(s.l, -k.l));
  return fx::fast_two_sum(s.h, t);
}

// a[i] for a lane-dependent i, by selects (no local-memory array)
template <int N>
__device__ __forceinline__ fx::df pick(const fx::df (&a)[N], int i) {
  fx::df r = a[0];
#pragma unroll
  for (int q = 1; q < N; ++q)
    if (i == q) r = a[q];
  return r;
}
template <int N>
__device__ __forceinline__ fx::df pick_acc(const fx::acc (&a)[N], int i) {
  fx::df r = fx::df{a[0].h, a[0].l};
#pragma unroll
  for (int q = 1; q < N; ++q)
    if (i == q) r = fx::df{a[q].h, a[q].l};
  return fx::df_norm(r);
}

// Central moment m (pairs uu, vv, ww, uv, uw, vw, psi psi) from the sums of
// the deviations (s1) and of their products (s2): (S_ab - S_a S_b / N) / N.
__device__ __forceinline__ double moment(const fx::acc (&s1)[5], const fx::acc (&s2)[7], int m, fx::df invN) {
  const int a = m == 6 ? 4 : (m < 3 ? m : (m == 5 ? 1 : 0));
  const int b = m == 6 ? 4 : (m < 3 ? m : (m == 3 ? 1 : 2));
  const fx::df Sa = pick_acc(s1, a), Sb = pick_acc(s1, b);
  const fx::df corr = fx::df_norm(fx::mul(fx::df_norm(fx::mul(Sa, Sb)), invN));
  return __longlong_as_double((long long)fx::df2d(fx::df_norm(fx::mul(fx::sub(pick_acc(s2, m), corr), invN))));
}

template <typename T>
__global__ void __launch_bounds__(256, 3) k_elem_stats_grp(const int32_t* __restrict__ seg,
                                                       const int32_t* __restrict__ pid, int32_t n_tri,
                                                       const T* __restrict__ u, const T* __restrict__ v,
                                                       const T* __restrict__ w, const T* __restrict__ om,
                                                       const T* __restrict__ ps, double* __restrict__ es) {
  const int lane = threadIdx.x & 31, j = lane & (kStatLanes - 1);
  const int64_t group = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kStatLanes;
  const int64_t n_groups = ((int64_t)gridDim.x * blockDim.x) / kStatLanes;
  // every lane of a warp runs the same number of rounds (the butterfly
  // below needs all 32 lanes)
  const int64_t rounds = (n_tri + n_groups - 1) / n_groups;
  int64_t e = group;
  for (int64_t r = 0; r < rounds; ++r, e += n_groups) {
    const bool live = e < n_tri;
    const int32_t beg = live ? seg[e] : 0, end = live ? seg[e + 1] : 0;
    const int32_t N = end - beg;
    {  // the next element of this group on its way to L2 (after a
       // reordering of the state its particles sit near their positions in
       // the grouped order)
      const int64_t en = e + n_groups;
      if (en < n_tri) {
        const int32_t nb = seg[en], ne = seg[en + 1];
        for (int32_t i = nb + 16 * j; i < ne; i += 16 * kStatLanes) {
          prefetch_l2(u + i); prefetch_l2(v + i); prefetch_l2(w + i); prefetch_l2(om + i); prefetch_l2(ps + i);
          if (pid) prefetch_l2(pid + i);
        }
      }
    }
    fx::df K[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) K[q] = fx::df{0.f, 0.f};
    if (N > 0) {
      const int32_t p0 = pid ? __ldg(pid + beg) : beg;
      K[0] = ld_df(u, p0); K[1] = ld_df(v, p0); K[2] = ld_df(w, p0); K[3] = ld_df(om, p0); K[4] = ld_df(ps, p0);
    }
    fx::acc s1[5], s2[7];
#pragma unroll
    for (int q = 0; q < 5; ++q) s1[q].init(fx::df{0.f, 0.f});
#pragma unroll
    for (int q = 0; q < 7; ++q) s2[q].init(fx::df{0.f, 0.f});
    // two particles per lane and iteration (positions i and i + 8), their
    // slots loaded one iteration ahead, so that ten state loads are in
    // flight before the first is needed; the sums still take the particles
    // in the lane's order i, i + 8, i + 16, ...
    auto slot = [&](int32_t i) { return pid ? __ldg(pid + i) : i; };
    int32_t qa = beg + j < end ? slot(beg + j) : 0;
    int32_t qb = beg + j + kStatLanes < end ? slot(beg + j + kStatLanes) : 0;
    auto acc1 = [&](fx::df xu, fx::df xv, fx::df xw, fx::df xm, fx::df xp) {
      // normalized, so that the dropped product of the low parts is below
      // 2^-48 of the product even when the deviation is far below the value
      const fx::df du = deviation(xu, K[0]);
      const fx::df dv = deviation(xv, K[1]);
      const fx::df dw = deviation(xw, K[2]);
      const fx::df dm = deviation(xm, K[3]);
      const fx::df dp = deviation(xp, K[4]);
      s1[0].add(du); s1[1].add(dv); s1[2].add(dw); s1[3].add(dm); s1[4].add(dp);
      s2[0].add(fx::mul(du, du));
      s2[1].add(fx::mul(dv, dv));
      s2[2].add(fx::mul(dw, dw));
      s2[3].add(fx::mul(du, dv));
      s2[4].add(fx::mul(du, dw));
      s2[5].add(fx::mul(dv, dw));
      s2[6].add(fx::mul(dp, dp));
    };
    for (int32_t i = beg + j; i < end; i += 2 * kStatLanes) {
      const int32_t pa = qa, pb = qb;
      const bool hb = i + kStatLanes < end;
      qa = i + 2 * kStatLanes < end ? slot(i + 2 * kStatLanes) : 0;
      qb = i + 3 * kStatLanes < end ? slot(i + 3 * kStatLanes) : 0;
      const fx::df au = ld_df(u, pa), av = ld_df(v, pa), aw = ld_df(w, pa), am = ld_df(om, pa), ap = ld_df(ps, pa);
      fx::df bu = au, bv = av, bw = aw, bm = am, bp = ap;
      if (hb) { bu = ld_df(u, pb); bv = ld_df(v, pb); bw = ld_df(w, pb); bm = ld_df(om, pb); bp = ld_df(ps, pb); }
      acc1(au, av, aw, am, ap);
      if (hb) acc1(bu, bv, bw, bm, bp);
    }
    // butterfly within the group of eight: every lane ends with the totals
#pragma unroll
    for (int o = kStatLanes / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < 5; ++q) acc_xor(s1[q], o);
#pragma unroll
      for (int q = 0; q < 7; ++q) acc_xor(s2[q], o);
    }
    if (!live) continue;
    double* out = es + e * PDF_NES;
    if (N == 0) {
#pragma unroll
      for (int q = 0; q < PDF_NES; ++q)
        if ((q & (kStatLanes - 1)) == j) out[q] = 0.0;
      continue;
    }
    // the 13 outputs (N, the five means, the seven central moments) are
    // shared out: lane j forms and writes outputs j and j + 8
    // (lanes 1-5 a mean, lanes 0-4 and 6-7 one moment each: one pass of
    // each formula per warp)
    const fx::df invN = fx::recip_df(N);
    if (j == 0) out[0] = (double)N;
    if (j >= 1 && j <= 5) {
      const fx::df Kq = pick(K, j - 1);
      const fx::df Sq = pick_acc(s1, j - 1);
      out[j] = __longlong_as_double((long long)fx::df2d(fx::add(Kq, fx::df_norm(fx::mul(Sq, invN)))));
    }
    const int m = j < 5 ? j + 2 : j - 6;  // output 6 + m; lane 5 has none
    if (j != 5) out[6 + m] = moment(s1, s2, m, invN);
  }
}

// 1 / c for the element counts of a node (the correctly rounded quotients,
// as the division gives them): GB300's FP64 pipe bounds the node passes,
// and a division costs it more than a dozen instructions.
constexpr int kRecipMax = 64;
struct RecipTable {
  double v[kRecipMax + 1];
  constexpr RecipTable() : v() {
    v[0] = 0.0;
    for (int c = 1; c <= kRecipMax; ++c) v[c] = 1.0 / (double)c;
  }
};
__device__ const RecipTable kRecip;
__device__ __forceinline__ double recip_count(int32_t c) {
  return c <= kRecipMax ? __ldg(&kRecip.v[c]) : 1.0 / (double)c;
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
      // s[0] = N >= 0: the bits of +0.0 (and -0.0) are not positive, those of
      // any N > 0 are (an integer test instead of an FP64 compare)
      if (__double_as_longlong(s[0]) <= 0) continue;
#pragma unroll
      for (int q = 0; q < PDF_NNS; ++q) acc[q] += s[1 + q];
      ++c;
    }
    if (c == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(kept), 1ULL);
      continue;
    }
    const double inv = recip_count(c);
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
    const double inv = recip_count(c > 0 ? c : 1);
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
    const double inv = recip_count(c > 0 ? c : 1);
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

// One stable pass of the radix sort on the digit at `shift`: tile
// histograms, the per-digit scan over the tiles, the scatter.  hist holds
// n_tiles * kBins entries, part kBins.
static pdf_status radix_pass(const int32_t* kin, const int32_t* vin, int64_t n, int shift, int64_t n_tiles,
                             int32_t* hist, int32_t* part, int32_t* kout, int32_t* vout, cudaStream_t st) {
  PDF_KERNEL("k_radix_hist", st, k_radix_hist<<<(unsigned)n_tiles, kSortThreads, 0, st>>>(kin, n, shift, n_tiles, hist););
  PDF_KERNEL("k_scan_bins", st, k_scan_bins<<<kBins, kScanThreads, 0, st>>>(hist, n_tiles, part););
  PDF_KERNEL("k_radix_scatter", st, k_radix_scatter<<<(unsigned)n_tiles, kScatterThreads, 0, st>>>(
                                        kin, vin, n, shift, n_tiles, hist, part, kout, vout););
  return PDF_OK;
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
    const pdf_status s = radix_pass(kin, vin, n, shift, P->n_tiles, P->hist, P->hist_part, P->keys[cur],
                                    P->vals[cur], st);
    if (s != PDF_OK) return s;
    kin = P->keys[cur];
    vin = P->vals[cur];
    cur ^= 1;
  }
  PDF_KERNEL("k_seg_offsets", st, k_seg_offsets<<<(unsigned)((seg_offsets_threads(n) + 255) / 256), 256, 0, st>>>(kin, n, n_tri, P->seg););
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

// Copies the state into the grouping's order, into the second set of state
// arrays (adopt_reorder then makes them the state).
static pdf_status launch_reorder(pdf_particles* P, cudaStream_t st) {
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
  // one thread per particle (0.31 ms at 15.9M particles against 0.46 ms
  // for a grid of 32 blocks per SM striding over them)
  PDF_KERNEL("k_reorder", st, k_reorder<<<(unsigned)((P->n + 255) / 256), 256, 0, st>>>(R););
  return PDF_OK;
}

// Adopts the copy (host pointers only; work issued afterwards sees it): the
// sorted order becomes the storage order (sorted_pid = NULL) and the element
// ids are the sorted keys.
static void adopt_reorder(pdf_particles* P) {
  std::swap(P->x, P->x2);
  std::swap(P->y, P->y2);
  std::swap(P->u, P->u2); std::swap(P->v, P->v2); std::swap(P->w, P->w2);
  std::swap(P->om, P->om2); std::swap(P->ps, P->ps2);
  std::swap(P->uf, P->uf2); std::swap(P->vf, P->vf2); std::swap(P->wf, P->wf2);
  std::swap(P->omf, P->omf2); std::swap(P->psf, P->psf2);
  std::swap(P->pid, P->pid2);
  std::swap(P->elem, P->keys[P->sorted_key_slot]);
  P->sorted_pid = nullptr;
}

pdf_status iecm_cond(pdf_particles* P, const int32_t* seg, const int32_t* order, cudaStream_t st);

// Element statistics of the grouped particles (seg, order) into P->es.
static pdf_status elem_stats(pdf_particles* P, const int32_t* seg, const int32_t* order, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  // one element per group of eight lanes up to 48 blocks of 256 per SM
  // (three resident at 80 registers); beyond that each group walks several
  // elements and prefetches the next one.  At 15.9M particles on 158,802
  // elements 3, 12, 24 and 48 blocks per SM took 0.29, 0.27, 0.25 and
  // 0.22 ms: with one element per group no group waits for a long one.
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)M.n_tri * kStatLanes + 255) / 256,
                                                           (int64_t)sm_count() * 48));
  if (P->precision == PDF_FP64)
    PDF_KERNEL("k_elem_stats", st, k_elem_stats_grp<fx::df><<<nb, 256, 0, st>>>(
                                       seg, order, M.n_tri, P->u, P->v, P->w, P->om, P->ps, P->es));
  else
    PDF_KERNEL("k_elem_stats", st, k_elem_stats_grp<float><<<nb, 256, 0, st>>>(
                                       seg, order, M.n_tri, P->uf, P->vf, P->wf, P->omf, P->psf, P->es));
  return PDF_OK;
}



// Node statistics and node derivatives from the element statistics P->es
// (sec. 3.3 second pass, sec. 3.4).
pdf_status node_stats_from_elements(pdf_particles* P, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  PDF_KERNEL("k_node_stats", st, k_node_stats<<<blocks_for(M.n_nodes, 128), 128, 0, st>>>(M.nse_off, M.nse, M.n_nodes, P->es, P->ns,
                                                          P->counters + 8););
  return node_derivs_from_node_stats(P, st);
}

pdf_status node_derivs_from_node_stats(pdf_particles* P, cudaStream_t st) {
  const MeshDev& M = P->mesh->d;
  PDF_KERNEL("k_elem_grad1", st, k_elem_grad1<<<blocks_for(M.n_tri, 128), 128, 0, st>>>(M.tri, M.dN, M.n_tri, P->ns, P->eg););
  PDF_KERNEL("k_node_grad1", st, k_node_grad1<<<blocks_for(M.n_nodes, 128), 128, 0, st>>>(M.nse_off, M.nse, M.n_nodes, P->eg, P->nd););
  PDF_KERNEL("k_elem_grad2", st, k_elem_grad2<<<blocks_for(M.n_tri, 128), 128, 0, st>>>(M.tri, M.dN, M.n_tri, P->nd, P->eg););
  PDF_KERNEL("k_node_grad2", st, k_node_grad2<<<blocks_for(M.n_nodes, 128), 128, 0, st>>>(M.nse_off, M.nse, M.n_nodes, P->eg, P->nd););
  return PDF_OK;
}

pdf_status estimate_stats(pdf_particles* P, cudaStream_t st) {
  pdf_status s = group_by_element(P, st);
  if (s != PDF_OK) return s;
  if (P->reorder_every > 0 && ++P->since_reorder >= P->reorder_every) {
    // (the copy beside the statistics on a second stream gained nothing:
    // both are limited by the same gathers)
    s = launch_reorder(P, st);
    if (s != PDF_OK) return s;
    adopt_reorder(P);
    P->since_reorder = 0;
  }
  s = elem_stats(P, P->seg, P->sorted_pid, st);
  if (s != PDF_OK) return s;
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
  const int32_t* kin = P->elem;
  const int32_t* vin = nullptr;
  int32_t* kout[2] = {passes == 2 ? keys_a : keys_b, keys_b};
  int32_t* vout[2] = {passes == 2 ? vals_a : vals_b, vals_b};
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kRadixBits;
    const pdf_status s = radix_pass(kin, vin, n, shift, n_tiles, hist, hist_part, kout[pass], vout[pass], st);
    if (s != PDF_OK) return s;
    kin = kout[pass];
    vin = vout[pass];
  }
  PDF_KERNEL("k_seg_offsets", st, k_seg_offsets<<<(unsigned)((seg_offsets_threads(n) + 255) / 256), 256, 0, st>>>(kin, n, M.n_tri, seg));
  pdf_status s = elem_stats(P, seg, vin, st);
  if (s != PDF_OK) return s;
  s = node_stats_from_elements(P, st);
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
  const int passes = std::max(1, (bits + kRadixBits - 1) / kRadixBits);
  const int32_t* kin = keys;
  const int32_t* vin = nullptr;
  int32_t* kout[2] = {k0, k1};
  int32_t* vout[2] = {v0, v1};
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kRadixBits;
    int32_t* ko = kout[pass & 1];
    int32_t* vo = vout[pass & 1];
    const pdf_status s = radix_pass(kin, vin, n, shift, n_tiles, hist, hist_part, ko, vo, st);
    if (s != PDF_OK) return s;
    kin = ko;
    vin = vo;
  }
  *keys_out = kin;
  *vals_out = vin;
  return PDF_OK;
}

}  // namespace pdfgb

// Sample-and-train: the RMI eCDF model of Sec. 2 / Sec. 6.1 (two layers,
// linear leaves, trained on a stratified 1% sample), plus the heavy-value set
// that feeds the equality buckets.
//
//  1. gather s keys at stratified offsets, as total-order keys;
//  2. sort of the sample: sample sort for 8-byte keys (ls_samplesort.cuh), LSD
//     radix sort for 4-byte keys (ls_radix.cuh);
//  3. FP64 least squares: root over all finite sample keys against their eCDF
//     rank (count of sample keys below x, ties take the first rank), then one
//     line per leaf over the keys the root routes to it; slopes clamped to >= 0
//     and each leaf's output clamped to [lo_l, hi_l] so that F is monotone;
//  4. the per-key lookup of the FP64 level-0 map: its f0 thresholds in the
//     total order (bisection over the FP64 model), an FP32 cell-index RMI
//     fitted to the same sample, and the bucket range of each of its cells
//     (no FP64 in the per-key path);
//  5. heavy values: sample runs of length >= tau, at most `hpb` per level-0
//     bucket (longest first), each given an equality slot.
// All reductions use a fixed order, so a model is bit-reproducible run to run.
#include <cfloat>

#include "ls_radix.cuh"
#include "ls_samplesort.cuh"
#include "ls_train.cuh"

namespace ls {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // SplitMix64 output function
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// x / d and x mod d by the reciprocal m = floor((2^64 - 1) / d) (Barrett
// reduction): floor(x * m / 2^64) is at most 2 below the quotient, and the
// corrections fix it exactly.
struct Div64 {
  uint64_t d, m;
};
static Div64 make_div64(uint64_t d) { return Div64{d, ~0ull / d}; }
__device__ __forceinline__ uint64_t div64(uint64_t x, const Div64& v, uint64_t* rem) {
  uint64_t q = __umul64hi(x, v.m);
  uint64_t r = x - q * v.d;
  if (r >= v.d) { r -= v.d; ++q; }
  if (r >= v.d) { r -= v.d; ++q; }
  *rem = r;
  return q;
}

// Stratified sample: i_k = floor(k n / s) + mix64(seed ^ k) mod max(1, floor(n / s)).
__device__ __forceinline__ uint64_t sample_index(uint64_t k, uint64_t n, uint64_t s, uint64_t seed,
                                                 const Div64& ds, const Div64& dst) {
  uint64_t base, r;
  if (n < (1ull << 32)) base = div64(k * n, ds, &r);  // k < s <= n: k n < 2^64
  else base = (uint64_t)(((unsigned __int128)k * n) / s);
  div64(mix64(seed ^ k), dst, &r);
  const uint64_t i = base + r;
  return i < n ? i : n - 1;  // (i < n by the formula; the clamp keeps the load in bounds)
}

// The sample (total-order keys).  When `spl` is given (the sample sort's
// path), CTA 0 instead draws the sample sort's evenly spaced oversample of the
// sample -- sample positions (8 t + q) s / SS_CAND, read from the input keys
// directly, so it overlaps the other CTAs' gathering -- sorts it and stores
// every SS_OVER-th key as a splitter, and clears the sample sort's counters.
template <int DT>
__global__ void __launch_bounds__(1024)
k_sample(const typename KT<DT>::U* __restrict__ keys, uint64_t n, uint64_t s, uint64_t seed,
         Div64 ds, Div64 dst, uint64_t* __restrict__ out, uint64_t* __restrict__ spl,
         uint32_t* __restrict__ cnt) {
  pdl_begin();
  if (spl && blockIdx.x == 0) {
    extern __shared__ uint64_t ss_c[];
    const uint32_t base = 8 * threadIdx.x;
    uint64_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      v[q] = KT<DT>::tk(keys[sample_index((uint64_t)(base + q) * s / SS_CAND, n, s, seed, ds, dst)]);
    for (uint32_t i = threadIdx.x; i <= SS_NB; i += blockDim.x) cnt[i] = 0;
    ss_sort_regs(v, ss_c, SS_CAND);
#pragma unroll
    for (int q = SS_OVER - 1; q < 8; q += SS_OVER) spl[(base + q) / SS_OVER] = v[q];
    return;
  }
  const uint64_t b0 = spl ? blockIdx.x - 1 : blockIdx.x, nb = spl ? gridDim.x - 1 : gridDim.x;
  for (uint64_t k = b0 * blockDim.x + threadIdx.x; k < s; k += nb * blockDim.x)
    out[k] = KT<DT>::tk(keys[sample_index(k, n, s, seed, ds, dst)]);
}

__global__ void k_train_init(DevModel* hdr, uint64_t s, uint32_t* leaf_beg, uint32_t* leaf_end,
                             int L, double* partials, ZeroList z, CallStatus* cs, uint32_t stall,
                             unsigned long long spin_limit) {
  pdl_begin();
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
#pragma unroll
  for (int r = 0; r < ZERO_REGIONS; ++r)
    if (z.p[r])
      for (uint32_t i = tid; i < z.words[r]; i += nth) ((uint32_t*)z.p[r])[i] = 0u;
  if (cs && tid == 0) { cs->word = 0u; cs->stall = stall; cs->spin_limit = spin_limit; }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    hdr->s = s;
    hdr->s_lo = ~0ull;
    hdr->s_fin = 0;
    hdr->nheavy = 0;
    hdr->heavy_len = 0;
    hdr->compact = 0;
    hdr->hash_probes = 0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
    leaf_beg[i] = 0;
    leaf_end[i] = 0;
  }
}

// Finite keys are contiguous in total order: [s_lo, s_hi).  In the sorted
// sample the two ends are where finiteness changes, so each is written once.
template <int DT>
__global__ void k_finite_range(const uint64_t* __restrict__ tk, uint64_t s, DevModel* hdr,
                               unsigned long long* hi_out) {
  pdl_begin();
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < s;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (!KT<DT>::finite(KT<DT>::from_tk(tk[k]))) continue;
    if (k == 0 || !KT<DT>::finite(KT<DT>::from_tk(tk[k - 1]))) hdr->s_lo = k;
    if (k + 1 == s || !KT<DT>::finite(KT<DT>::from_tk(tk[k + 1]))) *hi_out = k + 1;
  }
}

__global__ void k_finite_fix(DevModel* hdr, const unsigned long long* hi) {
  pdl_begin();
  if (hdr->s_lo == ~0ull || *hi <= hdr->s_lo) {
    hdr->s_lo = 0;
    hdr->s_fin = 0;
  } else {
    hdr->s_fin = *hi - hdr->s_lo;
  }
}

// first_rank[k]: index (within the finite range) of the first key equal to key k.
// Per block of FR_CHUNK keys: one bisection for the block's first key, then the
// latest run start at or before each key by a block max-scan.
constexpr int FR_THREADS = 1024;
constexpr int FR_PER = 2;
constexpr int FR_CHUNK = FR_THREADS * FR_PER;

__global__ void __launch_bounds__(FR_THREADS)
k_first_rank(const uint64_t* __restrict__ tk, const DevModel* hdr, uint32_t* __restrict__ rank,
             uint64_t s_cap) {
  pdl_begin();
  __shared__ uint32_t ws[33];
  __shared__ uint32_t s_r0;
  const uint64_t m = hdr->s_fin, lo = hdr->s_lo;
  const uint64_t* t = tk + lo;
  for (uint64_t k0 = (uint64_t)blockIdx.x * FR_CHUNK; k0 < m; k0 += (uint64_t)gridDim.x * FR_CHUNK) {
    if (threadIdx.x == 0) {
      const uint64_t v = t[k0];
      uint64_t a = 0, b = k0;  // lower_bound of the block's first key
      while (a < b) {
        const uint64_t mid = (a + b) >> 1;
        if (t[mid] < v) a = mid + 1; else b = mid;
      }
      s_r0 = (uint32_t)a;
    }
    uint32_t st[FR_PER], mx = 0;
#pragma unroll
    for (int j = 0; j < FR_PER; ++j) {
      const uint64_t k = k0 + (uint64_t)threadIdx.x * FR_PER + j;
      st[j] = 0;
      if (k < m && (k == 0 || t[k - 1] != t[k])) st[j] = (uint32_t)k;
      mx = max(mx, st[j]);
    }
    // inclusive max-scan of the thread maxima (warp shuffles, then warps)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = mx;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc = max(inc, y);
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      uint32_t w = lane < FR_THREADS / 32 ? ws[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w = max(w, y);
      }
      ws[lane] = w;
    }
    __syncthreads();
    uint32_t run = max(s_r0, wid ? ws[wid - 1] : 0u);
    run = max(run, __shfl_up_sync(0xffffffffu, inc, 1) * (lane ? 1u : 0u));
#pragma unroll
    for (int j = 0; j < FR_PER; ++j) {
      const uint64_t k = k0 + (uint64_t)threadIdx.x * FR_PER + j;
      run = max(run, st[j]);
      if (k < m) rank[k] = run;
    }
    __syncthreads();
  }
}

constexpr int FIT_THREADS = 256;

__device__ __forceinline__ double block_sum_d(double v, double* ws) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  double r = 0;
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

template <int DT>
__device__ __forceinline__ double sample_x(const uint64_t* tk, uint64_t lo, uint64_t k) {
  return KT<DT>::dbl(KT<DT>::from_tk(tk[lo + k]));
}

// s += (dx, dy, dx dx, dx dy) over points k0, k0 + step, ... < k1, in that
// order; the loads of four points are issued before their terms are added.
template <int DT>
__device__ __forceinline__ void fit_accumulate(const uint64_t* tk, const uint32_t* rank, uint64_t lo,
                                               uint64_t k0, uint64_t k1, uint64_t step, double xr,
                                               double yr, double inv_m, double (&s)[4]) {
  uint64_t k = k0;
  for (; k + 3 * step < k1; k += 4 * step) {
    double x[4];
    uint32_t rk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      x[q] = sample_x<DT>(tk, lo, k + q * step);
      rk[q] = rank[k + q * step];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double dx = x[q] - xr;
      const double dy = (double)rk[q] * inv_m - yr;
      s[0] += dx; s[1] += dy; s[2] += dx * dx; s[3] += dx * dy;
    }
  }
  for (; k < k1; k += step) {
    const double dx = sample_x<DT>(tk, lo, k) - xr;
    const double dy = (double)rank[k] * inv_m - yr;
    s[0] += dx; s[1] += dy; s[2] += dx * dx; s[3] += dx * dy;
  }
}

// Root least squares in one pass, shifted by the first point (x_r, y_r):
// sums of dx, dy, dx*dx, dx*dy per block (the leaves use the same formulas).
template <int DT>
__global__ void __launch_bounds__(FIT_THREADS)
k_fit_sums(const uint64_t* __restrict__ tk, const uint32_t* __restrict__ rank,
           const DevModel* hdr, double* partials) {
  pdl_begin();
  __shared__ double ws[33];
  const uint64_t m = hdr->s_fin, lo = hdr->s_lo;
  const uint64_t chunk = (m + gridDim.x - 1) / gridDim.x;
  const uint64_t b = blockIdx.x * chunk, e = min(m, b + chunk);
  const double inv_m = m ? 1.0 / (double)m : 0.0;
  const double xr = m ? sample_x<DT>(tk, lo, 0) : 0.0, yr = m ? (double)rank[0] * inv_m : 0.0;
  double s[4] = {0, 0, 0, 0};
  fit_accumulate<DT>(tk, rank, lo, b + threadIdx.x, e, blockDim.x, xr, yr, inv_m, s);
  for (int i = 0; i < 4; ++i) {
    const double t = block_sum_d(s[i], ws);
    if (threadIdx.x == 0) partials[4 * blockIdx.x + i] = t;
  }
}

template <int DT>
__global__ void k_fit_root(DevModel* hdr, const uint64_t* __restrict__ tk,
                           const uint32_t* __restrict__ rank, const double* partials, int nblk) {
  pdl_begin();
  // block partials summed lane-strided, then by a fixed warp tree (deterministic)
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int i = threadIdx.x; i < nblk; i += 32) {
    s0 += partials[4 * i]; s1 += partials[4 * i + 1];
    s2 += partials[4 * i + 2]; s3 += partials[4 * i + 3];
  }
  s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2); s3 = warp_sum(s3);
  if (threadIdx.x != 0) return;
  const uint64_t m = hdr->s_fin, lo = hdr->s_lo;
  if (!m) { hdr->root64[0] = 0.0; hdr->root64[1] = 0.0; hdr->root64[2] = 0.5; return; }
  const double xr = sample_x<DT>(tk, lo, 0), yr = (double)rank[0] / (double)m;
  const double cnt = (double)m;
  const double mdx = s0 / cnt, mdy = s1 / cnt;
  const double sxx = s2 - s0 * mdx, sxy = s3 - s0 * mdy;
  const double mx = xr + mdx;
  double a = (sxx > 0) ? sxy / sxx : 0.0;
  if (!(a >= 0) || !isfinite(a) || !isfinite(mx)) a = 0.0;
  hdr->root64[0] = a;
  hdr->root64[1] = isfinite(mx) ? mx : 0.0;
  hdr->root64[2] = yr + mdy;
}

// FP64 routing used in training: leaf = clamp(floor(L * (a (x - c) + b))).
__device__ __forceinline__ int leaf64(const double* r, int L, double x) {
  const double lin = (r[0] == 0.0) ? r[2] : __fma_rn(r[0], __dsub_rn(x, r[1]), r[2]);
  const double w = __dmul_rn((double)L, lin);
  if (!(w >= 0.0)) return 0;
  if (w >= (double)L) return L - 1;
  return (int)floor(w);
}

// Leaf ranges of the sorted sample.  The root's leaf is non-decreasing in the
// key (slope >= 0), so leaf l holds the keys from the first with leaf >= l to
// the first with leaf >= l + 1: one warp per leaf finds both by a 32-way
// search (each step probes 32 evenly spaced keys of the remaining range), in
// about log_33(s) dependent steps instead of a pass over every key.  Empty
// leaves keep [0, 0).
constexpr int RT_THREADS = 256;

template <int DT>
__device__ __forceinline__ uint64_t leaf_lower_bound(const uint64_t* tk, uint64_t lo, uint64_t m,
                                                     const double* r, int L, int t) {
  const int lane = threadIdx.x & 31;
  uint64_t a = 0, b = m;  // the answer lies in [a, b]
  while (b - a > 32) {
    const uint64_t p = a + ((b - a) * (uint64_t)(lane + 1)) / 33;
    const bool ge = leaf64(r, L, sample_x<DT>(tk, lo, p)) >= t;
    const unsigned bal = __ballot_sync(0xffffffffu, ge);
    const int f = bal ? __ffs(bal) - 1 : 32;
    const uint64_t pf = __shfl_sync(0xffffffffu, p, f & 31);
    const uint64_t pp = __shfl_sync(0xffffffffu, p, (f + 31) & 31);
    const uint64_t na = f == 0 ? a : pp + 1;
    const uint64_t nb = f == 32 ? b : pf;
    a = na;
    b = nb;
  }
  const uint64_t q = a + lane;
  const bool ge = q < b && leaf64(r, L, sample_x<DT>(tk, lo, q)) >= t;
  const unsigned bal = __ballot_sync(0xffffffffu, ge);
  return bal ? a + (uint64_t)(__ffs(bal) - 1) : b;
}

template <int DT>
__global__ void __launch_bounds__(RT_THREADS)
k_fit_route(const uint64_t* __restrict__ tk, const DevModel* hdr, int L, uint32_t* leaf_beg,
            uint32_t* leaf_end) {
  pdl_begin();
  const int l = (int)((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5);
  if (l >= L) return;  // whole warps
  const uint64_t m = hdr->s_fin, lo = hdr->s_lo;
  const double r[3] = {hdr->root64[0], hdr->root64[1], hdr->root64[2]};
  const uint64_t b = leaf_lower_bound<DT>(tk, lo, m, r, L, l);
  const uint64_t e = leaf_lower_bound<DT>(tk, lo, m, r, L, l + 1);
  if ((threadIdx.x & 31) == 0 && b < e) {
    leaf_beg[l] = (uint32_t)b;
    leaf_end[l] = (uint32_t)e;
  }
}

// Per-leaf least squares in deterministic work units.  Leaf l's points
// [beg, end) are cut into units of FIT_UNIT points; each unit sums, shifted by
// the leaf's first point (x_r, y_r), dx, dy, dx*dx, dx*dy; the leaf then adds
// its units in order.  Shifting by a point of the leaf keeps the one-pass
// formulas Sxx = sum dx^2 - (sum dx)^2 / n stable.
constexpr int FIT_UNIT = 2048;

__global__ void __launch_bounds__(1024)
k_fit_units_plan(const uint32_t* leaf_beg, const uint32_t* leaf_end, int L, uint32_t* ubase,
                 uint32_t* utotal, uint32_t ucap, uint32_t* err) {
  pdl_begin();
  // (ubase clamped to the unit buffer's ucap entries: leaf ranges that overlap,
  // which only an unsorted sample could give, flag an error instead of
  // writing past the buffer)
  __shared__ uint32_t ws[33];
  __shared__ uint32_t s_run;
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  for (int l0 = 0; l0 < L; l0 += blockDim.x) {
    const int l = l0 + threadIdx.x;
    uint32_t u = 0;
    if (l < L && leaf_end[l] > leaf_beg[l]) u = (leaf_end[l] - leaf_beg[l] + FIT_UNIT - 1) / FIT_UNIT;
    uint32_t tot;
    const uint32_t ex = block_excl_sum<uint32_t>(u, ws, &tot);
    if (l < L) ubase[l] = min(s_run + ex, ucap);
    __syncthreads();
    if (threadIdx.x == 0) s_run += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (s_run > ucap) set_error(err, ERR_BOUNDS);
    ubase[L] = min(s_run, ucap);
    *utotal = min(s_run, ucap);
  }
}

template <int DT>
__global__ void __launch_bounds__(FIT_THREADS)
k_fit_unit_sums(const uint64_t* __restrict__ tk, const uint32_t* __restrict__ rank,
                const DevModel* hdr, const uint32_t* leaf_beg, const uint32_t* leaf_end,
                const uint32_t* ubase, int L, const uint32_t* utotal, double* unit) {
  pdl_begin();
  __shared__ double ws[33];
  const uint64_t m = hdr->s_fin, lo = hdr->s_lo;
  const double inv_m = m ? 1.0 / (double)m : 0.0;
  const uint32_t U = *utotal;
  for (uint32_t u = blockIdx.x; u < U; u += gridDim.x) {
    int a = 0, b = L - 1;  // leaf: last l with ubase[l] <= u and a unit of its own
    while (a < b) { const int mid = (a + b + 1) >> 1; if (ubase[mid] <= u) a = mid; else b = mid - 1; }
    const int l = a;
    const uint64_t first = leaf_beg[l];
    const uint64_t kb = first + (uint64_t)(u - ubase[l]) * FIT_UNIT;
    const uint64_t ke = min((uint64_t)leaf_end[l], kb + FIT_UNIT);
    const double xr = sample_x<DT>(tk, lo, first), yr = (double)rank[first] * inv_m;
    double s[4] = {0, 0, 0, 0};
    fit_accumulate<DT>(tk, rank, lo, kb + threadIdx.x, ke, blockDim.x, xr, yr, inv_m, s);
    for (int i = 0; i < 4; ++i) {
      const double t = block_sum_d(s[i], ws);
      if (threadIdx.x == 0) unit[4 * (size_t)u + i] = t;
    }
  }
}

template <int DT>
__global__ void k_fit_leaf_final(const uint64_t* __restrict__ tk, const uint32_t* __restrict__ rank,
                                 const DevModel* hdr, const uint32_t* leaf_beg,
                                 const uint32_t* leaf_end, const uint32_t* ubase,
                                 const double* unit, int L, double* leaf) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int l = (int)((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5);  // one warp per leaf
  if (l >= L) return;
  double* q = leaf + 5 * (size_t)l;
  const uint64_t b = leaf_beg[l], e = leaf_end[l];
  if (e <= b) {
    if (lane == 0) { q[0] = 0; q[1] = 0; q[2] = -1; q[3] = -1; q[4] = 0; }
    return;
  }
  // units of the leaf summed in a fixed order: lane-strided, then a fixed tree
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (uint32_t u = ubase[l] + lane; u < ubase[l + 1]; u += 32) {
    s0 += unit[4 * (size_t)u]; s1 += unit[4 * (size_t)u + 1];
    s2 += unit[4 * (size_t)u + 2]; s3 += unit[4 * (size_t)u + 3];
  }
  s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2); s3 = warp_sum(s3);
  if (lane) return;
  const uint64_t m = hdr->s_fin, lo = hdr->s_lo;
  const double inv_m = 1.0 / (double)m;
  const double cnt = (double)(e - b);
  const double xr = sample_x<DT>(tk, lo, b), yr = (double)rank[b] * inv_m;
  const double mdx = s0 / cnt, mdy = s1 / cnt;
  const double sxx = s2 - s0 * mdx, sxy = s3 - s0 * mdy;
  double a = (e - b >= 2 && sxx > 0) ? sxy / sxx : 0.0;
  const double mx = xr + mdx;
  if (!(a >= 0) || !isfinite(a) || !isfinite(mx)) a = 0.0;
  q[0] = a;
  q[1] = isfinite(mx) ? mx : 0.0;
  q[2] = yr + mdy;
  q[3] = (double)rank[b] / (double)m;  // lo: eCDF of the leaf's first sample key
  q[4] = 0;
}

__device__ __forceinline__ float fp32_sat(double d) {  // round to FP32, finite
  if (d >= (double)FLT_MAX) return FLT_MAX;
  if (d <= -(double)FLT_MAX) return -FLT_MAX;
  return __double2float_rn(d);
}



// Empty leaves, hi bounds (hi_l = lo_{l+1}), and the FP32 records of the cell
// index (the RMI rewritten on x: L root(x) = L a x + L (b - a c); leaf
// F = clamp(a x + (b - a c), lo, hi)).
template <int DT>
__global__ void __launch_bounds__(1024)
k_fit_final(DevModel* hdr, int L, double* leaf, CellLeaf* cleaf) {
  pdl_begin();
  // the leaves' lo bounds staged in shared memory, so that the right-to-left
  // pass runs on shared loads rather than a chain of global round trips
  __shared__ double slo[MAX_LEAVES];
  __shared__ unsigned char emp[MAX_LEAVES];
  L = min(L, MAX_LEAVES);
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    slo[l] = leaf[5 * (size_t)l + 3];
    emp[l] = 0;
  }
  __syncthreads();
  // an empty leaf (lo < 0) takes the lo of the next non-empty leaf to its
  // right (1 past the last); one warp over L/32-leaf ranges
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int per = (L + 31) / 32;
    const int a = lane * per, b = min(L, a + per);
    int first = L;
    for (int l = b - 1; l >= a; --l)
      if (slo[l] >= 0) first = l;
    int suf = first;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_down_sync(0xffffffffu, suf, o);
      if (lane + o < 32) suf = min(suf, v);
    }
    int nxt = __shfl_down_sync(0xffffffffu, suf, 1);
    if (lane == 31) nxt = L;
    double next_lo = (nxt < L) ? slo[nxt] : 1.0;
    for (int l = b - 1; l >= a; --l) {
      if (slo[l] < 0) { slo[l] = next_lo; emp[l] = 1; }
      next_lo = slo[l];
    }
    if (lane == 0) {
      const double* r = hdr->root64;
      CellRoot cr;
      cr.A0 = fp32_sat(__dmul_rn((double)L, r[0]));
      cr.B0 = fp32_sat(__dmul_rn((double)L, __dsub_rn(r[2], __dmul_rn(r[0], r[1]))));
      cr.L = L;
      cr.pad = 0;
      hdr->croot = cr;
    }
  }
  __syncthreads();
  // hi_l = lo_{l+1} (1 for the last leaf); an empty leaf is the constant lo
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    double* q = leaf + 5 * (size_t)l;
    const double lo = slo[l], hi = l + 1 < L ? slo[l + 1] : 1.0;
    double A, c, B;
    if (emp[l]) {
      A = 0; c = 0; B = lo;
      q[0] = A; q[1] = c; q[2] = B;
    } else {
      A = q[0]; c = q[1]; B = q[2];
    }
    q[3] = lo;
    q[4] = hi;
    CellLeaf cl;
    cl.A = fp32_sat(A);
    cl.B = fp32_sat(__dsub_rn(B, __dmul_rn(A, c)));
    cl.LO = __double2float_rn(lo);
    cl.HI = __double2float_rn(hi);
    cleaf[l] = cl;
  }
}

// ---------------------------------------------------------------- level-0 thresholds
// The model in FP64, operation for operation: lin = a == 0 ? b : fma(a, x - c, b);
// leaf = clamp(floor(L * lin_root)); F = clamp(lin_leaf, lo, hi) (Sec. 2, Alg. 1).
__device__ __forceinline__ double lin64(double a, double x, double c, double b) {
  return a == 0.0 ? b : __fma_rn(a, __dsub_rn(x, c), b);
}
__device__ __forceinline__ double predict64(const double* r, const double* leaf, int L, double x) {
  const double w = __dmul_rn((double)L, lin64(r[0], x, r[1], r[2]));
  const int l = !(w >= 0.0) ? 0 : (w >= (double)L ? L - 1 : (int)floor(w));
  const double* q = leaf + 5 * (size_t)l;
  const double v = lin64(q[0], x, q[1], q[2]);
  if (!(v >= q[3])) return q[3];
  return v > q[4] ? q[4] : v;
}
// pos(t) = clamp(floor(F(x) * f0), 0, f0 - 1) for the key with total-order key t;
// NaNs take F = 0 / 1 by sign.
template <int DT>
__device__ __forceinline__ uint32_t pos64(uint64_t t, const double* r, const double* leaf, int L,
                                          uint32_t f0) {
  const typename KT<DT>::U u = KT<DT>::from_tk(t);
  double F;
  if (KT<DT>::is_nan(u)) F = KT<DT>::neg(u) ? 0.0 : 1.0;
  else F = predict64(r, leaf, L, KT<DT>::dbl(u));
  const double w = __dmul_rn(F, (double)f0);
  if (!(w >= 0.0)) return 0u;
  if (w >= (double)f0) return f0 - 1;
  return (uint32_t)floor(w);
}
template <int DT> struct TkRange {
  static constexpr uint64_t MAX = KT<DT>::W == 8 ? ~0ull : 0xFFFFFFFFull;
  static constexpr uint64_t NEVER = KT<DT>::W == 8 ? ~0ull : 0x100000000ull;
};

// Smallest t in [lo, hi] with pred(t), for a predicate non-decreasing in t
// with pred(hi) true, by one warp: each round the 32 lanes test 31 evenly
// spaced points and the interval shrinks to the gap holding the first true
// one (64-bit ranges take 13 rounds instead of 64 bisection steps).
template <typename Pred>
__device__ __forceinline__ uint64_t warp_first_true(uint64_t lo, uint64_t hi, Pred pred) {
  const int lane = threadIdx.x & 31;
  while (hi - lo >= 32) {
    const uint64_t step = (hi - lo) >> 5;
    const uint64_t p = lane < 31 ? lo + (uint64_t)(lane + 1) * step : hi;
    const unsigned bal = __ballot_sync(0xffffffffu, lane == 31 || pred(p));
    const int f = __ffs(bal) - 1;
    const uint64_t pf = __shfl_sync(0xffffffffu, p, f);
    const uint64_t pb = __shfl_sync(0xffffffffu, p, f > 0 ? f - 1 : 0);
    lo = f > 0 ? pb + 1 : lo;
    hi = pf;
  }
  const uint64_t p = lo + (uint64_t)lane;
  const unsigned bal = __ballot_sync(0xffffffffu, p >= hi || pred(p));
  return lo + (uint64_t)(__ffs(bal) - 1);
}

// thr[b] = min { t : pos(t) >= b } over the whole total order (pos is
// non-decreasing in t), one warp per bucket; warp f0 records the bucket of the
// largest key.
template <int DT>
__global__ void __launch_bounds__(128)
k_thresholds(DevModel* hdr, const double* __restrict__ leaf, int L, uint32_t f0, uint64_t* thr) {
  pdl_begin();
  const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b > f0) return;
  const double r[3] = {hdr->root64[0], hdr->root64[1], hdr->root64[2]};
  const uint64_t TMAX = TkRange<DT>::MAX;
  if (b == f0) {
    if (lane == 0) {
      hdr->pos_max = pos64<DT>(TMAX, r, leaf, L, f0);
      hdr->cell_span = 0;
    }
    return;
  }
  if (b == 0) { if (lane == 0) thr[0] = 0; return; }
  if (pos64<DT>(TMAX, r, leaf, L, f0) < b) { if (lane == 0) thr[b] = TkRange<DT>::NEVER; return; }
  const uint64_t t = warp_first_true(0ull, TMAX, [&](uint64_t x) { return pos64<DT>(x, r, leaf, L, f0) >= b; });
  if (lane == 0) thr[b] = t;
}

// #{ b in [1, f0) : thr[b] <= t }
__device__ __forceinline__ uint32_t thr_count(const uint64_t* thr, uint32_t f0, uint64_t t) {
  uint32_t lo = 1, hi = f0;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (thr[mid] <= t) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// Smallest total-order key whose cell is >= c (NEVER if there is none), by
// one warp.
template <int DT>
__device__ __forceinline__ uint64_t cell_start(uint32_t c, const CellRoot& cr,
                                               const CellLeaf* cleaf) {
  const uint64_t TMAX = TkRange<DT>::MAX;
  if (cell_of<DT>(KT<DT>::from_tk(TMAX), cr, cleaf) < c) return TkRange<DT>::NEVER;
  return warp_first_true(0ull, TMAX,
                         [&](uint64_t x) { return cell_of<DT>(KT<DT>::from_tk(x), cr, cleaf) >= c; });
}

// Cell table: for cell c, the bucket range [count(first key), count(last key)]
// of the keys whose cell is c (the cell map is non-decreasing in the key); one
// warp per cell.
template <int DT>
__global__ void k_cell_table(DevModel* hdr, const uint64_t* __restrict__ thr, uint32_t f0,
                             const CellLeaf* __restrict__ cleaf, uint32_t* cell) {
  pdl_begin();
  const uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= L0_CELLS) return;
  const uint64_t TMAX = TkRange<DT>::MAX, NEVER = TkRange<DT>::NEVER;
  const CellRoot cr = hdr->croot;
  const uint64_t a = c ? cell_start<DT>(c, cr, cleaf) : 0ull;
  const uint64_t e = c + 1 < L0_CELLS ? cell_start<DT>(c + 1, cr, cleaf) : NEVER;
  if ((threadIdx.x & 31) != 0) return;
  uint32_t lo, hi;
  if (a == NEVER || a > TMAX) {          // no key maps here
    lo = hi = thr_count(thr, f0, TMAX);
  } else {
    lo = thr_count(thr, f0, a);
    hi = (e == NEVER || e > TMAX) ? thr_count(thr, f0, TMAX) : (e > a ? thr_count(thr, f0, e - 1) : lo);
  }
  cell[c] = lo | (hi << 16);
  atomicMax(&hdr->cell_span, hi - lo);
}

// ---------------------------------------------------------------- heavy set
template <int DT>
__global__ void k_heavy_flags(const uint64_t* __restrict__ tk, const DevModel* hdr, uint64_t tau,
                              uint32_t* __restrict__ flags, uint64_t s_cap) {
  pdl_begin();
  const uint64_t m = hdr->s_fin, lo = hdr->s_lo;
  const uint64_t* t = tk + lo;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < s_cap;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t f = 0;
    if (k < m && tau >= 1 && k + tau - 1 < m) {
      const uint64_t v = t[k];
      if ((k == 0 || t[k - 1] != v) && t[k + tau - 1] == v) f = 1;
    }
    flags[k] = f;
  }
}

struct Cand {
  uint64_t tk;
  uint64_t len;
  uint32_t bucket;
  uint32_t pad;
};

template <int DT>
__global__ void k_heavy_compact(const uint64_t* __restrict__ tk, const DevModel* hdr,
                                const uint32_t* __restrict__ flags, const uint64_t* __restrict__ pos,
                                const uint64_t* __restrict__ thr, const uint32_t* __restrict__ cell,
                                const CellLeaf* __restrict__ cleaf, Cand* cand, uint64_t cand_cap) {
  pdl_begin();
  const uint64_t m = hdr->s_fin, lo = hdr->s_lo;
  const uint64_t* t = tk + lo;
  const L0Map q{thr, cell, cleaf, hdr->croot, hdr->pos_max, 0};
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (!flags[k]) continue;
    const uint64_t v = t[k];
    uint64_t a = k, b = m;  // upper_bound of v in [k, m)
    while (a < b) {
      const uint64_t mid = (a + b) >> 1;
      if (t[mid] <= v) a = mid + 1; else b = mid;
    }
    const uint64_t p = pos[k];
    if (p < cand_cap) {
      Cand c;
      c.tk = v;
      c.len = a - k;
      c.bucket = l0_bucket<DT>(KT<DT>::from_tk(v), q);
      c.pad = 0;
      cand[p] = c;
    }
  }
}

// One CTA per bucket: keep the hpb longest runs (ties: smaller key), listed
// by key.  A candidate's place is the number of the bucket's candidates that
// beat it (candidates are distinct values, so places are distinct); a bucket
// with more candidates than the shared copy holds takes one thread's insertion
// pass instead.
constexpr int SEL_THREADS = 256;
constexpr int SEL_CAP = 1024;

__global__ void __launch_bounds__(SEL_THREADS)
k_heavy_select(const Cand* __restrict__ cand, const uint64_t* ncand_ptr, uint64_t cand_cap,
               uint32_t f0, int hpb, uint64_t* sel, uint32_t* sellen, uint32_t* nh, DevModel* hdr) {
  pdl_begin();
  __shared__ uint64_t s_tk[SEL_CAP], s_len[SEL_CAP];
  __shared__ uint64_t s_top[MAX_HPB], s_toplen[MAX_HPB];  // the selected, by place
  __shared__ uint64_t s_ab[2];
  const uint32_t b = blockIdx.x;
  if (b >= f0) return;
  if (threadIdx.x < 2) {  // lower bounds of buckets b and b + 1 (candidates are in key order)
    const uint64_t nc = min(*ncand_ptr, cand_cap);
    const uint32_t bb = b + threadIdx.x;
    uint64_t lo = 0, hi = nc;
    while (lo < hi) { const uint64_t mid = (lo + hi) >> 1; if (cand[mid].bucket < bb) lo = mid + 1; else hi = mid; }
    s_ab[threadIdx.x] = lo;
  }
  __syncthreads();
  const uint64_t a = s_ab[0], k = s_ab[1] - a;
  const uint32_t cnt = (uint32_t)min(k, (uint64_t)hpb);
  if (k <= (uint64_t)SEL_CAP) {
    for (uint32_t i = threadIdx.x; i < k; i += SEL_THREADS) {
      s_tk[i] = cand[a + i].tk;
      s_len[i] = cand[a + i].len;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < k; i += SEL_THREADS) {
      const uint64_t t = s_tk[i], len = s_len[i];
      uint32_t place = 0;
      for (uint32_t j = 0; j < k; ++j)
        place += (s_len[j] > len || (s_len[j] == len && s_tk[j] < t)) ? 1u : 0u;
      if (place < cnt) { s_top[place] = t; s_toplen[place] = len; }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {  // key order among the selected
      const uint64_t t = s_top[threadIdx.x];
      uint32_t kr = 0;
      for (uint32_t q = 0; q < cnt; ++q) kr += s_top[q] < t ? 1u : 0u;
      sel[(size_t)b * hpb + kr] = t;
      sellen[(size_t)b * hpb + kr] = (uint32_t)min(s_toplen[threadIdx.x], (uint64_t)0xFFFFFFFFu);
    }
    if (threadIdx.x == 0) {
      unsigned long long len = 0;
      for (uint32_t q = 0; q < cnt; ++q) len += s_toplen[q];
      if (len) atomicAdd(&hdr->heavy_len, len);
      nh[b] = cnt;
    }
    return;
  }
  if (threadIdx.x != 0) return;
  uint64_t ktk[MAX_HPB], klen[MAX_HPB];
  int c = 0;
  for (uint64_t i = a; i < a + k; ++i) {
    const uint64_t t = cand[i].tk, len = cand[i].len;
    // insert into the top list ordered by (len desc, tk asc)
    int p = c;
    while (p > 0 && (klen[p - 1] < len || (klen[p - 1] == len && ktk[p - 1] > t))) --p;
    if (p >= hpb) continue;
    const int last = min(c, hpb - 1);
    for (int q = last; q > p; --q) { ktk[q] = ktk[q - 1]; klen[q] = klen[q - 1]; }
    ktk[p] = t; klen[p] = len;
    if (c < hpb) ++c;
  }
  unsigned long long len = 0;
  for (int i = 0; i < c; ++i) len += klen[i];
  if (len) atomicAdd(&hdr->heavy_len, len);
  for (int i = 1; i < c; ++i) {  // order by key, lengths alongside
    const uint64_t t = ktk[i], l = klen[i];
    int j = i;
    while (j > 0 && ktk[j - 1] > t) { ktk[j] = ktk[j - 1]; klen[j] = klen[j - 1]; --j; }
    ktk[j] = t;
    klen[j] = l;
  }
  for (int i = 0; i < c; ++i) {
    sel[(size_t)b * hpb + i] = ktk[i];
    sellen[(size_t)b * hpb + i] = (uint32_t)min(klen[i], (uint64_t)0xFFFFFFFFu);
  }
  nh[b] = (uint32_t)c;
}

template <int DT>
__global__ void __launch_bounds__(1024)
k_heavy_heads(const uint64_t* __restrict__ sel, const uint32_t* __restrict__ sellen,
              const uint32_t* __restrict__ nh, uint32_t f0, int hpb, DevModel* hdr,
              const CellLeaf* __restrict__ cleaf, BucketHead* heads, HeavyEntry* heavy,
              uint32_t* hlen) {
  pdl_begin();
  __shared__ uint32_t ws[33];
  __shared__ uint32_t s_run;
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  const CellRoot cr = hdr->croot;
  for (uint32_t b0 = 0; b0 < f0; b0 += blockDim.x) {
    const uint32_t b = b0 + threadIdx.x;
    const uint32_t c = b < f0 ? nh[b] : 0;
    uint32_t tot;
    const uint32_t ex = block_excl_sum<uint32_t>(c, ws, &tot);
    const uint32_t hoff = s_run + ex;
    if (b < f0) {
      BucketHead h;
      h.ext_base = b + 2 * hoff;
      h.hoff_nh = (hoff << 4) | c;
      heads[b] = h;
      for (uint32_t j = 0; j < c; ++j) {
        HeavyEntry he;
        he.tk = sel[(size_t)b * hpb + j];
        he.F = cell_F<DT>(KT<DT>::from_tk(he.tk), cr, cleaf);
        he.ext = h.ext_base + 2 * j + 1;
        heavy[hoff + j] = he;
        hlen[hoff + j] = sellen[(size_t)b * hpb + j];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_run += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint32_t H = s_run;
    BucketHead h;
    h.ext_base = f0 + 2 * H;
    h.hoff_nh = H << 4;
    heads[f0] = h;
    hdr->nheavy = H;
    hdr->n_ext = f0 + 2 * H;
    // equality keys dominate (> 1/4 of the sample): compact the others in K2
    hdr->compact = (4 * hdr->heavy_len > hdr->s_fin) ? 1u : 0u;
  }
}

// Heavy table, one CTA: each slot keeps the value hashing to it with the
// longest run in the sorted sample (ties: the smaller key), whatever the thread
// order: the caller zeroes the table, the candidates race with a 64-bit max of
// (run << 32 | ~index), and the winners then replace their packed records.
// Slots left free get a key of another slot (0, or 1 in slot 0), so a probe
// needs no emptiness test (hash_probes = 1 marks the table as built).
template <int DT>
__global__ void __launch_bounds__(1024)
k_heavy_hash(DevModel* hdr, const HeavyEntry* __restrict__ heavy, const uint32_t* __restrict__ hlen,
             unsigned long long* hkey, uint16_t* hval) {
  pdl_begin();
  const uint32_t H = hdr->nheavy;
  if (2 * H > HASH_SIZE) return;  // too full to help
  // (the bit pattern 2^64-1 is left to the full lookup; a zero run never wins)
  for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) {
    const uint64_t b = (uint64_t)KT<DT>::from_tk(heavy[i].tk);
    if (b != HASH_EMPTY)
      atomicMax(&hkey[heavy_hash(b)], (unsigned long long)hlen[i] << 32 | (uint32_t)~i);
  }
  __syncthreads();
  for (uint32_t p = threadIdx.x; p < HASH_SIZE; p += blockDim.x) {
    const unsigned long long w = hkey[p];
    const uint32_t i = ~(uint32_t)w;
    if ((w >> 32) != 0 && i < H) {
      hkey[p] = (uint64_t)KT<DT>::from_tk(heavy[i].tk);
      hval[p] = (uint16_t)heavy[i].ext;
    } else {
      hkey[p] = p == 0 ? 1ull : 0ull;  // heavy_hash(0) = 0, heavy_hash(1) != 0
      hval[p] = 0xFFFFu;
    }
  }
  if (threadIdx.x == 0 && H > 0) hdr->hash_probes = 1;
}

// ---------------------------------------------------------------- host enqueue
template <int DT>
static cudaError_t train_dt(const void* keys_v, uint64_t n, const TrainPlan& P, const TrainWs& W,
                            const ModelPtrs& M, uint32_t* err, cudaStream_t st, int num_sms) {
  typedef typename KT<DT>::U U;
  const U* keys = (const U*)keys_v;
  const uint64_t s = P.s;
  const int L = (int)P.L;
  const int gs = (int)std::min<uint64_t>((s + 255) / 256, 8ull * num_sms);
  ZeroList z = P.zero;
  // the heavy table, the sample's scan words and the finite-range maximum are
  // cleared here too (three memsets fewer); the caller's regions come first
  int zi = 0;
  while (zi < ZERO_REGIONS && z.p[zi]) ++zi;
  auto add = [&](void* p, size_t bytes) {
    if (zi < ZERO_REGIONS) { z.p[zi] = p; z.words[zi] = (uint32_t)(bytes / 4); ++zi; return true; }
    return false;
  };
  const bool z_hkey = add(M.hkey, HASH_SIZE * sizeof(uint64_t));
  const bool z_scan = add(W.scan_status, W.scan_status_bytes);
  const bool z_hi = add(W.hi, sizeof(unsigned long long));
  // the LSD radix sort's digit histograms and look-back words
  const bool radix = sample_by_radix(KT<DT>::W, s);
  const bool z_rs = radix && add(W.rs.hist, 8 * 256 * sizeof(uint32_t)) &&
                    add(W.rs.status, (rs_status_words(s) + 8) * sizeof(uint32_t));
  launch_k(k_train_init, std::max(16, (L + 255) / 256), 256, 0, st, M.hdr, s, M.leaf_beg, M.leaf_end,
           L, W.partials, z, P.cs, P.stall, P.spin_limit);
  const uint64_t stride = std::max<uint64_t>(1, n / s);
  cudaError_t e = cudaSuccess;
  // the sample sort for large samples of 8-byte keys (its splitters drawn by
  // the sampling kernel), else the LSD radix sort (sample_by_radix)
  const size_t smem = radix ? 0 : (size_t)SS_CAND * sizeof(uint64_t);
  if (!radix && (e = cudaFuncSetAttribute(k_sample<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)))
    return e;
  const int sg = std::max(1, (int)std::min<uint64_t>((s + 1023) / 1024, 2ull * num_sms)) + (radix ? 0 : 1);
  launch_k(k_sample<DT>, sg, 1024, smem, st, keys, n, s, P.seed, make_div64(s), make_div64(stride),
           W.smp_a, radix ? nullptr : W.ss.spl, radix ? nullptr : W.ss.cnt);
  add_launches(1);
  e = radix ? rs_sort_enqueue(W.smp_a, W.smp_b, s, nullptr, nullptr, W.rs, err, st, num_sms, z_rs)
            : ss_sort_enqueue(W.smp_a, W.smp_b, s, W.ss, err, st, num_sms, /*splitters_done=*/true);
  if (e) return e;
  if (!z_hi && (e = cudaMemsetAsync(W.hi, 0, sizeof(unsigned long long), st))) return e;
  launch_k(k_finite_range<DT>, std::max(1, gs), 256, 0, st, W.smp_a, s, M.hdr, W.hi);
  launch_k(k_finite_fix, 1, 1, 0, st, M.hdr, W.hi);
  const int fr = (int)std::min<uint64_t>((s + FR_CHUNK - 1) / FR_CHUNK, 4ull * num_sms);
  launch_k(k_first_rank, std::max(1, fr), FR_THREADS, 0, st, W.smp_a, M.hdr, W.rank, s);
  launch_k(k_fit_sums<DT>, FIT_BLOCKS, FIT_THREADS, 0, st, W.smp_a, W.rank, M.hdr, W.partials);
  launch_k(k_fit_root<DT>, 1, 32, 0, st, M.hdr, W.smp_a, W.rank, W.partials, FIT_BLOCKS);
  launch_k(k_fit_route<DT>, (32 * L + RT_THREADS - 1) / RT_THREADS, RT_THREADS, 0, st, W.smp_a, M.hdr, L,
           M.leaf_beg, M.leaf_end);
  launch_k(k_fit_units_plan, 1, 1024, 0, st, M.leaf_beg, M.leaf_end, L, W.ubase, W.utotal,
                                       (uint32_t)(s / FIT_UNIT + L + 2), err);
  {
    const unsigned ub = (unsigned)std::min<uint64_t>(s / FIT_UNIT + L + 1, 16ull * num_sms);
    launch_k(k_fit_unit_sums<DT>, ub, FIT_THREADS, 0, st, W.smp_a, W.rank, M.hdr, M.leaf_beg,
                                                   M.leaf_end, W.ubase, L, W.utotal, W.units);
  }
  launch_k(k_fit_leaf_final<DT>, (32 * L + 255) / 256, 256, 0, st, W.smp_a, W.rank, M.hdr, M.leaf_beg,
                                                       M.leaf_end, W.ubase, W.units, L, M.leaf64);
  launch_k(k_fit_final<DT>, 1, 1024, 0, st, M.hdr, L, M.leaf64, M.cleaf);
  launch_k(k_thresholds<DT>, (32 * (P.f0 + 1) + 127) / 128, 128, 0, st, M.hdr, M.leaf64, L, P.f0, M.thr);
  launch_k(k_cell_table<DT>, (32 * L0_CELLS + 127) / 128, 128, 0, st, M.hdr, M.thr, P.f0, M.cleaf, M.cell);
  // heavy values
  const uint64_t tau = P.tau;
  launch_k(k_heavy_flags<DT>, std::max(1, gs), 256, 0, st, W.smp_a, M.hdr, tau, W.flags, s);
  if (!z_scan && (e = cudaMemsetAsync(W.scan_status, 0, W.scan_status_bytes, st))) return e;
  const unsigned sblocks = (unsigned)std::max<uint64_t>(1, (s + SC_TILE - 1) / SC_TILE);
  launch_k(k_scan<uint32_t>, sblocks, SC_THREADS, 0, st, W.flags, W.cpos, s, nullptr,
           (uint64_t*)W.scan_status, (uint32_t*)((uint64_t*)W.scan_status + sblocks), err, 0u);
  launch_k(k_heavy_compact<DT>, std::max(1, gs), 256, 0, st, W.smp_a, M.hdr, W.flags, W.cpos, M.thr,
                                                      M.cell, M.cleaf, (Cand*)W.cand, W.cand_cap);
  launch_k(k_heavy_select, P.f0, SEL_THREADS, 0, st, (const Cand*)W.cand, W.cpos + s, W.cand_cap,
                                                     P.f0, (int)P.hpb, W.sel, W.sellen, W.nh, M.hdr);
  launch_k(k_heavy_heads<DT>, 1, 1024, 0, st, W.sel, W.sellen, W.nh, P.f0, (int)P.hpb, M.hdr, M.cleaf,
                                        M.heads, M.heavy, W.hlen);
  if (!z_hkey && (e = cudaMemsetAsync(M.hkey, 0, HASH_SIZE * sizeof(uint64_t), st))) return e;
  launch_k(k_heavy_hash<DT>, 1, 1024, 0, st, M.hdr, M.heavy, W.hlen, (unsigned long long*)M.hkey, M.hval);
  add_launches(20);
  return cudaGetLastError();
}

cudaError_t train_enqueue(int dt, const void* keys, uint64_t n, const TrainPlan& P,
                          const TrainWs& W, const ModelPtrs& M, uint32_t* err, cudaStream_t st,
                          int num_sms) {
  switch (dt) {
    case LS_F64: return train_dt<LS_F64>(keys, n, P, W, M, err, st, num_sms);
    case LS_U64: return train_dt<LS_U64>(keys, n, P, W, M, err, st, num_sms);
    case LS_F32: return train_dt<LS_F32>(keys, n, P, W, M, err, st, num_sms);
    case LS_U32: return train_dt<LS_U32>(keys, n, P, W, M, err, st, num_sms);
  }
  return cudaErrorInvalidValue;
}

cudaError_t sample_sort_u64_enqueue(uint64_t* a, uint64_t* b, uint64_t m, const SsWork& w,
                                    uint32_t* err, cudaStream_t st, int num_sms) {
  return ss_sort_enqueue(a, b, m, w, err, st, num_sms);
}

cudaError_t radix_sort_u64_enqueue(uint64_t* a, uint64_t* b, uint64_t m, const RsWork& w,
                                   uint32_t* err, cudaStream_t st, int num_sms) {
  return rs_sort_enqueue(a, b, m, nullptr, nullptr, w, err, st, num_sms);
}

}  // namespace ls

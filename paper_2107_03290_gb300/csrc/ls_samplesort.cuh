// Sort of the training sample (Sec. 6.1 trains the model on a 1% sample,
// which must be in key order to give each sample key its eCDF rank), as a
// sample sort of 64-bit total-order keys:
//
//  1. an evenly spaced oversample of SS_CAND keys, sorted by one CTA, gives
//     SS_P splitters (every SS_OVER-th);
//  2. each key goes to a gap between splitters (bucket 2j: keys strictly
//     between splitter j-1 and splitter j) or to a splitter's own value
//     (bucket 2j+1: keys equal to splitter j, already in order);
//  3. per-bucket sizes, their exclusive scan, and a scatter whose per-tile
//     bucket ranges are reserved with one atomic per (tile, bucket);
//  4. each gap sorted in shared memory by a bitonic network; a gap larger
//     than SS_CAP keys (rare: the oversample bounds the gaps with high
//     probability) is sorted in SS_CAP chunks and merged in global memory.
//
// There is no look-back chain and only five launches.  Keys equal to a
// splitter never need a sort, so heavy repeats cost one pass.
#pragma once
#include "ls_scan.cuh"

namespace ls {

constexpr int SS_CAND = SS_P * SS_OVER;    // oversample, sorted by one CTA
constexpr int SS_THREADS = 512;
constexpr int SS_KPT = 8;
constexpr int SS_TILE = SS_THREADS * SS_KPT;
constexpr int SS_CAP = 4096;               // gap sorted in one CTA's shared memory

// Bucket of key t: 2 * #{splitters < t} + [t equals the next splitter].
__device__ __forceinline__ uint32_t ss_bucket(const uint64_t* spl, uint64_t t) {
  uint32_t lo = 0;
#pragma unroll
  for (uint32_t s = SS_P / 2; s; s >>= 1)
    if (spl[lo + s - 1] < t) lo += s;
  if (spl[lo] < t) lo += 1;  // lo = #{spl < t} in [0, SS_P]
  return 2 * lo + ((lo < (uint32_t)SS_P && spl[lo] == t) ? 1u : 0u);
}

// Bitonic stages j < 8 of level k over the 8 consecutive elements v[0..8) at
// position base (pairs never leave an aligned group of 8).
__device__ __forceinline__ void ss_bitonic_regs(uint64_t* v, uint32_t base, uint32_t k, uint32_t jmax) {
#pragma unroll
  for (uint32_t j = 4; j > 0; j >>= 1) {
    if (j > jmax) continue;
#pragma unroll
    for (uint32_t p = 0; p < 8; ++p) {
      if (p & j) continue;
      const bool up = ((base + p) & k) == 0;
      const uint64_t x = v[p], y = v[p + j];
      if ((x > y) == up) { v[p] = y; v[p + j] = x; }
    }
  }
}

// Ascending bitonic sort of n keys (n a power of two, 256 <= n <= 8 * blockDim.x)
// held 8 consecutive keys per thread by the first n / 8 threads of the block
// (thread t: positions 8t .. 8t+7).  Stages whose pairs stay inside a thread
// run in registers, those inside a warp (8 <= j < 256) exchange through
// shuffles, and only the stages across warps (j >= 256) go through shared
// memory `sh` (n words).  Every thread of the block calls it (barriers).
__device__ __forceinline__ void ss_sort_regs(uint64_t (&v)[8], uint64_t* sh, uint32_t n) {
  const uint32_t t = threadIdx.x;
  const bool act = t < (n >> 3);  // whole warps: n / 8 is a multiple of 32
  const uint32_t base = 8 * t;
  if (act)
    for (uint32_t k = 2; k <= 8; k <<= 1) ss_bitonic_regs(v, base, k, k >> 1);
  for (uint32_t k = 16; k <= n; k <<= 1) {
    if (k > 256) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (act) sh[base + q] = v[q];
      __syncthreads();
      for (uint32_t j = k >> 1; j >= 256; j >>= 1) {
        for (uint32_t i = t; i < n / 2; i += blockDim.x) {
          const uint32_t p = 2 * i - (i & (j - 1)), q = p + j;
          const bool up = (p & k) == 0;
          const uint64_t x = sh[p], y = sh[q];
          if ((x > y) == up) { sh[p] = y; sh[q] = x; }
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (act) v[q] = sh[base + q];
    }
    if (act) {
      const bool up = (base & k) == 0;  // the same for the thread's 8 keys (k >= 16)
      for (uint32_t j = min(k >> 1, 128u); j >= 8; j >>= 1) {
        const uint32_t d = j >> 3;  // partner lane
        const bool keep_min = ((t & d) == 0) == up;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint64_t o = __shfl_xor_sync(0xffffffffu, v[q], d);
          v[q] = keep_min ? min(v[q], o) : max(v[q], o);
        }
      }
      ss_bitonic_regs(v, base, k, 4);
    }
  }
}

// The oversample sorted by one CTA of 1024 threads, 8 consecutive keys per
// thread (ss_sort_regs).
static __global__ void __launch_bounds__(1024)
k_ss_splitters(const uint64_t* __restrict__ keys, uint64_t m, uint64_t* __restrict__ spl,
               uint32_t* __restrict__ cnt) {
  pdl_begin();
  extern __shared__ uint64_t ss_c[];
  static_assert(SS_CAND == 8 * 1024, "8 keys per thread");
  const uint32_t base = 8 * threadIdx.x;
  uint64_t v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = keys[(uint64_t)(base + q) * m / SS_CAND];
  for (uint32_t i = threadIdx.x; i <= SS_NB; i += blockDim.x) cnt[i] = 0;
  ss_sort_regs(v, ss_c, SS_CAND);
  // every SS_OVER-th key of the sorted oversample (SS_OVER divides 8)
#pragma unroll
  for (int q = SS_OVER - 1; q < 8; q += SS_OVER) spl[(base + q) / SS_OVER] = v[q];
}

static __global__ void __launch_bounds__(SS_THREADS)
k_ss_count(const uint64_t* __restrict__ keys, uint64_t m, const uint64_t* __restrict__ spl,
           uint32_t* __restrict__ cnt) {
  pdl_begin();
  __shared__ uint64_t s_spl[SS_P];
  __shared__ uint32_t h[SS_NB];
  for (uint32_t i = threadIdx.x; i < SS_P; i += blockDim.x) s_spl[i] = spl[i];
  for (uint32_t i = threadIdx.x; i < SS_NB; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[ss_bucket(s_spl, keys[i])], 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < SS_NB; i += blockDim.x)
    if (h[i]) atomicAdd(&cnt[i], h[i]);
}

// beg = exclusive scan of cnt (beg[SS_NB] = m), cur = beg.
static __global__ void __launch_bounds__(1024)
k_ss_scan(const uint32_t* __restrict__ cnt, uint32_t* __restrict__ beg, uint32_t* __restrict__ cur) {
  pdl_begin();
  __shared__ uint32_t a[SS_NB + 1];
  __shared__ uint32_t ws[33];
  for (uint32_t i = threadIdx.x; i < SS_NB; i += blockDim.x) a[i] = cnt[i];
  __syncthreads();
  const uint32_t tot = block_scan_array<uint32_t>(a, SS_NB, ws);
  for (uint32_t i = threadIdx.x; i < SS_NB; i += blockDim.x) { beg[i] = a[i]; cur[i] = a[i]; }
  if (threadIdx.x == 0) beg[SS_NB] = tot;
}

static __global__ void __launch_bounds__(SS_THREADS)
k_ss_scatter(const uint64_t* __restrict__ keys, uint64_t m, const uint64_t* __restrict__ spl,
             uint32_t* __restrict__ cur, uint64_t* __restrict__ out, uint32_t* err) {
  pdl_begin();
  __shared__ uint64_t s_spl[SS_P];
  __shared__ uint32_t lc[SS_NB];  // per tile: counts, then output bases
  for (uint32_t i = threadIdx.x; i < SS_P; i += blockDim.x) s_spl[i] = spl[i];
  for (uint32_t i = threadIdx.x; i < SS_NB; i += blockDim.x) lc[i] = 0;
  __syncthreads();
  const uint64_t tiles = (m + SS_TILE - 1) / SS_TILE;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    uint64_t x[SS_KPT];
    uint32_t bk[SS_KPT], rk[SS_KPT];
#pragma unroll
    for (int k = 0; k < SS_KPT; ++k) {
      const uint64_t i = t * SS_TILE + (uint64_t)k * SS_THREADS + threadIdx.x;
      bk[k] = 0xFFFFFFFFu;
      rk[k] = 0;
      if (i < m) {
        x[k] = keys[i];
        bk[k] = ss_bucket(s_spl, x[k]);
        rk[k] = atomicAdd(&lc[bk[k]], 1u);
      }
    }
    __syncthreads();
    {  // reserve the tile's range of every bucket: independent atomics, issued together
      constexpr int PER = (SS_NB + SS_THREADS - 1) / SS_THREADS;
      uint32_t base[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const uint32_t b = q * SS_THREADS + threadIdx.x;
        const uint32_t c = b < (uint32_t)SS_NB ? lc[b] : 0u;
        base[q] = c ? atomicAdd(&cur[b], c) : 0u;
      }
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const uint32_t b = q * SS_THREADS + threadIdx.x;
        if (b < (uint32_t)SS_NB) lc[b] = base[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SS_KPT; ++k) {
      if (bk[k] == 0xFFFFFFFFu) continue;
      const uint64_t p = (uint64_t)lc[bk[k]] + rk[k];
      if (p < m) out[p] = x[k]; else set_error(err, ERR_BOUNDS);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < SS_NB; b += blockDim.x) lc[b] = 0;
    __syncthreads();
  }
}

// Number of elements of A among the first k outputs of the stable merge of
// A[0..na) and B[0..nb) (A first on ties).
__device__ __forceinline__ uint32_t ss_merge_path(const uint64_t* A, uint32_t na, const uint64_t* B,
                                                  uint32_t nb, uint32_t k) {
  uint32_t lo = k > nb ? k - nb : 0, hi = k < na ? k : na;
  while (lo < hi) {
    const uint32_t i = (lo + hi) >> 1;
    if (A[i] <= B[k - i - 1]) lo = i + 1; else hi = i;
  }
  return lo;
}

// Loads up to SS_CAP keys into registers (8 per thread), pads with the
// largest key to a power of two of at least 256 (up to 8 keys: one thread),
// sorts, writes the first `len` back.  Needs blockDim.x >= SS_CAP / 8.
__device__ __forceinline__ void ss_sort_chunk(const uint64_t* src, uint64_t* dst, uint32_t len,
                                              uint64_t* a) {
  if (len <= 8) {  // one thread: the 8-key network in registers
    if (threadIdx.x == 0) {
      uint64_t v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = q < (int)len ? src[q] : ~0ull;
      for (uint32_t k = 2; k <= 8; k <<= 1) ss_bitonic_regs(v, 0, k, k >> 1);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < (int)len) dst[q] = v[q];
    }
    __syncthreads();
    return;
  }
  uint32_t n2 = 256;
  while (n2 < len) n2 <<= 1;
  const uint32_t base = 8 * threadIdx.x;
  uint64_t v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = base + q < len ? src[base + q] : ~0ull;
  ss_sort_regs(v, a, n2);
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (base + q < len) dst[base + q] = v[q];
  __syncthreads();  // the merge passes read what the other threads wrote
}

// One CTA per gap: sorted from `in` into `out`.  The CTAs past the buckets
// copy the splitter-value buckets, a tile of positions at a time, so that a
// heavily repeated value does not fall to a single CTA.  A gap over SS_CAP
// keys: sorted chunks, then merge passes that alternate between the bucket's
// ranges of `out` and `in`.
static __global__ void __launch_bounds__(SS_THREADS)
k_ss_bucket_sort(uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                 const uint32_t* __restrict__ beg) {
  pdl_begin();
  __shared__ uint64_t a[SS_CAP];
  const uint32_t b = blockIdx.x;
  if (b >= (uint32_t)SS_NB) {
    uint32_t* sb = (uint32_t*)a;  // bucket starts (SS_NB + 1 words fit in a[])
    for (uint32_t i = threadIdx.x; i <= (uint32_t)SS_NB; i += blockDim.x) sb[i] = beg[i];
    __syncthreads();
    const uint32_t m = sb[SS_NB];
    for (uint64_t p = (uint64_t)(b - SS_NB) * blockDim.x + threadIdx.x; p < m;
         p += (uint64_t)(gridDim.x - SS_NB) * blockDim.x) {
      uint32_t lo = 0, hi = SS_NB - 1;  // last bucket starting at or before p
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (sb[mid] <= p) lo = mid; else hi = mid - 1;
      }
      if (lo & 1u) out[p] = in[p];
    }
    return;
  }
  if (b & 1u) return;
  const uint32_t a0 = beg[b], len = beg[b + 1] - a0;
  if (len == 0) return;
  if (len == 1) { if (threadIdx.x == 0) out[a0] = in[a0]; return; }
  if (len <= (uint32_t)SS_CAP) {
    ss_sort_chunk(in + a0, out + a0, len, a);
    return;
  }
  for (uint32_t c0 = 0; c0 < len; c0 += SS_CAP)
    ss_sort_chunk(in + a0 + c0, out + a0 + c0, min((uint32_t)SS_CAP, len - c0), a);
  uint64_t* src = out + a0;
  uint64_t* dst = in + a0;
  for (uint32_t w = SS_CAP; w < len; w <<= 1) {
    for (uint32_t p0 = 0; p0 < len; p0 += 2 * w) {
      const uint32_t na = min(w, len - p0);
      const uint32_t nb = len - p0 > w ? min(w, len - p0 - w) : 0u;
      const uint64_t* A = src + p0;
      const uint64_t* B = A + na;
      const uint32_t tot = na + nb;
      const uint32_t per = (tot + blockDim.x - 1) / blockDim.x;
      const uint32_t k0 = min(tot, threadIdx.x * per), k1 = min(tot, k0 + per);
      uint32_t i = ss_merge_path(A, na, B, nb, k0), j = k0 - i;
      for (uint32_t k = k0; k < k1; ++k) {
        const bool ta = i < na && (j >= nb || A[i] <= B[j]);
        dst[p0 + k] = ta ? A[i++] : B[j++];
      }
    }
    __syncthreads();
    uint64_t* t = src; src = dst; dst = t;
  }
  if (src != out + a0)
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) out[a0 + i] = src[i];
}

// Sorts a[0..m) (m < 2^32) using b[0..m) as scratch; the result is in a.
// splitters_done: the splitters and the cleared counters are already in `w`
// (the training's sampling kernel draws them from the input keys).
inline cudaError_t ss_sort_enqueue(uint64_t* a, uint64_t* b, uint64_t m, const SsWork& w,
                                   uint32_t* err, cudaStream_t st, int num_sms,
                                   bool splitters_done = false) {
  if (m < 2) return cudaSuccess;
  const unsigned g = (unsigned)std::max<uint64_t>(
      1, std::min<uint64_t>((m + SS_TILE - 1) / SS_TILE, 2ull * num_sms));
  if (!splitters_done) {
    const size_t smem = (size_t)SS_CAND * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(k_ss_splitters,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    launch_k(k_ss_splitters, 1, 1024, smem, st, a, m, w.spl, w.cnt);
    add_launches(1);
  }
  launch_k(k_ss_count, g, SS_THREADS, 0, st, a, m, w.spl, w.cnt);
  launch_k(k_ss_scan, 1, 1024, 0, st, w.cnt, w.beg, w.cur);
  launch_k(k_ss_scatter, g, SS_THREADS, 0, st, a, m, w.spl, w.cur, b, err);
  launch_k(k_ss_bucket_sort, SS_NB + 2 * num_sms, SS_THREADS, 0, st, b, a, w.beg);
  add_launches(4);
  return cudaGetLastError();
}

}  // namespace ls

// LSD radix sort of 64-bit total-order keys (8-bit digits; a digit that every
// key shares is skipped).  Sorts the training sample of 4-byte keys (Sec. 6.1:
// the model is trained on a 1% sample, which must be in key order to give each
// sample key its eCDF rank; their total-order keys leave four high digits
// constant) and serves ls_radix_sort_u64.
//
// Tile ranking is stable: warp w owns a contiguous run of the tile and walks it
// in order, keeping a private digit histogram; warps are then combined in warp
// order.  Across tiles the multi-CTA pass uses a decoupled look-back per digit.
#pragma once
#include "ls_scan.cuh"

namespace ls {

constexpr int RS_THREADS = 512;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;                      // keys per lane per tile
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 4096
constexpr uint32_t RS_FLAG_AGG = 1u << 30;
constexpr uint32_t RS_FLAG_INC = 2u << 30;
constexpr uint32_t RS_VAL = (1u << 30) - 1;

struct RsShared {
  uint32_t whist[RS_WARPS][256];
  uint32_t tile_excl[256];
  uint32_t run[256];      // single-CTA mode: running digit offsets
  uint32_t s_tile;
};

// Rank one tile: keys[r] for element base + w*256 + r*32 + lane.  After the
// call whist[w][d] holds the warp-exclusive offset of digit d in the tile and
// lrank[r] the rank inside the warp; tile_cnt (thread d < 256) the digit total.
template <typename DigitFn>
__device__ __forceinline__ void rs_rank_tile(RsShared& sh, const uint64_t* key, const bool* valid,
                                             uint32_t* lrank, DigitFn digit_of,
                                             uint32_t* tile_cnt_out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&sh.whist[0][0])[i] = 0;
  __syncthreads();
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const uint32_t d = valid[r] ? digit_of(key[r]) : 0x100u;
    // lanes holding the same 9-bit value (8-bit digit + invalid flag), by ballots
    unsigned peers = 0xffffffffu;
#pragma unroll
    for (int bit = 0; bit < 9; ++bit) {
      const unsigned bal = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
      peers &= ((d >> bit) & 1u) ? bal : ~bal;
    }
    const int leader = __ffs(peers) - 1;
    const uint32_t basec = valid[r] ? sh.whist[w][d] : 0u;
    __syncwarp();
    if (valid[r] && lane == leader) sh.whist[w][d] = basec + __popc(peers);
    __syncwarp();
    lrank[r] = basec + __popc(peers & lt);
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    const int d = threadIdx.x;
    uint32_t run = 0;
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      const uint32_t t = sh.whist[ww][d];
      sh.whist[ww][d] = run;
      run += t;
    }
    *tile_cnt_out = run;
  }
}

// Histogram of all 8 digits over keys[0..m) (m read from *m_dev if given).
static __global__ void k_rs_hist(const uint64_t* __restrict__ keys, uint64_t m_cap,
                          const uint64_t* m_dev, const uint64_t* off_dev,
                          uint32_t* __restrict__ hist) {
  pdl_begin();
  __shared__ uint32_t h[8][256];
  const uint64_t m = m_dev ? *m_dev : m_cap;
  const uint64_t off = off_dev ? *off_dev : 0;
  for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[off + i];
#pragma unroll
    for (int d = 0; d < 8; ++d) atomicAdd(&h[d][(k >> (8 * d)) & 255], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

// Exclusive scan of each digit's histogram; skip[d] = 1 when one digit value
// holds every key (the pass would be the identity).
static __global__ void k_rs_digit_scan(uint32_t* hist, uint32_t* skip, uint64_t m_cap,
                                const uint64_t* m_dev) {
  pdl_begin();
  __shared__ uint32_t ws[33];
  const uint64_t m = m_dev ? *m_dev : m_cap;
  for (int d = 0; d < 8; ++d) {
    const uint32_t c = hist[d * 256 + threadIdx.x];
    uint32_t tot;
    const uint32_t ex = block_excl_sum<uint32_t>(c, ws, &tot);
    const int full = __syncthreads_or(c == (uint32_t)m);
    hist[d * 256 + threadIdx.x] = ex;
    if (threadIdx.x == 0) skip[d] = full ? 1u : 0u;
    __syncthreads();
  }
}

// One LSD pass over digit `d` (multi-CTA, one tile per CTA, dynamic tile ids,
// decoupled look-back across tiles per digit).  `status` (tiles*256 words) and
// `tile_ctr` must be zero.  If skip[d], the CTA copies its tile unchanged.
static __global__ void __launch_bounds__(RS_THREADS)
k_rs_pass(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t m_cap,
          const uint64_t* m_dev, const uint64_t* off_dev, int d,
          const uint32_t* __restrict__ digit_off, const uint32_t* skip, uint32_t* status,
          uint32_t* tile_ctr, uint32_t* err) {
  pdl_begin();
  __shared__ RsShared sh;
  const uint64_t m = m_dev ? *m_dev : m_cap;
  const uint64_t off = off_dev ? *off_dev : 0;
  in += off;
  out += off;
  if (threadIdx.x == 0) sh.s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint64_t tile = sh.s_tile;
  const uint64_t base = tile * RS_TILE;
  if (base >= m) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t key[RS_ROUNDS];
  bool valid[RS_ROUNDS];
  uint32_t lrank[RS_ROUNDS];
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const uint64_t i = base + (uint64_t)w * (32 * RS_ROUNDS) + r * 32 + lane;
    valid[r] = i < m;
    key[r] = valid[r] ? in[i] : 0;
  }
  if (skip[d]) {
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      const uint64_t i = base + (uint64_t)w * (32 * RS_ROUNDS) + r * 32 + lane;
      if (valid[r]) out[i] = key[r];
    }
    return;
  }
  const int shift = 8 * d;
  uint32_t tcnt = 0;
  rs_rank_tile(sh, key, valid, lrank, [shift](uint64_t k) { return (uint32_t)(k >> shift) & 255u; },
               &tcnt);
  if (threadIdx.x < 256) {
    const int dg = threadIdx.x;
    uint32_t excl = 0;
    if (tile == 0) {
      st_release_u32(&status[dg], RS_FLAG_INC | tcnt);
    } else {
      st_release_u32(&status[tile * 256 + dg], RS_FLAG_AGG | tcnt);
      long long j = (long long)tile - 1;
      unsigned long long spins = 0;
      const unsigned long long lim = spin_limit_of(err);
      while (j >= 0) {
        const uint32_t v = ld_acquire_u32(&status[j * 256 + dg]);
        const uint32_t f = v & ~RS_VAL;
        if (f == 0) {
          if (++spins > lim) { set_error(err, ERR_TIMEOUT); break; }
          continue;
        }
        excl += v & RS_VAL;
        if (f == RS_FLAG_INC) break;
        --j;
      }
      st_release_u32(&status[tile * 256 + dg], RS_FLAG_INC | ((excl + tcnt) & RS_VAL));
    }
    sh.tile_excl[dg] = excl + digit_off[d * 256 + dg];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    if (!valid[r]) continue;
    const uint32_t dg = (uint32_t)(key[r] >> shift) & 255u;
    const uint64_t pos = (uint64_t)sh.tile_excl[dg] + sh.whist[w][dg] + lrank[r];
    if (pos < m) out[pos] = key[r];
    else set_error(err, ERR_BOUNDS);
  }
}

inline size_t rs_status_words(uint64_t m_cap) {
  const uint64_t tiles = (m_cap + RS_TILE - 1) / RS_TILE;
  return 8 * (tiles ? tiles : 1) * 256;
}

// Enqueue the 8 passes.  Every pass runs (a skipped digit copies), so after 8
// passes the sorted keys are back in `a`.
// `zeroed`: the caller has already cleared w.hist (8 * 256 words) and w.status
// (rs_status_words(m_cap) + 8 words) in stream order (no memsets here then).
inline cudaError_t rs_sort_enqueue(uint64_t* a, uint64_t* b, uint64_t m_cap, const uint64_t* m_dev,
                                   const uint64_t* off_dev, const RsWork& w, uint32_t* err,
                                   cudaStream_t st, int num_sms, bool zeroed = false) {
  const uint64_t tiles = (m_cap + RS_TILE - 1) / RS_TILE;
  if (tiles == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (!zeroed) {
    e = cudaMemsetAsync(w.hist, 0, 8 * 256 * sizeof(uint32_t), st);
    if (e) return e;
    e = cudaMemsetAsync(w.status, 0, rs_status_words(m_cap) * sizeof(uint32_t) + 8 * sizeof(uint32_t), st);
    if (e) return e;
  }
  int hb = (int)((m_cap + 4095) / 4096);
  if (hb > 4 * num_sms) hb = 4 * num_sms;
  if (hb < 1) hb = 1;
  launch_k(k_rs_hist, hb, 512, 0, st, a, m_cap, m_dev, off_dev, w.hist);
  launch_k(k_rs_digit_scan, 1, 256, 0, st, w.hist, w.skip, m_cap, m_dev);
  for (int d = 0; d < 8; ++d) {
    const uint64_t* src = (d & 1) ? b : a;
    uint64_t* dst = (d & 1) ? a : b;
    launch_k(k_rs_pass, (unsigned)tiles, RS_THREADS, 0, st, src, dst, m_cap, m_dev, off_dev, d, w.hist,
                                                     w.skip, w.status + (size_t)d * tiles * 256,
                                                     w.ctr + d, err);
  }
  add_launches(10);
  return cudaGetLastError();
}

}  // namespace ls

// Block-level helpers and the device-wide decoupled look-back scan
// (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", NVIDIA TR 2016).  Used for the bucket offsets (the running
// totals and write heads of Alg. 1 / Alg. 2), the level-1 sub-bucket offsets
// and the heavy-candidate compaction.
#pragma once
#include "ls_internal.cuh"

namespace ls {

template <typename T>
__device__ __forceinline__ T warp_incl_sum(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += y;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exclusive block scan of one value per thread; `ws` holds >= 32 T in smem.
// Returns the exclusive prefix; *total gets the block sum.  Deterministic.
template <typename T>
__device__ __forceinline__ T block_excl_sum(T v, T* ws, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const T inc = warp_incl_sum(v);
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? ws[lane] : T(0);
    const T wi = warp_incl_sum(w);
    if (lane < nw) ws[lane] = wi - w;
    if (lane == nw - 1) ws[32] = wi;
  }
  __syncthreads();
  const T r = ws[wid] + inc - v;
  if (total) *total = ws[32];
  __syncthreads();
  return r;
}

// Exclusive scan, in place, of an smem array a[0..len) by the whole block.
// Returns the total.  ws: >= 33 T of smem scratch.
template <typename T>
__device__ __forceinline__ T block_scan_array(T* a, int len, T* ws) {
  const int per = (len + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per;
  T s = 0;
  for (int i = 0; i < per; ++i)
    if (b + i < len) s += a[b + i];
  T tot;
  T run = block_excl_sum<T>(s, ws, &tot);
  for (int i = 0; i < per; ++i)
    if (b + i < len) { const T t = a[b + i]; a[b + i] = run; run += t; }
  __syncthreads();
  return tot;
}

// ---------------------------------------------------------------- device-wide scan
constexpr int SC_THREADS = 256;
constexpr int SC_PER = 16;
constexpr int SC_TILE = SC_THREADS * SC_PER;
constexpr uint64_t SC_FLAG_AGG = 1ull << 62;
constexpr uint64_t SC_FLAG_INC = 2ull << 62;
constexpr uint64_t SC_VAL = (1ull << 62) - 1;

// out[i] = sum(in[0..i)), out[M] = sum(in[0..M)).  `status` holds one word per
// tile and `tile_ctr` one counter; both must be zero at launch.  `M` is read
// from *M_dev when M_dev != nullptr (device-known lengths); grid covers M_cap.
// `stall_mask`: the STALL_* bit that, when set in the call's status block,
// keeps tile 0 from publishing (test injection of a wait that runs out).
template <typename In>
__global__ void __launch_bounds__(SC_THREADS)
k_scan(const In* __restrict__ in, uint64_t* __restrict__ out, uint64_t M_cap,
       const unsigned long long* M_dev, uint64_t* status, uint32_t* tile_ctr, uint32_t* err,
       uint32_t stall_mask = 0u) {
  pdl_begin();
  __shared__ uint64_t ws[33];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_excl;
  const uint64_t M = M_dev ? (uint64_t)*M_dev : M_cap;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint64_t tile = s_tile;
  const uint64_t base = tile * SC_TILE;
  if (base >= M) {
    // Nothing to scan in this tile, but tile 0 of an empty input writes out[0].
    if (tile == 0 && threadIdx.x == 0) out[0] = 0;
    return;
  }
  const uint64_t b0 = base + (uint64_t)threadIdx.x * SC_PER;
  uint64_t v[SC_PER];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SC_PER; ++i) {
    v[i] = (b0 + i < M) ? (uint64_t)in[b0 + i] : 0;
    s += v[i];
  }
  uint64_t tot;
  const uint64_t texcl = block_excl_sum<uint64_t>(s, ws, &tot);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    uint64_t excl = 0;
    if (tile == 0) {
      const bool stalled = (stall_of(err) & stall_mask) != 0u;
      if (lane == 0 && !stalled) st_release_u64(&status[0], SC_FLAG_INC | (tot & SC_VAL));
    } else {
      if (lane == 0) st_release_u64(&status[tile], SC_FLAG_AGG | (tot & SC_VAL));
      long long win = (long long)tile - 1;
      unsigned long long spins = 0;
      const unsigned long long lim = spin_limit_of(err);
      while (true) {
        const long long idx = win - lane;
        const uint64_t w = (idx >= 0) ? ld_acquire_u64(&status[idx]) : SC_FLAG_INC;
        const uint64_t flag = w & ~SC_VAL;
        const unsigned inv = __ballot_sync(0xffffffffu, flag == 0);
        const unsigned inc = __ballot_sync(0xffffffffu, flag == SC_FLAG_INC);
        const int first_inc = inc ? __ffs(inc) - 1 : 32;
        const unsigned need = (first_inc >= 31) ? 0xffffffffu : ((2u << first_inc) - 1u);
        if (inv & need) {
          if (++spins > lim) {
            if (lane == 0) set_error(err, ERR_TIMEOUT);
            break;
          }
          continue;
        }
        uint64_t val = (lane <= first_inc) ? (w & SC_VAL) : 0;
        val = warp_sum(val);
        excl += val;
        if (first_inc < 32) break;
        win -= 32;
      }
      if (lane == 0) st_release_u64(&status[tile], SC_FLAG_INC | ((excl + tot) & SC_VAL));
    }
    if (lane == 0) s_excl = excl;
  }
  __syncthreads();
  uint64_t run = s_excl + texcl;
#pragma unroll
  for (int i = 0; i < SC_PER; ++i) {
    if (b0 + i < M) out[b0 + i] = run;
    run += v[i];
    if (b0 + i + 1 == M) out[M] = run;
  }
}

}  // namespace ls

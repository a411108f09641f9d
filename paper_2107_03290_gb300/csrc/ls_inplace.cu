// In-place variant of the partitioning (Sec. 4.2: partitioning in place with
// fragments flushed over already-read positions, then Defragment; Alg. 1).
//
// Level 0 splits the whole array with the grid:
//   k_ip_frag0     one CTA per piece of the array: every key gets its extended
//                  slot (counted; equality keys are only counted, never moved:
//                  their ranges are filled afterwards), and the key of a
//                  regular bucket goes to that bucket's fragment in shared
//                  memory; a full fragment (one 128-byte block) is written to
//                  the next block slot at the front of the piece, which the
//                  piece has already read.  Leftovers go to a small per-piece
//                  area (P x f0 blocks, independent of n).
//   k_scan         slot counts -> slot offsets (the level-0 layout).
//   k_ip_prep0     per bucket: its slot range; per piece and bucket: where its
//                  blocks go among the bucket's.
//   k_ip_inv0      the device Defragment, by known destinations: a block's
//   k_ip_chain0    destination is its bucket's first slot + the blocks of its
//   k_ip_cycle0    bucket in earlier pieces + its rank in its piece.  The inverse
//                  map (who goes where) is built, about one slot in 32 (chosen
//                  by a hash of the slot) is copied out to a small area, and
//                  from every free destination (a copied-out or empty slot) one
//                  thread pulls blocks backwards along the inverse map until it
//                  meets a copied-out source or a slot nobody needs; the few
//                  cycles with no copied-out slot are rotated by their smallest
//                  slot.  No pointer atomics and no waits.
//   k_ip_save0     the overhang of a bucket's last block into the next
//                  bucket's head is saved;
//   k_ip_gaps0     each bucket's head and tail get its leftovers and its
//                  overhang.
// Each level-0 bucket's non-equality keys then lie at the start of its range
// (the equality ranges after them are filled last), as the out-of-place level 0
// leaves them in compaction mode, so k_classify0 makes the same jobs.
// The refinement levels (k_ip_refine) and the radix fallback split each
// segment in place inside one CTA (ls_inplace.cuh).
#include "ls_inplace.cuh"
#include "ls_partition.cuh"
#include "ls_partition_dev.cuh"
#include "ls_scan.cuh"

namespace ls {

// ---------------------------------------------------------------- level 0
struct Ip0Layout {
  L0Layout lay;          // the level-0 lookup tables and slot counters
  uint32_t frag;         // f0 fragments of one block
  uint32_t u32;          // 6 x f0 u32: fill, tile count, first slot, flushed, keys, blocks
  uint32_t total;
};

static Ip0Layout ip0_layout(int W, uint32_t L, uint32_t f0, uint32_t next) {
  const uint32_t hmax = (next - f0) / 2;
  for (int shared_leaves = 1; shared_leaves >= 0; --shared_leaves) {
    Ip0Layout y{};
    y.lay = l0_layout_hist(W, L, f0, next, hmax, shared_leaves != 0, false);
    size_t o = (size_t)y.lay.bar + 16;
    o = (o + 127) / 128 * 128;
    y.frag = (uint32_t)o;
    o += (size_t)f0 * IP_BLOCK_BYTES;
    y.u32 = (uint32_t)o;
    o += (size_t)6 * f0 * 4 + 16;
    y.total = (uint32_t)o;
    if (o <= L0_SMEM_LIMIT || !shared_leaves) return y;
  }
  return Ip0Layout{};
}

size_t ip_level0_smem(int dt, uint32_t L, uint32_t f0, uint32_t n_ext_max) {
  return ip0_layout(key_width(dt), L, f0, n_ext_max).total;
}

template <int DT>
__global__ void __launch_bounds__(IP0_THREADS, 1)
k_ip_frag0(Level0Args a, InPlace0 ip, Ip0Layout y) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr uint32_t B = IpBlk<U>::B;
  constexpr uint32_t NT = IP0_THREADS;
  extern __shared__ __align__(128) unsigned char sm[];
  const L0Layout& lay = y.lay;
  BucketHead* heads = (BucketHead*)(sm + lay.heads);
  uint32_t* ecnt = (uint32_t*)(sm + lay.cnt);
  const uint64_t* htk = (const uint64_t*)(sm + lay.htk);
  U* frag = (U*)(sm + y.frag);
  const uint32_t f0 = a.f0;
  uint32_t* ffill = (uint32_t*)(sm + y.u32);
  uint32_t* tcnt = ffill + f0;
  uint32_t* slot0 = ffill + 2 * f0;
  uint32_t* nfull = ffill + 3 * f0;
  uint32_t* kcnt = ffill + 4 * f0;
  uint32_t* nbk = ffill + 5 * f0;
  uint32_t* nsl = ffill + 6 * f0;
  const uint32_t next = min(a.M.hdr->n_ext, a.n_ext_max);
  const uint32_t H = min(a.M.hdr->nheavy, (next - f0) / 2);
  const L0Map q = load_tables(a, sm, lay, H);
  const uint32_t tid = threadIdx.x;
  for (uint32_t e = tid; e < next; e += NT) ecnt[e] = 0;
  for (uint32_t c = tid; c < f0; c += NT) ffill[c] = tcnt[c] = nfull[c] = kcnt[c] = nbk[c] = 0;
  if (tid == 0) *nsl = 0;
  __syncthreads();
  const uint32_t p = blockIdx.x;
  const uint64_t n = a.c.n;
  const uint64_t pb = (uint64_t)p * ip.PL;
  const uint64_t m = pb < n ? min(ip.PL, n - pb) : 0;
  U* X = (U*)a.keys + pb;
  const bool heavy = H > 0;
  for (uint64_t t0 = 0; t0 < m; t0 += IP0_TILE) {
    U u[IP0_KPT];
    uint32_t s[IP0_KPT], rk[IP0_KPT];
#pragma unroll
    for (int k = 0; k < IP0_KPT; ++k) {
      const uint64_t i = t0 + (uint64_t)k * NT + tid;
      u[k] = i < m ? X[i] : (U)0;
    }
    // all keys classified before any counter is touched (the lookups overlap)
    uint32_t ev[IP0_KPT];
#pragma unroll
    for (int k = 0; k < IP0_KPT; ++k) {
      const uint64_t i = t0 + (uint64_t)k * NT + tid;
      uint32_t pk = PK_EQ;
      ev[k] = IP_NONE;
      if (i < m)
        ev[k] = heavy ? classify_key<DT>(u[k], q, heads, htk, lay.hs, a.f0kf, a.kf, &pk)
                      : classify_plain<DT>(u[k], q, a.f0kf, a.kf, &pk);
      s[k] = (i < m && pk != PK_EQ) ? (pk & PK_B_MASK) : IP_NONE;
    }
#pragma unroll
    for (int k = 0; k < IP0_KPT; ++k) {
      if (ev[k] == IP_NONE) continue;
      if (ev[k] < next) atomicAdd(&ecnt[ev[k]], 1u);
      else { set_error(a.err, ERR_BOUNDS); s[k] = IP_NONE; }
    }
#pragma unroll
    for (int k = 0; k < IP0_KPT; ++k) rk[k] = s[k] != IP_NONE ? atomicAdd(&tcnt[s[k]], 1u) : 0u;
    __syncthreads();
    for (uint32_t c = tid; c < f0; c += NT) {
      const uint32_t t = tcnt[c];
      if (t) {
        const uint32_t nf = (ffill[c] + t) / B;
        nfull[c] = nf;
        if (nf) slot0[c] = atomicAdd(nsl, nf);
        kcnt[c] += t;
        nbk[c] += nf;
      }
    }
    __syncthreads();
    for (uint32_t c = tid; c < f0; c += NT) {
      if (nfull[c] && ffill[c]) {
        U* dst = X + (uint64_t)slot0[c] * B;
        for (uint32_t r = 0; r < ffill[c]; ++r) dst[r] = frag[c * B + r];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < IP0_KPT; ++k) {
      if (s[k] == IP_NONE) continue;
      const uint32_t c = s[k];
      const uint32_t pos = ffill[c] + rk[k];
      const uint32_t full = nfull[c] * B;
      if (pos < full) {
        const uint32_t sl = slot0[c] + pos / B;
        X[(uint64_t)sl * B + pos % B] = u[k];
        if (pos % B == B - 1) {  // the block's last key: its bucket and rank in the piece
          ip.tags[pb / B + sl] = (uint16_t)c;
          ip.prank[pb / B + sl] = nbk[c] - nfull[c] + pos / B;
        }
      } else {
        frag[c * B + (pos - full)] = u[k];
      }
    }
    __syncthreads();
    for (uint32_t c = tid; c < f0; c += NT) {
      const uint32_t t = tcnt[c];
      if (t) {
        ffill[c] = ffill[c] + t - nfull[c] * B;
        tcnt[c] = 0;
        nfull[c] = 0;
      }
    }
    __syncthreads();
  }
  // leftovers, counts, the piece's flushed blocks and its slots' read flags
  U* lo = (U*)ip.lo_keys + (size_t)p * f0 * B;
  for (uint32_t i = tid; i < f0 * B; i += NT) {
    const uint32_t c = i / B, r = i % B;
    if (r < ffill[c]) lo[i] = frag[i];
  }
  for (uint32_t c = tid; c < f0; c += NT) {
    ip.lo_cnt[(size_t)p * f0 + c] = ffill[c];
    ip.pnb[(size_t)p * f0 + c] = nbk[c];
    if (kcnt[c]) atomicAdd(&ip.cntb[c], (unsigned long long)kcnt[c]);
    if (nbk[c]) atomicAdd(&ip.nbk[c], nbk[c]);
  }
  for (uint32_t e = tid; e < next; e += NT)
    if (ecnt[e]) atomicAdd(&a.hist[e], ecnt[e]);
  if (tid == 0) ip.pslots[p] = *nsl;
  const uint64_t s0 = pb / B, s1 = (pb + m + B - 1) / B;
  for (uint64_t k = s0 + tid; k < s1; k += NT) {
    ip.flags[k] = 0;
    ip.inv[k] = IP_NONE;
  }
}

// Slot range and pointers of every bucket: bucket b's non-equality keys take
// [s_b, s_b + cntb[b]), s_b the first position of its range; its blocks go to
// slots [ceil(s_b / B), ...); its read range runs to the next bucket's first
// slot (the last bucket's to the array's last slot).
template <int DT>
__global__ void k_ip_prep0(Level0Args a, InPlace0 ip) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr uint32_t B = IpBlk<U>::B;
  const uint32_t f0 = a.f0;
  const uint64_t nslots = (a.c.n + B - 1) / B;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < f0; b += gridDim.x * blockDim.x) {
    const uint64_t s = a.offs[a.M.heads[b].ext_base];
    const uint64_t s1 = b + 1 < f0 ? a.offs[a.M.heads[b + 1].ext_base] : a.c.n;
    const uint64_t d = (s + B - 1) / B;
    const uint64_t D = b + 1 < f0 ? (s1 + B - 1) / B : nslots;
    if (d + ip.nbk[b] > D || s + ip.cntb[b] > s1 || D >= 0xFFFFFFFFull) set_error(a.err, ERR_BOUNDS);
    ip.sst[b] = s;
    ip.dsl[b] = (uint32_t)d;
    ip.dend[b] = (uint32_t)D;
    uint32_t run = 0;  // the bucket's blocks in earlier pieces
    for (uint32_t p = 0; p < ip.P; ++p) {
      const uint32_t t = ip.pnb[(size_t)p * f0 + b];
      ip.pnb[(size_t)p * f0 + b] = run;
      run += t;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 3) ip.hcount[threadIdx.x] = 0u;
}

constexpr int IP0_PERM_THREADS = 256;

struct Ip0Geo {
  uint64_t nslots, spp, ks;
  bool partial;
  uint32_t f0;
};
template <typename U>
__device__ __forceinline__ Ip0Geo ip0_geo(const Level0Args& a, const InPlace0& ip) {
  constexpr uint32_t B = IpBlk<U>::B;
  Ip0Geo g;
  g.nslots = (a.c.n + B - 1) / B;
  g.spp = ip.PL / B;
  g.ks = a.c.n / B;
  g.partial = (a.c.n % B) != 0;
  g.f0 = a.f0;
  return g;
}
__device__ __forceinline__ bool ip0_full(const InPlace0& ip, const Ip0Geo& g, uint64_t k) {
  const uint64_t pc = k / g.spp;
  return (k - pc * g.spp) < (uint64_t)ip.pslots[pc];
}
__device__ __forceinline__ uint64_t ip0_dest(const InPlace0& ip, const Ip0Geo& g, uint64_t k) {
  const uint32_t c = min((uint32_t)ip.tags[k], g.f0 - 1);
  return (uint64_t)ip.dsl[c] + ip.pnb[(size_t)(k / g.spp) * g.f0 + c] + ip.prank[k];
}

// The inverse map, and the hole blocks copied out.
template <int DT>
__global__ void __launch_bounds__(IP0_PERM_THREADS) k_ip_inv0(Level0Args a, InPlace0 ip) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr uint32_t B = IpBlk<U>::B;
  if (call_failed(a.err)) return;
  const Ip0Geo g = ip0_geo<U>(a, ip);
  const U* keys = (const U*)a.keys;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.nslots;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (!ip0_full(ip, g, k)) continue;
    const uint32_t c = min((uint32_t)ip.tags[k], g.f0 - 1);
    const uint64_t d = ip0_dest(ip, g, k);
    if (d >= (uint64_t)ip.dend[c]) { set_error(a.err, ERR_BOUNDS); continue; }
    ip.inv[d] = (uint32_t)k;
    if (ip_hole(k)) {
      const uint32_t hp = atomicAdd(ip.hcount, 1u);
      if (hp >= ip.hcap) { set_error(a.err, ERR_BOUNDS); continue; }
      U H[B];
      blk_load<U>(H, keys + k * B);
      blk_store<U>((U*)ip.hscr + (size_t)hp * B, H);
      ip.prank[k] = hp;
    }
  }
}

// The free destinations (a hole, or a slot that held no block), listed.
template <int DT>
__global__ void __launch_bounds__(IP0_PERM_THREADS) k_ip_starts0(Level0Args a, InPlace0 ip) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  if (call_failed(a.err)) return;
  const Ip0Geo g = ip0_geo<U>(a, ip);
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j0 = blockIdx.x * (uint64_t)blockDim.x; j0 < g.nslots; j0 += stride) {
    const uint64_t j = j0 + threadIdx.x;
    const bool st = j < g.nslots && ip.inv[j] != IP_NONE && (!ip0_full(ip, g, j) || ip_hole(j));
    const unsigned m = __ballot_sync(0xffffffffu, st);
    uint32_t base = 0;
    if (lane == 0 && m) base = atomicAdd(&ip.hcount[1], (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (st) {
      const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
      if (pos < ip.scap) ip.starts[pos] = (uint32_t)j;
      else set_error(a.err, ERR_BOUNDS);
    }
  }
}

// From every free destination, pull blocks backwards along the inverse map:
// each destination is filled once, by the one chain that reaches it, right
// after that chain has read the block that was there.  Chains are taken from
// the start list through a counter (32 at a time per warp), so that no thread
// walks several long ones while others are idle.
template <int DT>
__global__ void __launch_bounds__(IP0_PERM_THREADS) k_ip_chain0(Level0Args a, InPlace0 ip) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr uint32_t B = IpBlk<U>::B;
  if (call_failed(a.err)) return;
  const Ip0Geo g = ip0_geo<U>(a, ip);
  U* keys = (U*)a.keys;
  const uint32_t ns = min(ip.hcount[1], ip.scap);
  const uint32_t lane = threadIdx.x & 31;
  while (true) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&ip.hcount[2], 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= ns) break;
    const uint32_t si = base + lane;
    if (si >= ns) continue;
    const uint64_t j = ip.starts[si];
    uint32_t k = ip.inv[j];
    uint64_t cur = j;
    for (uint64_t step = 0; step <= g.nslots; ++step) {
      U H[B];
      const bool hole = ip_hole(k);
      // the next source is read with this block: one round trip per step
      const uint32_t nxt = hole ? IP_NONE : ip.inv[k];
      if (hole) blk_load<U>(H, (const U*)ip.hscr + (size_t)ip.prank[k] * B);
      else blk_load<U>(H, keys + (uint64_t)k * B);
      blk_store<U>((g.partial && cur == g.ks) ? (U*)ip.ovf : keys + cur * B, H);
      ip.flags[k] = 1;
      if (hole || nxt == IP_NONE) break;  // a hole's slot starts a chain of its own
      cur = k;
      k = nxt;
    }
  }
}

// Blocks on cycles that hold no hole (short ones, in practice) are rotated by
// the cycle's smallest slot; a block already at its destination stays.
constexpr uint64_t IP0_CYCLE_LIMIT = 1ull << 20;
template <int DT>
__global__ void __launch_bounds__(IP0_PERM_THREADS) k_ip_cycle0(Level0Args a, InPlace0 ip) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr uint32_t B = IpBlk<U>::B;
  if (call_failed(a.err)) return;
  const Ip0Geo g = ip0_geo<U>(a, ip);
  U* keys = (U*)a.keys;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.nslots;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (!ip0_full(ip, g, k) || ip_hole(k) || ip.flags[k]) continue;
    uint64_t j = ip0_dest(ip, g, k);
    if (j == k) continue;
    uint64_t mn = k, steps = 0;
    while (j != k && steps < IP0_CYCLE_LIMIT) {
      mn = j < mn ? j : mn;
      j = ip0_dest(ip, g, j);
      ++steps;
    }
    if (steps >= IP0_CYCLE_LIMIT) { set_error(a.err, ERR_TIMEOUT); continue; }
    if (mn != k) continue;  // another slot of the cycle rotates it
    U C[B];
    blk_load<U>(C, keys + k * B);
    j = ip0_dest(ip, g, k);
    while (j != k) {
      U T[B];
      blk_load<U>(T, keys + j * B);
      blk_store<U>(keys + j * B, C);
#pragma unroll
      for (uint32_t i = 0; i < B; ++i) C[i] = T[i];
      j = ip0_dest(ip, g, j);
    }
    blk_store<U>(keys + k * B, C);
  }
}

// Key at position p of the permuted array: the partial last slot was written
// to the overflow block.
template <typename U>
__device__ __forceinline__ U ip0_at(const U* keys, const InPlace0& ip, uint64_t n, uint64_t p) {
  constexpr uint32_t B = IpBlk<U>::B;
  const uint64_t ks = n / B;
  return ((n % B) != 0 && p >= ks * B) ? ((const U*)ip.ovf)[p - ks * B] : keys[p];
}

// The part of slot floor(s_b / B) from s_b on, when it holds the last block of
// an earlier bucket (its overhang), saved before any gap is written.
template <int DT>
__global__ void k_ip_save0(Level0Args a, InPlace0 ip) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr uint32_t B = IpBlk<U>::B;
  if (call_failed(a.err)) return;
  const uint32_t f0 = a.f0;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x + 1; b < f0; b += gridDim.x * blockDim.x) {
    const uint64_t s = ip.sst[b];
    if (s % B == 0) continue;
    const uint64_t k0 = s / B;
    uint32_t lo = 0, hi = b - 1;  // last bucket q < b with dsl[q] <= k0
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if ((uint64_t)ip.dsl[mid] <= k0) lo = mid; else hi = mid - 1;
    }
    if (!ip.nbk[lo] || k0 >= (uint64_t)ip.dsl[lo] + ip.nbk[lo]) continue;
    U* sv = (U*)ip.save + (size_t)b * B;
    for (uint64_t p = s; p < (k0 + 1) * B; ++p) sv[p - s] = ip0_at<U>((const U*)a.keys, ip, a.c.n, p);
  }
}

constexpr int IP0_GAP_THREADS = 256;

// Head [s_b, d_b B) and tail [(d_b + nb_b) B, s_b + cntb_b) of bucket b: its
// leftovers from every piece, then the overhang of its last block (read from
// the save area of the bucket whose head holds it, or in place where it lies
// in an equality range).  One CTA per bucket.
template <int DT>
__global__ void __launch_bounds__(IP0_GAP_THREADS) k_ip_gaps0(Level0Args a, InPlace0 ip) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr uint32_t B = IpBlk<U>::B;
  __shared__ unsigned long long ws[40];
  if (call_failed(a.err)) return;
  const uint32_t f0 = a.f0;
  U* keys = (U*)a.keys;
  const uint64_t n = a.c.n;
  const uint64_t ks = n / B;
  const bool partial = (n % B) != 0;
  for (uint32_t b = blockIdx.x; b < f0; b += gridDim.x) {
    const uint64_t s = ip.sst[b], e = s + ip.cntb[b];
    const uint32_t nb = ip.nbk[b];
    const uint64_t lo = nb ? (uint64_t)ip.dsl[b] * B : e;
    const uint64_t hi = nb ? lo + (uint64_t)nb * B : e;
    const uint64_t g1 = (lo < e ? lo : e) - s;
    const uint64_t g2 = hi < e ? e - hi : 0;
    const uint64_t ov = (nb && hi > e) ? hi - e : 0;
    auto pos = [&](uint64_t i) { return i < g1 ? s + i : hi + (i - g1); };
    // leftovers, piece by piece
    uint64_t base = 0;
    for (uint32_t p0 = 0; p0 < ip.P; p0 += IP0_GAP_THREADS) {
      const uint32_t pc = p0 + threadIdx.x;
      const unsigned long long c = pc < ip.P ? ip.lo_cnt[(size_t)pc * f0 + b] : 0u;
      unsigned long long tot;
      const unsigned long long ex = block_excl_sum<unsigned long long>(c, ws, &tot);
      if (base + tot + ov <= g1 + g2) {
        const U* src = (const U*)ip.lo_keys + ((size_t)pc * f0 + b) * B;
        for (uint32_t i = 0; i < c; ++i) keys[pos(base + ex + i)] = src[i];
      }
      base += tot;
    }
    if (base + ov != g1 + g2) {
      if (threadIdx.x == 0) set_error(a.err, ERR_BOUNDS);
      continue;
    }
    // the overhang
    for (uint64_t i = threadIdx.x; i < ov; i += blockDim.x) {
      const uint64_t p = e + i;
      U x;
      if (b + 1 < f0 && p >= ip.sst[b + 1]) {
        uint32_t l = b + 1, h = f0 - 1;  // last bucket t with sst[t] <= p
        while (l < h) {
          const uint32_t mid = (l + h + 1) >> 1;
          if (ip.sst[mid] <= p) l = mid; else h = mid - 1;
        }
        x = ((const U*)ip.save)[(size_t)l * B + (p - ip.sst[l])];
      } else {
        x = ip0_at<U>(keys, ip, n, p);
      }
      keys[pos(base + i)] = x;
    }
    // the bucket's keys in the partial last slot
    if (partial && nb && hi > ks * B) {
      const uint64_t p0 = ks * B > lo ? ks * B : lo;
      const uint64_t p1 = hi < e ? hi : e;
      for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) keys[p] = ((const U*)ip.ovf)[p - ks * B];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- refinement levels
// Alg. 2's level-1 position of a key inside its level-0 bucket b:
// clamp(floor(F(x) f0 Kf) - b Kf, 0, Kf - 1), plus the key's interval between
// the bucket's heavy values (so the ids follow the key order across them).
template <int DT>
struct IpModelSub {
  CellRoot croot;
  const CellLeaf* cleaf;
  float f0kf;
  int bkf, kf;
  const HeavyEntry* hv;
  uint32_t nh;
  __device__ uint32_t operator()(typename KT<DT>::U u) const {
    const float F = cell_F<DT>(u, croot, cleaf);
    const float w = F * f0kf;
    int sub = (w >= 0.0f ? (int)w : 0) - bkf;
    sub = sub < 0 ? 0 : (sub >= kf ? kf - 1 : sub);
    uint32_t j = 0;
    if (nh) {
      const uint64_t t = KT<DT>::tk(u);
      for (uint32_t i = 0; i < nh; ++i) j += hv[i].tk < t ? 1u : 0u;
    }
    return (uint32_t)sub + j;
  }
};

// A split by a line through the segment's key range (value or total order).
template <int DT>
struct IpRangeSub {
  RangeSplit rs;
  __device__ uint32_t operator()(typename KT<DT>::U u) const { return range_sub<DT>(u, rs); }
};

// Sub-bucket starts of a level-0 bucket with heavy values: interval j's ids
// start at sub(h_{j-1}) + j and its keys where the level-0 offsets put the
// interval; inside an interval the sub-buckets follow each other.
struct IpHeavyStarts {
  const HeavyEntry* hv;
  uint32_t nh;
  float f0kf;
  int bkf, kf;
  const uint64_t* l0offs;  // level-0 slot offsets
  uint32_t ext_base;
  uint64_t start;          // the job's first position
  template <int NT>
  __device__ void run(const uint32_t* cnt, unsigned long long* st, uint32_t f,
                      unsigned long long* ws) const {
    const uint32_t c = threadIdx.x;
    const unsigned long long v = c < f ? (unsigned long long)cnt[c] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_sum<unsigned long long>(v, ws, &tot);
    if (c < f) st[c] = ex;
    __syncthreads();
    unsigned long long val = 0;
    if (c < f) {
      uint32_t iv = 0, first = 0;
      for (uint32_t i = 0; i < nh; ++i) {
        const float w = hv[i].F * f0kf;
        int sub = (w >= 0.0f ? (int)w : 0) - bkf;
        sub = sub < 0 ? 0 : (sub >= kf ? kf - 1 : sub);
        const uint32_t hs = (uint32_t)sub + i + 1;  // first id of interval i + 1
        if (hs <= c) { iv = i + 1; first = hs; }
      }
      val = (l0offs[ext_base + 2 * iv] - start) + (st[c] - st[first]);
    }
    __syncthreads();
    if (c < f) st[c] = val;
  }
};

constexpr int IPR_THREADS = 512;
constexpr int IPR_KPT = 16;

size_t ip_cta_smem(int dt) {
  return (dt == LS_F64 || dt == LS_U64) ? IpCta<uint64_t>::SMEM : IpCta<uint32_t>::SMEM;
}

// One refinement level in place: each CTA takes jobs from a counter and splits
// a job's segment inside its own range (ls_inplace.cuh), by the model (mode 0)
// or by the job's key range (modes 1 and 2); sub-bucket counts and end
// positions go to the level's counters for k_l1_classify.
// CHAINS: the jobs whose range is wider than their keys (a level-0 bucket with
// heavy values: its sub-buckets sit between equality ranges), split with the
// defragment by known destinations; else the others, in rounds (measured
// faster there).  Each instantiation takes its jobs from its own counter.
template <int DT, bool CHAINS>
__global__ void __launch_bounds__(IPR_THREADS, 1)
k_ip_refine(typename KT<DT>::U* keys, ModelPtrs M, LevelArgs la, Level1Ws w, IpChainWs cw,
            uint32_t* err) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  typedef IpCta<U> Y;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ unsigned long long s_job;
  const L1Aux* aux = (const L1Aux*)w.aux;
  const uint64_t nj = w.totals[2];
  const uint32_t* cnt = (const uint32_t*)(sm + Y::OFF_U32) + 4 * Y::F;
  const unsigned long long* st = (const unsigned long long*)(sm + Y::OFF_ST);
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_job = call_failed(err) ? ~0ull : atomicAdd(&w.totals[CHAINS ? 5 : 3], 1ull);
    __syncthreads();
    const unsigned long long j = s_job;
    if (j >= nj) break;
    const Job job = la.in.jobs[j];
    const L1Aux x = aux[j];
    if ((job.span > job.m) != CHAINS) continue;  // the other instantiation's job
    U* X = job_keys(job, keys) + job.start;
    cw.seg_pos = job.start;
    if (la.mode && w.jmin[j] == w.jmax[j]) {  // homogeneous: one sub-bucket, filled later
      for (uint32_t c = threadIdx.x; c < x.f1; c += blockDim.x) {
        w.cnt[x.cbase + c] = c == 0 ? (uint32_t)job.m : 0u;
        w.cur[x.cbase + c] = job.start + (c == 0 ? job.m : 0ull);
      }
      continue;
    }
    if (la.mode == 0) {
      const uint32_t b = job.la;
      const BucketHead h = M.heads[b];
      IpModelSub<DT> sub;
      sub.croot = M.hdr->croot;
      sub.cleaf = M.cleaf;
      sub.f0kf = la.f0kf;
      sub.bkf = (int)(b * la.kf);
      sub.kf = (int)la.kf;
      sub.hv = M.heavy + (h.hoff_nh >> 4);
      sub.nh = job.lb;
      if (job.lb) {
        IpHeavyStarts hs{sub.hv, job.lb, la.f0kf, sub.bkf, sub.kf, la.l0offs, h.ext_base, job.start};
        ip_cta_partition<U, IPR_THREADS, IPR_KPT, CHAINS>(X, job.m, job.span, x.f1, sub, hs, sm, err, cw);
      } else {
        ip_cta_partition<U, IPR_THREADS, IPR_KPT, CHAINS>(X, job.m, job.span, x.f1, sub, IpPrefixStarts{}, sm, err, cw);
      }
    } else {
      IpRangeSub<DT> sub;
      sub.rs = range_split<DT>(w.jmin[j], w.jmax[j], x.f1, la.mode == 2);
      ip_cta_partition<U, IPR_THREADS, IPR_KPT, CHAINS>(X, job.m, job.span, x.f1, sub, IpPrefixStarts{}, sm, err, cw);
    }
    for (uint32_t c = threadIdx.x; c < x.f1; c += blockDim.x) {
      w.cnt[x.cbase + c] = cnt[c];
      w.cur[x.cbase + c] = job.start + st[c] + cnt[c];
    }
  }
}

// ---------------------------------------------------------------- host enqueue
template <int DT>
static cudaError_t ip_level0_dt(const Level0Args& a, const InPlace0& ip, const Lists& lists,
                                const SortLimits& lim, cudaStream_t st, int num_sms,
                                const Marks* mk, int mb) {
  const Ip0Layout y = ip0_layout(KT<DT>::W, a.L, a.f0, a.n_ext_max);
  launch_k(k_ip_frag0<DT>, ip.P, IP0_THREADS, y.total, st, a, ip, y);
  mark(mk, mb + 0, st);
  launch_k(k_scan<uint32_t>, a.scan_tiles, SC_THREADS, 0, st, a.hist, a.offs, (uint64_t)a.n_ext_max,
           nullptr, (uint64_t*)a.scan_status, (uint32_t*)((uint64_t*)a.scan_status + a.scan_tiles),
           a.err, STALL_L0_SCAN);
  mark(mk, mb + 1, st);
  launch_k(k_ip_prep0<DT>, (a.f0 + 255) / 256, 256, 0, st, a, ip);
  const unsigned pg = (unsigned)std::min<uint64_t>(
      std::max<uint64_t>(1, (a.c.n / IpBlk<typename KT<DT>::U>::B + IP0_PERM_THREADS - 1) / IP0_PERM_THREADS),
      16ull * num_sms);
  launch_k(k_ip_inv0<DT>, pg, IP0_PERM_THREADS, 0, st, a, ip);
  launch_k(k_ip_starts0<DT>, pg, IP0_PERM_THREADS, 0, st, a, ip);
  launch_k(k_ip_chain0<DT>, 8 * num_sms, IP0_PERM_THREADS, 0, st, a, ip);
  launch_k(k_ip_cycle0<DT>, pg, IP0_PERM_THREADS, 0, st, a, ip);
  launch_k(k_ip_save0<DT>, (a.f0 + 255) / 256, 256, 0, st, a, ip);
  launch_k(k_ip_gaps0<DT>, a.f0, IP0_GAP_THREADS, 0, st, a, ip);
  mark(mk, mb + 2, st);
  launch_classify0(DT, a, lists, lim, st);
  mark(mk, mb + 3, st);
  add_launches(9);
  return cudaGetLastError();
}

cudaError_t ip_level0_enqueue(int dt, const Level0Args& a, const InPlace0& ip, const Lists& lists,
                              const SortLimits& lim, cudaStream_t st, int num_sms,
                              const Marks* mk, int mb) {
  switch (dt) {
    case LS_F64: return ip_level0_dt<LS_F64>(a, ip, lists, lim, st, num_sms, mk, mb);
    case LS_U64: return ip_level0_dt<LS_U64>(a, ip, lists, lim, st, num_sms, mk, mb);
    case LS_F32: return ip_level0_dt<LS_F32>(a, ip, lists, lim, st, num_sms, mk, mb);
    case LS_U32: return ip_level0_dt<LS_U32>(a, ip, lists, lim, st, num_sms, mk, mb);
  }
  return cudaErrorInvalidValue;
}

template <int DT>
static cudaError_t ip_level_dt(void* keys, const ModelPtrs& M, const Lists& lists,
                               const LevelArgs& la, const SortLimits& lim, const Level1Ws& w,
                               const IpChainWs& cw, uint32_t* err, cudaStream_t st, int num_sms) {
  typedef typename KT<DT>::U U;
  launch_l1_plan(la, lim, w, err, st);
  if (la.mode) launch_l1_minmax(DT, keys, la, w, st, num_sms);
  launch_k(k_ip_refine<DT, false>, num_sms, IPR_THREADS, IpCta<U>::SMEM, st, (U*)keys, M, la, w, cw, err);
  if (la.mode == 0) {  // only the model's level has jobs wider than their keys
    launch_k(k_ip_refine<DT, true>, num_sms, IPR_THREADS, IpCta<U>::SMEM, st, (U*)keys, M, la, w, cw, err);
    add_launches(1);
  }
  launch_l1_classify(DT, lists, la, lim, w, M, err, st, num_sms);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t ip_levels_enqueue(int dt, void* keys, const ModelPtrs& M, const Lists& lists,
                              const SortLimits& lim, const Level1Ws& w, const InPlace0& ip,
                              uint32_t kf, float f0kf, const uint64_t* l0offs, uint32_t* err,
                              cudaStream_t st, int num_sms, bool range_levels) {
  // the level-0 defragment's per-slot arrays serve every split of the levels;
  // holes are reserved through the level's counter totals[4] (zeroed by its plan)
  IpChainWs cw{};
  cw.tags = ip.tags;
  cw.prank = ip.prank;
  cw.inv = ip.inv;
  cw.moved = ip.flags;
  cw.hscr = ip.hscr;
  cw.hctr = w.totals + 4;
  cw.hcap = ip.hcap;
  // as out of place: the model's split, then the value range, then the
  // total-order key range; at most IP_CTA_FMAX sub-buckets per split
  const JobList ins[3] = {lists.refine, lists.refine2, lists.refine3};
  const JobList outs[3] = {range_levels ? lists.refine2 : lists.fallback, lists.refine3,
                           lists.fallback};
  for (int lv = 0; lv < (range_levels ? 3 : 1); ++lv) {
    LevelArgs la{};
    la.in = ins[lv];
    la.next = outs[lv];
    la.mode = lv == 0 ? 0 : (lv == 1 ? 2 : 1);
    la.next_kind = (lv == 2 || !range_levels) ? JOB_FALLBACK : JOB_REFINE;
    la.kf = kf;
    la.target = lv == 2 ? 16 : lim.l1_target / 3;
    la.fmax = IP_CTA_FMAX;
    la.l0offs = l0offs;
    la.l0G = 1;
    la.f0kf = f0kf;
    la.in_place = 1;
    cudaError_t e = cudaErrorInvalidValue;
    switch (dt) {
      case LS_F64: e = ip_level_dt<LS_F64>(keys, M, lists, la, lim, w, cw, err, st, num_sms); break;
      case LS_U64: e = ip_level_dt<LS_U64>(keys, M, lists, la, lim, w, cw, err, st, num_sms); break;
      case LS_F32: e = ip_level_dt<LS_F32>(keys, M, lists, la, lim, w, cw, err, st, num_sms); break;
      case LS_U32: e = ip_level_dt<LS_U32>(keys, M, lists, la, lim, w, cw, err, st, num_sms); break;
    }
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t ip_configure(int dt, size_t smem0) {
  cudaError_t e = cudaSuccess;
#define LS_IPCFG(D)                                                                              \
  e = cudaFuncSetAttribute(k_ip_frag0<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0); \
  if (e) return e;                                                                               \
  e = cudaFuncSetAttribute(k_ip_refine<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                           (int)IpCta<typename KT<D>::U>::SMEM);                                 \
  if (e) return e;                                                                               \
  e = cudaFuncSetAttribute(k_ip_refine<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                           (int)IpCta<typename KT<D>::U>::SMEM);
  switch (dt) {
    case LS_F64: LS_IPCFG(LS_F64); break;
    case LS_U64: LS_IPCFG(LS_U64); break;
    case LS_F32: LS_IPCFG(LS_F32); break;
    case LS_U32: LS_IPCFG(LS_U32); break;
  }
#undef LS_IPCFG
  return e;
}

}  // namespace ls

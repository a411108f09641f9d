// In-place partitioning of LearnedSort 2.0 (Sec. 4.2, Alg. 1: fragments that
// are flushed back over already-read positions, then Defragment), shared by
// the level-0 pass of the in-place variant (ls_inplace.cu), its refinement
// levels (ls_inplace.cu) and its radix fallback (ls_bucket.cu).
//
// A segment X of m keys is split into f buckets (a non-decreasing bucket map
// sub(x)); bucket c ends up at [st[c], st[c] + cnt[c]) of [0, span), span >= m
// (gaps between buckets hold keys written later, e.g. equality fills).  The
// steps, all inside X:
//   A (fragment flush)  keys stream through per-bucket fragments of B keys
//                       (one 128-byte block); a full fragment is written to the
//                       next free block slot at the front of X, which the
//                       stream has already read.  Leftovers (< B keys per
//                       bucket) stay in the fragments.
//   B (defragment)      the blocks are permuted into bucket order: bucket c's
//                       blocks go to slots [d_c, d_c + nb_c), d_c =
//                       ceil(st[c] / B).  Two ways:
//                       * rounds: each bucket has a write pointer w (from d_c
//                         up) and a read pointer r (from the end of its slot
//                         range down), one 64-bit word w << 32 | (r + 1)
//                         updated by single atomics, so every slot is claimed
//                         exactly once, by a reader (its block is taken out
//                         and classified) or by a writer (a block of the
//                         bucket is put there; a block found there is carried
//                         on);
//                       * known destinations: step A records each block's
//                         bucket and rank, so its destination is d_c + rank;
//                         the blocks are pulled backwards along the inverse
//                         map in chains that start at free slots (holes copied
//                         out, or slots that held no block).
//   C (cleanup)         a bucket's block range starts at a block boundary, so
//                       its head [st, d*B) and tail [(d+nb)*B, end) are filled
//                       from its leftovers; its last block may overhang the
//                       next bucket's head, and those keys are saved first and
//                       written into the bucket's own gaps.
#pragma once
#include "ls_internal.cuh"
#include "ls_scan.cuh"

namespace ls {

constexpr uint32_t IP_BLOCK_BYTES = 128;  // one block: 16 keys of 8 bytes, 32 of 4
constexpr uint32_t IP_CTA_FMAX = 256;     // buckets of one CTA-local split
constexpr uint32_t IP_NONE = 0xFFFFFFFFu;

template <typename U>
struct IpBlk {
  static constexpr uint32_t B = IP_BLOCK_BYTES / sizeof(U);
};

// One block between global memory and registers (16-byte vector accesses when
// the block is 16-byte aligned, which holds for every block of a segment whose
// first key is).
template <typename U>
__device__ __forceinline__ void blk_load(U* h, const U* p) {
  constexpr uint32_t B = IpBlk<U>::B;
  if (((uintptr_t)p & 15) == 0) {
    const uint4* q = (const uint4*)p;
#pragma unroll
    for (uint32_t i = 0; i < IP_BLOCK_BYTES / 16; ++i) {
      const uint4 v = q[i];
      if (sizeof(U) == 8) {
        h[2 * i] = (U)(((unsigned long long)v.y << 32) | v.x);
        h[2 * i + 1] = (U)(((unsigned long long)v.w << 32) | v.z);
      } else {
        h[4 * i] = (U)v.x;
        h[4 * i + 1] = (U)v.y;
        h[4 * i + 2] = (U)v.z;
        h[4 * i + 3] = (U)v.w;
      }
    }
  } else {
#pragma unroll
    for (uint32_t i = 0; i < B; ++i) h[i] = p[i];
  }
}
template <typename U>
__device__ __forceinline__ void blk_store(U* p, const U* h) {
  constexpr uint32_t B = IpBlk<U>::B;
  if (((uintptr_t)p & 15) == 0) {
    uint4* q = (uint4*)p;
#pragma unroll
    for (uint32_t i = 0; i < IP_BLOCK_BYTES / 16; ++i) {
      uint4 v;
      if (sizeof(U) == 8) {
        v.x = (uint32_t)(unsigned long long)h[2 * i];
        v.y = (uint32_t)((unsigned long long)h[2 * i] >> 32);
        v.z = (uint32_t)(unsigned long long)h[2 * i + 1];
        v.w = (uint32_t)((unsigned long long)h[2 * i + 1] >> 32);
      } else {
        v.x = (uint32_t)h[4 * i];
        v.y = (uint32_t)h[4 * i + 1];
        v.z = (uint32_t)h[4 * i + 2];
        v.w = (uint32_t)h[4 * i + 3];
      }
      q[i] = v;
    }
  } else {
#pragma unroll
    for (uint32_t i = 0; i < B; ++i) p[i] = h[i];
  }
}

// Shared memory of the CTA-local split (at most IP_CTA_FMAX buckets).
template <typename U>
struct IpCta {
  static constexpr uint32_t F = IP_CTA_FMAX;
  static constexpr size_t OFF_FRAG = 0;                                 // F blocks
  static constexpr size_t OFF_SAVE = OFF_FRAG + (size_t)F * IP_BLOCK_BYTES;  // F blocks
  static constexpr size_t OFF_OVF = OFF_SAVE + (size_t)F * IP_BLOCK_BYTES;   // one block
  static constexpr size_t OFF_ST = OFF_OVF + IP_BLOCK_BYTES;           // F x u64
  static constexpr size_t OFF_PAIR = OFF_ST + 8 * (size_t)F;           // F x u64
  static constexpr size_t OFF_U32 = OFF_PAIR + 8 * (size_t)F;          // 7 x F x u32
  static constexpr size_t OFF_WS = OFF_U32 + 4 * 7 * (size_t)F;        // 40 x u64
  static constexpr size_t SMEM = OFF_WS + 8 * 40;
};

// Bucket starts of a split whose buckets follow each other without gaps:
// st[c] = cnt[0] + ... + cnt[c-1].
struct IpPrefixStarts {
  template <int NT>
  __device__ void run(const uint32_t* cnt, unsigned long long* st, uint32_t f,
                      unsigned long long* ws) const {
    const unsigned long long v = threadIdx.x < f ? (unsigned long long)cnt[threadIdx.x] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_sum<unsigned long long>(v, ws, &tot);
    if (threadIdx.x < f) st[threadIdx.x] = ex;
  }
};

// About one slot in 32, spread by a multiplicative hash of the slot index (no
// regular stride for a permutation to line up with): the holes of the
// defragment by known destinations.  A chain runs from a hole to the next one,
// so the longest chain is about 32 ln(#chains) blocks.
__device__ __forceinline__ bool ip_hole(uint64_t k) {
  return (((uint32_t)k * 0x9E3779B1u) >> 27) == 0u;
}

// Per-slot arrays for a CTA-local defragment by known destinations, indexed by
// the slot's absolute index floor(pos / B) (pos the slot's first key in the
// array): distinct for the whole slots of disjoint segments (a segment's
// partial last slot is kept in shared memory instead).
struct IpChainWs {
  uint16_t* tags;          // bucket of a flushed block
  uint32_t* prank;         // its rank among its bucket's blocks (a hole's: its place in hscr)
  uint32_t* inv;           // the slot whose block goes here
  uint8_t* moved;
  void* hscr;              // hole blocks, reserved through hctr
  unsigned long long* hctr;
  uint64_t hcap;
  uint64_t seg_pos;        // the segment's first key, as a position in the array
};

// Largest c in [0, f) with d[c] <= k (d[0] = 0, non-decreasing).
__device__ __forceinline__ uint32_t ip_bucket_of_slot(const uint32_t* d, uint32_t f, uint32_t k) {
  uint32_t lo = 0, hi = f - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (d[mid] <= k) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// CTA-local in-place split of X[0, m) into f <= IP_CTA_FMAX buckets laid out in
// [0, span) (steps A, B, C above, with the whole CTA on one segment).  NT
// threads, KPT keys per thread and tile.  CHAINS: step B by known destinations
// (the per-slot arrays of `cw`, falling back to rounds when the holes do not
// fit); else in rounds.  Sub: `uint32_t operator()(U) const`,
// the bucket of a key; Starts: `run<NT>(cnt, st, f, ws)` filling st.  On return
// (after a barrier) the CTA's shared memory holds cnt (u32 at OFF_U32 + 4*4*F)
// and st (u64 at OFF_ST) of every bucket.  Phase B runs in rounds: in each
// round threads without a block take one from a read pointer, a barrier, then
// threads holding a block make one write; a slot a reader took is therefore
// read before any writer of a later round (or of the same round's write half)
// stores into it, with no flag or wait.
template <typename U, int NT, int KPT, bool CHAINS, class Sub, class Starts>
__device__ void ip_cta_partition(U* X, uint64_t m, uint64_t span, uint32_t f, const Sub& sub,
                                 const Starts& starts, unsigned char* sm, uint32_t* err,
                                 const IpChainWs& cw) {
  typedef IpCta<U> Y;
  constexpr uint32_t B = IpBlk<U>::B;
  constexpr uint32_t F = Y::F;
  static_assert(NT >= (int)F && NT % 32 == 0, "one thread per bucket in the scans");
  U* frag = (U*)(sm + Y::OFF_FRAG);
  U* save = (U*)(sm + Y::OFF_SAVE);
  U* ovf = (U*)(sm + Y::OFF_OVF);
  unsigned long long* st = (unsigned long long*)(sm + Y::OFF_ST);
  unsigned long long* pair = (unsigned long long*)(sm + Y::OFF_PAIR);
  uint32_t* ffill = (uint32_t*)(sm + Y::OFF_U32);  // keys in the fragment
  uint32_t* tcnt = ffill + F;                      // keys of the tile (then: save offsets)
  uint32_t* slot0 = ffill + 2 * F;                 // first slot of the tile's flushes
  uint32_t* nfull = ffill + 3 * F;                 // blocks flushed by the tile
  uint32_t* cnt = ffill + 4 * F;                   // keys of the bucket
  uint32_t* nbk = ffill + 5 * F;                   // blocks of the bucket
  uint32_t* dd = ffill + 6 * F;                    // first slot of the bucket's range
  unsigned long long* ws = (unsigned long long*)(sm + Y::OFF_WS);
  uint32_t* nsl = (uint32_t*)(ws + 36);            // slots written in step A
  const uint32_t tid = threadIdx.x;
  if (f > F || f == 0 || (span + B - 1) / B >= 0x7FFFFFFFull || m > span) {
    if (tid == 0) set_error(err, ERR_BOUNDS);
    __syncthreads();
    return;
  }
  for (uint32_t c = tid; c < F; c += NT) {
    ffill[c] = tcnt[c] = nfull[c] = cnt[c] = nbk[c] = 0;
  }
  if (tid == 0) *nsl = 0;
  __syncthreads();
  // ---- A: fragment flush
  constexpr uint32_t T = NT * KPT;
  for (uint64_t t0 = 0; t0 < m; t0 += T) {
    U u[KPT];
    uint32_t s[KPT], rk[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const uint64_t i = t0 + (uint64_t)k * NT + tid;
      u[k] = i < m ? X[i] : (U)0;
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const uint64_t i = t0 + (uint64_t)k * NT + tid;
      s[k] = i < m ? min(sub(u[k]), f - 1) : IP_NONE;
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) rk[k] = s[k] != IP_NONE ? atomicAdd(&tcnt[s[k]], 1u) : 0u;
    __syncthreads();
    for (uint32_t c = tid; c < f; c += NT) {
      const uint32_t t = tcnt[c];
      if (t) {
        const uint32_t nf = (ffill[c] + t) / B;
        nfull[c] = nf;
        if (nf) slot0[c] = atomicAdd(nsl, nf);
        cnt[c] += t;
        nbk[c] += nf;
      }
    }
    __syncthreads();
    // the first flushed block of a bucket starts with its fragment's keys
    for (uint32_t c = tid; c < f; c += NT) {
      if (nfull[c] && ffill[c]) {
        U* dst = X + (uint64_t)slot0[c] * B;
        for (uint32_t q = 0; q < ffill[c]; ++q) dst[q] = frag[c * B + q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (s[k] == IP_NONE) continue;
      const uint32_t c = s[k];
      const uint32_t p = ffill[c] + rk[k];
      const uint32_t full = nfull[c] * B;
      if (p < full) {
        const uint32_t sl = slot0[c] + p / B;
        X[(uint64_t)sl * B + p % B] = u[k];
        if (CHAINS && p % B == B - 1) {  // the block's last key: its bucket and rank
          const uint64_t ab = cw.seg_pos / B + sl;
          cw.tags[ab] = (uint16_t)c;
          cw.prank[ab] = nbk[c] - nfull[c] + p / B;
        }
      } else {
        frag[c * B + (p - full)] = u[k];
      }
    }
    __syncthreads();
    for (uint32_t c = tid; c < f; c += NT) {
      const uint32_t t = tcnt[c];
      if (t) {
        ffill[c] = ffill[c] + t - nfull[c] * B;
        tcnt[c] = 0;
        nfull[c] = 0;
      }
    }
    __syncthreads();
  }
  // ---- bucket ranges
  starts.template run<NT>(cnt, st, f, ws);
  __syncthreads();
  const uint32_t nslots = (uint32_t)((span + B - 1) / B);
  const uint32_t nw = *nsl;
  const bool partial = (span % B) != 0;
  const uint32_t ks = (uint32_t)(span / B);  // the partial last slot
  for (uint32_t c = tid; c < f; c += NT) dd[c] = (uint32_t)((st[c] + B - 1) / B);
  __syncthreads();
  // The blocks of step A fill slots [0, nw); a bucket's read pointer starts at
  // its last slot below nw (slots above hold no block and need no reader: a
  // writer that reaches one finds it empty).
  bool bad = false;
  for (uint32_t c = tid; c < f; c += NT) {
    const uint32_t D = c + 1 < f ? dd[c + 1] : nslots;
    if (dd[c] + nbk[c] > D || st[c] + cnt[c] > (c + 1 < f ? st[c + 1] : span)) bad = true;
    pair[c] = ((unsigned long long)dd[c] << 32) | max(dd[c], min(D, nw));
  }
  if (__syncthreads_or(bad)) {  // inconsistent bucket ranges (cannot happen): keys untouched
    if (tid == 0) set_error(err, ERR_BOUNDS);
    return;
  }
  // ---- B by known destinations: a block goes to dd[c] + its rank in bucket c
  bool chains = CHAINS;
  if (CHAINS) {
    uint32_t* sh_u = (uint32_t*)(ws + 37);  // [0] local hole count, [1] the partial slot's source
    uint32_t* jctr = (uint32_t*)(ws + 39);  // the next slot to look at for a chain start
    unsigned long long* hbase = ws + 38;
    uint32_t hn = 0;
    for (uint32_t k = tid; k < nw; k += NT) hn += ip_hole(cw.seg_pos / B + k) ? 1u : 0u;
    unsigned long long htot;
    block_excl_sum<unsigned long long>((unsigned long long)hn, ws, &htot);
    if (tid == 0) {
      const unsigned long long b0 = htot ? atomicAdd(cw.hctr, htot) : 0ull;
      *hbase = (b0 + htot <= cw.hcap) ? b0 : ~0ull;
      sh_u[0] = 0;
      sh_u[1] = IP_NONE;
      *jctr = 0;
    }
    __syncthreads();
    chains = *hbase != ~0ull;
  }
  if (CHAINS && chains) {
    const uint64_t a0 = cw.seg_pos / B;
    uint32_t* sh_u = (uint32_t*)(ws + 37);
    uint32_t* jctr = (uint32_t*)(ws + 39);
    const unsigned long long hb = ws[38];
    for (uint32_t j = tid; j < nslots; j += NT) {
      if (partial && j == ks) continue;
      cw.inv[a0 + j] = IP_NONE;
      cw.moved[a0 + j] = 0;
    }
    __syncthreads();
    bool oob = false;
    for (uint32_t k = tid; k < nw; k += NT) {  // the inverse map, the holes copied out
      const uint32_t c = min((uint32_t)cw.tags[a0 + k], f - 1);
      const uint32_t d = dd[c] + cw.prank[a0 + k];
      if (d >= (c + 1 < f ? dd[c + 1] : nslots)) { oob = true; continue; }
      if (partial && d == ks) sh_u[1] = k;
      else cw.inv[a0 + d] = k;
      if (ip_hole(a0 + k)) {
        const unsigned long long hp = hb + atomicAdd(&sh_u[0], 1u);
        U H[B];
        blk_load<U>(H, X + (uint64_t)k * B);
        blk_store<U>((U*)cw.hscr + hp * B, H);
        cw.prank[a0 + k] = (uint32_t)hp;
      }
    }
    if (__syncthreads_or(oob)) {  // cannot happen: keys left as they are
      if (tid == 0) set_error(err, ERR_BOUNDS);
      return;
    }
    // chains from every free destination: a hole, or a slot at or above nw;
    // slots are taken from a counter, so that the threads stay busy until the
    // last chains end
    while (true) {
      const uint32_t j = atomicAdd(jctr, 1u);
      if (j >= nslots) break;
      uint32_t k = (partial && j == ks) ? sh_u[1] : cw.inv[a0 + j];
      if (k == IP_NONE || (j < nw && !ip_hole(a0 + j))) continue;
      uint32_t cur = j;
      for (uint32_t step = 0; step <= nw; ++step) {
        U H[B];
        const bool hole = ip_hole(a0 + k);
        const uint32_t nxt = hole ? IP_NONE : cw.inv[a0 + k];  // k < nw: a whole slot
        if (hole) blk_load<U>(H, (const U*)cw.hscr + (uint64_t)cw.prank[a0 + k] * B);
        else blk_load<U>(H, X + (uint64_t)k * B);
        blk_store<U>((partial && cur == ks) ? ovf : X + (uint64_t)cur * B, H);
        cw.moved[a0 + k] = 1;
        if (hole || nxt == IP_NONE) break;
        cur = k;
        k = nxt;
      }
    }
    __syncthreads();
    // cycles without a hole, rotated by their smallest slot
    for (uint32_t k = tid; k < nw; k += NT) {
      if (ip_hole(a0 + k) || cw.moved[a0 + k]) continue;
      auto dest = [&](uint32_t x) {
        return dd[min((uint32_t)cw.tags[a0 + x], f - 1)] + cw.prank[a0 + x];
      };
      uint32_t j = dest(k);
      if (j == k) continue;
      uint32_t mn = k, steps = 0;
      while (j != k && steps <= nw) { mn = min(mn, j); j = dest(j); ++steps; }
      if (steps > nw) { set_error(err, ERR_BOUNDS); continue; }
      if (mn != k) continue;
      U C[B];
      blk_load<U>(C, X + (uint64_t)k * B);
      j = dest(k);
      while (j != k) {
        U T[B];
        blk_load<U>(T, X + (uint64_t)j * B);
        blk_store<U>(X + (uint64_t)j * B, C);
#pragma unroll
        for (uint32_t i = 0; i < B; ++i) C[i] = T[i];
        j = dest(j);
      }
      blk_store<U>(X + (uint64_t)k * B, C);
    }
    __syncthreads();
  }
  // ---- B in rounds (no hole room, or no per-slot arrays); one ticket per slot below nw
  if (!chains) {
    uint32_t tick = tid;
    bool held = false;
    U H[B];
    uint32_t hs = 0;
    while (true) {
      if (!held && tick < nw) {
        const uint32_t c = ip_bucket_of_slot(dd, f, tick);
        tick += NT;
        const unsigned long long old = atomicAdd(&pair[c], ~0ull);
        const long long w = (long long)(old >> 32), r = (long long)(old & 0xFFFFFFFFull) - 1;
        if (r >= w) {  // r < nw: a slot holding a block
          blk_load<U>(H, X + (uint64_t)r * B);
          held = true;
          hs = min(sub(H[0]), f - 1);
        }
      }
      __syncthreads();
      if (held) {
        const unsigned long long old = atomicAdd(&pair[hs], 1ull << 32);
        const long long w = (long long)(old >> 32), r = (long long)(old & 0xFFFFFFFFull) - 1;
        const uint32_t D = hs + 1 < f ? dd[hs + 1] : nslots;
        if (w >= (long long)D) {
          set_error(err, ERR_BOUNDS);  // more blocks than room (cannot happen)
          held = false;
        } else {
          U* dst = (partial && (uint32_t)w == ks) ? ovf : X + (uint64_t)w * B;
          if (w <= r && (uint64_t)w < nw) {  // an unread block: carry it on
            U H2[B];
            blk_load<U>(H2, X + (uint64_t)w * B);
            blk_store<U>(dst, H);
#pragma unroll
            for (uint32_t i = 0; i < B; ++i) H[i] = H2[i];
            hs = min(sub(H[0]), f - 1);
          } else {  // a slot at or above nw, or one a reader emptied in an earlier half-round
            blk_store<U>(dst, H);
            held = false;
          }
        }
      }
      if (!__syncthreads_or(held || tick < nw)) break;
    }
  }
  // ---- C: cleanup
  uint32_t* svo = tcnt;  // per bucket: offset of its overhang in `save`
  for (uint32_t c = tid; c < f; c += NT) {
    uint32_t ov = 0;
    if (nbk[c]) {
      const uint64_t bhi = (uint64_t)(dd[c] + nbk[c]) * B, e = st[c] + cnt[c];
      if (bhi > e) ov = (uint32_t)(bhi - e);
    }
    svo[c] = ov;
  }
  __syncthreads();
  {
    const unsigned long long v = tid < f ? (unsigned long long)svo[tid] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_sum<unsigned long long>(v, ws, &tot);
    if (tid < f) svo[tid] = (uint32_t)ex;
  }
  __syncthreads();
  // the overhang of every bucket's last block, read before any gap is written
  // (positions in the partial last slot were written to `ovf`)
  for (uint32_t c = tid; c < f; c += NT) {
    if (!nbk[c]) continue;
    const uint64_t bhi = (uint64_t)(dd[c] + nbk[c]) * B, e = st[c] + cnt[c];
    for (uint64_t p = e; p < bhi; ++p) {
      const U x = (partial && p >= (uint64_t)ks * B) ? ovf[p - (uint64_t)ks * B] : X[p];
      save[svo[c] + (uint32_t)(p - e)] = x;
    }
  }
  __syncthreads();
  const int lane = tid & 31;
  for (uint32_t c = tid >> 5; c < f; c += NT / 32) {
    const uint64_t s0 = st[c], e = s0 + cnt[c];
    const uint32_t nb = nbk[c];
    const uint64_t lo = nb ? (uint64_t)dd[c] * B : e;
    const uint64_t hi = nb ? lo + (uint64_t)nb * B : e;
    const uint64_t g1 = (lo < e ? lo : e) - s0;
    const uint64_t g2 = hi < e ? e - hi : 0;
    const uint32_t left = ffill[c];
    const uint32_t ov = (nb && hi > e) ? (uint32_t)(hi - e) : 0u;
    if ((uint64_t)left + ov != g1 + g2) {
      if (lane == 0) set_error(err, ERR_BOUNDS);
      continue;
    }
    for (uint64_t q = lane; q < g1 + g2; q += 32) {
      const U x = q < left ? frag[c * B + (uint32_t)q] : save[svo[c] + (uint32_t)(q - left)];
      X[q < g1 ? s0 + q : hi + (q - g1)] = x;
    }
    if (partial && nb && hi > (uint64_t)ks * B) {  // the bucket's keys in the partial slot
      const uint64_t p0 = (uint64_t)ks * B > lo ? (uint64_t)ks * B : lo;
      const uint64_t p1 = hi < e ? hi : e;
      for (uint64_t p = p0 + lane; p < p1; p += 32) X[p] = ovf[p - (uint64_t)ks * B];
    }
  }
  __syncthreads();
}

}  // namespace ls

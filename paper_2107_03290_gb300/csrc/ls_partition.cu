// Model-based partitioning of LearnedSort 2.0 (Alg. 1) on the GPU.
//
// The paper's CPU Partition appends each key to a fixed-capacity fragment of
// its predicted bucket and flushes full fragments in place, so buckets never
// overflow (Sec. 4.2).  On the GPU the same goal -- each bucket gets exactly
// the space it needs -- is reached with a counting pre-pass (the exact-count
// alternative weighed in Sec. 4.2), which costs one extra streaming read:
//   K2 k_l0_hist     evaluates the model once per key: its extended slot
//                    (bucket, or an equality slot of a heavy value) counted in
//                    a per-CTA shared-memory histogram, and a packed id
//                    (bucket | level-1 id) stored for the scatter; when
//                    equality keys dominate, the other keys and their ids are
//                    packed into scratch;
//   K3 k_scan        decoupled look-back exclusive scan of the histograms,
//                    giving every (slot, CTA) its write head;
//   K4 k_l0_scatter  streams key and id tiles by TMA into shared memory, ranks
//                    keys by bucket inside the tile, stages them
//                    bucket-contiguously and writes full runs (keys and
//                    level-1 ids) to the other buffer;
//   k_classify0      turns slots into jobs (equality fill, in-bucket sort,
//                    level-1 re-partition).
// Level 1 (Alg. 2's re-partition of each bucket into sub-buckets) uses the
// sub-bucket ids from K2: sub = clamp(floor(F(x) * f0 * Kf) - b * Kf, 0, Kf-1),
// the paper's level-1 position with Kf sub-buckets per bucket, offset by the
// key's interval between the bucket's heavy values.
#include <cfloat>

#include "ls_partition.cuh"
#include "ls_partition_dev.cuh"
#include "ls_scan.cuh"
#include "ls_tma.cuh"

namespace ls {

// K4: double-buffered key and id tiles, per-bucket counters, offsets and
// cursors, staging records.
static L0Layout l0_layout_scatter(int W, uint32_t f0, uint32_t hmax, int tile) {
  L0Layout y{};
  size_t o = 0;
  auto al = [&](size_t a) { o = (o + a - 1) / a * a; };
  (void)hmax;
  const size_t nc = f0;
  y.bar = (uint32_t)o; o += 16;
  al(128); y.buf = (uint32_t)o; o += 2ull * tile * W;
  al(128); y.pbuf = (uint32_t)o; o += 2ull * tile * 4;
  y.ecnt = (uint32_t)o; o += nc * 4;
  y.soff = (uint32_t)o; o += (nc + 1) * 4;
  al(8); y.cursor = (uint32_t)o; o += nc * 8;
  y.gbase = (uint32_t)o; o += nc * 8;
  y.sinfo = (uint32_t)o; o += (size_t)tile * 2;
  y.sid = (uint32_t)o; o += (size_t)tile * 2;
  al(8); y.ws = (uint32_t)o; o += 33 * 8;
  y.total = (uint32_t)o;
  return y;
}

// K4's tile: P_TILE keys, or P_TILE_SMALL when the per-bucket arrays of a large
// fan-out leave too little shared memory.
static int scatter_tile(int W, uint32_t f0, uint32_t hmax) {
  return l0_layout_scatter(W, f0, hmax, P_TILE).total <= L0_SMEM_LIMIT ? P_TILE : P_TILE_SMALL;
}

size_t level0_smem_hist(int dt, uint32_t L, uint32_t f0, uint32_t n_ext_max) {
  return l0_layout_hist(key_width(dt), L, f0, n_ext_max, (n_ext_max - f0) / 2).total;
}
size_t level0_smem_scatter(int dt, uint32_t L, uint32_t f0, uint32_t n_ext_max) {
  (void)L;
  const uint32_t hmax = (n_ext_max - f0) / 2;
  return l0_layout_scatter(key_width(dt), f0, hmax, scatter_tile(key_width(dt), f0, hmax)).total;
}

__device__ __forceinline__ void chunk_of(const Chunking& c, uint32_t g, uint64_t* b, uint64_t* e) {
  uint64_t cb = c.a0 + (uint64_t)g * c.ch;
  uint64_t ce = cb + c.ch;
  if (cb > c.a1) cb = c.a1;
  if (ce > c.a1) ce = c.a1;
  *b = cb;
  *e = ce;
}


// ---------------------------------------------------------------- K2
// One model evaluation per key: extended slot e (counted), and the packed id
// b | sid << PK_B_BITS (PK_EQ for equality keys) stored at the key's position
// in the body.  sid = sub + j, sub the key's level-1 sub-bucket and j its
// interval between the bucket's heavy values: sub is non-decreasing in the key
// and the heavy values split the key order, so sid is an order-preserving id
// of the pair (j, sub) in [0, kf + nh).
// Two instantiations, launched back to back: HASHED handles calls whose
// heavy table is present (decided on the device by training), the other the
// rest; each returns at once when the call is not its kind.  In a call
// without heavy values the other one streams the chunk's keys through shared
// memory in double-buffered TMA tiles (the copy of the next tile overlaps the
// model evaluation of the current one).
template <int DT, bool HASHED>
__global__ void __launch_bounds__(H_THREADS, 1) k_l0_hist(Level0Args a, L0Layout lay) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  extern __shared__ __align__(128) unsigned char sm[];
  BucketHead* heads = (BucketHead*)(sm + lay.heads);
  uint32_t* cnt = (uint32_t*)(sm + lay.cnt);
  uint64_t* heavy = (uint64_t*)(sm + lay.htk);
  const U* keys = (const U*)a.keys;
  // compaction target: scratch, indexed like the ids (body-relative, so that every
  // chunk starts 16-byte aligned whatever the caller's pointer; head and tail
  // after the body)
  U* keys_w = (U*)a.scratch;
  uint32_t* pk = a.pk;
  const uint32_t next = min(a.M.hdr->n_ext, a.n_ext_max);
  const uint32_t H = min(a.M.hdr->nheavy, (next - a.f0) / 2);
  const uint32_t g = blockIdx.x;
  const uint64_t a0 = a.c.a0, nb = a.c.a1 - a.c.a0;
  const bool hashed = lay.hkey != NOT_SHARED && a.M.hdr->hash_probes > 0;
  if (hashed != HASHED) return;
  uint64_t cb, ce;
  chunk_of(a.c, g, &cb, &ce);
  const L0Map q = load_tables(a, sm, lay, H);
  for (uint32_t i = threadIdx.x; i < next; i += H_THREADS) cnt[i] = 0;
  // Compaction (equality keys dominate): the chunk's non-equality keys and
  // their ids are packed to the front of the chunk's range of scratch, so that
  // K4 reads only those (and writes its buckets back into the caller's array).
  const bool compact = a.may_compact && a.M.hdr->compact != 0;
  uint32_t* s_cpos = (uint32_t*)(sm + lay.ws);  // chunk lengths < 2^32
  if (threadIdx.x == 0) *s_cpos = 0;
  __syncthreads();
  if (g == 0) {  // unaligned head and tail: ids after the body
    const uint64_t nht = a0 + (a.c.n - a.c.a1);
    for (uint64_t k = threadIdx.x; k < nht; k += H_THREADS) {
      const uint64_t i = k < a0 ? k : a.c.a1 + (k - a0);
      uint32_t p;
      const U x = keys[i];
      const uint32_t e = classify_key<DT>(x, q, heads, heavy, lay.hs, a.f0kf, a.kf, &p);
      if (e < next) atomicAdd(&cnt[e], 1u); else set_error(a.err, ERR_BOUNDS);
      pk[nb + k] = p;
      if (compact) keys_w[nb + k] = x;  // K4 reads every key from scratch
    }
  }
  if (!HASHED && H == 0 && lay.tiles != NOT_SHARED) {
    // body chunk [cb, ce): 16-byte aligned, a multiple of 4 keys (as is every
    // tile), so each tile is one bulk copy
    TileStream<U, H_TILE> ts;
    ts.buf = (U*)(sm + lay.tiles);
    ts.bar = (uint64_t*)(sm + lay.bar);
    ts.src = keys + cb;
    ts.len = ce - cb;
    ts.nt = (uint32_t)((ts.len + H_TILE - 1) / H_TILE);
    if (threadIdx.x == 0) ts.init();
    __syncthreads();
    if (threadIdx.x == 0) { ts.issue(0); ts.issue(1); }
    for (uint32_t t = 0; t < ts.nt; ++t) {
      const U* tb = ts.wait(t, a.err);
      const uint32_t c = ts.count(t);
      uint32_t* pko = pk + (cb - a0) + (uint64_t)t * H_TILE;
      // every key of the step is classified before any counter is touched, so
      // that the table lookups of the thread's keys overlap (a shared-memory
      // atomic between them would order the loads)
      uint32_t ee[HT_KPT], pp[HT_KPT];
#pragma unroll
      for (int k = 0; k < HT_KPT; ++k) {
        const uint32_t i = k * H_THREADS + threadIdx.x;
        ee[k] = classify_plain<DT>(tb[i < c ? i : 0], q, a.f0kf, a.kf, &pp[k]);
      }
#pragma unroll
      for (int k = 0; k < HT_KPT; ++k) {
        const uint32_t i = k * H_THREADS + threadIdx.x;
        if (i < c) {
          if (ee[k] < next) atomicAdd(&cnt[ee[k]], 1u); else set_error(a.err, ERR_BOUNDS);
          pko[i] = pp[k];
        }
      }
      __syncthreads();  // every thread is done with buffer t & 1 before it is refilled
      if (threadIdx.x == 0) ts.issue(t + 2);
    }
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < a.n_ext_max; e += H_THREADS)
      a.hist[(size_t)e * a.c.G + g] = e < next ? cnt[e] : 0u;
    return;
  }
  const int lane = threadIdx.x & 31;
  // Heavy table path: a key equal to a heavy value is counted from one table
  // probe; the others queue per warp (QCAP entries) and take the full lookup
  // 32 at a time, so the lanes stay converged.
  const uint64_t* hk = (const uint64_t*)(sm + (hashed ? lay.hkey : 0));
  const uint16_t* hv = (const uint16_t*)(sm + (hashed ? lay.hval : 0));
  const int wid = threadIdx.x >> 5;
  U* qk = (U*)(sm + (hashed ? lay.queue : 0)) + (size_t)wid * QCAP;
  uint32_t* qi = (uint32_t*)(sm + (hashed ? lay.queue : 0) + (size_t)(H_THREADS / 32) * QCAP * sizeof(U)) +
                 (size_t)wid * QCAP;
  const unsigned lt = lanemask_lt();
  // Chunk-relative 32-bit positions (chunk lengths < 2^32).
  const U* kc = keys + cb;
  uint32_t* pkc = pk + (cb - a0);
  const uint32_t len = (uint32_t)(ce - cb);
  U* kwc = keys_w + (cb - a0);
  // full lookup of `valid` lanes' keys, then count and place the id
  auto finish = [&](bool valid, U x, uint32_t ri) {
    uint32_t pv = PK_EQ;
    if (valid) {
      const uint32_t e = classify_key<DT>(x, q, heads, heavy, lay.hs, a.f0kf, a.kf, &pv);
      if (e < next) atomicAdd(&cnt[e], 1u); else set_error(a.err, ERR_BOUNDS);
      if (!compact) pkc[ri] = pv;
    }
    if (compact) {
      const bool keep = valid && pv != PK_EQ;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      uint32_t wb = 0;
      if (lane == 0 && m) wb = atomicAdd(s_cpos, (uint32_t)__popc(m));
      wb = __shfl_sync(0xffffffffu, wb, 0);
      if (keep) {
        const uint32_t r = wb + __popc(m & lt);
        kwc[r] = x;
        pkc[r] = pv;
      }
    }
  };
  uint32_t nq = 0;  // the warp's queued misses, carried from step to step
  for (uint32_t base = 0; base < len; base += H_THREADS * H_KPT) {
    U u[H_KPT];
#pragma unroll
    for (int k = 0; k < H_KPT; ++k) {
      const uint32_t ri = base + k * H_THREADS + threadIdx.x;
      u[k] = ri < len ? kc[ri] : (U)0;
    }
    if (!HASHED) {  // every key takes the full lookup; the chains interleave
      uint32_t pp[H_KPT];
#pragma unroll
      for (int k = 0; k < H_KPT; ++k) {
        const uint32_t ri = base + k * H_THREADS + threadIdx.x;
        pp[k] = PK_EQ;
        if (ri < len) {
          const uint32_t e = classify_key<DT>(u[k], q, heads, heavy, lay.hs, a.f0kf, a.kf, &pp[k]);
          if (e < next) atomicAdd(&cnt[e], 1u); else set_error(a.err, ERR_BOUNDS);
          if (!compact) pkc[ri] = pp[k];
        }
      }
      if (compact) {
#pragma unroll
        for (int k = 0; k < H_KPT; ++k) {
          const bool keep = pp[k] != PK_EQ;
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          uint32_t wb = 0;
          if (lane == 0 && m) wb = atomicAdd(s_cpos, (uint32_t)__popc(m));
          wb = __shfl_sync(0xffffffffu, wb, 0);
          if (keep) {
            const uint32_t r = wb + __popc(m & lt);
            kwc[r] = u[k];
            pkc[r] = pp[k];
          }
        }
      }
      continue;
    }
#pragma unroll
    for (int k = 0; k < H_KPT; ++k) {
      const uint32_t ri = base + k * H_THREADS + threadIdx.x;
      bool miss = false;
      if (ri < len) {
        // one 8-byte probe: a hit is a heavy value; anything else (including a
        // heavy value that lost its slot) takes the full lookup (free slots
        // hold keys of other slots, so only a table key matches)
        const uint64_t bits = (uint64_t)u[k];
        const uint32_t slot = heavy_hash(bits);
        const uint32_t e = hk[slot] == bits ? (uint32_t)hv[slot] : 0xFFFFFFFFu;
        if (e != 0xFFFFFFFFu) {  // equality key: counted, never moved
          if (e < next) atomicAdd(&cnt[e], 1u); else set_error(a.err, ERR_BOUNDS);
          if (!compact) pkc[ri] = PK_EQ;
        } else {
          miss = true;
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, miss);
      if (miss) {
        const uint32_t pos = nq + __popc(m & lt);
        qk[pos] = u[k];
        qi[pos] = ri;
      }
      nq += __popc(m);
      if (nq >= 32) {
        __syncwarp();
        const U x = qk[lane];
        const uint32_t xi = qi[lane];
        U y = (U)0;
        uint32_t yi = 0;
        if (lane < nq - 32) { y = qk[32 + lane]; yi = qi[32 + lane]; }
        __syncwarp();
        if (lane < nq - 32) { qk[lane] = y; qi[lane] = yi; }
        nq -= 32;
        finish(true, x, xi);
        __syncwarp();
      }
    }
  }
  if (nq) {  // the last queued misses
    __syncwarp();
    const bool v = lane < nq;
    finish(v, v ? qk[lane] : (U)0, v ? qi[lane] : 0u);
    __syncwarp();
  }
  __syncthreads();
  if (compact) {  // pad to a multiple of 4 entries (equality marks)
    const uint64_t cpos = *s_cpos;  // (read after the loop's last barrier)
    const uint64_t r4 = (cpos + 3) & ~3ull;
    if (threadIdx.x < r4 - cpos) pk[cb - a0 + cpos + threadIdx.x] = PK_EQ;
    if (threadIdx.x == 0) a.ccount[g] = r4;
  }
  __syncthreads();
  for (uint32_t e = threadIdx.x; e < a.n_ext_max; e += H_THREADS)
    a.hist[(size_t)e * a.c.G + g] = e < next ? cnt[e] : 0u;
}

// ---------------------------------------------------------------- K4
// Key tiles and their packed ids stream in by TMA (double buffered).  Every
// non-equality key moves to its level-0 bucket: a bucket's non-equality keys
// gather at the start of the bucket's range in scratch, in chunk order (a
// bucket with heavy values is split between its intervals by level 1).  Per
// tile: each key's rank inside its bucket (shared atomics), an exclusive scan
// over the buckets gives the staging offsets, keys are staged
// bucket-contiguously and written out so that consecutive threads write
// consecutive addresses of a run; the level-1 ids follow their keys.
// Equality keys are skipped (their slots are filled later).
template <int DT, int TILE>
__global__ void __launch_bounds__(P_THREADS, 1) k_l0_scatter(Level0Args a, L0Layout lay) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr int KPT = TILE / P_THREADS;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = (uint64_t*)(sm + lay.bar);
  U* buf = (U*)(sm + lay.buf);
  uint32_t* pbuf = (uint32_t*)(sm + lay.pbuf);
  uint32_t* ecnt = (uint32_t*)(sm + lay.ecnt);
  uint32_t* soff = (uint32_t*)(sm + lay.soff);
  uint64_t* cursor = (uint64_t*)(sm + lay.cursor);
  uint64_t* gbase = (uint64_t*)(sm + lay.gbase);  // output of staged position s of bucket b: gbase[b] + s
  uint16_t* sinfo = (uint16_t*)(sm + lay.sinfo);   // staged keys' buckets
  uint16_t* sid = (uint16_t*)(sm + lay.sid);       // staged level-1 ids
  uint32_t* ws = (uint32_t*)(sm + lay.ws);
  // a failed scan (a wait that gave up) leaves the write heads unusable
  if (call_failed(a.err)) return;
  // input: the caller's array, or scratch where K2 compacted the chunks
  const bool compact = a.may_compact && a.M.hdr->compact;
  const U* keys = (const U*)a.keys;
  U* out = (U*)(compact ? a.keys : a.scratch);
  uint16_t* oid = a.sid;
  const uint64_t n = a.c.n;
  const uint32_t next = min(a.M.hdr->n_ext, a.n_ext_max);
  const uint32_t nc = a.f0;  // buckets
  const uint32_t g = blockIdx.x, G = a.c.G;
  const uint64_t a0 = a.c.a0, nb = a.c.a1 - a.c.a0;
  uint64_t cb, ce;
  chunk_of(a.c, g, &cb, &ce);
  if (compact) ce = cb + min(ce - cb, a.ccount[g]);  // packed keys
  // the body's first key: in the caller's array, or body-relative in scratch
  const U* body = compact ? (const U*)a.scratch : keys + a0;
  const uint32_t nt = (uint32_t)((ce - cb + TILE - 1) / TILE);
  auto tcount = [&](uint32_t t) {
    const uint64_t b = (uint64_t)t * TILE;
    return (uint32_t)min((uint64_t)TILE, ce - cb - b);
  };
  auto issue = [&](uint32_t t) {  // thread 0: keys and ids of tile t on one barrier
    if (t >= nt) return;
    const uint32_t c = tcount(t);
    uint64_t* br = bar + (t & 1);
    fence_proxy_async();
    mbar_arrive_expect_tx(br, c * (uint32_t)(sizeof(U) + 4));
    tma_load_1d_stream(buf + (size_t)(t & 1) * TILE, body + (cb - a0) + (size_t)t * TILE,
                       c * (uint32_t)sizeof(U), br);
    tma_load_1d_stream(pbuf + (size_t)(t & 1) * TILE, a.pk + (cb - a0) + (size_t)t * TILE, c * 4u,
                       br);
  };
  if (threadIdx.x == 0) { mbar_init(bar, 1); mbar_init(bar + 1, 1); fence_mbar_init(); }
  __syncthreads();
  if (threadIdx.x == 0) { issue(0); issue(1); }
  for (uint32_t i = threadIdx.x; i < nc; i += P_THREADS) ecnt[i] = 0;
  const BucketHead* heads = a.M.heads;
  // this chunk's place in bucket b: the bucket's start plus the non-equality
  // keys of b in earlier chunks (offs[e * G + g] - offs[e * G] over b's intervals)
  for (uint32_t b = threadIdx.x; b < nc; b += P_THREADS) {
    const BucketHead h = heads[b];
    const uint32_t nh = h.hoff_nh & 15u;
    uint64_t cur = h.ext_base < next ? a.offs[(size_t)h.ext_base * G] : n;
    for (uint32_t j = 0; j <= nh; ++j) {
      const uint32_t e = h.ext_base + 2 * j;
      if (e < next) cur += a.offs[(size_t)e * G + g] - a.offs[(size_t)e * G];
    }
    cursor[b] = cur;
  }
  __syncthreads();
  if (g == 0 && threadIdx.x == 0) {  // unaligned head and tail, one thread
    const uint64_t nht = a0 + (n - a.c.a1);
    for (uint64_t k = 0; k < nht; ++k) {
      const uint64_t i = k < a0 ? k : a.c.a1 + (k - a0);
      const uint32_t p = a.pk[nb + k];
      if (p == PK_EQ) continue;  // equality slot: filled later
      const uint32_t b = p & PK_B_MASK;
      if (b >= nc) { set_error(a.err, ERR_BOUNDS); continue; }
      const uint64_t dst = cursor[b]++;
      const U x = compact ? ((const U*)a.scratch)[nb + k] : keys[i];
      if (dst < n) { out[dst] = x; oid[dst] = (uint16_t)(p >> PK_B_BITS); }
      else set_error(a.err, ERR_BOUNDS);
    }
  }
  __syncthreads();
  for (uint32_t t = 0; t < nt; ++t) {
    mbar_wait(bar + (t & 1), (t >> 1) & 1, a.err);
    U* tb = buf + (size_t)(t & 1) * TILE;
    const uint32_t* pb = pbuf + (size_t)(t & 1) * TILE;
    const uint32_t cnt_t = tcount(t);
    U u[KPT];
    uint32_t pp[KPT], rk[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const uint32_t i = k * P_THREADS + threadIdx.x;
      u[k] = i < cnt_t ? tb[i] : (U)0;
      uint32_t p = i < cnt_t ? pb[i] : PK_EQ;
      if (p != PK_EQ && (p & PK_B_MASK) >= nc) { set_error(a.err, ERR_BOUNDS); p = PK_EQ; }
      pp[k] = p;
      rk[k] = p != PK_EQ ? atomicAdd(&ecnt[p & PK_B_MASK], 1u) : 0u;
    }
    __syncthreads();
    // the tile's bucket offsets; each bucket's output base moves past the tile
    uint32_t staged;
    {
      const uint32_t per = (nc + P_THREADS - 1) / P_THREADS;
      const uint32_t b0 = threadIdx.x * per;
      uint32_t sum = 0;
      for (uint32_t i = 0; i < per; ++i)
        if (b0 + i < nc) sum += ecnt[b0 + i];
      uint32_t run = block_excl_sum<uint32_t>(sum, ws, &staged);
      for (uint32_t i = 0; i < per; ++i) {
        const uint32_t b = b0 + i;
        if (b < nc) {
          const uint32_t c = ecnt[b];
          soff[b] = run;
          gbase[b] = cursor[b] - run;  // (mod 2^64)
          cursor[b] += c;
          ecnt[b] = 0;
          run += c;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; ++k) {  // stage bucket-contiguously
      if (pp[k] == PK_EQ) continue;
      const uint32_t b = pp[k] & PK_B_MASK;
      const uint32_t s = soff[b] + rk[k];
      if (s < (uint32_t)TILE) {
        tb[s] = u[k];
        sinfo[s] = (uint16_t)b;
        sid[s] = (uint16_t)(pp[k] >> PK_B_BITS);
      }
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < staged; s += P_THREADS) {
      const uint64_t dst = gbase[sinfo[s]] + s;
      if (dst < n) { out[dst] = tb[s]; oid[dst] = sid[s]; }
      else set_error(a.err, ERR_BOUNDS);
    }
    __syncthreads();
    if (threadIdx.x == 0) issue(t + 2);
  }
}

// ---------------------------------------------------------------- classify level 0
// Per extended slot: an equality slot becomes a fill job; the non-equality
// keys of a bucket without heavy values are sorted (or refined) where they
// are; those of a bucket with heavy values (gathered at the bucket's start in
// scratch) always take one level-1 job, which spreads them over the bucket's
// intervals.
template <int DT>
__global__ void k_classify0(Level0Args a, Lists lists, SortLimits lim) {
  pdl_begin();
  // after a failed level-0 step no job is made, so every later kernel of the
  // call finds empty lists (the keys are then unspecified, but every access
  // stays in bounds)
  if (call_failed(a.err)) return;
  const uint32_t next = min(a.M.hdr->n_ext, a.n_ext_max);
  const uint32_t G = a.c.G;
  const BucketHead* heads = a.M.heads;
  const HeavyEntry* heavy = a.M.heavy;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < next; e += gridDim.x * blockDim.x) {
    const uint64_t start = a.offs[(size_t)e * G];
    const uint64_t end = a.offs[(size_t)(e + 1) * G];
    uint32_t lo = 0, hi = a.f0;  // last b with ext_base <= e
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (heads[mid].ext_base <= e) lo = mid; else hi = mid - 1;
    }
    const uint32_t b = lo;
    const BucketHead h = heads[b];
    const uint32_t o = e - h.ext_base, nh = h.hoff_nh & 15u, hoff = h.hoff_nh >> 4;
    Job job;
    job.value = 0;
    job.src = (a.in_place || (a.may_compact && a.M.hdr->compact)) ? 0u : 1u;  // where level 0 put the keys
    job.pad = 0;
    job.kb = job.sb = 0;
    job.la = b;
    job.lb = 0;
    if (nh && (o & 1u)) {
      if (end <= start) continue;
      job.start = start;
      job.m = job.span = end - start;
      job.kind = JOB_FILL;
      job.value = (uint64_t)KT<DT>::from_tk(heavy[hoff + o / 2].tk);
      push_job(job.m >= FILL_BIG ? lists.fill_big : lists.fill, job, a.err);
      continue;
    }
    if (nh) {  // the bucket's non-equality keys, one job from its first slot
      if (o != 0) continue;
      uint64_t m = 0;
      for (uint32_t j = 0; j <= nh; ++j) {
        const uint32_t ej = e + 2 * j;
        if (ej < next) m += a.offs[(size_t)(ej + 1) * G] - a.offs[(size_t)ej * G];
      }
      if (m == 0) continue;
      const uint32_t eend = min(e + 2 * nh + 1, next);
      job.start = start;
      job.m = m;
      job.span = a.offs[(size_t)eend * G] - start;
      job.lb = nh;
      job.kind = JOB_REFINE;
      push_job(lists.refine, job, a.err);
      continue;
    }
    if (end <= start) continue;
    const uint64_t size = end - start;
    job.start = start;
    job.m = job.span = size;
    if (size <= lim.c_tiny) { job.kind = JOB_SORT; push_job(lists.sort_t, job, a.err); }
    else if (size <= lim.c_small) { job.kind = JOB_SORT; push_job(lists.sort_s, job, a.err); }
    else if (size <= lim.c_mid0) { job.kind = JOB_SORT; push_job(lists.sort_m0, job, a.err); }
    else if (size <= lim.c_mid) { job.kind = JOB_SORT; push_job(lists.sort_m, job, a.err); }
    else if (size <= lim.c_large) { job.kind = JOB_SORT; push_job(lists.sort_l, job, a.err); }
    else { job.kind = JOB_REFINE; push_job(lists.refine, job, a.err); }
  }
}

// ---------------------------------------------------------------- equality fill
// Large jobs are written by the whole grid, small ones by one CTA each (round
// robin), so thousands of small equality slots still fill in parallel; the
// 16-byte aligned body of a job is written with vector stores.
template <typename U>
__device__ __forceinline__ void fill_range(U* dst, uint64_t m, U v, uint64_t tid, uint64_t stride) {
  constexpr uint32_t V = 16 / sizeof(U);
  uint64_t head = ((16 - ((uintptr_t)dst & 15)) & 15) / sizeof(U);
  head = head < m ? head : m;
  const uint64_t body = (m - head) / V;
  const uint64_t tail0 = head + body * V;
  uint4 w;
  if (sizeof(U) == 8) {
    const uint64_t x = (uint64_t)v;
    w = make_uint4((uint32_t)x, (uint32_t)(x >> 32), (uint32_t)x, (uint32_t)(x >> 32));
  } else {
    const uint32_t x = (uint32_t)v;
    w = make_uint4(x, x, x, x);
  }
  uint4* vb = (uint4*)(dst + head);
  for (uint64_t i = tid; i < body; i += stride) vb[i] = w;
  const uint64_t ne = head + (m - tail0);
  for (uint64_t i = tid; i < ne; i += stride) dst[i < head ? i : tail0 + (i - head)] = v;
}

// Fill jobs are cut into units of FILL_UNIT keys and CTAs take units round
// robin (a unit's job found by bisection over the units' prefix, which every
// CTA scans for itself), so the stores spread evenly over the grid whatever
// the mix of job sizes.  More jobs than FILL_MAXJ: big jobs shared by the
// whole grid, small ones one CTA each.
constexpr uint32_t FILL_UNIT = 16384;
constexpr int FILL_MAXJ = 4096;

template <typename U>
__global__ void __launch_bounds__(256) k_fill(U* __restrict__ keys, JobList small, JobList big,
                                              const unsigned long long* __restrict__ from,
                                              const unsigned long long* __restrict__ upto) {
  pdl_begin();
  __shared__ uint32_t pre[FILL_MAXJ + 1];
  __shared__ uint32_t ws[33];
  // jobs [s0, s1) of `small` and [b0, b1) of `big`: from / upto hold {small, big}
  // positions (null: the list's start / its current count)
  const unsigned long long s1 = upto ? upto[0] : min(*small.count, small.cap);
  const unsigned long long b1 = upto ? upto[1] : min(*big.count, big.cap);
  const unsigned long long s0 = from ? min(from[0], s1) : 0ull;
  const unsigned long long b0 = from ? min(from[1], b1) : 0ull;
  const unsigned long long nb = b1 - b0, ns = s1 - s0;
  const unsigned long long nj = nb + ns;
  auto job_at = [&](unsigned long long j) -> const Job& {
    return j < nb ? big.jobs[b0 + j] : small.jobs[s0 + (j - nb)];
  };
  if (nj == 0) return;
  if (nj <= (unsigned long long)FILL_MAXJ) {
    for (uint32_t j = threadIdx.x; j < nj; j += blockDim.x)
      pre[j] = (uint32_t)((job_at(j).m + FILL_UNIT - 1) / FILL_UNIT);
    __syncthreads();
    const uint32_t T = block_scan_array<uint32_t>(pre, (int)nj, ws);  // exclusive, in place
    if (threadIdx.x == 0) pre[nj] = T;
    __syncthreads();
    for (uint32_t u = blockIdx.x; u < T; u += gridDim.x) {
      uint32_t lo = 0, hi = (uint32_t)nj - 1;  // last j with pre[j] <= u
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= u) lo = mid; else hi = mid - 1;
      }
      const Job& job = job_at(lo);
      const uint64_t off = (uint64_t)(u - pre[lo]) * FILL_UNIT;
      const uint64_t m = min((uint64_t)FILL_UNIT, job.m - off);
      fill_range<U>(job_keys(job, keys) + job.start + off, m, (U)job.value, threadIdx.x, blockDim.x);
    }
    return;
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (unsigned long long j = 0; j < nb; ++j) {
    const Job job = big.jobs[b0 + j];
    fill_range<U>(job_keys(job, keys) + job.start, job.m, (U)job.value, gtid, stride);
  }
  for (unsigned long long j = blockIdx.x; j < ns; j += gridDim.x) {
    const Job job = small.jobs[s0 + j];
    fill_range<U>(job_keys(job, keys) + job.start, job.m, (U)job.value, threadIdx.x, blockDim.x);
  }
}

// ---------------------------------------------------------------- level 1
__global__ void __launch_bounds__(1024)
k_l1_plan(LevelArgs la, SortLimits lim, Level1Ws w, uint32_t* err) {
  pdl_begin();
  __shared__ uint64_t ws[33];
  __shared__ uint64_t s_rt, s_rc;
  // this level's look-back words start at zero (cleared here rather than by a
  // memset between kernels); the scan runs two launches later
  for (size_t i = threadIdx.x; i < w.scan_status_bytes / 4; i += blockDim.x)
    ((uint32_t*)w.scan_status)[i] = 0u;
  L1Aux* aux = (L1Aux*)w.aux;
  const uint64_t nj = min((uint64_t)*la.in.count, min((uint64_t)la.in.cap, w.cap_jobs));
  if (threadIdx.x == 0) { s_rt = 0; s_rc = 0; }
  __syncthreads();
  for (uint64_t j0 = 0; j0 < nj; j0 += blockDim.x) {
    const uint64_t j = j0 + threadIdx.x;
    uint64_t tiles = 0, f1 = 0;
    if (j < nj) {
      Job job = la.in.jobs[j];
      // the model's split has the call's Kf sub-buckets per bucket (ids from
      // K2, plus one per heavy value's interval); a range split aims at
      // la.target keys per sub-bucket, at most la.fmax of them
      const uint64_t tg = (la.mode && job.pad) ? job.pad : (la.target ? la.target : 1);
      const uint64_t fmx = la.fmax ? min((uint64_t)la.fmax, (uint64_t)MAX_F1) : (uint64_t)MAX_F1;
      uint64_t f = (job.m + tg - 1) / tg;
      f = f < 2 ? 2 : (f > fmx ? fmx : f);
      if (la.mode == 0) f = la.kf + job.lb;  // ids sub + interval
      f1 = f;
      tiles = (job.m + L1_TILE - 1) / L1_TILE;
      w.jmin[j] = ~0ull;
      w.jmax[j] = 0ull;
    }
    uint64_t tt, tc;
    const uint64_t et = block_excl_sum<uint64_t>(tiles, ws, &tt);
    const uint64_t ec = block_excl_sum<uint64_t>(f1, ws, &tc);
    if (j < nj) {
      L1Aux x;
      x.tile_base = s_rt + et;
      x.cbase = s_rc + ec;
      x.pad0 = 0;
      x.f1 = (uint32_t)f1;
      x.pad = 0;
      aux[j] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_rt += tt; s_rc += tc; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    L1Aux x{};
    x.tile_base = s_rt;
    x.cbase = s_rc;
    aux[nj] = x;
    if (s_rc > w.cap_c) set_error(err, ERR_BOUNDS);
    w.totals[0] = s_rt;
    w.totals[1] = s_rc > w.cap_c ? w.cap_c : s_rc;
    w.totals[2] = nj;
    w.totals[3] = 0;  // job counter of the in-place split
    w.totals[4] = 0;  // its hole counter
    w.totals[5] = 0;  // job counter of its split by known destinations
  }
  // the level's sub-bucket counters (only the ones its jobs use) start at zero
  const uint64_t C = min((uint64_t)s_rc, w.cap_c);
  for (uint64_t i = threadIdx.x; i < C; i += blockDim.x) w.cnt[i] = 0;
}

// The tiles of a level are dealt to the CTAs in contiguous ranges: a CTA finds
// its first tile's job by bisection, then steps from job to job.
struct TileWalk {
  uint64_t t, t1, j, nbase;
};
__device__ __forceinline__ bool tile_walk_begin(const L1Aux* aux, uint64_t T, uint64_t nj,
                                                TileWalk& w) {
  const uint64_t per = (T + gridDim.x - 1) / gridDim.x;
  w.t = blockIdx.x * per;
  w.t1 = min(T, w.t + per);
  if (w.t >= w.t1) return false;
  w.j = aux_find_tile(aux, nj, w.t);
  w.nbase = aux[w.j + 1].tile_base;  // aux[nj] is the end sentinel
  return true;
}
__device__ __forceinline__ void tile_walk_job(const L1Aux* aux, TileWalk& w) {
  while (w.t >= w.nbase) { ++w.j; w.nbase = aux[w.j + 1].tile_base; }
}

// Total-order key range of every job of a range level (one atomic pair per tile).
template <int DT>
__global__ void __launch_bounds__(L1_THREADS, 4)
k_l1_minmax(const typename KT<DT>::U* keys, const typename KT<DT>::U* scratch, LevelArgs la,
            Level1Ws w) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  __shared__ unsigned long long s_min, s_max;
  const L1Aux* aux = (const L1Aux*)w.aux;
  const uint64_t T = w.totals[0], nj = w.totals[2];
  const int lane = threadIdx.x & 31;
  TileWalk tw;
  if (!tile_walk_begin(aux, T, nj, tw)) return;
  for (; tw.t < tw.t1; ++tw.t) {
    tile_walk_job(aux, tw);
    const uint64_t t = tw.t, j = tw.j;
    const Job job = la.in.jobs[j];
    const uint64_t off = (t - aux[j].tile_base) * L1_TILE;
    const uint32_t c = (uint32_t)min((uint64_t)L1_TILE, job.m - off);
    const U* src = (job.src ? job_scratch(job, scratch) : job_keys(job, keys)) + job.start + off;
    if (threadIdx.x == 0) { s_min = ~0ull; s_max = 0; }
    __syncthreads();
    unsigned long long mn = ~0ull, mx = 0;
    for (uint32_t i = threadIdx.x; i < c; i += blockDim.x) {
      const unsigned long long tk = KT<DT>::tk(src[i]);
      mn = min(mn, tk);
      mx = max(mx, tk);
    }
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) { atomicMin(&s_min, mn); atomicMax(&s_max, mx); }
    __syncthreads();
    if (threadIdx.x == 0) { atomicMin(&w.jmin[j], s_min); atomicMax(&w.jmax[j], s_max); }
    __syncthreads();
  }
}

template <int DT>
__global__ void __launch_bounds__(L1_THREADS, 4)
k_l1_hist(const typename KT<DT>::U* keys, const typename KT<DT>::U* scratch, ModelPtrs M,
          LevelArgs la, Level1Ws w) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  __shared__ uint32_t hc[MAX_F1];
  const L1Aux* aux = (const L1Aux*)w.aux;
  const uint64_t T = w.totals[0], nj = w.totals[2];
  TileWalk tw;
  if (!tile_walk_begin(aux, T, nj, tw)) return;
  // The CTA's consecutive tiles of one job form one span, counted into one
  // shared histogram that is added to the job's counters once.
  while (tw.t < tw.t1) {
    tile_walk_job(aux, tw);
    const uint64_t j = tw.j;
    const L1Aux x = aux[j];
    const Job job = la.in.jobs[j];
    const uint64_t te = min(tw.t1, tw.nbase);
    const uint64_t off = (tw.t - x.tile_base) * (uint64_t)L1_TILE;
    const uint64_t c = min((te - x.tile_base) * (uint64_t)L1_TILE, job.m) - off;
    tw.t = te;
    const U* src = (job.src ? job_scratch(job, scratch) : job_keys(job, keys)) + job.start + off;
    const uint16_t* ids = w.sid + job.start + off;
    RangeSplit rs{};
    if (la.mode) rs = range_split<DT>(w.jmin[j], w.jmax[j], x.f1, la.mode == 2);
    for (uint32_t s = threadIdx.x; s < x.f1; s += blockDim.x) hc[s] = 0;
    __syncthreads();
    if (la.mode) {
      constexpr int U8 = 8;  // independent loads in flight per thread
      for (uint64_t base = 0; base < c; base += blockDim.x * U8) {
        uint32_t sub[U8];
#pragma unroll
        for (int k = 0; k < U8; ++k) {
          const uint64_t i = base + k * blockDim.x + threadIdx.x;
          sub[k] = i < c ? range_sub<DT>(src[i], rs) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int k = 0; k < U8; ++k)
          if (sub[k] != 0xFFFFFFFFu) atomicAdd(&hc[sub[k]], 1u);
      }
    } else {  // the ids: 8 per 16-byte load over the span's aligned body, 4 loads in flight
      constexpr int UV = 4;
      const uint32_t f1m = x.f1 - 1;
      const uint64_t h = min(c, (uint64_t)((((16 - ((uintptr_t)ids & 15)) & 15)) >> 1));
      const uint64_t nv = (c - h) >> 3;
      const uint4* v = (const uint4*)(ids + h);
      for (uint64_t q0 = threadIdx.x; q0 < nv; q0 += UV * blockDim.x) {
        uint4 x4[UV];
#pragma unroll
        for (int r = 0; r < UV; ++r) {
          const uint64_t q = q0 + r * blockDim.x;
          x4[r] = q < nv ? v[q] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int r = 0; r < UV; ++r) {
          if (q0 + r * blockDim.x >= nv) break;
          const uint32_t wv[4] = {x4[r].x, x4[r].y, x4[r].z, x4[r].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            atomicAdd(&hc[min(wv[e] & 0xFFFFu, f1m)], 1u);
            atomicAdd(&hc[min(wv[e] >> 16, f1m)], 1u);
          }
        }
      }
      const uint64_t t0 = h + (nv << 3), ne = h + (c - t0);  // head, then tail
      for (uint64_t i = threadIdx.x; i < ne; i += blockDim.x)
        atomicAdd(&hc[min((uint32_t)ids[i < h ? i : t0 + (i - h)], f1m)], 1u);
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < x.f1; s += blockDim.x)
      if (hc[s]) atomicAdd(&w.cnt[x.cbase + s], hc[s]);
    __syncthreads();
  }
}

// First output position of every sub-bucket.  A level-0 bucket with heavy
// values has ids sub + j over its intervals j; interval j's ids start at
// sub(h_{j-1}) + j (h the bucket's heavy values, sub(h) from their stored F
// exactly as the level-0 pass computes a key's), and its keys start where the
// level-0 offsets put the interval.
__global__ void k_l1_cursor(LevelArgs la, Level1Ws w, ModelPtrs M) {
  pdl_begin();
  const L1Aux* aux = (const L1Aux*)w.aux;
  const uint64_t C = w.totals[1], nj = w.totals[2];
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < C;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = aux_find_c(aux, nj, c);
    const Job job = la.in.jobs[j];
    const uint64_t cbase = aux[j].cbase;
    uint64_t first = cbase, dst0 = job.start;
    if (la.mode == 0 && job.lb) {
      const uint32_t b = job.la, cc = (uint32_t)(c - cbase);
      const BucketHead h = M.heads[b];
      const uint32_t hoff = h.hoff_nh >> 4;
      uint32_t iv = 0, f = 0;
      for (uint32_t i = 0; i < job.lb; ++i) {
        const float wv = M.heavy[hoff + i].F * la.f0kf;
        int sub = (wv >= 0.0f ? (int)wv : 0) - (int)(b * la.kf);
        sub = sub < 0 ? 0 : (sub >= (int)la.kf ? (int)la.kf - 1 : sub);
        const uint32_t hs = (uint32_t)sub + i + 1;  // first id of interval i + 1
        if (hs <= cc) { iv = i + 1; f = hs; }
      }
      first = cbase + f;
      dst0 = la.l0offs[(size_t)(h.ext_base + 2 * iv) * la.l0G];
    }
    w.cur[c] = dst0 + (w.off[c] - w.off[first]);
  }
}

// Moves the keys of every refine job into its sub-buckets, from the buffer
// the job lives in to the other one (keys <-> scratch), same positions.
static_assert(MAX_F1 <= 1024 && L1_TILE <= (1 << 22), "sub | rank << 10 packing of the level-1 scatter");
template <int DT>
__global__ void __launch_bounds__(L1_THREADS, 3)
k_l1_scatter(typename KT<DT>::U* keys, typename KT<DT>::U* scratch, uint64_t n, ModelPtrs M,
             LevelArgs la, Level1Ws w, uint32_t* err) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  constexpr int KPT = L1_TILE / L1_THREADS;
  __shared__ uint32_t lc[MAX_F1 + 1];
  __shared__ unsigned long long gp[MAX_F1];
  __shared__ uint32_t ws[33];
  extern __shared__ __align__(16) unsigned char dsm[];
  U* stage = (U*)dsm;                                      // L1_TILE keys
  uint16_t* ids = (uint16_t*)(dsm + sizeof(U) * L1_TILE);  // L1_TILE slot ids
  const L1Aux* aux = (const L1Aux*)w.aux;
  const uint64_t T = w.totals[0], nj = w.totals[2];
  TileWalk tw;
  if (!tile_walk_begin(aux, T, nj, tw)) return;
  for (; tw.t < tw.t1; ++tw.t) {
    tile_walk_job(aux, tw);
    const uint64_t t = tw.t, j = tw.j;
    if (w.jmin[j] == w.jmax[j]) continue;  // homogeneous: filled, not moved
    const L1Aux x = aux[j];
    const Job job = la.in.jobs[j];
    const uint64_t off = (t - x.tile_base) * L1_TILE;
    const uint32_t c = (uint32_t)min((uint64_t)L1_TILE, job.m - off);
    const U* src = (job.src ? job_scratch(job, scratch) : job_keys(job, keys)) + job.start + off;
    const uint16_t* idsrc = w.sid + job.start + off;
    U* dstb = job.src ? job_keys(job, keys) : job_scratch(job, scratch);
    RangeSplit rs{};
    if (la.mode) rs = range_split<DT>(w.jmin[j], w.jmax[j], x.f1, la.mode == 2);
    for (uint32_t s = threadIdx.x; s <= x.f1; s += blockDim.x) lc[s] = 0;
    __syncthreads();
    U u[KPT];
    uint32_t sb[KPT];  // the id, then sub | rank << 10 (sub < MAX_F1 = 2^10, rank < L1_TILE)
#pragma unroll
    for (int k = 0; k < KPT; ++k) {  // all loads first, then the ranks
      const uint32_t i = k * L1_THREADS + threadIdx.x;
      u[k] = i < c ? src[i] : (U)0;
      sb[k] = i < c ? (la.mode ? 0u : (uint32_t)idsrc[i]) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      uint32_t sub = sb[k];
      if (sub != 0xFFFFFFFFu) {
        sub = la.mode ? range_sub<DT>(u[k], rs) : min(sub, x.f1 - 1);
        sb[k] = sub | (atomicAdd(&lc[sub], 1u) << 10);
      }
    }
    __syncthreads();
    block_scan_array<uint32_t>(lc, (int)x.f1, ws);
    if (threadIdx.x == 0) lc[x.f1] = c;
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < x.f1; s += blockDim.x) {
      const uint32_t cs = lc[s + 1] - lc[s];
      if (cs) gp[s] = atomicAdd(&w.cur[x.cbase + s], (unsigned long long)cs);
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (sb[k] != 0xFFFFFFFFu) {
        const uint32_t s = sb[k] & 1023u;
        const uint32_t p = lc[s] + (sb[k] >> 10);
        if (p < (uint32_t)L1_TILE) { stage[p] = u[k]; ids[p] = (uint16_t)s; }
      }
    }
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < c; p += blockDim.x) {
      const uint32_t s = ids[p];
      const uint64_t dst = gp[s] + (p - lc[s]);
      if (dst - job.start < job.span) dstb[dst] = stage[p]; else set_error(err, ERR_BOUNDS);
    }
    __syncthreads();
  }
}

template <int DT>
__global__ void k_l1_classify(Lists lists, LevelArgs la, SortLimits lim, Level1Ws w, ModelPtrs M,
                              int L, uint32_t* err) {
  pdl_begin();
  if (call_failed(err)) return;  // after a failed split no job is made
  const L1Aux* aux = (const L1Aux*)w.aux;
  const uint64_t C = w.totals[1], nj = w.totals[2];
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < C;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t cntc = la.in_place ? (uint64_t)w.cnt[c] : w.off[c + 1] - w.off[c];
    if (cntc == 0) continue;
    const uint64_t j = aux_find_c(aux, nj, c);
    const Job pj = la.in.jobs[j];
    Job job;
    job.value = 0;
    if (w.jmin[j] == w.jmax[j]) {  // all keys of the bucket are equal (Is-Homogeneous)
      job = pj;
      job.kind = JOB_FILL;
      job.value = (uint64_t)KT<DT>::from_tk(w.jmin[j]);
      push_job(job.m >= FILL_BIG ? lists.fill_big : lists.fill, job, err);
      continue;
    }
    job.start = w.cur[c] - cntc;  // the cursor ends past the sub-bucket's keys
    job.m = job.span = cntc;
    job.pad = 0;
    job.src = la.in_place ? pj.src : pj.src ^ 1u;  // split in place, or into the other buffer
    job.la = job.lb = 0;
    job.kb = pj.kb;
    job.sb = pj.sb;
    const uint32_t sk = la.mode ? JOB_SORT_RANGE : JOB_SORT;
    if (cntc <= lim.c_tiny) { job.kind = sk; push_job(lists.sort_t, job, err); }
    else if (cntc <= lim.c_small) { job.kind = sk; push_job(lists.sort_s, job, err); }
    else if (cntc <= lim.c_mid0) { job.kind = sk; push_job(lists.sort_m0, job, err); }
    else if (cntc <= lim.c_mid) { job.kind = sk; push_job(lists.sort_m, job, err); }
    else if (cntc <= lim.c_large) { job.kind = sk; push_job(lists.sort_l, job, err); }
    else { job.kind = la.next_kind; push_job(la.next, job, err); }
  }
}

// ---------------------------------------------------------------- host enqueue
template <int DT>
static cudaError_t level0_dt(const Level0Args& a, size_t sh, size_t ss, const Lists& lists,
                             const SortLimits& lim, cudaStream_t st, const Marks* mk, int mb) {
  const int W = KT<DT>::W;
  const uint32_t hmax = (a.n_ext_max - a.f0) / 2;
  const L0Layout lh = l0_layout_hist(W, a.L, a.f0, a.n_ext_max, hmax);
  const int tile = scatter_tile(W, a.f0, hmax);
  const L0Layout ls_ = l0_layout_scatter(W, a.f0, hmax, tile);
  launch_k(k_l0_hist<DT, false>, a.c.G, H_THREADS, sh, st, a, lh);
  if (lh.hkey != NOT_SHARED) launch_k(k_l0_hist<DT, true>, a.c.G, H_THREADS, sh, st, a, lh);
  mark(mk, mb + 0, st);
  const uint64_t M = (uint64_t)a.n_ext_max * a.c.G;
  launch_k(k_scan<uint32_t>, a.scan_tiles, SC_THREADS, 0, st, a.hist, a.offs, M, nullptr, (uint64_t*)a.scan_status,
      (uint32_t*)((uint64_t*)a.scan_status + a.scan_tiles), a.err, STALL_L0_SCAN);
  mark(mk, mb + 1, st);
  if (tile == P_TILE) launch_k(k_l0_scatter<DT, P_TILE>, a.c.G, P_THREADS, ss, st, a, ls_);
  else launch_k(k_l0_scatter<DT, P_TILE_SMALL>, a.c.G, P_THREADS, ss, st, a, ls_);
  mark(mk, mb + 2, st);
  launch_k(k_classify0<DT>, (a.n_ext_max + 255) / 256, 256, 0, st, a, lists, lim);
  mark(mk, mb + 3, st);
  add_launches(lh.hkey != NOT_SHARED ? 5 : 4);
  return cudaGetLastError();
}

static size_t l1_scatter_smem(int W) { return (size_t)L1_TILE * (W + 2); }

cudaError_t level0_configure(int dt, size_t sh, size_t ss) {
  cudaError_t e = cudaSuccess;
#define LS_CFG(D)                                                                               \
  e = cudaFuncSetAttribute(k_l0_hist<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh); \
  if (e) return e;                                                                              \
  e = cudaFuncSetAttribute(k_l0_hist<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh); \
  if (e) return e;                                                                              \
  e = cudaFuncSetAttribute(k_l1_scatter<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                           (int)l1_scatter_smem(KT<D>::W));                                     \
  if (e) return e;                                                                              \
  e = cudaFuncSetAttribute(k_l0_scatter<D, P_TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss); \
  if (e) return e;                                                                              \
  e = cudaFuncSetAttribute(k_l0_scatter<D, P_TILE_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
  switch (dt) {
    case LS_F64: LS_CFG(LS_F64); break;
    case LS_U64: LS_CFG(LS_U64); break;
    case LS_F32: LS_CFG(LS_F32); break;
    case LS_U32: LS_CFG(LS_U32); break;
  }
#undef LS_CFG
  return e;
}

cudaError_t level0_enqueue(int dt, const Level0Args& a, size_t sh, size_t ss, const Lists& lists,
                           const SortLimits& lim, cudaStream_t st, const Marks* mk, int mb) {
  switch (dt) {
    case LS_F64: return level0_dt<LS_F64>(a, sh, ss, lists, lim, st, mk, mb);
    case LS_U64: return level0_dt<LS_U64>(a, sh, ss, lists, lim, st, mk, mb);
    case LS_F32: return level0_dt<LS_F32>(a, sh, ss, lists, lim, st, mk, mb);
    case LS_U32: return level0_dt<LS_U32>(a, sh, ss, lists, lim, st, mk, mb);
  }
  return cudaErrorInvalidValue;
}

template <int DT>
static cudaError_t level_dt(void* keys, void* scratch, uint64_t n, const ModelPtrs& M,
                            const Lists& lists, const LevelArgs& la, const SortLimits& lim,
                            const Level1Ws& w, uint32_t* err, cudaStream_t st, int num_sms) {
  typedef typename KT<DT>::U U;
  launch_k(k_l1_plan, 1, 1024, 0, st, la, lim, w, err);
  const int grid = 4 * num_sms;  // the histogram and range passes hold 4 CTAs per SM
  if (la.mode) launch_k(k_l1_minmax<DT>, grid, L1_THREADS, 0, st, (const U*)keys, (const U*)scratch, la, w);
  launch_k(k_l1_hist<DT>, grid, L1_THREADS, 0, st, (const U*)keys, (const U*)scratch, M, la, w);
  const unsigned tiles = (unsigned)std::max<uint64_t>(1, (w.cap_c + SC_TILE - 1) / SC_TILE);
  launch_k(k_scan<uint32_t>, tiles, SC_THREADS, 0, st, w.cnt, w.off, w.cap_c, &w.totals[1],
           (uint64_t*)w.scan_status, (uint32_t*)((uint64_t*)w.scan_status + tiles), err, 0u);
  launch_k(k_l1_cursor, grid, 256, 0, st, la, w, M);
  // the scatter holds 3 CTAs per SM: one wave
  launch_k(k_l1_scatter<DT>, 3 * num_sms, L1_THREADS, l1_scatter_smem(KT<DT>::W), st, (U*)keys, (U*)scratch, n, M, la, w, err);
  launch_k(k_l1_classify<DT>, grid, 256, 0, st, lists, la, lim, w, M, M.L, err);
  add_launches(la.mode ? 7 : 6);
  return cudaGetLastError();
}

cudaError_t levels_enqueue(int dt, void* keys, void* scratch, uint64_t n, const ModelPtrs& M,
                           const Lists& lists, const SortLimits& lim, const Level1Ws& w,
                           const LevelArgs* lvs, int nlv, uint32_t* err, cudaStream_t st,
                           int num_sms) {
  for (int lv = 0; lv < nlv; ++lv) {
    const LevelArgs& la = lvs[lv];
    cudaError_t e = cudaErrorInvalidValue;
    switch (dt) {
      case LS_F64: e = level_dt<LS_F64>(keys, scratch, n, M, lists, la, lim, w, err, st, num_sms); break;
      case LS_U64: e = level_dt<LS_U64>(keys, scratch, n, M, lists, la, lim, w, err, st, num_sms); break;
      case LS_F32: e = level_dt<LS_F32>(keys, scratch, n, M, lists, la, lim, w, err, st, num_sms); break;
      case LS_U32: e = level_dt<LS_U32>(keys, scratch, n, M, lists, la, lim, w, err, st, num_sms); break;
    }
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t level1_enqueue(int dt, void* keys, void* scratch, uint64_t n, const ModelPtrs& M,
                           const Lists& lists, const SortLimits& lim, const Level1Ws& w,
                           uint32_t kf, float f0kf, const uint64_t* l0offs, uint32_t l0G,
                           uint32_t* err, cudaStream_t st, int num_sms, bool range_levels) {
  // level 1 splits by the model; levels 2 and 3 split what it could not by key
  // range (without them, level 1's leftovers go to the fallback)
  const JobList ins[3] = {lists.refine, lists.refine2, lists.refine3};
  const JobList outs[3] = {range_levels ? lists.refine2 : lists.fallback, lists.refine3,
                           lists.fallback};
  // re-splits of what the model left large: the value range first, then the
  // total-order key range (which separates clustered distinct values)
  LevelArgs lvs[3] = {};
  for (int lv = 0; lv < 3; ++lv) {
    lvs[lv].in = ins[lv];
    lvs[lv].next = outs[lv];
    lvs[lv].mode = lv == 0 ? 0 : (lv == 1 ? 2 : 1);
    lvs[lv].next_kind = (lv == 2 || !range_levels) ? JOB_FALLBACK : JOB_REFINE;
    lvs[lv].kf = kf;
    lvs[lv].target = lv == 2 ? 16 : lim.l1_target / 3;
    lvs[lv].fmax = lv == 2 ? 256 : MAX_F1;
    lvs[lv].l0offs = l0offs;
    lvs[lv].l0G = l0G;
    lvs[lv].f0kf = f0kf;
  }
  return levels_enqueue(dt, keys, scratch, n, M, lists, lim, w, lvs, range_levels ? 3 : 1, err, st,
                        num_sms);
}

cudaError_t launch_classify0(int dt, const Level0Args& a, const Lists& lists, const SortLimits& lim,
                             cudaStream_t st) {
  const unsigned g = (a.n_ext_max + 255) / 256;
  switch (dt) {
    case LS_F64: launch_k(k_classify0<LS_F64>, g, 256, 0, st, a, lists, lim); break;
    case LS_U64: launch_k(k_classify0<LS_U64>, g, 256, 0, st, a, lists, lim); break;
    case LS_F32: launch_k(k_classify0<LS_F32>, g, 256, 0, st, a, lists, lim); break;
    case LS_U32: launch_k(k_classify0<LS_U32>, g, 256, 0, st, a, lists, lim); break;
    default: return cudaErrorInvalidValue;
  }
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_l1_plan(const LevelArgs& la, const SortLimits& lim, const Level1Ws& w,
                           uint32_t* err, cudaStream_t st) {
  launch_k(k_l1_plan, 1, 1024, 0, st, la, lim, w, err);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_l1_minmax(int dt, const void* keys, const LevelArgs& la, const Level1Ws& w,
                             cudaStream_t st, int num_sms) {
  const int grid = 4 * num_sms;
  switch (dt) {
    case LS_F64: launch_k(k_l1_minmax<LS_F64>, grid, L1_THREADS, 0, st, (const uint64_t*)keys, (const uint64_t*)nullptr, la, w); break;
    case LS_U64: launch_k(k_l1_minmax<LS_U64>, grid, L1_THREADS, 0, st, (const uint64_t*)keys, (const uint64_t*)nullptr, la, w); break;
    case LS_F32: launch_k(k_l1_minmax<LS_F32>, grid, L1_THREADS, 0, st, (const uint32_t*)keys, (const uint32_t*)nullptr, la, w); break;
    case LS_U32: launch_k(k_l1_minmax<LS_U32>, grid, L1_THREADS, 0, st, (const uint32_t*)keys, (const uint32_t*)nullptr, la, w); break;
    default: return cudaErrorInvalidValue;
  }
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_l1_classify(int dt, const Lists& lists, const LevelArgs& la,
                               const SortLimits& lim, const Level1Ws& w, const ModelPtrs& M,
                               uint32_t* err, cudaStream_t st, int num_sms) {
  const int grid = 4 * num_sms;
  switch (dt) {
    case LS_F64: launch_k(k_l1_classify<LS_F64>, grid, 256, 0, st, lists, la, lim, w, M, M.L, err); break;
    case LS_U64: launch_k(k_l1_classify<LS_U64>, grid, 256, 0, st, lists, la, lim, w, M, M.L, err); break;
    case LS_F32: launch_k(k_l1_classify<LS_F32>, grid, 256, 0, st, lists, la, lim, w, M, M.L, err); break;
    case LS_U32: launch_k(k_l1_classify<LS_U32>, grid, 256, 0, st, lists, la, lim, w, M, M.L, err); break;
    default: return cudaErrorInvalidValue;
  }
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t fill_enqueue(int dt, void* keys, const Lists& lists, const unsigned long long* from,
                         const unsigned long long* upto, cudaStream_t st, int num_sms) {
  if (dt == LS_F64 || dt == LS_U64)
    launch_k(k_fill<uint64_t>, 4 * num_sms, 256, 0, st, (uint64_t*)keys, lists.fill, lists.fill_big, from, upto);
  else
    launch_k(k_fill<uint32_t>, 4 * num_sms, 256, 0, st, (uint32_t*)keys, lists.fill, lists.fill_big, from, upto);
  add_launches(1);
  return cudaGetLastError();
}

}  // namespace ls

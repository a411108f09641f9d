// In-bucket finish of LearnedSort 2.0 (Alg. 2): the model-based counting sort
// of each (sub-)bucket followed by the insertion-sort touch-up.
//
// One CTA per segment of m keys (m <= CAP) in shared memory:
//   slot(x) = clamp(floor((F(x) - Flo) * m / (Fhi - Flo)), 0, m - 1)
// evaluated per leaf with FP32 coefficients derived in FP64 for this segment
// (so the slot resolution is 1/m of the segment's eCDF range, not of [0,1]);
// histogram of slots -> exclusive scan (the running totals of Alg. 2) ->
// placement -> touch-up.  The slot map is monotone in the key, so keys of
// different slots are already in order and the touch-up only sorts each group
// of keys that share a slot: insertion sort (<= 8 keys, one thread), rank sort
// (<= 128, one warp) or a bitonic network over the group (one CTA).
//
// Segments the model cannot split below CAP keys go to the fallback: an LSD
// radix sort over the segment's varying total-order-key bytes, one CTA each.
#include <cfloat>

#include "ls_partition.cuh"
#include "ls_radix.cuh"
#include "ls_scan.cuh"

namespace ls {

constexpr int MAXL = 64;        // leaves with per-segment coefficients
constexpr int BIGCAP = 512;     // slot groups > 8 keys tracked per segment

struct Coef {
  float A, B, LO, HI;
  long long cq;
  int sh;
  int pad;
};

template <int DT, int THREADS, int KPT>
struct BucketCfg {
  typedef typename KT<DT>::U U;
  static constexpr int CAP = THREADS * KPT;
  static constexpr size_t OFF_OUT = 0;
  static constexpr size_t OFF_CNT = OFF_OUT + sizeof(U) * CAP;
  static constexpr size_t OFF_COEF = (OFF_CNT + 4 * (CAP + 1) + 15) / 16 * 16;
  static constexpr size_t OFF_BIG = OFF_COEF + sizeof(Coef) * MAXL;
  static constexpr size_t OFF_WS = OFF_BIG + 8 * BIGCAP;
  static constexpr size_t SMEM = OFF_WS + 8 * 40;
};

__device__ __forceinline__ float fp32_sat_d(double d) {
  if (d >= (double)FLT_MAX) return FLT_MAX;
  if (d <= -(double)FLT_MAX) return -FLT_MAX;
  return __double2float_rn(d);
}

template <int DT>
__device__ __forceinline__ void cmpswap(typename KT<DT>::U* a, uint32_t i, uint32_t j) {
  const typename KT<DT>::U x = a[i], y = a[j];
  if (KT<DT>::tk(x) > KT<DT>::tk(y)) { a[i] = y; a[j] = x; }
}

// Direction-free bitonic network over a[0..sz) with virtual +inf padding.
template <int DT>
__device__ void block_bitonic(typename KT<DT>::U* a, uint32_t sz) {
  uint32_t P = 1;
  while (P < sz) P <<= 1;
  for (uint32_t k = 2; k <= P; k <<= 1) {
    const uint32_t hk = k >> 1;
    for (uint32_t i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
      const uint32_t blk = i / hk, off = i % hk;
      const uint32_t lo = blk * k + off, hi = blk * k + k - 1 - off;
      if (hi < sz) cmpswap<DT>(a, lo, hi);
    }
    __syncthreads();
    for (uint32_t j = k >> 2; j >= 1; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
        const uint32_t blk = i / j, off = i % j;
        const uint32_t lo = blk * 2 * j + off, hi = lo + j;
        if (hi < sz) cmpswap<DT>(a, lo, hi);
      }
      __syncthreads();
    }
  }
}

template <int DT, int THREADS, int KPT>
__global__ void __launch_bounds__(THREADS)
k_bucket_sort(typename KT<DT>::U* keys, const typename KT<DT>::U* scratch, ModelPtrs M,
              JobList list, unsigned long long* ctr, uint32_t* err) {
  typedef typename KT<DT>::U U;
  typedef BucketCfg<DT, THREADS, KPT> C;
  extern __shared__ __align__(16) unsigned char sm[];
  U* out = (U*)(sm + C::OFF_OUT);
  uint32_t* cnt = (uint32_t*)(sm + C::OFF_CNT);
  Coef* coef = (Coef*)(sm + C::OFF_COEF);
  uint2* big = (uint2*)(sm + C::OFF_BIG);
  unsigned long long* ws = (unsigned long long*)(sm + C::OFF_WS);
  __shared__ unsigned long long s_job;
  __shared__ int s_lmin, s_lmax;
  __shared__ uint32_t s_nbig, s_all;
  __shared__ float s_S, s_T;
  __shared__ int s_mode;  // 0: per-leaf coefficients, 1: global F, 2: single slot
  const RootEval r = M.hdr->root;
  const int E = r.E;
  const unsigned long long nj = min(*list.count, list.cap);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  while (true) {
    if (threadIdx.x == 0) s_job = atomicAdd(ctr, 1ull);
    __syncthreads();
    const unsigned long long jid = s_job;
    if (jid >= nj) break;
    const Job job = list.jobs[jid];
    const uint32_t m = (uint32_t)job.m;
    if (job.m > (uint64_t)C::CAP) {  // classification guarantees m <= CAP
      if (threadIdx.x == 0) set_error(err, ERR_BOUNDS);
      __syncthreads();
      continue;
    }
    const U* src = (job.src ? scratch : keys) + job.start;
    // pass 1: load keys, leaf range
    U u[KPT];
    int lmin = 0x7fffffff, lmax = -1;
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const uint32_t i = k * THREADS + threadIdx.x;
      u[k] = i < m ? src[i] : (U)0;
      if (i < m && !KT<DT>::is_nan(u[k])) {
        int64_t q;
        const int l = predict_leaf<DT>(u[k], r, &q);
        lmin = min(lmin, l);
        lmax = max(lmax, l);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
      lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    }
    if (threadIdx.x == 0) { s_lmin = 0x7fffffff; s_lmax = -1; s_nbig = 0; s_all = 0; }
    for (uint32_t i = threadIdx.x; i <= m; i += THREADS) cnt[i] = 0;
    __syncthreads();
    if (lane == 0) { atomicMin(&s_lmin, lmin); atomicMax(&s_lmax, lmax); }
    __syncthreads();
    const int l0 = s_lmin, nl = s_lmax - s_lmin + 1;
    const double width = job.Fhi - job.Flo;
    const double scale = (double)m / width;
    const bool ok = (width > 0) && isfinite(scale) && m > 0;
    if (threadIdx.x == 0) {
      s_mode = !ok ? 2 : (nl >= 1 && nl <= MAXL ? 0 : 1);
      s_S = ok ? fp32_sat_d(scale) : 0.0f;
      s_T = ok ? fp32_sat_d(-job.Flo * scale) : 0.0f;
    }
    if (ok && nl >= 1 && nl <= MAXL) {
      for (int j = threadIdx.x; j < nl; j += THREADS) {
        const int l = l0 + j;
        const double* q = M.leaf64 + 5 * (size_t)l;
        const LeafEval le = M.leaf[l];
        Coef c;
        c.A = fp32_sat_d(ldexp(q[0], E + le.sh) * scale);
        c.B = fp32_sat_d((q[2] - job.Flo) * scale);
        c.LO = fp32_sat_d((q[3] - job.Flo) * scale);
        c.HI = fp32_sat_d((q[4] - job.Flo) * scale);
        c.cq = le.cq;
        c.sh = le.sh;
        c.pad = 0;
        coef[j] = c;
      }
    }
    __syncthreads();
    const int mode = s_mode;
    const float S = s_S, T = s_T;
    const float mlim = (float)(m - 1);
    // pass 2: slots, histogram, ranks
    uint32_t sl[KPT], rk[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const uint32_t i = k * THREADS + threadIdx.x;
      uint32_t s = 0xFFFFFFFFu;
      if (i < m) {
        const U x = u[k];
        if (KT<DT>::is_nan(x)) {
          s = KT<DT>::neg(x) ? 0u : m - 1;
        } else if (mode == 2) {
          s = 0;
        } else {
          float v;
          if (mode == 0) {
            int64_t q;
            const int l = predict_leaf<DT>(x, r, &q);
            const Coef c = coef[l - l0];
            v = __fmaf_rn(c.A, feature(q, c.cq, c.sh), c.B);
            v = fminf(fmaxf(v, c.LO), c.HI);
          } else {
            v = __fmaf_rn(predict_F<DT>(x, r, M.leaf), S, T);
          }
          s = (v > 0.0f) ? (v >= mlim ? m - 1 : (uint32_t)v) : 0u;
        }
      }
      sl[k] = s;
      const unsigned peers = __match_any_sync(0xffffffffu, s);
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (s != 0xFFFFFFFFu && lane == leader) old = atomicAdd(&cnt[s], (uint32_t)__popc(peers));
      old = __shfl_sync(0xffffffffu, old, leader);
      rk[k] = old + __popc(peers & lt);
    }
    __syncthreads();
    {
      // exclusive scan of cnt[0..m) in place (32-bit)
      const int per = (int)((m + THREADS - 1) / THREADS);
      const int b = threadIdx.x * per;
      uint32_t s = 0;
      for (int i = 0; i < per; ++i)
        if (b + i < (int)m) s += cnt[b + i];
      unsigned long long tot;
      unsigned long long run = block_excl_sum<unsigned long long>(s, ws, &tot);
      for (int i = 0; i < per; ++i)
        if (b + i < (int)m) { const uint32_t t = cnt[b + i]; cnt[b + i] = (uint32_t)run; run += t; }
      if (threadIdx.x == 0) cnt[m] = m;
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (sl[k] != 0xFFFFFFFFu) {
        const uint32_t p = cnt[sl[k]] + rk[k];
        if (p < m) out[p] = u[k]; else set_error(err, ERR_BOUNDS);
      }
    }
    __syncthreads();
    // touch-up: sort every group of keys that share a slot
    for (uint32_t s = threadIdx.x; s < m; s += THREADS) {
      const uint32_t a = cnt[s], b = cnt[s + 1];
      if (b <= a + 1) continue;
      const uint32_t sz = b - a;
      if (sz <= 8) {
        for (uint32_t i = a + 1; i < b; ++i) {
          const U x = out[i];
          const uint64_t t = KT<DT>::tk(x);
          uint32_t j = i;
          while (j > a && KT<DT>::tk(out[j - 1]) > t) { out[j] = out[j - 1]; --j; }
          out[j] = x;
        }
      } else {
        const uint32_t idx = atomicAdd(&s_nbig, 1u);
        if (idx < BIGCAP) big[idx] = make_uint2(a, sz);
        else s_all = 1;
      }
    }
    __syncthreads();
    if (s_all) {
      block_bitonic<DT>(out, m);
    } else {
      const uint32_t nb = s_nbig;
      for (uint32_t g = wid; g < nb; g += THREADS / 32) {
        const uint2 gr = big[g];
        if (gr.y > 128) continue;
        U x[4];
        uint32_t rank[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t i = lane + 32 * q;
          rank[q] = 0;
          x[q] = i < gr.y ? out[gr.x + i] : (U)0;
        }
        for (uint32_t j = 0; j < gr.y; ++j) {
          const uint64_t tj = KT<DT>::tk(out[gr.x + j]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t i = lane + 32 * q;
            const uint64_t ti = KT<DT>::tk(x[q]);
            rank[q] += (tj < ti || (tj == ti && j < i)) ? 1u : 0u;
          }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t i = lane + 32 * q;
          if (i < gr.y) out[gr.x + rank[q]] = x[q];
        }
        __syncwarp();
      }
      __syncthreads();
      for (uint32_t g = 0; g < nb; ++g) {
        const uint2 gr = big[g];
        if (gr.y <= 128) continue;
        const uint64_t t0 = KT<DT>::tk(out[gr.x]);
        int diff = 0;
        for (uint32_t i = threadIdx.x; i < gr.y; i += THREADS)
          diff |= KT<DT>::tk(out[gr.x + i]) != t0;
        if (__syncthreads_or(diff)) block_bitonic<DT>(out + gr.x, gr.y);
      }
    }
    __syncthreads();
    U* dst = keys + job.start;
    for (uint32_t i = threadIdx.x; i < m; i += THREADS) dst[i] = out[i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- fallback
template <int DT>
__global__ void __launch_bounds__(RS_THREADS)
k_fallback(typename KT<DT>::U* keys, typename KT<DT>::U* scratch, JobList list,
           unsigned long long* ctr, uint32_t* err) {
  typedef typename KT<DT>::U U;
  constexpr int NDIG = KT<DT>::W;
  __shared__ RsShared sh;
  __shared__ uint32_t hist[256];
  __shared__ uint32_t ws[33];
  __shared__ unsigned long long s_job, s_or, s_and;
  const unsigned long long nj = min(*list.count, list.cap);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  while (true) {
    if (threadIdx.x == 0) { s_job = atomicAdd(ctr, 1ull); s_or = 0; s_and = ~0ull; }
    __syncthreads();
    const unsigned long long jid = s_job;
    if (jid >= nj) break;
    const Job job = list.jobs[jid];
    const uint64_t m = job.m;
    U* X = (job.src ? scratch : keys) + job.start;
    U* Y = (job.src ? keys : scratch) + job.start;
    unsigned long long o = 0, a = ~0ull;
    for (uint64_t i = threadIdx.x; i < m; i += RS_THREADS) {
      const uint64_t t = KT<DT>::tk(X[i]);
      o |= t;
      a &= t;
    }
    for (int s = 16; s > 0; s >>= 1) {
      o |= __shfl_xor_sync(0xffffffffu, o, s);
      a &= __shfl_xor_sync(0xffffffffu, a, s);
    }
    if (lane == 0) { atomicOr(&s_or, o); atomicAnd(&s_and, a); }
    __syncthreads();
    const uint64_t diff = s_or ^ s_and;
    for (int d = 0; d < NDIG; ++d) {
      if (((diff >> (8 * d)) & 255u) == 0) continue;
      const int shift = 8 * d;
      if (threadIdx.x < 256) hist[threadIdx.x] = 0;
      __syncthreads();
      for (uint64_t i = threadIdx.x; i < m; i += RS_THREADS)
        atomicAdd(&hist[(KT<DT>::tk(X[i]) >> shift) & 255u], 1u);
      __syncthreads();
      uint32_t c = threadIdx.x < 256 ? hist[threadIdx.x] : 0u;
      uint32_t tot;
      const uint32_t ex = block_excl_sum<uint32_t>(c, ws, &tot);
      if (threadIdx.x < 256) sh.run[threadIdx.x] = ex;
      __syncthreads();
      for (uint64_t base = 0; base < m; base += RS_TILE) {
        uint64_t key[RS_ROUNDS];
        bool valid[RS_ROUNDS];
        uint32_t lrank[RS_ROUNDS];
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
          const uint64_t i = base + (uint64_t)w * (32 * RS_ROUNDS) + r * 32 + lane;
          valid[r] = i < m;
          key[r] = valid[r] ? (uint64_t)X[i] : 0;
        }
        uint32_t tcnt = 0;
        rs_rank_tile(sh, key, valid, lrank,
                     [shift](uint64_t k) { return (uint32_t)(KT<DT>::tk((U)k) >> shift) & 255u; },
                     &tcnt);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
          if (!valid[r]) continue;
          const uint32_t dg = (uint32_t)(KT<DT>::tk((U)key[r]) >> shift) & 255u;
          const uint64_t pos = (uint64_t)sh.run[dg] + sh.whist[w][dg] + lrank[r];
          if (pos < m) Y[pos] = (U)key[r]; else set_error(err, ERR_BOUNDS);
        }
        __syncthreads();
        if (threadIdx.x < 256) sh.run[threadIdx.x] += tcnt;
        __syncthreads();
      }
      U* t = X; X = Y; Y = t;
    }
    U* dst = keys + job.start;
    if (X != dst)
      for (uint64_t i = threadIdx.x; i < m; i += RS_THREADS) dst[i] = X[i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host enqueue
constexpr int BS_SMALL_T = 256, BS_SMALL_K = 8;    // CAP 2048
constexpr int BS_LARGE_T = 512, BS_LARGE_K = 16;   // CAP 8192

template <int DT>
static cudaError_t buckets_cfg_dt() {
  cudaError_t e = cudaFuncSetAttribute(k_bucket_sort<DT, BS_SMALL_T, BS_SMALL_K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BucketCfg<DT, BS_SMALL_T, BS_SMALL_K>::SMEM);
  if (e) return e;
  return cudaFuncSetAttribute(k_bucket_sort<DT, BS_LARGE_T, BS_LARGE_K>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)BucketCfg<DT, BS_LARGE_T, BS_LARGE_K>::SMEM);
}

cudaError_t buckets_configure(int dt) {
  switch (dt) {
    case LS_F64: return buckets_cfg_dt<LS_F64>();
    case LS_U64: return buckets_cfg_dt<LS_U64>();
    case LS_F32: return buckets_cfg_dt<LS_F32>();
    case LS_U32: return buckets_cfg_dt<LS_U32>();
  }
  return cudaErrorInvalidValue;
}

template <int DT>
static cudaError_t buckets_dt(void* keys, void* scratch, const ModelPtrs& M, const Lists& lists,
                              uint64_t cap_s, uint64_t cap_l, uint64_t cap_fb,
                              unsigned long long* ctrs, uint32_t* err, cudaStream_t st,
                              int num_sms, const Marks* mk, int mb) {
  typedef typename KT<DT>::U U;
  const unsigned gs = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_s, 1), 8ull * num_sms);
  const unsigned gl = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_l, 1), 2ull * num_sms);
  const unsigned gf = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_fb, 1), 2ull * num_sms);
  k_bucket_sort<DT, BS_SMALL_T, BS_SMALL_K>
      <<<gs, BS_SMALL_T, BucketCfg<DT, BS_SMALL_T, BS_SMALL_K>::SMEM, st>>>(
          (U*)keys, (const U*)scratch, M, lists.sort_s, ctrs + 0, err);
  mark(mk, mb + 0, st);
  k_bucket_sort<DT, BS_LARGE_T, BS_LARGE_K>
      <<<gl, BS_LARGE_T, BucketCfg<DT, BS_LARGE_T, BS_LARGE_K>::SMEM, st>>>(
          (U*)keys, (const U*)scratch, M, lists.sort_l, ctrs + 1, err);
  mark(mk, mb + 1, st);
  k_fallback<DT><<<gf, RS_THREADS, 0, st>>>((U*)keys, (U*)scratch, lists.fallback, ctrs + 2, err);
  mark(mk, mb + 2, st);
  add_launches(3);
  return cudaGetLastError();
}

cudaError_t buckets_enqueue(int dt, void* keys, void* scratch, uint64_t n, const ModelPtrs& M,
                            const Lists& lists, uint64_t cap_s, uint64_t cap_l, uint64_t cap_fb,
                            unsigned long long* ctrs, uint32_t* err, cudaStream_t st,
                            int num_sms, const Marks* mk, int mb) {
  (void)n;
  switch (dt) {
    case LS_F64: return buckets_dt<LS_F64>(keys, scratch, M, lists, cap_s, cap_l, cap_fb, ctrs, err, st, num_sms, mk, mb);
    case LS_U64: return buckets_dt<LS_U64>(keys, scratch, M, lists, cap_s, cap_l, cap_fb, ctrs, err, st, num_sms, mk, mb);
    case LS_F32: return buckets_dt<LS_F32>(keys, scratch, M, lists, cap_s, cap_l, cap_fb, ctrs, err, st, num_sms, mk, mb);
    case LS_U32: return buckets_dt<LS_U32>(keys, scratch, M, lists, cap_s, cap_l, cap_fb, ctrs, err, st, num_sms, mk, mb);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ls

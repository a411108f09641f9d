// In-bucket finish of LearnedSort 2.0 (Alg. 2): the counting sort of each
// (sub-)bucket followed by the insertion-sort touch-up.
//
// One CTA per segment of m keys (m <= CAP), keys held in registers, counts and
// the placed keys in shared memory.  Inside a segment the model is a straight
// line (a segment lies within the F range of one level-1 sub-bucket), so the
// slot map is that line drawn through the segment's own key range, evaluated
// on the total-order key without any per-key model lookup:
//   slot(x) = min(m - 1, floor(((tk(x) - tmin) >> sh) * m / (((tmax - tmin) >> sh) + 1)))
// (sh keeps the scaled range within 24 bits, so the conversion is exact and
// the map is non-decreasing); float segments whose range crosses binades use
// the line through the keys' FP32 images instead, which is non-decreasing
// too.  Histogram of slots -> exclusive scan (the
// running totals of Alg. 2) -> placement -> touch-up.  Keys of different
// slots are already in order, so the touch-up only orders each group of keys
// sharing a slot: a group that holds one value (duplicates) is in order as
// placed; in a group of several values every key of a group of at most 32
// counts the members below it and writes itself to its final place, and
// larger such groups are sorted by a bitonic network.
//
// Segments the levels could not split below CAP keys go to the fallback: per
// job one CTA splits by the top byte in which the segment's total-order keys
// differ (MSD), stops as soon as a piece holds one value, and finishes pieces
// of at most CAP keys with the same counting sort.
#include <cfloat>

#include "ls_inplace.cuh"
#include "ls_partition.cuh"
#include "ls_radix.cuh"
#include "ls_scan.cuh"

namespace ls {

constexpr int BIGCAP = 512;     // groups of several values above 32 keys tracked per segment
constexpr int STACK = 2048;     // fallback work stack entries per CTA

template <int DT, int THREADS, int KPT>
struct BucketCfg {
  typedef typename KT<DT>::U U;
  static constexpr int CAP = THREADS * KPT;
  static constexpr size_t OFF_OUT = 0;
  static constexpr size_t OFF_CNT = OFF_OUT + sizeof(U) * CAP;
  static constexpr size_t OFF_BIG = (OFF_CNT + 4 * (CAP + 1) + 15) / 16 * 16;
  static constexpr size_t OFF_WS = OFF_BIG + 8 * BIGCAP;
  static constexpr size_t OFF_MIX = OFF_WS + 8 * 40;       // CAP bytes: slot holds > 1 value
  static constexpr size_t SMEM = (OFF_MIX + CAP + 15) / 16 * 16;
  // fallback extras
  static constexpr size_t OFF_STACK = (SMEM + 15) / 16 * 16;
  static constexpr size_t OFF_HIST = OFF_STACK + 16 * STACK;
  static constexpr size_t SMEM_FB = OFF_HIST + 4 * 512;
};

struct SegShared {            // per-CTA scalars of the segment sort
  unsigned long long tmin, tmax;
  uint32_t nbig, all;
  float rscale;
  int sh;
  float fmin, fscale;         // value-linear map (floats spanning several binades)
  int vmap;
  uint32_t dense;             // some slot holds more than DENSE_RANK keys
};

// A segment in which some slot receives more than this many keys is treated
// as holding runs of duplicates (see the touch-up below).
constexpr uint32_t DENSE_RANK = 16;

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

__device__ __forceinline__ int bitlen64d(uint64_t v) { return v ? 64 - __clzll((long long)v) : 0; }

// Counting sort + touch-up of src[0..m) into dst[0..m) (dst may equal src).
template <int DT, int THREADS, int KPT>
__device__ void segment_sort(typename KT<DT>::U* dst, const typename KT<DT>::U* src, uint32_t m,
                             unsigned char* sm, SegShared& ss, uint32_t* err) {
  typedef typename KT<DT>::U U;
  typedef BucketCfg<DT, THREADS, KPT> C;
  U* out = (U*)(sm + C::OFF_OUT);
  uint32_t* cnt = (uint32_t*)(sm + C::OFF_CNT);
  uint2* big = (uint2*)(sm + C::OFF_BIG);
  uint8_t* mix = (uint8_t*)(sm + C::OFF_MIX);
  unsigned long long* ws = (unsigned long long*)(sm + C::OFF_WS);
  const int lane = threadIdx.x & 31;
  // load, total-order key range
  U u[KPT];
  unsigned long long mn = ~0ull, mx = 0;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const uint32_t i = k * THREADS + threadIdx.x;
    u[k] = i < m ? src[i] : (U)0;
    if (i < m) {
      const unsigned long long t = KT<DT>::tk(u[k]);
      mn = min(mn, t);
      mx = max(mx, t);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (threadIdx.x == 0) { ss.tmin = ~0ull; ss.tmax = 0; ss.nbig = 0; ss.all = 0; ss.dense = 0; }
  // every thread owns KPT consecutive counters (16-byte stores; the slots
  // beyond m stay zero, so the scan leaves m in them)
  static_assert(KPT % 4 == 0, "KPT counters per thread in 16-byte groups");
  uint4* cnt4 = (uint4*)cnt + threadIdx.x * (KPT / 4);
#pragma unroll
  for (int v = 0; v < KPT / 4; ++v) {
    cnt4[v] = make_uint4(0u, 0u, 0u, 0u);
    ((uint32_t*)mix)[threadIdx.x * (KPT / 4) + v] = 0u;
  }
  __syncthreads();
  if (lane == 0) { atomicMin(&ss.tmin, mn); atomicMax(&ss.tmax, mx); }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t R = ss.tmax - ss.tmin;
    const int bl = R ? 64 - __clzll((long long)R) : 0;
    const int sh = bl > 24 ? bl - 24 : 0;
    ss.sh = sh;
    ss.rscale = (float)m / ((float)(R >> sh) + 1.0f);
    // Floats whose range crosses binades (typically around zero) are spread
    // unevenly by a line in total-order key space (every binade gets the same
    // share of slots); a line through their FP32 images keeps the groups
    // short.  Both maps are non-decreasing in the key.
    ss.vmap = 0;
    if (DT == LS_F64 || DT == LS_F32) {
      const float a = key_f32<DT>(KT<DT>::from_tk(ss.tmin));
      const float b = key_f32<DT>(KT<DT>::from_tk(ss.tmax));
      const float span = b - a;
      if (((__float_as_uint(a) ^ __float_as_uint(b)) >> 23) != 0 && isfinite(a) && isfinite(b) &&
          span > 0.0f && isfinite(span)) {
        ss.vmap = 1;
        ss.fmin = a;
        ss.fscale = (float)m / span;
      }
    }
  }
  __syncthreads();
  const float rscale = ss.rscale;
  const int sh = ss.sh;
  const unsigned long long tmin = ss.tmin;
  const bool vmap = (DT == LS_F64 || DT == LS_F32) && ss.vmap != 0;
  const float fmin = ss.fmin, fscale = ss.fscale;
  // slots, histogram, ranks (packed slot | rank << 16; m <= 2^15)
  uint32_t sr[KPT];
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const uint32_t i = k * THREADS + threadIdx.x;
    uint32_t v = 0xFFFFFFFFu;
    if (i < m) {
      const float f = vmap ? (key_f32<DT>(u[k]) - fmin) * fscale
                           : __uint2float_rn((uint32_t)((KT<DT>::tk(u[k]) - tmin) >> sh)) * rscale;
      const uint32_t s = min((uint32_t)f, m - 1);
      v = s | (atomicAdd(&cnt[s], 1u) << 16);  // rank inside the slot
      if ((v >> 16) == DENSE_RANK) ss.dense = 1u;
    }
    sr[k] = v;
  }
  __syncthreads();
  {  // exclusive scan of the CAP counters (the running totals of Alg. 2)
    uint32_t c[KPT];
#pragma unroll
    for (int v = 0; v < KPT / 4; ++v) {
      const uint4 q = cnt4[v];
      c[4 * v] = q.x; c[4 * v + 1] = q.y; c[4 * v + 2] = q.z; c[4 * v + 3] = q.w;
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < KPT; ++i) { const uint32_t t = c[i]; c[i] = s; s += t; }
    unsigned long long tot;
    const uint32_t run = (uint32_t)block_excl_sum<unsigned long long>(s, ws, &tot);
#pragma unroll
    for (int v = 0; v < KPT / 4; ++v)
      cnt4[v] = make_uint4(run + c[4 * v], run + c[4 * v + 1], run + c[4 * v + 2], run + c[4 * v + 3]);
    if (threadIdx.x == 0) cnt[C::CAP] = m;
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    if (sr[k] != 0xFFFFFFFFu) {
      const uint32_t p = cnt[sr[k] & 0xFFFFu] + (sr[k] >> 16);
      if (p < m) out[p] = u[k]; else set_error(err, ERR_BOUNDS);
    }
  }
  __syncthreads();
  // In a segment with runs of duplicates (some slot over DENSE_RANK keys), a
  // slot group holding one value is in order as placed; the groups that hold
  // more than one are marked: every key compares itself with its group's
  // first member.  (Elsewhere every group has at most DENSE_RANK keys, and
  // the per-key ranking below is cheaper than the marking.)
  const bool dense = ss.dense != 0u;
  if (dense) {
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      if (sr[k] != 0xFFFFFFFFu && (sr[k] >> 16) != 0) {
        const uint32_t s = sr[k] & 0xFFFFu;
        if (KT<DT>::tk(out[cnt[s]]) != KT<DT>::tk(u[k])) mix[s] = 1;
      }
    }
    __syncthreads();
  }
  // Final positions straight from the registers.  Keys of different slots are
  // in order (the slot map is monotone); inside a group [a, b) of several
  // values a key's place is a + #{members smaller, or equal and placed
  // earlier}: the insertion-sort touch-up of Alg. 2 restricted to the group,
  // computed per key so that the lanes do not wait on each other.  Groups of
  // several values above GROUP_MAX keys are sorted cooperatively below.
  constexpr uint32_t GROUP_MAX = 32;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    if (sr[k] == 0xFFFFFFFFu) continue;
    const uint32_t s = sr[k] & 0xFFFFu;
    const uint32_t a = cnt[s], b = cnt[s + 1];
    if (b - a == 1 || (dense && !mix[s])) { dst[a + (sr[k] >> 16)] = u[k]; continue; }
    if (b - a > GROUP_MAX) {
      if ((sr[k] >> 16) == 0) {  // the group's first key records it
        const uint32_t idx = atomicAdd(&ss.nbig, 1u);
        if (idx < BIGCAP) big[idx] = make_uint2(a, b - a);
        else ss.all = 1;
      }
      continue;
    }
    const uint64_t t = KT<DT>::tk(u[k]);
    const uint32_t me = a + (sr[k] >> 16);
    uint32_t r = 0;
    for (uint32_t j = a; j < b; ++j) {
      const uint64_t tj = KT<DT>::tk(out[j]);
      r += (tj < t || (tj == t && j < me)) ? 1u : 0u;
    }
    dst[a + r] = u[k];
  }
  __syncthreads();
  const uint32_t nb = ss.nbig;
  if (nb == 0) return;
  if (ss.all) {  // too many large groups: sort the whole segment in shared memory
    block_bitonic<DT>(out, m);
    for (uint32_t i = threadIdx.x; i < m; i += THREADS) dst[i] = out[i];
    __syncthreads();
    return;
  }
  for (uint32_t g = 0; g < nb; ++g) {  // a large group of several values
    const uint2 gr = big[g];
    block_bitonic<DT>(out + gr.x, gr.y);
    for (uint32_t i = threadIdx.x; i < gr.y; i += THREADS) dst[gr.x + i] = out[gr.x + i];
    __syncthreads();
  }
}

template <int DT, int THREADS, int KPT>
__global__ void __launch_bounds__(THREADS, THREADS == 512 ? (KPT == 8 ? 3 : 2) : (KPT == 16 ? 3 : (THREADS == 128 ? 8 : 4)))
k_bucket_sort(typename KT<DT>::U* keys, const typename KT<DT>::U* scratch, ModelPtrs M,
              JobList list, unsigned long long* ctr, uint32_t* err) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  typedef BucketCfg<DT, THREADS, KPT> C;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ SegShared ss;
  __shared__ unsigned long long s_job;
  const unsigned long long nj = min(*list.count, list.cap);
  while (true) {
    if (threadIdx.x == 0) s_job = atomicAdd(ctr, 1ull);
    __syncthreads();
    const unsigned long long jid = s_job;
    if (jid >= nj) break;
    const Job job = list.jobs[jid];
    if (job.m > (uint64_t)C::CAP) {  // classification guarantees m <= CAP
      if (threadIdx.x == 0) set_error(err, ERR_BOUNDS);
      __syncthreads();
      continue;
    }
    const U* src = (job.src ? job_scratch(job, scratch) : job_keys(job, (U*)keys)) + job.start;
    segment_sort<DT, THREADS, KPT>(job_keys(job, keys) + job.start, src, (uint32_t)job.m, sm, ss,
                                   err);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- fallback
struct StackEnt {
  unsigned long long start;
  uint32_t m;
  uint32_t buf;  // 0: keys, 1: scratch
};

template <int DT>
__global__ void __launch_bounds__(512)
k_fallback(typename KT<DT>::U* keys, typename KT<DT>::U* scratch, ModelPtrs M, JobList list,
           unsigned long long* ctr, uint32_t* err) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  typedef BucketCfg<DT, 512, 16> C;
  extern __shared__ __align__(16) unsigned char sm[];
  StackEnt* stack = (StackEnt*)(sm + C::OFF_STACK);
  uint32_t* hist = (uint32_t*)(sm + C::OFF_HIST);
  uint32_t* cur = hist + 256;
  __shared__ SegShared ss;
  __shared__ unsigned long long s_job, s_or, s_and;
  __shared__ int s_top;
  __shared__ StackEnt s_e;
  __shared__ uint32_t ws32[33];
  const unsigned long long nj = min(*list.count, list.cap);
  const int lane = threadIdx.x & 31;
  while (true) {
    if (threadIdx.x == 0) s_job = atomicAdd(ctr, 1ull);
    __syncthreads();
    const unsigned long long jid = s_job;
    if (jid >= nj) break;
    const Job fjob = list.jobs[jid];
    U* const K = job_keys(fjob, keys);
    U* const S = job_scratch(fjob, scratch);
    if (threadIdx.x == 0) {
      const Job job = fjob;
      stack[0].start = job.start;
      stack[0].m = (uint32_t)job.m;
      stack[0].buf = job.src;
      s_top = 1;
    }
    __syncthreads();
    while (true) {
      if (threadIdx.x == 0) {
        if (s_top > 0) { s_e = stack[s_top - 1]; --s_top; }
        else s_e.m = 0xFFFFFFFFu;
        s_or = 0;
        s_and = ~0ull;
      }
      __syncthreads();
      const StackEnt e = s_e;
      if (e.m == 0xFFFFFFFFu) break;
      U* X = (e.buf ? S : K) + e.start;
      U* Y = (e.buf ? K : S) + e.start;
      U* D = K + e.start;
      if (e.m <= (uint32_t)C::CAP) {
        segment_sort<DT, 512, 16>(D, X, e.m, sm, ss, err);
        continue;
      }
      unsigned long long o = 0, a = ~0ull;
      for (uint32_t i = threadIdx.x; i < e.m; i += 512) {
        const uint64_t t = KT<DT>::tk(X[i]);
        o |= t;
        a &= t;
      }
      for (int s = 16; s > 0; s >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, s);
        a &= __shfl_xor_sync(0xffffffffu, a, s);
      }
      if (lane == 0) { atomicOr(&s_or, o); atomicAnd(&s_and, a); }
      if (threadIdx.x < 256) hist[threadIdx.x] = 0;
      __syncthreads();
      const uint64_t diff = s_or ^ s_and;
      if (diff == 0) {  // one value: already in order
        if (X != D)
          for (uint32_t i = threadIdx.x; i < e.m; i += 512) D[i] = X[i];
        __syncthreads();
        continue;
      }
      const int shift = ((63 - __clzll((long long)diff)) >> 3) << 3;  // top differing byte
      for (uint32_t i = threadIdx.x; i < e.m; i += 512)
        atomicAdd(&hist[(KT<DT>::tk(X[i]) >> shift) & 255u], 1u);
      __syncthreads();
      const uint32_t c = threadIdx.x < 256 ? hist[threadIdx.x] : 0u;
      uint32_t tot;
      const uint32_t ex = block_excl_sum<uint32_t>(c, ws32, &tot);
      if (threadIdx.x < 256) cur[threadIdx.x] = ex;
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < e.m; i += 512) {
        const U x = X[i];
        const uint32_t p = atomicAdd(&cur[(KT<DT>::tk(x) >> shift) & 255u], 1u);
        if (p < e.m) Y[p] = x; else set_error(err, ERR_BOUNDS);
      }
      __syncthreads();
      if (threadIdx.x < 256 && c > 0) {
        const int slot = atomicAdd(&s_top, 1);
        if (slot < STACK) {
          StackEnt ne;
          ne.start = e.start + ex;
          ne.m = c;
          ne.buf = e.buf ^ 1u;
          stack[slot] = ne;
        } else {
          set_error(err, ERR_BOUNDS);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && s_top > STACK) s_top = STACK;
      __syncthreads();
    }
  }
}

// Fallback of the in-place variant: the same MSD splits by the top differing
// byte, each done inside the segment (fragment flush, defragment, cleanup:
// ls_inplace.cuh) instead of into scratch.  The split's shared memory and the
// counting sort's share one region; the work stack follows it.
template <int DT>
struct IpFbCfg {
  typedef typename KT<DT>::U U;
  typedef BucketCfg<DT, 512, 16> C;
  static constexpr size_t AREA = C::SMEM > IpCta<U>::SMEM ? C::SMEM : IpCta<U>::SMEM;
  static constexpr size_t OFF_STACK = (AREA + 15) / 16 * 16;
  static constexpr size_t SMEM = OFF_STACK + 16 * STACK;
};

template <int DT>
struct IpDigit {
  int shift;
  __device__ uint32_t operator()(typename KT<DT>::U u) const {
    return (uint32_t)((KT<DT>::tk(u) >> shift) & 255u);
  }
};

template <int DT>
__global__ void __launch_bounds__(512, 1)
k_ip_fallback(typename KT<DT>::U* keys, JobList list, unsigned long long* ctr, uint32_t* err) {
  pdl_begin();
  typedef typename KT<DT>::U U;
  typedef IpFbCfg<DT> Q;
  typedef BucketCfg<DT, 512, 16> C;
  extern __shared__ __align__(16) unsigned char sm[];
  StackEnt* stack = (StackEnt*)(sm + Q::OFF_STACK);
  __shared__ SegShared ss;
  __shared__ unsigned long long s_job, s_or, s_and;
  __shared__ int s_top;
  __shared__ StackEnt s_e;
  const unsigned long long nj = min(*list.count, list.cap);
  const int lane = threadIdx.x & 31;
  const uint32_t* pcnt = (const uint32_t*)(sm + IpCta<U>::OFF_U32) + 4 * IpCta<U>::F;
  const unsigned long long* pst = (const unsigned long long*)(sm + IpCta<U>::OFF_ST);
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_job = call_failed(err) ? ~0ull : atomicAdd(ctr, 1ull);
    __syncthreads();
    const unsigned long long jid = s_job;
    if (jid >= nj) break;
    const Job fjob = list.jobs[jid];
    U* const K = job_keys(fjob, keys);
    if (threadIdx.x == 0) {
      stack[0].start = fjob.start;
      stack[0].m = (uint32_t)fjob.m;
      stack[0].buf = 0;
      s_top = 1;
    }
    __syncthreads();
    while (true) {
      if (threadIdx.x == 0) {
        if (s_top > 0) { s_e = stack[s_top - 1]; --s_top; }
        else s_e.m = 0xFFFFFFFFu;
        s_or = 0;
        s_and = ~0ull;
      }
      __syncthreads();
      const StackEnt e = s_e;
      if (e.m == 0xFFFFFFFFu) break;
      U* D = K + e.start;
      if (e.m <= (uint32_t)C::CAP) {
        segment_sort<DT, 512, 16>(D, D, e.m, sm, ss, err);
        continue;
      }
      unsigned long long o = 0, a = ~0ull;
      for (uint32_t i = threadIdx.x; i < e.m; i += 512) {
        const uint64_t t = KT<DT>::tk(D[i]);
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
      if (diff == 0) continue;  // one value: already in order
      const int shift = ((63 - __clzll((long long)diff)) >> 3) << 3;  // top differing byte
      ip_cta_partition<U, 512, 8, false>(D, e.m, e.m, 256u, IpDigit<DT>{shift}, IpPrefixStarts{}, sm,
                                         err, IpChainWs{});  // in rounds
      if (threadIdx.x < 256 && pcnt[threadIdx.x] > 1u) {
        const int slot = atomicAdd(&s_top, 1);
        if (slot < STACK) {
          StackEnt ne;
          ne.start = e.start + pst[threadIdx.x];
          ne.m = pcnt[threadIdx.x];
          ne.buf = 0;
          stack[slot] = ne;
        } else {
          set_error(err, ERR_BOUNDS);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && s_top > STACK) s_top = STACK;
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- host enqueue
constexpr int BS_TINY_T = 128, BS_TINY_K = 4;      // CAP 512
constexpr int BS_SMALL_T = 256, BS_SMALL_K = 8;    // CAP 2048
constexpr int BS_MID0_T = 384, BS_MID0_K = 8;      // CAP 3072
constexpr int BS_MID_T = 512, BS_MID_K = 8;        // CAP 4096
constexpr int BS_LARGE_T = 512, BS_LARGE_K = 16;   // CAP 8192

template <int DT>
static cudaError_t buckets_cfg_dt() {
  cudaError_t e = cudaFuncSetAttribute(k_bucket_sort<DT, BS_TINY_T, BS_TINY_K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BucketCfg<DT, BS_TINY_T, BS_TINY_K>::SMEM);
  if (e) return e;
  e = cudaFuncSetAttribute(k_bucket_sort<DT, BS_SMALL_T, BS_SMALL_K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BucketCfg<DT, BS_SMALL_T, BS_SMALL_K>::SMEM);
  if (e) return e;
  e = cudaFuncSetAttribute(k_bucket_sort<DT, BS_MID0_T, BS_MID0_K>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)BucketCfg<DT, BS_MID0_T, BS_MID0_K>::SMEM);
  if (e) return e;
  e = cudaFuncSetAttribute(k_bucket_sort<DT, BS_MID_T, BS_MID_K>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)BucketCfg<DT, BS_MID_T, BS_MID_K>::SMEM);
  if (e) return e;
  e = cudaFuncSetAttribute(k_bucket_sort<DT, BS_LARGE_T, BS_LARGE_K>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)BucketCfg<DT, BS_LARGE_T, BS_LARGE_K>::SMEM);
  if (e) return e;
  e = cudaFuncSetAttribute(k_fallback<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)BucketCfg<DT, 512, 16>::SMEM_FB);
  if (e) return e;
  static_assert(IpFbCfg<DT>::SMEM <= 227 * 1024, "in-place fallback shared memory");
  return cudaFuncSetAttribute(k_ip_fallback<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)IpFbCfg<DT>::SMEM);
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
                              int num_sms, const Marks* mk, int mb, bool in_place) {
  typedef typename KT<DT>::U U;
  const unsigned gs = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_s, 1), 8ull * num_sms);
  const unsigned gl = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_l, 1), 2ull * num_sms);
  const unsigned gf = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_fb, 1), 1ull * num_sms);
  {
    const unsigned gt = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_s, 1), 16ull * num_sms);
    launch_k(k_bucket_sort<DT, BS_TINY_T, BS_TINY_K>, gt, BS_TINY_T, BucketCfg<DT, BS_TINY_T, BS_TINY_K>::SMEM, st, (U*)keys, (const U*)scratch, M, lists.sort_t, ctrs + 6, err);
  }
  launch_k(k_bucket_sort<DT, BS_SMALL_T, BS_SMALL_K>, gs, BS_SMALL_T, BucketCfg<DT, BS_SMALL_T, BS_SMALL_K>::SMEM, st, (U*)keys, (const U*)scratch, M, lists.sort_s, ctrs + 0, err);
  mark(mk, mb + 0, st);
  {
    // segments of 2049..3072 keys: 384 threads, so that fewer key slots of a
    // thread stay empty than in the 4096-key class
    const unsigned gm0 = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_s, 1), 4ull * num_sms);
    launch_k(k_bucket_sort<DT, BS_MID0_T, BS_MID0_K>, gm0, BS_MID0_T, BucketCfg<DT, BS_MID0_T, BS_MID0_K>::SMEM, st, (U*)keys, (const U*)scratch, M, lists.sort_m0, ctrs + 9, err);
  }
  {
    const unsigned gm = (unsigned)std::min<uint64_t>(std::max<uint64_t>(cap_s, 1), 4ull * num_sms);
    launch_k(k_bucket_sort<DT, BS_MID_T, BS_MID_K>, gm, BS_MID_T, BucketCfg<DT, BS_MID_T, BS_MID_K>::SMEM, st, (U*)keys, (const U*)scratch, M, lists.sort_m, ctrs + 3, err);
  }
  launch_k(k_bucket_sort<DT, BS_LARGE_T, BS_LARGE_K>, gl, BS_LARGE_T, BucketCfg<DT, BS_LARGE_T, BS_LARGE_K>::SMEM, st, (U*)keys, (const U*)scratch, M, lists.sort_l, ctrs + 1, err);
  mark(mk, mb + 1, st);
  if (!in_place)
    launch_k(k_fallback<DT>, gf, 512, BucketCfg<DT, 512, 16>::SMEM_FB, st, (U*)keys, (U*)scratch, M,
             lists.fallback, ctrs + 2, err);
  else  // the in-place variant: no scratch, every job in the caller's array
    launch_k(k_ip_fallback<DT>, gf, 512, IpFbCfg<DT>::SMEM, st, (U*)keys, lists.fallback, ctrs + 2, err);
  add_launches(6);
  return cudaGetLastError();
}

cudaError_t buckets_enqueue(int dt, void* keys, void* scratch, uint64_t n, const ModelPtrs& M,
                            const Lists& lists, uint64_t cap_s, uint64_t cap_l, uint64_t cap_fb,
                            unsigned long long* ctrs, uint32_t* err, cudaStream_t st,
                            int num_sms, const Marks* mk, int mb, bool in_place) {
  (void)n;
  switch (dt) {
    case LS_F64: return buckets_dt<LS_F64>(keys, scratch, M, lists, cap_s, cap_l, cap_fb, ctrs, err, st, num_sms, mk, mb, in_place);
    case LS_U64: return buckets_dt<LS_U64>(keys, scratch, M, lists, cap_s, cap_l, cap_fb, ctrs, err, st, num_sms, mk, mb, in_place);
    case LS_F32: return buckets_dt<LS_F32>(keys, scratch, M, lists, cap_s, cap_l, cap_fb, ctrs, err, st, num_sms, mk, mb, in_place);
    case LS_U32: return buckets_dt<LS_U32>(keys, scratch, M, lists, cap_s, cap_l, cap_fb, ctrs, err, st, num_sms, mk, mb, in_place);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ls

// Internal definitions shared by the CUDA translation units of the learned
// sort (LearnedSort 2.0, arXiv 2107.03290).  Device code for sm_103a.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/atomic>

#include "../../include/ls.h"

namespace ls {

// ------------------------------------------------------------------ constants
constexpr int MAX_LEAVES = 4096;
constexpr int MAX_FANOUT = 4096;
constexpr int MAX_HPB = 8;          // equality buckets per level-0 bucket
constexpr int MAX_F1 = 1024;        // level-1 sub-buckets per segment
constexpr int64_t Q_SAT = (int64_t)1 << 62;
constexpr unsigned long long SPIN_LIMIT = 1ull << 26;  // bounded waits

// Device status word bits (ls_stream_status).
constexpr uint32_t ERR_TIMEOUT = 1u;
constexpr uint32_t ERR_BOUNDS = 2u;

// ------------------------------------------------------------------ key traits
// Keys are handled as raw bit patterns U; tk() is the total-order key, the
// ordering contract of ls.h (Sec. 4.2: the output is monotonically ordered).
template <int DT> struct KT;
template <> struct KT<LS_F64> {
  typedef uint64_t U;
  static constexpr int W = 8;
  __host__ __device__ static inline uint64_t tk(U u) { return (u >> 63) ? ~u : (u | (1ull << 63)); }
  __host__ __device__ static inline U from_tk(uint64_t t) { return (t >> 63) ? (t & ~(1ull << 63)) : ~t; }
  __device__ static inline bool is_nan(U u) { return ((u >> 52) & 0x7FF) == 0x7FF && (u & ((1ull << 52) - 1)); }
  __device__ static inline bool neg(U u) { return (u >> 63) != 0; }
  __device__ static inline bool finite(U u) { return ((u >> 52) & 0x7FF) != 0x7FF; }
  __device__ static inline double dbl(U u) { return __longlong_as_double((long long)u); }
};
template <> struct KT<LS_U64> {
  typedef uint64_t U;
  static constexpr int W = 8;
  __host__ __device__ static inline uint64_t tk(U u) { return u; }
  __host__ __device__ static inline U from_tk(uint64_t t) { return t; }
  __device__ static inline bool is_nan(U) { return false; }
  __device__ static inline bool neg(U) { return false; }
  __device__ static inline bool finite(U) { return true; }
  __device__ static inline double dbl(U u) { return __ull2double_rn(u); }
};
template <> struct KT<LS_F32> {
  typedef uint32_t U;
  static constexpr int W = 4;
  __host__ __device__ static inline uint64_t tk(U u) {
    return (u >> 31) ? (uint64_t)(~u) : (uint64_t)(u | 0x80000000u);
  }
  __host__ __device__ static inline U from_tk(uint64_t t) {
    const uint32_t v = (uint32_t)t;
    return (v >> 31) ? (v & 0x7FFFFFFFu) : ~v;
  }
  __device__ static inline bool is_nan(U u) { return ((u >> 23) & 0xFF) == 0xFF && (u & 0x7FFFFFu); }
  __device__ static inline bool neg(U u) { return (u >> 31) != 0; }
  __device__ static inline bool finite(U u) { return ((u >> 23) & 0xFF) != 0xFF; }
  __device__ static inline double dbl(U u) { return (double)__uint_as_float(u); }
};
template <> struct KT<LS_U32> {
  typedef uint32_t U;
  static constexpr int W = 4;
  __host__ __device__ static inline uint64_t tk(U u) { return u; }
  __host__ __device__ static inline U from_tk(uint64_t t) { return (uint32_t)t; }
  __device__ static inline bool is_nan(U) { return false; }
  __device__ static inline bool neg(U) { return false; }
  __device__ static inline bool finite(U) { return true; }
  __device__ static inline double dbl(U u) { return (double)u; }
};

// ------------------------------------------------------------------ fixed point
// q(x) = floor(x * 2^-E) saturated to [-2^62, 2^62]; |x| = M * 2^exp2.
// Integer arithmetic only (monotone in x by construction).
__device__ __forceinline__ int64_t fx_core(bool neg, uint64_t M, int exp2, int E) {
  if (M == 0) return 0;
  const int k = exp2 - E;
  uint64_t v;
  uint64_t rem = 0;
  if (k >= 0) {
    v = (k > 62 || M > (1ull << (62 - k))) ? (uint64_t)Q_SAT : (M << k);
  } else {
    const int j = -k;
    if (j >= 64) { v = 0; rem = 1; }
    else { v = M >> j; rem = (M & ((1ull << j) - 1)) != 0; }
  }
  int64_t q = neg ? -(int64_t)(v + rem) : (int64_t)v;
  q = q > Q_SAT ? Q_SAT : q;
  q = q < -Q_SAT ? -Q_SAT : q;
  return q;
}

__device__ __forceinline__ int64_t fx_f64bits(uint64_t u, int E) {
  const bool neg = (u >> 63) != 0;
  const int e = (int)((u >> 52) & 0x7FF);
  const uint64_t m = u & ((1ull << 52) - 1);
  if (e == 0x7FF) return neg ? -Q_SAT : Q_SAT;
  if (e == 0) return fx_core(neg, m, -1074, E);
  return fx_core(neg, m | (1ull << 52), e - 1075, E);
}

template <int DT> __device__ __forceinline__ int64_t fixed_point(typename KT<DT>::U u, int E);
template <> __device__ __forceinline__ int64_t fixed_point<LS_F64>(uint64_t u, int E) {
  return fx_f64bits(u, E);
}
template <> __device__ __forceinline__ int64_t fixed_point<LS_F32>(uint32_t u, int E) {
  const bool neg = (u >> 31) != 0;
  const int e = (int)((u >> 23) & 0xFF);
  const uint64_t m = u & ((1u << 23) - 1);
  if (e == 0xFF) return neg ? -Q_SAT : Q_SAT;
  if (e == 0) return fx_core(neg, m, -149, E);
  return fx_core(neg, m | (1u << 23), e - 150, E);
}
template <> __device__ __forceinline__ int64_t fixed_point<LS_U64>(uint64_t u, int E) {
  return fx_core(false, u, 0, E);
}
template <> __device__ __forceinline__ int64_t fixed_point<LS_U32>(uint32_t u, int E) {
  return fx_core(false, (uint64_t)u, 0, E);
}

// Centred feature: floor((q - cq) / 2^sh) clamped to +-(2^31 - 1), as float.
__device__ __forceinline__ float feature(int64_t q, int64_t cq, int sh) {
  int64_t d = (q - cq) >> sh;
  const int64_t LIM = 2147483647;
  d = d > LIM ? LIM : d;
  d = d < -LIM ? -LIM : d;
  return __int2float_rn((int)d);
}

// ------------------------------------------------------------------ model
struct LeafEval {      // 32 bytes, FP32 evaluation of one leaf
  long long cq;
  float A, B, LO, HI;
  int sh;
  int pad;
};
struct RootEval {
  long long cq;
  float A, B;
  int sh;
  int E;
  int L;
  int pad;
};

struct HeavyEntry {    // a heavy value of one level-0 bucket
  uint64_t tk;         // total-order key
  float F;             // FP32 eCDF estimate of the value
  uint32_t pad;
};

// Level-0 bucket head: first extended slot and heavy list [hoff, hoff+nh).
struct BucketHead {
  uint32_t ext_base;
  uint32_t hoff_nh;    // hoff << 4 | nh
};

// FP32 eCDF estimate F(x) in [0,1] for a non-NaN key; leaf from the root.
template <int DT>
__device__ __forceinline__ float predict_F(typename KT<DT>::U u, const RootEval& r,
                                           const LeafEval* __restrict__ leaves) {
  const int64_t q = fixed_point<DT>(u, r.E);
  const float v = __fmaf_rn(r.A, feature(q, r.cq, r.sh), r.B);
  int l;
  if (v >= (float)r.L) l = r.L - 1;
  else if (v > 0.0f) l = (int)v;
  else l = 0;
  const LeafEval le = leaves[l];
  float F = __fmaf_rn(le.A, feature(q, le.cq, le.sh), le.B);
  F = fmaxf(F, le.LO);
  F = fminf(F, le.HI);
  return F;
}

template <int DT>
__device__ __forceinline__ int predict_leaf(typename KT<DT>::U u, const RootEval& r, int64_t* q_out) {
  const int64_t q = fixed_point<DT>(u, r.E);
  *q_out = q;
  const float v = __fmaf_rn(r.A, feature(q, r.cq, r.sh), r.B);
  if (v >= (float)r.L) return r.L - 1;
  if (v > 0.0f) return (int)v;
  return 0;
}

// Level-0 bucket of a key (NaNs go to the end buckets by sign).
template <int DT>
__device__ __forceinline__ uint32_t bucket_of(typename KT<DT>::U u, const RootEval& r,
                                              const LeafEval* __restrict__ leaves, uint32_t f0) {
  if (KT<DT>::is_nan(u)) return KT<DT>::neg(u) ? 0u : f0 - 1;
  const float F = predict_F<DT>(u, r, leaves);
  const uint32_t b = (uint32_t)__fmul_rn(F, (float)f0);
  return b < f0 ? b : f0 - 1;
}

// Extended slot: regular bucket b with heavies h_1<..<h_k has slots
// ext_base + {0: <h_1, 1: =h_1, 2: (h_1,h_2), ..., 2k: >h_k}.
template <int DT>
__device__ __forceinline__ uint32_t ext_of(typename KT<DT>::U u, const RootEval& r,
                                           const LeafEval* __restrict__ leaves,
                                           const BucketHead* __restrict__ heads,
                                           const HeavyEntry* __restrict__ heavy, uint32_t f0) {
  const uint32_t b = bucket_of<DT>(u, r, leaves, f0);
  const BucketHead h = heads[b];
  uint32_t e = h.ext_base;
  const uint32_t nh = h.hoff_nh & 15u;
  if (nh) {
    const uint64_t t = KT<DT>::tk(u);
    const uint32_t ho = h.hoff_nh >> 4;
    for (uint32_t j = 0; j < nh; ++j) {
      const uint64_t hv = heavy[ho + j].tk;
      if (hv < t) e += 2;
      else { e += (hv == t) ? 1u : 0u; break; }
    }
  }
  return e;
}

// ------------------------------------------------------------------ jobs
// A segment of keys occupying [start, start+m) of buffer `src` (0: keys,
// 1: scratch); its keys' F estimates lie in [Flo, Fhi).  kind: what to do.
enum JobKind : uint32_t { JOB_SORT = 0, JOB_FILL = 1, JOB_REFINE = 2, JOB_FALLBACK = 3 };
struct Job {
  uint64_t start;
  uint64_t m;
  double Flo, Fhi;
  uint64_t value;      // FILL: the key bits to write
  uint32_t src;
  uint32_t kind;
};

// Job list: count + capacity-bounded array.
struct JobList {
  Job* jobs;
  unsigned long long* count;
  unsigned long long cap;
};

__device__ __forceinline__ void set_error(uint32_t* err, uint32_t bit) {
  if (err) atomicOr(err, bit);
}

__device__ __forceinline__ bool push_job(const JobList& L, const Job& j, uint32_t* err) {
  const unsigned long long i = atomicAdd(L.count, 1ull);
  if (i < L.cap) { L.jobs[i] = j; return true; }
  set_error(err, ERR_BOUNDS);
  return false;
}

// ------------------------------------------------------------------ memory order helpers
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  cuda::atomic_ref<uint64_t, cuda::thread_scope_device> a(*const_cast<uint64_t*>(p));
  return a.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  cuda::atomic_ref<uint64_t, cuda::thread_scope_device> a(*p);
  a.store(v, cuda::memory_order_release);
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  cuda::atomic_ref<uint32_t, cuda::thread_scope_device> a(*const_cast<uint32_t*>(p));
  return a.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  cuda::atomic_ref<uint32_t, cuda::thread_scope_device> a(*p);
  a.store(v, cuda::memory_order_release);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Work area of the LSD radix sort (ls_radix.cuh).  `ctr` must directly follow
// `status` in memory (one memset clears both).
struct RsWork {
  uint32_t* hist;     // 8 * 256 digit counts / offsets
  uint32_t* skip;     // 8
  uint32_t* status;   // 8 * tiles * 256 look-back words
  uint32_t* ctr;      // 8 tile counters
};

// ------------------------------------------------------------------ host-side plumbing
// Optional CUDA events recorded between kernels (per-kernel timing for stats).
struct Marks {
  cudaEvent_t* ev;
  int n;
};
inline void mark(const Marks* m, int i, cudaStream_t st) {
  if (m && m->ev && i < m->n) cudaEventRecord(m->ev[i], st);
}
// Number of kernel launches the library has enqueued (diagnostics).
void add_launches(unsigned k);
// Device address of the current device's status word (no allocation).
cudaError_t status_word_ptr(uint32_t** out);

// Model storage in device memory (one per sort call / array).
struct DevModel {
  RootEval root;           // FP32 evaluation of the root
  double root64[3];        // a, c, b
  uint64_t s, s_fin, s_lo; // sample size, finite keys, index of first finite
  uint32_t nheavy;
  uint32_t n_ext;
  uint64_t tau;
  double f_dummy;
};

struct ModelPtrs {         // device pointers of one model
  DevModel* hdr;
  double* leaf64;          // 5 * L
  LeafEval* leaf;          // L
  BucketHead* heads;       // f0 + 1
  HeavyEntry* heavy;       // max heavy
  uint32_t* leaf_beg;      // L (sample index ranges per leaf)
  uint32_t* leaf_end;      // L
};

}  // namespace ls

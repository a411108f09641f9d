// Internal definitions shared by the CUDA translation units of the learned
// sort (LearnedSort 2.0, arXiv 2107.03290).  Device code for sm_103a.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/atomic>

#include "../../include/ls.h"
#include "ls_call.h"

namespace ls {

// ------------------------------------------------------------------ constants
constexpr int MAX_LEAVES = 4096;
constexpr int MAX_FANOUT = 4096;
constexpr int MAX_HPB = 15;         // equality buckets per level-0 bucket (4-bit count)
constexpr int MAX_F1 = 1024;        // level-1 sub-buckets per segment
// Level-0 id of a key (histogram pass -> scatter pass): b | sid << PK_B_BITS
// for a non-equality key (b: its level-0 bucket; sid: its level-1 id), PK_EQ
// for a key equal to a heavy value.
constexpr int PK_B_BITS = 12;       // f0 <= MAX_FANOUT
constexpr uint32_t PK_B_MASK = (1u << PK_B_BITS) - 1;
constexpr uint32_t PK_EQ = 0xFFFFFFFFu;
constexpr unsigned long long SPIN_LIMIT = 1ull << 26;  // bounded waits

// Device status word bits (ls_stream_status).
constexpr uint32_t ERR_TIMEOUT = 1u;
constexpr uint32_t ERR_BOUNDS = 2u;

// Test injection: the first tile of the level-0 look-back scan never
// publishes its status, so the waits of the tiles after it run out.
constexpr uint32_t STALL_L0_SCAN = 1u;

__device__ __forceinline__ unsigned long long spin_limit_of(const uint32_t* err) {
  const unsigned long long s = err ? ((const CallStatus*)err)->spin_limit : 0ull;
  return s ? s : SPIN_LIMIT;
}
__device__ __forceinline__ uint32_t stall_of(const uint32_t* err) {
  return err ? ((const CallStatus*)err)->stall : 0u;
}
// True once the call has recorded an error (kernels that would consume the
// failed step's output return at once).
__device__ __forceinline__ bool call_failed(const uint32_t* err) {
  return err && *(volatile const uint32_t*)err != 0u;
}

// ------------------------------------------------------------------ launches
// Every kernel of the library is launched with programmatic stream
// serialization (programmatic dependent launch): the next kernel on the
// stream is scheduled as soon as the CTAs of the previous one have exited,
// without waiting for the grid's completion to be signalled, which hides most
// of the launch gap between the many short kernels of one call.  Each kernel
// therefore begins with pdl_begin(): it waits until the previous grid on the
// stream has completed and its memory is visible, before touching any memory.
// (No kernel triggers its dependents early: measured, letting the next
// kernel's CTAs occupy the SMs during the previous kernel's last wave made the
// training kernels slower.)  Launched without the attribute, the wait does
// nothing.
__device__ __forceinline__ void pdl_begin() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t c{};
  c.gridDim = grid;
  c.blockDim = block;
  c.dynamicSmemBytes = smem;
  c.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  c.attrs = at;
  c.numAttrs = 1;
  return cudaLaunchKernelEx(&c, kernel, static_cast<P>(args)...);
}

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

// ------------------------------------------------------------------ model
// Two evaluations of the same monotone model F:
//  * level 0 (buckets): the bucket of key x is pos(x) = clamp(floor(F(x) * f0),
//    0, f0-1) with F in FP64 (Alg. 1).  pos is non-decreasing in the
//    total-order key, so it is stored as its f0 thresholds
//      thr[b] = min { tk : pos(tk) >= b }   (thr[0] = 0)
//    and a key's bucket is the number of thresholds <= tk(x).  The search is
//    narrowed by a cell index: the same RMI evaluated in FP32 on a monotone
//    FP32 image of the key, cell = floor(F32(x) * L0_CELLS); the cell table
//    holds, per cell, the bucket range of the keys in it.  Any monotone cell
//    map gives the exact bucket; a good one only makes the ranges short;
// The same FP32 estimate (cell_F) also gives the level-1 sub-bucket of a key and
// the F value of each heavy value.
constexpr int L0_CELL_BITS = 12;
constexpr uint32_t L0_CELLS = 1u << L0_CELL_BITS;
constexpr uint32_t L0_TABLE = L0_CELLS;
struct HeavyEntry {    // a heavy value of one level-0 bucket
  uint64_t tk;         // total-order key
  float F;             // FP32 eCDF estimate of the value
  uint32_t ext;        // its equality slot
};

// Direct-mapped table of the heavy values (key bits -> equality slot): one
// 8-byte probe per key.  The table holds the raw bit patterns of the values
// (zero-extended for 4-byte keys; equal bits <=> equal total-order keys), so a
// probe needs no total-order conversion.  A slot keeps the most frequent of
// the values hashing to it; a free slot holds a key that hashes to another
// slot (0, or 1 in slot 0), so a probe never matches it.  The values that lost
// their slot, and the bit pattern HASH_EMPTY, are not in the table: their
// keys take the full lookup.
constexpr uint32_t HASH_SET_BITS = 13;
constexpr uint32_t HASH_SETS = 1u << HASH_SET_BITS;
constexpr uint32_t HASH_SIZE = HASH_SETS;          // entries (one per slot)
constexpr uint64_t HASH_EMPTY = ~0ull;
// Slot of a key's bits: the two halves folded, then 32-bit Fibonacci hashing.
__device__ __forceinline__ uint32_t heavy_hash(uint64_t bits) {
  const uint32_t f = (uint32_t)bits ^ (uint32_t)(bits >> 32);
  return (f * 0x9E3779B1u) >> (32 - HASH_SET_BITS);
}

// Level-0 bucket head: first extended slot and heavy list [hoff, hoff+nh).
struct __align__(8) BucketHead {   // one 8-byte load
  uint32_t ext_base;
  uint32_t hoff_nh;    // hoff << 4 | nh
};

// Monotone (non-decreasing) FP32 image of a non-NaN key: doubles are
// truncated toward zero (magnitudes below FLT_MIN become 0, above FLT_MAX
// infinity), integers converted toward zero.
template <int DT> __device__ __forceinline__ float key_f32(typename KT<DT>::U u);
template <> __device__ __forceinline__ float key_f32<LS_F64>(uint64_t u) {
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 896;  // FP32 biased exponent
  uint32_t mag = ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  mag = e <= 0 ? 0u : mag;
  mag = e >= 255 ? 0x7F800000u : mag;
  return __uint_as_float((hi & 0x80000000u) | mag);
}
template <> __device__ __forceinline__ float key_f32<LS_F32>(uint32_t u) { return __uint_as_float(u); }
template <> __device__ __forceinline__ float key_f32<LS_U64>(uint64_t u) { return __ull2float_rz(u); }
template <> __device__ __forceinline__ float key_f32<LS_U32>(uint32_t u) { return __uint2float_rz(u); }

struct CellRoot {          // FP32 RMI of the cell index, on key_f32(x)
  float A0, B0;            // w = A0 x + B0 = L * root(x)
  int L;
  int pad;
};
struct __align__(16) CellLeaf {  // F = clamp(A x + B, LO, HI), HI_l = LO_{l+1}; one 16-byte load
  float A, B, LO, HI;
};

// FP32 estimate of F on key_f32(x) (non-decreasing in the key: a >= 0 slopes,
// clamps with HI_l = LO_{l+1}); NaNs take 0 / 1 by sign.
template <int DT>
__device__ __forceinline__ float cell_F(typename KT<DT>::U u, const CellRoot& c,
                                        const CellLeaf* __restrict__ leaves) {
  const float x = key_f32<DT>(u);
  const float w = c.A0 == 0.0f ? c.B0 : __fmaf_rn(c.A0, x, c.B0);
  const int l = w >= 0.0f ? (w < (float)c.L ? (int)w : c.L - 1) : 0;
  const CellLeaf q = leaves[l];
  float F = q.A == 0.0f ? q.B : __fmaf_rn(q.A, x, q.B);
  F = fminf(fmaxf(F, q.LO), q.HI);
  if (KT<DT>::is_nan(u)) F = KT<DT>::neg(u) ? 0.0f : 1.0f;
  return F;
}

// Cell of a key: clamp(floor(F32(x) * L0_CELLS)).
template <int DT>
__device__ __forceinline__ uint32_t cell_of(typename KT<DT>::U u, const CellRoot& c,
                                            const CellLeaf* __restrict__ leaves) {
  const float v = cell_F<DT>(u, c, leaves) * (float)L0_CELLS;
  return v >= 0.0f ? (v < (float)L0_CELLS ? (uint32_t)v : L0_CELLS - 1) : 0u;
}

// Level-0 lookup tables (device or shared memory copies).
struct L0Map {
  const uint64_t* thr;     // f0 thresholds (thr[0] = 0)
  const uint32_t* cell;    // L0_CELLS entries: lo | hi << 16 (bucket range)
  const CellLeaf* cleaf;   // L cell-index leaves
  CellRoot croot;
  uint32_t pos_max;        // bucket of the largest total-order key
  uint32_t f0;             // buckets
};

// Largest b in [lo, hi] with thr[b] <= t (thr[lo] <= t holds).
__device__ __forceinline__ uint32_t thr_search(const uint64_t* thr, uint32_t lo, uint32_t hi,
                                               uint64_t t) {
  uint32_t b = lo;
  for (uint32_t s = hi > lo ? 1u << (31 - __clz((int)(hi - lo))) : 0u; s; s >>= 1) {
    const uint32_t nb = b + s;
    if (nb <= hi && thr[nb] <= t) b = nb;
  }
  return b;
}

// Level-0 bucket of a key (NaNs and infinities included: the thresholds cover
// the whole total order).
template <int DT>
__device__ __forceinline__ uint32_t l0_bucket(typename KT<DT>::U u, const L0Map& q) {
  const uint32_t c = q.cell[cell_of<DT>(u, q.croot, q.cleaf)];
  const uint32_t b = thr_search(q.thr, c & 0xFFFFu, c >> 16, KT<DT>::tk(u));
  return min(b, q.pos_max);
}

// Offset of key t among a bucket's ascending heavy values h[0..nh): 2 * #{h < t},
// plus 1 if t equals a heavy value (bisection).
__device__ __forceinline__ uint32_t heavy_offset(const uint64_t* h, uint32_t nh, uint64_t t) {
  uint32_t lo = 0, cnt = nh;
  while (cnt) {
    const uint32_t half = cnt >> 1;
    if (h[lo + half] < t) { lo += half + 1; cnt -= half + 1; } else cnt = half;
  }
  return 2 * lo + ((lo < nh && h[lo] == t) ? 1u : 0u);
}

// Extended slot: regular bucket b with heavies h_1<..<h_k has slots
// ext_base + {0: <h_1, 1: =h_1, 2: (h_1,h_2), ..., 2k: >h_k}.  `htk` holds the
// heavy values' total-order keys (bucket b's at [hoff, hoff + nh)).  Returns
// the slot; *bucket gets b and *nheavy its heavy count.
template <int DT>
__device__ __forceinline__ uint32_t ext_of2(typename KT<DT>::U u, const L0Map& q,
                                            const BucketHead* __restrict__ heads,
                                            const uint64_t* __restrict__ htk, uint32_t* bucket,
                                            uint32_t* nheavy = nullptr) {
  const uint64_t t = KT<DT>::tk(u);
  const uint32_t b = l0_bucket<DT>(u, q);
  *bucket = b;
  const BucketHead h = heads[b];
  uint32_t e = h.ext_base;
  const uint32_t nh = h.hoff_nh & 15u;
  if (nheavy) *nheavy = nh;
  if (nh) e += heavy_offset(htk + (h.hoff_nh >> 4), nh, t);
  return e;
}

template <int DT>
__device__ __forceinline__ uint32_t ext_of(typename KT<DT>::U u, const L0Map& q,
                                           const BucketHead* __restrict__ heads,
                                           const uint64_t* __restrict__ htk) {
  uint32_t b;
  return ext_of2<DT>(u, q, heads, htk, &b);
}

// ------------------------------------------------------------------ jobs
// A segment of keys occupying [start, start+m) of buffer `src` (0: keys,
// 1: scratch).  kind: what to do.
enum JobKind : uint32_t {
  JOB_SORT = 0,        // counting sort on the model's slot map
  JOB_FILL = 1,
  JOB_REFINE = 2,
  JOB_FALLBACK = 3,
  JOB_SORT_RANGE = 4,  // counting sort on the segment's key range (model could not split)
};
struct Job {
  uint64_t start;
  uint64_t m;
  uint64_t span;       // refine jobs: keys move within [start, start+span) of the other
                       // buffer (m, except for a level-0 bucket with heavy values, whose
                       // non-equality keys spread over the bucket's whole range)
  uint64_t pad;        // range-split jobs of the batched sort: keys per sub-bucket aimed at
                       // (0: the level's target)
  uint64_t value;      // FILL: the key bits to write
  uint32_t src;
  uint32_t kind;
  uint32_t la, lb;     // model refine jobs: level-0 bucket and its number of heavy values
  uint64_t kb, sb;     // batched arrays: this job's key / scratch array (0: the call's)
};

// Buffers of a job: its own array (batched sorts) or the call's.
template <typename U>
__device__ __forceinline__ U* job_keys(const Job& j, U* keys) { return j.kb ? (U*)j.kb : keys; }
template <typename U>
__device__ __forceinline__ U* job_scratch(const Job& j, U* scratch) {
  return j.sb ? (U*)j.sb : scratch;
}

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
// Work area of the training sample's sample sort (ls_samplesort.cuh).
constexpr int SS_OVER = 4;                 // oversample keys per splitter
constexpr int SS_P = 2048;                 // splitters
constexpr int SS_NB = 2 * SS_P + 1;        // buckets: gaps 2j, splitter values 2j+1
struct SsWork {
  uint64_t* spl;   // SS_P
  uint32_t* cnt;   // SS_NB + 1
  uint32_t* beg;   // SS_NB + 1
  uint32_t* cur;   // SS_NB + 1
};
inline size_t ss_work_words() { return (size_t)3 * (SS_NB + 1); }

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
// Persistent status block of `stream` on the current device (a slot of a
// static device array; no allocation).  Its word collects the errors of the
// calls on that stream until ls_stream_status reads and clears it.
cudaError_t stream_status_ptr(cudaStream_t stream, uint32_t** out);

// Model storage in device memory (one per sort call / array).
struct DevModel {
  double root64[3];        // a, c, b
  uint64_t s, s_fin, s_lo; // sample size, finite keys, index of first finite
  uint32_t nheavy;
  uint32_t n_ext;
  uint64_t tau;
  CellRoot croot;          // level-0 cell index (FP32 root)
  uint32_t cell_span;      // widest bucket range of a cell
  uint32_t pos_max;        // bucket of the largest total-order key
  unsigned long long heavy_len;  // sample keys equal to a selected heavy value
  uint32_t compact;        // 1: the level-0 histogram compacts non-equality keys
  uint32_t hash_probes;    // 1: the heavy table is built (0: no table)
};

__device__ __forceinline__ uint32_t bitlen32(uint32_t v) { return v ? 32u - __clz((int)v) : 0u; }

struct ModelPtrs {         // device pointers of one model
  DevModel* hdr;
  double* leaf64;          // 5 * L
  uint64_t* thr;           // f0 level-0 thresholds
  uint32_t* cell;          // L0_CELLS level-0 cell table
  CellLeaf* cleaf;         // L cell-index leaves
  uint64_t* hkey;          // HASH_SIZE heavy-table keys
  uint16_t* hval;          // HASH_SIZE heavy-table equality slots
  BucketHead* heads;       // f0 + 1
  HeavyEntry* heavy;       // max heavy
  uint32_t* leaf_beg;      // L (sample index ranges per leaf)
  int L;                   // leaves
  uint32_t* leaf_end;      // L
};

}  // namespace ls

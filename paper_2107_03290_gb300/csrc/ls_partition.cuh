// Host-side interface of the partitioning kernels (ls_partition.cu) and the
// in-bucket kernels (ls_bucket.cu).
#pragma once
#include "ls_internal.cuh"

namespace ls {

constexpr int P_THREADS = 1024;     // level-0 scatter CTAs
constexpr int H_THREADS = 1024;     // level-0 histogram CTAs
constexpr int P_TILE = 7168;        // keys per tile
constexpr int P_TILE_SMALL = 4096;  // keys per tile when many buckets leave less shared memory
constexpr int L1_THREADS = 512;
constexpr int L1_TILE = 4096;
constexpr uint64_t FILL_BIG = 1u << 15;   // fills this large are spread over the grid

// Contiguous chunk per CTA of the 16-byte aligned body [a0, a1); CTA 0 also
// handles the head [0, a0) and the tail [a1, n).
struct Chunking {
  uint64_t n, a0, a1, ch;
  uint32_t G;
};

struct Level0Args {
  const void* keys;
  void* scratch;
  Chunking c;
  ModelPtrs M;
  uint32_t f0;
  uint32_t n_ext_max;
  uint32_t L;
  uint32_t* hist;        // n_ext_max * G
  uint64_t* offs;        // n_ext_max * G + 1
  void* scan_status;     // scan work (status words + counter), zeroed by the caller
  uint32_t scan_tiles;
  uint32_t* err;
  uint32_t* pk;          // per key: compact slot | level-1 sub << 16 (body, then head/tail)
  uint16_t* sid;         // level-1 sub-bucket id at each scattered position
  uint32_t kf;           // level-1 sub-buckets per bucket
  float f0kf;            // f0 * kf
  uint64_t* ccount;      // per CTA: packed non-equality keys (compaction mode)
  uint32_t may_compact;  // 0: leave `keys` untouched (read-only callers)
  uint32_t in_place;     // 1: the in-place variant (buckets in `keys`, offsets with G = 1)
};

// The call's device counters (unsigned long long each): list counts and the
// in-bucket kernels' job counters, followed by the call's CallStatus.
//  [0] fill  [1] sort_s  [2] sort_l  [3] refine  [4] fallback  [5] refine2
//  [6] refine3  [7] sort_m  [8..11] job counters of sort_s, sort_l, fallback,
//  sort_m  [12] fill_big  [13] sort_t  [14] job counter of sort_t
//  [16] sort_m0  [17] job counter of sort_m0
constexpr int N_COUNTS = 20;

// Lists produced by classification (device-side counters).
struct Lists {
  JobList fill, sort_s, sort_l, refine, fallback;
  JobList refine2, refine3;  // segments the previous level left above c_large
  JobList sort_m;            // segments in (c_small, c_mid]
  JobList fill_big;          // fills of at least FILL_BIG keys (written by the whole grid)
  JobList sort_t;            // segments of at most c_tiny keys
  JobList sort_m0;           // segments in (c_small, c_mid0]
};

// One refinement level: split the jobs of `in` into sub-buckets, by the model
// (mode 0) or by the job's key range (modes 1 and 2); sub-buckets still above
// c_large go to `next` with kind next_kind.
struct LevelArgs {
  JobList in, next;
  int mode;              // 0: model ids; 1: total-order key range; 2: value range (floats)
  uint32_t next_kind;
  uint32_t kf;           // mode 0: sub-buckets per job (ids from the level-0 pass)
  uint32_t target;       // modes 1-2: keys per sub-bucket aimed at
  uint32_t fmax;         // modes 1-2: most sub-buckets per job (<= MAX_F1)
  // mode 0, jobs of level-0 buckets with heavy values: where each interval
  // starts (the level-0 slot offsets, G per slot) and the sub-bucket map
  const uint64_t* l0offs;
  uint32_t l0G;
  float f0kf;
  uint32_t in_place;     // 1: jobs split in place (counts in cnt, jobs stay in their buffer)
};

struct SortLimits {
  uint64_t c_tiny;       // segments up to this go to the tiny in-bucket kernel
  uint64_t c_small;      // ... up to this to the small one
  uint64_t c_mid0;       // ... up to this to the 384-thread one
  uint64_t c_mid;        // ... up to this to the middle one
  uint64_t c_large;      // ... up to this to the large kernel, above: refine/fallback
  uint64_t l1_target;    // target sub-bucket size of the level-1 split
};

struct Level1Ws {
  void* aux;             // per refine job: tile base, count base, f1, S, T
  unsigned long long* totals;   // [0] tiles, [1] counters, [2] jobs; the in-place split's
                                // [3] job counter (rounds), [4] hole counter, [5] job
                                // counter (known destinations) (8 words)
  uint32_t* cnt;         // counters (cap_c)
  uint64_t* off;         // cap_c + 1
  unsigned long long* cur;   // cap_c
  unsigned long long* jmin;  // per job
  unsigned long long* jmax;  // per job
  void* scan_status;
  size_t scan_status_bytes;
  const uint16_t* sid;   // level-1 ids (positions of the level-0 output)
  uint64_t cap_c;
  uint64_t cap_jobs;
  uint64_t cap_tiles;
};

// In-place variant (ls_inplace.cu): level 0 splits the caller's array in place
// (fragment flush over read positions, device defragment, cleanup); the
// refinement levels and the radix fallback split each segment in place inside
// one CTA.  Per-bucket arrays have f0 entries, per-piece ones P.
struct InPlace0 {
  uint32_t P;                  // pieces (one CTA each in the flush pass)
  uint64_t PL;                 // keys per piece (a multiple of the flush tile)
  uint8_t* flags;              // per block slot: set once its block has been moved
  uint16_t* tags;              // per flushed block slot: its bucket
  uint32_t* prank;             // per flushed block slot: its rank among its bucket's blocks
                               // of its piece (a hole's: its place in hscr)
  uint32_t* inv;               // per slot: the slot whose block goes there (IP_NONE: none)
  uint32_t* pnb;               // per piece and bucket: blocks flushed, then their prefix
  void* hscr;                  // the blocks of the hole slots (hcap blocks)
  uint32_t hcap;
  unsigned int* hcount;        // [0] holes copied, [1] chain starts, [2] starts taken
  uint32_t* starts;            // free destinations: where the defragment's chains start
  uint32_t scap;
  uint32_t* pslots;            // per piece: blocks flushed at its front
  void* lo_keys;               // per piece and bucket: leftover keys (one block each)
  uint32_t* lo_cnt;            // per piece and bucket: leftover count
  unsigned long long* cntb;    // per bucket: non-equality keys
  uint32_t* nbk;               // per bucket: full blocks
  uint32_t* dsl;               // per bucket: first slot of its range
  uint32_t* dend;              // per bucket: end of its slot range
  unsigned long long* sst;     // per bucket: first position
  void* save;                  // per bucket: one block (the overhang into its head)
  void* ovf;                   // one block: the partial last slot of the array
};
constexpr int IP0_THREADS = 1024;
constexpr int IP0_KPT = 8;
constexpr uint32_t IP0_TILE = IP0_THREADS * IP0_KPT;
constexpr uint32_t IP_FANOUT_MAX = 512;   // level-0 buckets of the in-place variant
size_t ip_level0_smem(int dt, uint32_t L, uint32_t f0, uint32_t n_ext_max);
size_t ip_cta_smem(int dt);
cudaError_t ip_configure(int dt, size_t smem0);
cudaError_t ip_level0_enqueue(int dt, const Level0Args& a, const InPlace0& ip, const Lists& lists,
                              const SortLimits& lim, cudaStream_t st, int num_sms,
                              const Marks* mk = nullptr, int mbase = 0);
cudaError_t ip_levels_enqueue(int dt, void* keys, const ModelPtrs& M, const Lists& lists,
                              const SortLimits& lim, const Level1Ws& w, const InPlace0& ip,
                              uint32_t kf, float f0kf, const uint64_t* l0offs, uint32_t* err,
                              cudaStream_t st, int num_sms, bool range_levels = true);

// Single launches of the level kernels (each counts itself in add_launches).
cudaError_t launch_classify0(int dt, const Level0Args& a, const Lists& lists, const SortLimits& lim,
                             cudaStream_t st);
cudaError_t launch_l1_plan(const LevelArgs& la, const SortLimits& lim, const Level1Ws& w,
                           uint32_t* err, cudaStream_t st);
cudaError_t launch_l1_minmax(int dt, const void* keys, const LevelArgs& la, const Level1Ws& w,
                             cudaStream_t st, int num_sms);
cudaError_t launch_l1_classify(int dt, const Lists& lists, const LevelArgs& la,
                               const SortLimits& lim, const Level1Ws& w, const ModelPtrs& M,
                               uint32_t* err, cudaStream_t st, int num_sms);

size_t level0_smem_hist(int dt, uint32_t L, uint32_t f0, uint32_t n_ext_max);
size_t level0_smem_scatter(int dt, uint32_t L, uint32_t f0, uint32_t n_ext_max);
cudaError_t level0_configure(int dt, size_t smem_hist, size_t smem_scatter);
cudaError_t level0_enqueue(int dt, const Level0Args& a, size_t smem_hist, size_t smem_scatter,
                           const Lists& lists, const SortLimits& lim, cudaStream_t st,
                           const Marks* mk = nullptr, int mbase = 0);
cudaError_t level1_enqueue(int dt, void* keys, void* scratch, uint64_t n, const ModelPtrs& M,
                           const Lists& lists, const SortLimits& lim, const Level1Ws& w,
                           uint32_t kf, float f0kf, const uint64_t* l0offs, uint32_t l0G,
                           uint32_t* err, cudaStream_t st, int num_sms, bool range_levels = true);
cudaError_t levels_enqueue(int dt, void* keys, void* scratch, uint64_t n, const ModelPtrs& M,
                           const Lists& lists, const SortLimits& lim, const Level1Ws& w,
                           const LevelArgs* lvs, int nlv, uint32_t* err, cudaStream_t st,
                           int num_sms);
// Fill jobs [from, upto) of the two fill lists ({small, big} positions in
// device memory; null: the start / the lists' counts when the kernel runs).
cudaError_t fill_enqueue(int dt, void* keys, const Lists& lists, const unsigned long long* from,
                         const unsigned long long* upto, cudaStream_t st, int num_sms);
cudaError_t buckets_configure(int dt);
cudaError_t buckets_enqueue(int dt, void* keys, void* scratch, uint64_t n, const ModelPtrs& M,
                            const Lists& lists, uint64_t cap_s, uint64_t cap_l,
                            uint64_t cap_fb, unsigned long long* job_ctrs, uint32_t* err,
                            cudaStream_t st, int num_sms, const Marks* mk = nullptr,
                            int mbase = 0, bool in_place = false);

}  // namespace ls

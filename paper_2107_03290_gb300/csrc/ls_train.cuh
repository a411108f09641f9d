// Host-side interface of the training step (ls_train.cu).
#pragma once
#include <algorithm>

#include "ls_internal.cuh"

namespace ls {

// Regions of the call's workspace that must start at zero, cleared by the
// first kernel of the training step instead of by separate memsets (a memset
// between two kernels would also break their dependent-launch overlap).
// Pointers and sizes are multiples of 4 bytes.
constexpr int ZERO_REGIONS = 10;
struct ZeroList {
  void* p[ZERO_REGIONS];
  uint32_t words[ZERO_REGIONS];  // 4-byte words
};

struct TrainPlan {
  uint64_t s;        // sample size
  uint64_t seed;
  uint64_t tau;      // heavy run-length threshold in the sample (UINT64_MAX: none)
  uint32_t L;        // leaves
  uint32_t f0;       // level-0 fan-out
  uint32_t hpb;      // heavy values per bucket (<= MAX_HPB)
  ZeroList zero;     // cleared by the first training kernel (unused entries: null)
  CallStatus* cs;    // the call's status block, initialised there too (null: none)
  uint32_t stall;
  unsigned long long spin_limit;
};

constexpr int FIT_BLOCKS = 304;     // blocks of the root least-squares sums

// The training sample is sorted by the LSD radix sort for 4-byte keys (their
// four constant high digits are skipped) and for samples of at most 2^17
// keys, whose few tiles per pass beat the sample sort's fixed cost (measured:
// 1M keys, a 10K-key sample: training 0.22 -> 0.20 ms); larger samples of
// 8-byte keys take the sample sort (200M keys: 0.54 ms against 0.61 ms).
inline bool sample_by_radix(int key_width, uint64_t s) { return key_width == 4 || s <= (1ull << 17); }

struct TrainWs {
  uint64_t* smp_a;           // s
  uint64_t* smp_b;           // s
  uint32_t* rank;            // s
  uint32_t* flags;           // s
  uint64_t* cpos;            // s + 1
  void* cand;                // cand_cap * 24 bytes
  uint64_t cand_cap;
  uint64_t* sel;             // f0 * hpb selected heavy values, per bucket by key
  uint32_t* sellen;          // f0 * hpb their sample run lengths
  uint32_t* hlen;            // f0 * hpb run length of each heavy-list entry
  uint32_t* nh;              // f0
  double* partials;          // 4 * FIT_BLOCKS
  uint32_t* ubase;           // L + 1 (first fit unit of each leaf)
  uint32_t* utotal;          // 1
  double* units;             // 4 * (s / 2048 + L + 1) unit partial sums
  unsigned long long* hi;    // 1
  void* scan_status;         // scan tiles * 8 + 16 bytes
  size_t scan_status_bytes;
  SsWork ss;                 // work area of the sample sort (8-byte keys)
  RsWork rs;                 // work area of the radix sort (4-byte keys)
};

cudaError_t train_enqueue(int dt, const void* keys, uint64_t n, const TrainPlan& P,
                          const TrainWs& W, const ModelPtrs& M, uint32_t* err, cudaStream_t st,
                          int num_sms);
cudaError_t sample_sort_u64_enqueue(uint64_t* a, uint64_t* b, uint64_t m, const SsWork& w,
                                    uint32_t* err, cudaStream_t st, int num_sms);
cudaError_t radix_sort_u64_enqueue(uint64_t* a, uint64_t* b, uint64_t m, const RsWork& w,
                                   uint32_t* err, cudaStream_t st, int num_sms);

}  // namespace ls

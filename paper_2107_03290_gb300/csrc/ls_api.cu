// Host runtime and C ABI of the learned sort (include/ls.h).
//
// Per call: plan (fan-out, sample size, heavy threshold, grid), carve one
// stream-ordered workspace allocation from a per-device memory pool, enqueue
// the hot path and return.  The path is, in stream order:
//   train (sample, sort sample, FP64 fit, FP32 evaluation, heavy set)
//   level 0: K2 histogram -> K3 look-back scan -> K4 scatter -> classify
//   level 1: re-partition of slots larger than one in-bucket CTA
//   equality / homogeneous fills, in-bucket counting sorts, radix fallback
// No host synchronization happens inside a call unless statistics are asked.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ls_inplace.cuh"
#include "ls_internal.cuh"
#include "ls_partition.cuh"
#include "ls_radix.cuh"
#include "ls_train.cuh"
#include "ls_tuned.h"

namespace ls {

// Persistent status blocks, one per stream that has called into the library
// (slot 0: the legacy default stream).  A stream's calls OR their errors into
// its block; ls_stream_status reads and clears it.  The slot of a stream is
// found in a fixed open-addressing table (no allocation); when the table is
// full, later streams share slots by hash.
constexpr int STATUS_SLOTS = 1024;
constexpr int MAX_DEVICES = 64;
__device__ CallStatus g_stream_status[STATUS_SLOTS];

struct SlotTable {
  std::atomic<uintptr_t> key[STATUS_SLOTS];   // stream handle + 1 (0: free)
  std::atomic<uint32_t> stall[STATUS_SLOTS];  // test hooks of ls_debug_set_wait
  std::atomic<unsigned long long> limit[STATUS_SLOTS];
};
static SlotTable g_slots[MAX_DEVICES];

static int slot_of(int dev, cudaStream_t st, bool insert) {
  if (dev < 0 || dev >= MAX_DEVICES) return 0;
  SlotTable& t = g_slots[dev];
  const uintptr_t k = (uintptr_t)st + 1;
  if (st == nullptr) {
    uintptr_t z = 0;
    t.key[0].compare_exchange_strong(z, k);
    return 0;
  }
  const uint64_t h = ((uint64_t)k * 0x9E3779B97F4A7C15ull) >> 40;
  for (int p = 0; p < STATUS_SLOTS - 1; ++p) {
    const int i = 1 + (int)((h + p) % (STATUS_SLOTS - 1));
    uintptr_t cur = t.key[i].load(std::memory_order_acquire);
    if (cur == k) return i;
    if (cur == 0) {
      if (!insert) return -1;
      if (t.key[i].compare_exchange_strong(cur, k) || cur == k) return i;
    }
  }
  return insert ? 1 + (int)(h % (STATUS_SLOTS - 1)) : -1;  // full: shared by hash
}

// Device address of the current device's persistent blocks (looked up once
// per device with that device current; no allocation of any kind).
static std::atomic<CallStatus*> g_slot_base[MAX_DEVICES];
static cudaError_t slot_base(int id, CallStatus** out) {
  if (id < 0 || id >= MAX_DEVICES) return cudaErrorInvalidDevice;
  CallStatus* b = g_slot_base[id].load(std::memory_order_acquire);
  if (!b) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_stream_status);
    if (e) return e;
    b = (CallStatus*)p;
    g_slot_base[id].store(b, std::memory_order_release);
  }
  *out = b;
  return cudaSuccess;
}

static std::atomic<unsigned long long> g_launches{0};
void add_launches(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ORs a call's error word into its persistent block (stream or request).
__global__ void k_status_fold(const CallStatus* __restrict__ local, CallStatus* to) {
  pdl_begin();
  const uint32_t w = local->word;
  if (w) atomicOr(&to->word, w);
}

// Pinned host staging for small uploads (the batched entry's job lists): a
// chunk is reused once the event recorded after its copy has completed, so
// uploads never go through pageable memory (which would wait for the stream).
struct Staging {
  void* host = nullptr;
  size_t bytes = 0;
  cudaEvent_t done = nullptr;
  bool busy = false;     // handed out, event not yet recorded
};

struct Device {
  int id = -1;
  int num_sms = 0;
  cudaMemPool_t pool = nullptr;
  CallStatus* slots = nullptr;   // device address of g_stream_status
  bool configured[4] = {false, false, false, false};
  std::vector<Staging> staging;
};

static std::mutex g_mu;
static std::map<int, Device> g_dev;

// A pinned chunk of at least `bytes` whose previous copy has completed.
static cudaError_t staging_acquire(Device* d, size_t bytes, Staging** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (Staging& s : d->staging) {
    if (!s.busy && s.bytes >= bytes && cudaEventQuery(s.done) == cudaSuccess) {
      s.busy = true;
      *out = &s;
      return cudaSuccess;
    }
  }
  Staging s;
  s.bytes = std::max<size_t>(bytes, 1 << 20);
  cudaError_t e = cudaHostAlloc(&s.host, s.bytes, cudaHostAllocDefault);
  if (e) return e;
  e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
  if (e) { cudaFreeHost(s.host); return e; }
  d->staging.reserve(64);
  if (d->staging.size() >= 64) { cudaFreeHost(s.host); cudaEventDestroy(s.done); return cudaErrorMemoryAllocation; }
  s.busy = true;
  d->staging.push_back(s);
  *out = &d->staging.back();
  return cudaSuccess;
}

static void staging_release(Staging* s) {
  std::lock_guard<std::mutex> lk(g_mu);
  s->busy = false;
}

static ls_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return LS_OK;
  if (e == cudaErrorMemoryAllocation) return LS_ERR_NOMEM;
  return LS_ERR_CUDA;
}

static cudaError_t get_device(Device** out) {
  int id;
  cudaError_t e = cudaGetDevice(&id);
  if (e) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  Device& d = g_dev[id];
  if (d.id < 0) {
    d.id = id;
    e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, id);
    if (e) return e;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = id;
    e = cudaMemPoolCreate(&d.pool, &props);
    if (e) return e;
    uint64_t thr = ~0ull;
    e = cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e) return e;
    e = slot_base(id, &d.slots);
    if (e) return e;
  }
  *out = &d;
  return cudaSuccess;
}

cudaError_t stream_status_ptr(cudaStream_t st, uint32_t** out) {
  int id;
  cudaError_t e = cudaGetDevice(&id);
  if (e) return e;
  CallStatus* b;
  if ((e = slot_base(id, &b))) return e;
  *out = &b[slot_of(id, st, true)].word;
  return cudaSuccess;
}

static CallOpts stream_opts(Device* d, cudaStream_t st) {
  const int i = slot_of(d->id, st, true);
  CallOpts o;
  o.fold_to = &d->slots[i];
  o.stall = 0;
  o.spin_limit = 0;
  if (d->id >= 0 && d->id < MAX_DEVICES) {
    o.stall = g_slots[d->id].stall[i].load(std::memory_order_relaxed);
    o.spin_limit = g_slots[d->id].limit[i].load(std::memory_order_relaxed);
  }
  return o;
}

static cudaError_t end_call(const unsigned long long* counts, size_t n_counts, const CallOpts& o,
                            cudaStream_t st) {
  launch_k(k_status_fold, 1, 1, 0, st, (const CallStatus*)(counts + n_counts), o.fold_to);
  add_launches(1);
  return cudaGetLastError();
}

static cudaError_t configure(Device* d, int dt) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (d->configured[dt]) return cudaSuccess;
  cudaError_t e = level0_configure(dt, 227 * 1024, 227 * 1024);
  if (e) return e;
  e = buckets_configure(dt);
  if (e) return e;
  e = ip_configure(dt, 227 * 1024);
  if (e) return e;
  d->configured[dt] = true;
  return cudaSuccess;
}

static int width_of(int dt) { return (dt == LS_F64 || dt == LS_U64) ? 8 : 4; }

// ---------------------------------------------------------------- planning
struct Plan {
  int dt, W;
  uint64_t n;
  uint32_t L, f0, hpb, n_ext_max;
  uint64_t s, tau, seed;
  Chunking c;
  SortLimits lim;
  uint64_t cap0, cap1, cap_c, cap_r, capj, cap_fill;
  uint32_t kf;
  size_t smem_hist, smem_scatter;
  uint32_t l0_scan_tiles;
  bool ip;                 // the in-place variant (LS_FLAG_IN_PLACE)
  uint32_t ip_P;           // in place: level-0 pieces
  uint64_t ip_PL;          // in place: keys per piece
  size_t smem_ip0;
};

static const size_t SMEM_LIMIT = 227 * 1024;

static void plan_call(const ls_params* prm, int dt, uint64_t n, uintptr_t addr, int num_sms,
                      Plan* P) {
  ls_params d;
  ls_default_params(&d);
  const ls_params& p = *prm;
  P->dt = dt;
  P->W = width_of(dt);
  P->n = n;
  P->L = std::min<uint32_t>(MAX_LEAVES, std::max<uint32_t>(1, p.leaves ? p.leaves : d.leaves));
  // level 0: 256 buckets, so that a 4096-key tile writes runs of ~16 keys
  P->f0 = std::min<uint32_t>(MAX_FANOUT, std::max<uint32_t>(1, p.fanout ? p.fanout : 256));
  // in place: one fragment block per bucket stays in shared memory
  P->ip = (p.flags & LS_FLAG_IN_PLACE) != 0;
  // (in place, the planner's fan-out is 512: more, smaller segments for the
  // one-CTA-per-segment level 1, measured 1-5% faster than 256 at 200M keys)
  if (P->ip) P->f0 = p.fanout ? std::min<uint32_t>(P->f0, IP_FANOUT_MAX) : IP_FANOUT_MAX;
  const uint32_t div = p.sample_div ? p.sample_div : d.sample_div;
  uint64_t s = (n + div - 1) / div;
  s = std::max<uint64_t>(s, std::min<uint64_t>(n, 2ull * P->L));
  if (p.sample_max) s = std::min<uint64_t>(s, p.sample_max);
  s = std::min<uint64_t>(s, n);
  s = std::min<uint64_t>(s, 1ull << 29);
  P->s = std::max<uint64_t>(s, 1);
  P->seed = p.seed;
  P->lim.c_tiny = 512;
  P->lim.c_small = 2048;
  P->lim.c_mid0 = 3072;
  P->lim.c_mid = 4096;
  P->lim.c_large = 8192;
  P->lim.l1_target = 3072;
  // heavy values: per-bucket count limited by shared memory of the scatter
  uint32_t hpb = (p.flags & LS_FLAG_NO_HEAVY) ? 0
                 : (p.heavy_per_bucket ? p.heavy_per_bucket : (P->f0 <= 512 ? MAX_HPB : 4));
  hpb = std::min<uint32_t>(hpb, MAX_HPB);
  while (true) {
    const uint32_t next = P->f0 * (1 + 2 * hpb);
    if (next < 65000 && (P->ip ? ip_level0_smem(dt, P->L, P->f0, next) <= SMEM_LIMIT
                               : (level0_smem_scatter(dt, P->L, P->f0, next) <= SMEM_LIMIT &&
                                  level0_smem_hist(dt, P->L, P->f0, next) <= SMEM_LIMIT)))
      break;
    if (hpb == 0) break;
    --hpb;
  }
  P->hpb = hpb;
  P->n_ext_max = P->f0 * (1 + 2 * hpb);
  const uint64_t hmc = p.heavy_min_count ? p.heavy_min_count : P->lim.c_large / 2;
  if (hpb == 0) {
    P->tau = P->s + 1;
  } else {
    const unsigned __int128 num = (unsigned __int128)hmc * P->s + n - 1;
    P->tau = std::max<uint64_t>(2, (uint64_t)(num / n));
  }
  // chunking of the aligned body
  // body: 16-byte aligned keys, a multiple of 4 keys per chunk so that the
  // 4-byte ids of a chunk are 16-byte aligned too
  const uint64_t V = 4;
  uint64_t a0 = ((16 - (addr & 15)) & 15) / P->W;
  a0 = std::min<uint64_t>(a0, n);
  const uint64_t nb = ((n - a0) / V) * V;
  P->c.n = n;
  P->c.a0 = a0;
  P->c.a1 = a0 + nb;
  uint64_t G = std::min<uint64_t>((uint64_t)num_sms, std::max<uint64_t>(1, (nb + P_TILE - 1) / P_TILE));
  uint64_t ch = (nb + G - 1) / G;
  ch = (ch + V - 1) / V * V;
  if (ch == 0) ch = V;
  P->c.ch = ch;
  P->c.G = (uint32_t)G;
  if (P->ip) {
    // level 0 in place: pieces of whole flush tiles, one CTA each, the level-0
    // offsets kept once per slot (G = 1)
    P->c.a0 = 0;
    P->c.a1 = n;
    P->c.ch = n;
    P->c.G = 1;
    G = 1;
    const uint64_t tiles = std::max<uint64_t>(1, (n + IP0_TILE - 1) / IP0_TILE);
    const uint64_t pieces = std::min<uint64_t>((uint64_t)num_sms, tiles);
    P->ip_PL = (tiles + pieces - 1) / pieces * IP0_TILE;
    P->ip_P = (uint32_t)((n + P->ip_PL - 1) / P->ip_PL);
    P->smem_ip0 = ip_level0_smem(dt, P->L, P->f0, P->n_ext_max);
  } else {
    P->ip_P = 0;
    P->ip_PL = 0;
    P->smem_ip0 = 0;
  }
  P->smem_hist = level0_smem_hist(dt, P->L, P->f0, P->n_ext_max);
  P->smem_scatter = level0_smem_scatter(dt, P->L, P->f0, P->n_ext_max);
  // level-1 sub-buckets per bucket: buckets of about l1_target keys each
  const uint64_t per = (uint64_t)P->f0 * P->lim.l1_target;
  // (ids sub + interval stay below MAX_F1 with up to MAX_HPB heavy values)
  P->kf = (uint32_t)std::min<uint64_t>(MAX_F1 - MAX_HPB, std::max<uint64_t>(1, (n + per - 1) / per));
  // in place, a split keeps at most IP_CTA_FMAX sub-buckets (ids sub + interval)
  if (P->ip) P->kf = std::min<uint32_t>(P->kf, IP_CTA_FMAX - MAX_HPB - 1);
  P->cap0 = P->n_ext_max + 16;
  P->cap_r = n / (P->lim.c_large + 1) + 16;     // jobs a refinement level can pass on
  P->capj = std::max(P->cap0, P->cap_r);        // jobs of one refinement level
  // sub-buckets of one level: level 1 splits at most one job per level-0
  // bucket into Kf + (its heavy values) sub-buckets; a key-range level at
  // most n / 32 + n / (l1_target / 3) + its jobs
  P->cap_c = std::max((uint64_t)(P->kf + MAX_HPB) * (P->f0 + 16),
                      n / 32 + n / (P->lim.l1_target / 3) + P->capj) + 64;
  P->cap1 = P->cap_c + P->cap0;
  // fills: the equality slots, and one per homogeneous job of the two
  // key-range levels
  P->cap_fill = P->n_ext_max + 2 * P->cap_r + 64;
  const uint64_t M = (uint64_t)P->n_ext_max * G;
  P->l0_scan_tiles = (uint32_t)std::max<uint64_t>(1, (M + SC_TILE - 1) / SC_TILE);
}

// ---------------------------------------------------------------- workspace
struct Carver {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    off = (off + 255) / 256 * 256;
    const size_t o = off;
    off += count * sizeof(T);
    return o;
  }
};

struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
  // offsets
  size_t o_scratch, o_smp_a, o_smp_b, o_rank, o_flags, o_cpos, o_cand, o_sel, o_sellen, o_hlen, o_nh, o_part, o_hi,
      o_tscan, o_ss_spl, o_ss_words, o_rs_hist, o_rs_skip, o_rs_status, o_hdr, o_leaf64, o_thr, o_cell, o_cleaf, o_hkey, o_hval, o_heads, o_heavy,
      o_lbeg, o_lend, o_hist, o_offs, o_l0scan, o_jobs_fill, o_jobs_s, o_jobs_l, o_jobs_m, o_jobs_m0, o_jobs_fb2, o_jobs_t, o_jobs_r,
      o_jobs_fb, o_jobs_r2, o_jobs_r3, o_pk, o_sid, o_ccount, o_counts, o_aux, o_tot, o_l1cnt, o_l1off, o_l1cur, o_jmin, o_jmax, o_l1scan,
      o_ubase, o_units;
  // in place
  size_t o_ip_flags, o_ip_tags, o_ip_prank, o_ip_inv, o_ip_pnb, o_ip_hscr, o_ip_hcount, o_ip_pslots,
      o_ip_lokeys, o_ip_locnt, o_ip_cntb, o_ip_nbk, o_ip_dsl, o_ip_dend, o_ip_sst, o_ip_save, o_ip_ovf,
      o_ip_starts;
  uint32_t ip_hcap, ip_scap;
  size_t tscan_bytes, rs_status_bytes, l0scan_bytes, l1scan_bytes;
  uint64_t cand_cap;
};

// Jobs of more than `m` keys cover disjoint key ranges: at most n / (m + 1) of them.
static uint64_t cap_above(uint64_t n, uint64_t m) { return n / (m + 1) + 16; }

static void layout_ws(const Plan& P, Workspace* w, bool with_scratch) {
  Carver c;
  const uint64_t s = P.s;
  w->o_scratch = c.take<uint8_t>(with_scratch ? P.n * P.W : 0);
  w->o_smp_a = c.take<uint64_t>(s);
  w->o_smp_b = c.take<uint64_t>(s);
  w->o_rank = c.take<uint32_t>(s);
  w->o_flags = c.take<uint32_t>(s);
  w->o_cpos = c.take<uint64_t>(s + 1);
  w->cand_cap = s / std::max<uint64_t>(1, P.tau) + 2;
  w->o_cand = c.take<uint8_t>(w->cand_cap * 24);
  w->o_sel = c.take<uint64_t>((size_t)P.f0 * std::max<uint32_t>(1, P.hpb));
  w->o_sellen = c.take<uint32_t>((size_t)P.f0 * std::max<uint32_t>(1, P.hpb));
  w->o_hlen = c.take<uint32_t>((size_t)P.f0 * std::max<uint32_t>(1, P.hpb));
  w->o_nh = c.take<uint32_t>(P.f0);
  w->o_part = c.take<double>(4 * FIT_BLOCKS);
  w->o_ubase = c.take<uint32_t>(P.L + 2);
  w->o_units = c.take<double>(4 * (P.s / 2048 + P.L + 2));
  w->o_hi = c.take<uint64_t>(1);
  const uint64_t stiles = std::max<uint64_t>(1, (s + SC_TILE - 1) / SC_TILE);
  w->tscan_bytes = stiles * 8 + 16;
  w->o_tscan = c.take<uint8_t>(w->tscan_bytes);
  w->o_ss_spl = c.take<uint64_t>(SS_P);
  w->o_ss_words = c.take<uint32_t>(ss_work_words());
  const bool narrow = sample_by_radix(P.W, s);  // the sample is sorted by radix
  w->o_rs_hist = c.take<uint32_t>(narrow ? 8 * 256 : 0);
  w->o_rs_skip = c.take<uint32_t>(narrow ? 8 : 0);
  w->rs_status_bytes = narrow ? rs_status_words(s) * 4 + 8 * 4 : 0;
  w->o_rs_status = c.take<uint8_t>(w->rs_status_bytes);
  w->o_hdr = c.take<DevModel>(1);
  w->o_leaf64 = c.take<double>(5 * (size_t)P.L);
  w->o_thr = c.take<uint64_t>(P.f0);
  w->o_cell = c.take<uint32_t>(L0_CELLS);
  w->o_cleaf = c.take<CellLeaf>(P.L);
  w->o_hkey = c.take<uint64_t>(HASH_SIZE);
  w->o_hval = c.take<uint16_t>(HASH_SIZE);
  w->o_heads = c.take<BucketHead>(P.f0 + 1);
  w->o_heavy = c.take<HeavyEntry>((size_t)P.f0 * std::max<uint32_t>(1, P.hpb));
  w->o_lbeg = c.take<uint32_t>(P.L);
  w->o_lend = c.take<uint32_t>(P.L);
  w->o_hist = c.take<uint32_t>((size_t)P.n_ext_max * P.c.G);
  w->o_offs = c.take<uint64_t>((size_t)P.n_ext_max * P.c.G + 1);
  w->l0scan_bytes = (size_t)P.l0_scan_tiles * 8 + 16;
  w->o_l0scan = c.take<uint8_t>(w->l0scan_bytes);
  w->o_jobs_fill = c.take<Job>(P.cap_fill);
  w->o_jobs_s = c.take<Job>(cap_above(P.n, P.lim.c_tiny));
  w->o_jobs_l = c.take<Job>(cap_above(P.n, P.lim.c_mid));
  w->o_jobs_m = c.take<Job>(cap_above(P.n, P.lim.c_small));
  w->o_jobs_m0 = c.take<Job>(cap_above(P.n, P.lim.c_small));
  w->o_jobs_fb2 = c.take<Job>(cap_above(P.n, FILL_BIG - 1));
  w->o_jobs_t = c.take<Job>(P.cap1);
  w->o_jobs_r = c.take<Job>(P.cap0);
  w->o_jobs_fb = c.take<Job>(cap_above(P.n, P.lim.c_large));
  w->o_pk = c.take<uint32_t>(with_scratch ? P.n + 16 : 0);
  w->o_ccount = c.take<uint64_t>(P.c.G + 1);
  w->o_sid = c.take<uint16_t>(with_scratch ? P.n + 16 : 0);
  w->o_jobs_r2 = c.take<Job>(P.cap_r);
  w->o_jobs_r3 = c.take<Job>(P.cap_r);
  w->o_counts = c.take<unsigned long long>(N_COUNTS + 2);  // counters + the call's CallStatus
  w->o_aux = c.take<uint8_t>((P.capj + 1) * 32);
  w->o_tot = c.take<unsigned long long>(8);
  w->o_l1cnt = c.take<uint32_t>(P.cap_c);
  w->o_l1off = c.take<uint64_t>(P.cap_c + 1);
  w->o_l1cur = c.take<unsigned long long>(P.cap_c);
  w->o_jmin = c.take<unsigned long long>(P.capj);
  w->o_jmax = c.take<unsigned long long>(P.capj);
  const uint64_t l1tiles = std::max<uint64_t>(1, (P.cap_c + SC_TILE - 1) / SC_TILE);
  w->l1scan_bytes = l1tiles * 8 + 16;
  w->o_l1scan = c.take<uint8_t>(w->l1scan_bytes);
  if (P.ip) {
    const uint64_t B = IP_BLOCK_BYTES / P.W;
    const uint64_t blocks = (uint64_t)P.ip_P * P.f0;
    const uint64_t slots = (P.n + B - 1) / B;
    w->o_ip_flags = c.take<uint8_t>(slots + 16);
    w->o_ip_tags = c.take<uint16_t>(slots + 16);
    w->o_ip_prank = c.take<uint32_t>(slots + 16);
    w->o_ip_inv = c.take<uint32_t>(slots + 16);
    w->o_ip_pnb = c.take<uint32_t>(blocks);
    // holes: one slot in 32 on average; room for twice that
    w->ip_hcap = (uint32_t)(slots / 16 + 1024);
    w->o_ip_hscr = c.take<uint8_t>((size_t)w->ip_hcap * IP_BLOCK_BYTES);
    w->o_ip_hcount = c.take<uint32_t>(4);
    // chain starts: destinations that are holes or held no block (the slots
    // freed by equality keys among them), at most one per slot
    w->ip_scap = (uint32_t)(slots + 16);
    w->o_ip_starts = c.take<uint32_t>(w->ip_scap);
    w->o_ip_pslots = c.take<uint32_t>(P.ip_P);
    w->o_ip_lokeys = c.take<uint8_t>(blocks * IP_BLOCK_BYTES);
    w->o_ip_locnt = c.take<uint32_t>(blocks);
    w->o_ip_cntb = c.take<unsigned long long>(P.f0);
    w->o_ip_nbk = c.take<uint32_t>(P.f0);
    w->o_ip_dsl = c.take<uint32_t>(P.f0);
    w->o_ip_dend = c.take<uint32_t>(P.f0);
    w->o_ip_sst = c.take<unsigned long long>(P.f0);
    w->o_ip_save = c.take<uint8_t>((size_t)P.f0 * IP_BLOCK_BYTES);
    w->o_ip_ovf = c.take<uint8_t>(IP_BLOCK_BYTES);
  }
  w->bytes = c.off + 256;
}

template <typename T>
static T* at(const Workspace& w, size_t o) {
  return (T*)((char*)w.base + o);
}

struct Bound {
  ModelPtrs M;
  TrainWs T;
  Lists lists;
  Level1Ws l1;
  unsigned long long* counts;  // [0..7], [12], [13] list counts, [8..11], [14] job counters
};

static Bound bind(const Plan& P, const Workspace& w) {
  Bound b{};
  b.M.hdr = at<DevModel>(w, w.o_hdr);
  b.M.leaf64 = at<double>(w, w.o_leaf64);
  b.M.thr = at<uint64_t>(w, w.o_thr);
  b.M.cell = at<uint32_t>(w, w.o_cell);
  b.M.cleaf = at<CellLeaf>(w, w.o_cleaf);
  b.M.hkey = at<uint64_t>(w, w.o_hkey);
  b.M.hval = at<uint16_t>(w, w.o_hval);
  b.M.heads = at<BucketHead>(w, w.o_heads);
  b.M.heavy = at<HeavyEntry>(w, w.o_heavy);
  b.M.leaf_beg = at<uint32_t>(w, w.o_lbeg);
  b.M.L = (int)P.L;
  b.M.leaf_end = at<uint32_t>(w, w.o_lend);
  TrainWs& T = b.T;
  T.smp_a = at<uint64_t>(w, w.o_smp_a);
  T.smp_b = at<uint64_t>(w, w.o_smp_b);
  T.rank = at<uint32_t>(w, w.o_rank);
  T.flags = at<uint32_t>(w, w.o_flags);
  T.cpos = at<uint64_t>(w, w.o_cpos);
  T.cand = at<void>(w, w.o_cand);
  T.cand_cap = w.cand_cap;
  T.sel = at<uint64_t>(w, w.o_sel);
  T.sellen = at<uint32_t>(w, w.o_sellen);
  T.hlen = at<uint32_t>(w, w.o_hlen);
  T.nh = at<uint32_t>(w, w.o_nh);
  T.partials = at<double>(w, w.o_part);
  T.ubase = at<uint32_t>(w, w.o_ubase);
  T.utotal = T.ubase + P.L + 1;
  T.units = at<double>(w, w.o_units);
  T.hi = at<unsigned long long>(w, w.o_hi);
  T.scan_status = at<void>(w, w.o_tscan);
  T.scan_status_bytes = w.tscan_bytes;
  T.ss.spl = at<uint64_t>(w, w.o_ss_spl);
  T.ss.cnt = at<uint32_t>(w, w.o_ss_words);
  T.ss.beg = T.ss.cnt + (SS_NB + 1);
  T.ss.cur = T.ss.beg + (SS_NB + 1);
  T.rs.hist = at<uint32_t>(w, w.o_rs_hist);
  T.rs.skip = at<uint32_t>(w, w.o_rs_skip);
  T.rs.status = at<uint32_t>(w, w.o_rs_status);
  T.rs.ctr = T.rs.status + rs_status_words(P.s);
  b.counts = at<unsigned long long>(w, w.o_counts);
  auto mk = [&](size_t o, unsigned long long* cnt, uint64_t cap) {
    JobList l;
    l.jobs = at<Job>(w, o);
    l.count = cnt;
    l.cap = cap;
    return l;
  };
  b.lists.fill = mk(w.o_jobs_fill, b.counts + 0, P.cap_fill);
  b.lists.sort_s = mk(w.o_jobs_s, b.counts + 1, cap_above(P.n, P.lim.c_tiny));
  b.lists.sort_l = mk(w.o_jobs_l, b.counts + 2, cap_above(P.n, P.lim.c_mid));
  b.lists.sort_m = mk(w.o_jobs_m, b.counts + 7, cap_above(P.n, P.lim.c_small));
  b.lists.fill_big = mk(w.o_jobs_fb2, b.counts + 12, cap_above(P.n, FILL_BIG - 1));
  b.lists.sort_t = mk(w.o_jobs_t, b.counts + 13, P.cap1);
  b.lists.sort_m0 = mk(w.o_jobs_m0, b.counts + 16, cap_above(P.n, P.lim.c_small));
  b.lists.refine = mk(w.o_jobs_r, b.counts + 3, P.cap0);
  b.lists.fallback = mk(w.o_jobs_fb, b.counts + 4, cap_above(P.n, P.lim.c_large));
  b.lists.refine2 = mk(w.o_jobs_r2, b.counts + 5, P.cap_r);
  b.lists.refine3 = mk(w.o_jobs_r3, b.counts + 6, P.cap_r);
  Level1Ws& l = b.l1;
  l.aux = at<void>(w, w.o_aux);
  l.totals = at<unsigned long long>(w, w.o_tot);
  l.cnt = at<uint32_t>(w, w.o_l1cnt);
  l.off = at<uint64_t>(w, w.o_l1off);
  l.cur = at<unsigned long long>(w, w.o_l1cur);
  l.jmin = at<unsigned long long>(w, w.o_jmin);
  l.jmax = at<unsigned long long>(w, w.o_jmax);
  l.scan_status = at<void>(w, w.o_l1scan);
  l.sid = at<uint16_t>(w, w.o_sid);
  l.scan_status_bytes = w.l1scan_bytes;
  l.cap_c = P.cap_c;
  l.cap_jobs = P.capj;
  l.cap_tiles = 0;
  return b;
}

// ---------------------------------------------------------------- the sort
constexpr int NMARK = 11;  // start, train, K2, K3, K4, classify, level1, fill, K5s, K5l, fallback
struct Events {
  cudaEvent_t ev[NMARK];
  bool on = false;
};

#define LS_TRY(x)                       \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return e_;   \
  } while (0)

static cudaError_t enqueue_train(const Plan& P, const Bound& b, const void* keys, Device* d,
                                 uint32_t* err, cudaStream_t st, const ZeroList* zero = nullptr,
                                 CallStatus* cs = nullptr, const CallOpts* o = nullptr) {
  TrainPlan tp{};
  if (zero) tp.zero = *zero;
  tp.cs = cs;
  tp.stall = o ? o->stall : 0u;
  tp.spin_limit = o ? o->spin_limit : 0ull;
  tp.s = P.s;
  tp.seed = P.seed;
  tp.tau = P.tau;
  tp.L = P.L;
  tp.f0 = P.f0;
  tp.hpb = P.hpb;
  return train_enqueue(P.dt, keys, P.n, tp, b.T, b.M, err, st, d->num_sms);
}

static Level0Args level0_args(const Plan& P, const Bound& b, const Workspace& w, const void* keys,
                              uint32_t* err) {
  Level0Args a{};
  a.keys = keys;
  a.scratch = at<void>(w, w.o_scratch);
  a.c = P.c;
  a.M = b.M;
  a.f0 = P.f0;
  a.n_ext_max = P.n_ext_max;
  a.L = P.L;
  a.hist = at<uint32_t>(w, w.o_hist);
  a.offs = at<uint64_t>(w, w.o_offs);
  a.scan_status = at<void>(w, w.o_l0scan);
  a.scan_tiles = P.l0_scan_tiles;
  a.err = err;
  a.pk = at<uint32_t>(w, w.o_pk);
  a.sid = at<uint16_t>(w, w.o_sid);
  a.kf = P.kf;
  a.ccount = at<uint64_t>(w, w.o_ccount);
  a.may_compact = 1;
  a.f0kf = (float)((double)P.f0 * P.kf);
  a.in_place = P.ip ? 1u : 0u;
  return a;
}

// The two key-range levels after the model's level 1 run for arrays above 2^22
// keys; below, a segment the model's split leaves above the in-bucket limit
// goes straight to the radix fallback (one CTA per segment), and 13 launches
// that would find no work are not made.
static bool range_levels(uint64_t n) { return n > (1ull << 22); }

static InPlace0 inplace0_of(const Plan& P, const Workspace& w) {
  InPlace0 ip{};
  ip.P = P.ip_P;
  ip.PL = P.ip_PL;
  ip.flags = at<uint8_t>(w, w.o_ip_flags);
  ip.tags = at<uint16_t>(w, w.o_ip_tags);
  ip.prank = at<uint32_t>(w, w.o_ip_prank);
  ip.inv = at<uint32_t>(w, w.o_ip_inv);
  ip.pnb = at<uint32_t>(w, w.o_ip_pnb);
  ip.hscr = at<void>(w, w.o_ip_hscr);
  ip.hcap = w.ip_hcap;
  ip.hcount = at<unsigned int>(w, w.o_ip_hcount);
  ip.starts = at<uint32_t>(w, w.o_ip_starts);
  ip.scap = w.ip_scap;
  ip.pslots = at<uint32_t>(w, w.o_ip_pslots);
  ip.lo_keys = at<void>(w, w.o_ip_lokeys);
  ip.lo_cnt = at<uint32_t>(w, w.o_ip_locnt);
  ip.cntb = at<unsigned long long>(w, w.o_ip_cntb);
  ip.nbk = at<uint32_t>(w, w.o_ip_nbk);
  ip.dsl = at<uint32_t>(w, w.o_ip_dsl);
  ip.dend = at<uint32_t>(w, w.o_ip_dend);
  ip.sst = at<unsigned long long>(w, w.o_ip_sst);
  ip.save = at<void>(w, w.o_ip_save);
  ip.ovf = at<void>(w, w.o_ip_ovf);
  return ip;
}

// The in-place variant: level 0 and every refinement split inside the
// caller's array (no n-key scratch), then the same fills and in-bucket sorts.
static cudaError_t enqueue_sort_ip(const Plan& P, const Workspace& w, void* keys, Device* d,
                                   cudaStream_t st, Events* ev, const CallOpts& o) {
  const Bound b = bind(P, w);
  Marks mk{ev && ev->on ? ev->ev : nullptr, NMARK};
  uint32_t* err = (uint32_t*)(b.counts + N_COUNTS);
  ZeroList z{};
  z.p[0] = b.counts;
  z.words[0] = N_COUNTS * 2;
  z.p[1] = at<void>(w, w.o_l0scan);
  z.words[1] = (uint32_t)(w.l0scan_bytes / 4);
  z.p[2] = at<void>(w, w.o_hist);           // level-0 slot counts (accumulated)
  z.words[2] = P.n_ext_max;
  z.p[3] = at<void>(w, w.o_ip_cntb);
  z.words[3] = 2 * P.f0;
  z.p[4] = at<void>(w, w.o_ip_nbk);
  z.words[4] = P.f0;
  mark(&mk, 0, st);
  LS_TRY(enqueue_train(P, b, keys, d, err, st, &z, (CallStatus*)err, &o));
  mark(&mk, 1, st);
  Level0Args a = level0_args(P, b, w, keys, err);
  a.scratch = nullptr;
  a.pk = nullptr;
  a.sid = nullptr;
  a.may_compact = 0;
  const InPlace0 ip = inplace0_of(P, w);
  LS_TRY(ip_level0_enqueue(P.dt, a, ip, b.lists, P.lim, st, d->num_sms, &mk, 2));
  LS_TRY(ip_levels_enqueue(P.dt, keys, b.M, b.lists, P.lim, b.l1, ip, P.kf, a.f0kf, a.offs, err,
                           st, d->num_sms, range_levels(P.n)));
  mark(&mk, 6, st);
  LS_TRY(fill_enqueue(P.dt, keys, b.lists, nullptr, nullptr, st, d->num_sms));
  mark(&mk, 7, st);
  LS_TRY(buckets_enqueue(P.dt, keys, nullptr, P.n, b.M, b.lists, P.cap1, P.cap1, P.cap1,
                         b.counts + 8, err, st, d->num_sms, &mk, 8, true));
  LS_TRY(end_call(b.counts, N_COUNTS, o, st));
  mark(&mk, 10, st);
  return cudaSuccess;
}

static cudaError_t enqueue_sort(const Plan& P, const Workspace& w, void* keys, Device* d,
                                cudaStream_t st, Events* ev, const CallOpts& o) {
  if (P.ip) return enqueue_sort_ip(P, w, keys, d, st, ev, o);
  const Bound b = bind(P, w);
  Marks mk{ev && ev->on ? ev->ev : nullptr, NMARK};
  uint32_t* err = (uint32_t*)(b.counts + N_COUNTS);  // the call's own CallStatus
  // the first training kernel zeroes the list counters and the level-0 scan
  // words and initialises the call's status block (no memsets in the stream)
  ZeroList z{};
  z.p[0] = b.counts;
  z.words[0] = N_COUNTS * 2;
  z.p[1] = at<void>(w, w.o_l0scan);
  z.words[1] = (uint32_t)(w.l0scan_bytes / 4);
  mark(&mk, 0, st);
  LS_TRY(enqueue_train(P, b, keys, d, err, st, &z, (CallStatus*)err, &o));
  mark(&mk, 1, st);
  const Level0Args a = level0_args(P, b, w, keys, err);
  LS_TRY(level0_enqueue(P.dt, a, P.smem_hist, P.smem_scatter, b.lists, P.lim, st, &mk, 2));
  LS_TRY(level1_enqueue(P.dt, keys, a.scratch, P.n, b.M, b.lists, P.lim, b.l1, P.kf, a.f0kf,
                        a.offs, P.c.G, err, st, d->num_sms, range_levels(P.n)));
  mark(&mk, 6, st);
  LS_TRY(fill_enqueue(P.dt, keys, b.lists, nullptr, nullptr, st, d->num_sms));
  mark(&mk, 7, st);
  LS_TRY(buckets_enqueue(P.dt, keys, a.scratch, P.n, b.M, b.lists, P.cap1, P.cap1, P.cap1,
                         b.counts + 8, err, st, d->num_sms, &mk, 8));
  LS_TRY(end_call(b.counts, N_COUNTS, o, st));
  mark(&mk, 10, st);
  return cudaSuccess;
}

static ls_status validate(const void* keys, size_t n, int dt) {
  if (dt < LS_F64 || dt > LS_U32) return LS_ERR_INVALID;
  if (n > 0 && !keys) return LS_ERR_INVALID;
  const int W = width_of(dt);
  if ((uintptr_t)keys % W) return LS_ERR_INVALID;
  if (n >= (1ull << 62) / W) return LS_ERR_INVALID;
  return LS_OK;
}

int pool_alloc(void** p, size_t bytes, CUstream_st* st) {
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return (int)e;
  return (int)cudaMallocFromPoolAsync(p, bytes, d->pool, (cudaStream_t)st);
}

void pool_free(void* p, CUstream_st* st) { cudaFreeAsync(p, (cudaStream_t)st); }

static cudaError_t ws_alloc(Device* d, Workspace* w, cudaStream_t st) {
  return cudaMallocFromPoolAsync(&w->base, w->bytes, d->pool, st);
}

static void fill_stats(const Plan& P, const Workspace& w, Events* ev, ls_stats* stats,
                       uint64_t launches) {
  std::memset(stats, 0, sizeof(*stats));
  if (ev->on) {
    auto el = [&](int a, int b) {
      float ms = 0;
      cudaEventElapsedTime(&ms, ev->ev[a], ev->ev[b]);
      return (double)ms;
    };
    stats->ms_total = el(0, 10);
    stats->ms_train = el(0, 1);
    stats->ms_hist = el(1, 2);
    stats->ms_scan = el(2, 3);
    stats->ms_scatter = el(3, 4);
    stats->ms_classify = el(4, 5);
    stats->ms_level1 = el(5, 6);
    stats->ms_fill = el(6, 7);
    stats->ms_sort_small = el(7, 8);
    stats->ms_sort_large = el(8, 9);
    stats->ms_fallback = el(9, 10);
  }
  stats->n_launches = launches;
  stats->workspace_bytes = w.bytes;
  DevModel hdr;
  cudaMemcpy(&hdr, at<void>(w, w.o_hdr), sizeof(hdr), cudaMemcpyDeviceToHost);
  unsigned long long counts[N_COUNTS];
  cudaMemcpy(counts, at<void>(w, w.o_counts), sizeof(counts), cudaMemcpyDeviceToHost);
  stats->sample_size = hdr.s;
  stats->sample_finite = hdr.s_fin;
  stats->fanout = P.f0;
  stats->leaves = P.L;
  stats->n_heavy = hdr.nheavy;
  stats->n_ext = hdr.n_ext;
  stats->n_level1 = counts[3];
  stats->n_segments = counts[1] + counts[2] + counts[7] + counts[13] + counts[16];
  stats->n_fallback = counts[4];
  stats->n_range = counts[5] + counts[6];
  // largest slot and equality keys from the level-0 offsets
  const uint32_t next = std::min<uint32_t>(hdr.n_ext, P.n_ext_max);
  std::vector<uint64_t> offs((size_t)P.n_ext_max * P.c.G + 1);
  cudaMemcpy(offs.data(), at<void>(w, w.o_offs), offs.size() * 8, cudaMemcpyDeviceToHost);
  std::vector<BucketHead> heads(P.f0 + 1);
  cudaMemcpy(heads.data(), at<void>(w, w.o_heads), heads.size() * sizeof(BucketHead),
             cudaMemcpyDeviceToHost);
  uint64_t mx = 0, eq = 0;
  uint32_t b = 0;
  for (uint32_t e = 0; e < next; ++e) {
    while (b + 1 <= P.f0 && heads[b + 1].ext_base <= e) ++b;
    const uint64_t sz = offs[(size_t)(e + 1) * P.c.G] - offs[(size_t)e * P.c.G];
    const uint32_t o = e - heads[b].ext_base, nh = heads[b].hoff_nh & 15u;
    if (nh && (o & 1u)) eq += sz; else mx = std::max(mx, sz);
  }
  stats->max_bucket = mx;
  stats->n_eq_keys = eq;
  stats->n_fill = counts[0] + counts[12];
  auto job_keys = [&](size_t off, uint64_t cnt, uint64_t cap, uint64_t* mxm) {
    std::vector<Job> jobs((size_t)std::min(cnt, cap));
    if (!jobs.empty())
      cudaMemcpy(jobs.data(), at<void>(w, off), jobs.size() * sizeof(Job), cudaMemcpyDeviceToHost);
    uint64_t sum = 0;
    for (const Job& j : jobs) {
      sum += j.m;
      if (mxm) *mxm = std::max<uint64_t>(*mxm, j.m);
    }
    return sum;
  };
  stats->n_fallback_keys = job_keys(w.o_jobs_fb, counts[4], cap_above(P.n, P.lim.c_large),
                                    &stats->max_fallback);
  stats->n_large_keys = job_keys(w.o_jobs_l, counts[2], cap_above(P.n, P.lim.c_mid), nullptr) +
                        job_keys(w.o_jobs_m, counts[7], cap_above(P.n, P.lim.c_small), nullptr) +
                        job_keys(w.o_jobs_m0, counts[16], cap_above(P.n, P.lim.c_small), nullptr);
}

}  // namespace ls

using namespace ls;

extern "C" {

void ls_default_params(ls_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->fanout = 0;               // planner's choice (Sec. 6.1's 1000 on request)
  p->leaves = 1000;
  p->sample_div = 100;
  p->heavy_per_bucket = 0;     // planner's choice
  p->sample_max = 0;
  p->seed = 0;
  p->heavy_min_count = 0;
  p->flags = 0;
}

const char* ls_status_string(ls_status s) {
  switch (s) {
    case LS_OK: return "ok";
    case LS_ERR_INVALID: return "invalid argument";
    case LS_ERR_NOMEM: return "out of memory";
    case LS_ERR_CUDA: return "CUDA error";
    case LS_ERR_TIMEOUT: return "device wait timed out";
    case LS_ERR_BUSY: return "busy: admission refused";
    case LS_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

}  // extern "C"

ls_status ls::sort_call(void* keys, size_t n, ls_dtype dtype, CUstream_st* stream,
                        const ls_params* params, ls_stats* stats, const CallOpts* opts) {
  const ls_status v = validate(keys, n, dtype);
  if (v) return v;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n < 2) return LS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  if ((e = configure(d, dtype))) return to_status(e);
  const CallOpts o = opts ? *opts : stream_opts(d, st);
  ls_params p;
  if (params) p = *params; else ls_default_params(&p);
  Plan P;
  plan_call(&p, dtype, n, (uintptr_t)keys, d->num_sms, &P);
  if (P.ip ? P.smem_ip0 > SMEM_LIMIT : (P.smem_hist > SMEM_LIMIT || P.smem_scatter > SMEM_LIMIT))
    return LS_ERR_INVALID;
  Workspace w;
  layout_ws(P, &w, !P.ip);
  if ((e = ws_alloc(d, &w, st))) return to_status(e);
  Events ev;
  if (stats) {
    ev.on = true;
    for (int i = 0; i < NMARK; ++i) cudaEventCreate(&ev.ev[i]);
  }
  const unsigned long long l0 = g_launches.load();
  e = enqueue_sort(P, w, keys, d, st, &ev, o);
  const unsigned long long l1 = g_launches.load();
  if (e == cudaSuccess && stats) {
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) fill_stats(P, w, &ev, stats, l1 - l0);
  }
  cudaFreeAsync(w.base, st);
  if (stats)
    for (int i = 0; i < NMARK; ++i) cudaEventDestroy(ev.ev[i]);
  return to_status(e);
}

extern "C" {

ls_status ls_sort_ex(void* keys, size_t n, ls_dtype dtype, void* stream, const ls_params* params,
                     ls_stats* stats) {
  return sort_call(keys, n, dtype, (cudaStream_t)stream, params, stats, nullptr);
}

size_t ls_workspace_bytes(size_t n, ls_dtype dtype, const ls_params* params) {
  if (dtype < LS_F64 || dtype > LS_U32 || n < 2) return 0;
  Device* d;
  if (get_device(&d) != cudaSuccess) return 0;
  ls_params p;
  if (params) p = *params; else ls_default_params(&p);
  Plan P;
  plan_call(&p, dtype, n, 0, d->num_sms, &P);
  Workspace w;
  layout_ws(P, &w, !P.ip);
  return w.bytes;
}

ls_status ls_sort(void* keys, size_t n, ls_dtype dtype, void* stream) {
  return sort_call(keys, n, dtype, (cudaStream_t)stream, nullptr, nullptr, nullptr);
}

// Batched sort of many independent arrays in one launch sequence.  Every job
// record names its own array (and its region of one shared scratch buffer), so
// thousands of arrays share the same kernels: arrays of at most 8192 keys are
// in-bucket jobs from the start; larger ones enter the key-range levels (each
// array split by a line through its own key range, twice), and all finish in
// the shared in-bucket sort, fill and fallback launches.
ls_status ls_sort_batch(void* const* keys, const size_t* n, size_t count, ls_dtype dtype,
                        void* stream) {
  return batch_call(keys, n, count, dtype, (cudaStream_t)stream, nullptr);
}

ls_status ls_sort_batch_ex(void* const* keys, const size_t* n, size_t count, ls_dtype dtype,
                           void* stream, const ls_batch_params* params) {
  return batch_call(keys, n, count, dtype, (cudaStream_t)stream, nullptr, params);
}

}  // extern "C"

ls_status ls::batch_call(void* const* keys, const size_t* n, size_t count, ls_dtype dtype,
                         CUstream_st* stream, const CallOpts* opts, const ls_batch_params* bp) {
  if (count > 0 && (!keys || !n)) return LS_ERR_INVALID;
  if (dtype < LS_F64 || dtype > LS_U32) return LS_ERR_INVALID;
  const int W = width_of(dtype);
  uint64_t N = 0;
  for (size_t i = 0; i < count; ++i) {
    const ls_status v = validate(keys[i], n[i], dtype);
    if (v) return v;
    if (n[i] >= 2) N += n[i];
  }
  if (N == 0) return LS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  if ((e = configure(d, dtype))) return to_status(e);
  const CallOpts o = opts ? *opts : stream_opts(d, st);
  SortLimits lim;
  lim.c_tiny = 512;
  lim.c_small = 2048;
  lim.c_mid0 = 3072;
  lim.c_mid = 4096;
  lim.c_large = 8192;
  lim.l1_target = 3072;
  const uint64_t capj = count + N / (lim.c_large + 1) + 16;
  const uint64_t cap_c = N / 32 + N / (lim.l1_target / 3) + capj + 64;
  const uint64_t cap1 = cap_c + count + 64;
  // workspace
  Carver c;
  const size_t o_scr = c.take<uint8_t>(N * W);
  size_t o_list[11];
  const uint64_t caps[11] = {cap1, cap1, cap1, cap1, cap1, capj, capj, cap1, capj, cap1, cap1};
  for (int i = 0; i < 11; ++i) o_list[i] = c.take<Job>(caps[i]);
  const size_t o_counts = c.take<unsigned long long>(N_COUNTS + 2);  // counters + CallStatus
  const size_t o_aux = c.take<uint8_t>((capj + 1) * 32);
  const size_t o_tot = c.take<unsigned long long>(8);
  const size_t o_cnt = c.take<uint32_t>(cap_c);
  const size_t o_off = c.take<uint64_t>(cap_c + 1);
  const size_t o_cur = c.take<unsigned long long>(cap_c);
  const size_t o_jmin = c.take<unsigned long long>(capj);
  const size_t o_jmax = c.take<unsigned long long>(capj);
  const uint64_t tiles = std::max<uint64_t>(1, (cap_c + SC_TILE - 1) / SC_TILE);
  const size_t scan_bytes = (tiles + 1) * sizeof(uint64_t) + 16;
  const size_t o_scan = c.take<uint8_t>(scan_bytes);
  Workspace w;
  w.bytes = c.off + 256;
  if ((e = ws_alloc(d, &w, st))) return to_status(e);
  unsigned long long* counts = at<unsigned long long>(w, o_counts);
  auto mk = [&](int i, int ci) {
    JobList l;
    l.jobs = at<Job>(w, o_list[i]);
    l.count = counts + ci;
    l.cap = caps[i];
    return l;
  };
  Lists lists;
  lists.fill = mk(0, 0);
  lists.sort_s = mk(1, 1);
  lists.sort_l = mk(2, 2);
  lists.fallback = mk(3, 4);
  lists.sort_m = mk(4, 7);
  lists.refine2 = mk(5, 5);
  lists.refine3 = mk(6, 6);
  lists.fill_big = mk(7, 12);
  lists.refine = mk(8, 3);
  lists.sort_t = mk(9, 13);
  lists.sort_m0 = mk(10, 16);
  // initial jobs, one per array
  std::vector<Job> jt, js, jm0, jm, jl, jr;
  uint64_t off = 0;
  char* scr = at<char>(w, o_scr);
  for (size_t i = 0; i < count; ++i) {
    if (n[i] < 2) continue;
    Job j{};
    j.start = 0;
    j.m = n[i];
    j.span = n[i];
    j.src = 0;
    j.kb = (uint64_t)(uintptr_t)keys[i];
    j.sb = (uint64_t)(uintptr_t)(scr + off * W);
    off += n[i];
    if (n[i] <= lim.c_tiny) { j.kind = JOB_SORT_RANGE; jt.push_back(j); }
    else if (n[i] <= lim.c_small) { j.kind = JOB_SORT_RANGE; js.push_back(j); }
    else if (n[i] <= lim.c_mid0) { j.kind = JOB_SORT_RANGE; jm0.push_back(j); }
    else if (n[i] <= lim.c_mid) { j.kind = JOB_SORT_RANGE; jm.push_back(j); }
    else if (n[i] <= lim.c_large) { j.kind = JOB_SORT_RANGE; jl.push_back(j); }
    else {
      j.kind = JOB_REFINE;
      int c = 0;  // the array's size class picks its first split's target
      while (c < 2 && n[i] > TUNED_CLASS_MAX[c]) ++c;
      j.pad = (bp && bp->split_target[c]) ? bp->split_target[c] : TUNED_SPLIT_TARGET[c];
      jr.push_back(j);
    }
  }
  unsigned long long hc[N_COUNTS + 2] = {0};  // list counters, then the call's CallStatus
  {
    CallStatus cs{0u, o.stall, o.spin_limit};
    std::memcpy(&hc[N_COUNTS], &cs, sizeof(cs));
  }
  hc[1] = js.size(); hc[7] = jm.size(); hc[2] = jl.size(); hc[5] = jr.size(); hc[13] = jt.size();
  hc[16] = jm0.size();
  // one pinned upload: the counters, then the five initial lists
  const size_t up_bytes = sizeof(hc) + (jt.size() + js.size() + jm0.size() + jm.size() + jl.size() + jr.size()) * sizeof(Job);
  Staging* sg = nullptr;
  if (!e) e = staging_acquire(d, up_bytes, &sg);
  if (!e) {
    char* hp = (char*)sg->host;
    std::memcpy(hp, hc, sizeof(hc));
    size_t o = sizeof(hc);
    auto put = [&](const std::vector<Job>& v, int i) {
      if (v.empty()) return cudaSuccess;
      std::memcpy(hp + o, v.data(), v.size() * sizeof(Job));
      cudaError_t r = cudaMemcpyAsync(at<void>(w, o_list[i]), hp + o, v.size() * sizeof(Job),
                                      cudaMemcpyHostToDevice, st);
      o += v.size() * sizeof(Job);
      return r;
    };
    e = cudaMemcpyAsync(counts, hp, sizeof(hc), cudaMemcpyHostToDevice, st);
    if (!e) e = put(jt, 9);
    if (!e) e = put(js, 1);
    if (!e) e = put(jm0, 10);
    if (!e) e = put(jm, 4);
    if (!e) e = put(jl, 2);
    if (!e) e = put(jr, 5);
    if (!e) e = cudaEventRecord(sg->done, st);
  }
  if (sg) staging_release(sg);
  if (!e) {
    Level1Ws l{};
    l.aux = at<void>(w, o_aux);
    l.totals = at<unsigned long long>(w, o_tot);
    l.cnt = at<uint32_t>(w, o_cnt);
    l.off = at<uint64_t>(w, o_off);
    l.cur = at<unsigned long long>(w, o_cur);
    l.jmin = at<unsigned long long>(w, o_jmin);
    l.jmax = at<unsigned long long>(w, o_jmax);
    l.scan_status = at<void>(w, o_scan);
    l.scan_status_bytes = scan_bytes;
    l.sid = nullptr;
    l.cap_c = cap_c;
    l.cap_jobs = capj;
    // value range, value range again, total-order key range, then the fallback
    LevelArgs lv[3] = {};
    lv[0].in = lists.refine2; lv[0].next = lists.refine3; lv[0].mode = 2;
    lv[0].next_kind = JOB_REFINE; lv[0].kf = 0; lv[0].target = lim.l1_target;
    lv[1].in = lists.refine3; lv[1].next = lists.refine; lv[1].mode = 2;
    lv[1].next_kind = JOB_REFINE; lv[1].kf = 0; lv[1].target = lim.l1_target / 3;
    lv[2].in = lists.refine; lv[2].next = lists.fallback; lv[2].mode = 1;
    lv[2].next_kind = JOB_FALLBACK; lv[2].kf = 0; lv[2].target = 16;
    lv[0].fmax = lv[1].fmax = MAX_F1;
    lv[2].fmax = 256;
    ModelPtrs M{};
    uint32_t* err = (uint32_t*)(counts + N_COUNTS);
    e = levels_enqueue(dtype, nullptr, nullptr, N, M, lists, lim, l, lv, 3, err, st, d->num_sms);
    if (!e) e = fill_enqueue(dtype, nullptr, lists, nullptr, nullptr, st, d->num_sms);
    if (!e) e = buckets_enqueue(dtype, nullptr, nullptr, N, M, lists, cap1, cap1, cap1, counts + 8,
                                err, st, d->num_sms, nullptr, 0);
    if (!e) e = end_call(counts, N_COUNTS, o, st);
  }
  cudaFreeAsync(w.base, st);
  return to_status(e);
}

extern "C" {

ls_status ls_sort_host(void* host_keys, size_t n, ls_dtype dtype, void* stream,
                       const ls_params* params) {
  const ls_status v = validate(host_keys, n, dtype);
  if (v) return v;
  if (n < 2) return LS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  const size_t bytes = n * (size_t)width_of(dtype);
  void* dk = nullptr;
  if ((e = cudaMallocFromPoolAsync(&dk, bytes, d->pool, st))) return to_status(e);
  e = cudaMemcpyAsync(dk, host_keys, bytes, cudaMemcpyHostToDevice, st);
  ls_status s = LS_OK;
  if (e == cudaSuccess) s = ls_sort_ex(dk, n, dtype, stream, params, nullptr);
  if (e == cudaSuccess && s == LS_OK) e = cudaMemcpyAsync(host_keys, dk, bytes, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(dk, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (s != LS_OK) return s;
  if (e == cudaSuccess) e = e2;
  return to_status(e);
}

ls_status ls_stream_status(void* stream) {
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  cudaStream_t st = (cudaStream_t)stream;
  if ((e = cudaStreamSynchronize(st))) return to_status(e);
  const int i = slot_of(d->id, st, false);
  if (i < 0) return LS_OK;  // no call on this stream yet
  uint32_t* word = &d->slots[i].word;
  uint32_t w = 0;
  if ((e = cudaMemcpyAsync(&w, word, sizeof(w), cudaMemcpyDeviceToHost, st))) return to_status(e);
  if ((e = cudaStreamSynchronize(st))) return to_status(e);
  if (w) {
    if ((e = cudaMemsetAsync(word, 0, sizeof(uint32_t), st))) return to_status(e);
    if ((e = cudaStreamSynchronize(st))) return to_status(e);
  }
  if (w & ERR_TIMEOUT) return LS_ERR_TIMEOUT;
  if (w & ERR_BOUNDS) return LS_ERR_CUDA;
  return LS_OK;
}

ls_status ls_train(const void* keys, size_t n, ls_dtype dtype, void* stream,
                   const ls_params* params, ls_model_export* out) {
  const ls_status v = validate(keys, n, dtype);
  if (v) return v;
  if (!out || n == 0) return LS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  if ((e = configure(d, dtype))) return to_status(e);
  ls_params p;
  if (params) p = *params; else ls_default_params(&p);
  p.flags &= ~LS_FLAG_IN_PLACE;  // the model alone: the regular plan
  Plan P;
  plan_call(&p, dtype, n, (uintptr_t)keys, d->num_sms, &P);
  if (out->leaves < P.L) return LS_ERR_INVALID;
  Workspace w;
  layout_ws(P, &w, false);
  if ((e = ws_alloc(d, &w, st))) return to_status(e);
  const Bound b = bind(P, w);
  uint32_t* err = &d->slots[slot_of(d->id, st, true)].word;
  e = enqueue_train(P, b, keys, d, err, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    DevModel hdr;
    cudaMemcpy(&hdr, b.M.hdr, sizeof(hdr), cudaMemcpyDeviceToHost);
    out->sample_size = hdr.s;
    out->sample_finite = hdr.s_fin;
    std::memcpy(out->root, hdr.root64, sizeof(out->root));
    out->tau = P.tau;
    out->n_heavy = hdr.nheavy;
    if (out->leaf) cudaMemcpy(out->leaf, b.M.leaf64, 5 * sizeof(double) * P.L, cudaMemcpyDeviceToHost);
    out->pos_max = hdr.pos_max;
    if (out->thr && out->fanout >= P.f0)
      cudaMemcpy(out->thr, b.M.thr, sizeof(uint64_t) * P.f0, cudaMemcpyDeviceToHost);
    out->fanout = P.f0;
    if (out->sorted_sample_tk)
      cudaMemcpy(out->sorted_sample_tk, b.T.smp_a, 8 * P.s, cudaMemcpyDeviceToHost);
    if (out->heavy_tk && hdr.nheavy) {
      std::vector<HeavyEntry> hv(hdr.nheavy);
      cudaMemcpy(hv.data(), b.M.heavy, sizeof(HeavyEntry) * hdr.nheavy, cudaMemcpyDeviceToHost);
      for (uint32_t j = 0; j < std::min<uint32_t>(hdr.nheavy, out->max_heavy); ++j)
        out->heavy_tk[j] = hv[j].tk;
    }
    e = cudaGetLastError();
  }
  cudaFreeAsync(w.base, st);
  cudaStreamSynchronize(st);
  return to_status(e);
}

ls_status ls_level0_histogram(const void* keys, size_t n, ls_dtype dtype, void* stream,
                              const ls_params* params, uint64_t* hist_host, size_t max_ext,
                              size_t* n_ext) {
  const ls_status v = validate(keys, n, dtype);
  if (v) return v;
  if (!hist_host || !n_ext || n == 0) return LS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  if ((e = configure(d, dtype))) return to_status(e);
  ls_params p;
  if (params) p = *params; else ls_default_params(&p);
  p.flags &= ~LS_FLAG_IN_PLACE;  // the out-of-place histogram pass
  Plan P;
  plan_call(&p, dtype, n, (uintptr_t)keys, d->num_sms, &P);
  Workspace w;
  layout_ws(P, &w, true);
  if ((e = ws_alloc(d, &w, st))) return to_status(e);
  const Bound b = bind(P, w);
  uint32_t* err = &d->slots[slot_of(d->id, st, true)].word;
  e = cudaMemsetAsync(b.counts, 0, N_COUNTS * sizeof(unsigned long long), st);
  if (!e) e = enqueue_train(P, b, keys, d, err, st);
  if (!e) e = cudaMemsetAsync(at<void>(w, w.o_l0scan), 0, w.l0scan_bytes, st);
  Level0Args a0 = level0_args(P, b, w, keys, err);
  a0.may_compact = 0;  // the histogram entry point leaves `keys` as it is
  if (!e) e = level0_enqueue(P.dt, a0, P.smem_hist, P.smem_scatter,
                             b.lists, P.lim, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (!e) {
    DevModel hdr;
    cudaMemcpy(&hdr, b.M.hdr, sizeof(hdr), cudaMemcpyDeviceToHost);
    const uint32_t next = std::min<uint32_t>(hdr.n_ext, P.n_ext_max);
    std::vector<uint64_t> offs((size_t)P.n_ext_max * P.c.G + 1);
    cudaMemcpy(offs.data(), at<void>(w, w.o_offs), offs.size() * 8, cudaMemcpyDeviceToHost);
    *n_ext = next;
    for (uint32_t x = 0; x < next && x < max_ext; ++x)
      hist_host[x] = offs[(size_t)(x + 1) * P.c.G] - offs[(size_t)x * P.c.G];
    e = cudaGetLastError();
  }
  cudaFreeAsync(w.base, st);
  cudaStreamSynchronize(st);
  return to_status(e);
}

uint64_t ls_kernel_launches(void) { return g_launches.load(); }

ls_status ls_debug_set_wait(void* stream, uint32_t stall, uint64_t spin_limit) {
  Device* d;
  const cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  if (d->id < 0 || d->id >= MAX_DEVICES) return LS_ERR_INVALID;
  const int i = slot_of(d->id, (cudaStream_t)stream, true);
  g_slots[d->id].stall[i].store(stall & STALL_L0_SCAN, std::memory_order_relaxed);
  g_slots[d->id].limit[i].store(spin_limit, std::memory_order_relaxed);
  return LS_OK;
}

ls_status ls_radix_sort_u64(uint64_t* keys, size_t count, void* stream) {
  if (count > 0 && !keys) return LS_ERR_INVALID;
  if (count < 2) return LS_OK;
  if (count >= (1ull << 30)) return LS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  Carver c;
  const size_t o_tmp = c.take<uint64_t>(count);
  const size_t o_hist = c.take<uint32_t>(8 * 256);
  const size_t o_skip = c.take<uint32_t>(8);
  const size_t o_stat = c.take<uint8_t>(rs_status_words(count) * 4 + 32);
  void* base = nullptr;
  if ((e = cudaMallocFromPoolAsync(&base, c.off + 256, d->pool, st))) return to_status(e);
  RsWork rw;
  rw.hist = (uint32_t*)((char*)base + o_hist);
  rw.skip = (uint32_t*)((char*)base + o_skip);
  rw.status = (uint32_t*)((char*)base + o_stat);
  rw.ctr = rw.status + rs_status_words(count);
  e = radix_sort_u64_enqueue(keys, (uint64_t*)((char*)base + o_tmp), count, rw,
                             &d->slots[slot_of(d->id, st, true)].word, st,
                             d->num_sms);
  cudaFreeAsync(base, st);
  return to_status(e);
}

ls_status ls_sample_sort_u64(uint64_t* keys, size_t count, void* stream) {
  if (count > 0 && !keys) return LS_ERR_INVALID;
  if (count < 2) return LS_OK;
  if (count >= (1ull << 32)) return LS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Device* d;
  cudaError_t e = get_device(&d);
  if (e) return to_status(e);
  Carver c;
  const size_t o_tmp = c.take<uint64_t>(count);
  const size_t o_spl = c.take<uint64_t>(SS_P);
  const size_t o_words = c.take<uint32_t>(ss_work_words());
  void* base = nullptr;
  if ((e = cudaMallocFromPoolAsync(&base, c.off + 256, d->pool, st))) return to_status(e);
  SsWork sw;
  sw.spl = (uint64_t*)((char*)base + o_spl);
  sw.cnt = (uint32_t*)((char*)base + o_words);
  sw.beg = sw.cnt + (SS_NB + 1);
  sw.cur = sw.beg + (SS_NB + 1);
  e = sample_sort_u64_enqueue(keys, (uint64_t*)((char*)base + o_tmp), count, sw,
                              &d->slots[slot_of(d->id, st, true)].word, st,
                              d->num_sms);
  cudaFreeAsync(base, st);
  return to_status(e);
}

}  // extern "C"

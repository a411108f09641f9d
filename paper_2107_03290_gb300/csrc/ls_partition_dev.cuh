// Device helpers shared by the partitioning kernels (ls_partition.cu) and the
// in-place partition (ls_inplace.cu): the level-0 lookup tables in shared
// memory and a key's extended slot (Alg. 1's prediction), and the per-job
// bookkeeping and key-range maps of the refinement levels (Alg. 2's
// re-partition).
#pragma once
#include "ls_partition.cuh"

namespace ls {

struct L0Layout {
  uint32_t bar, buf, pbuf, thr, cell, cleaf, heads, htk, cnt, ecnt, soff, cursor, gbase, sinfo, sid,
      ws, hkey, hval, queue, tiles, total;
  uint32_t hs;           // K2: heavy values per bucket row (power of two > per-bucket maximum)
};

// Row width of the padded per-bucket heavy table of K2.
inline uint32_t heavy_stride(uint32_t f0, uint32_t next) {
  const uint32_t hpb = f0 ? (next - f0) / (2 * f0) : 0;
  if (!hpb) return 0;
  uint32_t hs = 1;
  while (hs <= hpb) hs <<= 1;
  return hs;
}

// The cell-index leaves stay in global memory (read through L1) when the
// shared copy would not fit.
constexpr size_t L0_SMEM_LIMIT = 227 * 1024;
constexpr uint32_t NOT_SHARED = 0xFFFFFFFFu;
constexpr int H_KPT = 6;             // keys per thread and step of K2's table-lookup loop
constexpr int HT_KPT = 8;            // keys per thread of K2's TMA tiles (calls without heavy values)

// K2: the lookup tables and the extended-slot counters.
inline int key_width(int dt) { return (dt == LS_F64 || dt == LS_U64) ? 8 : 4; }

constexpr int QCAP = 64;              // K2 per-warp queue of keys missing the heavy table
constexpr int H_TILE = H_THREADS * HT_KPT;  // K2 keys per TMA tile (calls without heavy values)

inline L0Layout l0_layout_hist(int W, uint32_t L, uint32_t f0, uint32_t next, uint32_t hmax,
                               bool cleaf_shared = true, bool hashed = true) {
  L0Layout y{};
  (void)hmax;
  y.hs = heavy_stride(f0, next);
  size_t o = 0;
  auto al = [&](size_t a) { o = (o + a - 1) / a * a; };
  al(16); y.thr = (uint32_t)o; o += (size_t)f0 * 8;
  y.cell = (uint32_t)o; o += (size_t)L0_CELLS * 4;
  y.cleaf = NOT_SHARED;
  if (cleaf_shared) { al(16); y.cleaf = (uint32_t)o; o += (size_t)L * sizeof(CellLeaf); }
  al(16); y.heads = (uint32_t)o; o += (size_t)(f0 + 1) * sizeof(BucketHead);
  y.htk = (uint32_t)o; o += (size_t)f0 * y.hs * 8;
  y.cnt = (uint32_t)o; o += (size_t)(next + 1) * 4;
  al(8); y.ws = (uint32_t)o; o += 33 * 8;
  y.bar = (uint32_t)o; o += 16;  // two mbarriers of the TMA tiles
  // The rest holds either the heavy table with the miss queues (the HASHED
  // instantiation) or the double-buffered TMA key tiles (the other one, in
  // calls without heavy values): the two kernels never use both.
  al(128);
  const size_t rest = o;
  y.hkey = y.hval = y.queue = NOT_SHARED;
  if (hashed && y.hs) {  // heavy table and per-warp miss queues
    al(16); y.hkey = (uint32_t)o; o += (size_t)HASH_SIZE * 8;
    y.hval = (uint32_t)o; o += (size_t)HASH_SIZE * 2;
    al(16); y.queue = (uint32_t)o; o += (size_t)(H_THREADS / 32) * QCAP * (W + 4);
  }
  const size_t tiles_end = rest + 2ull * H_TILE * W;
  y.tiles = tiles_end <= L0_SMEM_LIMIT ? (uint32_t)rest : NOT_SHARED;
  if (y.tiles != NOT_SHARED && tiles_end > o) o = tiles_end;
  y.total = (uint32_t)o;
  if (hashed && y.hs && o > L0_SMEM_LIMIT) return l0_layout_hist(W, L, f0, next, hmax, cleaf_shared, false);
  if (cleaf_shared && o > L0_SMEM_LIMIT) return l0_layout_hist(W, L, f0, next, hmax, false, false);
  return y;
}

// Shared-memory copies of the level-0 tables; returns the lookup over them.
__device__ __forceinline__ L0Map load_tables(const Level0Args& a, unsigned char* sm,
                                             const L0Layout& lay, uint32_t H) {
  uint64_t* thr = (uint64_t*)(sm + lay.thr);
  uint32_t* cell = (uint32_t*)(sm + lay.cell);
  CellLeaf* cleaf = lay.cleaf == NOT_SHARED ? a.M.cleaf : (CellLeaf*)(sm + lay.cleaf);
  BucketHead* heads = (BucketHead*)(sm + lay.heads);
  uint64_t* htk = (uint64_t*)(sm + lay.htk);
  for (uint32_t i = threadIdx.x; i < a.f0; i += blockDim.x) thr[i] = a.M.thr[i];
  for (uint32_t i = threadIdx.x; i < L0_CELLS; i += blockDim.x) cell[i] = a.M.cell[i];
  if (lay.cleaf != NOT_SHARED)
    for (uint32_t i = threadIdx.x; i < a.L; i += blockDim.x) cleaf[i] = a.M.cleaf[i];
  for (uint32_t i = threadIdx.x; i <= a.f0; i += blockDim.x) heads[i] = a.M.heads[i];
  // bucket b's heavy values at htk[j * f0 + b] (column-major, so lanes probing
  // different buckets hit different banks), padded with the largest key
  for (uint32_t i = threadIdx.x; i < a.f0 * lay.hs; i += blockDim.x) {
    const uint32_t j = i / a.f0, b = i % a.f0;
    const uint32_t hn = a.M.heads[b].hoff_nh;
    const uint32_t nh = hn & 15u, ho = hn >> 4;
    htk[i] = (j < nh && ho + j < H) ? a.M.heavy[ho + j].tk : ~0ull;
  }
  if (lay.hkey != NOT_SHARED) {
    uint64_t* hk = (uint64_t*)(sm + lay.hkey);
    uint16_t* hv = (uint16_t*)(sm + lay.hval);
    for (uint32_t i = threadIdx.x; i < HASH_SIZE; i += blockDim.x) { hk[i] = a.M.hkey[i]; hv[i] = a.M.hval[i]; }
  }
  const DevModel* h = a.M.hdr;
  return L0Map{thr, cell, cleaf, h->croot, h->pos_max, a.f0};
}

// 2 * #{heavy < t} + [t is heavy] over bucket b's padded row (hs entries at
// stride f0, ascending, padded with the largest key): fixed bisection steps,
// no divergence.
__device__ __forceinline__ uint32_t heavy_offset_row(const uint64_t* h, uint32_t f0, uint32_t hs,
                                                     uint32_t nh, uint64_t t) {
  uint32_t lo = 0;
  for (uint32_t s = hs >> 1; s; s >>= 1)
    if (h[(size_t)(lo + s - 1) * f0] < t) lo += s;
  if (h[(size_t)lo * f0] < t) lo += 1;  // lo: #{h < t} over the row
  lo = min(lo, nh);
  return 2 * lo + ((lo < nh && h[(size_t)lo * f0] == t) ? 1u : 0u);
}

template <int DT>
__device__ __forceinline__ uint32_t classify_key(typename KT<DT>::U u, const L0Map& q,
                                                 const BucketHead* heads, const uint64_t* htk,
                                                 uint32_t hs, float f0kf, uint32_t kf,
                                                 uint32_t* packed) {
  const float F = cell_F<DT>(u, q.croot, q.cleaf);
  const float v = F * (float)L0_CELLS;
  const uint32_t cl = v >= 0.0f ? (v < (float)L0_CELLS ? (uint32_t)v : L0_CELLS - 1) : 0u;
  const uint32_t r = q.cell[cl];
  const uint64_t t = KT<DT>::tk(u);
  const uint32_t b = min(thr_search(q.thr, r & 0xFFFFu, r >> 16, t), q.pos_max);
  const BucketHead h = heads[b];
  uint32_t e = h.ext_base;
  const uint32_t nh = h.hoff_nh & 15u;
  if (nh) e += heavy_offset_row(htk + b, q.f0, hs, nh, t);
  const float w = F * f0kf;
  int sub = (w >= 0.0f ? (int)w : 0) - (int)(b * kf);
  sub = sub < 0 ? 0 : (sub >= (int)kf ? (int)kf - 1 : sub);
  const uint32_t o = e - h.ext_base;
  *packed = (o & 1u) ? PK_EQ : (b | ((uint32_t)sub + (o >> 1)) << PK_B_BITS);
  return e;
}

// Bucket and packed id of a key in a call without heavy values (every bucket
// is one slot: e = b).
template <int DT>
__device__ __forceinline__ uint32_t classify_plain(typename KT<DT>::U u, const L0Map& q,
                                                   float f0kf, uint32_t kf, uint32_t* packed) {
  const float F = cell_F<DT>(u, q.croot, q.cleaf);
  const float v = F * (float)L0_CELLS;
  const uint32_t cl = v >= 0.0f ? (v < (float)L0_CELLS ? (uint32_t)v : L0_CELLS - 1) : 0u;
  const uint32_t r = q.cell[cl];
  const uint32_t b = min(thr_search(q.thr, r & 0xFFFFu, r >> 16, KT<DT>::tk(u)), q.pos_max);
  const float w = F * f0kf;
  int sub = (w >= 0.0f ? (int)w : 0) - (int)(b * kf);
  sub = sub < 0 ? 0 : (sub >= (int)kf ? (int)kf - 1 : sub);
  *packed = b | (uint32_t)sub << PK_B_BITS;
  return b;
}

struct L1Aux {
  uint64_t tile_base;
  uint64_t cbase;
  uint64_t pad0;
  uint32_t f1;
  uint32_t pad;
};

// Split of one refine job: by the model's F (the level-1 Partition of Alg. 2)
// or, for segments the model could not split, linearly over the segment's key
// range: on the FP32 image of the key for floating-point keys (value space,
// where a float range is close to linear in density), else, or when the image
// cannot resolve the range, on the total-order key (an integer map, exact at
// any width).  Both maps are non-decreasing in the key.
struct RangeSplit {
  unsigned long long tmin;
  unsigned long long mul;
  uint32_t sh;
  uint32_t fe;
  float xmin, xscale;    // value-space map when xscale > 0
};

template <int DT>
__device__ __forceinline__ RangeSplit range_split(unsigned long long tmin, unsigned long long tmax,
                                                  uint32_t f1, bool value_space) {
  RangeSplit s;
  const unsigned long long R = tmax - tmin;
  const int bl = R ? 64 - __clzll((long long)R) : 0;
  s.sh = bl > 32 ? (uint32_t)(bl - 32) : 0u;
  const unsigned long long Q = R >> s.sh;                      // < 2^32
  const unsigned long long fe = min((unsigned long long)f1, Q + 1);
  s.mul = (fe << 32) / (Q + 1);                                // <= 2^32
  s.tmin = tmin;
  s.fe = (uint32_t)fe;
  s.xmin = 0.0f;
  s.xscale = 0.0f;
  if (value_space && (DT == LS_F64 || DT == LS_F32)) {
    const float x0 = key_f32<DT>(KT<DT>::from_tk(tmin));
    const float x1 = key_f32<DT>(KT<DT>::from_tk(tmax));
    const float sc = (float)f1 / (x1 - x0);
    if (x1 > x0 && isfinite(x0) && isfinite(x1) && isfinite(sc) && sc > 0.0f) {
      s.xmin = x0;
      s.xscale = sc;
      s.fe = f1;
    }
  }
  return s;
}
template <int DT>
__device__ __forceinline__ uint32_t range_sub(typename KT<DT>::U u, const RangeSplit& s) {
  if (s.xscale > 0.0f) {
    const float v = (key_f32<DT>(u) - s.xmin) * s.xscale;
    return v > 0.0f ? min((uint32_t)v, s.fe - 1) : 0u;         // NaN keys cannot occur here
  }
  const unsigned long long d = (KT<DT>::tk(u) - s.tmin) >> s.sh;
  return (uint32_t)((d * s.mul) >> 32);                        // < min(f1, Q + 1)
}

__device__ __forceinline__ uint64_t aux_find_tile(const L1Aux* aux, uint64_t nj, uint64_t t) {
  uint64_t lo = 0, hi = nj;  // first index with tile_base > t, minus one
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (aux[mid].tile_base <= t) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}
__device__ __forceinline__ uint64_t aux_find_c(const L1Aux* aux, uint64_t nj, uint64_t c) {
  uint64_t lo = 0, hi = nj;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (aux[mid].cbase <= c) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

}  // namespace ls

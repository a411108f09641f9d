// Argsort and key-value sort on top of the learned sort.
//
// A key and its position are packed into one 64-bit composite key whose
// unsigned order is the key's total order, ties broken by position; the
// composites go through the whole learned sort (ls_sort on 64-bit unsigned
// keys: sample, RMI fit, both partition levels, in-bucket counting sorts) and
// the positions come back out as the permutation.  Ties keep their input
// order, so the permutation is the unique stable one.
//  * 4-byte keys: composite = tk(x) << 32 | i, one sort.
//  * 8-byte keys: two stable passes, least significant half first (the LSD
//    order of a radix sort, with the learned sort as the pass):
//      pass 1: c1 = lo32(tk(x_i)) << 32 | i, sorted;
//      pass 2: c2 = hi32(tk(x_{i_j})) << 32 | j, for the key i_j at position
//              j of pass 1, sorted;
//    the key at rank r is then i_{j_r}: ordered by (hi, lo, i), i.e. by the
//    total-order key with ties in input order.
// Keys and values are then gathered through the permutation.
#include <algorithm>

#include "ls_internal.cuh"

namespace ls {

constexpr int PR_THREADS = 256;

template <int DT>
__global__ void __launch_bounds__(PR_THREADS)
k_pack_key(const typename KT<DT>::U* __restrict__ keys, uint64_t n, int half,
           uint64_t* __restrict__ c) {
  pdl_begin();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = KT<DT>::tk(keys[i]);
    // 4-byte keys: the whole key (half = 0); 8-byte keys: the low (half = 1)
    // or high (half = 2) 32 bits of the total-order key
    const uint64_t part = half == 0 ? t : (half == 1 ? (t & 0xFFFFFFFFull) : (t >> 32));
    c[i] = part << 32 | i;
  }
}

// Pass 2 of 8-byte keys: c2[j] = hi32(tk(keys[i_j])) << 32 | j, i_j = lo32(c1[j]).
template <int DT>
__global__ void __launch_bounds__(PR_THREADS)
k_pack_hi(const typename KT<DT>::U* __restrict__ keys, const uint64_t* __restrict__ c1,
          uint64_t n, uint64_t* __restrict__ c2, uint32_t* err) {
  pdl_begin();
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)c1[j];
    if (i >= n) { set_error(err, ERR_BOUNDS); c2[j] = j; continue; }
    c2[j] = (KT<DT>::tk(keys[i]) >> 32) << 32 | j;
  }
}

// perm[r] = lo32(c[r]) (one pass), or lo32(c1[lo32(c2[r])]) (two passes).
__global__ void __launch_bounds__(PR_THREADS)
k_perm(const uint64_t* __restrict__ c2, const uint64_t* __restrict__ c1, uint64_t n,
       uint32_t* __restrict__ perm, uint32_t* err) {
  pdl_begin();
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
       r += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t j = (uint32_t)c2[r];
    if (c1) {
      if (j >= n) { set_error(err, ERR_BOUNDS); j = 0; }
      j = (uint32_t)c1[j];
    }
    perm[r] = j < n ? j : 0u;
    if (j >= n) set_error(err, ERR_BOUNDS);
  }
}

// out[r] = in[perm[r]] for elements of W bytes.
template <typename T>
__global__ void __launch_bounds__(PR_THREADS)
k_gather(const T* __restrict__ in, const uint32_t* __restrict__ perm, uint64_t n,
         T* __restrict__ out) {
  pdl_begin();
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
       r += (uint64_t)gridDim.x * blockDim.x)
    out[r] = in[perm[r]];
}

static unsigned pr_grid(uint64_t n, int num_sms) {
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + PR_THREADS - 1) / PR_THREADS,
                                                             16ull * num_sms));
}

template <int DT>
static cudaError_t pack_dt(const void* keys, uint64_t n, int half, uint64_t* c, cudaStream_t st,
                           int num_sms) {
  typedef typename KT<DT>::U U;
  return launch_k(k_pack_key<DT>, pr_grid(n, num_sms), PR_THREADS, 0, st, (const U*)keys, n, half,
                  c);
}

template <int DT>
static cudaError_t pack_hi_dt(const void* keys, const uint64_t* c1, uint64_t n, uint64_t* c2,
                              uint32_t* err, cudaStream_t st, int num_sms) {
  typedef typename KT<DT>::U U;
  return launch_k(k_pack_hi<DT>, pr_grid(n, num_sms), PR_THREADS, 0, st, (const U*)keys, c1, n,
                  c2, err);
}

static int key_bytes(int dt) { return (dt == LS_F64 || dt == LS_U64) ? 8 : 4; }

static ls_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return LS_OK;
  return e == cudaErrorMemoryAllocation ? LS_ERR_NOMEM : LS_ERR_CUDA;
}

// Stable argsort of `keys` into the device array `perm` (n < 2^32).
static ls_status argsort_impl(const void* keys, uint32_t* perm, uint64_t n, int dt,
                              cudaStream_t st) {
  if (n == 0) return LS_OK;
  if (n == 1) return status_of(cudaMemsetAsync(perm, 0, sizeof(uint32_t), st));
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (!e) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t* err = nullptr;
  if (!e) e = stream_status_ptr(st, &err);
  if (e) return status_of(e);
  const bool two = key_bytes(dt) == 8;
  uint64_t* c1 = nullptr;
  uint64_t* c2 = nullptr;
  if ((e = (cudaError_t)pool_alloc((void**)&c1, n * 8 * (two ? 2 : 1), st))) return status_of(e);
  if (two) c2 = c1 + n;
  ls_status rc = LS_OK;
  switch (dt) {
    case LS_F64: e = pack_dt<LS_F64>(keys, n, 1, c1, st, num_sms); break;
    case LS_U64: e = pack_dt<LS_U64>(keys, n, 1, c1, st, num_sms); break;
    case LS_F32: e = pack_dt<LS_F32>(keys, n, 0, c1, st, num_sms); break;
    default: e = pack_dt<LS_U32>(keys, n, 0, c1, st, num_sms); break;
  }
  add_launches(1);
  if (!e) rc = sort_call(c1, n, LS_U64, st, nullptr, nullptr, nullptr);
  if (!e && rc == LS_OK && two) {
    e = dt == LS_F64 ? pack_hi_dt<LS_F64>(keys, c1, n, c2, err, st, num_sms)
                     : pack_hi_dt<LS_U64>(keys, c1, n, c2, err, st, num_sms);
    add_launches(1);
    if (!e) rc = sort_call(c2, n, LS_U64, st, nullptr, nullptr, nullptr);
  }
  if (!e && rc == LS_OK) {
    e = launch_k(k_perm, pr_grid(n, num_sms), PR_THREADS, 0, st, (const uint64_t*)(two ? c2 : c1),
                 (const uint64_t*)(two ? c1 : nullptr), n, perm, err);
    add_launches(1);
  }
  pool_free(c1, st);
  if (e) return status_of(e);
  return rc;
}

static ls_status check_args(const void* keys, size_t n, int dt) {
  if (dt < LS_F64 || dt > LS_U32) return LS_ERR_INVALID;
  if (n > 0 && !keys) return LS_ERR_INVALID;
  if ((uintptr_t)keys % key_bytes(dt)) return LS_ERR_INVALID;
  if (n >= (1ull << 32)) return LS_ERR_INVALID;  // positions are 32-bit
  return LS_OK;
}

}  // namespace ls

using namespace ls;

extern "C" {

ls_status ls_argsort(const void* keys, uint32_t* perm, size_t n, ls_dtype dtype, void* stream) {
  const ls_status v = check_args(keys, n, dtype);
  if (v) return v;
  if (n > 0 && (!perm || ((uintptr_t)perm & 3))) return LS_ERR_INVALID;
  return argsort_impl(keys, perm, n, dtype, (cudaStream_t)stream);
}

ls_status ls_sort_pairs(void* keys, void* values, size_t n, ls_dtype dtype, uint32_t value_bytes,
                        void* stream) {
  const ls_status v = check_args(keys, n, dtype);
  if (v) return v;
  if (value_bytes != 4 && value_bytes != 8) return LS_ERR_INVALID;
  if (n > 0 && (!values || ((uintptr_t)values % value_bytes))) return LS_ERR_INVALID;
  if (n < 2) return LS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (!e) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e) return status_of(e);
  const size_t kb = (size_t)key_bytes(dtype);
  const size_t tb = std::max<size_t>(kb, value_bytes);
  void* base = nullptr;
  const size_t perm_bytes = (n * 4 + 255) / 256 * 256;
  if ((e = (cudaError_t)pool_alloc(&base, perm_bytes + n * tb, st))) return status_of(e);
  uint32_t* perm = (uint32_t*)base;
  void* tmp = (char*)base + perm_bytes;
  ls_status rc = argsort_impl(keys, perm, n, dtype, st);
  const unsigned g = pr_grid(n, num_sms);
  auto gather = [&](void* arr, size_t w) {
    cudaError_t r = w == 8 ? launch_k(k_gather<uint64_t>, g, PR_THREADS, 0, st,
                                      (const uint64_t*)arr, (const uint32_t*)perm, (uint64_t)n,
                                      (uint64_t*)tmp)
                           : launch_k(k_gather<uint32_t>, g, PR_THREADS, 0, st,
                                      (const uint32_t*)arr, (const uint32_t*)perm, (uint64_t)n,
                                      (uint32_t*)tmp);
    add_launches(1);
    if (!r) r = cudaMemcpyAsync(arr, tmp, n * w, cudaMemcpyDeviceToDevice, st);
    return r;
  };
  if (rc == LS_OK) e = gather(keys, kb);
  if (rc == LS_OK && !e) e = gather(values, value_bytes);
  pool_free(base, st);
  if (rc != LS_OK) return rc;
  return status_of(e);
}

}  // extern "C"

// 1-D TMA bulk copies (cp.async.bulk) into shared memory, completed on an
// mbarrier.  Used to stream key tiles of the level-0 passes into shared memory.
// Every wait is bounded: on timeout the status word gets ERR_TIMEOUT.
#pragma once
#include "ls_internal.cuh"

namespace ls {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Same, with an L2 evict-first policy: streamed-once data should not push
// out lines that other traffic (partially written output runs) still needs.
__device__ __forceinline__ void tma_load_1d_stream(void* dst, const void* src, uint32_t bytes,
                                                   uint64_t* bar) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* err) {
  unsigned long long spins = 0;
  const unsigned long long lim = spin_limit_of(err);
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > lim) { set_error(err, ERR_TIMEOUT); return false; }
  }
  return true;
}

// Double-buffered stream of tiles of a contiguous, 16-byte aligned range of
// keys (length a multiple of 16 bytes).  Thread 0 issues the copies.
template <typename U, int T>
struct TileStream {
  U* buf;              // 2 * T elements of shared memory
  uint64_t* bar;       // 2 mbarriers
  const U* src;
  uint64_t len;
  uint32_t nt;

  __device__ uint32_t count(uint32_t t) const {
    const uint64_t b = (uint64_t)t * T;
    return (uint32_t)(len - b < (uint64_t)T ? len - b : (uint64_t)T);
  }
  __device__ void issue(uint32_t t) {
    if (t >= nt) return;
    const uint32_t bytes = count(t) * (uint32_t)sizeof(U);
    uint64_t* br = bar + (t & 1);
    fence_proxy_async();
    mbar_arrive_expect_tx(br, bytes);
    tma_load_1d(buf + (size_t)(t & 1) * T, src + (size_t)t * T, bytes, br);
  }
  // thread 0 only; caller syncs afterwards
  __device__ void init() {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    fence_mbar_init();
  }
  __device__ U* wait(uint32_t t, uint32_t* err) {
    mbar_wait(bar + (t & 1), (t >> 1) & 1, err);
    return buf + (size_t)(t & 1) * T;
  }
};

}  // namespace ls

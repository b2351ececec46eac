// Bulk-copy (TMA) and mbarrier primitives for sm_100+ in inline PTX, and the
// bounded waits the streaming kernels use.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace msrep {

// Error codes a kernel ORs into the device error word it is given (the
// word is read and cleared by msrep_device_status).
enum : int { kErrWaitTimeout = 1 };

// An mbarrier wait that has not completed after this many polls, or after
// this many SM clock cycles (about a second), is treated as a failure; the
// copies it waits for take microseconds.
constexpr uint32_t kWaitPolls = 1u << 24;
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// make mbarrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same buffers
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`.  Returns false (and records the
// failure in *err) if the phase did not complete within kWaitPolls polls or
// `max_cycles` SM clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          long long max_cycles = kWaitCycles) {
  const long long t0 = clock64();
  for (uint32_t i = 0; i < kWaitPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > max_cycles) break;
  }
  atomicOr(err, kErrWaitTimeout);
  return false;
}

// Bulk copy of `bytes` (a multiple of 16) from global `src` (16-byte
// aligned) to shared `dst` (16-byte aligned); completion is signalled as
// transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Plan of one array segment copy: elements [e0, e1) of an array of `len`
// elements of `es` bytes.  The copied range starts at e0 rounded down to
// `align` elements (16-byte multiple) and ends at e1 rounded up to `align`,
// clipped to the 16-byte-aligned part of the array; elements of [e0, e1)
// past the clip (the last few of the array) are left to plain loads.
struct SegCopy {
  int64_t base;   // first element held in shared memory
  int64_t cend;   // end of the bulk-copied part
  uint32_t bytes; // bulk bytes (multiple of 16, may be 0)
};

__device__ __forceinline__ SegCopy seg_plan(int64_t e0, int64_t e1, int64_t len, int es,
                                            int align) {
  SegCopy c;
  c.base = e0 & ~int64_t(align - 1);
  int64_t want = (e1 + align - 1) & ~int64_t(align - 1);
  const int64_t per16 = 16 / es;
  int64_t cap = len & ~(per16 - 1);  // 16-byte aligned end of the array
  if (want > cap) want = cap;
  if (want < c.base) want = c.base;
  c.cend = want;
  c.bytes = static_cast<uint32_t>((want - c.base) * es);
  return c;
}

}  // namespace msrep

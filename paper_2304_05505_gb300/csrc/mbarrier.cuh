// Shared-memory mbarrier helpers of the TMA-fed kernels (inline PTX,
// sm_90 and later).  Every wait is bounded: about 2 s of clock64 (or the
// shorter limit stored beside the error word), after which the waiting thread
// sets its code in an error word the host reads, so that a lost transfer ends
// the kernel with an error status instead of a hang.  The drain after a
// failed wait always takes the full limit.
#pragma once

#include <stdint.h>

namespace {

constexpr long long WAIT_LIMIT = 4000000000LL;   // clock64 cycles (~2 s)

// The limit of the waits that report to the error word `err`: the 64-bit
// value at err + 2 (bytes 8-15 of the word's 64-byte block) when positive (a
// test sets a short one to make waits run out), else WAIT_LIMIT.
__device__ __forceinline__ long long wait_limit(const int* err) {
  const long long v = *reinterpret_cast<const volatile long long*>(err + 2);
  return v > 0 ? v : WAIT_LIMIT;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the phase of parity `parity` to complete.  Gives up after
// WAIT_LIMIT cycles (setting `code` in the error word) or as soon as another
// CTA has set the error word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  const long long t0 = clock64();
  long long limit = WAIT_LIMIT;
  for (uint32_t it = 0;; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) limit = wait_limit(err);   // read only when the first test fails
    if ((it & 255) == 255 && *(volatile int*)err != 0) return false;
    if (clock64() - t0 > limit) {
      atomicOr(err, code);
      return false;
    }
  }
}

// The same wait taken by a whole warp, with one answer for every lane.  Lane
// 0 polls with a growing sleep (up to 256 ns) so that waiting epilogue and
// converter warps leave the issue slots to the warps doing work.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, int* err, int code) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    const long long t0 = clock64();
    long long limit = WAIT_LIMIT;
    uint32_t ns = 8;
    for (uint32_t it = 0;; it++) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(bar), "r"(parity)
          : "memory");
      if (done) break;
      if (it == 0) limit = wait_limit(err);
      if ((it & 15) == 15 && *(volatile int*)err != 0) { ok = 0; break; }
      if (clock64() - t0 > limit) {
        atomicOr(err, code);
        ok = 0;
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
    }
  }
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Bounded wait that ignores the error word: used after a failed wait, so that
// a copy still in flight lands before the block exits.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_LIMIT) return false;
  }
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 3-D tiled TMA load of one box at (c0, c1, c2) into dst, completing on bar.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* map, uint32_t bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// 2-D tiled TMA load of one box at (c0, c1) into dst, completing on bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

}  // namespace

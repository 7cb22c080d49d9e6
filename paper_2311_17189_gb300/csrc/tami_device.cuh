// Device helpers shared by the libtami kernels (forward and adjoint translation units), and
// the host-side launch helpers they share.  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "tami_internal.h"
#include "tami_devmath.cuh"

namespace tami {
namespace dev {

constexpr long long kSpinLimit = 1ll << 24;  // bound on every device-side wait

// Final reduction of per-block partial sums, in a fixed order for a given number of rows: thread
// t of a kFinBlock-thread block adds rows t, t + kFinBlock, ... in turn, then the block adds the
// threads' sums pairwise in a fixed tree.  The result is in s[] of thread 0.
constexpr int kFinBlock = 256;

template <int NC>
__device__ __forceinline__ void fixed_tree_sum(double (&s)[NC], double (*sh)[kFinBlock]) {
  const int t = threadIdx.x;
  for (int k = 0; k < NC; ++k) sh[k][t] = s[k];
  __syncthreads();
  for (int w = kFinBlock / 2; w > 0; w >>= 1) {
    if (t < w)
      for (int k = 0; k < NC; ++k) sh[k][t] += sh[k][t + w];
    __syncthreads();
  }
  for (int k = 0; k < NC; ++k) s[k] = sh[k][0];
}

__host__ __device__ __forceinline__ int align16(int b) { return (b + 15) & ~15; }


// Bulk copy (TMA, cp.async.bulk) of `bytes` (multiple of 16, both addresses 16-byte aligned)
// into shared memory, completed on the mbarrier `bar` (initialised once with count 1 by
// mbar_init).  `parity` is the phase being completed: 0 for the first use, then alternating.
// The caller must __syncthreads() before a re-fill so that no thread still reads the old data.
// Every wait is bounded; on timeout the status word is set and the copy is waited for again.
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  if (threadIdx.x == 0) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

// Thread 0 only: arm `bar` for `bytes` bytes in total and start the copy of bytes0 bytes from src0
// to dst0 and, if bytes1 > 0, of bytes1 bytes from src1 to dst1 (all multiples of 16, addresses
// 16-byte aligned), both completing on `bar`.
__device__ __forceinline__ void bulk_issue(unsigned char* dst0, const unsigned char* src0, int bytes0,
                                           unsigned char* dst1, const unsigned char* src1, int bytes1,
                                           unsigned long long* bar) {
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  // order this block's earlier generic-proxy reads of the destinations before the async-proxy writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes0 + bytes1) : "memory");
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"((uint32_t)__cvta_generic_to_shared(dst0)), "l"(src0), "r"(bytes0), "r"(b) : "memory");
  if (bytes1 > 0)
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst1)), "l"(src1), "r"(bytes1), "r"(b) : "memory");
}

// Every thread: wait, bounded, for phase `parity` of `bar`; on timeout the status word is set and
// the copy is waited for again (bounded), so that it has landed before the block goes on or exits.
// `limit` bounds the first wait (kSpinLimit unless a test shortens it, tami_debug_set_wait_limit);
// the second is always bounded by kSpinLimit.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, int* status,
                                          long long limit = kSpinLimit) {
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  uint32_t done = 0;
  for (long long it = 0; it < limit && !done; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(b), "r"(parity) : "memory");
    if (!done && it > 64) __nanosleep(64);
  }
  if (!done) {
    if (status) atomicExch(status, TAMI_ETIMEOUT);
    for (long long j = 0; j < kSpinLimit && !done; ++j) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                   : "=r"(done) : "r"(b), "r"(parity) : "memory");
      __nanosleep(256);
    }
  }
  return done != 0;
}

__device__ __forceinline__ bool bulk_stage(unsigned char* dst, const unsigned char* src, int bytes,
                                           unsigned long long* bar, uint32_t parity, int* status,
                                           long long limit = kSpinLimit) {
  if (threadIdx.x == 0) bulk_issue(dst, src, bytes, nullptr, nullptr, 0, bar);
  return mbar_wait(bar, parity, status, limit);
}

// One-shot staging of a table: [src, src + bytes0) to dst and, if bytes1 > 0, [src1, src1 + bytes1)
// right after it; the decision to go on is the same in every thread of the block.
__device__ __forceinline__ bool stage_table(unsigned char* dst, const unsigned char* src, int bytes0,
                                            int* status, long long limit, const unsigned char* src1 = nullptr,
                                            int bytes1 = 0) {
  __shared__ __align__(8) unsigned long long bar;
  mbar_init(&bar);
  __syncthreads();
  if (threadIdx.x == 0) bulk_issue(dst, src, bytes0, dst + bytes0, src1, bytes1, &bar);
  const bool ok = mbar_wait(&bar, 0u, status, limit);
  return !__syncthreads_or(!ok);
}

// ------------------------------------------------------------------------------- host helpers
inline int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return TAMI_ECUDA;
}

struct DeviceProps { int sms = 0; size_t smem_optin = 0; };
inline DeviceProps device_props(int dev) {
  static std::mutex mu;
  static DeviceProps cache[64];
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64) return DeviceProps{};
  if (!cache[dev].sms) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
      cache[dev].sms = p.multiProcessorCount;
      cache[dev].smem_optin = p.sharedMemPerBlockOptin;
    }
  }
  return cache[dev];
}

}  // namespace dev
}  // namespace tami

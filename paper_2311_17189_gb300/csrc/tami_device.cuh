// Device helpers shared by the libtami kernels (forward and adjoint translation units), and
// the host-side launch helpers they share.  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "tami_internal.h"

namespace tami {
namespace dev {

constexpr int kBlock = 128;                 // threads per block = samples per tile
constexpr long long kSpinLimit = 1ll << 24;  // bound on every device-side wait

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

// [0,1) from 53 bits of two words, then k = 2 pi u - pi with one rounding
__device__ __forceinline__ double to_momentum(uint32_t hi, uint32_t lo) {
  unsigned long long m = ((unsigned long long)hi << 21) | (unsigned long long)(lo >> 11);
  double u = __dmul_rn(__ull2double_rn(m), 0x1.0p-53);
  const double pi = 0x1.921fb54442d18p+1;
  return fma(u, 2.0 * pi, -pi);
}

// cos and sin: Cody-Waite reduction by pi (three-part constant), k = n pi + r, |r| <= pi/2, then
// Taylor series in r (to r^24 for cos, r^25 for sin) and the sign (-1)^n (W. J. Cody and
// W. Waite, 1980).  Every operation is an explicit fma or a rounded mul intrinsic, so the result
// is the same on any IEEE machine that follows the same recipe.
__device__ __forceinline__ double cw_reduce(double k, double& odd_sign) {
  const double inv_pi = 0x1.45f306dc9c883p-2;
  const double P1 = 0x1.921fb54442d18p+1, P2 = 0x1.1a62633145c07p-53, P3 = -0x1.f1976b7ed8fbcp-109;
  const double n = rint(__dmul_rn(k, inv_pi));
  double r = fma(-n, P1, k);
  r = fma(-n, P2, r);
  r = fma(-n, P3, r);
  odd_sign = ((long long)n & 1) ? -1.0 : 1.0;
  return r;
}

__device__ __forceinline__ double cw_cos_poly(double z) {
  double pc = 0x1.f2cf01972f578p-80;
  pc = fma(pc, z, -0x1.0ce396db7f853p-70);
  pc = fma(pc, z, 0x1.e542ba4020225p-62);
  pc = fma(pc, z, -0x1.6827863b97d97p-53);
  pc = fma(pc, z, 0x1.ae7f3e733b81fp-45);
  pc = fma(pc, z, -0x1.93974a8c07c9dp-37);
  pc = fma(pc, z, 0x1.1eed8eff8d898p-29);
  pc = fma(pc, z, -0x1.27e4fb7789f5cp-22);
  pc = fma(pc, z, 0x1.a01a01a01a01ap-16);
  pc = fma(pc, z, -0x1.6c16c16c16c17p-10);
  pc = fma(pc, z, 0x1.5555555555555p-5);
  pc = fma(pc, z, -0x1.0000000000000p-1);
  return fma(z, pc, 1.0);
}

__device__ __forceinline__ double cw_cos(double k) {
  double sg;
  const double r = cw_reduce(k, sg);
  const double c = cw_cos_poly(__dmul_rn(r, r));
  return sg < 0.0 ? -c : c;
}

__device__ __forceinline__ void cw_sincos(double k, double& s_out, double& c_out) {
  double sg;
  const double r = cw_reduce(k, sg);
  const double z = __dmul_rn(r, r);
  const double cr = cw_cos_poly(z);
  double ps = 0x1.3f3ccdd165fa9p-84;
  ps = fma(ps, z, -0x1.761b41316381ap-75);
  ps = fma(ps, z, 0x1.71b8ef6dcf572p-66);
  ps = fma(ps, z, -0x1.2f49b46814157p-57);
  ps = fma(ps, z, 0x1.952c77030ad4ap-49);
  ps = fma(ps, z, -0x1.ae7f3e733b81fp-41);
  ps = fma(ps, z, 0x1.6124613a86d09p-33);
  ps = fma(ps, z, -0x1.ae64567f544e4p-26);
  ps = fma(ps, z, 0x1.71de3a556c734p-19);
  ps = fma(ps, z, -0x1.a01a01a01a01ap-13);
  ps = fma(ps, z, 0x1.1111111111111p-7);
  ps = fma(ps, z, -0x1.5555555555555p-3);
  const double sr = fma(__dmul_rn(r, z), ps, r);
  s_out = sg < 0.0 ? -sr : sr;
  c_out = sg < 0.0 ? -cr : cr;
}

// E = mu - eps(k),  eps(k) = -2t(cos kx + cos ky) - 4t' cos kx cos ky
__device__ __forceinline__ double line_energy(double kx, double ky, double t, double tp, double mu) {
  const double cx = cw_cos(kx), cy = cw_cos(ky);
  const double sum = __dadd_rn(cx, cy);
  const double prod = __dmul_rn(cx, cy);
  return fma(4.0 * tp, prod, fma(2.0 * t, sum, mu));
}

// 1/d: hardware estimate refined by one third-order Newton-Raphson step,
// r <- r (1 + e + e^2), e = 1 - d r  (error e^3).
__device__ __forceinline__ double rcp(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// d^k/dx^k g at (g, h = 1 - g): (-beta)^k sum_i (-1)^i A(k,i) g^(i+1) h^(k-i), A = Eulerian
__device__ __forceinline__ double fermi_poly(int k, double g, double h, double beta) {
  if (k == 0) return g;
  double gh = g * h;
  if (k == 1) return -beta * gh;
  double d = h - g;
  if (k == 2) return beta * beta * gh * d;
  if (k == 3) return -beta * beta * beta * gh * fma(d, d, -2.0 * gh);
  double b4 = beta * beta * beta * beta;
  double h2 = h * h, g2 = g * g;
  if (k == 4) return b4 * gh * (h2 * h - 11.0 * g * h2 + 11.0 * g2 * h - g2 * g);
  return -b4 * beta * gh * (h2 * h2 - 26.0 * g * h2 * h + 66.0 * g2 * h2 - 26.0 * g2 * g * h + g2 * g2);
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

__device__ __forceinline__ bool bulk_stage(unsigned char* dst, const unsigned char* src, int bytes,
                                           unsigned long long* bar, uint32_t parity, int* status) {
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  if (threadIdx.x == 0) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    // order this block's earlier generic-proxy reads of dst before the async-proxy writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(d), "l"(src), "r"(bytes), "r"(b) : "memory");
  }
  uint32_t done = 0;
  for (long long it = 0; it < kSpinLimit && !done; ++it) {
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

__device__ __forceinline__ bool stage_table(unsigned char* dst, const unsigned char* src, int bytes, int* status) {
  // one-shot staging: init the barrier, copy, wait on phase 0
  __shared__ __align__(8) unsigned long long bar;
  mbar_init(&bar);
  __syncthreads();
  const bool ok = bulk_stage(dst, src, bytes, &bar, 0u, status);
  // the decision to go on must be the same in every thread of the block
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

// Device helpers of the transport kernels: the Philox4x32-10 draw stream and
// order-preserving integer keys of binary64 values.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcgpu {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64-bit products mixed with the other counter words and the key,
// the key advancing by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Per-packet uniform stream.  Draw d uses Philox block d/2 with counter
// (d/2, packet, iteration, 0); words (x,y) for even d, (z,w) for odd d;
// u53 = (wa >> 5) 2^26 + (wb >> 6).
struct DrawStream {
  uint32_t k0, k1, packet, iteration;
  uint32_t d, spare_a, spare_b;

  __device__ __forceinline__ void init(uint32_t key0, uint32_t key1, uint32_t pid, uint32_t it) {
    k0 = key0; k1 = key1; packet = pid; iteration = it; d = 0; spare_a = 0; spare_b = 0;
  }
  __device__ __forceinline__ uint64_t next_u53() {
    uint32_t wa, wb;
    if ((d & 1u) == 0u) {
      const uint4 o = philox4x32_10(make_uint4(d >> 1, packet, iteration, 0u), k0, k1);
      wa = o.x; wb = o.y; spare_a = o.z; spare_b = o.w;
    } else {
      wa = spare_a; wb = spare_b;
    }
    ++d;
    return (static_cast<uint64_t>(wa >> 5) << 26) | static_cast<uint64_t>(wb >> 6);
  }
  // z in (0, 1]
  __device__ __forceinline__ double open0() { return __ull2double_rn(next_u53() + 1ull) * 0x1.0p-53; }
  // z in [0, 1)
  __device__ __forceinline__ double closed0() { return __ull2double_rn(next_u53()) * 0x1.0p-53; }
  __device__ __forceinline__ float closed0f() { return static_cast<float>(next_u53() >> 29) * 0x1.0p-24f; }
};

// Integer key with the same order as the binary64 value (all finite values,
// both zeros equal-ish: -0 sorts just below +0).  Comparisons of keys run on
// the integer pipe instead of the (slow) binary64 pipe.
__device__ __forceinline__ long long okey(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ long long okey_bits(long long b) {
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ int okey32(float v) {
  const int b = __float_as_int(v);
  return b ^ ((b >> 31) & 0x7fffffff);
}

constexpr long long kKeyNegInf = (long long)0x800fffffffffffffll;  // okey(-inf)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace mcgpu

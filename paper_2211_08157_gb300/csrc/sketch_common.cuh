// Device helpers shared by the sketch kernels (sketch.cu, sketch_seg.cu):
// the 2-bit base code, Wang's integer hash restricted to 2k bits in the
// arithmetic forms the kernels use, and division by the pattern weight.
#pragma once

#include "common.cuh"

namespace god {
namespace {

__device__ __forceinline__ uint32_t base_code(uint8_t b) {
  const uint32_t c = b & 0xDFu;  // upper-case letters; other bytes stay non-ACGT
  return c == 'A' ? 0u : c == 'C' ? 1u : c == 'G' ? 2u : c == 'T' ? 3u : 4u;
}

// (x * c + a) mod 2^64 from two 32-bit multiply-adds.
__device__ __forceinline__ uint64_t mad_c64(uint64_t x, uint32_t c, uint64_t a) {
  uint64_t lo;
  uint32_t hi;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(lo) : "r"((uint32_t)x), "r"(c), "l"(a));
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(hi) : "r"((uint32_t)(x >> 32)), "r"(c), "r"((uint32_t)(lo >> 32)));
  return ((uint64_t)hi << 32) | (uint32_t)lo;
}

// x ^ (x >> S) for 0 < S < 32, on the two 32-bit halves.
template <int S>
__device__ __forceinline__ uint64_t xorshr64(uint64_t x) {
  const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
  return ((uint64_t)(hi ^ (hi >> S)) << 32) | (lo ^ __funnelshift_r(lo, hi, S));
}

// Wang's 64-bit integer hash restricted to 2k bits. Its shift-add steps are
// multiplications by constants: ~x + (x << 21) = x * (2^21 - 1) - 1,
// x + (x << 3) + (x << 8) = 265 x, x + (x << 2) + (x << 4) = 21 x and
// x + (x << 31) = (2^31 + 1) x (mod 2^64), so each is one 64 x 32-bit
// multiply-add. HM (hash mode) 2: 2k > 32, the mask only touches the high
// half; HM 1: 32 < 2k <= 46, the high half has at most 14 bits, so every
// right shift (by 14, 24 or 28) leaves it zero and only the low half changes.
// HM 0: the same steps in 32-bit arithmetic give the identical value.
template <int S>
__device__ __forceinline__ uint64_t xorshr64_narrow(uint64_t x) {
  const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
  return ((uint64_t)hi << 32) | (lo ^ __funnelshift_r(lo, hi, S));
}

template <int HM>
__device__ __forceinline__ uint64_t wang_mix(uint64_t key, uint64_t mask) {
  if (HM == 2) {
    uint64_t x = key;
    x = mad_c64(x, 0x1FFFFFu, ~0ULL) & mask;
    x = xorshr64<24>(x);
    x = mad_c64(x, 265u, 0) & mask;
    x = xorshr64<14>(x);
    x = mad_c64(x, 21u, 0) & mask;
    x = xorshr64<28>(x);
    x = mad_c64(x, 0x80000001u, 0) & mask;
    return x;
  } else if (HM == 1) {
    uint64_t x = key;
    x = mad_c64(x, 0x1FFFFFu, ~0ULL) & mask;
    x = xorshr64_narrow<24>(x);
    x = mad_c64(x, 265u, 0) & mask;
    x = xorshr64_narrow<14>(x);
    x = mad_c64(x, 21u, 0) & mask;
    x = xorshr64_narrow<28>(x);
    x = mad_c64(x, 0x80000001u, 0) & mask;
    return x;
  } else {
    uint32_t x = (uint32_t)key;
    const uint32_t m = (uint32_t)mask;
    x = (x * 0x1FFFFFu + 0xFFFFFFFFu) & m;
    x = x ^ (x >> 24);
    x = (x * 265u) & m;
    x = x ^ (x >> 14);
    x = (x * 21u) & m;
    x = x ^ (x >> 28);
    x = (x * 0x80000001u) & m;
    return x;
  }
}

// q = j / x, r = j mod x with xinv = floor((2^32 - 1) / x): the estimate
// umulhi(j, xinv) is q or q - 1 for every j < 2^32, so one correction step.
__device__ __forceinline__ void divmod_x(uint32_t j, uint32_t x, uint32_t xinv, uint32_t& q, uint32_t& r) {
  q = __umulhi(j, xinv);
  r = j - q * x;
  if (r >= x) {
    r -= x;
    ++q;
  }
}

}  // namespace
}  // namespace god

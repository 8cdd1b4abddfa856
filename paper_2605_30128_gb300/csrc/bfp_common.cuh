// Block floating-point (BFP) block codec of Section III-C-3, shared by the stream kernels
// (bfp.cu) and the step kernel that reads the residual from a 12-bit stream (stencil.cu).
//
// Four FP32 values form one block of N_bits = 4 n_bits bits: the low 8 bits hold the
// shared biased exponent e = e_max + 127 (2^(e_max-1) <= max |x_i| < 2^e_max; e = 0
// marks an all-zero block), the rest four two's-complement coefficients of
// v = n_bits - 2 bits, q_i = round(x_i 2^(v-1-e_max)) clamped above at 2^(v-1) - 1;
// decoding gives q_i 2^(e_max-v+1).  The word layout of a block in a stream and the
// choices where the section is silent are stated in bfp.cu.
#pragma once

#include <cstdint>
#include <cstring>

#include "internal.h"

namespace rcf {
namespace {

__host__ __device__ __forceinline__ uint32_t bits_of(float x) {
  uint32_t u;
  memcpy(&u, &x, sizeof(u));
  return u;
}
__host__ __device__ __forceinline__ float float_of(uint32_t u) {
  float x;
  memcpy(&x, &u, sizeof(x));
  return x;
}
// 2^k for -126 <= k <= 127
__host__ __device__ __forceinline__ float pow2i(int k) { return float_of(uint32_t(k + 127) << 23); }
// x 2^k for |k| <= 252, as two power-of-two products (each factor a normal number)
__host__ __device__ __forceinline__ float scale_pow2(float x, int k) {
  const int h = k / 2;
  return (x * pow2i(h)) * pow2i(k - h);
}

template <int V>
__host__ __device__ __forceinline__ uint64_t bfp_encode4(const float x[4]) {
  constexpr int QMAX = (1 << (V - 1)) - 1;
  const float m = fmaxf(fmaxf(fabsf(x[0]), fabsf(x[1])), fmaxf(fabsf(x[2]), fabsf(x[3])));
  if (!(m > 0.0f)) return 0;                                // all zero
  const int f = int((bits_of(m) >> 23) & 0xFFu);            // biased FP32 exponent of the max
  int emax = f == 0 ? -126 : f - 126;                       // 2^(emax-1) <= m < 2^emax
  if (emax > 128) emax = 128;                               // non-finite input: unspecified code
  const float lo = emax == 128 ? -float(QMAX) : -float(QMAX + 1);
  uint64_t w = uint64_t(emax + 127);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float s = rintf(scale_pow2(x[i], V - 1 - emax));        // round half to even
    s = fminf(fmaxf(s, lo), float(QMAX));
    const int q = int(s);
    w |= uint64_t(uint32_t(q) & ((1u << V) - 1u)) << (8 + i * V);
  }
  return w;
}

template <int V>
__host__ __device__ __forceinline__ void bfp_decode4(uint64_t w, float y[4]) {
  const int e = int(w & 0xFFu);
  const int k = e - 127 - V + 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int fld = int((w >> (8 + i * V)) & ((1u << V) - 1u));
    const int q = fld >= (1 << (V - 1)) ? fld - (1 << V) : fld;   // restore the sign bits
    y[i] = e == 0 ? 0.0f : scale_pow2(float(q), k);
  }
}

// one block's bytes in the stream: 8 bytes as one word, 6 as three 2-byte words, 5 as bytes
template <int NB>
struct BlockIO;
template <>
struct BlockIO<16> {
  static __device__ __forceinline__ void store(unsigned char* s, int64_t b, uint64_t w) {
    reinterpret_cast<uint64_t*>(s)[b] = w;
  }
  static __device__ __forceinline__ uint64_t load(const unsigned char* s, int64_t b) {
    return __ldg(reinterpret_cast<const unsigned long long*>(s) + b);
  }
};
template <>
struct BlockIO<12> {
  static __device__ __forceinline__ void store(unsigned char* s, int64_t b, uint64_t w) {
    uint16_t* p = reinterpret_cast<uint16_t*>(s) + 3 * b;
    p[0] = uint16_t(w);
    p[1] = uint16_t(w >> 16);
    p[2] = uint16_t(w >> 32);
  }
  static __device__ __forceinline__ uint64_t load(const unsigned char* s, int64_t b) {
    const unsigned short* p = reinterpret_cast<const unsigned short*>(s) + 3 * b;
    return uint64_t(__ldg(p)) | (uint64_t(__ldg(p + 1)) << 16) | (uint64_t(__ldg(p + 2)) << 32);
  }
};
template <>
struct BlockIO<10> {
  static __device__ __forceinline__ void store(unsigned char* s, int64_t b, uint64_t w) {
    unsigned char* p = s + 5 * b;
#pragma unroll
    for (int j = 0; j < 5; ++j) p[j] = static_cast<unsigned char>(w >> (8 * j));
  }
  static __device__ __forceinline__ uint64_t load(const unsigned char* s, int64_t b) {
    const unsigned char* p = s + 5 * b;
    uint64_t w = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) w |= uint64_t(__ldg(p + j)) << (8 * j);
    return w;
  }
};

// Block decode without integer-to-float conversions (same values as bfp_decode4<V>): with
// k = e - 127 - V + 1 (the scale 2^(e_max - V + 1)), coefficient q is placed in the float
// 3 2^22 + q by adding q to the bits of 3 2^22 (exact for |q| < 2^22), and one FMA
// (3 2^22 + q) 2^k - 3 2^22 2^k gives q 2^k exactly: the product and the constant are exact
// and their sum is representable.  Valid for -126 <= k <= 104 (2^k normal, 3 2^(22+k) finite);
// zero blocks and the other exponents take the general path.
template <int V>
__device__ __forceinline__ void bfp_decode4_fast(uint64_t w, float y[4]) {
  const int e = int(w & 0xFFu);
  const int k = e - 127 - V + 1;
  if (e != 0 && k >= -126 && k <= 104) {
    const float s = __int_as_float((k + 127) << 23);
    const float c = -12582912.0f * s;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // the field with its sign bit flipped is q + 2^(V-1)
      const uint32_t fld = uint32_t(w >> (8 + V * i)) & ((1u << V) - 1u);
      const float m = __int_as_float(int(0x4B400000u - (1u << (V - 1)) + (fld ^ (1u << (V - 1)))));
      y[i] = __fmaf_rn(m, s, c);
    }
  } else {
    bfp_decode4<V>(w, y);
  }
}
__device__ __forceinline__ void bfp12_decode(uint64_t w, float y[4]) { bfp_decode4_fast<10>(w, y); }

// Block b of a 12-bit stream (6 bytes at byte 6 b, as three little-endian 16-bit words)
// read with one aligned 4-byte and one 2-byte load and no byte outside the block: for even
// b the word at 6 b and the half-word at 6 b + 4, for odd b the half-word at 6 b and the
// word at 6 b + 2.  The stream must start on a 4-byte boundary.  The loads (bfp12_fetch)
// and their assembly into the block (bfp12_join) are separate so that a caller can issue
// the loads well before it needs the values.
__device__ __forceinline__ void bfp12_fetch(const unsigned char* __restrict__ s, int64_t b, uint32_t& w,
                                            uint32_t& h) {
  const int odd = int(b & 1);
  const unsigned char* blk = s + 6 * b;
  w = __ldg(reinterpret_cast<const unsigned int*>(blk + 2 * odd));
  h = __ldg(reinterpret_cast<const unsigned short*>(blk + 4 - 4 * odd));
}
__device__ __forceinline__ uint64_t bfp12_join(int odd, uint32_t w, uint32_t h) {
  return odd ? (uint64_t(h) | (uint64_t(w) << 16)) : (uint64_t(w) | (uint64_t(h) << 32));
}

}  // namespace
}  // namespace rcf

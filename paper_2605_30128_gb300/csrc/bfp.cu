// Block floating-point (BFP) codec of Section III-C-3.
//
// Four FP32 values form one block of N_bits = 4 n_bits bits: the low 8 bits hold the
// shared biased exponent e = e_max + 127 (2^(e_max-1) <= max |x_i| < 2^e_max; e = 0
// marks an all-zero block), the rest four two's-complement coefficients of
// v = n_bits - 2 bits, q_i = round(x_i 2^(v-1-e_max)) clamped above at 2^(v-1) - 1;
// decoding gives q_i 2^(e_max-v+1).  n_bits = 16, 12, 10: 8, 6 or 5 bytes per block,
// written by one thread as one 8-byte, three 2-byte or five 1-byte stores, so no
// storage word is shared by two blocks (the section's layout).
//
// Choices where the section is silent: round to nearest even; coefficient i in bits
// [8 + i v, 8 + (i+1) v), the word little-endian; a block whose largest magnitude is
// subnormal takes e_max = -126; at e_max = 128 the lower clamp is -(2^(v-1) - 1), so
// that no decoded value overflows FP32; a ragged tail block is completed with zeros.
//
// All scaling is by powers of two, split into two factors that are normal FP32
// numbers, so every product is exact (or, when it underflows, far below 1/2, where
// the rounded coefficient is 0 either way): the only rounding is the rint of the
// quantisation, and decoding is exact.  The block helpers (bfp_common.cuh) are
// __host__ __device__ so that their arithmetic can be checked on a CPU as well.
#include <cstring>

#include "bfp_common.cuh"

namespace rcf {
namespace {

constexpr int kBfpThreads = 256;
constexpr int kBfpUnroll = 4;   // blocks per thread per pass (independent loads in flight)

// Thread t of the grid handles blocks t, t + S, t + 2S, ... (S = threads in the grid),
// kBfpUnroll of them per pass.  vec4: x is 16-byte aligned (whole blocks load as float4).
template <int NB>
__global__ void __launch_bounds__(kBfpThreads) bfp_encode_kernel(const float* __restrict__ x, int64_t n,
                                                                   unsigned char* __restrict__ s, int vec4) {
  constexpr int V = NB - 2;
  const int64_t nblk = (n + 3) / 4;
  const int64_t S = int64_t(gridDim.x) * blockDim.x;
  for (int64_t b0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b0 < nblk; b0 += S * kBfpUnroll) {
    float v[kBfpUnroll][4];
#pragma unroll
    for (int u = 0; u < kBfpUnroll; ++u) {
      const int64_t b = b0 + u * S;
      if (b >= nblk) break;
      if (vec4 && 4 * b + 4 <= n) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(x) + b);
        v[u][0] = t.x; v[u][1] = t.y; v[u][2] = t.z; v[u][3] = t.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[u][j] = 4 * b + j < n ? x[4 * b + j] : 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < kBfpUnroll; ++u) {
      const int64_t b = b0 + u * S;
      if (b >= nblk) break;
      BlockIO<NB>::store(s, b, bfp_encode4<V>(v[u]));
    }
  }
}

template <int NB>
__global__ void __launch_bounds__(kBfpThreads) bfp_decode_kernel(const unsigned char* __restrict__ s, int64_t n,
                                                                   float* __restrict__ y, int vec4) {
  constexpr int V = NB - 2;
  const int64_t nblk = (n + 3) / 4;
  const int64_t S = int64_t(gridDim.x) * blockDim.x;
  for (int64_t b0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b0 < nblk; b0 += S * kBfpUnroll) {
    uint64_t w[kBfpUnroll];
#pragma unroll
    for (int u = 0; u < kBfpUnroll; ++u) {
      const int64_t b = b0 + u * S;
      if (b >= nblk) break;
      w[u] = BlockIO<NB>::load(s, b);
    }
#pragma unroll
    for (int u = 0; u < kBfpUnroll; ++u) {
      const int64_t b = b0 + u * S;
      if (b >= nblk) break;
      float r[4];
      bfp_decode4<V>(w[u], r);
      if (vec4 && 4 * b + 4 <= n) {
        reinterpret_cast<float4*>(y)[b] = make_float4(r[0], r[1], r[2], r[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * b + j < n) y[4 * b + j] = r[j];
      }
    }
  }
}

// Decode with 16-byte loads (stream and values 16-byte aligned): each warp takes a chunk of
// 32 consecutive blocks, whose 192 (12 bits) or 160 (10 bits) stream bytes its first 12 or
// 10 lanes load as 16-byte words into shared memory; then lane l assembles block l from
// there, decodes it and stores its 4 values as one 16-byte word (coalesced across the
// warp).  Chunks c < nchunks hold only whole 4-value groups; the caller decodes the rest
// with bfp_decode_kernel.
template <int NB>
__global__ void __launch_bounds__(kBfpThreads) bfp_decode_vec_kernel(const uint4* __restrict__ s, int64_t nchunks,
                                                                       float4* __restrict__ y) {
  constexpr int V = NB - 2, BYTES = NB / 2, WORDS = 32 * BYTES / 16;   // 16-byte words per chunk: 12 or 10
  constexpr int CH = 2;                                                // chunks in flight per warp
  static_assert(32 * BYTES % 16 == 0, "a chunk is whole 16-byte words");
  __shared__ uint4 buf[kBfpThreads / 32][CH][WORDS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x / 32);
  for (int64_t c0 = int64_t(blockIdx.x) * (blockDim.x / 32) + wid; c0 < nchunks; c0 += CH * nw) {
#pragma unroll
    for (int h = 0; h < CH; ++h) {
      const int64_t c = c0 + h * nw;
      if (lane < WORDS && c < nchunks) buf[wid][h][lane] = __ldg(s + c * WORDS + lane);
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < CH; ++h) {
      const int64_t c = c0 + h * nw;
      if (c >= nchunks) break;
      const unsigned char* b = reinterpret_cast<const unsigned char*>(buf[wid][h]) + lane * BYTES;
      uint64_t w = 0;
#pragma unroll
      for (int j = 0; j < BYTES; ++j) w |= uint64_t(b[j]) << (8 * j);
      float r[4];
      bfp_decode4_fast<V>(w, r);
      y[c * 32 + lane] = make_float4(r[0], r[1], r[2], r[3]);
    }
    __syncwarp();   // the chunks' words are read before the next pass overwrites them
  }
}

// 12-bit storage of a residual block (the FP32 recurrence with R kept as a BFP stream):
// every block of x is encoded into s and x is overwritten by the decoded values, so
// that the uses of R that read x and those that read s see the same numbers.  x is
// 16-byte aligned and n a multiple of 4 (whole node 4-tuples).
__global__ void __launch_bounds__(kBfpThreads) bfp12_round_trip_kernel(float* __restrict__ x, int64_t nblk,
                                                                         unsigned char* __restrict__ s) {
  const int64_t S = int64_t(gridDim.x) * blockDim.x;
  for (int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b < nblk; b += S) {
    const float4 t = reinterpret_cast<const float4*>(x)[b];
    float v[4] = {t.x, t.y, t.z, t.w};
    const uint64_t w = bfp_encode4<10>(v);
    BlockIO<12>::store(s, b, w);
    bfp_decode4<10>(w, v);
    reinterpret_cast<float4*>(x)[b] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

int bfp_bytes_per_block(int nbits) {
  switch (nbits) {
    case 16: return 8;
    case 12: return 6;
    case 10: return 5;
    default: return 0;
  }
}

// grid: one pass of kBfpUnroll blocks per thread, at most 16 resident-size CTAs per SM of 152
unsigned bfp_grid(int64_t nblk) {
  const int64_t per_cta = int64_t(kBfpThreads) * kBfpUnroll;
  return unsigned(std::min<int64_t>((nblk + per_cta - 1) / per_cta, 152 * 16));
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* a0 = static_cast<const char*>(a);
  const char* b0 = static_cast<const char*>(b);
  return a0 < b0 + nb && b0 < a0 + na;
}

int check_bfp_args(rcf_ctx* ctx, const void* vals, int64_t n, int nbits, const void* stream, const char* vname) {
  const int nb = bfp_bytes_per_block(nbits);
  if (nb == 0) return fail(ctx, RCF_EINVAL, "n_bits must be 16, 12 or 10 (got %d)", nbits);
  if (n < 0) return fail(ctx, RCF_EINVAL, "n < 0");
  if (n == 0) return RCF_OK;
  if (!vals || !stream) return fail(ctx, RCF_EINVAL, "NULL %s or stream", vname);
  if (reinterpret_cast<uintptr_t>(vals) % 4) return fail(ctx, RCF_EINVAL, "%s must be 4-byte aligned", vname);
  const size_t salign = nbits == 16 ? 8 : nbits == 12 ? 2 : 1;
  if (reinterpret_cast<uintptr_t>(stream) % salign)
    return fail(ctx, RCF_EINVAL, "stream must be %zu-byte aligned at %d bits", salign, nbits);
  const size_t sbytes = size_t((n + 3) / 4) * nb;
  if (ranges_overlap(vals, sizeof(float) * size_t(n), stream, sbytes))
    return fail(ctx, RCF_EINVAL, "%s overlaps the stream", vname);
  return RCF_OK;
}

}  // namespace
}  // namespace rcf

namespace rcf {
int launch_bfp12_round_trip(rcf_ctx* ctx, float* x, int64_t n, unsigned char* s) {
  if (n <= 0) return RCF_OK;
  const int64_t nblk = n / 4;
  bfp12_round_trip_kernel<<<bfp_grid(nblk), kBfpThreads, 0, ctx->stream>>>(x, nblk, s);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}
}  // namespace rcf

using namespace rcf;

extern "C" int64_t rcf_bfp_stream_bytes(int64_t n, int nbits) {
  const int nb = bfp_bytes_per_block(nbits);
  if (nb == 0 || n < 0) return -1;
  return ((n + 3) / 4) * nb;
}

extern "C" int rcf_bfp_encode(rcf_ctx* ctx, const float* x, int64_t n, int nbits, void* stream) {
  if (!ctx) return RCF_EINVAL;
  RCF_TRY(check_bfp_args(ctx, x, n, nbits, stream, "x"));
  if (n == 0) return RCF_OK;
  const int64_t nblk = (n + 3) / 4;
  const int vec4 = (reinterpret_cast<uintptr_t>(x) % 16) == 0;
  unsigned char* s = static_cast<unsigned char*>(stream);
  const unsigned grid = bfp_grid(nblk);
  switch (nbits) {
    case 16: bfp_encode_kernel<16><<<grid, kBfpThreads, 0, ctx->stream>>>(x, n, s, vec4); break;
    case 12: bfp_encode_kernel<12><<<grid, kBfpThreads, 0, ctx->stream>>>(x, n, s, vec4); break;
    default: bfp_encode_kernel<10><<<grid, kBfpThreads, 0, ctx->stream>>>(x, n, s, vec4); break;
  }
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

extern "C" int rcf_bfp_decode(rcf_ctx* ctx, const void* stream, int64_t n, int nbits, float* y) {
  if (!ctx) return RCF_EINVAL;
  RCF_TRY(check_bfp_args(ctx, y, n, nbits, stream, "y"));
  if (n == 0) return RCF_OK;
  const int vec4 = (reinterpret_cast<uintptr_t>(y) % 16) == 0;
  const unsigned char* s = static_cast<const unsigned char*>(stream);
  if (nbits != 16 && vec4 && (reinterpret_cast<uintptr_t>(stream) % 16) == 0) {
    // whole chunks of 32 blocks through 16-byte words, the rest below
    const int bpg = 32;
    const int64_t ngroups = (n / 4) / bpg;
    if (ngroups > 0) {
      const unsigned g = unsigned(std::min<int64_t>((ngroups + kBfpThreads / 16 - 1) / (kBfpThreads / 16), 152 * 16));
      if (nbits == 12)
        bfp_decode_vec_kernel<12><<<g, kBfpThreads, 0, ctx->stream>>>(reinterpret_cast<const uint4*>(s), ngroups,
                                                                          reinterpret_cast<float4*>(y));
      else
        bfp_decode_vec_kernel<10><<<g, kBfpThreads, 0, ctx->stream>>>(reinterpret_cast<const uint4*>(s), ngroups,
                                                                          reinterpret_cast<float4*>(y));
      RCF_CHECK_LAUNCH(ctx);
    }
    const int64_t done = ngroups * bpg * 4;   // values decoded
    if (done == n) return RCF_OK;
    s += done / 4 * bfp_bytes_per_block(nbits);
    y += done;
    n -= done;
  }
  const unsigned grid2 = bfp_grid((n + 3) / 4);
  switch (nbits) {
    case 16: bfp_decode_kernel<16><<<grid2, kBfpThreads, 0, ctx->stream>>>(s, n, y, vec4); break;
    case 12: bfp_decode_kernel<12><<<grid2, kBfpThreads, 0, ctx->stream>>>(s, n, y, vec4); break;
    default: bfp_decode_kernel<10><<<grid2, kBfpThreads, 0, ctx->stream>>>(s, n, y, vec4); break;
  }
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

// C = A^H diag(w) B for tall complex FP64 blocks (K rows, K >> m, n), in double-float
// arithmetic on the FP32 pipes: the Gram matrix of Cholesky-QR (w = lumped mass) and the
// projected matrix Y^H (H Y) of Rayleigh-Ritz (w = 1), Algorithm 1's RR step.
//
// GB300 runs FP64 GEMMs at about 1 TFLOP/s (cuBLAS ZGEMM/ZHERK), so at 10^6 rows and 10^3
// columns these products take seconds to tens of seconds.  Here every FP64 input is split
// into a float pair with integer operations, every product is formed exactly with one FMA
// (c_h x_h = p + e) plus the cross terms, and the sums run with Knuth's TwoSum (the
// compensated dot product of Ogita, Rump and Oishi), giving about 2^-46 relative to the sum
// of the magnitudes of the terms.
//
// Summation is blocked: each stage of 16 rows accumulates into a fresh pair, which is then
// added to the running pair by a normalised double-float addition.  (Accumulating a long
// sum in one pair would let the low word collect ~n TwoSum errors of the size eps |sum|
// and lose accuracy once n eps is no longer small; blocked, the error grows with the
// number of stages and stays near eps^2 |sum| per stage.)
//
// Tiling: a block computes a 64 x 64 tile of C over one chunk of the K rows (split-K);
// 256 threads, each 4 x 4 outputs strided by 16 (conflict-free shared-memory reads); the
// K rows stream through shared memory 16 at a time as (hi, lo) pairs.  The partial tiles
// of the chunks are summed by a second kernel in double-float and written as FP64.
// With lower = 1 only tiles on or below the diagonal are formed (Hermitian C = A^H A).
#include <algorithm>

#include "internal.h"

namespace rcf {
namespace {

constexpr int TM = 64, TN = 64, KT = 16, NTHR = 256;

__device__ __forceinline__ float2 add2(float2 x, float2 y) { return __fadd2_rn(x, y); }
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(make_float2(-1.f, -1.f), y, x); }

// S (hi, lo pairs of two components) += c x, c = (ch, cl) a scalar pair
__device__ __forceinline__ void tap(float2& Sh, float2& Sl, float ch, float cl, float2 xh, float2 xl) {
  const float2 c2 = make_float2(ch, ch), nc2 = make_float2(-ch, -ch), l2 = make_float2(cl, cl);
  const float2 np = __fmul2_rn(nc2, xh);          // -p
  float2 t = __ffma2_rn(c2, xh, np);              // c_h x_h - p, exact
  t = __ffma2_rn(c2, xl, t);
  t = __ffma2_rn(l2, xh, t);
  const float2 s = sub2(Sh, np);
  const float2 bp = sub2(s, Sh);
  const float2 da = sub2(Sh, sub2(s, bp));
  const float2 db = add2(np, bp);
  Sh = s;
  Sl = add2(Sl, add2(t, sub2(da, db)));
}

// (Sh, Sl) += (bh, bl), both unevaluated pairs; the result normalised (|Sl| <= ulp(Sh) / 2)
__device__ __forceinline__ void dfacc(float2& Sh, float2& Sl, float2 bh, float2 bl) {
  const float2 s = add2(Sh, bh);
  const float2 bp = sub2(s, Sh);
  const float2 err = add2(sub2(Sh, sub2(s, bp)), sub2(bh, bp));
  const float2 l = add2(add2(Sl, bl), err);
  Sh = add2(s, l);
  Sl = sub2(l, sub2(Sh, s));
}

// FP64 -> (hi, lo) with integer operations (as in the double-float residual): hi the top
// 24 significand bits, lo the next 29 rounded to 24; (0, 0) below 2^-126.
__device__ __forceinline__ float2 split(double x) {
  const unsigned hw = static_cast<unsigned>(__double2hiint(x));
  const unsigned lw = static_cast<unsigned>(__double2loint(x));
  const unsigned sgn = hw & 0x80000000u;
  const int E = int((hw >> 20) & 0x7FFu);
  const int e32 = E - 896, es = E - 948;
  float h = __uint_as_float(sgn | (static_cast<unsigned>(e32) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  float l = __fmul_rn(__uint2float_rn(lw & 0x1FFFFFFFu), __uint_as_float(static_cast<unsigned>(es) << 23));
  l = __uint_as_float(__float_as_uint(l) | sgn);
  if (es <= 0) l = __uint_as_float(sgn);
  if (e32 <= 0) h = __uint_as_float(sgn);
  if (e32 >= 255) { h = __uint_as_float(sgn | 0x7F800000u); l = 0.f; }
  return make_float2(h, l);
}

// scalar double-float product, normalised (weights times an input)
__device__ __forceinline__ float2 dfmul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}

struct TNArgs {
  const double* A; int64_t lda;   // complex, K x m, column-major (ld in complex elements)
  const double* B; int64_t ldb;   // complex, K x n
  const double* w;                // weight of complex row k: w[k >> 1] (the node's lumped mass); may be null
  int64_t K; int m, n;
  int lower;                      // form only tiles with row tile >= column tile
  int64_t kchunk;                 // rows per chunk
  float* part;                    // [nchunks][ntiles][TM][TN] x (re_h, im_h, re_l, im_l)
  int tiles_m, tiles_n;
};

// tile index t -> (tile row, tile column): all tiles, or the lower triangle row by row
__device__ __forceinline__ void tile_of(int t, int tiles_n, int lower, int& ti, int& tj) {
  if (!lower) {
    ti = t / tiles_n;
    tj = t - ti * tiles_n;
    return;
  }
  // lower triangle: row r has r + 1 tiles; t = r (r + 1) / 2 + c
  int r = int((sqrtf(8.f * float(t) + 1.f) - 1.f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  ti = r;
  tj = t - r * (r + 1) / 2;
}

// grid (ntiles, nchunks), NTHR threads
__global__ void __launch_bounds__(NTHR, 1) gemm_tn_df_kernel(const TNArgs a) {
  __shared__ float2 Ah[KT][TM], Al[KT][TM], Bh[KT][TN], Bl[KT][TN];   // (re, im) pairs: 32 KB
  int ti, tj;
  tile_of(blockIdx.x, a.tiles_n, a.lower, ti, tj);
  const int i0 = ti * TM, j0 = tj * TN;
  const int64_t k0 = int64_t(blockIdx.y) * a.kchunk;
  const int64_t k1 = k0 + a.kchunk < a.K ? k0 + a.kchunk : a.K;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // outputs (i0 + ty + 16 u, j0 + tx + 16 v)

  float2 Sh[4][4], Sl[4][4];   // (re, im) hi and lo
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Sh[u][v] = Sl[u][v] = make_float2(0.f, 0.f);

  for (int64_t kb = k0; kb < k1; kb += KT) {
    // stage KT rows of the 64 A columns and 64 B columns: thread -> (row kk, column c)
    __syncthreads();
    for (int e = threadIdx.x; e < KT * TM; e += NTHR) {
      const int kk = e % KT, c = e / KT;
      const int64_t k = kb + kk;
      float2 ar = make_float2(0.f, 0.f), ai = ar, br = ar, bi = ar;
      if (k < k1) {
        if (i0 + c < a.m) {
          const double2 x = reinterpret_cast<const double2*>(a.A + 2 * (int64_t(i0 + c) * a.lda))[k];
          ar = split(x.x);
          ai = split(x.y);
          if (a.w) {
            const float2 wk = split(a.w[k >> 1]);
            ar = dfmul(ar, wk);
            ai = dfmul(ai, wk);
          }
        }
        if (j0 + c < a.n) {
          const double2 y = reinterpret_cast<const double2*>(a.B + 2 * (int64_t(j0 + c) * a.ldb))[k];
          br = split(y.x);
          bi = split(y.y);
        }
      }
      Ah[kk][c] = make_float2(ar.x, ai.x);
      Al[kk][c] = make_float2(ar.y, ai.y);
      Bh[kk][c] = make_float2(br.x, bi.x);
      Bl[kk][c] = make_float2(br.y, bi.y);
    }
    __syncthreads();
    float2 Bh_[4][4], Bl_[4][4];   // this stage's sums
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) Bh_[u][v] = Bl_[u][v] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int kk = 0; kk < KT; ++kk) {
      float2 ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { ah[u] = Ah[kk][ty + 16 * u]; al[u] = Al[kk][ty + 16 * u]; }
#pragma unroll
      for (int v = 0; v < 4; ++v) { bh[v] = Bh[kk][tx + 16 * v]; bl[v] = Bl[kk][tx + 16 * v]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          // conj(a) b = a_r (b_r, b_i) + a_i (b_i, -b_r)
          tap(Bh_[u][v], Bl_[u][v], ah[u].x, al[u].x, bh[v], bl[v]);
          tap(Bh_[u][v], Bl_[u][v], ah[u].y, al[u].y, make_float2(bh[v].y, -bh[v].x),
              make_float2(bl[v].y, -bl[v].x));
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) dfacc(Sh[u][v], Sl[u][v], Bh_[u][v], Bl_[u][v]);
  }
  // partial tile
  float4* out = reinterpret_cast<float4*>(a.part) +
                (int64_t(blockIdx.y) * gridDim.x + blockIdx.x) * (TM * TN);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v)
      out[(ty + 16 * u) * TN + tx + 16 * v] = make_float4(Sh[u][v].x, Sh[u][v].y, Sl[u][v].x, Sl[u][v].y);
}

// C[i + j ldc] = sum over chunks of the partial tiles (double-float), written as FP64
__global__ void gemm_tn_reduce_kernel(const float* __restrict__ part, int nchunks, int ntiles, int tiles_n,
                                      int lower, int m, int n, double* __restrict__ C, int64_t ldc) {
  const int t = blockIdx.x;
  int ti, tj;
  tile_of(t, tiles_n, lower, ti, tj);
  for (int e = threadIdx.x; e < TM * TN; e += blockDim.x) {
    const int il = e / TN, jl = e - il * TN;
    const int i = ti * TM + il, j = tj * TN + jl;
    if (i >= m || j >= n) continue;
    float2 sh = make_float2(0.f, 0.f), sl = sh;
    for (int c = 0; c < nchunks; ++c) {
      const float4 p = reinterpret_cast<const float4*>(part)[(int64_t(c) * ntiles + t) * (TM * TN) + e];
      // (sh, sl) += (p.xy, p.zw): TwoSum of the hi parts, lo parts added
      dfacc(sh, sl, make_float2(p.x, p.y), make_float2(p.z, p.w));
    }
    reinterpret_cast<double2*>(C)[int64_t(j) * ldc + i] =
        make_double2(double(sh.x) + double(sl.x), double(sh.y) + double(sl.y));
  }
}

}  // namespace

int launch_gemm_tn_df(rcf_ctx* ctx, const double* A, int64_t lda, const double* B, int64_t ldb,
                      const double* w, int64_t K, int m, int n, int lower, double* C, int64_t ldc) {
  if (m <= 0 || n <= 0) return RCF_OK;
  TNArgs a{};
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.w = w;
  a.K = K; a.m = m; a.n = n; a.lower = lower;
  a.tiles_m = (m + TM - 1) / TM;
  a.tiles_n = (n + TN - 1) / TN;
  if (lower && a.tiles_m != a.tiles_n) return fail(ctx, RCF_EINVAL, "lower needs a square C");
  const int ntiles = lower ? a.tiles_m * (a.tiles_m + 1) / 2 : a.tiles_m * a.tiles_n;
  // enough chunks for about eight blocks per SM-slot on 152 SMs, each at least 1024 rows
  int64_t nchunks = std::max<int64_t>(1, (8 * 152 + ntiles - 1) / ntiles);
  nchunks = std::min<int64_t>(nchunks, std::max<int64_t>(1, K / 1024));
  int64_t kchunk = (K + nchunks - 1) / nchunks;
  kchunk = (kchunk + KT - 1) / KT * KT;
  nchunks = (K + kchunk - 1) / kchunk;
  a.kchunk = kchunk;
  float* part = nullptr;
  RCF_TRY(workspace(ctx, WS_GEMM_PART, sizeof(float4) * size_t(TM * TN) * ntiles * nchunks,
                    reinterpret_cast<void**>(&part)));
  a.part = part;
  gemm_tn_df_kernel<<<dim3(unsigned(ntiles), unsigned(nchunks)), NTHR, 0, ctx->stream>>>(a);
  RCF_CHECK_LAUNCH(ctx);
  gemm_tn_reduce_kernel<<<unsigned(ntiles), 256, 0, ctx->stream>>>(part, int(nchunks), ntiles, a.tiles_n, lower,
                                                                   m, n, C, ldc);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

}  // namespace rcf

// Device helpers shared by the step kernels (stencil.cu, stencil_tma.cu): 4-tuples of
// a node's spinor values (re_up, im_up, re_dn, im_dn), packed FMAs, loads, the 2x2
// spinor potential, the 1D coefficient tables and the tile shapes.
#pragma once

#include "internal.h"

namespace rcf {
namespace {

template <typename Real>
struct alignas(4 * sizeof(Real)) R4 {
  Real v[4];
};

template <typename Real>
__device__ __forceinline__ R4<Real> zero4() {
  R4<Real> r;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.v[i] = Real(0);
  return r;
}

template <typename Real>
__device__ __forceinline__ void fma4(R4<Real>& acc, Real c, const R4<Real>& x) {
#pragma unroll
  for (int i = 0; i < 4; ++i) acc.v[i] = fma(c, x.v[i], acc.v[i]);
}
// FP32: two packed FFMA2 (sm_100+) per 4-tuple
template <>
__device__ __forceinline__ void fma4<float>(R4<float>& acc, float c, const R4<float>& x) {
  const float2 cc = make_float2(c, c);
  const float2 lo = __ffma2_rn(cc, make_float2(x.v[0], x.v[1]), make_float2(acc.v[0], acc.v[1]));
  const float2 hi = __ffma2_rn(cc, make_float2(x.v[2], x.v[3]), make_float2(acc.v[2], acc.v[3]));
  acc.v[0] = lo.x; acc.v[1] = lo.y; acc.v[2] = hi.x; acc.v[3] = hi.y;
}

__device__ __forceinline__ R4<float> ldg4(const R4<float>* p) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  R4<float> r;
  r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  return r;
}
__device__ __forceinline__ R4<double> ldg4(const R4<double>* p) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  R4<double> r;
  r.v[0] = a.x; r.v[1] = a.y; r.v[2] = b.x; r.v[3] = b.y;
  return r;
}
// plain (coherent) load for buffers that the same kernel may write (prev aliases out)
template <typename Real>
__device__ __forceinline__ R4<Real> ld4(const R4<Real>* p) {
  return *p;
}
template <typename Real>
__device__ __forceinline__ void st4(R4<Real>* p, const R4<Real>& x) {
  *p = x;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename Real>
__device__ __forceinline__ void cp_async_r4(R4<Real>* dst, const R4<Real>* src) {
#pragma unroll
  for (int i = 0; i < int(sizeof(R4<Real>) / 16); ++i)
    cp_async16(reinterpret_cast<char*>(dst) + 16 * i, reinterpret_cast<const char*>(src) + 16 * i);
}

// ---- storage types: multivectors kept in St, arithmetic in Real ----
// Conversion of a node's 4-tuple between storage and arithmetic (round to nearest even).
template <typename Real, typename St>
struct Cvt;
template <typename R>
struct Cvt<R, R> {
  static __device__ __forceinline__ R4<R> in(const R4<R>& x) { return x; }
  static __device__ __forceinline__ R4<R> out(const R4<R>& x) { return x; }
};
template <>
struct Cvt<float, __half> {
  static __device__ __forceinline__ R4<float> in(const R4<__half>& x) {
    const __half2* h = reinterpret_cast<const __half2*>(&x);   // the tuple is two half2 words
    const float2 a = __half22float2(h[0]);
    const float2 b = __half22float2(h[1]);
    R4<float> r;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = b.x; r.v[3] = b.y;
    return r;
  }
  static __device__ __forceinline__ R4<__half> out(const R4<float>& x) {
    R4<__half> r;
    __half2* h = reinterpret_cast<__half2*>(&r);
    h[0] = __floats2half2_rn(x.v[0], x.v[1]);
    h[1] = __floats2half2_rn(x.v[2], x.v[3]);
    return r;
  }
};
template <>
struct Cvt<float, __nv_bfloat16> {
  static __device__ __forceinline__ R4<float> in(const R4<__nv_bfloat16>& x) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&x);
    const float2 a = __bfloat1622float2(h[0]);
    const float2 b = __bfloat1622float2(h[1]);
    R4<float> r;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = b.x; r.v[3] = b.y;
    return r;
  }
  static __device__ __forceinline__ R4<__nv_bfloat16> out(const R4<float>& x) {
    R4<__nv_bfloat16> r;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&r);
    h[0] = __floats2bfloat162_rn(x.v[0], x.v[1]);
    h[1] = __floats2bfloat162_rn(x.v[2], x.v[3]);
    return r;
  }
};

// read-only load of a stored 4-tuple
template <typename St>
__device__ __forceinline__ R4<St> ldgs(const R4<St>* p) {
  if constexpr (sizeof(R4<St>) == 8) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    R4<St> r;
    static_assert(sizeof(r) == sizeof(t), "8-byte tuple");
    __builtin_memcpy(&r, &t, sizeof(t));
    return r;
  } else {
    return ldg4(p);
  }
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
// asynchronous copy of one stored 4-tuple (8, 16 or 32 bytes)
template <typename St>
__device__ __forceinline__ void cp_async_s4(R4<St>* dst, const R4<St>* src) {
  if constexpr (sizeof(R4<St>) == 8) cp_async8(dst, src);
  else cp_async_r4(dst, src);
}

// 2x2 spinor potential (Eq. hloc): [[pv + bz, bx - i by], [bx + i by, pv - bz]] u
template <typename Real>
__device__ __forceinline__ void add_potential(R4<Real>& acc, const R4<Real>& pot, const R4<Real>& u) {
  const Real pv = pot.v[0], bx = pot.v[1], by = pot.v[2], bz = pot.v[3];
  const Real ur = u.v[0], ui = u.v[1], dr = u.v[2], di = u.v[3];
  // up row
  acc.v[0] += (pv + bz) * ur + bx * dr + by * di;
  acc.v[1] += (pv + bz) * ui + bx * di - by * dr;
  // down row
  acc.v[2] += bx * ur - by * ui + (pv - bz) * dr;
  acc.v[3] += bx * ui + by * ur + (pv - bz) * di;
}

// Thread -> node of a TX x TY tile (TX, TY multiples of P), grouped by node class so that
// the element-vertex branches are uniform within most warps: first the nodes interior in
// both x and y, then x-vertex nodes, then y-vertex nodes, then nodes that are vertices in
// both (row-major within each class).  A vertex node's 1D row spans two elements (2P + 2
// taps instead of P + 1); in row-major order every warp holds vertex lanes and all its
// lanes pay for them.
template <int P, int TX, int TY>
__device__ __forceinline__ void tile_position(int tid, int& lx, int& ly) {
  if constexpr (P == 1) {   // every node is a vertex
    lx = tid % TX;
    ly = tid / TX;
  } else {
    constexpr int nxv = TX / P, nxi = TX - nxv, nyv = TY / P, nyi = TY - nyv;
    constexpr int n0 = nxi * nyi, n1 = n0 + nxv * nyi, n2 = n1 + nxi * nyv;
    auto interior = [](int i) { return (i / (P - 1)) * P + 1 + i % (P - 1); };
    if (tid < n0) {
      lx = interior(tid % nxi);
      ly = interior(tid / nxi);
    } else if (tid < n1) {
      const int i = tid - n0;
      lx = (i % nxv) * P;
      ly = interior(i / nxv);
    } else if (tid < n2) {
      const int i = tid - n1;
      lx = interior(i % nxi);
      ly = (i / nxi) * P;
    } else {
      const int i = tid - n2;
      lx = (i % nxv) * P;
      ly = (i / nxv) * P;
    }
  }
}

template <typename Real, int P>
struct KTab {
  Real c[3][P + 1][P + 1];
};

// Tile shapes (multiples of P so that tiles start on element vertices), blocks per SM
// and ring depth of the step kernel.
// FP32 (HBM bound): a tile one element high (TY = P, at least about 5 rows) and about
// 24 nodes wide, with as many blocks per SM as 128 registers allow.  Timed on a GB300
// (256-vector step, 2M DoF at p = 5): 20x10 two blocks per SM 4.05 ms, 50x5/2 3.67,
// 25x10/2 3.71, 50x10/1 3.85, 25x5/4 3.60, 25x5/4 with a 6-deep ring and two planes per
// barrier 3.57 (kept); with no arithmetic at all the 20x10 form still took 3.65 ms, so
// the tile shape, through the DRAM access pattern and the number of independent blocks,
// is what sets the time.  p = 6 (3.46M DoF): 24x18/1 7.28 ms, 24x12/1 8.85, 30x6/2 7.31,
// 24x6/3 6.62 (kept).
// FP64 (ALU bound): about 8 x 8, one block per SM.
template <typename Real, int P>
struct TileOf {
  static constexpr bool f32 = sizeof(Real) == 4;
  static constexpr int TX = f32 ? P * ((24 + P - 1) / P) : P * ((8 + P - 1) / P);
  static constexpr int TY_MIN = (120 + TX - 1) / TX;   // FP32: at least ~120 threads per block
  static constexpr int TY = f32 ? P * ((TY_MIN + P - 1) / P) : P * ((8 + P - 1) / P);
  static constexpr int WARPS = (TX * TY + 31) / 32;
  static constexpr int MINB = f32 ? (65536 / (WARPS * 32 * 128) < 1 ? 1 : 65536 / (WARPS * 32 * 128)) : 1;
  static constexpr int NST = f32 ? 6 : 4;   // cp.async ring depth (NST - ZB planes in flight)
  static constexpr bool OWN = false;        // own Z_{k-1}, R planes through the ring (else registers)
  static constexpr int ZB = f32 ? 2 : 1;    // planes per block barrier
};

}  // namespace
}  // namespace rcf

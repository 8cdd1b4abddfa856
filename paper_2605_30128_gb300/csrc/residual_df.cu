// Eigen-residual R = H X - M X diag(lambda) (Algorithm 1; Eq. rChFSIrecurrence takes R
// as its source term) in double-float arithmetic on the FP32 pipes.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate, so an FP64 stencil pass over a
// 256-vector block is ALU bound at roughly twenty times the cost of an FP32 step.
// Here every FP64 quantity is carried as an unevaluated pair (hi, lo) of floats and
// every product-sum uses error-free transformations: the product c_h x_h is split
// exactly into p + e with one FMA, the cross terms c_h x_l + c_l x_h join e, and the
// running sum absorbs p with Knuth's TwoSum while the rounding errors collect in the
// low word (the compensated dot product of Ogita, Rump and Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005).  The result matches an FP64
// evaluation to about 2^-46 relative to the sum of |terms|; the R-ChFSI recurrence
// then reads its FP32 rounding, which this kernel writes directly.
//
// FP64 inputs (X, the projector coefficients) are split into pairs with integer
// operations only (no FP64 instruction): hi keeps the top 24 significand bits, lo the
// next 29 bits rounded to 24.  The coefficient tables, the potential and the mass
// weights are split on the host.
//
// Kernel organisation follows the FP32 step kernel (z-marching TX x TY column tiles,
// a cp.async ring of halo planes, incremental z accumulation), with raw FP64 planes
// in the ring, converted once per plane into a double-buffered (hi, lo) plane, and the
// tile's potential and nonlocal terms staged through the same ring.  Threads are
// grouped by node class (tile_position) so that the element-vertex branches are
// uniform within warps: this kernel is ALU bound, and a divergent vertex branch costs
// every lane of the warp.
#include "internal.h"
#include "stencil_common.cuh"

namespace rcf {
namespace {

// ---- double-float arithmetic on packed pairs of components ----

struct DF2 {   // two components, each hi + lo
  float2 h, l;
};
struct DF4 {   // a node's spinor: (re_up, im_up) and (re_dn, im_dn)
  DF2 a, b;
};
struct Coef {  // a coefficient c = h + l, duplicated for packed operations; nh = -h
  float2 h, nh, l;
};

__device__ __forceinline__ float2 add2(float2 x, float2 y) { return __fadd2_rn(x, y); }
// x - y with one rounding (an FMA with -1 has no intermediate rounding)
__device__ __forceinline__ float2 sub2(float2 x, float2 y) {
  return __ffma2_rn(make_float2(-1.f, -1.f), y, x);
}
__device__ __forceinline__ DF2 zero2() { return DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ DF4 zero4df() { return DF4{zero2(), zero2()}; }

// S += c x with an exact product and an error-free running sum
__device__ __forceinline__ void tap(DF2& S, const Coef& c, const DF2& x) {
  const float2 np = __fmul2_rn(c.nh, x.h);      // -p, p = RN(c_h x_h)
  float2 t = __ffma2_rn(c.h, x.h, np);           // c_h x_h - p, exact
  t = __ffma2_rn(c.h, x.l, t);
  t = __ffma2_rn(c.l, x.h, t);
  const float2 s = sub2(S.h, np);                // TwoSum(S.h, p)
  const float2 bp = sub2(s, S.h);
  const float2 da = sub2(S.h, sub2(s, bp));
  const float2 db = add2(np, bp);                // -(p - bp)
  S.h = s;
  S.l = add2(S.l, add2(t, sub2(da, db)));
}
__device__ __forceinline__ void tap4(DF4& S, const Coef& c, const DF4& x) {
  tap(S.a, c, x.a);
  tap(S.b, c, x.b);
}
// S += x
__device__ __forceinline__ void dfadd(DF2& S, const DF2& x) {
  const float2 s = add2(S.h, x.h);
  const float2 bp = sub2(s, S.h);
  const float2 da = sub2(S.h, sub2(s, bp));
  const float2 db = sub2(x.h, bp);
  S.h = s;
  S.l = add2(S.l, add2(x.l, add2(da, db)));
}
__device__ __forceinline__ void dfadd4(DF4& S, const DF4& x) {
  dfadd(S.a, x.a);
  dfadd(S.b, x.b);
}
__device__ __forceinline__ DF2 swap2(const DF2& x) {
  return DF2{make_float2(x.h.y, x.h.x), make_float2(x.l.y, x.l.x)};
}
// coefficient from per-component (hi, lo) pairs
__device__ __forceinline__ Coef coef2(float2 h, float2 l) {
  return Coef{h, make_float2(-h.x, -h.y), l};
}
__device__ __forceinline__ Coef coef1(float h, float l) {
  return coef2(make_float2(h, h), make_float2(l, l));
}

// scalar double-float product, normalised
__device__ __forceinline__ float2 dfmul1(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}
// scalar double-float sum, normalised
__device__ __forceinline__ float2 dfadd1(float2 x, float2 y) {
  const float s = __fadd_rn(x.x, y.x);
  const float bp = __fsub_rn(s, x.x);
  const float err = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s, bp)), __fsub_rn(y.x, bp));
  const float l = __fadd_rn(__fadd_rn(x.y, y.y), err);
  const float h = __fadd_rn(s, l);
  return make_float2(h, __fsub_rn(l, __fsub_rn(h, s)));
}

// FP64 -> (hi, lo) with integer operations.  hi: the sign, exponent and top 23
// fraction bits (truncation); lo: the remaining 29 fraction bits, converted to float
// (rounded to 24 bits) and scaled by 2^(E - 1075).  |x - hi - lo| <= 2^-48 |x| for
// 2^-74 <= |x| < 2^128; below 2^-126 the pair is (0, 0), below 2^-74 lo is 0
// (absolute error < 2^-97); beyond the float range hi is infinite.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned hw = static_cast<unsigned>(__double2hiint(x));
  const unsigned lw = static_cast<unsigned>(__double2loint(x));
  const unsigned sgn = hw & 0x80000000u;
  const int E = int((hw >> 20) & 0x7FFu);
  const int e32 = E - 896;   // float biased exponent of hi
  const int es = E - 948;    // float biased exponent of 2^(E - 1075)
  const unsigned f23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const unsigned r = lw & 0x1FFFFFFFu;
  float h = __uint_as_float(sgn | (static_cast<unsigned>(e32) << 23) | f23);
  float l = __fmul_rn(__uint2float_rn(r), __uint_as_float(static_cast<unsigned>(es) << 23));
  l = __uint_as_float(__float_as_uint(l) | sgn);
  if (es <= 0) l = __uint_as_float(sgn);
  if (e32 <= 0) h = __uint_as_float(sgn);
  if (e32 >= 255) { h = __uint_as_float(sgn | 0x7F800000u); l = 0.f; }
  hi = h;
  lo = l;
}

struct alignas(16) D4 {   // a node's four doubles in shared memory
  double v[4];
};

__device__ __forceinline__ void split4(const D4& d, float4& h, float4& l) {
  split_f64(d.v[0], h.x, l.x);
  split_f64(d.v[1], h.y, l.y);
  split_f64(d.v[2], h.z, l.z);
  split_f64(d.v[3], h.w, l.w);
}
__device__ __forceinline__ DF4 df4_of(float4 h, float4 l) {
  return DF4{DF2{make_float2(h.x, h.y), make_float2(l.x, l.y)},
             DF2{make_float2(h.z, h.w), make_float2(l.z, l.w)}};
}
__device__ __forceinline__ DF4 load_split(const double* p) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *(reinterpret_cast<const double2*>(p) + 1);
  float4 h, l;
  split_f64(a.x, h.x, l.x);
  split_f64(a.y, h.y, l.y);
  split_f64(b.x, h.z, l.z);
  split_f64(b.y, h.w, l.w);
  return df4_of(h, l);
}

// 16-byte asynchronous copy that zero-fills instead of reading when !pred
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, bool pred) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}

// ---- kernel ----

// row-scaled 1D operators (D^{-1} K) and 1D lumped-mass weights, as double-float pairs
template <int P>
struct DFTabs {
  Coef c[3][P + 1][P + 1];
  float2 wg[3][P];   // wg[d][a]: vertex (a = 0) h w_0, interior h w_a / 2
};

struct ResidualDFArgs {
  const double* X;  int64_t ldx;      // c128 [nvec][ldx]
  float* Rh;        float* Rl;        // c64 [nvec][ldr]: FP32 rounding of R and the remainder
  int64_t ldr;                        // (Rl may be null)
  const float* pot;                   // [nnodes][8]: (pv+bz, pv-bz, bx, by)/M_I hi, then lo
  const int* nodemap;                 // [nnodes] index into the projector-support union, -1 outside
  const float* nls;                   // [nunion][nvec][8] sum_a beta C2 (hi4, lo4)
  const float* neglam;                // [2][nvec]: hi, lo of -lambda_v
  int nvec;
};

template <int P, int TX, int TY, int NST>
constexpr size_t df_smem_bytes() {
  constexpr int W = TX + P + 1, H = TY + P + 1, HALO = W * H, NT = TX * TY;
  return size_t(NST) * HALO * sizeof(D4)            // raw FP64 planes
         + size_t(NST) * 4 * NT * sizeof(float4)    // tile potential and nonlocal terms (hi, lo)
         + size_t(2) * 2 * HALO * sizeof(float4)    // converted planes (hi, lo), double buffered
         + size_t(3) * (P + 1) * (P + 1) * sizeof(Coef);
}

// Tiles as the FP32 step kernel's (one element high, about 24 nodes wide), a 2-deep ring
// (one plane in flight: the kernel is ALU bound), and as many blocks per SM (at most
// three) as 227 KB of shared memory and the registers hold.  Timed on a GB300 at p = 5 (256 vectors, 2M
// DoF, kernel alone): 20x10/2 blocks with a 3-deep ring 18.2 ms, 20x10/2 ring 2 18.1,
// 25x5/2 ring 3 19.1, 25x10/2 ring 2 16.0, 25x5/3 ring 2 15.9 (kept).
template <int P>
struct DFTile {
  static constexpr int TX = TileOf<float, P>::TX;
  static constexpr int TY = TileOf<float, P>::TY;
  static constexpr int NST = 2;
  static constexpr int FIT_SMEM = int((227u * 1024u) / df_smem_bytes<P, TX, TY, NST>());
  // registers a thread needs without spilling grow with the P z-accumulators (~96 + 12 P)
  static constexpr int FIT_REGS = 65536 / (((TX * TY + 31) / 32) * 32 * (96 + 12 * P));
  static constexpr int FIT = FIT_SMEM < FIT_REGS ? FIT_SMEM : FIT_REGS;
  static constexpr int MINB = FIT < 1 ? 1 : (FIT > 3 ? 3 : FIT);
};

template <int P, int TX, int TY, int NST>
__global__ void __launch_bounds__(TX* TY, DFTile<P>::MINB)
    residual_df_kernel(const ResidualDFArgs a, const DFTabs<P> tb, const int Gx, const int Gy, const int Gz) {
  constexpr int W = TX + P + 1;
  constexpr int H = TY + P + 1;
  constexpr int NT = TX * TY;
  constexpr int HALO = W * H;
  constexpr int KMAX = (HALO + NT - 1) / NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  D4* RAW = reinterpret_cast<D4*>(smem_raw);                       // [NST][HALO]
  float4* TT = reinterpret_cast<float4*>(RAW + NST * HALO);        // [NST][4][NT]: pot h, pot l, nl h, nl l
  float4* SH = TT + NST * 4 * NT;                                  // [2][HALO]
  float4* SL = SH + 2 * HALO;                                      // [2][HALO]
  Coef* CT = reinterpret_cast<Coef*>(SL + 2 * HALO);               // [3][P+1][P+1]: x, y, z
  const Coef* CZ = CT + 2 * (P + 1) * (P + 1);

  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * (P + 1) * (P + 1); i += NT) CT[i] = (&tb.c[0][0][0])[i];

  int lx, ly;
  tile_position<P, TX, TY>(tid, lx, ly);
  const int ntx = (Gx + TX - 1) / TX;
  const int x0 = (blockIdx.x % ntx) * TX;
  const int y0 = (blockIdx.x / ntx) * TY;
  const int v = blockIdx.y;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool active = (gx < Gx) && (gy < Gy);
  const int nz = Gz / P;
  const int64_t plane = int64_t(Gx) * Gy;
  const int64_t col = active ? int64_t(gx) + int64_t(Gx) * gy : 0;
  const double* Xv = a.X + 2 * int64_t(v) * a.ldx;

  int hs[KMAX], hg[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = tid + k * NT;
    hs[k] = -1;
    hg[k] = 0;
    if (e < HALO) {
      const int r = e / W, c = e - r * W;
      if ((r >= P && r < P + TY) || (c >= P && c < P + TX)) {
        int xx = (x0 - P + c) % Gx;
        if (xx < 0) xx += Gx;
        int yy = (y0 - P + r) % Gy;
        if (yy < 0) yy += Gy;
        hs[k] = e;
        hg[k] = xx + Gx * yy;
      }
    }
  }

  // support flags of the planes in flight (bit z % 32) and the next plane's union index
  unsigned supp = 0;
  int nm_next = -1;
  auto load_nm = [&](int z) {
    nm_next = (a.nodemap && active && z < Gz) ? a.nodemap[col + int64_t(z) * plane] : -1;
  };
  auto issue_plane = [&](int z, int s) {
    D4* st = RAW + s * HALO;
    const double* src = Xv + 4 * (int64_t(z) * plane);
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      if (hs[k] >= 0) {
        cp_async16(&st[hs[k]].v[0], src + 4 * int64_t(hg[k]));
        cp_async16(&st[hs[k]].v[2], src + 4 * int64_t(hg[k]) + 2);
      }
    if (active) {
      const int64_t I = col + int64_t(z) * plane;
      float4* t = TT + s * 4 * NT;
      cp_async16(&t[0 * NT + tid], a.pot + 8 * I);
      cp_async16(&t[1 * NT + tid], a.pot + 8 * I + 4);
      const bool in = nm_next >= 0;
      const float* nsrc = in ? a.nls + 8 * (int64_t(nm_next) * a.nvec + v) : a.pot;
      cp_async16_zfill(&t[2 * NT + tid], nsrc, in);
      cp_async16_zfill(&t[3 * NT + tid], nsrc + 4, in);
      if (in) supp |= 1u << (z & 31);
      else supp &= ~(1u << (z & 31));
    }
    cp_async_commit();
  };

  // element -1 (planes Gz-P .. Gz-1) contributes row P of its 1D matrix to vertex plane 0
  DF4 accn = zero4df();
  if (active) {
#pragma unroll
    for (int c = 0; c < P; ++c) tap4(accn, tb.c[2][P][c], load_split(Xv + 4 * (col + int64_t(Gz - P + c) * plane)));
  }

  load_nm(0);
#pragma unroll
  for (int s = 0; s < NST - 1; ++s) {
    if (s < Gz) {
      issue_plane(s, s);
      load_nm(s + 1);
    } else {
      cp_async_commit();
    }
  }
  int zload = NST - 1;

  __syncthreads();  // tables visible
  const int ax = lx % P, by = ly % P;
  const float2 wxy = dfmul1(tb.wg[0][ax], tb.wg[1][by]);
  const Coef nlam = coef1(a.neglam[v], a.neglam[a.nvec + v]);
  const Coef* cxr = CT + (0 * (P + 1) + ax) * (P + 1);
  const Coef* cxv = CT + (0 * (P + 1) + P) * (P + 1);
  const Coef* cyr = CT + (1 * (P + 1) + by) * (P + 1);
  const Coef* cyv = CT + (1 * (P + 1) + P) * (P + 1);

  DF4 acc[P];
  auto emit = [&](int ez) {
    if (!active) return;
#pragma unroll
    for (int cc = 0; cc < P; ++cc) {
      const int64_t I = col + int64_t(ez * P + cc) * plane;
      const float2 m = dfmul1(wxy, tb.wg[2][cc]);
      const Coef mc = coef1(m.x, m.y);
      DF4 r = zero4df();
      tap4(r, mc, acc[cc]);
      // normalise: hi = RN(h + l) is the FP32 rounding of R, lo the remainder
      float4 oh, ol;
      {
        const float2 h0 = add2(r.a.h, r.a.l), h1 = add2(r.b.h, r.b.l);
        oh = make_float4(h0.x, h0.y, h1.x, h1.y);
        const float2 l0 = sub2(r.a.l, sub2(h0, r.a.h)), l1 = sub2(r.b.l, sub2(h1, r.b.h));
        ol = make_float4(l0.x, l0.y, l1.x, l1.y);
      }
      *reinterpret_cast<float4*>(a.Rh + 2 * int64_t(v) * a.ldr + 4 * I) = oh;
      if (a.Rl) *reinterpret_cast<float4*>(a.Rl + 2 * int64_t(v) * a.ldr + 4 * I) = ol;
    }
  };

  // planes in order; c = local index of the plane in its z element.  The loop is not
  // unrolled (the body is large); the branches on c are uniform across the block.
  int c = 0, ez = 0;
  for (int z = 0; z < Gz; ++z) {
    const int s = z % NST;
    cp_async_wait<NST - 2>();
    // convert this thread's copies of plane z into the (hi, lo) plane z & 1
    {
      const D4* st = RAW + s * HALO;
      float4* dh = SH + (z & 1) * HALO;
      float4* dl = SL + (z & 1) * HALO;
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (hs[k] >= 0) {
          float4 h, l;
          split4(st[hs[k]], h, l);
          dh[hs[k]] = h;
          dl[hs[k]] = l;
        }
    }
    __syncthreads();
    if (zload < Gz) {
      issue_plane(zload, zload % NST);
      load_nm(zload + 1);
    } else {
      cp_async_commit();
    }
    ++zload;

    const float4* Ph = SH + (z & 1) * HALO;
    const float4* Pl = SL + (z & 1) * HALO;
    auto node = [&](int k) { return df4_of(Ph[k], Pl[k]); };
    const DF4 u = node((ly + P) * W + lx + P);
    DF4 self = zero4df();
    {
      const int row = (ly + P) * W;
      const int cb = lx - ax + P;
#pragma unroll
      for (int q = 0; q <= P; ++q) tap4(self, cxr[q], node(row + cb + q));
      if (ax == 0) {
#pragma unroll
        for (int q = 0; q <= P; ++q) tap4(self, cxv[q], node(row + cb - P + q));
      }
      const int rb = ly - by + P;
#pragma unroll
      for (int q = 0; q <= P; ++q) tap4(self, cyr[q], node((rb + q) * W + lx + P));
      if (by == 0) {
#pragma unroll
        for (int q = 0; q <= P; ++q) tap4(self, cyv[q], node((rb - P + q) * W + lx + P));
      }
    }
    // spinor potential and -lambda: [[pv+bz-l, bx-i by], [bx+i by, pv-bz-l]] u
    {
      const float4* t = TT + s * 4 * NT;
      const float4 ph = t[0 * NT + tid], pl = t[1 * NT + tid];
      const float2 dA = dfadd1(make_float2(ph.x, pl.x), make_float2(nlam.h.x, nlam.l.x));
      const float2 dD = dfadd1(make_float2(ph.y, pl.y), make_float2(nlam.h.x, nlam.l.x));
      const Coef cA = coef1(dA.x, dA.y), cD = coef1(dD.x, dD.y), cBx = coef1(ph.z, pl.z);
      const Coef cBy = coef2(make_float2(ph.w, -ph.w), make_float2(pl.w, -pl.w));    // ( by, -by)
      const Coef cnBy = coef2(make_float2(-ph.w, ph.w), make_float2(-pl.w, pl.w));   // (-by,  by)
      tap(self.a, cA, u.a);
      tap(self.a, cBx, u.b);
      tap(self.a, cBy, swap2(u.b));
      tap(self.b, cBx, u.a);
      tap(self.b, cnBy, swap2(u.a));
      tap(self.b, cD, u.b);
      if (supp & (1u << (z & 31))) dfadd4(self, df4_of(t[2 * NT + tid], t[3 * NT + tid]));
    }
    if (c == 0) {
      // the vertex plane closes element ez-1 (its local node P) and opens element ez
      tap4(accn, tb.c[2][P][P], u);
      if (ez > 0) {
#pragma unroll
        for (int cc = 0; cc < P; ++cc) tap4(acc[cc], tb.c[2][cc][P], u);
        emit(ez - 1);
      }
      acc[0] = accn;
      dfadd4(acc[0], self);
#pragma unroll
      for (int cc = 1; cc < P; ++cc) acc[cc] = zero4df();
#pragma unroll
      for (int cc = 0; cc < P; ++cc) tap4(acc[cc], tb.c[2][cc][0], u);
      accn = zero4df();
      tap4(accn, tb.c[2][P][0], u);
    } else {
      const Coef* cz = CZ + c;   // column c of the z operator: cz[cc * (P + 1)] = C_z[cc][c]
#pragma unroll
      for (int cc = 1; cc < P; ++cc)
        if (cc == c) dfadd4(acc[cc], self);
#pragma unroll
      for (int cc = 0; cc < P; ++cc) tap4(acc[cc], cz[cc * (P + 1)], u);
      tap4(accn, cz[P * (P + 1)], u);
    }
    if (++c == P) { c = 0; ++ez; }
  }
  // the last element closes on plane Gz = 0 (periodic)
  if (active) {
    const DF4 u0 = load_split(Xv + 4 * col);
#pragma unroll
    for (int cc = 0; cc < P; ++cc) tap4(acc[cc], tb.c[2][cc][P], u0);
  }
  emit(nz - 1);
  cp_async_wait<0>();
}

// (hi, lo) of n doubles
__global__ void split_kernel(int64_t n, const double* __restrict__ x, float* __restrict__ hi,
                             float* __restrict__ lo) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float h, l;
    split_f64(x[i], h, l);
    hi[i] = h;
    lo[i] = l;
  }
}

// NLs[u][v] = sum over the support entries at union node u of beta_e C2[atom_e][.][v]
// (the nonlocal term before the mass factor), thread per (u, v)
constexpr int kGatherThreads = 128;
__global__ void __launch_bounds__(kGatherThreads)
    nl_gather_df_kernel(const int* __restrict__ uoff, const int* __restrict__ uent,
                        const int* __restrict__ atom, const float* __restrict__ betadf,
                        const float* __restrict__ c2h, const float* __restrict__ c2l, int nvec,
                        float* __restrict__ nls) {
  const int u = blockIdx.x;
  const int v = blockIdx.y * kGatherThreads + threadIdx.x;
  if (v >= nvec) return;
  DF2 sa = zero2(), sb = zero2();
  const int k0 = uoff[u], k1 = uoff[u + 1];
  for (int k = k0; k < k1; ++k) {
    const int e = uent[k];
    const int at = atom[e];
#pragma unroll
    for (int f6 = 0; f6 < 6; ++f6) {
      const Coef b = coef1(betadf[12 * int64_t(e) + 2 * f6], betadf[12 * int64_t(e) + 2 * f6 + 1]);
      const int64_t i0 = 2 * ((int64_t(at) * 12 + 2 * f6) * nvec + v);
      const int64_t i1 = 2 * ((int64_t(at) * 12 + 2 * f6 + 1) * nvec + v);
      tap(sa, b, DF2{*reinterpret_cast<const float2*>(c2h + i0), *reinterpret_cast<const float2*>(c2l + i0)});
      tap(sb, b, DF2{*reinterpret_cast<const float2*>(c2h + i1), *reinterpret_cast<const float2*>(c2l + i1)});
    }
  }
  float4* o = reinterpret_cast<float4*>(nls + 8 * (int64_t(u) * nvec + v));
  o[0] = make_float4(sa.h.x, sa.h.y, sb.h.x, sb.h.y);
  o[1] = make_float4(sa.l.x, sa.l.y, sb.l.x, sb.l.y);
}

void split_host(double x, float* h, float* l) {
  *h = float(x);
  *l = float(x - double(*h));
}
Coef coef_host(double x) {
  float h, l;
  split_host(x, &h, &l);
  return Coef{make_float2(h, h), make_float2(-h, -h), make_float2(l, l)};
}

template <int P>
int launch_df_p(rcf_ctx* ctx, const rcf_op* op, const ResidualDFArgs& args) {
  constexpr int TX = DFTile<P>::TX, TY = DFTile<P>::TY, NST = DFTile<P>::NST;
  const rcf_mesh* m = op->mesh;
  Tables t;
  build_tables(m, TAB_ROW_SCALED, &t);
  DFTabs<P> tb;
  for (int d = 0; d < 3; ++d) {
    for (int i = 0; i <= P; ++i)
      for (int j = 0; j <= P; ++j) tb.c[d][i][j] = coef_host(t.c[d][i][j]);
    for (int i = 0; i < P; ++i) {
      const double w = (i == 0) ? m->h[d] * m->w[0] : 0.5 * m->h[d] * m->w[i];
      float h, l;
      split_host(w, &h, &l);
      tb.wg[d][i] = make_float2(h, l);
    }
  }
  constexpr size_t smem = df_smem_bytes<P, TX, TY, NST>();
  auto kern = residual_df_kernel<P, TX, TY, NST>;
  if (smem > 48 * 1024) RCF_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int ntx = (m->G[0] + TX - 1) / TX, nty = (m->G[1] + TY - 1) / TY;
  dim3 grid(ntx * nty, args.nvec);
  kern<<<grid, TX * TY, smem, ctx->stream>>>(args, tb, m->G[0], m->G[1], m->G[2]);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

}  // namespace

int launch_split_f64(rcf_ctx* ctx, int64_t n, const double* x, float* hi, float* lo) {
  if (n <= 0) return RCF_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  split_kernel<<<unsigned(blocks), 256, 0, ctx->stream>>>(n, x, hi, lo);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_residual_df(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                       const double* neglam_d, float* Rh, float* Rl, int64_t ldr) {
  if (nvec <= 0) return RCF_OK;
  const rcf_mesh* m = op->mesh;
  if (op->fm) return fail(ctx, RCF_ENOTSUP, "the double-float residual is not available with the full consistent mass");
  if (!op->d_potdf) return fail(ctx, RCF_EINVAL, "potential not set");
  ResidualDFArgs args{};
  args.X = X; args.ldx = ldx;
  args.Rh = Rh; args.Rl = Rl; args.ldr = ldr;
  args.pot = op->d_potdf;
  args.nvec = nvec;
  float* lam = nullptr;
  RCF_TRY(workspace(ctx, WS_DF_LAM, sizeof(float) * 2 * size_t(nvec), reinterpret_cast<void**>(&lam)));
  RCF_TRY(launch_split_f64(ctx, nvec, neglam_d, lam, lam + nvec));
  args.neglam = lam;
  const ProjAtoms& pa = op->proj;
  if (pa.natoms > 0 && pa.nunion > 0) {
    // C = P^H X (FP64), C2 = Delta C, split, then the per-node sums over the supports
    const size_t nc = size_t(24) * pa.natoms * nvec;
    double *C = nullptr, *C2 = nullptr;
    float* c2df = nullptr;
    float* nls = nullptr;
    RCF_TRY(workspace(ctx, WS_NLC, sizeof(double) * nc, reinterpret_cast<void**>(&C)));
    RCF_TRY(workspace(ctx, WS_NLC2, sizeof(double) * nc, reinterpret_cast<void**>(&C2)));
    RCF_TRY(workspace(ctx, WS_DF_C2, sizeof(float) * 2 * nc, reinterpret_cast<void**>(&c2df)));
    RCF_TRY(workspace(ctx, WS_DF_NL, sizeof(float) * 8 * size_t(pa.nunion) * nvec, reinterpret_cast<void**>(&nls)));
    RCF_TRY(launch_nl_project<double>(ctx, op, X, ldx, nvec, 1, C));
    RCF_TRY(launch_nl_delta<double>(ctx, op, C, nvec, 1.0, C2));
    RCF_TRY(launch_split_f64(ctx, int64_t(nc), C2, c2df, c2df + nc));
    dim3 grid(unsigned(pa.nunion), unsigned((nvec + kGatherThreads - 1) / kGatherThreads));
    nl_gather_df_kernel<<<grid, kGatherThreads, 0, ctx->stream>>>(pa.d_uoff, pa.d_uent, pa.d_atom, pa.d_betadf,
                                                                  c2df, c2df + nc, nvec, nls);
    RCF_CHECK_LAUNCH(ctx);
    args.nodemap = pa.d_nodemap;
    args.nls = nls;
  }
  switch (m->p) {
    case 1: return launch_df_p<1>(ctx, op, args);
    case 2: return launch_df_p<2>(ctx, op, args);
    case 3: return launch_df_p<3>(ctx, op, args);
    case 4: return launch_df_p<4>(ctx, op, args);
    case 5: return launch_df_p<5>(ctx, op, args);
    case 6: return launch_df_p<6>(ctx, op, args);
    case 7: return launch_df_p<7>(ctx, op, args);
    case 8: return launch_df_p<8>(ctx, op, args);
    default: return fail(ctx, RCF_ENOTSUP, "degree p=%d not built (1..8)", m->p);
  }
}

}  // namespace rcf

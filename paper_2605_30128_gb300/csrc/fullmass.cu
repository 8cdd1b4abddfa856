// The Hamiltonian and mass with the full consistent mass and Gauss-Legendre quadrature
// (Section III-A; Section III-B-2): the paper's noncollinear setting, where the filter uses a
// diagonal D (the GLL-integrated mass) in place of M^-1 and R-ChFSI still converges to the
// eigenpairs of H x = eps M x.
//
// With nq >= p + 1 Gauss points per direction the cell integrals of the kinetic term and of
// the mass are exact, and on a uniform mesh the assembled matrices are tensor products of
// assembled 1D matrices: M = Mz (x) My (x) Mx and the kinetic term
// 1/2 (Kz My Mx + Mz Ky Mx + Mz My Kx), with K the 1D stiffness (2/h) K1 and M the 1D
// consistent mass (h/2) M1, both banded (the nodes of an element, two elements at a vertex).
// They are applied by sum factorisation in three node passes, one per direction:
//   x: t1 = Mx u, t2 = Kx u;  y: s1 = My t1, s2 = Ky t1 + My t2;  z: K u = Kz s1 + Mz s2
// (the 1/2 folded into the K tables), and M u = Mz My Mx u the same way.
// The potential V I + B . sigma is given at the Gauss points and couples all nodes of a cell:
// per cell and vector, the nodal spinor values are interpolated to the nq^3 points (three
// 1D contractions with the Lagrange table B1 [nq][np]), multiplied by w_q |J| (V I + B . sigma),
// projected back (the transposed contractions) and written to a per-cell buffer; a node pass
// then sums the contributions of the (up to 8) cells of each node, with no atomics.
// The spin-orbit projector columns int N_I beta are computed with the same Gauss rule at
// set-up and applied by the nonlocal kernels of the lumped operator.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <vector>

#include "bfp_common.cuh"
#include "internal.h"
#include "stencil_common.cuh"

namespace rcf {
namespace {

__device__ __forceinline__ int wrapi(int i, int G) { return i < 0 ? i + G : (i >= G ? i - G : i); }

// 4 reals of node I of vector v (complex spinor: re up, im up, re down, im down)
template <typename Real>
__device__ __forceinline__ R4<Real> ld_node(const Real* base, int64_t ld, int v, int64_t I) {
  return ldg4(reinterpret_cast<const R4<Real>*>(base + 2 * int64_t(v) * ld) + I);
}
template <typename Real>
__device__ __forceinline__ void st_node(Real* base, int64_t ld, int v, int64_t I, const R4<Real>& x) {
  st4(reinterpret_cast<R4<Real>*>(base + 2 * int64_t(v) * ld) + I, x);
}

// One 1D pass along direction d: out1 = c1 * in1 + c2 * in2, out2 = c3 * in1 + c4 * in2
// (tables [p][2p + 1] by local position and offset; null tables, inputs and outputs skipped)
template <typename Real>
__global__ void fm_pass_kernel(int d, int p, int Gx, int Gy, int Gz, const Real* __restrict__ c1,
                               const Real* __restrict__ c2, const Real* __restrict__ c3,
                               const Real* __restrict__ c4, const Real* __restrict__ in1,
                               const Real* __restrict__ in2, int64_t ldin, Real* __restrict__ out1,
                               Real* __restrict__ out2, int64_t ldout) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (I >= int64_t(Gx) * Gy * Gz) return;
  const int idx[3] = {int(I % Gx), int((I / Gx) % Gy), int(I / (int64_t(Gx) * Gy))};
  const int G[3] = {Gx, Gy, Gz};
  const int64_t stride = d == 0 ? 1 : (d == 1 ? int64_t(Gx) : int64_t(Gx) * Gy);
  const int i = idx[d], a = i % p;
  const int lo = a == 0 ? -p : -a, hi = a == 0 ? p : p - a;
  const int64_t base = I - int64_t(i) * stride;
  R4<Real> o1 = zero4<Real>(), o2 = zero4<Real>();
  const int row = a * (2 * p + 1) + p;
  for (int o = lo; o <= hi; ++o) {
    const int64_t J = base + int64_t(wrapi(i + o, G[d])) * stride;
    const R4<Real> x1 = ld_node(in1, ldin, v, J);
    if (c1) fma4(o1, c1[row + o], x1);
    if (c3) fma4(o2, c3[row + o], x1);
    if (in2) {
      const R4<Real> x2 = ld_node(in2, ldin, v, J);
      if (c2) fma4(o1, c2[row + o], x2);
      if (c4) fma4(o2, c4[row + o], x2);
    }
  }
  if (out1) st_node(out1, ldout, v, I, o1);
  if (out2) st_node(out2, ldout, v, I, o2);
}

// Per cell e and vector v: E[v][e][l] = sum_q N_l(x_q) w_q |J| (V_q I + B_q . sigma) u(x_q),
// u(x_q) = sum_l' N_l'(x_q) u_{node(e, l')} (u = dinv in if dinv is given), by sum
// factorisation: each 1D contraction is done by one thread per line of the cell, with the
// line's values in registers, so that shared memory holds only the intermediate blocks:
//   1. gather + x:  line (b, c): u[a] from HBM -> A[qx + nq (b + NP c)]
//   2. y:           line (qx, c): A[. b .] -> Bf[qx + nq (qy + nq c)]
//   3. z, potential, z back: line (qx, qy): Bf[. c] -> u at the nq points of the line ->
//                   times w_q |J| (V + B . sigma) -> projected back onto c -> A[qx + nq (qy + nq c)]
//   4. y back:      line (qx, c): A[. qy .] -> Bf[qx + nq (b + NP c)]
//   5. x back:      line (b, c): Bf[qx . .] -> E[a + NP (b + NP c)] in HBM
// A block takes one cell and NVB vectors (the cell's potential read once for them); SB
// tuples per vector and buffer.  B1 [nq][NP]: the Lagrange basis at the Gauss nodes.
template <typename Real, int P>
__global__ void __launch_bounds__(256) fm_cell_kernel(int nq, int nx, int ny, int nz, const Real* __restrict__ B1,
                                                      const Real* __restrict__ vq, const Real* __restrict__ in,
                                                      int64_t ldin, const Real* __restrict__ dinv,
                                                      Real* __restrict__ E, int nvec, int NVB, int SB) {
  using V4 = R4<Real>;
  constexpr int NP = P + 1, NL = NP * NP * NP;
  extern __shared__ __align__(16) unsigned char fm_cell_smem[];
  V4* A = reinterpret_cast<V4*>(fm_cell_smem);   // [NVB][SB]
  V4* Bf = A + size_t(NVB) * SB;                  // [NVB][SB]
  V4* VQ = Bf + size_t(NVB) * SB;                 // [nq^3] the cell's w_q |J| (V, Bx, By, Bz)
  Real* B = reinterpret_cast<Real*>(VQ + nq * nq * nq);   // [nq][NP]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t e = blockIdx.x;
  const int v0 = blockIdx.y * NVB, nvb = min(NVB, nvec - v0);
  const int ex = int(e % nx), ey = int((e / nx) % ny), ez = int(e / (int64_t(nx) * ny));
  const int Gx = nx * P, Gy = ny * P, Gz = nz * P;
  const int nq2 = nq * nq, nq3 = nq2 * nq;
  for (int i = tid; i < nq * NP; i += nt) B[i] = B1[i];
  {
    const V4* vc4 = reinterpret_cast<const V4*>(vq) + e * int64_t(nq3);
    for (int i = tid; i < nq3; i += nt) VQ[i] = ldg4(vc4 + i);
  }
  __syncthreads();
  // 1. gather and interpolate along x
  for (int t = tid; t < nvb * NP * NP; t += nt) {
    const int j = t / (NP * NP), line = t - j * NP * NP;
    const int b = line % NP, c = line / NP;
    int yy = ey * P + b, zz = ez * P + c;
    if (yy >= Gy) yy -= Gy;
    if (zz >= Gz) zz -= Gz;
    const int64_t rowI = int64_t(Gx) * (yy + int64_t(Gy) * zz);
    const V4* x = reinterpret_cast<const V4*>(in + 2 * int64_t(v0 + j) * ldin);
    V4 u[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      int xx = ex * P + a;
      if (xx >= Gx) xx -= Gx;
      u[a] = ldg4(x + rowI + xx);
      if (dinv) {
        const Real d = dinv[rowI + xx];
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) u[a].v[c4] *= d;
      }
    }
    V4* out = A + size_t(j) * SB + nq * line;
#pragma unroll 4
    for (int qx = 0; qx < nq; ++qx) {
      V4 s = zero4<Real>();
#pragma unroll
      for (int a = 0; a < NP; ++a) fma4(s, B[qx * NP + a], u[a]);
      out[qx] = s;
    }
  }
  __syncthreads();
  // 2. along y
  for (int t = tid; t < nvb * nq * NP; t += nt) {
    const int j = t / (nq * NP), line = t - j * nq * NP;
    const int qx = line % nq, c = line / nq;
    const V4* src = A + size_t(j) * SB;
    V4 u[NP];
#pragma unroll
    for (int b = 0; b < NP; ++b) u[b] = src[qx + nq * (b + NP * c)];
    V4* out = Bf + size_t(j) * SB;
#pragma unroll 4
    for (int qy = 0; qy < nq; ++qy) {
      V4 s = zero4<Real>();
#pragma unroll
      for (int b = 0; b < NP; ++b) fma4(s, B[qy * NP + b], u[b]);
      out[qx + nq * (qy + nq * c)] = s;
    }
  }
  __syncthreads();
  // 3. along z to the points, the spinor potential, and back along z
  for (int t = tid; t < nvb * nq2; t += nt) {
    const int j = t / nq2, qxy = t - j * nq2;
    const V4* src = Bf + size_t(j) * SB;
    V4 u[NP], o[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      u[c] = src[qxy + nq2 * c];
      o[c] = zero4<Real>();
    }
#pragma unroll 4
    for (int qz = 0; qz < nq; ++qz) {
      V4 w = zero4<Real>();
#pragma unroll
      for (int c = 0; c < NP; ++c) fma4(w, B[qz * NP + c], u[c]);
      const V4 pq = VQ[qxy + nq2 * qz];
      const Real V = pq.v[0], Bx = pq.v[1], By = pq.v[2], Bz = pq.v[3];
      // up = (V + Bz) u_up + (Bx - i By) u_dn ; dn = (Bx + i By) u_up + (V - Bz) u_dn
      V4 h;
      h.v[0] = (V + Bz) * w.v[0] + Bx * w.v[2] + By * w.v[3];
      h.v[1] = (V + Bz) * w.v[1] + Bx * w.v[3] - By * w.v[2];
      h.v[2] = Bx * w.v[0] - By * w.v[1] + (V - Bz) * w.v[2];
      h.v[3] = Bx * w.v[1] + By * w.v[0] + (V - Bz) * w.v[3];
#pragma unroll
      for (int c = 0; c < NP; ++c) fma4(o[c], B[qz * NP + c], h);
    }
    V4* out = A + size_t(j) * SB;
#pragma unroll
    for (int c = 0; c < NP; ++c) out[qxy + nq2 * c] = o[c];
  }
  __syncthreads();
  // 4. back along y
  for (int t = tid; t < nvb * nq * NP; t += nt) {
    const int j = t / (nq * NP), line = t - j * nq * NP;
    const int qx = line % nq, c = line / nq;
    const V4* src = A + size_t(j) * SB;
    V4 o[NP];
#pragma unroll
    for (int b = 0; b < NP; ++b) o[b] = zero4<Real>();
#pragma unroll 4
    for (int qy = 0; qy < nq; ++qy) {
      const V4 w = src[qx + nq * (qy + nq * c)];
#pragma unroll
      for (int b = 0; b < NP; ++b) fma4(o[b], B[qy * NP + b], w);
    }
    V4* out = Bf + size_t(j) * SB;
#pragma unroll
    for (int b = 0; b < NP; ++b) out[qx + nq * (b + NP * c)] = o[b];
  }
  __syncthreads();
  // 5. back along x, to the cell buffer
  for (int t = tid; t < nvb * NP * NP; t += nt) {
    const int j = t / (NP * NP), line = t - j * NP * NP;
    const V4* src = Bf + size_t(j) * SB + nq * line;
    V4 o[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) o[a] = zero4<Real>();
#pragma unroll 4
    for (int qx = 0; qx < nq; ++qx) {
      const V4 w = src[qx];
#pragma unroll
      for (int a = 0; a < NP; ++a) fma4(o[a], B[qx * NP + a], w);
    }
    V4* out = reinterpret_cast<V4*>(E) + (int64_t(v0 + j) * gridDim.x + e) * NL + NP * line;
#pragma unroll
    for (int a = 0; a < NP; ++a) out[a] = o[a];
  }
}

// Element matrices of the fused x-y pass: K and M along x (d = 0) and y (d = 1), [P + 1][P + 1]
template <typename Real, int P>
struct XYTab {
  Real k[2][P + 1][P + 1], m[2][P + 1][P + 1];
};

// Tile of the fused x-y pass: whole elements, about 32 x 16 nodes
template <int P>
struct XYTile {
  static constexpr int NEX = (32 + P - 1) / P, NEY = (16 + P - 1) / P;   // elements per tile row / column
  static constexpr int TX = NEX * P, TY = NEY * P;
  static constexpr int UY = TY + P + 1;                                     // t rows: y0 - P .. y0 + TY
  static constexpr int THREADS = 128;
};

// The x and y passes of one z plane, fused: over a tile of whole elements,
//   s1 = My Mx u,  s2 = Ky Mx u + My Kx u      (u = dinv in if dinv is given, else in)
// One thread per (row, element) of the tile takes the element's P + 1 nodes and the left
// element's P nodes straight from memory (the neighbouring threads' loads hit L1), and
// writes t1 = Mx u and t2 = Kx u of the element's P nodes (a vertex sums its two elements'
// rows) for the rows y0 - P .. y0 + TY into shared memory; then one thread per (column,
// element) does the same along y from shared memory and writes s1 and s2.  Each staged value
// is read about twice instead of once per tap.  Grid (x-y tiles, Gz, nvec).
template <typename Real, int P>
__global__ void __launch_bounds__(XYTile<P>::THREADS) fm_xy_kernel(const XYTab<Real, P> tab, int Gx, int Gy,
                                                                   const Real* __restrict__ in, int64_t ldin,
                                                                   const Real* __restrict__ dinv,
                                                                   Real* __restrict__ s1, Real* __restrict__ s2,
                                                                   int64_t lds) {
  using T = XYTile<P>;
  using V4 = R4<Real>;
  constexpr int TX = T::TX, UY = T::UY, NP = P + 1;
  extern __shared__ __align__(16) unsigned char fm_xy_smem[];
  V4* T1 = reinterpret_cast<V4*>(fm_xy_smem);   // [UY][TX]
  V4* T2 = T1 + UY * TX;
  XYTab<Real, P>* tb = reinterpret_cast<XYTab<Real, P>*>(T2 + UY * TX);
  const int tid = threadIdx.x, nt = T::THREADS;
  const int ntx = (Gx + TX - 1) / TX;
  const int x0 = (blockIdx.x % ntx) * TX, y0 = (blockIdx.x / ntx) * T::TY;
  const int z = blockIdx.y, v = blockIdx.z;
  const int64_t plane = int64_t(Gx) * Gy, zoff = int64_t(z) * plane;
  for (int i = tid; i < int(sizeof(XYTab<Real, P>) / sizeof(Real)); i += nt)
    reinterpret_cast<Real*>(tb)[i] = reinterpret_cast<const Real*>(&tab)[i];
  __syncthreads();
  const V4* src = reinterpret_cast<const V4*>(in + 2 * int64_t(v) * ldin) + zoff;
  // x: item (r, ei): row y = y0 - P + r, element ei of the tile (nodes x0 + ei P .. + P - 1)
  for (int t = tid; t < UY * T::NEX; t += nt) {
    const int r = t / T::NEX, ei = t - r * T::NEX;
    const int xe = x0 + ei * P;
    if (xe >= Gx) continue;
    int yy = (y0 - P + r) % Gy;
    if (yy < 0) yy += Gy;
    const int64_t row = int64_t(Gx) * yy;
    V4 u[2 * P + 1];   // x = xe - P .. xe + P
#pragma unroll
    for (int q = 0; q <= 2 * P; ++q) {
      int xx = (xe - P + q) % Gx;
      if (xx < 0) xx += Gx;
      u[q] = ldg4(src + row + xx);
      if (dinv) {
        const Real d = dinv[zoff + row + xx];
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) u[q].v[c4] *= d;
      }
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
      V4 m1 = zero4<Real>(), k1 = zero4<Real>();
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        fma4(m1, tb->m[0][a][q], u[P + q]);
        fma4(k1, tb->k[0][a][q], u[P + q]);
      }
      if (a == 0) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          fma4(m1, tb->m[0][P][q], u[q]);
          fma4(k1, tb->k[0][P][q], u[q]);
        }
      }
      T1[r * TX + ei * P + a] = m1;
      T2[r * TX + ei * P + a] = k1;
    }
  }
  __syncthreads();
  // y: item (cx, ej): column x0 + cx, element ej of the tile (rows y0 + ej P .. + P - 1)
  for (int t = tid; t < TX * T::NEY; t += nt) {
    const int ej = t / TX, cx = t - ej * TX;
    const int gx = x0 + cx, ye = y0 + ej * P;
    if (gx >= Gx || ye >= Gy) continue;
    V4 t1[2 * P + 1], t2[2 * P + 1];   // staged rows ej P .. ej P + 2 P (y = ye - P .. ye + P)
#pragma unroll
    for (int q = 0; q <= 2 * P; ++q) {
      t1[q] = T1[(ej * P + q) * TX + cx];
      t2[q] = T2[(ej * P + q) * TX + cx];
    }
#pragma unroll
    for (int b = 0; b < P; ++b) {
      V4 o1 = zero4<Real>(), o2 = zero4<Real>();
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const Real my = tb->m[1][b][q];
        fma4(o1, my, t1[P + q]);
        fma4(o2, tb->k[1][b][q], t1[P + q]);
        fma4(o2, my, t2[P + q]);
      }
      if (b == 0) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const Real my = tb->m[1][P][q];
          fma4(o1, my, t1[q]);
          fma4(o2, tb->k[1][P][q], t1[q]);
          fma4(o2, my, t2[q]);
        }
      }
      const int64_t I = zoff + gx + int64_t(Gx) * (ye + b);
      st4(reinterpret_cast<V4*>(s1 + 2 * int64_t(v) * lds) + I, o1);
      if (s2) st4(reinterpret_cast<V4*>(s2 + 2 * int64_t(v) * lds) + I, o2);
    }
  }
}

// z-direction element matrices of the fused z pass: K and M, element-local [P + 1][P + 1]
template <typename Real, int P>
struct ZTab {
  Real k[P + 1][P + 1], m[P + 1][P + 1];
};

// The z pass fused with the potential's node gather and the recurrence combination.  One
// thread per (x, y) column of one vector marches through the z planes as the lumped step
// kernel does: input plane c of element ez adds K[cc][c] s1 + M[cc][c] s2 to the element's
// outputs cc (registers), and the element's P planes are written when its closing vertex
// plane arrives, each as
//   T = K u (the z pass) + the per-cell potential terms E of the up to 8 cells of the node
//   mode 3 (H D^-1): out = A T + B in + C prev + g[v] rv
//   mode 2 (D^-1 H): out = A dinv T + B in + C prev + g[v] rv
// (in, prev, rv, E may be null; rv_bfp: R read from its 12-bit BFP stream instead of rv,
// block v nnodes + node).  Grid (ceil(Gx Gy / 128), nvec).
template <typename Real, int P>
__global__ void __launch_bounds__(128) fm_z_kernel(const ZTab<Real, P> zt, int Gx, int Gy, int Gz,
                                                   const Real* __restrict__ s1, const Real* __restrict__ s2,
                                                   int64_t lds, const Real* __restrict__ E, int mode, Real A,
                                                   Real B, const Real* __restrict__ in, int64_t ldin, Real C,
                                                   const Real* prev, int64_t ldprev, const double* __restrict__ g,
                                                   const Real* __restrict__ rv, int64_t ldrv,
                                                   const unsigned char* __restrict__ rv_bfp,
                                                   const Real* __restrict__ dinv, Real* out, int64_t ldout) {
  using V4 = R4<Real>;
  const int64_t plane = int64_t(Gx) * Gy;
  const int64_t col = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (col >= plane) return;
  const int i = int(col % Gx), j = int(col / Gx);
  const int nx = Gx / P, ny = Gy / P, nzc = Gz / P;
  constexpr int NL = (P + 1) * (P + 1) * (P + 1);
  const V4* S1 = reinterpret_cast<const V4*>(s1 + 2 * int64_t(v) * lds) + col;
  const V4* S2 = reinterpret_cast<const V4*>(s2 + 2 * int64_t(v) * lds) + col;
  const V4* Ev = E ? reinterpret_cast<const V4*>(E) + int64_t(v) * nx * ny * nzc * NL : nullptr;
  const Real gv = ((rv || rv_bfp) && g) ? Real(g[v]) : Real(0);
  // x and y cells of this column: (cell, local) pairs, two at an element vertex
  int cxe[2], cxl[2], cye[2], cyl[2];
  const int ax = i % P, ay = j % P;
  cxe[0] = i / P; cxl[0] = ax; cxe[1] = (i / P + nx - 1) % nx; cxl[1] = P;
  cye[0] = j / P; cyl[0] = ay; cye[1] = (j / P + ny - 1) % ny; cyl[1] = P;
  const int ncx = ax == 0 ? 2 : 1, ncy = ay == 0 ? 2 : 1;

  V4 acc[P];
  auto emit = [&](int ez) {
#pragma unroll
    for (int cc = 0; cc < P; ++cc) {
      const int k = ez * P + cc;
      const int64_t I = col + int64_t(k) * plane;
      V4 t = acc[cc];
      if (Ev) {
        for (int zc = 0; zc < (cc == 0 ? 2 : 1); ++zc) {
          const int ez2 = zc == 0 ? ez : (ez + nzc - 1) % nzc, lz = zc == 0 ? cc : P;
          for (int yc = 0; yc < ncy; ++yc)
            for (int xc = 0; xc < ncx; ++xc) {
              const int64_t e = cxe[xc] + int64_t(nx) * (cye[yc] + int64_t(ny) * ez2);
              const V4 w = ldg4(Ev + e * NL + cxl[xc] + (P + 1) * (cyl[yc] + (P + 1) * lz));
#pragma unroll
              for (int c4 = 0; c4 < 4; ++c4) t.v[c4] += w.v[c4];
            }
        }
      }
      const Real a = mode == 2 ? A * dinv[I] : A;
      V4 o = zero4<Real>();
      fma4(o, a, t);
      if (in && B != Real(0)) fma4(o, B, ldg4(reinterpret_cast<const V4*>(in + 2 * int64_t(v) * ldin) + I));
      if (prev) fma4(o, C, ld4(reinterpret_cast<const V4*>(prev + 2 * int64_t(v) * ldprev) + I));
      if (rv_bfp && g) {
        if constexpr (std::is_same<Real, float>::value) {
          uint32_t w, h;
          const int64_t b = int64_t(v) * plane * Gz + I;
          bfp12_fetch(rv_bfp, b, w, h);
          V4 r;
          bfp12_decode(bfp12_join(int(b & 1), w, h), r.v);
          fma4(o, gv, r);
        }
      } else if (rv && g) {
        fma4(o, gv, ldg4(reinterpret_cast<const V4*>(rv + 2 * int64_t(v) * ldrv) + I));
      }
      st4(reinterpret_cast<V4*>(out + 2 * int64_t(v) * ldout) + I, o);
    }
  };
  auto contrib = [&](V4& dst, int row, int c, const V4& a1, const V4& a2) {
    fma4(dst, zt.k[row][c], a1);
    fma4(dst, zt.m[row][c], a2);
  };
  // element -1 (planes Gz - P .. Gz - 1) adds row P of its matrices to the vertex plane 0
  V4 accn = zero4<Real>();
#pragma unroll
  for (int c = 0; c < P; ++c) {
    const int64_t o = int64_t(Gz - P + c) * plane;
    contrib(accn, P, c, ldg4(S1 + o), ldg4(S2 + o));
  }
  V4 n1 = ldg4(S1), n2 = ldg4(S2);   // the next plane, one ahead
  for (int ez = 0; ez < nzc; ++ez) {
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const int z = ez * P + c;
      const V4 a1 = n1, a2 = n2;
      if (z + 1 < Gz) {
        n1 = ldg4(S1 + int64_t(z + 1) * plane);
        n2 = ldg4(S2 + int64_t(z + 1) * plane);
      }
      if (c == 0) {
        contrib(accn, P, P, a1, a2);
        if (ez > 0) {
#pragma unroll
          for (int cc = 0; cc < P; ++cc) contrib(acc[cc], cc, P, a1, a2);
          emit(ez - 1);
        }
        acc[0] = accn;
#pragma unroll
        for (int cc = 1; cc < P; ++cc) acc[cc] = zero4<Real>();
#pragma unroll
        for (int cc = 0; cc < P; ++cc) contrib(acc[cc], cc, 0, a1, a2);
        accn = zero4<Real>();
        contrib(accn, P, 0, a1, a2);
      } else {
#pragma unroll
        for (int cc = 0; cc < P; ++cc) contrib(acc[cc], cc, c, a1, a2);
        contrib(accn, P, c, a1, a2);
      }
    }
  }
  // the last element closes on plane Gz = 0 (periodic)
  {
    const V4 a1 = ldg4(S1), a2 = ldg4(S2);
#pragma unroll
    for (int cc = 0; cc < P; ++cc) contrib(acc[cc], cc, P, a1, a2);
  }
  emit(nzc - 1);
}

// T[I] += sum over the cells e containing node I of E[v][e][local index of I in e]
template <typename Real>
__global__ void fm_gather_kernel(int p, int nx, int ny, int nz, int64_t ncells, const Real* __restrict__ E,
                                 Real* __restrict__ T, int64_t ldt) {
  const int Gx = nx * p, Gy = ny * p, Gz = nz * p;
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (I >= int64_t(Gx) * Gy * Gz) return;
  const int i = int(I % Gx), j = int((I / Gx) % Gy), k = int(I / (int64_t(Gx) * Gy));
  const int np = p + 1;
  // per direction: (cell, local) pairs; a vertex belongs to the element on each side
  int ce[3][2], cl[3][2], cn[3];
  const int idx[3] = {i, j, k}, nc[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d) {
    const int a = idx[d] % p, el = idx[d] / p;
    ce[d][0] = el;
    cl[d][0] = a;
    cn[d] = 1;
    if (a == 0) {
      ce[d][1] = (el + nc[d] - 1) % nc[d];
      cl[d][1] = p;
      cn[d] = 2;
    }
  }
  const R4<Real>* Ev = reinterpret_cast<const R4<Real>*>(E) + int64_t(v) * ncells * (np * np * np);
  R4<Real> s = ld4(reinterpret_cast<const R4<Real>*>(T + 2 * int64_t(v) * ldt) + I);
  for (int z = 0; z < cn[2]; ++z)
    for (int y = 0; y < cn[1]; ++y)
      for (int x = 0; x < cn[0]; ++x) {
        const int64_t e = ce[0][x] + int64_t(nx) * (ce[1][y] + int64_t(ny) * ce[2][z]);
        const int l = cl[0][x] + np * (cl[1][y] + np * cl[2][z]);
        const R4<Real> w = Ev[e * (np * np * np) + l];
#pragma unroll
        for (int c = 0; c < 4; ++c) s.v[c] += w.v[c];
      }
  st_node(T, ldt, v, I, s);
}

// elementwise combinations on node tuples (complex rows r < rows, vector v):
//   mode 0: out = B in + C prev + g[v] rv                 (the argument of M in form H)
//   mode 1: out = A T + W                                  (form H, W = M (B in + ...))
//   mode 2: out = A dinv T + B in + C prev + g[v] rv       (form D^-1 H)
//   mode 3: out = A T + B in + C prev + g[v] rv            (form H D^-1)
//   mode 4: out = dinv in                                  (the scaled input of H D^-1)
template <typename Real>
__global__ void fm_combine_kernel(int mode, int64_t nodes, Real A, const Real* __restrict__ T, int64_t ldt,
                                  const Real* __restrict__ W, int64_t ldw, Real B, const Real* in, int64_t ldin,
                                  Real C, const Real* prev, int64_t ldprev, const double* __restrict__ g,
                                  const Real* rv, int64_t ldrv, const double* __restrict__ dinv, Real* out,
                                  int64_t ldout) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (I >= nodes) return;
  auto at = [&](const Real* b, int64_t ld) {
    return ld4(reinterpret_cast<const R4<Real>*>(b + 2 * int64_t(v) * ld) + I);
  };
  R4<Real> o = zero4<Real>();
  if (mode == 4) {
    fma4(o, Real(dinv[I]), at(in, ldin));
  } else {
    if (mode == 1 || mode == 2 || mode == 3) fma4(o, mode == 2 ? Real(A * dinv[I]) : A, at(T, ldt));
    if (mode == 1) {
      const R4<Real> w = at(W, ldw);
#pragma unroll
      for (int c = 0; c < 4; ++c) o.v[c] += w.v[c];
    } else {
      if (in && B != Real(0)) fma4(o, B, at(in, ldin));
      if (prev) fma4(o, C, at(prev, ldprev));
      if (rv && g) fma4(o, Real(g[v]), at(rv, ldrv));
    }
  }
  st4(reinterpret_cast<R4<Real>*>(out + 2 * int64_t(v) * ldout) + I, o);
}

}  // namespace
}  // namespace rcf

namespace rcf {
namespace {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre polynomial from the
// Chebyshev guess; the standard construction, e.g. Numerical Recipes' gauleg)
void gauss_legendre(int n, std::vector<double>* x, std::vector<double>* w) {
  x->assign(n, 0.0);
  w->assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), pp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double z1 = z;
      z = z1 - p1 / pp;
      if (std::fabs(z - z1) < 1e-16) break;
    }
    (*x)[i] = -z;
    (*x)[n - 1 - i] = z;
    (*w)[i] = (*w)[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

// Lagrange basis l_a on the nodes xi at the point t (product formula)
double lagrange(const std::vector<double>& xi, int a, double t) {
  double v = 1.0;
  for (size_t b = 0; b < xi.size(); ++b)
    if (int(b) != a) v *= (t - xi[b]) / (xi[a] - xi[b]);
  return v;
}

template <typename T>
int upload_vec(rcf_ctx* ctx, T** dst, const std::vector<T>& v) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (v.empty()) return RCF_OK;
  RCF_CUDA(ctx, cudaMalloc(dst, sizeof(T) * v.size()));
  RCF_CUDA(ctx, cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return RCF_OK;
}

template <typename Real>
const Real* fm_tab(const FullMass* fm);
template <>
const double* fm_tab<double>(const FullMass* fm) { return fm->d_tab64; }
template <>
const float* fm_tab<float>(const FullMass* fm) { return fm->d_tab32; }
template <typename Real>
const Real* fm_b1(const FullMass* fm);
template <>
const double* fm_b1<double>(const FullMass* fm) { return fm->d_B1_64; }
template <>
const float* fm_b1<float>(const FullMass* fm) { return fm->d_B1_32; }
template <typename Real>
const Real* fm_vq(const FullMass* fm);
template <>
const double* fm_vq<double>(const FullMass* fm) { return fm->d_vq64; }
template <>
const float* fm_vq<float>(const FullMass* fm) { return fm->d_vq32; }

// table of kind (0 = K, 1 = M) and direction d: [p][2p + 1]
template <typename Real>
const Real* table(const rcf_op* op, int kind, int d) {
  const int p = op->mesh->p;
  return fm_tab<Real>(op->fm) + (size_t(kind) * 3 + d) * size_t(p) * (2 * p + 1);
}

template <typename Real>
int pass(rcf_ctx* ctx, const rcf_op* op, int d, const Real* c1, const Real* c2, const Real* c3, const Real* c4,
         const Real* in1, const Real* in2, int64_t ldin, Real* out1, Real* out2, int64_t ldout, int nvec) {
  const rcf_mesh* m = op->mesh;
  fm_pass_kernel<Real><<<dim3(unsigned((m->nnodes + 255) / 256), nvec), 256, 0, ctx->stream>>>(
      d, m->p, m->G[0], m->G[1], m->G[2], c1, c2, c3, c4, in1, in2, ldin, out1, out2, ldout);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

template <typename Real>
int combine(rcf_ctx* ctx, const rcf_op* op, int mode, int nvec, Real A, const Real* T, int64_t ldt,
            const Real* W, int64_t ldw, Real B, const Real* in, int64_t ldin, Real C, const Real* prev,
            int64_t ldprev, const double* g, const Real* rv, int64_t ldrv, Real* out, int64_t ldout) {
  const rcf_mesh* m = op->mesh;
  fm_combine_kernel<Real><<<dim3(unsigned((m->nnodes + 255) / 256), nvec), 256, 0, ctx->stream>>>(
      mode, m->nnodes, A, T, ldt, W, ldw, B, in, ldin, C, prev, ldprev, g, rv, ldrv, m->d_inv_mass64, out, ldout);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

template <typename Real>
int ws_block(rcf_ctx* ctx, int slot, const rcf_op* op, int nvec, Real** p) {
  return workspace(ctx, slot, sizeof(Real) * 4 * size_t(op->mesh->nnodes) * nvec, reinterpret_cast<void**>(p));
}

// 1 / M_I in the arithmetic type (the FP32 copy is the rounding of the FP64 one)
template <typename Real>
const Real* inv_mass_of(const rcf_mesh* m);
template <>
const double* inv_mass_of<double>(const rcf_mesh* m) { return m->d_inv_mass64; }
template <>
const float* inv_mass_of<float>(const rcf_mesh* m) { return m->d_inv_mass32; }

// the per-cell Gauss-point potential for degree P: E (cell buffer, [nvec][cells][(P+1)^3]
// tuples) from in (times dinv if given); vectors per block from the shared memory they need
template <typename Real, int P>
int launch_fm_cell_p(rcf_ctx* ctx, const rcf_op* op, const Real* in, int64_t ldin, const Real* dinv, Real* E,
                     int nvec) {
  const rcf_mesh* m = op->mesh;
  const FullMass* fm = op->fm;
  constexpr int NP = P + 1;
  const int nq = fm->nq;
  const int SB = std::max(nq * NP * NP, nq * nq * NP);
  const size_t per_vec = 2 * size_t(SB) * sizeof(R4<Real>);
  // vectors per block: every phase's lines (at most max(NP^2, nq NP, nq^2) per vector) in one
  // pass of the 256 threads, within ~96 KB of shared memory
  const int lines = std::max({NP * NP, nq * NP, nq * nq});
  const int NVB = int(std::max<size_t>(
      1, std::min<size_t>({8, size_t(256 / lines), size_t(96 * 1024) / per_vec, size_t(nvec)})));
  const size_t smem = NVB * per_vec + sizeof(R4<Real>) * nq * nq * nq + sizeof(Real) * nq * NP;
  auto kern = fm_cell_kernel<Real, P>;
  if (smem > 48 * 1024) RCF_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  kern<<<dim3(unsigned(m->ncells), unsigned((nvec + NVB - 1) / NVB)), 256, smem, ctx->stream>>>(
      nq, m->n[0], m->n[1], m->n[2], fm_b1<Real>(fm), fm_vq<Real>(fm), in, ldin, dinv, E, nvec, NVB, SB);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}
template <typename Real>
int launch_fm_cell(rcf_ctx* ctx, const rcf_op* op, const Real* in, int64_t ldin, const Real* dinv, Real* E,
                   int nvec) {
  switch (op->mesh->p) {
    case 1: return launch_fm_cell_p<Real, 1>(ctx, op, in, ldin, dinv, E, nvec);
    case 2: return launch_fm_cell_p<Real, 2>(ctx, op, in, ldin, dinv, E, nvec);
    case 3: return launch_fm_cell_p<Real, 3>(ctx, op, in, ldin, dinv, E, nvec);
    case 4: return launch_fm_cell_p<Real, 4>(ctx, op, in, ldin, dinv, E, nvec);
    case 5: return launch_fm_cell_p<Real, 5>(ctx, op, in, ldin, dinv, E, nvec);
    case 6: return launch_fm_cell_p<Real, 6>(ctx, op, in, ldin, dinv, E, nvec);
    case 7: return launch_fm_cell_p<Real, 7>(ctx, op, in, ldin, dinv, E, nvec);
    case 8: return launch_fm_cell_p<Real, 8>(ctx, op, in, ldin, dinv, E, nvec);
    default: return fail(ctx, RCF_ENOTSUP, "degree p=%d not built (1..8)", op->mesh->p);
  }
}

// T = H u (kinetic with the consistent 1D masses, Gauss-point potential, projectors); u, T
// node-tuple blocks with ld = 2M
template <typename Real>
int hamiltonian_fm(rcf_ctx* ctx, const rcf_op* op, const Real* u, int64_t ldu, int nvec, Real* T) {
  const rcf_mesh* m = op->mesh;
  const FullMass* fm = op->fm;
  const int64_t ld = 2 * m->nnodes;
  Real *t1, *t2, *s1, *s2;
  RCF_TRY(ws_block<Real>(ctx, WS_FM_T1, op, nvec, &t1));
  RCF_TRY(ws_block<Real>(ctx, WS_FM_T2, op, nvec, &t2));
  RCF_TRY(ws_block<Real>(ctx, WS_FM_S1, op, nvec, &s1));
  RCF_TRY(ws_block<Real>(ctx, WS_FM_S2, op, nvec, &s2));
  const Real *Kx = table<Real>(op, 0, 0), *Ky = table<Real>(op, 0, 1), *Kz = table<Real>(op, 0, 2);
  const Real *Mx = table<Real>(op, 1, 0), *My = table<Real>(op, 1, 1), *Mz = table<Real>(op, 1, 2);
  RCF_TRY(pass<Real>(ctx, op, 0, Mx, nullptr, Kx, nullptr, u, nullptr, ldu, t1, t2, ld, nvec));
  RCF_TRY(pass<Real>(ctx, op, 1, My, nullptr, Ky, My, t1, t2, ld, s1, s2, ld, nvec));
  RCF_TRY(pass<Real>(ctx, op, 2, Kz, Mz, nullptr, nullptr, s1, s2, ld, T, nullptr, ld, nvec));
  // Gauss-point potential: per-cell contributions, then summed at the nodes
  if (fm_vq<Real>(fm)) {
    const int np = m->p + 1;
    Real* E;
    RCF_TRY(workspace(ctx, WS_FM_CELL, sizeof(Real) * 4 * size_t(m->ncells) * np * np * np * nvec,
                      reinterpret_cast<void**>(&E)));
    RCF_TRY(launch_fm_cell<Real>(ctx, op, u, ldu, nullptr, E, nvec));
    fm_gather_kernel<Real><<<dim3(unsigned((m->nnodes + 255) / 256), nvec), 256, 0, ctx->stream>>>(
        m->p, m->n[0], m->n[1], m->n[2], m->ncells, E, T, ld);
    RCF_CHECK_LAUNCH(ctx);
  }
  // spin-orbit projectors: the columns int N_I beta are stored as beta' = column / D_I, so the
  // lumped operator's kernels with the D weights apply them
  if (op->proj.natoms > 0) {
    const size_t bytes = sizeof(Real) * 24 * size_t(op->proj.natoms) * nvec;
    Real *Cc, *C2;
    RCF_TRY(workspace(ctx, WS_NLC, bytes, reinterpret_cast<void**>(&Cc)));
    RCF_TRY(workspace(ctx, WS_NLC2, bytes, reinterpret_cast<void**>(&C2)));
    RCF_TRY((launch_nl_project<Real, Real>(ctx, op, u, ldu, nvec, 1, Cc)));
    RCF_TRY(launch_nl_delta<Real>(ctx, op, Cc, nvec, Real(1), C2));
    RCF_TRY((launch_nl_addback<Real, Real>(ctx, op, C2, nvec, 1, T, ld)));
  }
  return RCF_OK;
}

}  // namespace

// the fused z pass for degree P
// (mass_only: out = Mz s1, Mz in the slot that multiplies s1 and no second input)
template <typename Real, int P>
int launch_fm_z(rcf_ctx* ctx, const rcf_op* op, const Real* s1, const Real* s2, int64_t lds, const Real* E,
                int mode, const StepArgs<Real, Real>& a, bool mass_only = false) {
  const rcf_mesh* m = op->mesh;
  const int np = P + 1;
  ZTab<Real, P> zt;
  for (int r = 0; r < np; ++r)
    for (int c = 0; c < np; ++c) {
      const Real kz = Real(op->fm->el[size_t(2) * np * np + size_t(r) * np + c]);
      const Real mz = Real(op->fm->el[size_t(5) * np * np + size_t(r) * np + c]);
      zt.k[r][c] = mass_only ? mz : kz;
      zt.m[r][c] = mass_only ? Real(0) : mz;
    }
  if (mass_only) s2 = s1;   // read but multiplied by zero
  const int64_t cols = int64_t(m->G[0]) * m->G[1];
  fm_z_kernel<Real, P><<<dim3(unsigned((cols + 127) / 128), a.nvec), 128, 0, ctx->stream>>>(
      zt, m->G[0], m->G[1], m->G[2], s1, s2, lds, E, mode, a.A, a.B, a.in, a.ld_in, a.C, a.prev, a.ld_prev, a.g,
      a.rv, a.ld_rv, a.rv_bfp, inv_mass_of<Real>(m), a.out, a.ld_out);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

// the fused x-y pass for degree P
template <typename Real, int P>
int launch_fm_xy(rcf_ctx* ctx, const rcf_op* op, const StepArgs<Real, Real>& a, const Real* dinv, Real* s1,
                 Real* s2, int64_t lds) {
  using T = XYTile<P>;
  const rcf_mesh* m = op->mesh;
  constexpr int NP = P + 1;
  XYTab<Real, P> tb;
  for (int d = 0; d < 2; ++d)
    for (int r = 0; r < NP; ++r)
      for (int c = 0; c < NP; ++c) {
        tb.k[d][r][c] = Real(op->fm->el[(size_t(d) * NP + r) * NP + c]);
        tb.m[d][r][c] = Real(op->fm->el[(size_t(3 + d) * NP + r) * NP + c]);
      }
  const size_t smem = 2 * size_t(T::UY) * T::TX * sizeof(R4<Real>) + sizeof(XYTab<Real, P>);
  auto kern = fm_xy_kernel<Real, P>;
  if (smem > 48 * 1024) RCF_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int ntx = (m->G[0] + T::TX - 1) / T::TX, nty = (m->G[1] + T::TY - 1) / T::TY;
  kern<<<dim3(unsigned(ntx * nty), unsigned(m->G[2]), unsigned(a.nvec)), T::THREADS, smem, ctx->stream>>>(
      tb, m->G[0], m->G[1], a.in, a.ld_in, dinv, s1, s2, lds);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

// Forms H D^-1 and D^-1 H of the recurrence step with the full mass, in three launches (plus
// the projectors): the fused x-y pass per plane (s1, s2), the per-cell Gauss-point potential
// (E), and the z pass fused with the node gather of E and the combination.  About 230 B per
// node and vector move through HBM (u read twice, s1 and s2 written and read, E written and
// read, in, Z_{k-1}, R read, out written) against ~390 B for the pass-by-pass form.
template <typename Real>
int apply_fm_fused(rcf_ctx* ctx, const rcf_op* op, int form, const StepArgs<Real, Real>& a) {
  const rcf_mesh* m = op->mesh;
  const FullMass* fm = op->fm;
  const int nvec = a.nvec, p = m->p;
  const int64_t ld = 2 * m->nnodes;
  if (m->G[2] > 65535 || nvec > 65535) return fail(ctx, RCF_ENOTSUP, "grid too large for the fused full-mass pass");
  Real *s1, *s2;
  RCF_TRY(ws_block<Real>(ctx, WS_FM_S1, op, nvec, &s1));
  RCF_TRY(ws_block<Real>(ctx, WS_FM_S2, op, nvec, &s2));
  const Real* dinv = form == RCF_FORM_H_DINV ? inv_mass_of<Real>(m) : nullptr;
  switch (p) {
    case 1: RCF_TRY((launch_fm_xy<Real, 1>(ctx, op, a, dinv, s1, s2, ld))); break;
    case 2: RCF_TRY((launch_fm_xy<Real, 2>(ctx, op, a, dinv, s1, s2, ld))); break;
    case 3: RCF_TRY((launch_fm_xy<Real, 3>(ctx, op, a, dinv, s1, s2, ld))); break;
    case 4: RCF_TRY((launch_fm_xy<Real, 4>(ctx, op, a, dinv, s1, s2, ld))); break;
    case 5: RCF_TRY((launch_fm_xy<Real, 5>(ctx, op, a, dinv, s1, s2, ld))); break;
    case 6: RCF_TRY((launch_fm_xy<Real, 6>(ctx, op, a, dinv, s1, s2, ld))); break;
    case 7: RCF_TRY((launch_fm_xy<Real, 7>(ctx, op, a, dinv, s1, s2, ld))); break;
    case 8: RCF_TRY((launch_fm_xy<Real, 8>(ctx, op, a, dinv, s1, s2, ld))); break;
    default: return fail(ctx, RCF_ENOTSUP, "degree p=%d not built (1..8)", p);
  }
  Real* E = nullptr;
  if (fm_vq<Real>(fm)) {
    const int np = p + 1;
    RCF_TRY(workspace(ctx, WS_FM_CELL, sizeof(Real) * 4 * size_t(m->ncells) * np * np * np * nvec,
                      reinterpret_cast<void**>(&E)));
    RCF_TRY(launch_fm_cell<Real>(ctx, op, a.in, a.ld_in, dinv, E, nvec));
  }
  const int mode = form == RCF_FORM_H_DINV ? 3 : 2;
  switch (p) {
    case 1: RCF_TRY((launch_fm_z<Real, 1>(ctx, op, s1, s2, ld, E, mode, a))); break;
    case 2: RCF_TRY((launch_fm_z<Real, 2>(ctx, op, s1, s2, ld, E, mode, a))); break;
    case 3: RCF_TRY((launch_fm_z<Real, 3>(ctx, op, s1, s2, ld, E, mode, a))); break;
    case 4: RCF_TRY((launch_fm_z<Real, 4>(ctx, op, s1, s2, ld, E, mode, a))); break;
    case 5: RCF_TRY((launch_fm_z<Real, 5>(ctx, op, s1, s2, ld, E, mode, a))); break;
    case 6: RCF_TRY((launch_fm_z<Real, 6>(ctx, op, s1, s2, ld, E, mode, a))); break;
    case 7: RCF_TRY((launch_fm_z<Real, 7>(ctx, op, s1, s2, ld, E, mode, a))); break;
    case 8: RCF_TRY((launch_fm_z<Real, 8>(ctx, op, s1, s2, ld, E, mode, a))); break;
    default: return fail(ctx, RCF_ENOTSUP, "degree p=%d not built (1..8)", p);
  }
  // spin-orbit projectors onto out: the columns are stored as beta' = column / D_I, so the
  // lumped operator's weights give P^H D^-1 in / P^H in and add D P C' / P C' (times A)
  if (op->proj.natoms > 0) {
    const size_t bytes = sizeof(Real) * 24 * size_t(op->proj.natoms) * nvec;
    Real *Cc, *C2;
    RCF_TRY(workspace(ctx, WS_NLC, bytes, reinterpret_cast<void**>(&Cc)));
    RCF_TRY(workspace(ctx, WS_NLC2, bytes, reinterpret_cast<void**>(&C2)));
    RCF_TRY((launch_nl_project<Real, Real>(ctx, op, a.in, a.ld_in, nvec, form == RCF_FORM_DINV_H ? 1 : 0, Cc)));
    RCF_TRY(launch_nl_delta<Real>(ctx, op, Cc, nvec, a.A, C2));
    RCF_TRY((launch_nl_addback<Real, Real>(ctx, op, C2, nvec, form == RCF_FORM_H_DINV ? 1 : 0, a.out, a.ld_out)));
  }
  return RCF_OK;
}

// Y = M X: the x-y kernel's s1 = My Mx X and the z march with Mz (two launches)
template <typename Real>
int mass_apply_fm(rcf_ctx* ctx, const rcf_op* op, const Real* X, int64_t ldx, int nvec, Real* Y, int64_t ldy) {
  const rcf_mesh* m = op->mesh;
  if (nvec == 0) return RCF_OK;
  if (m->G[2] > 65535 || nvec > 65535) return fail(ctx, RCF_ENOTSUP, "grid too large for the fused full-mass pass");
  const int64_t ld = 2 * m->nnodes;
  Real* s1;
  RCF_TRY(ws_block<Real>(ctx, WS_FM_S1, op, nvec, &s1));
  StepArgs<Real, Real> a{};
  a.in = X; a.ld_in = ldx;
  a.out = Y; a.ld_out = ldy;
  a.A = Real(1); a.B = Real(0); a.C = Real(0);
  a.nvec = nvec;
  switch (m->p) {
#define RCF_FM_MASS(P)                                                                     \
    case P:                                                                                \
      RCF_TRY((launch_fm_xy<Real, P>(ctx, op, a, nullptr, s1, nullptr, ld)));              \
      return launch_fm_z<Real, P>(ctx, op, s1, nullptr, ld, nullptr, 3, a, true);
    RCF_FM_MASS(1) RCF_FM_MASS(2) RCF_FM_MASS(3) RCF_FM_MASS(4)
    RCF_FM_MASS(5) RCF_FM_MASS(6) RCF_FM_MASS(7) RCF_FM_MASS(8)
#undef RCF_FM_MASS
    default: return fail(ctx, RCF_ENOTSUP, "degree p=%d not built (1..8)", m->p);
  }
}

template <typename Real>
int apply_full_fm(rcf_ctx* ctx, const rcf_op* op, int form, const StepArgs<Real, Real>& a) {
  const int nvec = a.nvec;
  if (nvec == 0) return RCF_OK;
  if (a.rv_bfp && !std::is_same<Real, float>::value)
    return fail(ctx, RCF_ENOTSUP, "a BFP residual stream needs FP32 storage");
  if (form == RCF_FORM_H_DINV || form == RCF_FORM_DINV_H) return apply_fm_fused<Real>(ctx, op, form, a);
  if (a.rv_bfp) return fail(ctx, RCF_ENOTSUP, "BFP storage of R applies to the recurrence forms only");
  const int64_t ld = 2 * op->mesh->nnodes;
  const Real* u = a.in;
  int64_t ldu = a.ld_in;
  if (form == RCF_FORM_H_DINV) {   // u = D^-1 in
    Real* U;
    RCF_TRY(ws_block<Real>(ctx, WS_FM_U, op, nvec, &U));
    RCF_TRY(combine<Real>(ctx, op, 4, nvec, Real(0), nullptr, 0, nullptr, 0, Real(0), a.in, a.ld_in, Real(0),
                          nullptr, 0, nullptr, nullptr, 0, U, ld));
    u = U;
    ldu = ld;
  }
  Real* T;
  RCF_TRY(ws_block<Real>(ctx, WS_FM_T, op, nvec, &T));
  RCF_TRY(hamiltonian_fm<Real>(ctx, op, u, ldu, nvec, T));
  if (form == RCF_FORM_H) {
    // out = A T + M (B in + C prev + g rv)
    Real *W, *MW;
    RCF_TRY(ws_block<Real>(ctx, WS_FM_W, op, nvec, &W));
    RCF_TRY(ws_block<Real>(ctx, WS_FM_U, op, nvec, &MW));
    RCF_TRY(combine<Real>(ctx, op, 0, nvec, Real(0), nullptr, 0, nullptr, 0, a.B, a.in, a.ld_in, a.C, a.prev,
                          a.ld_prev, a.g, a.rv, a.ld_rv, W, ld));
    RCF_TRY(mass_apply_fm<Real>(ctx, op, W, ld, nvec, MW, ld));
    return combine<Real>(ctx, op, 1, nvec, a.A, T, ld, MW, ld, Real(0), nullptr, 0, Real(0), nullptr, 0, nullptr,
                         nullptr, 0, a.out, a.ld_out);
  }
  return combine<Real>(ctx, op, form == RCF_FORM_DINV_H ? 2 : 3, nvec, a.A, T, ld, nullptr, 0, a.B, a.in, a.ld_in,
                       a.C, a.prev, a.ld_prev, a.g, a.rv, a.ld_rv, a.out, a.ld_out);
}

template int apply_full_fm<double>(rcf_ctx*, const rcf_op*, int, const StepArgs<double, double>&);
template int apply_full_fm<float>(rcf_ctx*, const rcf_op*, int, const StepArgs<float, float>&);
template int mass_apply_fm<double>(rcf_ctx*, const rcf_op*, const double*, int64_t, int, double*, int64_t);
template int mass_apply_fm<float>(rcf_ctx*, const rcf_op*, const float*, int64_t, int, float*, int64_t);

void free_fm(FullMass* fm) {
  if (!fm) return;
  for (void* p : {static_cast<void*>(fm->d_tab64), static_cast<void*>(fm->d_tab32), static_cast<void*>(fm->d_B1_64),
                  static_cast<void*>(fm->d_B1_32), static_cast<void*>(fm->d_vq64), static_cast<void*>(fm->d_vq32)})
    if (p) cudaFree(p);
  delete fm;
}

}  // namespace rcf

namespace rcf {

// V, B at the Gauss points ([ncells][nq^3], [3][ncells][nq^3], host) -> w_q |J| (V, Bx, By, Bz)
int fm_set_potential(rcf_ctx* ctx, rcf_op* op, const double* V, const double* B) {
  FullMass* fm = op->fm;
  const rcf_mesh* m = op->mesh;
  const int nq = fm->nq, nq3 = nq * nq * nq;
  const size_t npt = size_t(m->ncells) * nq3;
  std::vector<double> vq(4 * npt, 0.0);
  for (int64_t e = 0; e < m->ncells; ++e)
    for (int q = 0; q < nq3; ++q) {
      const double wq = fm->gw[q % nq] * fm->gw[(q / nq) % nq] * fm->gw[q / (nq * nq)] * m->detJ;
      const size_t i = size_t(e) * nq3 + q;
      vq[4 * i] = V ? wq * V[i] : 0.0;
      for (int d = 0; d < 3; ++d) vq[4 * i + 1 + d] = B ? wq * B[d * npt + i] : 0.0;
    }
  for (double x : vq)
    if (!std::isfinite(x)) return fail(ctx, RCF_EINVAL, "potential contains a non-finite value");
  std::vector<float> v32(vq.begin(), vq.end());
  RCF_TRY(upload_vec(ctx, &fm->d_vq64, vq));
  RCF_TRY(upload_vec(ctx, &fm->d_vq32, v32));
  return RCF_OK;
}

// Projector columns int N_I beta_{j,i} by the Gauss rule, as (node, atom, beta' = column / D_I)
// entries, nodes ascending per atom (the nodes whose column is not zero)
int fm_projector_entries(rcf_ctx* ctx, const rcf_op* op, int natoms, const double* pos, const double* width,
                         double rcut_factor, std::vector<int>* node, std::vector<int>* atom,
                         std::vector<double>* beta, std::vector<int>* offsets) {
  const FullMass* fm = op->fm;
  const rcf_mesh* m = op->mesh;
  const int p = m->p, np = p + 1, nq = fm->nq, nq3 = nq * nq * nq, nl = np * np * np;
  const double pi = 3.14159265358979323846;
  offsets->assign(natoms + 1, 0);
  std::vector<double> col;
  for (int a = 0; a < natoms; ++a) {
    double Nj[2], s2[2], rj2[2];
    for (int j = 0; j < 2; ++j) {
      const double s = width[2 * a + j];
      if (!(s > 0.0)) return fail(ctx, RCF_EINVAL, "projector width must be > 0");
      Nj[j] = std::sqrt(2.0 / (std::pow(pi, 1.5) * std::pow(s, 5)));
      s2[j] = s * s;
      rj2[j] = (rcut_factor * s) * (rcut_factor * s);
    }
    col.assign(size_t(m->nnodes) * 6, 0.0);
    std::vector<char> touched(m->nnodes, 0);
    for (int64_t e = 0; e < m->ncells; ++e) {
      const int ex = int(e % m->n[0]), ey = int((e / m->n[0]) % m->n[1]), ez = int(e / (int64_t(m->n[0]) * m->n[1]));
      const int ec[3] = {ex, ey, ez};
      for (int q = 0; q < nq3; ++q) {
        const int ql[3] = {q % nq, (q / nq) % nq, q / (nq * nq)};
        double d[3], r2 = 0.0;
        for (int k = 0; k < 3; ++k) {
          const double xk = ec[k] * m->h[k] + (fm->gx[ql[k]] + 1.0) * m->h[k] / 2.0;
          double dd = xk - pos[3 * a + k];
          dd -= m->L[k] * std::nearbyint(dd / m->L[k]);
          d[k] = dd;
          r2 += dd * dd;
        }
        double g[2];
        bool any = false;
        for (int j = 0; j < 2; ++j) {
          g[j] = r2 < rj2[j] ? Nj[j] * std::exp(-r2 / (2.0 * s2[j])) : 0.0;
          any = any || g[j] != 0.0;
        }
        if (!any) continue;
        const double wq = fm->gw[ql[0]] * fm->gw[ql[1]] * fm->gw[ql[2]] * m->detJ;
        for (int l = 0; l < nl; ++l) {
          const int la = l % np, lb = (l / np) % np, lc = l / (np * np);
          const double N = fm->B1[ql[0] * np + la] * fm->B1[ql[1] * np + lb] * fm->B1[ql[2] * np + lc];
          const int64_t I = (ex * p + la) % m->G[0] +
                            int64_t(m->G[0]) * ((ey * p + lb) % m->G[1] + int64_t(m->G[1]) * ((ez * p + lc) % m->G[2]));
          touched[I] = 1;
          for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 3; ++i) col[size_t(I) * 6 + 3 * j + i] += wq * N * g[j] * d[i];
        }
      }
    }
    for (int64_t I = 0; I < m->nnodes; ++I) {
      if (!touched[I]) continue;
      bool nz = false;
      for (int c = 0; c < 6; ++c) nz = nz || col[size_t(I) * 6 + c] != 0.0;
      if (!nz) continue;
      node->push_back(int(I));
      atom->push_back(a);
      for (int c = 0; c < 6; ++c) beta->push_back(col[size_t(I) * 6 + c] / m->mass[I]);
    }
    (*offsets)[a + 1] = int(node->size());
  }
  return RCF_OK;
}

}  // namespace rcf

using namespace rcf;

extern "C" int rcf_op_set_gauss(rcf_op* op, int nq) {
  if (!op) return RCF_EINVAL;
  rcf_ctx* ctx = op->ctx;
  const rcf_mesh* m = op->mesh;
  const int p = m->p, np = p + 1;
  if (nq < p + 1 || nq > 12) return fail(ctx, RCF_EINVAL, "nq must be in [p + 1, 12] (got %d for p = %d)", nq, p);
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  FullMass* fm = new FullMass();
  fm->nq = nq;
  gauss_legendre(nq, &fm->gx, &fm->gw);
  fm->B1.resize(size_t(nq) * np);
  for (int q = 0; q < nq; ++q)
    for (int a = 0; a < np; ++a) fm->B1[size_t(q) * np + a] = lagrange(m->xi, a, fm->gx[q]);
  // element matrices on [-1, 1]: stiffness (exact with the GLL rule), mass (Gauss rule)
  std::vector<double> M1(size_t(np) * np, 0.0);
  for (int a = 0; a < np; ++a)
    for (int b = 0; b < np; ++b)
      for (int q = 0; q < nq; ++q) M1[size_t(a) * np + b] += fm->gw[q] * fm->B1[size_t(q) * np + a] * fm->B1[size_t(q) * np + b];
  const int W = 2 * p + 1;
  fm->tab.assign(size_t(2) * 3 * p * W, 0.0);
  for (int kind = 0; kind < 2; ++kind)
    for (int d = 0; d < 3; ++d) {
      const double sc = kind == 0 ? 0.5 * 2.0 / m->h[d] : m->h[d] / 2.0;
      const double* E = kind == 0 ? m->K1.data() : M1.data();
      double* T = fm->tab.data() + (size_t(kind) * 3 + d) * p * W;
      for (int a = 0; a < p; ++a)
        for (int q = 0; q <= p; ++q) {
          if (a == 0) {
            T[q] += sc * E[size_t(p) * np + q];            // element on the left: local p, offset q - p
            T[p + q] += sc * E[q];                         // element on the right: local 0, offset q
          } else {
            T[size_t(a) * W + q - a + p] += sc * E[size_t(a) * np + q];
          }
        }
    }
  fm->el.assign(size_t(6) * np * np, 0.0);
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < np * np; ++a) {
      fm->el[size_t(d) * np * np + a] = 0.5 * 2.0 / m->h[d] * m->K1[a];
      fm->el[size_t(3 + d) * np * np + a] = m->h[d] / 2.0 * M1[a];
    }
  std::vector<float> t32(fm->tab.begin(), fm->tab.end()), b32(fm->B1.begin(), fm->B1.end());
  int st = upload_vec(ctx, &fm->d_tab64, fm->tab);
  if (st == RCF_OK) st = upload_vec(ctx, &fm->d_tab32, t32);
  if (st == RCF_OK) st = upload_vec(ctx, &fm->d_B1_64, fm->B1);
  if (st == RCF_OK) st = upload_vec(ctx, &fm->d_B1_32, b32);
  if (st != RCF_OK) {
    free_fm(fm);
    return st;
  }
  free_fm(op->fm);
  op->fm = fm;
  return RCF_OK;
}

extern "C" int rcf_op_gauss_points(const rcf_op* op, double* out) {
  if (!op || !out) return RCF_EINVAL;
  if (!op->fm) return fail(op->ctx, RCF_EINVAL, "the operator has no Gauss quadrature (rcf_op_set_gauss)");
  const rcf_mesh* m = op->mesh;
  const int nq = op->fm->nq, nq3 = nq * nq * nq;
  for (int64_t e = 0; e < m->ncells; ++e) {
    const int ec[3] = {int(e % m->n[0]), int((e / m->n[0]) % m->n[1]), int(e / (int64_t(m->n[0]) * m->n[1]))};
    for (int q = 0; q < nq3; ++q) {
      const int ql[3] = {q % nq, (q / nq) % nq, q / (nq * nq)};
      for (int d = 0; d < 3; ++d)
        out[(size_t(e) * nq3 + q) * 3 + d] = ec[d] * m->h[d] + (op->fm->gx[ql[d]] + 1.0) * m->h[d] / 2.0;
    }
  }
  return RCF_OK;
}

extern "C" int rcf_mass_apply(rcf_ctx* ctx, const rcf_op* op, const void* X, int64_t ldx, int nvec, void* Y,
                              int64_t ldy, int prec) {
  if (!ctx || !op) return RCF_EINVAL;
  if (prec != RCF_FP64 && prec != RCF_FP32) return fail(ctx, RCF_EINVAL, "unknown precision %d", prec);
  const int64_t rows = 2 * op->mesh->nnodes;
  const size_t real = prec == RCF_FP64 ? 8 : 4;
  if (nvec < 0) return fail(ctx, RCF_EINVAL, "nvec < 0");
  if (nvec == 0) return RCF_OK;
  if (!X || !Y || ldx < rows || ldy < rows || (ldx & 1) || (ldy & 1) ||
      (reinterpret_cast<uintptr_t>(X) % (4 * real)) || (reinterpret_cast<uintptr_t>(Y) % (4 * real)))
    return fail(ctx, RCF_EINVAL, "X or Y: NULL, misaligned, or leading dimension below 2M / odd");
  const char* x0 = static_cast<const char*>(X);
  const char* y0 = static_cast<const char*>(Y);
  if (x0 < y0 + size_t(ldy) * nvec * 2 * real && y0 < x0 + size_t(ldx) * nvec * 2 * real)
    return fail(ctx, RCF_EINVAL, "Y overlaps X");
  if (op->fm) {
    if (prec == RCF_FP64)
      return mass_apply_fm<double>(ctx, op, static_cast<const double*>(X), ldx, nvec, static_cast<double*>(Y), ldy);
    return mass_apply_fm<float>(ctx, op, static_cast<const float*>(X), ldx, nvec, static_cast<float*>(Y), ldy);
  }
  if (prec == RCF_FP64)   // the diagonal mass of the lumped operator
    return launch_scale_mass(ctx, op->mesh, static_cast<const double*>(X), ldx, nvec, 1.0, static_cast<double*>(Y), ldy);
  return fail(ctx, RCF_ENOTSUP, "the diagonal mass is applied in FP64 only");
}

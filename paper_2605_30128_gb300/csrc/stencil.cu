// Matrix-free local Hamiltonian step on the periodic GLL spectral-element mesh.
//
// On a uniform mesh with GLL quadrature collocated at the nodes, the
// assembled kinetic matrix of the cell-level form (Eq. cellHam, stages i-iii
// of Section III-B-3) factors into three 1D banded operators:
//   K = 1/2 (K1g (x) Wg (x) Wg + Wg (x) K1g (x) Wg + Wg (x) Wg (x) K1g),
//   M = Wg (x) Wg (x) Wg,
// so (D^{-1} K u)_{ijk} = sum_d (A_d u)_{along d} with 1D matrices A_d that
// couple only the nodes of one 1D element (two for element vertices).  The
// same holds for K D^{-1}.  This is the same matrix as the cell-assembled one;
// the kernel evaluates it node by node ("owner computes"), so no cell buffer,
// no scatter and no atomics are needed.
//
// Data layout: column-major multivectors; vector v is a 3D field of nodes
// I = x + Gx (y + Gy z), each node a 4-tuple (re_up, im_up, re_dn, im_dn).
// A block owns a TX x TY tile of (x, y) columns of one vector and marches
// through all z planes.  Each plane (tile plus the x/y halo of one element
// width) is staged in shared memory by cp.async through an NST-deep ring
// (NST-1 planes in flight); the tile's own potential, previous iterate and
// residual, which no other thread needs, go straight to registers one plane
// ahead.  4-wide FP32 updates use packed FFMA2.  The z direction is
// accumulated incrementally: when plane c of a 1D element arrives, its
// contribution A Cz[cc][c] u_c is added to all P outputs of the element, and
// the element's P planes are written when its closing vertex plane arrives.
// Every input element is read from L2/HBM once per plane visit; outputs are
// written once.
#include <type_traits>

#include "bfp_common.cuh"
#include "internal.h"
#include "stencil_common.cuh"

namespace rcf {
namespace {

// shared-memory elements of one ring stage: the plane tile with its one-element x/y halo
template <int P, int TX, int TY>
__host__ __device__ constexpr int stage_elems(bool own) {
  return (TX + P + 1) * (TY + P + 1) + (own ? 2 * TX * TY : 0);
}

// OWN: the tile's own Z_{k-1} and R planes travel through the cp.async ring with the
// halo (NST-1 planes ahead) instead of register prefetch one plane ahead.
// ZB: planes consumed per block barrier (1 or 2); NST - ZB planes are in flight.
// St: storage type of the multivectors (arithmetic in Real; a 16-bit St halves the traffic)
// RBF (FP32): the residual term reads R from a 12-bit BFP stream (a.rv_bfp, one block per
// node 4-tuple, 6 bytes instead of 16), decoded in registers
template <typename Real, typename St, int P, int TX, int TY, int NST, bool OWN, int ZB, bool RBF>
__global__ void __launch_bounds__(TX* TY, TileOf<Real, P>::MINB)
    step_kernel(const StepArgs<Real, St> a, const KTab<Real, P> tab, const int Gx, const int Gy,
                const int Gz) {
  // tab holds A * (x, y, z 1D operators); see launch_p.
  constexpr int W = TX + P + 1;        // staged columns: x0 - P .. x0 + TX
  constexpr int H = TY + P + 1;        // staged rows:    y0 - P .. y0 + TY
  constexpr int NT = TX * TY;
  constexpr int HALO = H * W;
  constexpr int KMAX = (HALO + NT - 1) / NT;
  constexpr int STAGE = stage_elems<P, TX, TY>(OWN);
  static_assert(STAGE == HALO + (OWN ? 2 * NT : 0), "one stage: the plane tile with its halo (+ own planes)");
  using V4 = R4<Real>;
  using S4 = R4<St>;
  using CV = Cvt<Real, St>;
  static_assert(!RBF || (std::is_same<Real, float>::value && std::is_same<St, float>::value && !OWN),
                "BFP residual: FP32 storage, own planes through registers");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S4* S = reinterpret_cast<S4*>(smem_raw);                        // [NST][STAGE]
  Real* ST = reinterpret_cast<Real*>(S + NST * STAGE);           // [2][P+1][P+1] x and y tables

  const int tid = threadIdx.x;
  for (int i = tid; i < 2 * (P + 1) * (P + 1); i += NT) ST[i] = (&tab.c[0][0][0])[i];

  // FP64 is bound by the FP64 pipe: threads grouped by node class (tile_position), so that
  // the element-vertex taps are executed by the vertex warps only.  FP32 is latency bound
  // and keeps the row-major order (its rows of consecutive nodes read shared memory
  // without bank conflicts).
  int lx = tid % TX, ly = tid / TX;
  if constexpr (sizeof(Real) == 8) tile_position<P, TX, TY>(tid, lx, ly);
  const int ntx = (Gx + TX - 1) / TX;
  const int x0 = (blockIdx.x % ntx) * TX;
  const int y0 = (blockIdx.x / ntx) * TY;
  const int v = blockIdx.y;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool active = (gx < Gx) && (gy < Gy);
  const int nz = Gz / P;
  const int64_t plane = int64_t(Gx) * Gy;
  const int64_t col = active ? int64_t(gx) + int64_t(Gx) * gy : 0;

  const S4* in = reinterpret_cast<const S4*>(a.in + 2 * int64_t(v) * a.ld_in);
  const S4* prev = a.prev ? reinterpret_cast<const S4*>(a.prev + 2 * int64_t(v) * a.ld_prev) : nullptr;
  const S4* rv = a.rv ? reinterpret_cast<const S4*>(a.rv + 2 * int64_t(v) * a.ld_rv) : nullptr;
  S4* out = reinterpret_cast<S4*>(a.out + 2 * int64_t(v) * a.ld_out);
  const V4* pot = reinterpret_cast<const V4*>(a.pot);

  // this thread's share of the halo plane: shared-memory slot and in-plane offset (periodic wrap)
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

  auto issue_plane = [&](int z, int s) {
    S4* st = S + s * STAGE;
    const S4* src = in + int64_t(z) * plane;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      if (hs[k] >= 0) cp_async_s4(st + hs[k], src + hg[k]);
    if (OWN && active) {
      const int64_t I = col + int64_t(z) * plane;
      if (prev) cp_async_s4(st + HALO + tid, prev + I);
      if (rv) cp_async_s4(st + HALO + NT + tid, rv + I);
    }
    cp_async_commit();
  };
  // this thread's potential, previous iterate and residual of one plane, one plane ahead.
  // prev may alias out: each element is read here before this thread writes it.
  V4 npot = zero4<Real>(), nprev = zero4<Real>(), nrv = zero4<Real>();
  uint32_t nrw = 0, nrh = 0;   // RBF: the raw words of R's block, decoded when consumed
  const int64_t rblk0 = int64_t(v) * plane * Gz + col;   // RBF: block of node (col, z = 0)
  auto fetch_own = [&](int z) {
    if (!active) return;
    const int64_t I = col + int64_t(z) * plane;
    npot = ldg4(pot + I);
    if (!OWN) {
      if (prev) nprev = CV::in(ldgs(prev + I));
      if constexpr (RBF) {
        bfp12_fetch(a.rv_bfp, rblk0 + int64_t(z) * plane, nrw, nrh);
      } else if (rv) {
        nrv = CV::in(ldgs(rv + I));
      }
    }
  };

  // element -1 (planes Gz-P .. Gz-1) contributes row P of its 1D matrix to the vertex plane 0
  V4 accn = zero4<Real>();
  if (active) {
#pragma unroll
    for (int c = 0; c < P; ++c) fma4(accn, tab.c[2][P][c], CV::in(ldgs(in + col + int64_t(Gz - P + c) * plane)));
  }

  static_assert(ZB == 1 || ZB == 2, "one or two planes per barrier");
  static_assert(NST >= 2 * ZB + 1, "ring too shallow");
#pragma unroll
  for (int s = 0; s < NST - ZB; ++s) {
    if (s < Gz) issue_plane(s, s);
    else cp_async_commit();
  }
  int zload = NST - ZB;
  fetch_own(0);

  __syncthreads();  // tables visible
  const int ax = lx % P, by = ly % P;
  Real cx[P + 1], cy[P + 1];
#pragma unroll
  for (int q = 0; q <= P; ++q) {
    cx[q] = ST[(0 * (P + 1) + ax) * (P + 1) + q];
    cy[q] = ST[(1 * (P + 1) + by) * (P + 1) + q];
  }
  const Real* cxv = ST + (0 * (P + 1) + P) * (P + 1);   // vertex rows (left element)
  const Real* cyv = ST + (1 * (P + 1) + P) * (P + 1);
  const Real A = a.A, B = a.B, C = a.C;
  const Real gv = a.g ? Real(a.g[v]) : Real(0);

  V4 acc[P];
  V4 u0 = zero4<Real>();

  auto emit = [&](int ez) {
    if (!active) return;
#pragma unroll
    for (int cc = 0; cc < P; ++cc) {
      const int64_t I = col + int64_t(ez * P + cc) * plane;
      V4 r = acc[cc];
      if (a.scale_out) {
        const Real mI = Real(a.mass[I]);
#pragma unroll
        for (int i = 0; i < 4; ++i) r.v[i] *= mI;
      }
      st4(out + I, CV::out(r));
    }
  };

  for (int ez = 0; ez < nz; ++ez) {
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const int z = ez * P + c;
      if (ZB == 1 || (z & 1) == 0) {
        // planes z .. z + ZB - 1 have landed; the stages of the previous ZB planes are free
        cp_async_wait<NST - 2 * ZB>();
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ZB; ++j) {
          if (zload < Gz) issue_plane(zload, zload % NST);
          else cp_async_commit();
          ++zload;
        }
      }
      const S4* Pl = S + (z % NST) * STAGE;
      const V4 u = CV::in(Pl[(ly + P) * W + lx + P]);
      const V4 cpot = npot;
      const V4 cprev = OWN ? (prev ? CV::in(Pl[HALO + tid]) : zero4<Real>()) : nprev;
      V4 crv = OWN ? (rv ? CV::in(Pl[HALO + NT + tid]) : zero4<Real>()) : nrv;
      const uint32_t crw = nrw, crh = nrh;
      if (z + 1 < Gz) fetch_own(z + 1);
      // x and y terms (tables carry the factor A)
      V4 self = zero4<Real>();
      {
        const S4* row = Pl + (ly + P) * W;
        const int cb = lx - ax + P;
#pragma unroll
        for (int q = 0; q <= P; ++q) fma4(self, cx[q], CV::in(row[cb + q]));
        if (ax == 0) {
#pragma unroll
          for (int q = 0; q <= P; ++q) fma4(self, cxv[q], CV::in(row[cb - P + q]));
        }
        const int rb = ly - by + P;
#pragma unroll
        for (int q = 0; q <= P; ++q) fma4(self, cy[q], CV::in(Pl[(rb + q) * W + lx + P]));
        if (by == 0) {
#pragma unroll
          for (int q = 0; q <= P; ++q) fma4(self, cyv[q], CV::in(Pl[(rb - P + q) * W + lx + P]));
        }
      }
      // A (potential) u + B u + C prev + g rv
      {
        V4 hp = zero4<Real>();
        add_potential(hp, cpot, u);
        fma4(self, A, hp);
        fma4(self, B, u);
        if (prev) fma4(self, C, cprev);
        if constexpr (RBF) {
          float r[4];
          bfp12_decode(bfp12_join(int((rblk0 + int64_t(z) * plane) & 1), crw, crh), r);
#pragma unroll
          for (int i = 0; i < 4; ++i) crv.v[i] = r[i];
        }
        if (RBF || rv) fma4(self, gv, crv);
      }
      if (c == 0) {
        // the vertex plane closes element ez-1 (its local node P) and opens element ez
        fma4(accn, tab.c[2][P][P], u);
        if (ez > 0) {
#pragma unroll
          for (int cc = 0; cc < P; ++cc) fma4(acc[cc], tab.c[2][cc][P], u);
          emit(ez - 1);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[0].v[i] = accn.v[i] + self.v[i];
#pragma unroll
        for (int cc = 1; cc < P; ++cc) acc[cc] = zero4<Real>();
#pragma unroll
        for (int cc = 0; cc < P; ++cc) fma4(acc[cc], tab.c[2][cc][0], u);
        accn = zero4<Real>();
        fma4(accn, tab.c[2][P][0], u);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[c].v[i] += self.v[i];
#pragma unroll
        for (int cc = 0; cc < P; ++cc) fma4(acc[cc], tab.c[2][cc][c], u);
        fma4(accn, tab.c[2][P][c], u);
      }
    }
  }
  // the last element closes on plane Gz = 0 (periodic), read again here rather than kept in
  // registers through the march
  if (active) u0 = CV::in(ldgs(in + col));
#pragma unroll
  for (int cc = 0; cc < P; ++cc) fma4(acc[cc], tab.c[2][cc][P], u0);
  emit(nz - 1);
  cp_async_wait<0>();
}

template <typename Real, typename St, int P>
int launch_p(rcf_ctx* ctx, const rcf_mesh* m, const Tables& t, const StepArgs<Real, St>& a) {
  constexpr int TX = TileOf<Real, P>::TX, TY = TileOf<Real, P>::TY;
  constexpr int NST = TileOf<Real, P>::NST;
  constexpr bool OWN = TileOf<Real, P>::OWN;
  constexpr int ZB = TileOf<Real, P>::ZB;
  // the kernel multiplies the operator by A through its tables
  KTab<Real, P> kt;
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i <= P; ++i)
      for (int j = 0; j <= P; ++j) kt.c[d][i][j] = Real(double(a.A) * t.c[d][i][j]);
  const int ntx = (m->G[0] + TX - 1) / TX, nty = (m->G[1] + TY - 1) / TY;
  const size_t stage = size_t(stage_elems<P, TX, TY>(OWN));
  const size_t smem = size_t(NST) * stage * sizeof(R4<St>) + 2 * (P + 1) * (P + 1) * sizeof(Real);
  auto launch = [&](auto kern) -> int {
    if (smem > 48 * 1024)
      RCF_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    dim3 grid(ntx * nty, a.nvec);
    kern<<<grid, TX * TY, smem, ctx->stream>>>(a, kt, m->G[0], m->G[1], m->G[2]);
    RCF_CHECK_LAUNCH(ctx);
    return RCF_OK;
  };
  if constexpr (std::is_same<Real, float>::value && std::is_same<St, float>::value) {
    if (a.rv_bfp) return launch(step_kernel<Real, St, P, TX, TY, NST, OWN, ZB, true>);
  }
  return launch(step_kernel<Real, St, P, TX, TY, NST, OWN, ZB, false>);
}

}  // namespace

void build_tables(const rcf_mesh* m, int kind, Tables* t) {
  // C_d[a][a'] = 1/2 (2/h_d) K1[a][a'] / Wg(a'') with a'' = a' (column scaled,
  // H D^{-1}) or a'' = a (row scaled, D^{-1} H); Wg = (h/2) w at interior
  // nodes and h w_0 at vertices (two elements meet there).
  const int P = m->p, np = m->np;
  for (int d = 0; d < 3; ++d) {
    const double h = m->h[d];
    for (int i = 0; i <= kMaxP; ++i)
      for (int j = 0; j <= kMaxP; ++j) t->c[d][i][j] = 0.0;
    auto wg = [&](int a) { return (a == 0 || a == P) ? h * m->w[0] : 0.5 * h * m->w[a]; };
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) {
        const double k = 0.5 * (2.0 / h) * m->K1[i * np + j];
        t->c[d][i][j] = k / (kind == TAB_COL_SCALED ? wg(j) : wg(i));
      }
  }
}

template <typename Real, typename St>
int launch_step(rcf_ctx* ctx, const rcf_mesh* m, const Tables& t, const StepArgs<Real, St>& a) {
  if (a.nvec <= 0) return RCF_OK;
  if (a.rv_bfp && !(std::is_same<Real, float>::value && std::is_same<St, float>::value))
    return fail(ctx, RCF_ENOTSUP, "a BFP residual stream needs FP32 storage");
  if constexpr (sizeof(Real) == 4 && sizeof(St) == 4) {
    if (ctx->step_kernel == RCF_STEP_TMA && !a.rv_bfp) {
      bool used = false;
      RCF_TRY(launch_step_tma(ctx, m, t, a, &used));
      if (used) return RCF_OK;
    }
  }
  switch (m->p) {
    case 1: return launch_p<Real, St, 1>(ctx, m, t, a);
    case 2: return launch_p<Real, St, 2>(ctx, m, t, a);
    case 3: return launch_p<Real, St, 3>(ctx, m, t, a);
    case 4: return launch_p<Real, St, 4>(ctx, m, t, a);
    case 5: return launch_p<Real, St, 5>(ctx, m, t, a);
    case 6: return launch_p<Real, St, 6>(ctx, m, t, a);
    case 7: return launch_p<Real, St, 7>(ctx, m, t, a);
    case 8: return launch_p<Real, St, 8>(ctx, m, t, a);
    default: return fail(ctx, RCF_ENOTSUP, "degree p=%d not built (1..8)", m->p);
  }
}

template int launch_step<float, float>(rcf_ctx*, const rcf_mesh*, const Tables&, const StepArgs<float, float>&);
template int launch_step<double, double>(rcf_ctx*, const rcf_mesh*, const Tables&, const StepArgs<double, double>&);
template int launch_step<float, __half>(rcf_ctx*, const rcf_mesh*, const Tables&, const StepArgs<float, __half>&);
template int launch_step<float, __nv_bfloat16>(rcf_ctx*, const rcf_mesh*, const Tables&,
                                               const StepArgs<float, __nv_bfloat16>&);

}  // namespace rcf

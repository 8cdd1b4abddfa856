// FP32 step kernel with Tensor Memory Accelerator (TMA) plane loads and mbarrier
// producer/consumer staging (sm_90+ bulk tensor copies, used here on sm_103a).
//
// Same operation and z-marching organisation as step_kernel in stencil.cu
// (Eq. rChFSIrecurrence / Eq. ChFSIrecurrence on the GLL stencil form of Eq. cellHam),
// but each plane of a TX x TY tile arrives as five TMA boxes issued by one producer
// thread: the owned tile B (TX x TY), the left and right x strips XA (P x TY) and
// XC (1 x TY), and the top and bottom y strips YA (TX x P) and YC (TX x 1).  Each
// strip starts at a periodic-wrapped coordinate and never crosses the domain edge,
// so no ghost layers are needed.  Consumers wait on a "full" mbarrier per ring
// stage and release it per warp on an "empty" mbarrier; there is no block-wide
// barrier per plane, and the copies take no consumer instructions.  Every wait is
// bounded; on time-out the kernel records an error word and returns after its own
// copies have landed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"
#include "stencil_common.cuh"

namespace rcf {
namespace {

// Pipeline waits give up after the context's limit of try_wait polls (rcf_set_wait_limit,
// default 2^24).  The wait for a block's own copies in flight before it exits uses a separate,
// fixed limit, so that a small pipeline limit never lets a block exit with a copy still
// writing to its shared memory.
constexpr long kDrainLimit = 1L << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait; false after `limit` polls (at once for limit 0)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long limit) {
  for (long it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int v,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(z), "r"(v), "r"(bar)
      : "memory");
}

// Tensor maps of one input multivector, one per box shape.
struct Maps {
  CUtensorMap b, xa, xc, ya, yc;
};

// Stage layout (R4<float> elements, each piece 128-byte aligned): B [TY][TX], XA [TY][P],
// XC [TY][1], YA [P][TX], YC [1][TX].
template <int P, int TX, int TY>
struct Stage {
  static constexpr int pad(int n) { return (n + 7) / 8 * 8; }
  static constexpr int B = 0;
  static constexpr int XA = B + pad(TX * TY);
  static constexpr int XC = XA + pad(P * TY);
  static constexpr int YA = XC + pad(TY);
  static constexpr int YC = YA + pad(TX * P);
  static constexpr int SIZE = YC + pad(TX);
  static constexpr uint32_t TX_BYTES = 16u * (TX * TY + P * TY + TY + TX * P + TX);
};

// blocks per SM for a block of consumer warps plus one producer warp at 128 registers
template <int TX, int TY>
constexpr int tma_minb() {
  return 65536 / (((TX * TY + 31) / 32 + 1) * 32 * 128) < 1 ? 1 : 65536 / (((TX * TY + 31) / 32 + 1) * 32 * 128);
}

template <int P, int TX, int TY, int NST>
__global__ void __launch_bounds__((((TX * TY) + 31) / 32 + 1) * 32, tma_minb<TX, TY>())
    step_kernel_tma(const StepArgs<float> a, const KTab<float, P> tab, const __grid_constant__ Maps maps,
                    const int Gx, const int Gy, const int Gz, int* err, const long wait_limit) {
  using V4 = R4<float>;
  using ST_ = Stage<P, TX, TY>;
  constexpr int NT = TX * TY;
  constexpr int NCW = (NT + 31) / 32;   // consumer warps; the last warp is the producer
  extern __shared__ __align__(128) unsigned char smem_raw[];
  V4* S = reinterpret_cast<V4*>(smem_raw);                                   // [NST][SIZE]
  uint64_t* bars = reinterpret_cast<uint64_t*>(S + NST * ST_::SIZE);         // full[NST], empty[NST]
  float* TB = reinterpret_cast<float*>(bars + 2 * NST);                      // [2][P+1][P+1]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(TB + 2 * (P + 1) * (P + 1));

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 2 * (P + 1) * (P + 1); i += blockDim.x) TB[i] = (&tab.c[0][0][0])[i];
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(bars + s), 1);
      mbar_init(smem_u32(bars + NST + s), NCW);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int ntx = Gx / TX;
  const int x0 = (blockIdx.x % ntx) * TX;
  const int y0 = (blockIdx.x / ntx) * TY;
  const int v = blockIdx.y;

  if (warp == NCW) {
    // ---- producer: one lane issues the five boxes of every plane ----
    if (lane == 0) {
      const int xa = (x0 - P + Gx) % Gx, xc = (x0 + TX) % Gx;
      const int ya = (y0 - P + Gy) % Gy, yc = (y0 + TY) % Gy;
      int issued = 0;
      bool ok = true;
      for (int z = 0; z < Gz && ok; ++z) {
        const int s = z % NST, k = z / NST;
        if (k >= 1 && !mbar_wait(smem_u32(bars + NST + s), (k - 1) & 1, wait_limit)) {
          ok = false;
          break;
        }
        if (*abort_flag) { ok = false; break; }
        const uint32_t full = smem_u32(bars + s);
        const uint32_t base = smem_u32(S + s * ST_::SIZE);
        mbar_expect_tx(full, ST_::TX_BYTES);
        tma_load_5d(base + 16 * ST_::B, &maps.b, x0, y0, z, v, full);
        tma_load_5d(base + 16 * ST_::XA, &maps.xa, xa, y0, z, v, full);
        tma_load_5d(base + 16 * ST_::XC, &maps.xc, xc, y0, z, v, full);
        tma_load_5d(base + 16 * ST_::YA, &maps.ya, x0, ya, z, v, full);
        tma_load_5d(base + 16 * ST_::YC, &maps.yc, x0, yc, z, v, full);
        ++issued;
      }
      if (!ok) {
        atomicExch(err, 1);
        *abort_flag = 1;
        // let the copies already issued land before the block's shared memory goes away
        for (int z = (issued > NST ? issued - NST : 0); z < issued; ++z)
          mbar_wait(smem_u32(bars + z % NST), (z / NST) & 1, kDrainLimit);
      }
    }
    return;
  }

  // ---- consumers ----
  const bool real = tid < NT;
  const int lx = real ? tid % TX : 0, ly = real ? tid / TX : 0;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool active = real;   // tiles divide the mesh, so every real thread owns a node
  const int nz = Gz / P;
  const int64_t plane = int64_t(Gx) * Gy;
  const int64_t col = int64_t(gx) + int64_t(Gx) * gy;
  const V4* in = reinterpret_cast<const V4*>(a.in + 2 * int64_t(v) * a.ld_in);
  const V4* prev = a.prev ? reinterpret_cast<const V4*>(a.prev + 2 * int64_t(v) * a.ld_prev) : nullptr;
  const V4* rv = a.rv ? reinterpret_cast<const V4*>(a.rv + 2 * int64_t(v) * a.ld_rv) : nullptr;
  V4* out = reinterpret_cast<V4*>(a.out + 2 * int64_t(v) * a.ld_out);
  const V4* pot = reinterpret_cast<const V4*>(a.pot);

  V4 npot = zero4<float>(), nprev = zero4<float>(), nrv = zero4<float>();
  auto fetch_own = [&](int z) {
    if (!active) return;
    const int64_t I = col + int64_t(z) * plane;
    npot = ldg4(pot + I);
    if (prev) nprev = ldg4(prev + I);
    if (rv) nrv = ldg4(rv + I);
  };
  V4 accn = zero4<float>();
  if (active) {
#pragma unroll
    for (int c = 0; c < P; ++c) fma4(accn, tab.c[2][P][c], ldg4(in + col + int64_t(Gz - P + c) * plane));
  }
  fetch_own(0);

  const int ax = lx % P, by = ly % P;
  const int es = lx - ax, er = ly - by;
  const bool last_x = (es + P == TX), last_y = (er + P == TY);
  float cx[P + 1], cy[P + 1];
#pragma unroll
  for (int q = 0; q <= P; ++q) {
    cx[q] = TB[(0 * (P + 1) + ax) * (P + 1) + q];
    cy[q] = TB[(1 * (P + 1) + by) * (P + 1) + q];
  }
  const float* cxv = TB + (0 * (P + 1) + P) * (P + 1);
  const float* cyv = TB + (1 * (P + 1) + P) * (P + 1);
  const float A = a.A, B = a.B, C = a.C;
  const float gv = a.g ? float(a.g[v]) : 0.f;

  V4 acc[P];
  V4 u0 = zero4<float>();
  auto emit = [&](int ez) {
    if (!active) return;
#pragma unroll
    for (int cc = 0; cc < P; ++cc) {
      const int64_t I = col + int64_t(ez * P + cc) * plane;
      V4 r = acc[cc];
      if (a.scale_out) {
        const float mI = float(a.mass[I]);
#pragma unroll
        for (int i = 0; i < 4; ++i) r.v[i] *= mI;
      }
      st4(out + I, r);
    }
  };

  bool ok = true;
  for (int ez = 0; ez < nz && ok; ++ez) {
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const int z = ez * P + c;
      const int s = z % NST;
      if (!mbar_wait(smem_u32(bars + s), (z / NST) & 1, wait_limit) || *abort_flag) {
        ok = false;
        break;
      }
      const V4* Sb = S + s * ST_::SIZE;
      const V4* Bt = Sb + ST_::B;
      const V4 u = Bt[ly * TX + lx];
      V4 self = zero4<float>();
      {
        // x: right element; its closing vertex is in XC for the tile's last element
        const V4* row = Bt + ly * TX;
#pragma unroll
        for (int q = 0; q < P; ++q) fma4(self, cx[q], row[es + q]);
        fma4(self, cx[P], last_x ? Sb[ST_::XC + ly] : row[es + P]);
        if (ax == 0) {
          if (lx == 0) {
            const V4* xa = Sb + ST_::XA + ly * P;
#pragma unroll
            for (int q = 0; q < P; ++q) fma4(self, cxv[q], xa[q]);
            fma4(self, cxv[P], row[0]);
          } else {
#pragma unroll
            for (int q = 0; q <= P; ++q) fma4(self, cxv[q], row[es - P + q]);
          }
        }
        // y: right element, closing vertex row in YC for the tile's last element
#pragma unroll
        for (int q = 0; q < P; ++q) fma4(self, cy[q], Bt[(er + q) * TX + lx]);
        fma4(self, cy[P], last_y ? Sb[ST_::YC + lx] : Bt[(er + P) * TX + lx]);
        if (by == 0) {
          if (ly == 0) {
            const V4* ya = Sb + ST_::YA;
#pragma unroll
            for (int q = 0; q < P; ++q) fma4(self, cyv[q], ya[q * TX + lx]);
            fma4(self, cyv[P], Bt[lx]);
          } else {
#pragma unroll
            for (int q = 0; q <= P; ++q) fma4(self, cyv[q], Bt[(er - P + q) * TX + lx]);
          }
        }
      }
      // this warp is done with the stage
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(bars + NST + s));

      const V4 cpot = npot, cprev = nprev, crv = nrv;
      if (z + 1 < Gz) fetch_own(z + 1);
      {
        V4 hp = zero4<float>();
        add_potential(hp, cpot, u);
        fma4(self, A, hp);
        fma4(self, B, u);
        if (prev) fma4(self, C, cprev);
        if (rv) fma4(self, gv, crv);
      }
      if (c == 0) {
        fma4(accn, tab.c[2][P][P], u);
        if (ez > 0) {
#pragma unroll
          for (int cc = 0; cc < P; ++cc) fma4(acc[cc], tab.c[2][cc][P], u);
          emit(ez - 1);
        } else {
          u0 = u;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[0].v[i] = accn.v[i] + self.v[i];
#pragma unroll
        for (int cc = 1; cc < P; ++cc) acc[cc] = zero4<float>();
#pragma unroll
        for (int cc = 0; cc < P; ++cc) fma4(acc[cc], tab.c[2][cc][0], u);
        accn = zero4<float>();
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
  if (!ok) {
    if (lane == 0) atomicExch(err, 1);
    *abort_flag = 1;
    return;
  }
#pragma unroll
  for (int cc = 0; cc < P; ++cc) fma4(acc[cc], tab.c[2][cc][P], u0);
  emit(nz - 1);
}

// ---- host side ----

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// map of the 5D view (4 floats, x, y, z, vector) with a (4, bx, by, 1, 1) box
bool encode_map(CUtensorMap* map, const float* base, const rcf_mesh* m, int64_t ld, int nvec, int bx,
                int by) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[5] = {4, cuuint64_t(m->G[0]), cuuint64_t(m->G[1]), cuuint64_t(m->G[2]), cuuint64_t(nvec)};
  const cuuint64_t strides[4] = {16, 16 * cuuint64_t(m->G[0]), 16 * cuuint64_t(m->G[0]) * m->G[1],
                                 8 * cuuint64_t(ld)};
  const cuuint32_t box[5] = {4, cuuint32_t(bx), cuuint32_t(by), 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<float*>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int P>
int launch_tma_p(rcf_ctx* ctx, const rcf_mesh* m, const Tables& t, const StepArgs<float>& a, bool* used) {
  constexpr int TX = TileOf<float, P>::TX, TY = TileOf<float, P>::TY;
  constexpr int NST = 4;
  using ST_ = Stage<P, TX, TY>;
  *used = false;
  if (m->G[0] % TX != 0 || m->G[1] % TY != 0) return RCF_OK;
  if ((reinterpret_cast<uintptr_t>(a.in) & 15) != 0 || (a.ld_in & 1) != 0) return RCF_OK;
  Maps maps;
  if (!encode_map(&maps.b, a.in, m, a.ld_in, a.nvec, TX, TY) ||
      !encode_map(&maps.xa, a.in, m, a.ld_in, a.nvec, P, TY) ||
      !encode_map(&maps.xc, a.in, m, a.ld_in, a.nvec, 1, TY) ||
      !encode_map(&maps.ya, a.in, m, a.ld_in, a.nvec, TX, P) ||
      !encode_map(&maps.yc, a.in, m, a.ld_in, a.nvec, TX, 1))
    return RCF_OK;   // fall back to the cp.async kernel
  KTab<float, P> kt;
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i <= P; ++i)
      for (int j = 0; j <= P; ++j) kt.c[d][i][j] = float(double(a.A) * t.c[d][i][j]);
  const size_t smem = size_t(NST) * ST_::SIZE * sizeof(R4<float>) + 2 * NST * sizeof(uint64_t) +
                      2 * (P + 1) * (P + 1) * sizeof(float) + 16;
  auto kern = step_kernel_tma<P, TX, TY, NST>;
  if (smem > 48 * 1024) RCF_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int threads = ((TX * TY + 31) / 32 + 1) * 32;
  dim3 grid((m->G[0] / TX) * (m->G[1] / TY), a.nvec);
  kern<<<grid, threads, smem, ctx->stream>>>(a, kt, maps, m->G[0], m->G[1], m->G[2], ctx->d_err,
                                             long(ctx->wait_limit));
  RCF_CHECK_LAUNCH(ctx);
  *used = true;
  return RCF_OK;
}

}  // namespace

int launch_step_tma(rcf_ctx* ctx, const rcf_mesh* m, const Tables& t, const StepArgs<float>& a, bool* used) {
  *used = false;
  if (!ctx->d_err) return RCF_OK;
  switch (m->p) {
    case 4: return launch_tma_p<4>(ctx, m, t, a, used);
    case 5: return launch_tma_p<5>(ctx, m, t, a, used);
    case 6: return launch_tma_p<6>(ctx, m, t, a, used);
    default: return RCF_OK;
  }
}

}  // namespace rcf

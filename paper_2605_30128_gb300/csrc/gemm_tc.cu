// FP64-accurate products for Cholesky-QR and Rayleigh-Ritz on the bf16 tensor cores
// (Algorithm 1, RR step; Section III-C-4).
//
// Method: the error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).  Every row a of
// the left operand and every column b of the right one is scaled by a power of two,
// 2^e, with max |x| <= 2^(e-1), and written as T balanced digits of BETA bits,
//     x = 2^e sum_{s=1..T} d_s 2^(-BETA s) + r,   d_s integer, |d_s| <= 2^(BETA-1),
//     |r| <= 2^(e - BETA T - 1),
// each digit exactly representable in bf16 (|d| <= 128).  The product is
//     sum_k a_k b_k = 2^(e_a + e_b) sum_{s + t <= T + 1} 2^(-BETA (s + t)) sum_k d^a_{s,k} d^b_{t,k}
// (the omitted s + t > T + 1 terms are below the truncation r).  Each digit product
// is at most 2^14 in magnitude, so a sum over WIN = 1024 consecutive k is an integer of
// magnitude <= 2^24: the tensor core's FP32 accumulation of such a window is exact.
// Each (window, s, t) accumulator is drained from tensor memory into two 64-bit
// fixed-point sums per output entry, one for the weights w = s + t <= 4 (kept in tensor
// memory) and one for w >= 5 (kept in registers), each with every shift a left shift: the
// digit products are summed exactly, and the only roundings are the digit truncation and
// the final conversion to FP64.
//
// Kernel: one CTA per 128 x 128 output tile and K range, persistent over its
// windows.  Warp 0 issues the TMA loads of the two operand tiles (128 rows x 64 k,
// bf16, 128-byte swizzle) into a 6-stage shared-memory ring; warp 1 (one thread)
// issues tcgen05.mma (M = N = 128, K = 16, FP32 accumulate) into one of two
// 128-column accumulators in tensor memory; warps 4..11 (two warpgroups, given most of
// the registers by setmaxnreg) drain the other accumulator (tcgen05.ld) into the
// fixed-point sums (each warp: 32 rows x 64 columns).  Every wait is bounded; on time-out the CTA records an error
// word, waits (bounded) for its copies and MMAs in flight, frees its tensor memory
// and returns.  All copies use this GPU's own memory; no cluster, no multicast.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"

namespace rcf {
namespace tc {

constexpr int BETA = 8;          // bits per digit
constexpr int T = 7;             // digits per operand entry (56 bits): FP64-accurate products
constexpr int T_LOW = 3;         // 24 bits: the FP32-accurate off-diagonal rotation of Section III-C-4
constexpr int WIN = 1024;        // k per exact FP32 window
constexpr int BK = 64;           // k per staged tile (128 bytes of bf16: one swizzle row)
constexpr int TM = 128, TN = 128;
constexpr int NSTAGE = 6;
constexpr int FIX_HI = 34;       // fixed point of the weights 2..4 (in units of weight-2 products)
constexpr int FIX_LO = 32;       // fixed point of the weights 5..8 (in units of weight-5 products)
constexpr int W_SPLIT = 2;       // w - 2 <= W_SPLIT: the tensor-memory sum
constexpr int LAUNCH_WINDOWS = 8;   // windows per CTA per launch (bounds |F| < 2^63)
constexpr int NTHREADS = 384;    // three warpgroups: producer + MMA (+2 idle warps), two drain groups
// register split (setmaxnreg): launched with 168 per thread (65536 / 384 rounded down to 8);
// warpgroup 0 drops to 40 and the two drain warpgroups rise to 232:
// 128 x 40 + 256 x 232 = 64512 = 384 x 168
constexpr int REG_LAUNCH = 168, REG_LOW = 40, REG_HIGH = 232;
static_assert(128 * REG_LOW + 256 * REG_HIGH <= NTHREADS * REG_LAUNCH, "register split above the launch total");
constexpr int TILE_BYTES = TM * BK * 2;   // 16 KB per operand tile
constexpr unsigned long long WAIT_NS = 2000000000ull;   // every wait gives up after 2 s
constexpr int E_NONFINITE = 1 << 14;   // exponent of a row or column holding an Inf or a NaN

template <int TD>
struct Prod {
  static constexpr int N = TD * (TD + 1) / 2;   // digit products with s + t <= TD + 1
  unsigned char s[N], t[N];
};

// products in slice-major order: the T + 1 - s products of left slice s follow one another,
// so its window tiles are re-read from L2 rather than from HBM
template <int TD>
__host__ __device__ constexpr Prod<TD> make_products() {
  Prod<TD> p{};
  int n = 0;
  for (int s = 1; s <= TD; ++s)
    for (int t = 1; s + t <= TD + 1; ++t) {
      p.s[n] = (unsigned char)(s - 1);
      p.t[n] = (unsigned char)(t - 1);
      ++n;
    }
  return p;
}

__constant__ Prod<T> kProdFull = make_products<T>();
__constant__ Prod<T_LOW> kProdLow = make_products<T_LOW>();
template <int TD>
__device__ __forceinline__ const Prod<TD>& products();
template <>
__device__ __forceinline__ const Prod<T>& products<T>() {
  return kProdFull;
}
template <>
__device__ __forceinline__ const Prod<T_LOW>& products<T_LOW>() {
  return kProdLow;
}

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
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: false after WAIT_NS, or as soon as another role has aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  const unsigned long long t0 = now_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0 && (*abort_flag || now_ns() - t0 > WAIT_NS)) return false;
  }
}
// bounded wait that ignores the abort flag: for copies and MMAs already in flight, which must
// complete before the CTA releases its shared and tensor memory
__device__ __forceinline__ bool mbar_wait_inflight(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0 && now_ns() - t0 > WAIT_NS) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int k, int row, int s,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(k), "r"(row), "r"(s), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major tile of rows x 64 bf16 with the 128-byte swizzle
// (8-row groups 1024 bytes apart), start address advanced by 32 bytes per K = 16 step
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFF);
  d |= uint64_t(1) << 16;                  // leading byte offset (unused with the swizzle)
  d |= uint64_t(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 bytes
  d |= uint64_t(1) << 46;                  // descriptor version
  d |= uint64_t(2) << 61;                  // 128-byte swizzle
  return d;
}
// instruction descriptor: D FP32, A and B bf16, both K-major, M = 128, N = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TN >> 3) << 17) | (uint32_t(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 32 lanes x 32 columns of 32-bit words from / to tensor memory
__device__ __forceinline__ void tmem_ld32u(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32u(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_ld8u(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st8u(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
               ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct GemmArgs {
  int m, n;            // output rows (A rows) and columns (B rows)
  int64_t k0;          // first k of this launch
  int nwin;            // windows (WIN k each, the last one may be shorter) per CTA
  int64_t kend;        // one past the last k of this launch
  const int* ea;       // [m] row exponents of A
  const int* eb;       // [n] row exponents of B
  double* out;         // out[split * ss + row * rs + (col >> 1) * cs2 + (col & 1)] (+)= value
  int64_t ss, rs, cs2;
  int accumulate;      // add to out instead of overwriting
  int lower_n;         // > 0: skip tiles whose column block (mod lower_n) lies above the diagonal
  int* err;
};

template <int TD>
__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                      const GemmArgs g) {
  constexpr int NPROD = Prod<TD>::N;
  const Prod<TD>& kProd = products<TD>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-aligned operand ring, then barriers
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = base;                                   // [NSTAGE][TILE_BYTES]
  unsigned char* sB = base + NSTAGE * TILE_BYTES;             // [NSTAGE][TILE_BYTES]
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * NSTAGE * TILE_BYTES);
  uint64_t* full = bars;                 // [NSTAGE] TMA landed
  uint64_t* empty = bars + NSTAGE;       // [NSTAGE] MMAs done with the stage
  uint64_t* acc_full = bars + 2 * NSTAGE;       // [2] accumulator ready for draining
  uint64_t* acc_empty = bars + 2 * NSTAGE + 2;  // [2] accumulator drained
  uint64_t* fin = bars + 2 * NSTAGE + 4;        // all MMAs complete (abort path)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSTAGE + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntn = (g.n + TN - 1) / TN;
  const int row0 = (blockIdx.x / ntn) * TM, col0 = (blockIdx.x % ntn) * TN;
  if (g.lower_n > 0 && col0 % g.lower_n > row0) return;   // Hermitian: upper blocks not needed
  const int64_t kbeg = g.k0 + int64_t(blockIdx.y) * g.nwin * WIN;
  const int64_t kstop = min(g.kend, kbeg + int64_t(g.nwin) * WIN);
  const int nw = kstop > kbeg ? int((kstop - kbeg + WIN - 1) / WIN) : 0;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(smem_u32(full + s), 1);
      mbar_init(smem_u32(empty + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(acc_full + b), 1);
      mbar_init(smem_u32(acc_empty + b), 8);   // one arrival per draining warp
    }
    mbar_init(smem_u32(fin), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // tensor memory: two 128-column accumulators, then the high-weight sums
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // number of (window, product) accumulators and k-tiles in each window
  auto ktiles = [&](int w) -> int {
    const int64_t a = kbeg + int64_t(w) * WIN;
    const int64_t b = min(kstop, a + WIN);
    return int((b - a + BK - 1) / BK);
  };

  if (warp < 4) {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_LOW));
  if (warp == 0) {
    // ---- producer ----
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int w = 0; w < nw && ok; ++w) {
        const int nt = ktiles(w);
        for (int p = 0; p < NPROD && ok; ++p) {
          for (int kt = 0; kt < nt; ++kt, ++it) {
            const int st = it % NSTAGE, ph = it / NSTAGE;
            if (ph >= 1 && !mbar_wait(smem_u32(empty + st), (ph - 1) & 1, abort_flag)) {
              ok = false;
              break;
            }
            const int k = int(kbeg + int64_t(w) * WIN + int64_t(kt) * BK);
            const uint32_t fb = smem_u32(full + st);
            mbar_expect_tx(fb, 2 * TILE_BYTES);
            tma_load_3d(smem_u32(sA + st * TILE_BYTES), &mapA, k, row0, kProd.s[p], fb);
            tma_load_3d(smem_u32(sB + st * TILE_BYTES), &mapB, k, col0, kProd.t[p], fb);
          }
        }
      }
      if (!ok) {
        atomicExch(g.err, 1);
        *abort_flag = 1;
      }
      // the copies still in flight land before the CTA can exit (separate fixed limit)
      for (int j = (it > NSTAGE ? it - NSTAGE : 0); j < it; ++j)
        mbar_wait_inflight(smem_u32(full + j % NSTAGE), (j / NSTAGE) & 1);
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int it = 0, acc = 0;
      bool ok = true;
      for (int w = 0; w < nw && ok; ++w) {
        const int nt = ktiles(w);
        for (int p = 0; p < NPROD && ok; ++p, ++acc) {
          const int b = acc & 1, use = acc >> 1;
          if (use >= 1 && !mbar_wait(smem_u32(acc_empty + b), (use - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + uint32_t(b * TN);
          for (int kt = 0; kt < nt; ++kt, ++it) {
            const int st = it % NSTAGE, ph = it / NSTAGE;
            if (!mbar_wait(smem_u32(full + st), ph & 1, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + st * TILE_BYTES), b0 = smem_u32(sB + st * TILE_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              mma_bf16(d, smem_desc(a0 + 32 * kk), smem_desc(b0 + 32 * kk), (kt > 0 || kk > 0) ? 1u : 0u);
            mma_commit(smem_u32(empty + st));
          }
          if (ok) mma_commit(smem_u32(acc_full + b));
        }
      }
      if (!ok) {
        atomicExch(g.err, 1);
        *abort_flag = 1;
      }
      // every MMA issued so far completes before tensor memory is released
      mma_commit(smem_u32(fin));
      mbar_wait_inflight(smem_u32(fin), 0);
    }
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_HIGH));
    // ---- drain: warps 4..11; lanes quarter (warp % 4), columns half (warp - 4) / 4 ----
    const int q = warp & 3, half = (warp - 4) >> 2;
    const int r = row0 + 32 * q + lane;
    // high-weight sums in tensor memory: low words at columns 256 + c, high words at 384 + c
    const uint32_t lane_base = tmem + (uint32_t(32 * q) << 16);
    const uint32_t fh_lo = lane_base + uint32_t(2 * TN + 64 * half), fh_hi = fh_lo + TN;
    {
      uint32_t z[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) z[c] = 0u;
      for (int h = 0; h < 8; ++h) {
        tmem_st8u(fh_lo + 8 * h, z);
        tmem_st8u(fh_hi + 8 * h, z);
      }
      tmem_wait_st();
    }
    long long F[64];   // low-weight sum
#pragma unroll
    for (int c = 0; c < 64; ++c) F[c] = 0;
    int acc = 0;
    bool ok = true;
    for (int w = 0; w < nw && ok; ++w) {
#pragma unroll 1
      for (int p = 0; p < NPROD; ++p, ++acc) {
        const int b = acc & 1, use = acc >> 1;
        if (!mbar_wait(smem_u32(acc_full + b), use & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int wgt = int(kProd.s[p]) + int(kProd.t[p]);   // (s - 1) + (t - 1) = w - 2
        const uint32_t ta = lane_base + uint32_t(b * TN + 64 * half);
        if (wgt <= W_SPLIT) {
          // exact integers |v| <= 2^24 shifted left into the tensor-memory sum
          const int sh = FIX_HI - BETA * wgt;
#pragma unroll 1
          for (int h = 0; h < 8; ++h) {
            uint32_t v[8], lo[8], hi[8];
            tmem_ld8u(ta + 8 * h, v);
            tmem_ld8u(fh_lo + 8 * h, lo);
            tmem_ld8u(fh_hi + 8 * h, hi);
            tmem_wait_ld();
            if (h == 7) {   // the whole accumulator read: it may be reused
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(acc_empty + b));
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const long long f = static_cast<long long>((static_cast<unsigned long long>(hi[c]) << 32) | lo[c]) +
                                  (static_cast<long long>(__float2int_rn(__uint_as_float(v[c]))) << sh);
              lo[c] = static_cast<uint32_t>(f);
              hi[c] = static_cast<uint32_t>(static_cast<unsigned long long>(f) >> 32);
            }
            tmem_st8u(fh_lo + 8 * h, lo);
            tmem_st8u(fh_hi + 8 * h, hi);
            tmem_wait_st();
          }
        } else {
          const int sh = FIX_LO - BETA * (wgt - W_SPLIT - 1);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(ta + 32 * h, v);
            if (h == 1) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(acc_empty + b));
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) F[32 * h + c] += static_cast<long long>(__float2int_rn(v[c])) << sh;
          }
        }
      }
    }
    if (!ok) {
      if (lane == 0) atomicExch(g.err, 1);
      *abort_flag = 1;
    } else {
      const int e_r = r < g.m ? g.ea[r] : 0;
      double* o = g.out + int64_t(blockIdx.y) * g.ss + int64_t(r) * g.rs;
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        uint32_t lo[8], hi[8];
        tmem_ld8u(fh_lo + 8 * h, lo);   // warp-wide loads, before any lane leaves
        tmem_ld8u(fh_hi + 8 * h, hi);
        tmem_wait_ld();
        if (r >= g.m) continue;
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
          const int col = col0 + 64 * half + 8 * h + c;
          if (col >= g.n) break;
          double v[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int cc = col + u;
            if (cc >= g.n) {
              v[u] = 0.0;
              continue;
            }
            const int e = e_r + g.eb[cc];
            const long long fh = static_cast<long long>((static_cast<unsigned long long>(hi[c + u]) << 32) | lo[c + u]);
            v[u] = e >= E_NONFINITE ? __longlong_as_double(0x7FF8000000000000ll)
                                    : ldexp(double(fh), e - FIX_HI - 2 * BETA) +
                                          ldexp(double(F[8 * h + c + u]), e - FIX_LO - 3 * BETA - 2 * BETA);
          }
          double* dst = o + int64_t(col >> 1) * g.cs2;
          if (g.accumulate) {
            dst[0] += v[0];
            if (col + 1 < g.n) dst[1] += v[1];
          } else {
            dst[0] = v[0];
            if (col + 1 < g.n) dst[1] = v[1];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// ---------------------------------------------------------------------------------------
// operand digits
// ---------------------------------------------------------------------------------------

// e with max <= 2^(e - 1) (max = f 2^x, f in [1/2, 1): e = x + 1); 0 for max = 0;
// E_NONFINITE for an Inf or NaN maximum (its digits come out zero, its outputs NaN)
__device__ __forceinline__ int scale_exponent(double mx) {
  if (!(mx <= 1.7976931348623157e308)) return E_NONFINITE;
  if (!(mx > 0.0)) return 0;
  int x;
  frexp(mx, &x);
  return x + 1;
}

// T balanced digits of x 2^-e (|x| <= 2^(e-1)) in integer arithmetic on the bits of x
// (GB300 runs FP64 at a small fraction of its integer rate): X = round(x 2^(8T - e)) is a
// 64-bit integer with |X| <= 2^(8T - 1) (error <= 2^(e - 8T - 1), the truncation bound of
// T digits), written as X = sum_s d_s 2^(8 (T - 1 - s)) with the low digits in
// [-128, 127] and the top one in [-128, 128].
template <int TD>
__device__ __forceinline__ void digits(double x, int e, float (&d)[TD]) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int ex = int((b >> 52) & 0x7FF);
  unsigned long long m = b & ((1ull << 52) - 1);
  if (ex != 0) m |= 1ull << 52;                 // value = m 2^(max(ex, 1) - 1075)
  const int sh = (ex != 0 ? ex : 1) - 1075 + BETA * TD - e;
  long long X;
  if (sh >= 0)
    X = static_cast<long long>(m << sh);        // sh <= 3 when |x| <= 2^(e-1)
  else if (sh < -62)
    X = 0;
  else
    X = static_cast<long long>((m + (1ull << (-sh - 1))) >> (-sh));
  if (b >> 63) X = -X;
#pragma unroll
  for (int s = TD - 1; s > 0; --s) {
    const long long q = ((X + 128) & 255) - 128;
    d[s] = float(int(q));
    X = (X - q) >> BETA;
  }
  d[0] = float(int(X));
}

// |x| as ordered integer bits (non-negative doubles compare like their bit patterns)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ double block_max(unsigned long long v, unsigned long long* red) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < int(blockDim.x >> 5) ? red[l] : 0ull;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return __longlong_as_double(static_cast<long long>(v));
}

// Column operand of a product over the complex rows r0 .. r0 + nr - 1 of X (column j:
// vector j, complex rows interleaved (re, im)), each row optionally weighted by w[row / 2]
// (the lumped mass of its node).  Row j of the digit matrix holds the reals of column j,
// k = 2 (r - r0) + c; with pair_rows, row ncol + j holds J x_j: (im, -re) per complex
// entry, so that sum_k X_i[k] (J X_j)[k] = Im (x_i^H x_j).  Digits [T][rows][ldk] bf16,
// k >= 2 nr zero; exponents e[row].  One block per column.
__global__ void slice_cols_kernel(const double* __restrict__ X, int64_t ldx, int ncol, int64_t r0, int64_t nr,
                                  const double* __restrict__ w, int pair_rows, int64_t ldk, int rows_total,
                                  __nv_bfloat16* __restrict__ D, int* __restrict__ e_out) {
  __shared__ unsigned long long red[32];
  const int j = blockIdx.x;
  const double2* x = reinterpret_cast<const double2*>(X + 2 * int64_t(j) * ldx) + r0;
  unsigned long long mb = 0;
  for (int64_t r = threadIdx.x; r < nr; r += blockDim.x) {
    double2 v = x[r];
    if (w) {
      const double m = w[(r0 + r) >> 1];
      v.x *= m;
      v.y *= m;
    }
    mb = max(mb, max(abs_bits(v.x), abs_bits(v.y)));
  }
  const double mx = block_max(mb, red);
  const int e = scale_exponent(mx);
  if (threadIdx.x == 0) {
    e_out[j] = e;
    if (pair_rows) e_out[ncol + j] = e;
  }
  const int64_t slice = int64_t(rows_total) * ldk;
  __nv_bfloat162* dj = reinterpret_cast<__nv_bfloat162*>(D + int64_t(j) * ldk);
  __nv_bfloat162* dp = reinterpret_cast<__nv_bfloat162*>(D + int64_t(ncol + j) * ldk);
  for (int64_t r = threadIdx.x; r < ldk / 2; r += blockDim.x) {
    float dr[T], di[T];
    if (r < nr) {
      double2 v = x[r];
      if (w) {
        const double m = w[(r0 + r) >> 1];
        v.x *= m;
        v.y *= m;
      }
      digits<T>(v.x, e, dr);
      digits<T>(v.y, e, di);
    } else {
#pragma unroll
      for (int s = 0; s < T; ++s) dr[s] = di[s] = 0.f;
    }
#pragma unroll
    for (int s = 0; s < T; ++s) {
      dj[s * slice / 2 + r] = __floats2bfloat162_rn(dr[s], di[s]);
      if (pair_rows) dp[s * slice / 2 + r] = __floats2bfloat162_rn(di[s], -dr[s]);
    }
  }
}

// Row operand of the product Y Q over complex rows r0 .. r0 + nr - 1 of Y (n columns):
// row r of the digit matrix holds [Re Y(r, :), Im Y(r, :)], k = i and n + i.  Exponent
// of row r = that of max_i max(|Re|, |Im|).  One thread per row.
__global__ void row_exponent_kernel(const double* __restrict__ Y, int64_t ldy, int n, int64_t r0, int64_t nr,
                                    int* __restrict__ e_out) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= nr) return;
  unsigned long long mb = 0;
  for (int i = 0; i < n; ++i) {
    const double2 v = reinterpret_cast<const double2*>(Y + 2 * int64_t(i) * ldy)[r0 + r];
    mb = max(mb, max(abs_bits(v.x), abs_bits(v.y)));
  }
  e_out[r] = scale_exponent(__longlong_as_double(static_cast<long long>(mb)));
}

// digits of a 32-row x 32-column tile of Y, transposed through shared memory so that
// each row's digits are written contiguously along k.  Grid (row tiles, column tiles).
template <int TD>
__global__ void __launch_bounds__(256) slice_rows_kernel(const double* __restrict__ Y, int64_t ldy, int n,
                                                         int64_t r0, int64_t nr, const int* __restrict__ e_row,
                                                         int64_t ldk, __nv_bfloat16* __restrict__ D) {
  __shared__ __nv_bfloat16 sd[TD][32][66];   // [s][row][k: 32 re then 32 im] (+2 padding)
  const int rt = blockIdx.x, it = blockIdx.y;
  const int lr = threadIdx.x & 31, ib = threadIdx.x >> 5;
  const int64_t r = int64_t(rt) * 32 + lr;
  const int e = r < nr ? e_row[r] : 0;
  for (int jj = 0; jj < 4; ++jj) {
    const int li = ib + 8 * jj, i = it * 32 + li;
    float dr[TD], di[TD];
    if (r < nr && i < n) {
      const double2 v = reinterpret_cast<const double2*>(Y + 2 * int64_t(i) * ldy)[r0 + r];
      digits<TD>(v.x, e, dr);
      digits<TD>(v.y, e, di);
    } else {
#pragma unroll
      for (int s = 0; s < TD; ++s) dr[s] = di[s] = 0.f;
    }
#pragma unroll
    for (int s = 0; s < TD; ++s) {
      sd[s][lr][li] = __float2bfloat16_rn(dr[s]);
      sd[s][lr][32 + li] = __float2bfloat16_rn(di[s]);
    }
  }
  __syncthreads();
  // write: per (s, row, part) 32 bf16, as 2-element pieces
  const int64_t slice = int64_t(nr) * ldk;
  for (int t = threadIdx.x; t < TD * 32 * 2 * 16; t += 256) {
    const int piece = t & 15, part = (t >> 4) & 1, lrow = (t >> 5) & 31, s = t >> 10;
    const int64_t rr = int64_t(rt) * 32 + lrow;
    const int i0 = it * 32 + piece * 2;
    if (rr >= nr || i0 >= n) continue;
    __nv_bfloat16* dst = D + s * slice + rr * ldk + (part ? n : 0) + i0;
    dst[0] = sd[s][lrow][part * 32 + piece * 2];
    if (i0 + 1 < n) dst[1] = sd[s][lrow][part * 32 + piece * 2 + 1];
  }
}

// Column operand of Y Q for a complex n x n matrix Q (column-major, Q(i, j) at i + j ldq):
// output column 2j = (Re Q(:, j); -Im Q(:, j)), 2j + 1 = (Im Q(:, j); Re Q(:, j)), so that
// [Re y, Im y] . col 2j = Re (y Q)_j and . col 2j + 1 = Im (y Q)_j.  offdiag: Q(j, j) is
// taken as zero (the off-diagonal part of Section III-C-4).  One block per j.
template <int TD>
__global__ void slice_rotation_kernel(const double* __restrict__ Q, int64_t ldq, int n, int64_t ldk, int offdiag,
                                      __nv_bfloat16* __restrict__ D, int* __restrict__ e_out) {
  __shared__ unsigned long long red[32];
  const int j = blockIdx.x;
  const double2* q = reinterpret_cast<const double2*>(Q + 2 * int64_t(j) * ldq);
  unsigned long long mb = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!(offdiag && i == j)) mb = max(mb, max(abs_bits(q[i].x), abs_bits(q[i].y)));
  const double mx = block_max(mb, red);
  const int e = scale_exponent(mx);
  if (threadIdx.x == 0) e_out[2 * j] = e_out[2 * j + 1] = e;
  const int64_t slice = int64_t(2 * n) * ldk;
  __nv_bfloat16* c0 = D + int64_t(2 * j) * ldk;
  __nv_bfloat16* c1 = D + int64_t(2 * j + 1) * ldk;
  for (int k = threadIdx.x; k < ldk; k += blockDim.x) {
    float a[TD], b[TD];
    const int i = k < n ? k : k - n;
    if (k < 2 * n && !(offdiag && i == j)) {
      const double2 v = q[i];
      digits<TD>(k < n ? v.x : -v.y, e, a);   // column 2j
      digits<TD>(k < n ? v.y : v.x, e, b);    // column 2j + 1
    } else {
#pragma unroll
      for (int s = 0; s < TD; ++s) a[s] = b[s] = 0.f;
    }
#pragma unroll
    for (int s = 0; s < TD; ++s) {
      c0[s * slice + k] = __float2bfloat16_rn(a[s]);
      c1[s * slice + k] = __float2bfloat16_rn(b[s]);
    }
  }
}

// S(i, j) = sum over slots of C[i][j] + i C[i][nz + j]  (i < n, j < nz; lower: i >= j only),
// C [slot][n][2 nz]
__global__ void gram_reduce_kernel(const double* __restrict__ C, int nslot, int n, int nz, int64_t slot_stride,
                                   double* __restrict__ S, int64_t lds, int lower) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n || (lower && i < j)) return;
  double re = 0.0, im = 0.0;
  for (int s = 0; s < nslot; ++s) {
    const double* c = C + s * slot_stride + int64_t(i) * 2 * nz;
    re += c[j];
    im += c[nz + j];
  }
  reinterpret_cast<double2*>(S)[i + int64_t(j) * lds] = make_double2(re, im);
}

// X(r, j) += Q(j, j) Y(r, j) in FP64 (the diagonal part of the rotation, Section III-C-4)
__global__ void add_diag_kernel(const double* __restrict__ Y, int64_t ldy, const double* __restrict__ Q,
                                int64_t ldq, int64_t nrows, double* __restrict__ X, int64_t ldx) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r >= nrows) return;
  const double2 q = reinterpret_cast<const double2*>(Q)[j + int64_t(j) * ldq];
  const double2 y = reinterpret_cast<const double2*>(Y + 2 * int64_t(j) * ldy)[r];
  double2* x = reinterpret_cast<double2*>(X + 2 * int64_t(j) * ldx) + r;
  const double2 o = *x;
  *x = make_double2(o.x + (q.x * y.x - q.y * y.y), o.y + (q.x * y.y + q.y * y.x));
}

}  // namespace tc
}  // namespace rcf

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
namespace rcf {
namespace tc {
namespace {

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

// digits [T][rows][ldk] bf16 viewed as (k < kdim, row, s) with (64, 128, 1) boxes and the
// 128-byte swizzle; k >= kdim and rows beyond `rows` read as zero
int encode_digits(rcf_ctx* ctx, CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t ldk,
                  int64_t kdim, int td = T) {
  auto fn = encode_fn();
  if (!fn) return fail(ctx, RCF_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ldk % BK != 0)
    return fail(ctx, RCF_EINVAL, "digit buffer misaligned");
  const cuuint64_t dims[3] = {cuuint64_t(kdim), cuuint64_t(rows), cuuint64_t(td)};
  const cuuint64_t strides[2] = {cuuint64_t(ldk) * 2, cuuint64_t(rows) * cuuint64_t(ldk) * 2};
  const cuuint32_t box[3] = {BK, TM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(base), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, RCF_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
  return RCF_OK;
}

constexpr size_t kSmem = 1024 + 2 * NSTAGE * TILE_BYTES + 256;

// C (+)= A B^T over k in [k0, kend) for the digit maps; splits CTAs per tile along k
template <int TD>
int launch_gemm(rcf_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, int m, int n, int64_t k0,
                int64_t kend, int splits, const int* ea, const int* eb, double* out, int64_t ss, int64_t rs,
                int64_t cs2, int lower_n, bool overwrite) {
  static bool attr = false;
  if (!attr) {
    RCF_CUDA(ctx, cudaFuncSetAttribute(ozaki_gemm_kernel<TD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(kSmem)));
    attr = true;
  }
  const int tiles = ((m + TM - 1) / TM) * ((n + TN - 1) / TN);
  for (int64_t k = k0; k < kend;) {
    const int64_t wins = (kend - k + WIN - 1) / WIN;
    const int nwin = int(std::min<int64_t>(LAUNCH_WINDOWS, (wins + splits - 1) / splits));
    const int ny = int(std::min<int64_t>(splits, (wins + nwin - 1) / nwin));
    GemmArgs g;
    g.m = m;
    g.n = n;
    g.k0 = k;
    g.nwin = nwin;
    g.kend = kend;
    g.ea = ea;
    g.eb = eb;
    g.out = out;
    g.ss = ss;
    g.rs = rs;
    g.cs2 = cs2;
    g.accumulate = (overwrite && k == k0) ? 0 : 1;
    g.lower_n = lower_n;
    g.err = ctx->d_err;
    ozaki_gemm_kernel<TD><<<dim3(tiles, ny), NTHREADS, kSmem, ctx->stream>>>(ma, mb, g);
    RCF_CHECK_LAUNCH(ctx);
    k += int64_t(ny) * nwin * WIN;
  }
  return RCF_OK;
}

int sm_count(rcf_ctx* ctx) {
  static int n = 0;
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || n <= 0) n = 152;
  }
  return n;
}

}  // namespace
}  // namespace tc

// C (n x nz complex, column-major, ldc) = Y^H diag(w) Z over all complex rows (w the weight
// of row r is w[r / 2], null: 1); lower: only C(i, j), i >= j, for Z = Y (Hermitian Gram).
int tc_gemm_tn(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* w, const double* Z, int64_t ldz,
               int nz, int64_t nrows, double* C, int64_t ldc, int lower) {
  using namespace tc;
  if (!ctx->d_err) return fail(ctx, RCF_ENOTSUP, "tensor-core products need the device error word");
  lower = lower && Z == Y && nz == n && n % TM == 0;
  // complex rows per chunk: digits of both operands within ~8 GB, whole windows
  int64_t kc = int64_t(8) << 30;
  kc /= int64_t(T) * 2 * 2 * (n + 2 * int64_t(nz));
  kc = std::max<int64_t>(WIN / 2, kc / (WIN / 2) * (WIN / 2));
  kc = std::min<int64_t>(kc, (nrows + WIN / 2 - 1) / (WIN / 2) * (WIN / 2));
  const int64_t ldk = 2 * kc;
  __nv_bfloat16 *DA = nullptr, *DB = nullptr;
  int* E = nullptr;
  RCF_TRY(workspace(ctx, WS_TC_A, sizeof(__nv_bfloat16) * T * size_t(n) * ldk, reinterpret_cast<void**>(&DA)));
  RCF_TRY(workspace(ctx, WS_TC_B, sizeof(__nv_bfloat16) * T * size_t(2 * nz) * ldk, reinterpret_cast<void**>(&DB)));
  RCF_TRY(workspace(ctx, WS_TC_E, sizeof(int) * size_t(n + 2 * nz), reinterpret_cast<void**>(&E)));
  const int tiles_m = (n + TM - 1) / TM, tiles_n = (2 * nz + TN - 1) / TN;
  const int tiles = lower ? tiles_m * (tiles_m + 1) : tiles_m * tiles_n;   // computed tiles
  const int splits = std::max(1, std::min(64, sm_count(ctx) / std::max(1, tiles)));
  double* P = nullptr;
  const size_t slot = size_t(n) * 2 * nz;
  RCF_TRY(workspace(ctx, WS_TC_C, sizeof(double) * slot * splits, reinterpret_cast<void**>(&P)));
  RCF_CUDA(ctx, cudaMemsetAsync(P, 0, sizeof(double) * slot * splits, ctx->stream));
  CUtensorMap ma, mb;
  RCF_TRY(encode_digits(ctx, &ma, DA, n, ldk, ldk));          // k padding written as zeros
  RCF_TRY(encode_digits(ctx, &mb, DB, 2 * nz, ldk, ldk));
  for (int64_t r0 = 0; r0 < nrows; r0 += kc) {
    const int64_t nr = std::min(kc, nrows - r0);
    slice_cols_kernel<<<n, 512, 0, ctx->stream>>>(Y, ldy, n, r0, nr, nullptr, 0, ldk, n, DA, E);
    RCF_CHECK_LAUNCH(ctx);
    slice_cols_kernel<<<nz, 512, 0, ctx->stream>>>(Z, ldz, nz, r0, nr, w, 1, ldk, 2 * nz, DB, E + n);
    RCF_CHECK_LAUNCH(ctx);
    RCF_TRY(launch_gemm<T>(ctx, ma, mb, n, 2 * nz, 0, 2 * nr, splits, E, E + n, P, int64_t(slot), 2 * int64_t(nz),
                           2, lower ? n : 0, false));
  }
  gram_reduce_kernel<<<dim3((n + 127) / 128, nz), 128, 0, ctx->stream>>>(P, splits, n, nz, int64_t(slot), C, ldc,
                                                                        lower);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

namespace tc {
namespace {

// X = Y Q with TD digits per entry (offdiag: Q's diagonal taken as zero), row chunks of Y
template <int TD>
int rotate_chunks(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Q, int64_t ldq, int64_t nrows,
                  double* X, int64_t ldx, int offdiag) {
  const int64_t ldk = (2 * int64_t(n) + BK - 1) / BK * BK;
  int64_t rc = (int64_t(6) << 30) / (int64_t(TD) * 2 * ldk);
  rc = std::max<int64_t>(TM, rc / TM * TM);
  rc = std::min<int64_t>(rc, (nrows + TM - 1) / TM * TM);
  __nv_bfloat16 *DA = nullptr, *DB = nullptr;
  int* E = nullptr;
  RCF_TRY(workspace(ctx, WS_TC_A, sizeof(__nv_bfloat16) * TD * size_t(rc) * ldk, reinterpret_cast<void**>(&DA)));
  RCF_TRY(workspace(ctx, WS_TC_B, sizeof(__nv_bfloat16) * TD * size_t(2 * n) * ldk, reinterpret_cast<void**>(&DB)));
  RCF_TRY(workspace(ctx, WS_TC_E, sizeof(int) * size_t(rc + 2 * n), reinterpret_cast<void**>(&E)));
  slice_rotation_kernel<TD><<<n, 256, 0, ctx->stream>>>(Q, ldq, n, ldk, offdiag, DB, E + rc);
  RCF_CHECK_LAUNCH(ctx);
  CUtensorMap mb;
  RCF_TRY(encode_digits(ctx, &mb, DB, 2 * n, ldk, 2 * int64_t(n), TD));
  for (int64_t r0 = 0; r0 < nrows; r0 += rc) {
    const int64_t nr = std::min(rc, nrows - r0);
    CUtensorMap ma;
    RCF_TRY(encode_digits(ctx, &ma, DA, nr, ldk, 2 * int64_t(n), TD));
    row_exponent_kernel<<<unsigned((nr + 255) / 256), 256, 0, ctx->stream>>>(Y, ldy, n, r0, nr, E);
    RCF_CHECK_LAUNCH(ctx);
    slice_rows_kernel<TD><<<dim3(unsigned((nr + 31) / 32), unsigned((n + 31) / 32)), 256, 0, ctx->stream>>>(
        Y, ldy, n, r0, nr, E, ldk, DA);
    RCF_CHECK_LAUNCH(ctx);
    // one launch covers K = 2n <= LAUNCH_WINDOWS windows: the output is written, not added to
    RCF_TRY(launch_gemm<TD>(ctx, ma, mb, int(nr), 2 * n, 0, 2 * n, 1, E, E + rc, X + 2 * r0, 0, 2, 2 * ldx, 0,
                            true));
  }
  return RCF_OK;
}

}  // namespace
}  // namespace tc

// X (nrows x n complex, ldx) = Y Q for a device n x n complex Q (ldq).  mixed = false:
// FP64-accurate, X may equal Y (ldx == ldy).  mixed = true (Section III-C-4): Y Q_offdiag at
// FP32-level accuracy (3 digits) plus Y diag(Q) in FP64; X must not overlap Y.
int tc_rotate(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Q, int64_t ldq, int64_t nrows,
              double* X, int64_t ldx, bool mixed) {
  using namespace tc;
  if (!ctx->d_err) return fail(ctx, RCF_ENOTSUP, "tensor-core products need the device error word");
  if (2 * n > LAUNCH_WINDOWS * WIN)
    return fail(ctx, RCF_ENOTSUP, "tensor-core rotation supports up to %d vectors", LAUNCH_WINDOWS * WIN / 2);
  const char* x0 = reinterpret_cast<const char*>(X);
  const char* y0 = reinterpret_cast<const char*>(Y);
  const bool overlap = x0 < y0 + size_t(ldy) * n * 16 && y0 < x0 + size_t(ldx) * n * 16;
  if (mixed) {
    if (overlap) return fail(ctx, RCF_EINVAL, "the mixed-precision rotation cannot write over its input");
    RCF_TRY(rotate_chunks<T_LOW>(ctx, Y, ldy, n, Q, ldq, nrows, X, ldx, 1));
    add_diag_kernel<<<dim3(unsigned((nrows + 255) / 256), n), 256, 0, ctx->stream>>>(Y, ldy, Q, ldq, nrows, X, ldx);
    RCF_CHECK_LAUNCH(ctx);
    return RCF_OK;
  }
  if (X != Y && overlap)
    return fail(ctx, RCF_EINVAL, "rotation output overlaps its input (only X == Y is allowed)");
  if (X == Y && ldx != ldy) return fail(ctx, RCF_EINVAL, "in-place rotation needs equal leading dimensions");
  return rotate_chunks<T>(ctx, Y, ldy, n, Q, ldq, nrows, X, ldx, 0);
}

}  // namespace rcf

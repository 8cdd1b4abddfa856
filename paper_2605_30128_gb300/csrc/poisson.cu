// Periodic FE Poisson solve: matrix-free Laplacian K x and preconditioned CG with a
// Chebyshev-Jacobi preconditioner (Section III-B-1; Algorithm pcg_fusion), FP64.
//
// K_IJ = int grad N_I . grad N_J on the periodic GLL mesh.  On a uniform mesh the assembled
// matrix is K = c_x K1g (x) Wg (x) Wg + c_y Wg (x) K1g (x) Wg + c_z Wg (x) Wg (x) K1g, with K1g
// and Wg the assembled 1D reference stiffness and GLL mass and c_d = (2 / h_d)^2 h_x h_y h_z / 8,
// so K x is one pass over the nodes: per direction a 1D stencil along that direction
// (the nodes of the element, both elements at a vertex) scaled by the GLL weights of the
// other two directions.  One thread per node, neighbours through L1/L2 (a scalar field of a
// million nodes is 8 MB: the whole solve is L2-resident on GB300).
//
// PCG in the paper's fused arrangement, all scalars kept on the device (no host round trip
// inside an iteration except the convergence test): w = K p; eta = p.w; alpha = delta/eta;
// x += alpha p and r += alpha w in one pass; z = P^-1 r; (delta_new, gamma) = (r.z, r.r) in
// one reduction; beta = delta_new/delta; p = -z + beta p.
// P^-1 = chi(A) diag(K)^-1, A = diag(K)^-1 K, chi the degree-m polynomial of Chebyshev
// semi-iteration on [a, b] (textbook three-term recurrence); each of its steps is one
// fused K x pass that also updates the iterate, its residual and the next direction.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace rcf {
namespace {

constexpr int kMaxTap = 2 * kMaxP + 1;

// per direction d and local position a (0 = element vertex), coefficients of offsets
// -p .. p along d (zero outside the support), scaled by c_d; wg[a] = assembled 1D GLL weight
struct LapTables {
  double c[3][kMaxP][kMaxTap];
  double wg[kMaxP];
};

__device__ __forceinline__ int wrap(int i, int G) { return i < 0 ? i + G : (i >= G ? i - G : i); }

// (K x)_I for the node (i, j, k)
template <int P>
__device__ __forceinline__ double lap_node(const LapTables& t, const double* __restrict__ x, int i, int j, int k,
                                           int Gx, int Gy, int Gz) {
  const int64_t sy = Gx, sz = int64_t(Gx) * Gy;
  const int ai = i % P, aj = j % P, ak = k % P;
  const double* row = x + j * sy + k * sz;
  double sx_ = 0.0, sy_ = 0.0, sz_ = 0.0;
  const int lo_i = ai == 0 ? -P : -ai, hi_i = ai == 0 ? P : P - ai;
#pragma unroll
  for (int o = -P; o <= P; ++o)
    if (o >= lo_i && o <= hi_i) sx_ += t.c[0][ai][o + P] * row[wrap(i + o, Gx)];
  const double* col = x + i + k * sz;
  const int lo_j = aj == 0 ? -P : -aj, hi_j = aj == 0 ? P : P - aj;
#pragma unroll
  for (int o = -P; o <= P; ++o)
    if (o >= lo_j && o <= hi_j) sy_ += t.c[1][aj][o + P] * col[wrap(j + o, Gy) * sy];
  const double* pil = x + i + j * sy;
  const int lo_k = ak == 0 ? -P : -ak, hi_k = ak == 0 ? P : P - ak;
#pragma unroll
  for (int o = -P; o <= P; ++o)
    if (o >= lo_k && o <= hi_k) sz_ += t.c[2][ak][o + P] * pil[wrap(k + o, Gz) * sz];
  return t.wg[aj] * t.wg[ak] * sx_ + t.wg[ai] * t.wg[ak] * sy_ + t.wg[ai] * t.wg[aj] * sz_;
}

template <int P>
__global__ void laplacian_kernel(const LapTables t, const double* __restrict__ x, double* __restrict__ y, int Gx,
                                 int Gy, int Gz) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = int64_t(Gx) * Gy * Gz;
  if (I >= n) return;
  const int i = int(I % Gx), j = int((I / Gx) % Gy), k = int(I / (int64_t(Gx) * Gy));
  y[I] = lap_node<P>(t, x, i, j, k, Gx, Gy, Gz);
}

// one Chebyshev semi-iteration step fused with its K x: at every node
//   y += d;  res -= (K d) / Kdiag;  d_next = c1 d + c2 res
template <int P>
__global__ void cheb_step_kernel(const LapTables t, const double* __restrict__ d, const double* __restrict__ kdiag,
                                 double* __restrict__ y, double* __restrict__ res, double* __restrict__ dnext,
                                 double c1, double c2, int Gx, int Gy, int Gz) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = int64_t(Gx) * Gy * Gz;
  if (I >= n) return;
  const int i = int(I % Gx), j = int((I / Gx) % Gy), k = int(I / (int64_t(Gx) * Gy));
  const double kd = lap_node<P>(t, d, i, j, k, Gx, Gy, Gz);
  const double dI = d[I];
  y[I] += dI;
  const double r = res[I] - kd / kdiag[I];
  res[I] = r;
  dnext[I] = c1 * dI + c2 * r;
}

// start of the preconditioner: g = r / Kdiag, res = g, d = g / theta, y = 0
__global__ void cheb_init_kernel(int64_t n, const double* __restrict__ r, const double* __restrict__ kdiag,
                                 double inv_theta, double* __restrict__ y, double* __restrict__ res,
                                 double* __restrict__ d) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= n) return;
  const double g = r[I] / kdiag[I];
  y[I] = 0.0;
  res[I] = g;
  d[I] = g * inv_theta;
}

// Device scalars of one solve: [0] eta, [1] delta, [2] delta_new, [3] gamma
enum { S_ETA = 0, S_DELTA = 1, S_DNEW = 2, S_GAMMA = 3, S_COUNT = 4 };
constexpr int kRedBlocks = 304;   // 2 x 152 SMs
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = l < int(blockDim.x >> 5) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;   // valid in thread 0
}

// partial[b] = sum over this block's grid-stride share of a.b (and of c.c if c given)
__global__ void __launch_bounds__(kRedThreads) dot_partial_kernel(int64_t n, const double* __restrict__ a,
                                                                  const double* __restrict__ b,
                                                                  const double* __restrict__ c,
                                                                  double* __restrict__ partial) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; I < n; I += int64_t(gridDim.x) * blockDim.x) {
    s0 += a[I] * b[I];
    if (c) s1 += c[I] * c[I];
  }
  s0 = block_sum(s0, sh);
  __syncthreads();
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s0;
    partial[gridDim.x + blockIdx.x] = s1;
  }
}

// scal[i0] = sum of partial[0 .. nb), scal[i1] = sum of partial[nb .. 2 nb) (i1 < 0: none);
// fixed order, so the result does not depend on timing
__global__ void __launch_bounds__(kRedThreads) dot_final_kernel(const double* __restrict__ partial, int nb,
                                                                double* __restrict__ scal, int i0, int i1) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    s0 += partial[b];
    s1 += partial[nb + b];
  }
  s0 = block_sum(s0, sh);
  __syncthreads();
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    scal[i0] = s0;
    if (i1 >= 0) scal[i1] = s1;
  }
}

// x += alpha p, r += alpha w with alpha = delta / eta read from the device scalars
__global__ void pcg_update_kernel(int64_t n, const double* __restrict__ scal, const double* __restrict__ p,
                                  const double* __restrict__ w, double* __restrict__ x, double* __restrict__ r) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= n) return;
  const double alpha = scal[S_DELTA] / scal[S_ETA];
  x[I] += alpha * p[I];
  r[I] += alpha * w[I];
}

// p = -z + beta p, beta = delta_new / delta (first: p = -z)
__global__ void pcg_direction_kernel(int64_t n, const double* __restrict__ scal, const double* __restrict__ z,
                                     double* __restrict__ p, int first) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= n) return;
  p[I] = first ? -z[I] : -z[I] + (scal[S_DNEW] / scal[S_DELTA]) * p[I];
}

// delta <- delta_new (one thread, after the direction update has read both)
__global__ void pcg_shift_kernel(double* scal) { scal[S_DELTA] = scal[S_DNEW]; }

// r = K x - f  (K x already in r)
__global__ void sub_kernel(int64_t n, const double* __restrict__ f, double* __restrict__ r) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I < n) r[I] -= f[I];
}

void build_lap_tables(const rcf_mesh* m, LapTables* t, std::vector<double>* kdiag_1d) {
  const int p = m->p, np = m->np;
  *t = LapTables{};
  const double J = m->detJ;   // h_x h_y h_z / 8
  for (int a = 0; a < p; ++a) t->wg[a] = a == 0 ? m->w[0] + m->w[p] : m->w[a];
  for (int d = 0; d < 3; ++d) {
    const double cd = 4.0 / (m->h[d] * m->h[d]) * J;
    for (int a = 0; a < p; ++a) {
      if (a == 0) {
        for (int q = 0; q <= p; ++q) {   // element on the left (local p), on the right (local 0)
          t->c[d][0][q] += cd * m->K1[p * np + q];          // offset q - p
          t->c[d][0][p + q] += cd * m->K1[0 * np + q];      // offset q
        }
      } else {
        for (int q = 0; q <= p; ++q) t->c[d][a][q - a + p] += cd * m->K1[a * np + q];
      }
    }
  }
  kdiag_1d->assign(3 * p, 0.0);
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < p; ++a) (*kdiag_1d)[d * p + a] = t->c[d][a][p];
}

template <int P>
int launch_lap(rcf_ctx* ctx, const rcf_mesh* m, const LapTables& t, const double* x, double* y) {
  const int64_t n = m->nnodes;
  laplacian_kernel<P><<<unsigned((n + 255) / 256), 256, 0, ctx->stream>>>(t, x, y, m->G[0], m->G[1], m->G[2]);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int lap(rcf_ctx* ctx, const rcf_mesh* m, const LapTables& t, const double* x, double* y) {
  switch (m->p) {
    case 1: return launch_lap<1>(ctx, m, t, x, y);
    case 2: return launch_lap<2>(ctx, m, t, x, y);
    case 3: return launch_lap<3>(ctx, m, t, x, y);
    case 4: return launch_lap<4>(ctx, m, t, x, y);
    case 5: return launch_lap<5>(ctx, m, t, x, y);
    case 6: return launch_lap<6>(ctx, m, t, x, y);
    case 7: return launch_lap<7>(ctx, m, t, x, y);
    default: return launch_lap<8>(ctx, m, t, x, y);
  }
}

template <int P>
int launch_cheb(rcf_ctx* ctx, const rcf_mesh* m, const LapTables& t, const double* d, const double* kdiag,
                double* y, double* res, double* dnext, double c1, double c2) {
  const int64_t n = m->nnodes;
  cheb_step_kernel<P><<<unsigned((n + 255) / 256), 256, 0, ctx->stream>>>(t, d, kdiag, y, res, dnext, c1, c2,
                                                                         m->G[0], m->G[1], m->G[2]);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int cheb(rcf_ctx* ctx, const rcf_mesh* m, const LapTables& t, const double* d, const double* kdiag, double* y,
         double* res, double* dnext, double c1, double c2) {
  switch (m->p) {
    case 1: return launch_cheb<1>(ctx, m, t, d, kdiag, y, res, dnext, c1, c2);
    case 2: return launch_cheb<2>(ctx, m, t, d, kdiag, y, res, dnext, c1, c2);
    case 3: return launch_cheb<3>(ctx, m, t, d, kdiag, y, res, dnext, c1, c2);
    case 4: return launch_cheb<4>(ctx, m, t, d, kdiag, y, res, dnext, c1, c2);
    case 5: return launch_cheb<5>(ctx, m, t, d, kdiag, y, res, dnext, c1, c2);
    case 6: return launch_cheb<6>(ctx, m, t, d, kdiag, y, res, dnext, c1, c2);
    case 7: return launch_cheb<7>(ctx, m, t, d, kdiag, y, res, dnext, c1, c2);
    default: return launch_cheb<8>(ctx, m, t, d, kdiag, y, res, dnext, c1, c2);
  }
}

}  // namespace
}  // namespace rcf

namespace rcf {
namespace {

__global__ void kdiag_kernel(const LapTables t, int P, double* __restrict__ kd, int Gx, int Gy, int Gz) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= int64_t(Gx) * Gy * Gz) return;
  const int ai = int(I % Gx) % P, aj = int((I / Gx) % Gy) % P, ak = int(I / (int64_t(Gx) * Gy)) % P;
  kd[I] = t.c[0][ai][P] * t.wg[aj] * t.wg[ak] + t.c[1][aj][P] * t.wg[ai] * t.wg[ak] +
          t.c[2][ak][P] * t.wg[ai] * t.wg[aj];
}

// Gershgorin bound of the spectrum of diag(K)^-1 K: max over the local positions of
// sum_J |K_IJ| / K_II (every node of a uniform mesh is one of p^3 local positions)
double gershgorin_top(const LapTables& t, int p) {
  double best = 0.0;
  for (int ai = 0; ai < p; ++ai)
    for (int aj = 0; aj < p; ++aj)
      for (int ak = 0; ak < p; ++ak) {
        const int a[3] = {ai, aj, ak};
        double row = 0.0, diag = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double wp = t.wg[a[(d + 1) % 3]] * t.wg[a[(d + 2) % 3]];
          for (int o = 0; o <= 2 * p; ++o) row += std::fabs(t.c[d][a[d]][o]) * wp;
          diag += t.c[d][a[d]][p] * wp;
        }
        best = std::max(best, row / diag);
      }
  return best;
}

int check_field(rcf_ctx* ctx, const void* p, const char* name) {
  if (!p) return fail(ctx, RCF_EINVAL, "%s is NULL", name);
  if (reinterpret_cast<uintptr_t>(p) & 7) return fail(ctx, RCF_EINVAL, "%s is not 8-byte aligned", name);
  return RCF_OK;
}

}  // namespace
}  // namespace rcf

using namespace rcf;

extern "C" int rcf_laplacian(rcf_ctx* ctx, const rcf_mesh* mesh, const double* x, double* y) {
  if (!ctx || !mesh) return RCF_EINVAL;
  RCF_TRY(check_field(ctx, x, "x"));
  RCF_TRY(check_field(ctx, y, "y"));
  const char* a = reinterpret_cast<const char*>(x);
  const char* b = reinterpret_cast<const char*>(y);
  const size_t bytes = sizeof(double) * size_t(mesh->nnodes);
  if (a < b + bytes && b < a + bytes) return fail(ctx, RCF_EINVAL, "y overlaps x");
  LapTables t;
  std::vector<double> kd1;
  build_lap_tables(mesh, &t, &kd1);
  return lap(ctx, mesh, t, x, y);
}

extern "C" int rcf_poisson_pcg(rcf_ctx* ctx, const rcf_mesh* mesh, const double* f, double* x, int cheb_degree,
                               double a, double b, double tol, int maxit, int* iterations, double* residual) {
  if (!ctx || !mesh) return RCF_EINVAL;
  RCF_TRY(check_field(ctx, f, "f"));
  RCF_TRY(check_field(ctx, x, "x"));
  if (!iterations || !residual) return fail(ctx, RCF_EINVAL, "iterations and residual must be host pointers");
  if (cheb_degree < 0 || maxit < 0 || !(tol >= 0.0)) return fail(ctx, RCF_EINVAL, "bad degree, tolerance or limit");
  if (cheb_degree > 0 && b > 0.0 && !(0.0 < a && a < b))
    return fail(ctx, RCF_EINVAL, "the Chebyshev interval needs 0 < a < b");
  const int64_t n = mesh->nnodes;
  {
    const char* pf = reinterpret_cast<const char*>(f);
    const char* px = reinterpret_cast<const char*>(x);
    const size_t bytes = sizeof(double) * size_t(n);
    if (pf < px + bytes && px < pf + bytes) return fail(ctx, RCF_EINVAL, "x overlaps f");
  }
  LapTables t;
  std::vector<double> kd1;
  build_lap_tables(mesh, &t, &kd1);
  if (cheb_degree > 0 && !(b > 0.0)) {   // interval from the Gershgorin bound
    b = gershgorin_top(t, mesh->p);
    a = b / 20.0;
  }
  // r, z, p, w, res, d0, d1, kdiag; reduction partials; device scalars
  double* ws = nullptr;
  const size_t vec = size_t(n);
  RCF_TRY(workspace(ctx, WS_PCG, sizeof(double) * (8 * vec + 2 * kRedBlocks + S_COUNT), reinterpret_cast<void**>(&ws)));
  double *r = ws, *z = ws + vec, *p = ws + 2 * vec, *w = ws + 3 * vec, *res = ws + 4 * vec;
  double *d0 = ws + 5 * vec, *d1 = ws + 6 * vec, *kd = ws + 7 * vec;
  double* part = ws + 8 * vec;
  double* scal = part + 2 * kRedBlocks;
  const unsigned gb = unsigned((n + 255) / 256);
  kdiag_kernel<<<gb, 256, 0, ctx->stream>>>(t, mesh->p, kd, mesh->G[0], mesh->G[1], mesh->G[2]);
  RCF_CHECK_LAUNCH(ctx);
  // Chebyshev semi-iteration constants on [a, b]
  const double theta = 0.5 * (b + a), dlt = 0.5 * (b - a), sigma1 = theta / dlt;
  std::vector<double> c1(std::max(cheb_degree, 1)), c2(std::max(cheb_degree, 1));
  {
    double rho = 1.0 / sigma1;
    for (int s = 0; s < cheb_degree; ++s) {
      const double rn = 1.0 / (2.0 * sigma1 - rho);
      c1[s] = rn * rho;
      c2[s] = 2.0 * rn / dlt;
      rho = rn;
    }
  }
  auto precond = [&](const double* rr, double* zz) -> int {
    if (cheb_degree == 0) {   // plain Jacobi
      cheb_init_kernel<<<gb, 256, 0, ctx->stream>>>(n, rr, kd, 1.0, res, zz, d0);
      RCF_CHECK_LAUNCH(ctx);
      return RCF_OK;
    }
    cheb_init_kernel<<<gb, 256, 0, ctx->stream>>>(n, rr, kd, 1.0 / theta, zz, res, d0);
    RCF_CHECK_LAUNCH(ctx);
    double *dc = d0, *dn = d1;
    for (int s = 0; s < cheb_degree; ++s) {
      RCF_TRY(cheb(ctx, mesh, t, dc, kd, zz, res, dn, c1[s], c2[s]));
      std::swap(dc, dn);
    }
    return RCF_OK;
  };
  auto dots = [&](const double* u, const double* v, const double* c, int i0, int i1) -> int {
    dot_partial_kernel<<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(n, u, v, c, part);
    RCF_CHECK_LAUNCH(ctx);
    dot_final_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, scal, i0, i1);
    RCF_CHECK_LAUNCH(ctx);
    return RCF_OK;
  };
  double gamma = 0.0;
  auto read_gamma = [&]() -> int {
    RCF_CUDA(ctx, cudaMemcpyAsync(&gamma, scal + S_GAMMA, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RCF_OK;
  };
  // r = K x - f; z = P^-1 r; delta = r.z, gamma = r.r; p = -z
  RCF_TRY(lap(ctx, mesh, t, x, r));
  sub_kernel<<<gb, 256, 0, ctx->stream>>>(n, f, r);
  RCF_CHECK_LAUNCH(ctx);
  RCF_TRY(precond(r, z));
  RCF_TRY(dots(r, z, r, S_DELTA, S_GAMMA));
  pcg_direction_kernel<<<gb, 256, 0, ctx->stream>>>(n, scal, z, p, 1);
  RCF_CHECK_LAUNCH(ctx);
  RCF_TRY(read_gamma());
  int it = 0;
  while (std::sqrt(gamma) >= tol && it < maxit) {
    RCF_TRY(lap(ctx, mesh, t, p, w));                       // w = K p
    RCF_TRY(dots(p, w, nullptr, S_ETA, -1));                 // eta = p.w
    pcg_update_kernel<<<gb, 256, 0, ctx->stream>>>(n, scal, p, w, x, r);   // x += alpha p, r += alpha w
    RCF_CHECK_LAUNCH(ctx);
    RCF_TRY(precond(r, z));                                  // z = P^-1 r
    RCF_TRY(dots(r, z, r, S_DNEW, S_GAMMA));                 // (delta_new, gamma)
    pcg_direction_kernel<<<gb, 256, 0, ctx->stream>>>(n, scal, z, p, 0);   // p = -z + beta p
    RCF_CHECK_LAUNCH(ctx);
    pcg_shift_kernel<<<1, 1, 0, ctx->stream>>>(scal);
    RCF_CHECK_LAUNCH(ctx);
    ++it;
    RCF_TRY(read_gamma());
    if (!std::isfinite(gamma)) return fail(ctx, RCF_ECUDA, "PCG residual is not finite at iteration %d", it);
  }
  *iterations = it;
  *residual = std::sqrt(gamma);
  return RCF_OK;
}

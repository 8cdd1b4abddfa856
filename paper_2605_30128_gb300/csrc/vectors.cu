// Elementwise and reduction kernels on column-major complex multivectors:
// mass scalings, the R-ChFSI recovery Y = D^{-1} Z_q + X Lambda_q (Algorithm
// 1), FP64 -> FP32 shadows, column norms, Lanczos vector updates, and the
// node-level bilinear derivative reductions of the adjoint.
#include <type_traits>

#include "internal.h"

namespace rcf {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n, int t = kThreads) { return unsigned((n + t - 1) / t); }

// grid (blocks over rows, nvec); x, y complex: 2 doubles per row
__global__ void scale_mass_kernel(const double* __restrict__ mass, int64_t rows, const double* x,
                                  int64_t ldx, double pw, double* y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const double m = mass[r >> 1];
  double s = 1.0;
  if (pw == 1.0) s = m;
  else if (pw == -1.0) s = 1.0 / m;
  else if (pw == 0.5) s = sqrt(m);
  else if (pw == -0.5) s = 1.0 / sqrt(m);
  const double2 a = reinterpret_cast<const double2*>(x + 2 * int64_t(v) * ldx)[r];
  reinterpret_cast<double2*>(y + 2 * int64_t(v) * ldy)[r] = make_double2(s * a.x, s * a.y);
}

// Y = zs D^{-1} Z + X lam[v]; the D^{-1} Z term in the precision of Z, the rest in FP64
__global__ void recover_kernel_f32(const float* __restrict__ invm, int64_t rows, const float* __restrict__ Z,
                                   int64_t ldz, float zs, const double* __restrict__ X, int64_t ldx,
                                   const double* __restrict__ lam, double* __restrict__ Y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const float d = zs * invm[r >> 1];
  const float2 z = reinterpret_cast<const float2*>(Z + 2 * int64_t(v) * ldz)[r];
  const double2 xv = reinterpret_cast<const double2*>(X + 2 * int64_t(v) * ldx)[r];
  const double l = lam[v];
  reinterpret_cast<double2*>(Y + 2 * int64_t(v) * ldy)[r] =
      make_double2(fma(l, xv.x, double(d * z.x)), fma(l, xv.y, double(d * z.y)));
}

__global__ void recover_kernel_f64(const double* __restrict__ invm, int64_t rows, const double* __restrict__ Z,
                                   int64_t ldz, double zs, const double* __restrict__ X, int64_t ldx,
                                   const double* __restrict__ lam, double* __restrict__ Y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const double d = zs * invm[r >> 1];
  const double2 z = reinterpret_cast<const double2*>(Z + 2 * int64_t(v) * ldz)[r];
  const double2 xv = reinterpret_cast<const double2*>(X + 2 * int64_t(v) * ldx)[r];
  const double l = lam[v];
  reinterpret_cast<double2*>(Y + 2 * int64_t(v) * ldy)[r] = make_double2(fma(d, z.x, l * xv.x), fma(d, z.y, l * xv.y));
}

__global__ void to_c64_kernel(int64_t rows, const double* __restrict__ x, int64_t ldx,
                              float* __restrict__ y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const double2 a = reinterpret_cast<const double2*>(x + 2 * int64_t(v) * ldx)[r];
  reinterpret_cast<float2*>(y + 2 * int64_t(v) * ldy)[r] = make_float2(float(a.x), float(a.y));
}

__global__ void c64_to_c128_kernel(int64_t rows, const float* __restrict__ x, int64_t ldx,
                                   double* __restrict__ y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const float2 a = reinterpret_cast<const float2*>(x + 2 * int64_t(v) * ldx)[r];
  reinterpret_cast<double2*>(y + 2 * int64_t(v) * ldy)[r] = make_double2(a.x, a.y);
}

__global__ void copy_c128_kernel(int64_t rows, const double* __restrict__ x, int64_t ldx,
                                 double* __restrict__ y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  reinterpret_cast<double2*>(y + 2 * int64_t(v) * ldy)[r] =
      reinterpret_cast<const double2*>(x + 2 * int64_t(v) * ldx)[r];
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// block-level sum: registers -> warp shuffle -> shared memory -> one atomic per block
__device__ __forceinline__ void block_atomic_add(double val, double* dst) {
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  val = warp_sum_d(val);
  if (lane == 0) red[wid] = val;
  __syncthreads();
  if (wid == 0) {
    double s = lane < int(blockDim.x >> 5) ? red[lane] : 0.0;
    s = warp_sum_d(s);
    if (lane == 0) atomicAdd(dst, s);
  }
}

// grid (blocks over rows with grid-stride, nvec)
__global__ void colnorm2_kernel(int64_t rows, const double* __restrict__ x, int64_t ldx,
                                double* nrm2) {
  const int v = blockIdx.y;
  const double2* xv = reinterpret_cast<const double2*>(x + 2 * int64_t(v) * ldx);
  double s = 0.0;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows;
       r += int64_t(gridDim.x) * blockDim.x) {
    const double2 a = xv[r];
    s += a.x * a.x + a.y * a.y;
  }
  block_atomic_add(s, nrm2 + v);
}

// per column the largest modulus of any real or imaginary part of a complex64 block, as float
// bits (non-negative floats order like their bit patterns, so atomicMax is exact and the
// result does not depend on the order of the updates); cmax pre-zeroed
__global__ void colmax_f32_kernel(int64_t rows, const float* __restrict__ x, int64_t ldx,
                                  unsigned* __restrict__ cmax) {
  const int v = blockIdx.y;
  const float2* xv = reinterpret_cast<const float2*>(x + 2 * int64_t(v) * ldx);
  float m = 0.f;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows;
       r += int64_t(gridDim.x) * blockDim.x) {
    const float2 a = xv[r];
    m = fmaxf(m, fmaxf(fabsf(a.x), fabsf(a.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(cmax + v, __float_as_uint(m));
}

// scale[v] = 2^e with the column maximum in [2^(e-1), 2^e) (1 for a zero or non-finite
// column), inv[v] = 2^-e: exact scalings, so the scaled values lie in (-1, 1)
__global__ void pow2_scale_kernel(const unsigned* __restrict__ cmax, int n, double* __restrict__ scale,
                                  float* __restrict__ inv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const float m = __uint_as_float(cmax[v]);
  int e = 0;
  if (m > 0.f && m <= 3.4e38f) {
    frexpf(m, &e);   // m = f 2^e, f in [1/2, 1)
    e = e < -120 ? -120 : (e > 120 ? 120 : e);
  }
  scale[v] = ldexp(1.0, e);
  inv[v] = ldexpf(1.0f, -e);
}

// y = x * inv[v], rounded to the storage type
template <typename St>
__global__ void to_storage_kernel(int64_t rows, const float* __restrict__ x, int64_t ldx,
                                  const float* __restrict__ inv, St* __restrict__ y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const float2 a = reinterpret_cast<const float2*>(x + 2 * int64_t(v) * ldx)[r];
  const float s = inv[v];
  St* o = y + 2 * int64_t(v) * ldy + 2 * r;
  if constexpr (std::is_same_v<St, __half>) {
    *reinterpret_cast<__half2*>(o) = __floats2half2_rn(a.x * s, a.y * s);
  } else {
    *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(a.x * s, a.y * s);
  }
}

// Y = D^{-1} Z zscale[v] + X lam[v] with Z stored in a 16-bit type
template <typename St>
__global__ void recover_scaled_kernel(const float* __restrict__ invm, int64_t rows, const St* __restrict__ Z,
                                      int64_t ldz, const double* __restrict__ zscale,
                                      const double* __restrict__ X, int64_t ldx,
                                      const double* __restrict__ lam, double* __restrict__ Y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const St* zp = Z + 2 * int64_t(v) * ldz + 2 * r;
  float2 z;
  if constexpr (std::is_same_v<St, __half>) z = __half22float2(*reinterpret_cast<const __half2*>(zp));
  else z = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(zp));
  const double d = double(invm[r >> 1]) * zscale[v];
  const double2 xv = reinterpret_cast<const double2*>(X + 2 * int64_t(v) * ldx)[r];
  const double l = lam[v];
  reinterpret_cast<double2*>(Y + 2 * int64_t(v) * ldy)[r] =
      make_double2(fma(l, xv.x, d * z.x), fma(l, xv.y, d * z.y));
}

__global__ void sqrt_kernel(double* v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = sqrt(v[i]);
}

__global__ void dot_re_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                              double* out) {
  double s = 0.0;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x) {
    const double2 x = reinterpret_cast<const double2*>(a)[r];
    const double2 y = reinterpret_cast<const double2*>(b)[r];
    s += x.x * y.x + x.y * y.y;
  }
  block_atomic_add(s, out);
}

// w = w - alpha v - beta vprev
__global__ void lanczos_update_kernel(int64_t n, double* w, const double* __restrict__ v,
                                      const double* __restrict__ vprev, double alpha, double beta) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double2 x = reinterpret_cast<double2*>(w)[r];
  const double2 a = reinterpret_cast<const double2*>(v)[r];
  const double2 b = reinterpret_cast<const double2*>(vprev)[r];
  x.x -= alpha * a.x + beta * b.x;
  x.y -= alpha * a.y + beta * b.y;
  reinterpret_cast<double2*>(w)[r] = x;
}

__global__ void scale_vec_kernel(int64_t n, const double* __restrict__ x, double s, double* y) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double2 a = reinterpret_cast<const double2*>(x)[r];
  reinterpret_cast<double2*>(y)[r] = make_double2(s * a.x, s * a.y);
}

// node-level bilinear derivatives, thread per node, loop over vectors (no atomics)
template <typename Real>
__global__ void grad_local_kernel(const double* __restrict__ mass, int64_t nnodes,
                                  const Real* __restrict__ W, int64_t ldw, const Real* __restrict__ U,
                                  int64_t ldu, int nvec, double wgt, int u_dinv,
                                  double* __restrict__ g) {
  const int64_t I = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nnodes) return;
  const double us = u_dinv ? 1.0 / mass[I] : 1.0;
  double s0 = 0, sx = 0, sy = 0, sz = 0;
  for (int v = 0; v < nvec; ++v) {
    const Real* w = W + 2 * (int64_t(v) * ldw) + 4 * I;
    const Real* u = U + 2 * (int64_t(v) * ldu) + 4 * I;
    const double wr = w[0], wi = w[1], xr = w[2], xi = w[3];     // W up, W down
    const double ur = us * u[0], ui = us * u[1], dr = us * u[2], di = us * u[3];
    // Re conj(a) b = ar br + ai bi ; Re conj(a) (i b) = ar (-bi) + ai br
    s0 += wr * ur + wi * ui + xr * dr + xi * di;
    // sigma_x: up <- down, down <- up
    sx += wr * dr + wi * di + xr * ur + xi * ui;
    // sigma_y: up <- -i down, down <- i up
    sy += (wr * di - wi * dr) + (-xr * ui + xi * ur);
    // sigma_z
    sz += wr * ur + wi * ui - xr * dr - xi * di;
  }
  g[I] += wgt * s0;
  g[nnodes + I] += wgt * sx;
  g[2 * nnodes + I] += wgt * sy;
  g[3 * nnodes + I] += wgt * sz;
}

// dV[e][l] += |J| w_l g0[I(e,l)], dB[d][e][l] += |J| w_l g_{1+d}[I(e,l)]
__global__ void grad_to_quadrature_kernel(int nx, int ny, int nz, int p, int Gx, int Gy, int Gz,
                                          const double* __restrict__ wq, int64_t nnodes,
                                          const double* __restrict__ g, double* dV, double* dB) {
  const int np = p + 1, nloc = np * np * np;
  const int64_t ncells = int64_t(nx) * ny * nz;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= ncells * nloc) return;
  const int64_t e = t / nloc;
  const int l = int(t % nloc);
  const int a = l % np, b = (l / np) % np, c = l / (np * np);
  const int ex = int(e % nx), ey = int((e / nx) % ny), ez = int(e / (int64_t(nx) * ny));
  const int i = (ex * p + a) % Gx, j = (ey * p + b) % Gy, k = (ez * p + c) % Gz;
  const int64_t I = i + int64_t(Gx) * (j + int64_t(Gy) * k);
  const double w = wq[l];
  dV[t] += w * g[I];
  const int64_t nq = ncells * nloc;
  dB[t] += w * g[nnodes + I];
  dB[nq + t] += w * g[2 * nnodes + I];
  dB[2 * nq + t] += w * g[3 * nnodes + I];
}

}  // namespace

int launch_scale_mass(rcf_ctx* ctx, const rcf_mesh* m, const double* x, int64_t ldx, int nvec,
                      double pw, double* y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  const int64_t rows = 2 * m->nnodes;
  scale_mass_kernel<<<dim3(blocks_for(rows), nvec), kThreads, 0, ctx->stream>>>(m->d_mass, rows, x,
                                                                                  ldx, pw, y, ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

template <>
int launch_recover<float>(rcf_ctx* ctx, const rcf_mesh* m, const float* Z, int64_t ldz, double zs,
                          const double* X, int64_t ldx, const double* lam, int nvec, double* Y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  const int64_t rows = 2 * m->nnodes;
  recover_kernel_f32<<<dim3(blocks_for(rows), nvec), kThreads, 0, ctx->stream>>>(
      m->d_inv_mass32, rows, Z, ldz, float(zs), X, ldx, lam, Y, ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}
template <>
int launch_recover<double>(rcf_ctx* ctx, const rcf_mesh* m, const double* Z, int64_t ldz, double zs,
                           const double* X, int64_t ldx, const double* lam, int nvec, double* Y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  const int64_t rows = 2 * m->nnodes;
  recover_kernel_f64<<<dim3(blocks_for(rows), nvec), kThreads, 0, ctx->stream>>>(
      m->d_inv_mass64, rows, Z, ldz, zs, X, ldx, lam, Y, ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_to_c64(rcf_ctx* ctx, int64_t rows, const double* x, int64_t ldx, int nvec, float* y,
                  int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  to_c64_kernel<<<dim3(blocks_for(rows), nvec), kThreads, 0, ctx->stream>>>(rows, x, ldx, y, ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_c64_to_c128(rcf_ctx* ctx, int64_t rows, const float* x, int64_t ldx, int nvec,
                       double* y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  c64_to_c128_kernel<<<dim3(blocks_for(rows), nvec), kThreads, 0, ctx->stream>>>(rows, x, ldx, y,
                                                                                  ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_copy_c128(rcf_ctx* ctx, int64_t rows, const double* x, int64_t ldx, int nvec,
                     double* y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  copy_c128_kernel<<<dim3(blocks_for(rows), nvec), kThreads, 0, ctx->stream>>>(rows, x, ldx, y,
                                                                                ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_colmax_f32(rcf_ctx* ctx, int64_t rows, const float* x, int64_t ldx, int nvec, unsigned* cmax) {
  if (nvec <= 0) return RCF_OK;
  const unsigned nb = unsigned(std::min<int64_t>(blocks_for(rows), 152));
  colmax_f32_kernel<<<dim3(nb, nvec), kThreads, 0, ctx->stream>>>(rows, x, ldx, cmax);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_pow2_scale(rcf_ctx* ctx, const unsigned* cmax, int n, double* scale, float* inv) {
  if (n <= 0) return RCF_OK;
  pow2_scale_kernel<<<unsigned((n + 127) / 128), 128, 0, ctx->stream>>>(cmax, n, scale, inv);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

template <typename St>
int launch_to_storage(rcf_ctx* ctx, int64_t rows, const float* x, int64_t ldx, int nvec, const float* inv,
                      St* y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  to_storage_kernel<St><<<dim3(blocks_for(rows), nvec), kThreads, 0, ctx->stream>>>(rows, x, ldx, inv, y, ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}
template int launch_to_storage<__half>(rcf_ctx*, int64_t, const float*, int64_t, int, const float*, __half*, int64_t);
template int launch_to_storage<__nv_bfloat16>(rcf_ctx*, int64_t, const float*, int64_t, int, const float*,
                                              __nv_bfloat16*, int64_t);

template <typename St>
int launch_recover_scaled(rcf_ctx* ctx, const rcf_mesh* m, const St* Z, int64_t ldz, const double* zscale,
                          const double* X, int64_t ldx, const double* lam, int nvec, double* Y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  const int64_t rows = 2 * m->nnodes;
  recover_scaled_kernel<St><<<dim3(blocks_for(rows), nvec), kThreads, 0, ctx->stream>>>(
      m->d_inv_mass32, rows, Z, ldz, zscale, X, ldx, lam, Y, ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}
template int launch_recover_scaled<__half>(rcf_ctx*, const rcf_mesh*, const __half*, int64_t, const double*,
                                           const double*, int64_t, const double*, int, double*, int64_t);
template int launch_recover_scaled<__nv_bfloat16>(rcf_ctx*, const rcf_mesh*, const __nv_bfloat16*, int64_t,
                                                  const double*, const double*, int64_t, const double*, int,
                                                  double*, int64_t);

int launch_colnorm2(rcf_ctx* ctx, int64_t rows, const double* x, int64_t ldx, int nvec,
                    double* nrm2) {
  if (nvec <= 0) return RCF_OK;
  const unsigned nb = unsigned(std::min<int64_t>(blocks_for(rows), 152));
  colnorm2_kernel<<<dim3(nb, nvec), kThreads, 0, ctx->stream>>>(rows, x, ldx, nrm2);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_sqrt_inplace(rcf_ctx* ctx, double* v, int n) {
  if (n <= 0) return RCF_OK;
  sqrt_kernel<<<blocks_for(n), kThreads, 0, ctx->stream>>>(v, n);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_dot_re(rcf_ctx* ctx, int64_t n, const double* a, const double* b, double* out) {
  const unsigned nb = unsigned(std::min<int64_t>(blocks_for(n), 304));
  dot_re_kernel<<<nb, kThreads, 0, ctx->stream>>>(n, a, b, out);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_lanczos_update(rcf_ctx* ctx, int64_t n, double* w, const double* v,
                          const double* vprev, double alpha, double beta) {
  lanczos_update_kernel<<<blocks_for(n), kThreads, 0, ctx->stream>>>(n, w, v, vprev, alpha, beta);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

int launch_scale_vec(rcf_ctx* ctx, int64_t n, const double* x, double s, double* y) {
  scale_vec_kernel<<<blocks_for(n), kThreads, 0, ctx->stream>>>(n, x, s, y);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

template <typename Real>
int launch_grad_local(rcf_ctx* ctx, const rcf_mesh* m, const Real* W, int64_t ldw, const Real* U,
                      int64_t ldu, int nvec, double wgt, int u_dinv, double* gnode) {
  if (nvec <= 0) return RCF_OK;
  grad_local_kernel<Real><<<blocks_for(m->nnodes), kThreads, 0, ctx->stream>>>(
      m->d_mass, m->nnodes, W, ldw, U, ldu, nvec, wgt, u_dinv, gnode);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}
template int launch_grad_local<float>(rcf_ctx*, const rcf_mesh*, const float*, int64_t,
                                      const float*, int64_t, int, double, int, double*);
template int launch_grad_local<double>(rcf_ctx*, const rcf_mesh*, const double*, int64_t,
                                       const double*, int64_t, int, double, int, double*);

int launch_grad_to_quadrature(rcf_ctx* ctx, const rcf_mesh* m, const double* gnode, double* dV,
                              double* dB) {
  // quadrature weights w_l |J| in a small scratch buffer
  double* wq = nullptr;
  RCF_TRY(workspace(ctx, WS_COEF, sizeof(double) * m->nloc, reinterpret_cast<void**>(&wq)));
  std::vector<double> h(m->nloc);
  for (int c = 0; c < m->np; ++c)
    for (int b = 0; b < m->np; ++b)
      for (int a = 0; a < m->np; ++a)
        h[a + m->np * (b + m->np * c)] = m->w[a] * m->w[b] * m->w[c] * m->detJ;
  RCF_CUDA(ctx, cudaMemcpyAsync(wq, h.data(), sizeof(double) * m->nloc, cudaMemcpyHostToDevice,
                                ctx->stream));
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // h is a stack buffer
  const int64_t n = m->ncells * m->nloc;
  grad_to_quadrature_kernel<<<blocks_for(n), kThreads, 0, ctx->stream>>>(
      m->n[0], m->n[1], m->n[2], m->p, m->G[0], m->G[1], m->G[2], wq, m->nnodes, gnode, dV, dB);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

}  // namespace rcf

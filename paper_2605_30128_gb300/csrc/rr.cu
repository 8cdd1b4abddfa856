// Cholesky-QR2 and the Rayleigh-Ritz step in FP64 (Algorithm 1, RR step; Section III-C-4).
//
// The Gram matrix S = Y^H M Y is accumulated over row chunks as a Hermitian
// rank-k update of W = M^{1/2} Y (ZHERK), factorised S = L L^H (ZPOTRF) and
// applied as Y <- Y L^{-H} (ZTRSM); twice.  A non-positive pivot triggers one
// shifted pass (shifted Cholesky-QR) before giving up with RCF_ENOTSPD.  The
// projected matrix A = Y^H H Y is formed from column chunks of H Y (the
// library's own matrix-free product) with ZGEMM, diagonalised by ZHEEVD, and
// the rotation X = Y Q is one ZGEMM.  These are plain dense library
// routines; the problem-specific work (H Y, the M weighting) runs in this
// library's kernels.
#include <algorithm>
#include <cmath>
#include <tuple>
#include <vector>

#include "internal.h"

namespace rcf {
namespace {

__global__ void sqrt_mass_rows_kernel(const double* __restrict__ mass, const double* __restrict__ Y,
                                      int64_t ldy, int64_t r0, int64_t cr, double* __restrict__ W) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= cr) return;
  const double s = sqrt(mass[(r0 + r) >> 1]);
  const double2 y = reinterpret_cast<const double2*>(Y + 2 * int64_t(v) * ldy)[r0 + r];
  reinterpret_cast<double2*>(W + 2 * int64_t(v) * cr)[r] = make_double2(s * y.x, s * y.y);
}

const char* cublas_name(cublasStatus_t s) {
  switch (s) {
    case CUBLAS_STATUS_SUCCESS: return "success";
    case CUBLAS_STATUS_NOT_INITIALIZED: return "not initialized";
    case CUBLAS_STATUS_ALLOC_FAILED: return "alloc failed";
    case CUBLAS_STATUS_INVALID_VALUE: return "invalid value";
    case CUBLAS_STATUS_EXECUTION_FAILED: return "execution failed";
    default: return "error";
  }
}

#define RCF_BLAS(ctx, expr)                                                                  \
  do {                                                                                       \
    cublasStatus_t _s = (expr);                                                              \
    if (_s != CUBLAS_STATUS_SUCCESS)                                                         \
      return fail((ctx), RCF_ECUDA, "cuBLAS %s failed: %s", #expr, cublas_name(_s));         \
  } while (0)
#define RCF_SOLVER(ctx, expr)                                                                \
  do {                                                                                       \
    cusolverStatus_t _s = (expr);                                                            \
    if (_s != CUSOLVER_STATUS_SUCCESS)                                                       \
      return fail((ctx), RCF_ECUDA, "cuSOLVER %s failed: status %d", #expr, int(_s));        \
  } while (0)

// W[v][r] = w_I Y[v][r0 + r], I = (r0 + r) / 2 (w null: copy), for complex rows r < cr
__global__ void weight_rows_kernel(const double* __restrict__ w, const double* __restrict__ Y, int64_t ldy,
                                   int64_t r0, int64_t cr, double* __restrict__ W) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= cr) return;
  const double s = w ? w[(r0 + r) >> 1] : 1.0;
  const double2 y = reinterpret_cast<const double2*>(Y + 2 * int64_t(v) * ldy)[r0 + r];
  reinterpret_cast<double2*>(W + 2 * int64_t(v) * cr)[r] = make_double2(s * y.x, s * y.y);
}

// C (n x nz, ldc) = Y^H diag(w) Z in the given arithmetic; lower: Z == Y and only C(i, j),
// i >= j, is needed (the Hermitian Gram matrix)
int inner_product(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Z, int64_t ldz, int nz,
                  int64_t nrows, const double* w, double* C, int64_t ldc, int arith, int lower) {
  if (arith == RCF_RR_TC || arith == RCF_RR_MIXED) return tc_gemm_tn(ctx, Y, ldy, n, w, Z, ldz, nz, nrows, C, ldc, lower);
  if (arith == RCF_RR_DF) {
    if (ldc != n) return fail(ctx, RCF_ENOTSUP, "double-float products need ldc == n");
    return launch_gemm_tn_df(ctx, Y, ldy, Z, ldz, w, nrows, n, nz, lower && Z == Y && nz == n, C, ldc);
  }
  if (nrows > INT32_MAX || ldy > INT32_MAX || ldz > INT32_MAX || ldc > INT32_MAX)
    return fail(ctx, RCF_ENOTSUP, "dimensions above 2^31 are not supported by the BLAS path");
  int64_t cr = std::max<int64_t>(1024, (int64_t(1) << 26) / std::max(nz, 1));   // ~1 GiB chunks
  cr = std::min<int64_t>(cr, nrows);
  double* W = nullptr;
  const bool herk = lower && Z == Y && nz == n && w != nullptr;
  const int wc = herk ? n : nz;
  RCF_TRY(workspace(ctx, WS_RR_W, sizeof(double) * 2 * size_t(cr) * wc, reinterpret_cast<void**>(&W)));
  const double one = 1.0, zero = 0.0;
  const cuDoubleComplex onec = make_cuDoubleComplex(1.0, 0.0), zeroc = make_cuDoubleComplex(0.0, 0.0);
  auto* Cz = reinterpret_cast<cuDoubleComplex*>(C);
  for (int64_t r0 = 0; r0 < nrows; r0 += cr) {
    const int64_t c = std::min(cr, nrows - r0);
    if (herk) {   // W = M^{1/2} Y, S = W^H W
      sqrt_mass_rows_kernel<<<dim3(unsigned((c + 255) / 256), n), 256, 0, ctx->stream>>>(w, Y, ldy, r0, c, W);
      RCF_CHECK_LAUNCH(ctx);
      RCF_BLAS(ctx, cublasZherk(ctx->blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_C, n, int(c), &one,
                                reinterpret_cast<const cuDoubleComplex*>(W), int(c), r0 == 0 ? &zero : &one, Cz,
                                int(ldc)));
    } else {
      weight_rows_kernel<<<dim3(unsigned((c + 255) / 256), nz), 256, 0, ctx->stream>>>(w, Z, ldz, r0, c, W);
      RCF_CHECK_LAUNCH(ctx);
      RCF_BLAS(ctx, cublasZgemm(ctx->blas, CUBLAS_OP_C, CUBLAS_OP_N, n, nz, int(c), &onec,
                                reinterpret_cast<const cuDoubleComplex*>(Y + 2 * r0), int(ldy),
                                reinterpret_cast<const cuDoubleComplex*>(W), int(c), r0 == 0 ? &zeroc : &onec, Cz,
                                int(ldc)));
    }
  }
  return RCF_OK;
}

// X = Y Q (n x n complex Q, ldq) in the given arithmetic; TC allows X == Y
int rotate(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Q, int64_t ldq, int64_t nrows,
           double* X, int64_t ldx, int arith) {
  if (arith == RCF_RR_TC) return tc_rotate(ctx, Y, ldy, n, Q, ldq, nrows, X, ldx);
  if (arith == RCF_RR_MIXED) return tc_rotate(ctx, Y, ldy, n, Q, ldq, nrows, X, ldx, true);
  if (nrows > INT32_MAX || ldy > INT32_MAX || ldx > INT32_MAX)
    return fail(ctx, RCF_ENOTSUP, "dimensions above 2^31 are not supported by the BLAS path");
  const char* x0 = reinterpret_cast<const char*>(X);
  const char* y0 = reinterpret_cast<const char*>(Y);
  if (x0 < y0 + size_t(ldy) * n * 16 && y0 < x0 + size_t(ldx) * n * 16)
    return fail(ctx, RCF_EINVAL, "the FP64 rotation cannot write over its input");
  const cuDoubleComplex onec = make_cuDoubleComplex(1.0, 0.0), zeroc = make_cuDoubleComplex(0.0, 0.0);
  RCF_BLAS(ctx, cublasZgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, int(nrows), n, n, &onec,
                            reinterpret_cast<const cuDoubleComplex*>(Y), int(ldy),
                            reinterpret_cast<const cuDoubleComplex*>(Q), int(ldq), &zeroc,
                            reinterpret_cast<cuDoubleComplex*>(X), int(ldx)));
  return RCF_OK;
}

// U(i, j) = conj(Linv(j, i)) for i <= j, 0 below: U = L^{-H} from the lower factor Linv = L^{-1}
__global__ void inverse_adjoint_kernel(const double* __restrict__ Li, int n, double* __restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  double2 v = make_double2(0.0, 0.0);
  if (i <= j) {
    const double2 l = reinterpret_cast<const double2*>(Li)[j + int64_t(i) * n];
    v = make_double2(l.x, -l.y);
  }
  reinterpret_cast<double2*>(U)[i + int64_t(j) * n] = v;
}

// S = Y^H M Y  (lower triangle), S: n x n
int gram(rcf_ctx* ctx, const rcf_op* op, const double* Y, int64_t ldy, int n, cuDoubleComplex* S) {
  const int64_t N = 2 * op->mesh->nnodes;
  if (op->fm) {   // the full consistent mass: S = Y^H (M Y), column chunks of M Y
    const int cb = std::min(n, 256);
    double* T = nullptr;
    RCF_TRY(workspace(ctx, WS_RR_T, sizeof(double) * 2 * size_t(N) * cb, reinterpret_cast<void**>(&T)));
    for (int c0 = 0; c0 < n; c0 += cb) {
      const int nc = std::min(cb, n - c0);
      RCF_TRY(mass_apply_fm<double>(ctx, op, Y + 2 * int64_t(c0) * ldy, ldy, nc, T, N));
      RCF_TRY(inner_product(ctx, Y, ldy, n, T, N, nc, N, nullptr, reinterpret_cast<double*>(S + size_t(c0) * n), n,
                            ctx->rr_arith, 0));
    }
    return RCF_OK;
  }
  return inner_product(ctx, Y, ldy, n, Y, ldy, n, N, op->mesh->d_mass, reinterpret_cast<double*>(S), n,
                       ctx->rr_arith, 1);
}

// one Cholesky-QR pass; returns RCF_ENOTSPD (without touching Y) on breakdown unless shifted
int cholqr_pass(rcf_ctx* ctx, const rcf_op* op, double* Y, int64_t ldy, int n, bool shift) {
  const int64_t N = 2 * op->mesh->nnodes;
  cuDoubleComplex* S = nullptr;
  int* info = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_S, sizeof(cuDoubleComplex) * size_t(n) * n, reinterpret_cast<void**>(&S)));
  RCF_TRY(workspace(ctx, WS_RR_INFO, sizeof(int) * 4, reinterpret_cast<void**>(&info)));
  RCF_TRY(gram(ctx, op, Y, ldy, n, S));
  if (shift) {
    // shifted Cholesky-QR: S += 11 (N n + n (n + 1)) u tr(S) I   (tr(S) >= ||S||_2 for SPD S)
    std::vector<cuDoubleComplex> h(size_t(n) * n);
    RCF_CUDA(ctx, cudaMemcpyAsync(h.data(), S, sizeof(cuDoubleComplex) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += h[size_t(i) * n + i].x;
    const double sh = 11.0 * (double(N) * n + double(n) * (n + 1)) * 1.1102230246251565e-16 * tr;
    for (int i = 0; i < n; ++i) h[size_t(i) * n + i].x += sh;
    RCF_CUDA(ctx, cudaMemcpyAsync(S, h.data(), sizeof(cuDoubleComplex) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  int lwork = 0;
  RCF_SOLVER(ctx, cusolverDnZpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, S, n, &lwork));
  cuDoubleComplex* work = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_WORK, sizeof(cuDoubleComplex) * size_t(std::max(lwork, 1)), reinterpret_cast<void**>(&work)));
  RCF_SOLVER(ctx, cusolverDnZpotrf(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, S, n, work, lwork, info));
  int hinfo = 0;
  std::vector<cuDoubleComplex> diag(n);   // the factor's diagonal: a NaN in Y leaves it non-finite
  RCF_CUDA(ctx, cudaMemcpy2DAsync(diag.data(), sizeof(cuDoubleComplex), S, sizeof(cuDoubleComplex) * (n + 1),
                                  sizeof(cuDoubleComplex), n, cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hinfo != 0)
    return fail(ctx, RCF_ENOTSPD, "Cholesky-QR: Gram matrix not positive definite (pivot %d)", hinfo);
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(diag[i].x) || !(diag[i].x > 0.0))
      return fail(ctx, RCF_ENOTSPD, "Cholesky-QR: Gram factor not finite and positive (column %d)", i + 1);
  if (ctx->rr_arith == RCF_RR_TC || ctx->rr_arith == RCF_RR_MIXED) {
    // Y <- Y L^{-H}: invert the n x n factor (TRTRI), apply its adjoint as a rotation in place
    size_t dbytes = 0, hbytes = 0;
    RCF_SOLVER(ctx, cusolverDnXtrtri_bufferSize(ctx->solver, CUBLAS_FILL_MODE_LOWER, CUBLAS_DIAG_NON_UNIT, n,
                                                CUDA_C_64F, S, n, &dbytes, &hbytes));
    void* dwork = nullptr;
    RCF_TRY(workspace(ctx, WS_RR_WORK, std::max<size_t>(dbytes, 16), &dwork));
    std::vector<unsigned char> hwork(std::max<size_t>(hbytes, 16));
    RCF_SOLVER(ctx, cusolverDnXtrtri(ctx->solver, CUBLAS_FILL_MODE_LOWER, CUBLAS_DIAG_NON_UNIT, n, CUDA_C_64F, S,
                                     n, dwork, dbytes, hwork.data(), hbytes, info));
    double* U = nullptr;
    RCF_TRY(workspace(ctx, WS_TC_Q, sizeof(cuDoubleComplex) * size_t(n) * n, reinterpret_cast<void**>(&U)));
    inverse_adjoint_kernel<<<dim3(unsigned((n + 127) / 128), n), 128, 0, ctx->stream>>>(
        reinterpret_cast<const double*>(S), n, U);
    RCF_CHECK_LAUNCH(ctx);
    RCF_TRY(tc_rotate(ctx, Y, ldy, n, U, n, N, Y, ldy));
    RCF_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // hwork is host memory of this frame
    if (hinfo != 0) return fail(ctx, RCF_ENOTSPD, "Cholesky-QR: triangular factor singular (%d)", hinfo);
    return RCF_OK;
  }
  const cuDoubleComplex onec = make_cuDoubleComplex(1.0, 0.0);
  RCF_BLAS(ctx, cublasZtrsm(ctx->blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_C,
                            CUBLAS_DIAG_NON_UNIT, int(N), n, &onec, S, n,
                            reinterpret_cast<cuDoubleComplex*>(Y), int(ldy)));
  return RCF_OK;
}

}  // namespace
}  // namespace rcf

using namespace rcf;

namespace rcf {
namespace {

int check_y(rcf_ctx* ctx, const rcf_op* op, const double* Y, int64_t ldy, int nvec) {
  const int64_t N = 2 * op->mesh->nnodes;
  if (nvec <= 0) return fail(ctx, RCF_EINVAL, "nvec must be >= 1");
  if (!Y) return fail(ctx, RCF_EINVAL, "NULL argument");
  if (ldy < N || (ldy & 1)) return fail(ctx, RCF_EINVAL, "bad leading dimension");
  if (ldy > INT32_MAX || N > INT32_MAX)
    return fail(ctx, RCF_ENOTSUP, "leading dimensions above 2^31 are not supported by the BLAS path");
  return RCF_OK;
}

// Cholesky-QR2, with one shifted pass in front if the first factorisation breaks down
int cholqr2(rcf_ctx* ctx, const rcf_op* op, double* Y, int64_t ldy, int nvec) {
  int s = cholqr_pass(ctx, op, Y, ldy, nvec, false);
  if (s == RCF_ENOTSPD) {
    RCF_TRY(cholqr_pass(ctx, op, Y, ldy, nvec, true));
    RCF_TRY(cholqr_pass(ctx, op, Y, ldy, nvec, false));
  } else if (s != RCF_OK) {
    return s;
  }
  return cholqr_pass(ctx, op, Y, ldy, nvec, false);
}

// projection, eigensolve and rotation for an M-orthonormal Y
int rr_orth(rcf_ctx* ctx, const rcf_op* op, const double* Y, int64_t ldy, int nvec, double* X_out,
            int64_t ldx, double* ritz_out) {
  const int64_t N = 2 * op->mesh->nnodes;
  // A = Y^H H Y, column chunks of H Y
  cuDoubleComplex* A = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_S, sizeof(cuDoubleComplex) * size_t(nvec) * nvec, reinterpret_cast<void**>(&A)));
  const int cb = std::min(nvec, 256);
  double* T = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_T, sizeof(double) * 2 * size_t(N) * cb, reinterpret_cast<void**>(&T)));
  for (int c0 = 0; c0 < nvec; c0 += cb) {
    const int nc = std::min(cb, nvec - c0);
    RCF_TRY(rcf_apply(ctx, op, RCF_FORM_H, Y + 2 * int64_t(c0) * ldy, ldy, nc, T, N, RCF_FP64));
    RCF_TRY(inner_product(ctx, Y, ldy, nvec, T, N, nc, N, nullptr, reinterpret_cast<double*>(A + size_t(c0) * nvec),
                          nvec, ctx->rr_arith, 0));
  }
  double* w = nullptr;
  int* info = nullptr;
  RCF_TRY(workspace(ctx, WS_NORM, sizeof(double) * nvec, reinterpret_cast<void**>(&w)));
  RCF_TRY(workspace(ctx, WS_RR_INFO, sizeof(int) * 4, reinterpret_cast<void**>(&info)));
  int lwork = 0;
  RCF_SOLVER(ctx, cusolverDnZheevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                              nvec, A, nvec, w, &lwork));
  cuDoubleComplex* work = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_WORK, sizeof(cuDoubleComplex) * size_t(std::max(lwork, 1)), reinterpret_cast<void**>(&work)));
  RCF_SOLVER(ctx, cusolverDnZheevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nvec, A,
                                   nvec, w, work, lwork, info));
  RCF_TRY(rotate(ctx, Y, ldy, nvec, reinterpret_cast<const double*>(A), nvec, N, X_out, ldx,
                 ctx->rr_arith == RCF_RR_DF ? RCF_RR_FP64 : ctx->rr_arith));
  int hinfo = 0;
  RCF_CUDA(ctx, cudaMemcpyAsync(ritz_out, w, sizeof(double) * nvec, cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hinfo != 0) return fail(ctx, RCF_ECUDA, "ZHEEVD did not converge (info %d)", hinfo);
  return RCF_OK;
}

int check_xy(rcf_ctx* ctx, const rcf_op* op, const double* Y, int64_t ldy, int nvec, const double* X_out,
             int64_t ldx, const double* ritz_out) {
  RCF_TRY(check_y(ctx, op, Y, ldy, nvec));
  const int64_t N = 2 * op->mesh->nnodes;
  if (!X_out || !ritz_out) return fail(ctx, RCF_EINVAL, "NULL argument");
  if (ldx < N || (ldx & 1)) return fail(ctx, RCF_EINVAL, "bad leading dimension");
  if (ldx > INT32_MAX) return fail(ctx, RCF_ENOTSUP, "leading dimensions above 2^31 are not supported by the BLAS path");
  const char* y0 = reinterpret_cast<const char*>(Y);
  const char* x0 = reinterpret_cast<const char*>(X_out);
  if (y0 < x0 + size_t(ldx) * nvec * 16 && x0 < y0 + size_t(ldy) * nvec * 16)
    return fail(ctx, RCF_EINVAL, "X_out overlaps Y");
  return RCF_OK;
}

}  // namespace
}  // namespace rcf

extern "C" int rcf_cholqr2(rcf_ctx* ctx, const rcf_op* op, double* Y, int64_t ldy, int nvec) {
  if (!ctx || !op) return RCF_EINVAL;
  RCF_TRY(check_y(ctx, op, Y, ldy, nvec));
  RCF_TRY(cholqr2(ctx, op, Y, ldy, nvec));
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RCF_OK;
}

extern "C" int rcf_rayleigh_ritz_orth(rcf_ctx* ctx, const rcf_op* op, const double* Y, int64_t ldy, int nvec,
                                      double* X_out, int64_t ldx, double* ritz_out) {
  if (!ctx || !op) return RCF_EINVAL;
  RCF_TRY(check_xy(ctx, op, Y, ldy, nvec, X_out, ldx, ritz_out));
  return rr_orth(ctx, op, Y, ldy, nvec, X_out, ldx, ritz_out);
}

extern "C" int rcf_rayleigh_ritz(rcf_ctx* ctx, const rcf_op* op, double* Y, int64_t ldy, int nvec,
                                 double* X_out, int64_t ldx, double* ritz_out) {
  if (!ctx || !op) return RCF_EINVAL;
  RCF_TRY(check_xy(ctx, op, Y, ldy, nvec, X_out, ldx, ritz_out));
  RCF_TRY(cholqr2(ctx, op, Y, ldy, nvec));
  return rr_orth(ctx, op, Y, ldy, nvec, X_out, ldx, ritz_out);
}

// ---------------------------------------------------------------------------
// cotangent of the Ritz values (no counterpart in the paper)
// ---------------------------------------------------------------------------
namespace rcf {
namespace {

// y[v][r] = s[v] x[v][r] (complex rows r < rows)
__global__ void scale_cols_kernel(int64_t rows, const double* __restrict__ x, int64_t ldx,
                                  const double* __restrict__ s, double* __restrict__ y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const double2 a = reinterpret_cast<const double2*>(x + 2 * int64_t(v) * ldx)[r];
  reinterpret_cast<double2*>(y + 2 * int64_t(v) * ldy)[r] = make_double2(s[v] * a.x, s[v] * a.y);
}

}  // namespace
}  // namespace rcf

extern "C" int rcf_ritz_cotangent(rcf_ctx* ctx, const rcf_op* op, const double* Y, int64_t ldy,
                                  const double* X, int64_t ldx, int nvec, const double* theta,
                                  const double* thetabar, double* Ybar, int64_t ldb, double* dV,
                                  double* dB, double* dh) {
  if (!ctx || !op) return RCF_EINVAL;
  if (op->fm) return fail(ctx, RCF_ENOTSUP, "the Ritz cotangent is not available with the full consistent mass");
  RCF_TRY(check_y(ctx, op, Y, ldy, nvec));
  RCF_TRY(check_y(ctx, op, X, ldx, nvec));
  RCF_TRY(check_y(ctx, op, Ybar, ldb, nvec));
  if (!theta || !thetabar) return fail(ctx, RCF_EINVAL, "theta and thetabar must be host arrays");
  if ((dV == nullptr) != (dB == nullptr)) return fail(ctx, RCF_EINVAL, "dV and dB must both be given or both NULL");
  const int n = nvec;
  const int64_t N = 2 * op->mesh->nnodes;
  auto overl = [&](const double* a, int64_t la, const double* b, int64_t lb) {
    const char* a0 = reinterpret_cast<const char*>(a);
    const char* b0 = reinterpret_cast<const char*>(b);
    return a0 < b0 + size_t(lb) * n * 16 && b0 < a0 + size_t(la) * n * 16;
  };
  if (overl(Ybar, ldb, Y, ldy) || overl(Ybar, ldb, X, ldx)) return fail(ctx, RCF_EINVAL, "Ybar overlaps Y or X");
  // S = Y^H M Y and T = Y^H M X (n x n); Q = S^-1 T, so that X = Y Q
  cuDoubleComplex *S = nullptr, *T = nullptr, *Cm = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_S, sizeof(cuDoubleComplex) * 3 * size_t(n) * n, reinterpret_cast<void**>(&S)));
  T = S + size_t(n) * n;
  Cm = T + size_t(n) * n;
  RCF_TRY(inner_product(ctx, Y, ldy, n, Y, ldy, n, N, op->mesh->d_mass, reinterpret_cast<double*>(S), n,
                        ctx->rr_arith, 0));
  RCF_TRY(inner_product(ctx, Y, ldy, n, X, ldx, n, N, op->mesh->d_mass, reinterpret_cast<double*>(T), n,
                        ctx->rr_arith, 0));
  int* info = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_INFO, sizeof(int) * 4, reinterpret_cast<void**>(&info)));
  int lwork = 0;
  RCF_SOLVER(ctx, cusolverDnZpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, S, n, &lwork));
  cuDoubleComplex* work = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_WORK, sizeof(cuDoubleComplex) * size_t(std::max(lwork, 1)), reinterpret_cast<void**>(&work)));
  RCF_SOLVER(ctx, cusolverDnZpotrf(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, S, n, work, lwork, info));
  int hinfo = 0;
  RCF_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hinfo != 0) return fail(ctx, RCF_ENOTSPD, "Ritz cotangent: Y^H M Y not positive definite (pivot %d)", hinfo);
  RCF_SOLVER(ctx, cusolverDnZpotrs(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, n, S, n, T, n, info));
  // Cm[j][i] = 2 thetabar_j conj(Q[i][j])  (column-major: Cm(j, i) at j + i n)
  std::vector<cuDoubleComplex> Qh(size_t(n) * n), Ch(size_t(n) * n);
  RCF_CUDA(ctx, cudaMemcpyAsync(Qh.data(), T, sizeof(cuDoubleComplex) * Qh.size(), cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hinfo != 0) return fail(ctx, RCF_ECUDA, "ZPOTRS failed (info %d)", hinfo);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const cuDoubleComplex q = Qh[size_t(j) * n + i];   // Q(i, j)
      Ch[size_t(i) * n + j] = make_cuDoubleComplex(2.0 * thetabar[j] * q.x, -2.0 * thetabar[j] * q.y);
    }
  RCF_CUDA(ctx, cudaMemcpyAsync(Cm, Ch.data(), sizeof(cuDoubleComplex) * Ch.size(), cudaMemcpyHostToDevice, ctx->stream));
  // Ybar = sum over column chunks of (H - theta M) X_chunk  Cm[chunk rows, :]
  const int cb = std::min(n, 256);
  double* Rx = nullptr;
  RCF_TRY(workspace(ctx, WS_RR_T, sizeof(double) * 2 * size_t(N) * cb, reinterpret_cast<void**>(&Rx)));
  double* sc = nullptr;
  if (dV) {
    RCF_TRY(workspace(ctx, WS_NORM, sizeof(double) * n, reinterpret_cast<void**>(&sc)));
    RCF_CUDA(ctx, cudaMemcpyAsync(sc, thetabar, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  }
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  for (int c0 = 0; c0 < n; c0 += cb) {
    const int nc = std::min(cb, n - c0);
    RCF_TRY(rcf_residual(ctx, op, X + 2 * int64_t(c0) * ldx, ldx, nc, theta + c0, Rx, N, nullptr));
    RCF_BLAS(ctx, cublasZgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, int(N), n, nc, &one,
                              reinterpret_cast<const cuDoubleComplex*>(Rx), int(N), Cm + c0, n,
                              c0 == 0 ? &zero : &one, reinterpret_cast<cuDoubleComplex*>(Ybar), int(ldb)));
    if (dV) {
      // direct term: sum_j thetabar_j x_j^H dH x_j, with W = X_chunk diag(thetabar) written
      // over Rx (stream order puts it after the product that read Rx)
      scale_cols_kernel<<<dim3(unsigned((N + 255) / 256), nc), 256, 0, ctx->stream>>>(
          N, X + 2 * int64_t(c0) * ldx, ldx, sc + c0, Rx, N);
      RCF_CHECK_LAUNCH(ctx);
      RCF_TRY(rcf_grad_bilinear(ctx, op, Rx, N, X + 2 * int64_t(c0) * ldx, ldx, nc, 1.0, dV, dB, dh));
    }
  }
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RCF_OK;
}

extern "C" int rcf_inner(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Z, int64_t ldz, int nz,
                         int64_t nrows, const double* w, double* C, int64_t ldc, int arith) {
  if (!ctx) return RCF_EINVAL;
  if (!Y || !Z || !C) return fail(ctx, RCF_EINVAL, "NULL argument");
  if (n <= 0 || nz <= 0 || nrows <= 0) return fail(ctx, RCF_EINVAL, "sizes must be >= 1");
  if (ldy < nrows || ldz < nrows || (ldy & 1) || (ldz & 1) || ldc < n)
    return fail(ctx, RCF_EINVAL, "bad leading dimension");
  if (w && (nrows & 1)) return fail(ctx, RCF_EINVAL, "a node weight needs an even number of rows");
  if (arith != RCF_RR_FP64 && arith != RCF_RR_DF && arith != RCF_RR_TC && arith != RCF_RR_MIXED)
    return fail(ctx, RCF_EINVAL, "unknown arithmetic %d", arith);
  if (((reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(Z) | reinterpret_cast<uintptr_t>(C)) & 15) != 0)
    return fail(ctx, RCF_EINVAL, "buffers must be 16-byte aligned");
  const char* c0 = reinterpret_cast<const char*>(C);
  const size_t cb = size_t(ldc) * nz * 16;
  for (auto [p, ld, m] : {std::tuple<const double*, int64_t, int>{Y, ldy, n}, {Z, ldz, nz}}) {
    const char* p0 = reinterpret_cast<const char*>(p);
    if (c0 < p0 + size_t(ld) * m * 16 && p0 < c0 + cb) return fail(ctx, RCF_EINVAL, "C overlaps an input");
  }
  return inner_product(ctx, Y, ldy, n, Z, ldz, nz, nrows, w, C, ldc, arith, 0);
}

extern "C" int rcf_rotate(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Q, int64_t ldq,
                          int64_t nrows, double* X, int64_t ldx, int arith) {
  if (!ctx) return RCF_EINVAL;
  if (!Y || !Q || !X) return fail(ctx, RCF_EINVAL, "NULL argument");
  if (n <= 0 || nrows <= 0) return fail(ctx, RCF_EINVAL, "sizes must be >= 1");
  if (ldy < nrows || ldx < nrows || (ldy & 1) || (ldx & 1) || ldq < n)
    return fail(ctx, RCF_EINVAL, "bad leading dimension");
  if (arith != RCF_RR_FP64 && arith != RCF_RR_TC && arith != RCF_RR_MIXED)
    return fail(ctx, RCF_EINVAL, "unknown arithmetic %d", arith);
  if (((reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(Q) | reinterpret_cast<uintptr_t>(X)) & 15) != 0)
    return fail(ctx, RCF_EINVAL, "buffers must be 16-byte aligned");
  const char* q0 = reinterpret_cast<const char*>(Q);
  const char* x0 = reinterpret_cast<const char*>(X);
  if (q0 < x0 + size_t(ldx) * n * 16 && x0 < q0 + size_t(ldq) * n * 16) return fail(ctx, RCF_EINVAL, "X overlaps Q");
  return rotate(ctx, Y, ldy, n, Q, ldq, nrows, X, ldx, arith);
}

// Host drivers: Hamiltonian-multivector products, the FP64 residual, the
// ChFSI / R-ChFSI filters (Section III-B-2), the Lanczos bound, and the
// checkpointed reverse-mode filter derivative.
#include <algorithm>
#include <cmath>
#include <vector>

#include <type_traits>

#include "internal.h"

namespace rcf {
namespace {

template <typename Real>
const Real* pot_of(const rcf_op* op);
template <>
const double* pot_of<double>(const rcf_op* op) { return op->d_pot64; }
template <>
const float* pot_of<float>(const rcf_op* op) { return op->d_pot32; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_block(rcf_ctx* ctx, const rcf_op* op, const void* p, int64_t ld, int nvec, size_t real,
                const char* name) {
  const int64_t rows = 2 * op->mesh->nnodes;
  if (nvec < 0) return fail(ctx, RCF_EINVAL, "%s: nvec < 0", name);
  if (nvec == 0) return RCF_OK;
  if (!p) return fail(ctx, RCF_EINVAL, "%s is NULL", name);
  if (ld < rows || (ld & 1)) return fail(ctx, RCF_EINVAL, "%s: ld=%lld must be even and >= 2M=%lld", name, (long long)ld, (long long)rows);
  if (!aligned(p, 4 * real)) return fail(ctx, RCF_EINVAL, "%s: base must be %zu-byte aligned", name, 4 * real);
  return RCF_OK;
}

constexpr int kHostSlots = 2;   // device slots per direction of rcf_filter_host

// status of a CUDA call, recorded in the context (for use where RCF_CUDA cannot return)
int cuda_check(rcf_ctx* ctx, cudaError_t e) {
  return e == cudaSuccess ? RCF_OK : cuda_fail(ctx, e, "CUDA call", __FILE__, __LINE__);
}

// do two multivectors (nvec columns of ld complex elements of size_a / size_b bytes) overlap
bool overlaps(const void* a, int64_t lda, size_t size_a, const void* b, int64_t ldb, size_t size_b, int nvec) {
  if (!a || !b || nvec == 0) return false;
  const char* a0 = static_cast<const char*>(a);
  const char* b0 = static_cast<const char*>(b);
  const char* a1 = a0 + size_t(lda) * nvec * size_a;
  const char* b1 = b0 + size_t(ldb) * nvec * size_b;
  return a0 < b1 && b0 < a1;
}
bool overlaps(const void* a, int64_t lda, const void* b, int64_t ldb, int nvec, size_t cplx) {
  return overlaps(a, lda, cplx, b, ldb, cplx, nvec);
}

// Chebyshev scalars (Eq. ChFSIrecurrence): c, e, sigma[1..q]
struct Cheb {
  double c, e;
  std::vector<double> sigma;  // index 1..q
};
int cheb_scalars(rcf_ctx* ctx, const double* bounds, int q, Cheb* out) {
  if (!bounds) return fail(ctx, RCF_EINVAL, "bounds is NULL");
  const double lmin = bounds[0], lT = bounds[1], lmax = bounds[2];
  if (!(lmin < lT && lT < lmax) || !std::isfinite(lmin) || !std::isfinite(lmax))
    return fail(ctx, RCF_EINVAL, "need lambda_min < lambda_T < lambda_max (got %g, %g, %g)", lmin, lT, lmax);
  if (q < 1) return fail(ctx, RCF_EINVAL, "degree must be >= 1");
  out->c = 0.5 * (lmax + lT);
  out->e = 0.5 * (lmax - lT);
  out->sigma.assign(q + 1, 0.0);
  out->sigma[1] = out->e / (lmin - out->c);
  for (int k = 1; k < q; ++k) out->sigma[k + 1] = 1.0 / (2.0 / out->sigma[1] - out->sigma[k]);
  return RCF_OK;
}

// Lambda_k = C_k(Lambda) by the same three-term recurrence, FP64 (text after Eq. rChFSIrecurrence)
void ritz_filter_values(const Cheb& ch, const double* lam, int nvec, int q, std::vector<double>* L) {
  L->assign(size_t(q + 1) * nvec, 0.0);
  for (int v = 0; v < nvec; ++v) {
    (*L)[v] = 1.0;
    if (q >= 1) (*L)[size_t(nvec) + v] = ch.sigma[1] * (lam[v] - ch.c) / ch.e;
  }
  for (int k = 1; k < q; ++k) {
    const double a = 2.0 * ch.sigma[k + 1] / ch.e, b = ch.sigma[k] * ch.sigma[k + 1];
    for (int v = 0; v < nvec; ++v)
      (*L)[size_t(k + 1) * nvec + v] =
          a * (lam[v] - ch.c) * (*L)[size_t(k) * nvec + v] - b * (*L)[size_t(k - 1) * nvec + v];
  }
}

// y[v] += coef[v] x[v] over `rows` complex rows
template <typename Real>
__global__ void axpy_cols_kernel(int64_t rows, const Real* __restrict__ x, int64_t ldx,
                                 const double* __restrict__ coef, Real* y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const Real c = Real(coef[v]);
  const Real* xs = x + 2 * (int64_t(v) * ldx + r);
  Real* ys = y + 2 * (int64_t(v) * ldy + r);
  ys[0] += c * xs[0];
  ys[1] += c * xs[1];
}
template <typename Real>
int launch_axpy_cols(rcf_ctx* ctx, int64_t rows, const Real* x, int64_t ldx, const double* coef,
                     int nvec, Real* y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  axpy_cols_kernel<Real><<<dim3(unsigned((rows + 255) / 256), nvec), 256, 0, ctx->stream>>>(
      rows, x, ldx, coef, y, ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

// y = s x (Real), column-major blocks
template <typename Real>
__global__ void scale_cols_kernel(int64_t rows, const Real* __restrict__ x, int64_t ldx, Real s,
                                  Real* y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (r >= rows) return;
  const Real* xs = x + 2 * (int64_t(v) * ldx + r);
  Real* ys = y + 2 * (int64_t(v) * ldy + r);
  ys[0] = s * xs[0];
  ys[1] = s * xs[1];
}
template <typename Real>
int launch_scale_cols(rcf_ctx* ctx, int64_t rows, const Real* x, int64_t ldx, Real s, int nvec,
                      Real* y, int64_t ldy) {
  if (nvec <= 0) return RCF_OK;
  scale_cols_kernel<Real><<<dim3(unsigned((rows + 255) / 256), nvec), 256, 0, ctx->stream>>>(
      rows, x, ldx, s, y, ldy);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

// Symmetric tridiagonal extreme eigenvalues by Sturm-sequence bisection.
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double d = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    d = a[i] - x - (i ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++cnt;
  }
  return cnt;
}
double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int k) {
  // k-th smallest eigenvalue (0-based)
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < a.size(); ++i) {
    const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (sturm_count(a, b, mid) > k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

// Hamiltonian-multivector product with the nonlocal part.
//   form H_DINV: out = A (H D^{-1}) in + ...       (R-ChFSI, Eq. rChFSIrecurrence)
//   form DINV_H: out = A (D^{-1} H) in + ...       (ChFSI, Eq. ChFSIrecurrence)
//   form H:      out = M (A (D^{-1} H_loc) in + B in + C prev + g rv) + A H_nloc in
template <typename Real, typename St>
int apply_full(rcf_ctx* ctx, const rcf_op* op, int form, const StepArgs<Real, St>& a0) {
  if (op->fm) {   // full consistent mass: form H's M is the full mass (fullmass.cu)
    if constexpr (std::is_same<Real, St>::value)
      return apply_full_fm<Real>(ctx, op, form, a0);
    else
      return fail(ctx, RCF_ENOTSUP, "16-bit storage is not available with the full mass");
  }
  StepArgs<Real, St> a = a0;
  a.pot = pot_of<Real>(op);
  a.mass = op->mesh->d_mass;
  Tables t;
  build_tables(op->mesh, form == RCF_FORM_H_DINV ? TAB_COL_SCALED : TAB_ROW_SCALED, &t);
  int proj_mass = 1, add_mass = 1;
  if (form == RCF_FORM_H_DINV) { proj_mass = 0; add_mass = 1; a.scale_out = 0; }
  else if (form == RCF_FORM_DINV_H) { proj_mass = 1; add_mass = 0; a.scale_out = 0; }
  else { proj_mass = 1; add_mass = 1; a.scale_out = 1; }
  const bool nl = op->proj.natoms > 0 && a.nvec > 0;
  Real *C = nullptr, *C2 = nullptr;
  if (nl) {
    const size_t bytes = sizeof(Real) * 24 * size_t(op->proj.natoms) * a.nvec;
    RCF_TRY(workspace(ctx, WS_NLC, bytes, reinterpret_cast<void**>(&C)));
    RCF_TRY(workspace(ctx, WS_NLC2, bytes, reinterpret_cast<void**>(&C2)));
    RCF_TRY((launch_nl_project<Real, St>(ctx, op, a.in, a.ld_in, a.nvec, proj_mass, C)));
    RCF_TRY(launch_nl_delta<Real>(ctx, op, C, a.nvec, a.A, C2));
  }
  RCF_TRY((launch_step<Real, St>(ctx, op->mesh, t, a)));
  if (nl) RCF_TRY((launch_nl_addback<Real, St>(ctx, op, C2, a.nvec, add_mass, a.out, a.ld_out)));
  return RCF_OK;
}
template int apply_full<float, float>(rcf_ctx*, const rcf_op*, int, const StepArgs<float, float>&);
template int apply_full<double, double>(rcf_ctx*, const rcf_op*, int, const StepArgs<double, double>&);
template int apply_full<float, __half>(rcf_ctx*, const rcf_op*, int, const StepArgs<float, __half>&);
template int apply_full<float, __nv_bfloat16>(rcf_ctx*, const rcf_op*, int, const StepArgs<float, __nv_bfloat16>&);

namespace {

template <typename Real, typename St = Real>
StepArgs<Real, St> step_args(const St* in, int64_t ldin, St* out, int64_t ldout, int nvec, Real A,
                             Real B) {
  StepArgs<Real, St> a{};
  a.in = in; a.ld_in = ldin;
  a.out = out; a.ld_out = ldout;
  a.A = A; a.B = B; a.C = Real(0);
  a.nvec = nvec;
  return a;
}

// FP64 residual R = H X - M X diag(lam) into R (c128); lam_d device [nvec]
int residual_impl(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                  const double* neglam_d, double* R, int64_t ldr) {
  StepArgs<double> a = step_args<double>(X, ldx, R, ldr, nvec, 1.0, 0.0);
  a.rv = X; a.ld_rv = ldx; a.g = neglam_d;
  return apply_full<double>(ctx, op, RCF_FORM_H, a);
}

// One R-ChFSI step (Eq. rChFSIrecurrence) for k >= 1:
//   out = a_k H D^{-1} (zs Zk) - a_k c (zs Zk) + cp * Zkm1 + g[v] R
// Rbfp (FP32): the g[v] R term reads R from its 12-bit BFP stream instead of R.
template <typename Real, typename St = Real>
int rchfsi_step(rcf_ctx* ctx, const rcf_op* op, const Cheb& ch, int k, const St* Zk, double zs,
                const St* Zkm1, double cp, const St* R, const double* g, St* out, int64_t ld,
                int nvec, const unsigned char* Rbfp = nullptr) {
  const double ak = 2.0 * ch.sigma[k + 1] / ch.e;
  StepArgs<Real, St> a = step_args<Real, St>(Zk, ld, out, ld, nvec, Real(ak * zs), Real(-ak * ch.c * zs));
  if (Zkm1) { a.prev = Zkm1; a.ld_prev = ld; a.C = Real(cp); }
  if (Rbfp) a.rv_bfp = Rbfp;
  else { a.rv = R; a.ld_rv = ld; }
  a.g = g;
  return apply_full<Real, St>(ctx, op, RCF_FORM_H_DINV, a);
}

// R-ChFSI coefficient table of a block (q + 1 rows of nvec): row 0: -Lambda; rows k = 1 .. q-1:
// a_k Lambda_k (the R term of step k); row q: Lambda_q (the recovery)
void rchfsi_table(const Cheb& ch, const double* lam_h, int nvec, int q, double* tab) {
  std::vector<double> L;
  ritz_filter_values(ch, lam_h, nvec, q, &L);
  for (int v = 0; v < nvec; ++v) tab[v] = -lam_h[v];
  for (int k = 1; k < q; ++k) {
    const double ak = 2.0 * ch.sigma[k + 1] / ch.e;
    for (int v = 0; v < nvec; ++v) tab[size_t(k) * nvec + v] = ak * L[size_t(k) * nvec + v];
  }
  for (int v = 0; v < nvec; ++v) tab[size_t(q) * nvec + v] = L[size_t(q) * nvec + v];
}
// the table into the context's coefficient slot (one host-to-device copy on the context's stream)
int upload_rchfsi_table(rcf_ctx* ctx, const Cheb& ch, const double* lam_h, int nvec, int q, const double** out) {
  std::vector<double> tab(size_t(q + 1) * nvec);
  rchfsi_table(ch, lam_h, nvec, q, tab.data());
  double* tab_d = nullptr;
  RCF_TRY(workspace(ctx, WS_COEF, sizeof(double) * tab.size(), reinterpret_cast<void**>(&tab_d)));
  RCF_CUDA(ctx, cudaMemcpyAsync(tab_d, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, ctx->stream));
  *out = tab_d;
  return RCF_OK;
}

// df: the residual in double-float arithmetic, written straight to its FP32 rounding
// (FP32 recurrence, q >= 2); otherwise in FP64 and rounded by a separate pass.
// bfp (FP32, q >= 2): R stored as a 12-bit BFP stream (Section III-C-3's block format, one
// block per node 4-tuple): its FP32 rounding is encoded once and replaced by the decoded
// values, and every step reads its g[v] R term from the stream (6 bytes per node and vector
// instead of 16).  The recurrence is linear in R, so the storage rounding of R enters the
// result as R-ChFSI applied to that rounding: an error proportional to ||R||.
// tab_dev: the block's coefficient table already on the device (else it is built and uploaded).
template <typename Real>
int rchfsi_block(rcf_ctx* ctx, const rcf_op* op, const Cheb& ch, int q, const double* X, int64_t ldx,
                 int nvec, const double* lam_h, double* Y, int64_t ldy, bool df = false, bool bfp = false,
                 const double* tab_dev = nullptr) {
  const rcf_mesh* m = op->mesh;
  const int64_t rows = 2 * m->nnodes;
  const int64_t ld = rows;   // internal buffers: ld = 2M
  // device coefficient table: row 0: -Lambda; rows k=1..q-1: a_k Lambda_k; row q: Lambda_q
  const double* tab_d = tab_dev;
  if (!tab_d) RCF_TRY(upload_rchfsi_table(ctx, ch, lam_h, nvec, q, &tab_d));

  const double s = ch.sigma[1] / ch.e;
  const double* lamq_d = tab_d + size_t(q) * nvec;
  df = df && sizeof(Real) == sizeof(float) && q >= 2;
  double* R64 = nullptr;
  if (!df) {
    RCF_TRY(workspace(ctx, WS_R64, sizeof(double) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&R64)));
    RCF_TRY(residual_impl(ctx, op, X, ldx, nvec, tab_d, R64, ld));
  }
  if (q == 1) {
    RCF_TRY(launch_recover<double>(ctx, m, R64, ld, s, X, ldx, lamq_d, nvec, Y, ldy));
  } else {
    const Real* R = nullptr;
    unsigned char* Rbfp = nullptr;
    if (sizeof(Real) == sizeof(double)) {
      R = reinterpret_cast<const Real*>(R64);
    } else {
      float* R32 = nullptr;
      RCF_TRY(workspace(ctx, WS_R32, sizeof(float) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&R32)));
      if (df) RCF_TRY(launch_residual_df(ctx, op, X, ldx, nvec, tab_d, R32, nullptr, ld));
      else RCF_TRY(launch_to_c64(ctx, rows, R64, ld, nvec, R32, ld));
      if (bfp) {
        const int64_t nvals = 2 * ld * int64_t(nvec);
        RCF_TRY(workspace(ctx, WS_RBFP, size_t((nvals / 4) * 6 + 16), reinterpret_cast<void**>(&Rbfp)));
        RCF_TRY(launch_bfp12_round_trip(ctx, R32, nvals, Rbfp));
      }
      R = reinterpret_cast<const Real*>(R32);
    }
    Real *ZA = nullptr, *ZB = nullptr;
    RCF_TRY(workspace(ctx, WS_ZA, sizeof(Real) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&ZA)));
    RCF_TRY(workspace(ctx, WS_ZB, sizeof(Real) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&ZB)));
    // k = 1: Z_2 = a_1 H D^-1 (s R) - a_1 c s R + a_1 Lambda_1 R   (Z_0 = 0)
    RCF_TRY((rchfsi_step<Real, Real>(ctx, op, ch, 1, R, s, nullptr, 0.0, R, tab_d + nvec, ZA, ld, nvec, Rbfp)));
    // Z_1 = s R is never materialised: it is R with the scale folded into the coefficients.
    const Real* Zkm1 = R;
    double zps = s;
    Real* Zk = ZA;
    for (int k = 2; k < q; ++k) {
      const double bk = ch.sigma[k] * ch.sigma[k + 1];
      Real* out = (Zkm1 == R) ? ZB : const_cast<Real*>(Zkm1);   // in place over Z_{k-1}
      RCF_TRY((rchfsi_step<Real, Real>(ctx, op, ch, k, Zk, 1.0, Zkm1, -bk * zps, R,
                                       tab_d + size_t(k) * nvec, out, ld, nvec, Rbfp)));
      Zkm1 = Zk;
      zps = 1.0;
      Zk = out;
    }
    RCF_TRY(launch_recover<Real>(ctx, m, Zk, ld, 1.0, X, ldx, lamq_d, nvec, Y, ldy));
  }
  return RCF_OK;
}

// R-ChFSI with the recurrence vectors Z_k, Z_{k-1} and R stored in a 16-bit float type
// (FP32 arithmetic): the residual in double-float arithmetic, each column of R scaled by
// the power of two that puts its largest entry in [1/2, 1) before rounding (exact, and
// independent of summation order; the recurrence is linear in (Z, R), so the scale
// returns exactly in the recovery), q >= 2.
template <typename St>
int rchfsi_block16(rcf_ctx* ctx, const rcf_op* op, const Cheb& ch, int q, const double* X, int64_t ldx,
                   int nvec, const double* lam_h, double* Y, int64_t ldy, const double* tab_dev = nullptr) {
  if (q < 2) return rchfsi_block<float>(ctx, op, ch, q, X, ldx, nvec, lam_h, Y, ldy, true, false, tab_dev);
  const rcf_mesh* m = op->mesh;
  const int64_t rows = 2 * m->nnodes;
  const int64_t ld = rows;
  const double* tab_d = tab_dev;
  if (!tab_d) RCF_TRY(upload_rchfsi_table(ctx, ch, lam_h, nvec, q, &tab_d));
  // R (double-float) -> FP32 rounding -> column scale -> 16-bit copy
  float* R32 = nullptr;
  RCF_TRY(workspace(ctx, WS_R32, sizeof(float) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&R32)));
  RCF_TRY(launch_residual_df(ctx, op, X, ldx, nvec, tab_d, R32, nullptr, ld));
  double* sc = nullptr;   // [scale] doubles, then [inv] floats, then [column max] bits
  RCF_TRY(workspace(ctx, WS_SCALE, (sizeof(double) + sizeof(float) + sizeof(unsigned)) * size_t(nvec),
                    reinterpret_cast<void**>(&sc)));
  double* scale = sc;
  float* inv = reinterpret_cast<float*>(sc + nvec);
  unsigned* cmax = reinterpret_cast<unsigned*>(inv + nvec);
  RCF_CUDA(ctx, cudaMemsetAsync(cmax, 0, sizeof(unsigned) * nvec, ctx->stream));
  RCF_TRY(launch_colmax_f32(ctx, rows, R32, ld, nvec, cmax));
  RCF_TRY(launch_pow2_scale(ctx, cmax, nvec, scale, inv));
  St* R = nullptr;
  RCF_TRY(workspace(ctx, WS_R16, sizeof(St) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&R)));
  RCF_TRY(launch_to_storage<St>(ctx, rows, R32, ld, nvec, inv, R, ld));
  St *ZA = nullptr, *ZB = nullptr;
  RCF_TRY(workspace(ctx, WS_ZA, sizeof(St) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&ZA)));
  RCF_TRY(workspace(ctx, WS_ZB, sizeof(St) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&ZB)));
  const double s = ch.sigma[1] / ch.e;
  RCF_TRY((rchfsi_step<float, St>(ctx, op, ch, 1, R, s, nullptr, 0.0, R, tab_d + nvec, ZA, ld, nvec)));
  const St* Zkm1 = R;
  double zps = s;
  St* Zk = ZA;
  for (int k = 2; k < q; ++k) {
    const double bk = ch.sigma[k] * ch.sigma[k + 1];
    St* out = (Zkm1 == R) ? ZB : const_cast<St*>(Zkm1);
    RCF_TRY((rchfsi_step<float, St>(ctx, op, ch, k, Zk, 1.0, Zkm1, -bk * zps, R, tab_d + size_t(k) * nvec, out,
                                    ld, nvec)));
    Zkm1 = Zk;
    zps = 1.0;
    Zk = out;
  }
  return launch_recover_scaled<St>(ctx, m, Zk, ld, scale, X, ldx, tab_d + size_t(q) * nvec, nvec, Y, ldy);
}


// ChFSI (Eq. ChFSIrecurrence) in FP64 on c128 blocks
int chfsi_block64(rcf_ctx* ctx, const rcf_op* op, const Cheb& ch, int q, const double* X, int64_t ldx,
                  int nvec, double* Y, int64_t ldy) {
  const int64_t ld = 2 * op->mesh->nnodes;
  const double s = ch.sigma[1] / ch.e;
  if (q == 1) {
    StepArgs<double> a = step_args<double>(X, ldx, Y, ldy, nvec, s, -s * ch.c);
    return apply_full<double>(ctx, op, RCF_FORM_DINV_H, a);
  }
  double *YA = nullptr, *YB = nullptr;
  RCF_TRY(workspace(ctx, WS_ZA, sizeof(double) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&YA)));
  RCF_TRY(workspace(ctx, WS_ZB, sizeof(double) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&YB)));
  {
    StepArgs<double> a = step_args<double>(X, ldx, YA, ld, nvec, s, -s * ch.c);
    RCF_TRY(apply_full<double>(ctx, op, RCF_FORM_DINV_H, a));
  }
  const double* Yk = YA;
  int64_t ldk = ld;
  const double* Ykm1 = X;
  int64_t ldkm1 = ldx;
  for (int k = 1; k < q; ++k) {
    const double ak = 2.0 * ch.sigma[k + 1] / ch.e, bk = ch.sigma[k] * ch.sigma[k + 1];
    double* out;
    int64_t ldo;
    if (k == q - 1) { out = Y; ldo = ldy; }
    else if (Ykm1 == X) { out = (Yk == YA) ? YB : YA; ldo = ld; }
    else { out = const_cast<double*>(Ykm1); ldo = ld; }
    StepArgs<double> a = step_args<double>(Yk, ldk, out, ldo, nvec, ak, -ak * ch.c);
    a.prev = Ykm1; a.ld_prev = ldkm1; a.C = -bk;
    RCF_TRY(apply_full<double>(ctx, op, RCF_FORM_DINV_H, a));
    Ykm1 = Yk; ldkm1 = ldk;
    Yk = out; ldk = ldo;
  }
  return RCF_OK;
}

// ChFSI in FP32 (complex64 recurrence from a rounded copy of X), result widened to c128
int chfsi_block32(rcf_ctx* ctx, const rcf_op* op, const Cheb& ch, int q, const double* X, int64_t ldx,
                  int nvec, double* Y, int64_t ldy) {
  const int64_t rows = 2 * op->mesh->nnodes, ld = rows;
  float *X32 = nullptr, *YA = nullptr;
  RCF_TRY(workspace(ctx, WS_R32, sizeof(float) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&X32)));
  RCF_TRY(workspace(ctx, WS_ZA, sizeof(float) * 2 * size_t(ld) * nvec, reinterpret_cast<void**>(&YA)));
  RCF_TRY(launch_to_c64(ctx, rows, X, ldx, nvec, X32, ld));
  const double s = ch.sigma[1] / ch.e;
  {
    StepArgs<float> a = step_args<float>(X32, ld, YA, ld, nvec, float(s), float(-s * ch.c));
    RCF_TRY(apply_full<float>(ctx, op, RCF_FORM_DINV_H, a));
  }
  float* bufs[2] = {X32, YA};   // Y_{k+1} overwrites Y_{k-1} in place
  int ikm1 = 0, ik = 1;
  for (int k = 1; k < q; ++k) {
    const double ak = 2.0 * ch.sigma[k + 1] / ch.e, bk = ch.sigma[k] * ch.sigma[k + 1];
    const int io = ikm1;   // in place over Y_{k-1}
    StepArgs<float> a = step_args<float>(bufs[ik], ld, bufs[io], ld, nvec, float(ak), float(-ak * ch.c));
    a.prev = bufs[ikm1]; a.ld_prev = ld; a.C = float(-bk);
    RCF_TRY(apply_full<float>(ctx, op, RCF_FORM_DINV_H, a));
    ikm1 = ik;
    ik = io;
  }
  return launch_c64_to_c128(ctx, rows, bufs[ik], ld, nvec, Y, ldy);
}

}  // namespace
}  // namespace rcf

using namespace rcf;

namespace rcf {
namespace {

// one band block of the filter in the requested mode and precision
// tab: the block's R-ChFSI coefficient table on the device, or null (built and uploaded here)
int filter_block(rcf_ctx* ctx, const rcf_op* op, const Cheb& ch, int q, int mode, int prec, const double* X,
                 int64_t ldx, int n, const double* lam, double* Y, int64_t ldy, const double* tab = nullptr) {
  if (mode == RCF_RCHFSI) {
    switch (prec) {
      case RCF_FP64: return rchfsi_block<double>(ctx, op, ch, q, X, ldx, n, lam, Y, ldy, false, false, tab);
      case RCF_FP32: return rchfsi_block<float>(ctx, op, ch, q, X, ldx, n, lam, Y, ldy, false, false, tab);
      case RCF_FP32_DF: return rchfsi_block<float>(ctx, op, ch, q, X, ldx, n, lam, Y, ldy, true, false, tab);
      case RCF_FP16: return rchfsi_block16<__half>(ctx, op, ch, q, X, ldx, n, lam, Y, ldy, tab);
      case RCF_BF16: return rchfsi_block16<__nv_bfloat16>(ctx, op, ch, q, X, ldx, n, lam, Y, ldy, tab);
      case RCF_FP32_BFP12:
        return rchfsi_block<float>(ctx, op, ch, q, X, ldx, n, lam, Y, ldy, false, true, tab);
      default: return fail(ctx, RCF_EINVAL, "unknown precision %d", prec);
    }
  }
  if (prec == RCF_FP64) return chfsi_block64(ctx, op, ch, q, X, ldx, n, Y, ldy);
  return chfsi_block32(ctx, op, ch, q, X, ldx, n, Y, ldy);
}

// precision and mode of rcf_filter / rcf_filter_host
int check_filter_mode(rcf_ctx* ctx, int mode, int prec) {
  if (mode != RCF_CHFSI && mode != RCF_RCHFSI) return fail(ctx, RCF_EINVAL, "unknown mode %d", mode);
  if (prec < RCF_FP64 || prec > RCF_FP32_BFP12) return fail(ctx, RCF_EINVAL, "unknown precision %d", prec);
  if (prec >= RCF_FP32_DF && mode != RCF_RCHFSI)
    return fail(ctx, RCF_EINVAL, "precision %d applies to R-ChFSI only (it reshapes the residual)", prec);
  return RCF_OK;
}

// bytes of one real of a multivector in precision prec (rcf_apply, rcf_cheb_step)
size_t real_bytes(int prec) {
  switch (prec) {
    case RCF_FP64: return 8;
    case RCF_FP32: return 4;
    case RCF_FP16: case RCF_BF16: return 2;
    default: return 0;
  }
}

}  // namespace
}  // namespace rcf

extern "C" int rcf_apply(rcf_ctx* ctx, const rcf_op* op, int form, const void* X, int64_t ldx,
                         int nvec, void* Y, int64_t ldy, int prec) {
  if (!ctx || !op) return RCF_EINVAL;
  if (form < 0 || form > 2) return fail(ctx, RCF_EINVAL, "unknown form %d", form);
  if (prec == RCF_FP32_BFP12) return fail(ctx, RCF_EINVAL, "RCF_FP32_BFP12 applies to rcf_filter and rcf_cheb_step");
  const size_t real = real_bytes(prec);
  if (real == 0) return fail(ctx, RCF_EINVAL, "unknown precision %d", prec);
  RCF_TRY(check_block(ctx, op, X, ldx, nvec, real, "X"));
  RCF_TRY(check_block(ctx, op, Y, ldy, nvec, real, "Y"));
  if (overlaps(X, ldx, Y, ldy, nvec, 2 * real)) return fail(ctx, RCF_EINVAL, "Y overlaps X");
  if (nvec == 0) return RCF_OK;
  auto run = [&](auto tag) {
    using St = decltype(tag);
    using Real = std::conditional_t<std::is_same_v<St, double>, double, float>;
    StepArgs<Real, St> a = step_args<Real, St>(static_cast<const St*>(X), ldx, static_cast<St*>(Y), ldy, nvec,
                                               Real(1), Real(0));
    return apply_full<Real, St>(ctx, op, form, a);
  };
  switch (prec) {
    case RCF_FP64: return run(double{});
    case RCF_FP32: return run(float{});
    case RCF_FP16: return run(__half{});
    default: return run(__nv_bfloat16{});
  }
}

extern "C" int rcf_cheb_step(rcf_ctx* ctx, const rcf_op* op, int form, int prec, const void* Zk,
                             const void* Zkm1, const void* R, int64_t ld, int nvec, double alpha,
                             double beta, double gamma, const double* g, void* out) {
  if (!ctx || !op) return RCF_EINVAL;
  if (form < 0 || form > 2) return fail(ctx, RCF_EINVAL, "unknown form %d", form);
  const bool bfp = prec == RCF_FP32_BFP12;   // Zk, Zkm1, out complex64; R a 12-bit BFP stream
  const size_t real = bfp ? 4 : real_bytes(prec);
  if (real == 0) return fail(ctx, RCF_EINVAL, "unknown precision %d", prec);
  RCF_TRY(check_block(ctx, op, Zk, ld, nvec, real, "Zk"));
  RCF_TRY(check_block(ctx, op, out, ld, nvec, real, "out"));
  if (Zkm1) RCF_TRY(check_block(ctx, op, Zkm1, ld, nvec, real, "Zkm1"));
  const int64_t nn = op->mesh->nnodes;
  if (R && bfp) {
    if (!aligned(R, 4)) return fail(ctx, RCF_EINVAL, "R: the BFP stream must be 4-byte aligned");
    if (op->fm && form == RCF_FORM_H) return fail(ctx, RCF_ENOTSUP, "BFP storage of R applies to the recurrence forms");
  } else if (R) {
    RCF_TRY(check_block(ctx, op, R, ld, nvec, real, "R"));
  }
  const bool r_over = bfp ? overlaps(R, nn, 6, out, ld, 2 * real, nvec) : overlaps(R, ld, out, ld, nvec, 2 * real);
  if (overlaps(Zk, ld, out, ld, nvec, 2 * real) || r_over) return fail(ctx, RCF_EINVAL, "out overlaps Zk or R");
  if (Zkm1 && Zkm1 != out && overlaps(Zkm1, ld, out, ld, nvec, 2 * real))
    return fail(ctx, RCF_EINVAL, "out partly overlaps Zkm1");
  if (R && !g) return fail(ctx, RCF_EINVAL, "R given without g");
  if (nvec == 0) return RCF_OK;
  auto run = [&](auto tag) {
    using St = decltype(tag);
    using Real = std::conditional_t<std::is_same_v<St, double>, double, float>;
    StepArgs<Real, St> a = step_args<Real, St>(static_cast<const St*>(Zk), ld, static_cast<St*>(out), ld, nvec,
                                               Real(alpha), Real(beta));
    if (Zkm1) { a.prev = static_cast<const St*>(Zkm1); a.ld_prev = ld; a.C = Real(gamma); }
    if (R && bfp) { a.rv_bfp = static_cast<const unsigned char*>(R); a.g = g; }
    else if (R) { a.rv = static_cast<const St*>(R); a.ld_rv = ld; a.g = g; }
    return apply_full<Real, St>(ctx, op, form, a);
  };
  switch (prec) {
    case RCF_FP64: return run(double{});
    case RCF_FP32: case RCF_FP32_BFP12: return run(float{});
    case RCF_FP16: return run(__half{});
    default: return run(__nv_bfloat16{});
  }
}

extern "C" int64_t rcf_launch_count(const rcf_ctx* ctx) { return ctx ? ctx->launches : -1; }

extern "C" int rcf_residual(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                            const double* ritz, double* R, int64_t ldr, double* colnorm) {
  if (!ctx || !op) return RCF_EINVAL;
  RCF_TRY(check_block(ctx, op, X, ldx, nvec, 8, "X"));
  if (nvec == 0) return RCF_OK;
  if (!ritz) return fail(ctx, RCF_EINVAL, "ritz is NULL");
  const int64_t rows = 2 * op->mesh->nnodes;
  if (R) {
    RCF_TRY(check_block(ctx, op, R, ldr, nvec, 8, "R"));
    if (overlaps(X, ldx, R, ldr, nvec, 16)) return fail(ctx, RCF_EINVAL, "R overlaps X");
  } else {
    ldr = rows;
    RCF_TRY(workspace(ctx, WS_R64, sizeof(double) * 2 * size_t(ldr) * nvec, reinterpret_cast<void**>(&R)));
  }
  std::vector<double> neg(nvec);
  for (int v = 0; v < nvec; ++v) neg[v] = -ritz[v];
  double* neg_d = nullptr;
  RCF_TRY(workspace(ctx, WS_COEF, sizeof(double) * nvec, reinterpret_cast<void**>(&neg_d)));
  RCF_CUDA(ctx, cudaMemcpyAsync(neg_d, neg.data(), sizeof(double) * nvec, cudaMemcpyHostToDevice, ctx->stream));
  RCF_TRY(residual_impl(ctx, op, X, ldx, nvec, neg_d, R, ldr));
  if (colnorm) {
    RCF_CUDA(ctx, cudaMemsetAsync(colnorm, 0, sizeof(double) * nvec, ctx->stream));
    RCF_TRY(launch_colnorm2(ctx, rows, R, ldr, nvec, colnorm));
    RCF_TRY(launch_sqrt_inplace(ctx, colnorm, nvec));
  }
  // neg is a host stack buffer read by an async copy
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RCF_OK;
}

extern "C" int rcf_residual_df(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                               const double* ritz, float* Rh, float* Rl, int64_t ldr) {
  if (!ctx || !op) return RCF_EINVAL;
  RCF_TRY(check_block(ctx, op, X, ldx, nvec, 8, "X"));
  if (nvec == 0) return RCF_OK;
  if (!ritz) return fail(ctx, RCF_EINVAL, "ritz is NULL");
  RCF_TRY(check_block(ctx, op, Rh, ldr, nvec, 4, "Rh"));
  if (Rl) {
    RCF_TRY(check_block(ctx, op, Rl, ldr, nvec, 4, "Rl"));
    if (overlaps(Rh, ldr, Rl, ldr, nvec, 8)) return fail(ctx, RCF_EINVAL, "Rl overlaps Rh");
  }
  if (overlaps(X, ldx, 16, Rh, ldr, 8, nvec) || (Rl && overlaps(X, ldx, 16, Rl, ldr, 8, nvec)))
    return fail(ctx, RCF_EINVAL, "R overlaps X");
  std::vector<double> neg(nvec);
  for (int v = 0; v < nvec; ++v) neg[v] = -ritz[v];
  double* neg_d = nullptr;
  RCF_TRY(workspace(ctx, WS_COEF, sizeof(double) * nvec, reinterpret_cast<void**>(&neg_d)));
  RCF_CUDA(ctx, cudaMemcpyAsync(neg_d, neg.data(), sizeof(double) * nvec, cudaMemcpyHostToDevice, ctx->stream));
  RCF_TRY(launch_residual_df(ctx, op, X, ldx, nvec, neg_d, Rh, Rl, ldr));
  // neg is a host stack buffer read by an async copy
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RCF_OK;
}

extern "C" int rcf_filter(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                          const double* ritz, int degree, const double bounds[3], int mode, int prec,
                          int block, double* Y, int64_t ldy) {
  if (!ctx || !op) return RCF_EINVAL;
  RCF_TRY(check_block(ctx, op, X, ldx, nvec, 8, "X"));
  RCF_TRY(check_block(ctx, op, Y, ldy, nvec, 8, "Y"));
  if (overlaps(X, ldx, Y, ldy, nvec, 16)) return fail(ctx, RCF_EINVAL, "Y overlaps X");
  RCF_TRY(check_filter_mode(ctx, mode, prec));
  if (mode == RCF_RCHFSI && !ritz && nvec > 0) return fail(ctx, RCF_EINVAL, "ritz is NULL");
  Cheb ch;
  RCF_TRY(cheb_scalars(ctx, bounds, degree, &ch));
  if (nvec == 0) return RCF_OK;
  const int nb = (block <= 0 || block > nvec) ? nvec : block;
  for (int b0 = 0; b0 < nvec; b0 += nb) {
    const int n = std::min(nb, nvec - b0);
    const double* Xb = X + 2 * int64_t(b0) * ldx;
    double* Yb = Y + 2 * int64_t(b0) * ldy;
    RCF_TRY(filter_block(ctx, op, ch, degree, mode, prec, Xb, ldx, n, ritz ? ritz + b0 : nullptr, Yb, ldy));
    // one block in flight at a time (the next block's table goes into the same device slot)
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return check_device_error(ctx);
}

extern "C" int rcf_filter_host(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                               const double* ritz, int degree, const double bounds[3], int mode, int prec,
                               int block, double* Y, int64_t ldy) {
  if (!ctx || !op) return RCF_EINVAL;
  const int64_t rows = 2 * op->mesh->nnodes;
  if (nvec < 0) return fail(ctx, RCF_EINVAL, "nvec < 0");
  if (nvec > 0 && (!X || !Y)) return fail(ctx, RCF_EINVAL, "NULL X or Y");
  if (ldx < rows || ldy < rows) return fail(ctx, RCF_EINVAL, "leading dimension below 2M");
  if (overlaps(X, ldx, Y, ldy, nvec, 16)) return fail(ctx, RCF_EINVAL, "Y overlaps X");
  RCF_TRY(check_filter_mode(ctx, mode, prec));
  if (mode == RCF_RCHFSI && !ritz && nvec > 0) return fail(ctx, RCF_EINVAL, "ritz is NULL");
  Cheb ch;
  RCF_TRY(cheb_scalars(ctx, bounds, degree, &ch));
  if (nvec == 0) return RCF_OK;
  for (cudaStream_t* st : {&ctx->copy_in, &ctx->copy_out})
    if (!*st) RCF_CUDA(ctx, cudaStreamCreateWithFlags(st, cudaStreamNonBlocking));
  const int nb = (block <= 0 || block > nvec) ? nvec : block;
  const int nblk = (nvec + nb - 1) / nb;
  // S device slots for X blocks and S for Y blocks (ld = 2M): the next block is copied
  // in and the previous one copied out while a block is filtered
  const int S = std::min(nblk, kHostSlots);
  const size_t bytes = sizeof(double) * 2 * size_t(rows) * nb;
  double* dxs = nullptr;
  double* dys = nullptr;
  RCF_TRY(workspace(ctx, WS_HX0, bytes * S, reinterpret_cast<void**>(&dxs)));
  RCF_TRY(workspace(ctx, WS_HY0, bytes * S, reinterpret_cast<void**>(&dys)));
  auto dx = [&](int b) { return dxs + 2 * size_t(rows) * nb * (b % S); };
  auto dy = [&](int b) { return dys + 2 * size_t(rows) * nb * (b % S); };
  // events: X block landed, block filtered (its X slot free, Y ready), Y slot copied out
  std::vector<cudaEvent_t> ev_in(nblk), ev_done(nblk), ev_out(nblk);
  auto make = [&](std::vector<cudaEvent_t>& v) -> int {
    for (auto& e : v) RCF_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return RCF_OK;
  };
  int st = make(ev_in);
  if (st == RCF_OK) st = make(ev_done);
  if (st == RCF_OK) st = make(ev_out);
  auto copy_rows = [&](double* dst, int64_t ldd, const double* src, int64_t lds, int n, cudaMemcpyKind kind,
                       cudaStream_t s) -> int {
    RCF_CUDA(ctx, cudaMemcpy2DAsync(dst, sizeof(double) * 2 * ldd, src, sizeof(double) * 2 * lds,
                                    sizeof(double) * 2 * rows, n, kind, s));
    return RCF_OK;
  };
  auto count = [&](int b) { return std::min(nb, nvec - b * nb); };
  // R-ChFSI: every block's coefficient table built and uploaded here, in one copy queued
  // before the first block copy, so that no small host-to-device copy waits behind a block
  // copy on the copy engine in the middle of the pipeline (a filter whose table upload is
  // queued behind an 8 GB block copy starts only when that copy ends)
  std::vector<size_t> tab_off(nblk + 1, 0);
  const double* tabs_d = nullptr;
  if (st == RCF_OK && mode == RCF_RCHFSI) {
    for (int b = 0; b < nblk; ++b) tab_off[b + 1] = tab_off[b] + size_t(degree + 1) * count(b);
    std::vector<double> tabs(tab_off[nblk]);
    for (int b = 0; b < nblk; ++b) rchfsi_table(ch, ritz + int64_t(b) * nb, count(b), degree, tabs.data() + tab_off[b]);
    double* d = nullptr;
    st = workspace(ctx, WS_HTAB, sizeof(double) * tabs.size(), reinterpret_cast<void**>(&d));
    if (st == RCF_OK)
      st = cuda_check(ctx, cudaMemcpyAsync(d, tabs.data(), sizeof(double) * tabs.size(), cudaMemcpyHostToDevice,
                                           ctx->stream));
    tabs_d = d;
  }
  // block b into its X slot once the block that used the slot before (b - S) is filtered
  auto copy_in = [&](int b) -> int {
    if (b >= S) RCF_TRY(cuda_check(ctx, cudaStreamWaitEvent(ctx->copy_in, ev_done[b - S], 0)));
    RCF_TRY(copy_rows(dx(b), rows, X + 2 * int64_t(b) * nb * ldx, ldx, count(b), cudaMemcpyHostToDevice,
                      ctx->copy_in));
    return cuda_check(ctx, cudaEventRecord(ev_in[b], ctx->copy_in));
  };
  if (st == RCF_OK) st = copy_in(0);
  for (int b = 0; b < nblk && st == RCF_OK; ++b) {
    const int n = count(b);
    st = cuda_check(ctx, cudaStreamWaitEvent(ctx->stream, ev_in[b], 0));
    if (st == RCF_OK && b >= S) st = cuda_check(ctx, cudaStreamWaitEvent(ctx->stream, ev_out[b - S], 0));
    if (st == RCF_OK) {
      double* xs = dx(b);
      double* ys = dy(b);
      st = filter_block(ctx, op, ch, degree, mode, prec, xs, rows, n, ritz ? ritz + int64_t(b) * nb : nullptr,
                        ys, rows, tabs_d ? tabs_d + tab_off[b] : nullptr);
    }
    if (st == RCF_OK) st = cuda_check(ctx, cudaEventRecord(ev_done[b], ctx->stream));
    // The next block's copy is queued now and runs while this block is filtered (host-to-
    // device copies of one device run in issue order; the coefficient tables went ahead of
    // all block copies, above).
    if (st == RCF_OK && b + 1 < nblk) st = copy_in(b + 1);
    // copy the filtered block out while the next one is filtered
    if (st == RCF_OK) st = cuda_check(ctx, cudaStreamWaitEvent(ctx->copy_out, ev_done[b], 0));
    if (st == RCF_OK)
      st = copy_rows(Y + 2 * int64_t(b) * nb * ldy, ldy, dy(b), rows, n, cudaMemcpyDeviceToHost, ctx->copy_out);
    if (st == RCF_OK) st = cuda_check(ctx, cudaEventRecord(ev_out[b], ctx->copy_out));
    // one block of filter work in flight at a time: the next is queued once this one has run
    if (st == RCF_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream));
  }
  // drain both copy streams (also on failure, before the events go away)
  cudaStreamSynchronize(ctx->copy_in);
  cudaStreamSynchronize(ctx->copy_out);
  for (auto* v : {&ev_in, &ev_done, &ev_out})
    for (auto e : *v)
      if (e) cudaEventDestroy(e);
  if (st != RCF_OK) return st;
  return check_device_error(ctx);
}

extern "C" int rcf_lanczos_bounds(rcf_ctx* ctx, const rcf_op* op, int nsteps, const double* v0,
                                  double* theta_min, double* upper) {
  if (!ctx || !op) return RCF_EINVAL;
  if (!v0 || !theta_min || !upper) return fail(ctx, RCF_EINVAL, "NULL argument");
  if (nsteps < 1) return fail(ctx, RCF_EINVAL, "nsteps must be >= 1");
  const rcf_mesh* m = op->mesh;
  const int64_t n = 2 * m->nnodes;   // complex entries
  double* buf = nullptr;
  RCF_TRY(workspace(ctx, WS_LANCZOS, sizeof(double) * (2 * 4 * size_t(n) + 8), reinterpret_cast<void**>(&buf)));
  double *v = buf, *vprev = buf + 2 * n, *w = buf + 4 * n, *t = buf + 6 * n, *dot = buf + 8 * n;
  double h = 0.0;
  RCF_CUDA(ctx, cudaMemsetAsync(dot, 0, sizeof(double), ctx->stream));
  RCF_TRY(launch_dot_re(ctx, n, v0, v0, dot));
  RCF_CUDA(ctx, cudaMemcpyAsync(&h, dot, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (!(h > 0.0)) return fail(ctx, RCF_EINVAL, "v0 is zero");
  RCF_TRY(launch_scale_vec(ctx, n, v0, 1.0 / std::sqrt(h), v));
  RCF_CUDA(ctx, cudaMemsetAsync(vprev, 0, sizeof(double) * 2 * n, ctx->stream));
  std::vector<double> al, be;
  double beta_prev = 0.0;
  for (int j = 0; j < nsteps; ++j) {
    // w = D^{-1/2} H D^{-1/2} v
    RCF_TRY(launch_scale_mass(ctx, m, v, n, 1, -0.5, t, n));
    StepArgs<double> a = step_args<double>(t, n, w, n, 1, 1.0, 0.0);
    RCF_TRY(apply_full<double>(ctx, op, RCF_FORM_H, a));
    RCF_TRY(launch_scale_mass(ctx, m, w, n, 1, -0.5, w, n));
    double alpha = 0.0, bnew = 0.0;
    RCF_CUDA(ctx, cudaMemsetAsync(dot, 0, sizeof(double), ctx->stream));
    RCF_TRY(launch_dot_re(ctx, n, v, w, dot));
    RCF_CUDA(ctx, cudaMemcpyAsync(&alpha, dot, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RCF_TRY(launch_lanczos_update(ctx, n, w, v, vprev, alpha, beta_prev));
    RCF_CUDA(ctx, cudaMemsetAsync(dot, 0, sizeof(double), ctx->stream));
    RCF_TRY(launch_dot_re(ctx, n, w, w, dot));
    RCF_CUDA(ctx, cudaMemcpyAsync(&bnew, dot, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    bnew = std::sqrt(bnew);
    al.push_back(alpha);
    be.push_back(bnew);
    if (j + 1 < nsteps) {
      if (!(bnew > 0.0)) break;   // invariant subspace found
      RCF_CUDA(ctx, cudaMemcpyAsync(vprev, v, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, ctx->stream));
      RCF_TRY(launch_scale_vec(ctx, n, w, 1.0 / bnew, v));
      beta_prev = bnew;
    }
  }
  std::vector<double> off(be.begin(), be.end() - 1);
  *theta_min = tridiag_eig(al, off, 0);
  *upper = tridiag_eig(al, off, int(al.size()) - 1) + std::fabs(be.back());
  return RCF_OK;
}

extern "C" int rcf_grad_bilinear(rcf_ctx* ctx, const rcf_op* op, const double* W, int64_t ldw,
                                 const double* U, int64_t ldu, int nvec, double weight, double* dV,
                                 double* dB, double* dh) {
  if (op && op->fm) return fail(ctx, RCF_ENOTSUP, "gradients are not available with the full consistent mass");
  if (!ctx || !op) return RCF_EINVAL;
  RCF_TRY(check_block(ctx, op, W, ldw, nvec, 8, "W"));
  RCF_TRY(check_block(ctx, op, U, ldu, nvec, 8, "U"));
  if (!dV || !dB) return fail(ctx, RCF_EINVAL, "dV and dB must be device buffers");
  if (nvec == 0) return RCF_OK;
  const rcf_mesh* m = op->mesh;
  double* g = nullptr;
  RCF_TRY(workspace(ctx, WS_GRAD, sizeof(double) * 4 * size_t(m->nnodes) + 16 * sizeof(double) * std::max(1, op->proj.natoms), reinterpret_cast<void**>(&g)));
  RCF_CUDA(ctx, cudaMemsetAsync(g, 0, sizeof(double) * (4 * size_t(m->nnodes) + 2 * std::max(1, op->proj.natoms)), ctx->stream));
  RCF_TRY(launch_grad_local<double>(ctx, m, W, ldw, U, ldu, nvec, weight, 0, g));
  RCF_TRY(launch_grad_to_quadrature(ctx, m, g, dV, dB));
  if (dh && op->proj.natoms > 0) {
    const int na = op->proj.natoms;
    double* gh = g + 4 * m->nnodes;
    double *CW = nullptr, *CU = nullptr;
    const size_t bytes = sizeof(double) * 24 * size_t(na) * nvec;
    RCF_TRY(workspace(ctx, WS_NLC, bytes, reinterpret_cast<void**>(&CW)));
    RCF_TRY(workspace(ctx, WS_NLC2, bytes, reinterpret_cast<void**>(&CU)));
    RCF_TRY(launch_nl_project<double>(ctx, op, W, ldw, nvec, 1, CW));
    RCF_TRY(launch_nl_project<double>(ctx, op, U, ldu, nvec, 1, CU));
    RCF_TRY(launch_grad_h<double>(ctx, op, CW, CU, nvec, weight, gh));
    std::vector<double> tmp(2 * na);
    RCF_CUDA(ctx, cudaMemcpyAsync(tmp.data(), gh, sizeof(double) * 2 * na, cudaMemcpyDeviceToHost, ctx->stream));
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 2 * na; ++i) dh[i] += tmp[i];
  }
  return RCF_OK;
}

namespace rcf {
namespace {

// Reverse sweep of the R-ChFSI filter in precision Real (see rcf_adjoint_filter).
template <typename Real>
int adjoint_impl(rcf_ctx* ctx, const rcf_op* op, const Cheb& ch, int q, const double* X, int64_t ldx,
                 int nvec, const double* lam_h, const double* Ybar, int64_t ldyb, int kc, double* gnode,
                 double* gh) {
  const rcf_mesh* m = op->mesh;
  const int64_t rows = 2 * m->nnodes, ld = rows;
  const size_t blk = sizeof(Real) * 2 * size_t(ld) * nvec;   // one block in Real
  const size_t blk64 = sizeof(double) * 2 * size_t(ld) * nvec;
  // coefficient table (rows as in rchfsi_block) + a_k rows for Rbar
  std::vector<double> L;
  ritz_filter_values(ch, lam_h, nvec, q, &L);
  std::vector<double> tab(size_t(q + 1) * nvec);
  for (int v = 0; v < nvec; ++v) tab[v] = -lam_h[v];
  for (int k = 1; k < q; ++k) {
    const double ak = 2.0 * ch.sigma[k + 1] / ch.e;
    for (int v = 0; v < nvec; ++v) tab[size_t(k) * nvec + v] = ak * L[size_t(k) * nvec + v];
  }
  for (int v = 0; v < nvec; ++v) tab[size_t(q) * nvec + v] = ch.sigma[1] / ch.e;   // s, for Rbar += s Zbar_1
  double* tab_d = nullptr;
  RCF_TRY(workspace(ctx, WS_COEF, sizeof(double) * tab.size(), reinterpret_cast<void**>(&tab_d)));
  RCF_CUDA(ctx, cudaMemcpyAsync(tab_d, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, ctx->stream));

  // R (FP64, then Real copy)
  double* R64 = nullptr;
  RCF_TRY(workspace(ctx, WS_R64, blk64, reinterpret_cast<void**>(&R64)));
  RCF_TRY(residual_impl(ctx, op, X, ldx, nvec, tab_d, R64, ld));
  Real* R = nullptr;
  if (sizeof(Real) == sizeof(double)) R = reinterpret_cast<Real*>(R64);
  else {
    float* R32 = nullptr;
    RCF_TRY(workspace(ctx, WS_R32, blk, reinterpret_cast<void**>(&R32)));
    RCF_TRY(launch_to_c64(ctx, rows, R64, ld, nvec, R32, ld));
    R = reinterpret_cast<Real*>(R32);
  }
  const double s = ch.sigma[1] / ch.e;
  // checkpoints: pairs (Z_{k-1}, Z_k) at k = 1 + j kc, and a segment buffer of kc blocks
  const int nseg = (q - 1 + kc - 1) / kc;   // segments cover k = 1 .. q-1
  char* ck = nullptr;
  char* seg = nullptr;
  RCF_TRY(workspace(ctx, WS_CKPT, blk * size_t(2 * std::max(nseg, 1)), reinterpret_cast<void**>(&ck)));
  RCF_TRY(workspace(ctx, WS_ADJ_U, blk * size_t(kc + 1), reinterpret_cast<void**>(&seg)));
  auto ckp = [&](int j, int which) { return reinterpret_cast<Real*>(ck + blk * size_t(2 * j + which)); };
  auto segp = [&](int i) { return reinterpret_cast<Real*>(seg + blk * size_t(i)); };
  Real *ZA = nullptr, *ZB = nullptr;
  RCF_TRY(workspace(ctx, WS_ZA, blk, reinterpret_cast<void**>(&ZA)));
  RCF_TRY(workspace(ctx, WS_ZB, blk, reinterpret_cast<void**>(&ZB)));

  // forward step helper: out = Z_{k+1} from (Z_k, Z_{k-1}); Z_0 = 0 (kprev null)
  auto fwd = [&](int k, const Real* Zk, const Real* Zkm1, Real* out) {
    const double bk = ch.sigma[k] * ch.sigma[k + 1];
    return rchfsi_step<Real>(ctx, op, ch, k, Zk, 1.0, Zkm1, -bk, R, tab_d + size_t(k) * nvec, out, ld, nvec);
  };
  // forward sweep storing checkpoints. Z_1 = s R materialised.
  {
    Real* z1 = ckp(0, 1);
    RCF_TRY(launch_scale_cols<Real>(ctx, rows, R, ld, Real(s), nvec, z1, ld));
    RCF_CUDA(ctx, cudaMemsetAsync(ckp(0, 0), 0, blk, ctx->stream));
    const Real* Zkm1 = ckp(0, 0);
    const Real* Zk = z1;
    for (int k = 1; k < q - 1; ++k) {   // produce Z_{k+1} for k+1 <= q-1 (Z_q is not needed)
      // in place over Z_{k-1} when it is a scratch buffer, never over a checkpoint
      Real* out = (Zkm1 == ZA || Zkm1 == ZB) ? const_cast<Real*>(Zkm1) : (Zk == ZA ? ZB : ZA);
      RCF_TRY(fwd(k, Zk, k == 1 ? nullptr : Zkm1, out));
      const int kn = k + 1;
      if ((kn - 1) % kc == 0) {
        const int j = (kn - 1) / kc;
        RCF_CUDA(ctx, cudaMemcpyAsync(ckp(j, 0), Zk, blk, cudaMemcpyDeviceToDevice, ctx->stream));
        RCF_CUDA(ctx, cudaMemcpyAsync(ckp(j, 1), out, blk, cudaMemcpyDeviceToDevice, ctx->stream));
        Zkm1 = ckp(j, 0);
        Zk = ckp(j, 1);
      } else {
        Zkm1 = Zk;
        Zk = out;
      }
    }
  }
  // reverse sweep buffers: Zbar (3 rotating), Rbar, projections
  Real *B0 = nullptr, *B1 = nullptr, *B2 = nullptr, *Rbar = nullptr;
  RCF_TRY(workspace(ctx, WS_ADJ_A, blk, reinterpret_cast<void**>(&B0)));
  RCF_TRY(workspace(ctx, WS_ADJ_B, blk, reinterpret_cast<void**>(&B1)));
  RCF_TRY(workspace(ctx, WS_ADJ_C, blk * 2, reinterpret_cast<void**>(&B2)));
  Rbar = reinterpret_cast<Real*>(reinterpret_cast<char*>(B2) + blk);
  RCF_CUDA(ctx, cudaMemsetAsync(Rbar, 0, blk, ctx->stream));
  Real *CW = nullptr, *CU = nullptr;
  const int na = op->proj.natoms;
  if (na > 0) {
    const size_t bytes = sizeof(Real) * 24 * size_t(na) * nvec;
    RCF_TRY(workspace(ctx, WS_NLC, bytes, reinterpret_cast<void**>(&CW)));
    RCF_TRY(workspace(ctx, WS_NLC2, bytes, reinterpret_cast<void**>(&CU)));
  }
  // Zbar_q = D^{-1} Ybar (in Real)
  Real* zbk1 = B0;   // Zbar_{k+1}
  Real* zbk2 = nullptr;   // Zbar_{k+2}
  if (sizeof(Real) == sizeof(double)) {
    RCF_TRY(launch_scale_mass(ctx, m, Ybar, ldyb, nvec, -1.0, reinterpret_cast<double*>(zbk1), ld));
  } else {
    double* tmp64 = R64;   // R64 is no longer needed in FP64 once R32 exists
    RCF_TRY(launch_scale_mass(ctx, m, Ybar, ldyb, nvec, -1.0, tmp64, ld));
    RCF_TRY(launch_to_c64(ctx, rows, tmp64, ld, nvec, reinterpret_cast<float*>(zbk1), ld));
  }
  Real* freebufs[2] = {B1, B2};
  for (int j = nseg - 1; j >= 0; --j) {
    const int k0 = 1 + j * kc;
    const int k1 = std::min(k0 + kc - 1, q - 1);
    // recompute Z_{k0} .. Z_{k1} into seg[0 .. k1-k0]
    RCF_CUDA(ctx, cudaMemcpyAsync(segp(0), ckp(j, 1), blk, cudaMemcpyDeviceToDevice, ctx->stream));
    for (int k = k0; k < k1; ++k) {
      const Real* Zk = segp(k - k0);
      const Real* Zkm1 = (k == k0) ? ckp(j, 0) : segp(k - k0 - 1);
      RCF_TRY(fwd(k, Zk, k == 1 ? nullptr : Zkm1, segp(k - k0 + 1)));
    }
    for (int k = k1; k >= k0; --k) {
      const double ak = 2.0 * ch.sigma[k + 1] / ch.e;
      const Real* Zk = segp(k - k0);
      // gradient: a_k Re tr(Zbar_{k+1}^H dH D^{-1} Z_k)
      RCF_TRY(launch_grad_local<Real>(ctx, m, zbk1, ld, Zk, ld, nvec, ak, 1, gnode));
      if (na > 0 && gh) {
        RCF_TRY(launch_nl_project<Real>(ctx, op, zbk1, ld, nvec, 1, CW));   // P^H Zbar = beta^T M Zbar
        RCF_TRY(launch_nl_project<Real>(ctx, op, Zk, ld, nvec, 0, CU));     // P^H D^{-1} Z = beta^T Z
        RCF_TRY(launch_grad_h<Real>(ctx, op, CW, CU, nvec, ak, gh));
      }
      // Rbar += a_k Lambda_k Zbar_{k+1}
      RCF_TRY(launch_axpy_cols<Real>(ctx, rows, zbk1, ld, tab_d + size_t(k) * nvec, nvec, Rbar, ld));
      // Zbar_k = a_k (D^{-1} H - c) Zbar_{k+1} - b_{k+1} Zbar_{k+2}
      Real* out = zbk2 ? zbk2 : freebufs[0];
      StepArgs<Real> a = step_args<Real>(zbk1, ld, out, ld, nvec, Real(ak), Real(-ak * ch.c));
      if (zbk2) { a.prev = zbk2; a.ld_prev = ld; a.C = Real(-ch.sigma[k + 1] * ch.sigma[k + 2]); }
      RCF_TRY(apply_full<Real>(ctx, op, RCF_FORM_DINV_H, a));
      zbk2 = zbk1;
      zbk1 = out;
      // the third buffer: whichever of B0, B1, B2 is neither zbk1 nor zbk2
      Real* cand[3] = {B0, B1, B2};
      for (Real* c : cand)
        if (c != zbk1 && c != zbk2) { freebufs[0] = c; break; }
    }
  }
  // Rbar += s Zbar_1
  RCF_TRY(launch_axpy_cols<Real>(ctx, rows, zbk1, ld, tab_d + size_t(q) * nvec, nvec, Rbar, ld));
  // gradient of R = H X - M X Lambda: Re tr(Rbar^H dH X), with X in Real
  const Real* XR = nullptr;
  if (sizeof(Real) == sizeof(double)) {
    XR = reinterpret_cast<const Real*>(X);
    RCF_TRY(launch_grad_local<Real>(ctx, m, Rbar, ld, XR, ldx, nvec, 1.0, 0, gnode));
    if (na > 0 && gh) {
      RCF_TRY(launch_nl_project<Real>(ctx, op, Rbar, ld, nvec, 1, CW));
      RCF_TRY(launch_nl_project<Real>(ctx, op, XR, ldx, nvec, 1, CU));
      RCF_TRY(launch_grad_h<Real>(ctx, op, CW, CU, nvec, 1.0, gh));
    }
  } else {
    // widen Rbar to FP64 and use the FP64 X
    double* Rb64 = R64;
    RCF_TRY(launch_c64_to_c128(ctx, rows, reinterpret_cast<const float*>(Rbar), ld, nvec, Rb64, ld));
    RCF_TRY(launch_grad_local<double>(ctx, m, Rb64, ld, X, ldx, nvec, 1.0, 0, gnode));
    if (na > 0 && gh) {
      double *CW64 = nullptr, *CU64 = nullptr;
      const size_t bytes = sizeof(double) * 24 * size_t(na) * nvec;
      RCF_TRY(workspace(ctx, WS_NLC, bytes, reinterpret_cast<void**>(&CW64)));
      RCF_TRY(workspace(ctx, WS_NLC2, bytes, reinterpret_cast<void**>(&CU64)));
      RCF_TRY(launch_nl_project<double>(ctx, op, Rb64, ld, nvec, 1, CW64));
      RCF_TRY(launch_nl_project<double>(ctx, op, X, ldx, nvec, 1, CU64));
      RCF_TRY(launch_grad_h<double>(ctx, op, CW64, CU64, nvec, 1.0, gh));
    }
  }
  return RCF_OK;
}

}  // namespace
}  // namespace rcf

extern "C" int rcf_adjoint_filter(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx,
                                  int nvec, const double* ritz, int degree, const double bounds[3],
                                  int mode, int prec, const double* Ybar, int64_t ldyb,
                                  int ckpt_every, double* dV, double* dB, double* dh) {
  if (op && op->fm) return fail(ctx, RCF_ENOTSUP, "the adjoint filter is not available with the full consistent mass");
  if (!ctx || !op) return RCF_EINVAL;
  RCF_TRY(check_block(ctx, op, X, ldx, nvec, 8, "X"));
  RCF_TRY(check_block(ctx, op, Ybar, ldyb, nvec, 8, "Ybar"));
  if (mode != RCF_RCHFSI) return fail(ctx, RCF_ENOTSUP, "the adjoint is built for mode RCF_RCHFSI");
  if (prec != RCF_FP64 && prec != RCF_FP32) return fail(ctx, RCF_EINVAL, "unknown precision %d", prec);
  if (!dV || !dB) return fail(ctx, RCF_EINVAL, "dV and dB must be device buffers");
  if (nvec > 0 && !ritz) return fail(ctx, RCF_EINVAL, "ritz is NULL");
  if (ckpt_every < 1) return fail(ctx, RCF_EINVAL, "ckpt_every must be >= 1");
  Cheb ch;
  RCF_TRY(cheb_scalars(ctx, bounds, degree + 1, &ch));   // sigma up to q+1 for b_{k+1}
  if (nvec == 0) return RCF_OK;
  const rcf_mesh* m = op->mesh;
  const int na = op->proj.natoms;
  double* g = nullptr;
  RCF_TRY(workspace(ctx, WS_GRAD, sizeof(double) * (4 * size_t(m->nnodes) + 2 * size_t(std::max(na, 1))), reinterpret_cast<void**>(&g)));
  RCF_CUDA(ctx, cudaMemsetAsync(g, 0, sizeof(double) * (4 * size_t(m->nnodes) + 2 * size_t(std::max(na, 1))), ctx->stream));
  double* gh = (dh && na > 0) ? g + 4 * m->nnodes : nullptr;
  if (degree == 1) {
    // Y = D^{-1} s R + X Lambda_1: Rbar = s D^{-1} Ybar
    double* R64 = nullptr;
    RCF_TRY(workspace(ctx, WS_R64, sizeof(double) * 4 * size_t(m->nnodes) * nvec, reinterpret_cast<void**>(&R64)));
    const int64_t ld = 2 * m->nnodes;
    RCF_TRY(launch_scale_mass(ctx, m, Ybar, ldyb, nvec, -1.0, R64, ld));
    const double s = ch.sigma[1] / ch.e;
    RCF_TRY(launch_grad_local<double>(ctx, m, R64, ld, X, ldx, nvec, s, 0, g));
    if (gh) {
      double *CW = nullptr, *CU = nullptr;
      const size_t bytes = sizeof(double) * 24 * size_t(na) * nvec;
      RCF_TRY(workspace(ctx, WS_NLC, bytes, reinterpret_cast<void**>(&CW)));
      RCF_TRY(workspace(ctx, WS_NLC2, bytes, reinterpret_cast<void**>(&CU)));
      RCF_TRY(launch_nl_project<double>(ctx, op, R64, ld, nvec, 1, CW));
      RCF_TRY(launch_nl_project<double>(ctx, op, X, ldx, nvec, 1, CU));
      RCF_TRY(launch_grad_h<double>(ctx, op, CW, CU, nvec, s, gh));
    }
  } else if (prec == RCF_FP64) {
    RCF_TRY((adjoint_impl<double>(ctx, op, ch, degree, X, ldx, nvec, ritz, Ybar, ldyb, ckpt_every, g, gh)));
  } else {
    RCF_TRY((adjoint_impl<float>(ctx, op, ch, degree, X, ldx, nvec, ritz, Ybar, ldyb, ckpt_every, g, gh)));
  }
  RCF_TRY(launch_grad_to_quadrature(ctx, m, g, dV, dB));
  if (gh) {
    std::vector<double> tmp(2 * na);
    RCF_CUDA(ctx, cudaMemcpyAsync(tmp.data(), gh, sizeof(double) * 2 * na, cudaMemcpyDeviceToHost, ctx->stream));
    RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 2 * na; ++i) dh[i] += tmp[i];
  }
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RCF_OK;
}

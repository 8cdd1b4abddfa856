// Context, mesh and operator set-up (host, FP64), status reporting, scratch memory.
//
// Mesh (Section III-A, Eq. FEWfns): GLL nodes by Newton's iteration on
// (1 - x^2) P_p'(x) with the Legendre three-term recurrence, weights
// 2 / (p (p+1) P_p^2), Lagrange derivative matrix by barycentric weights
// (Berrut & Trefethen, SIAM Review 2004), 1D stiffness K1 = D^T diag(w) D.
// Operator (Eq. hloc, Eq. hnloc, Eq. cellHam): per-node 2x2 potential blocks
// and the spin-orbit projectors, uploaded once.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <vector>

#include "internal.h"

namespace rcf {

int fail(rcf_ctx* ctx, int status, const char* fmt, ...) {
  if (ctx) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return status;
}

int cuda_fail(rcf_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
  const int st = (e == cudaErrorMemoryAllocation) ? RCF_ENOMEM : RCF_ECUDA;
  return fail(ctx, st, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

int workspace(rcf_ctx* ctx, int slot, size_t bytes, void** out) {
  if (slot < 0 || slot >= WS_COUNT) return fail(ctx, RCF_EINVAL, "bad workspace slot");
  if (ctx->ws_ptr.size() < size_t(WS_COUNT)) {
    ctx->ws_ptr.resize(WS_COUNT, nullptr);
    ctx->ws_size.resize(WS_COUNT, 0);
  }
  bytes = std::max<size_t>((bytes + 255) & ~size_t(255), 256);
  if (ctx->ws_size[slot] < bytes) {
    if (ctx->ws_ptr[slot]) {
      RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      RCF_CUDA(ctx, cudaFree(ctx->ws_ptr[slot]));
    }
    ctx->ws_ptr[slot] = nullptr;
    ctx->ws_size[slot] = 0;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, RCF_ENOMEM, "scratch allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->ws_ptr[slot] = p;
    ctx->ws_size[slot] = bytes;
  }
  *out = ctx->ws_ptr[slot];
  return RCF_OK;
}

namespace {

void gll(int p, std::vector<double>* xi, std::vector<double>* w) {
  const int n = p + 1;
  const double pi = 3.14159265358979323846;
  std::vector<double> x(n), xold(n), P(size_t(n) * n);
  for (int i = 0; i < n; ++i) x[i] = std::cos(pi * i / p);   // Chebyshev-Gauss-Lobatto start
  for (int it = 0; it < 100; ++it) {
    xold = x;
    for (int i = 0; i < n; ++i) {
      P[size_t(i) * n + 0] = 1.0;
      if (p >= 1) P[size_t(i) * n + 1] = x[i];
      for (int k = 2; k <= p; ++k)
        P[size_t(i) * n + k] = ((2.0 * k - 1.0) * x[i] * P[size_t(i) * n + k - 1] - (k - 1.0) * P[size_t(i) * n + k - 2]) / k;
    }
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) {
      x[i] = xold[i] - (x[i] * P[size_t(i) * n + p] - P[size_t(i) * n + p - 1]) / (n * P[size_t(i) * n + p]);
      dmax = std::max(dmax, std::fabs(x[i] - xold[i]));
    }
    if (dmax < 1e-16) break;
  }
  xi->assign(n, 0.0);
  w->assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    // P_p at the final nodes
    double p0 = 1.0, p1 = x[i];
    for (int k = 2; k <= p; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x[i] * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double Pp = (p == 0) ? 1.0 : p1;
    (*xi)[n - 1 - i] = x[i];   // ascending
    (*w)[n - 1 - i] = 2.0 / (p * (p + 1.0) * Pp * Pp);
  }
  (*xi)[0] = -1.0;
  (*xi)[n - 1] = 1.0;
}

void derivative_matrix(const std::vector<double>& xi, std::vector<double>* D) {
  const int n = int(xi.size());
  std::vector<double> lam(n, 1.0);
  for (int a = 0; a < n; ++a)
    for (int m = 0; m < n; ++m)
      if (m != a) lam[a] /= (xi[a] - xi[m]);
  D->assign(size_t(n) * n, 0.0);
  for (int q = 0; q < n; ++q) {
    double diag = 0.0;
    for (int a = 0; a < n; ++a) {
      if (a == q) continue;
      const double v = (lam[a] / lam[q]) / (xi[q] - xi[a]);
      (*D)[size_t(q) * n + a] = v;
      diag -= v;
    }
    (*D)[size_t(q) * n + q] = diag;
  }
}

inline int64_t node_of(const rcf_mesh* m, int64_t e, int l) {
  const int np = m->np;
  const int a = l % np, b = (l / np) % np, c = l / (np * np);
  const int ex = int(e % m->n[0]), ey = int((e / m->n[0]) % m->n[1]), ez = int(e / (int64_t(m->n[0]) * m->n[1]));
  const int i = (ex * m->p + a) % m->G[0], j = (ey * m->p + b) % m->G[1], k = (ez * m->p + c) % m->G[2];
  return i + int64_t(m->G[0]) * (j + int64_t(m->G[1]) * k);
}

inline double wq(const rcf_mesh* m, int l) {
  const int np = m->np;
  return m->w[l % np] * m->w[(l / np) % np] * m->w[l / (np * np)] * m->detJ;
}

inline double node_coord(const rcf_mesh* m, int d, int idx) {
  return (idx / m->p) * m->h[d] + (m->xi[idx % m->p] + 1.0) * m->h[d] / 2.0;
}

template <typename T>
int upload(rcf_ctx* ctx, T** dst, const T* src, size_t n) {
  if (*dst) { cudaFree(*dst); *dst = nullptr; }
  if (n == 0) return RCF_OK;
  RCF_CUDA(ctx, cudaMalloc(reinterpret_cast<void**>(dst), sizeof(T) * n));
  RCF_CUDA(ctx, cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice));
  return RCF_OK;
}

void free_proj(ProjAtoms* pa) {
  cudaFree(pa->d_offsets); cudaFree(pa->d_node); cudaFree(pa->d_atom);
  cudaFree(pa->d_beta64); cudaFree(pa->d_beta32); cudaFree(pa->d_delta64); cudaFree(pa->d_delta32);
  cudaFree(pa->d_nodemap); cudaFree(pa->d_unode); cudaFree(pa->d_uoff); cudaFree(pa->d_uent);
  cudaFree(pa->d_betadf);
  *pa = ProjAtoms();
}

void build_delta(const rcf_ctx* ctx, ProjAtoms* pa, const double* pj) {
  pa->delta.assign(size_t(pa->natoms) * 288, 0.0);
  for (int a = 0; a < pa->natoms; ++a)
    for (int j = 0; j < 2; ++j)
      for (int f = 0; f < 6; ++f)
        for (int g = 0; g < 6; ++g) {
          const double h = pa->hcoup[2 * a + j];
          const size_t dst = size_t(a) * 288 + 2 * ((6 * j + f) * 12 + 6 * j + g);
          pa->delta[dst] = h * pj[2 * (j * 36 + f * 6 + g)];
          pa->delta[dst + 1] = h * pj[2 * (j * 36 + f * 6 + g) + 1];
        }
  (void)ctx;
}

}  // namespace
}  // namespace rcf

using namespace rcf;

extern "C" const char* rcf_status_string(int s) {
  switch (s) {
    case RCF_OK: return "ok";
    case RCF_EINVAL: return "invalid argument";
    case RCF_ENOMEM: return "out of memory";
    case RCF_ECUDA: return "CUDA error";
    case RCF_ENOTSPD: return "Gram matrix not positive definite";
    case RCF_ETIMEOUT: return "device wait timed out";
    case RCF_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

extern "C" const char* rcf_last_error(const rcf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

extern "C" int rcf_create(rcf_ctx** out, int device, void* stream) {
  if (!out) return RCF_EINVAL;
  *out = nullptr;
  rcf_ctx* ctx = new rcf_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  auto bail = [&](int st) {
    if (ctx->blas) cublasDestroy(ctx->blas);
    if (ctx->solver) cusolverDnDestroy(ctx->solver);
    if (ctx->d_pj) cudaFree(ctx->d_pj);
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return st;
  };
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return bail(RCF_ECUDA); }
  if (cublasCreate(&ctx->blas) != CUBLAS_STATUS_SUCCESS) return bail(RCF_ECUDA);
  if (cublasSetStream(ctx->blas, ctx->stream) != CUBLAS_STATUS_SUCCESS) return bail(RCF_ECUDA);
  if (cusolverDnCreate(&ctx->solver) != CUSOLVER_STATUS_SUCCESS) return bail(RCF_ECUDA);
  if (cusolverDnSetStream(ctx->solver, ctx->stream) != CUSOLVER_STATUS_SUCCESS) return bail(RCF_ECUDA);
  double pj[144];
  channel_projector_table(pj);
  if (cudaMalloc(&ctx->d_pj, sizeof(pj)) != cudaSuccess) { cudaGetLastError(); return bail(RCF_ENOMEM); }
  if (cudaMemcpy(ctx->d_pj, pj, sizeof(pj), cudaMemcpyHostToDevice) != cudaSuccess) return bail(RCF_ECUDA);
  if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return bail(RCF_ENOMEM); }
  if (cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) return bail(RCF_ECUDA);
  *out = ctx;
  return RCF_OK;
}

extern "C" int rcf_set_step_kernel(rcf_ctx* ctx, int kind) {
  if (!ctx) return RCF_EINVAL;
  if (kind != RCF_STEP_CPASYNC && kind != RCF_STEP_TMA) return fail(ctx, RCF_EINVAL, "unknown step kernel %d", kind);
  ctx->step_kernel = kind;
  return RCF_OK;
}

extern "C" int rcf_set_rr_arith(rcf_ctx* ctx, int kind) {
  if (!ctx) return RCF_EINVAL;
  if (kind != RCF_RR_FP64 && kind != RCF_RR_DF && kind != RCF_RR_TC && kind != RCF_RR_MIXED)
    return fail(ctx, RCF_EINVAL, "unknown Rayleigh-Ritz arithmetic %d", kind);
  ctx->rr_arith = kind;
  return RCF_OK;
}

extern "C" int64_t rcf_workspace_bytes(const rcf_ctx* ctx) {
  if (!ctx) return -1;
  int64_t b = 0;
  for (size_t i = 0; i < ctx->ws_ptr.size(); ++i)
    if (ctx->ws_ptr[i]) b += int64_t(ctx->ws_size[i]);
  return b;
}

extern "C" int rcf_set_wait_limit(rcf_ctx* ctx, int64_t polls) {
  if (!ctx) return RCF_EINVAL;
  if (polls < 0) return fail(ctx, RCF_EINVAL, "wait limit must be >= 0 polls");
  ctx->wait_limit = polls;
  return RCF_OK;
}

extern "C" int rcf_destroy(rcf_ctx* ctx) {
  if (!ctx) return RCF_OK;
  cudaStreamSynchronize(ctx->stream);
  for (void* p : ctx->ws_ptr) if (p) cudaFree(p);
  if (ctx->blas) cublasDestroy(ctx->blas);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  if (ctx->d_pj) cudaFree(ctx->d_pj);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
  if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
  delete ctx;
  return RCF_OK;
}

namespace rcf {
int check_device_error(rcf_ctx* ctx) {
  if (!ctx->d_err) return RCF_OK;
  int h = 0;
  RCF_CUDA(ctx, cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h != 0) {
    RCF_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    return fail(ctx, RCF_ETIMEOUT, "a device-side wait timed out (kernel returned early; results invalid)");
  }
  return RCF_OK;
}
}  // namespace rcf

extern "C" int rcf_sync(rcf_ctx* ctx) {
  if (!ctx) return RCF_EINVAL;
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return check_device_error(ctx);
}

extern "C" int rcf_mesh_create(rcf_ctx* ctx, const int ncell[3], const double side[3], int p, rcf_mesh** out) {
  if (!ctx || !out || !ncell || !side) return fail(ctx, RCF_EINVAL, "NULL argument");
  *out = nullptr;
  if (p < 1 || p > kMaxP) return fail(ctx, RCF_ENOTSUP, "degree p=%d outside 1..%d", p, kMaxP);
  for (int d = 0; d < 3; ++d) {
    if (ncell[d] < 1) return fail(ctx, RCF_EINVAL, "ncell[%d] must be >= 1", d);
    if (!(side[d] > 0.0) || !std::isfinite(side[d])) return fail(ctx, RCF_EINVAL, "side[%d] must be > 0", d);
    if (int64_t(ncell[d]) * p > (1 << 20)) return fail(ctx, RCF_EINVAL, "too many nodes along %d", d);
  }
  rcf_mesh* m = new rcf_mesh();
  m->ctx = ctx;
  m->p = p;
  m->np = p + 1;
  m->nnodes = 1;
  m->ncells = 1;
  for (int d = 0; d < 3; ++d) {
    m->n[d] = ncell[d];
    m->L[d] = side[d];
    m->h[d] = side[d] / ncell[d];
    m->G[d] = ncell[d] * p;
    m->nnodes *= m->G[d];
    m->ncells *= ncell[d];
  }
  if (m->nnodes > (int64_t(1) << 31) - 1) { delete m; return fail(ctx, RCF_EINVAL, "more than 2^31 nodes"); }
  m->nloc = m->np * m->np * m->np;
  gll(p, &m->xi, &m->w);
  derivative_matrix(m->xi, &m->D);
  m->K1.assign(size_t(m->np) * m->np, 0.0);
  for (int a = 0; a < m->np; ++a)
    for (int b = 0; b < m->np; ++b) {
      double s = 0.0;
      for (int q = 0; q < m->np; ++q) s += m->w[q] * m->D[size_t(q) * m->np + a] * m->D[size_t(q) * m->np + b];
      m->K1[size_t(a) * m->np + b] = s;
    }
  m->detJ = m->h[0] * m->h[1] * m->h[2] / 8.0;
  m->mass.assign(size_t(m->nnodes), 0.0);
  for (int64_t e = 0; e < m->ncells; ++e)
    for (int l = 0; l < m->nloc; ++l) m->mass[size_t(node_of(m, e, l))] += wq(m, l);
  std::vector<double> inv64(size_t(m->nnodes));
  std::vector<float> inv32(size_t(m->nnodes));
  for (int64_t I = 0; I < m->nnodes; ++I) {
    inv64[I] = 1.0 / m->mass[I];
    inv32[I] = float(inv64[I]);
  }
  cudaError_t err = cudaMalloc(&m->d_mass, sizeof(double) * m->nnodes);
  if (err == cudaSuccess) err = cudaMemcpy(m->d_mass, m->mass.data(), sizeof(double) * m->nnodes, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMalloc(&m->d_inv_mass64, sizeof(double) * m->nnodes);
  if (err == cudaSuccess) err = cudaMemcpy(m->d_inv_mass64, inv64.data(), sizeof(double) * m->nnodes, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMalloc(&m->d_inv_mass32, sizeof(float) * m->nnodes);
  if (err == cudaSuccess) err = cudaMemcpy(m->d_inv_mass32, inv32.data(), sizeof(float) * m->nnodes, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    cudaFree(m->d_mass);
    cudaFree(m->d_inv_mass64);
    cudaFree(m->d_inv_mass32);
    delete m;
    return cuda_fail(ctx, err, "mass upload", __FILE__, __LINE__);
  }
  *out = m;
  return RCF_OK;
}

extern "C" int rcf_mesh_destroy(rcf_mesh* m) {
  if (!m) return RCF_OK;
  cudaFree(m->d_mass);
  cudaFree(m->d_inv_mass64);
  cudaFree(m->d_inv_mass32);
  delete m;
  return RCF_OK;
}

extern "C" int rcf_mesh_info(const rcf_mesh* m, int64_t* nnodes, int64_t* ncells, int* nloc) {
  if (!m) return RCF_EINVAL;
  if (nnodes) *nnodes = m->nnodes;
  if (ncells) *ncells = m->ncells;
  if (nloc) *nloc = m->nloc;
  return RCF_OK;
}

extern "C" int rcf_mesh_connectivity(const rcf_mesh* m, int32_t* out) {
  if (!m || !out) return RCF_EINVAL;
  for (int64_t e = 0; e < m->ncells; ++e)
    for (int l = 0; l < m->nloc; ++l) out[e * m->nloc + l] = int32_t(node_of(m, e, l));
  return RCF_OK;
}

extern "C" int rcf_mesh_quadrature_points(const rcf_mesh* m, double* out) {
  if (!m || !out) return RCF_EINVAL;
  const int np = m->np;
  for (int64_t e = 0; e < m->ncells; ++e) {
    const int ex = int(e % m->n[0]), ey = int((e / m->n[0]) % m->n[1]), ez = int(e / (int64_t(m->n[0]) * m->n[1]));
    const int ec[3] = {ex, ey, ez};
    for (int l = 0; l < m->nloc; ++l) {
      const int loc[3] = {l % np, (l / np) % np, l / (np * np)};
      for (int d = 0; d < 3; ++d)
        out[(e * m->nloc + l) * 3 + d] = ec[d] * m->h[d] + (m->xi[loc[d]] + 1.0) * m->h[d] / 2.0;
    }
  }
  return RCF_OK;
}

extern "C" int rcf_mesh_mass(const rcf_mesh* m, double* out) {
  if (!m || !out) return RCF_EINVAL;
  std::memcpy(out, m->mass.data(), sizeof(double) * m->nnodes);
  return RCF_OK;
}

extern "C" int rcf_op_create(rcf_ctx* ctx, const rcf_mesh* mesh, rcf_op** out) {
  if (!ctx || !mesh || !out) return fail(ctx, RCF_EINVAL, "NULL argument");
  *out = nullptr;
  rcf_op* op = new rcf_op();
  op->ctx = ctx;
  op->mesh = mesh;
  int s = rcf_potential_set(op, nullptr, nullptr, 0);
  if (s != RCF_OK) { rcf_op_destroy(op); return s; }
  *out = op;
  return RCF_OK;
}

extern "C" int rcf_op_destroy(rcf_op* op) {
  if (!op) return RCF_OK;
  if (op->ctx) cudaStreamSynchronize(op->ctx->stream);
  cudaFree(op->d_pot64);
  cudaFree(op->d_pot32);
  cudaFree(op->d_potdf);
  free_proj(&op->proj);
  free_fm(op->fm);
  delete op;
  return RCF_OK;
}

extern "C" int rcf_potential_set(rcf_op* op, const double* V, const double* B, int on_device) {
  if (!op) return RCF_EINVAL;
  rcf_ctx* ctx = op->ctx;
  const rcf_mesh* m = op->mesh;
  const size_t nq = size_t(m->ncells) * (op->fm ? op->fm->nq * op->fm->nq * op->fm->nq : m->nloc);
  std::vector<double> hv, hb;
  if (V && on_device) {
    hv.resize(nq);
    RCF_CUDA(ctx, cudaMemcpy(hv.data(), V, sizeof(double) * nq, cudaMemcpyDeviceToHost));
    V = hv.data();
  }
  if (B && on_device) {
    hb.resize(3 * nq);
    RCF_CUDA(ctx, cudaMemcpy(hb.data(), B, sizeof(double) * 3 * nq, cudaMemcpyDeviceToHost));
    B = hb.data();
  }
  if (op->fm) return fm_set_potential(ctx, op, V, B);
  std::vector<double> pot(4 * size_t(m->nnodes), 0.0);
  if (V || B) {
    for (int64_t e = 0; e < m->ncells; ++e)
      for (int l = 0; l < m->nloc; ++l) {
        const size_t I = size_t(node_of(m, e, l));
        const size_t q = size_t(e) * m->nloc + l;
        const double w = wq(m, l);
        if (V) pot[4 * I] += w * V[q];
        if (B)
          for (int d = 0; d < 3; ++d) pot[4 * I + 1 + d] += w * B[d * nq + q];
      }
    for (int64_t I = 0; I < m->nnodes; ++I)
      for (int c = 0; c < 4; ++c) pot[4 * I + c] /= m->mass[I];
  }
  for (double x : pot)
    if (!std::isfinite(x)) return fail(ctx, RCF_EINVAL, "potential contains a non-finite value");
  std::vector<float> pot32(pot.begin(), pot.end());
  // double-float copy for the residual: (pv+bz, pv-bz, bx, by) / M_I, hi then lo
  std::vector<float> potdf(8 * size_t(m->nnodes));
  for (int64_t I = 0; I < m->nnodes; ++I) {
    const double* q = &pot[4 * I];
    const double c[4] = {q[0] + q[3], q[0] - q[3], q[1], q[2]};
    for (int k = 0; k < 4; ++k) {
      const float h = float(c[k]);
      potdf[8 * I + k] = h;
      potdf[8 * I + 4 + k] = float(c[k] - double(h));
    }
  }
  RCF_TRY(upload(ctx, &op->d_pot64, pot.data(), pot.size()));
  RCF_TRY(upload(ctx, &op->d_pot32, pot32.data(), pot32.size()));
  RCF_TRY(upload(ctx, &op->d_potdf, potdf.data(), potdf.size()));
  return RCF_OK;
}

extern "C" int rcf_projectors_set(rcf_op* op, int natoms, const double* pos, const double* width,
                                  const double* h, double rcut_factor) {
  if (!op) return RCF_EINVAL;
  rcf_ctx* ctx = op->ctx;
  const rcf_mesh* m = op->mesh;
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  free_proj(&op->proj);
  if (natoms == 0) return RCF_OK;
  if (natoms < 0 || !pos || !width || !h) return fail(ctx, RCF_EINVAL, "bad projector arguments");
  if (!(rcut_factor > 0.0)) return fail(ctx, RCF_EINVAL, "rcut_factor must be > 0");
  ProjAtoms pa;
  pa.natoms = natoms;
  pa.offsets.assign(natoms + 1, 0);
  pa.hcoup.assign(h, h + 2 * natoms);
  const double pi = 3.14159265358979323846;
  if (op->fm) RCF_TRY(fm_projector_entries(ctx, op, natoms, pos, width, rcut_factor, &pa.node, &pa.atom, &pa.beta,
                                           &pa.offsets));
  for (int a = 0; a < natoms && !op->fm; ++a) {
    for (int j = 0; j < 2; ++j)
      if (!(width[2 * a + j] > 0.0)) return fail(ctx, RCF_EINVAL, "projector width must be > 0");
    const double rc = rcut_factor * std::max(width[2 * a], width[2 * a + 1]);
    // candidate indices per axis (minimum image), ascending
    std::vector<int> cand[3];
    std::vector<double> off[3];
    for (int d = 0; d < 3; ++d) {
      for (int i = 0; i < m->G[d]; ++i) {
        double dd = node_coord(m, d, i) - pos[3 * a + d];
        dd -= m->L[d] * std::nearbyint(dd / m->L[d]);
        if (std::fabs(dd) < rc) { cand[d].push_back(i); off[d].push_back(dd); }
      }
    }
    double Nj[2], s2[2], rj2[2];
    for (int j = 0; j < 2; ++j) {
      const double s = width[2 * a + j];
      Nj[j] = std::sqrt(2.0 / (std::pow(pi, 1.5) * std::pow(s, 5)));
      s2[j] = s * s;
      rj2[j] = (rcut_factor * s) * (rcut_factor * s);
    }
    for (size_t kz = 0; kz < cand[2].size(); ++kz)
      for (size_t ky = 0; ky < cand[1].size(); ++ky)
        for (size_t kx = 0; kx < cand[0].size(); ++kx) {
          const double d[3] = {off[0][kx], off[1][ky], off[2][kz]};
          const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          if (!(r2 < rc * rc)) continue;
          const int64_t I = cand[0][kx] + int64_t(m->G[0]) * (cand[1][ky] + int64_t(m->G[1]) * cand[2][kz]);
          pa.node.push_back(int(I));
          pa.atom.push_back(a);
          for (int j = 0; j < 2; ++j) {
            const double g = (r2 < rj2[j]) ? Nj[j] * std::exp(-r2 / (2.0 * s2[j])) : 0.0;
            for (int i = 0; i < 3; ++i) pa.beta.push_back(g * d[i]);
          }
        }
    pa.offsets[a + 1] = int(pa.node.size());
  }
  pa.nent = int64_t(pa.node.size());
  std::vector<double> pj(144);
  channel_projector_table(pj.data());
  build_delta(ctx, &pa, pj.data());
  std::vector<float> b32(pa.beta.begin(), pa.beta.end()), d32(pa.delta.begin(), pa.delta.end());
  RCF_TRY(upload(ctx, &pa.d_offsets, pa.offsets.data(), pa.offsets.size()));
  RCF_TRY(upload(ctx, &pa.d_node, pa.node.data(), pa.node.size()));
  RCF_TRY(upload(ctx, &pa.d_atom, pa.atom.data(), pa.atom.size()));
  RCF_TRY(upload(ctx, &pa.d_beta64, pa.beta.data(), pa.beta.size()));
  RCF_TRY(upload(ctx, &pa.d_beta32, b32.data(), b32.size()));
  RCF_TRY(upload(ctx, &pa.d_delta64, pa.delta.data(), pa.delta.size()));
  RCF_TRY(upload(ctx, &pa.d_delta32, d32.data(), d32.size()));
  // union of the supports: entry ids grouped by node, node -> union index
  {
    std::vector<int> order(pa.nent);
    for (int64_t e = 0; e < pa.nent; ++e) order[e] = int(e);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return pa.node[x] < pa.node[y]; });
    std::vector<int> nodemap(m->nnodes, -1), uoff(1, 0), unode;
    for (int64_t k = 0; k < pa.nent; ++k) {
      const int I = pa.node[order[k]];
      if (k == 0 || pa.node[order[k - 1]] != I) {
        if (k > 0) uoff.push_back(int(k));
        nodemap[I] = int(uoff.size()) - 1;
        unode.push_back(I);
      }
    }
    if (pa.nent > 0) uoff.push_back(int(pa.nent));
    pa.nunion = int(uoff.size()) - 1;
    std::vector<float> bdf(12 * size_t(pa.nent));
    for (size_t i = 0; i < 6 * size_t(pa.nent); ++i) {
      const float h = float(pa.beta[i]);
      bdf[2 * i] = h;
      bdf[2 * i + 1] = float(pa.beta[i] - double(h));
    }
    RCF_TRY(upload(ctx, &pa.d_nodemap, nodemap.data(), nodemap.size()));
    RCF_TRY(upload(ctx, &pa.d_unode, unode.data(), unode.size()));
    RCF_TRY(upload(ctx, &pa.d_uoff, uoff.data(), uoff.size()));
    RCF_TRY(upload(ctx, &pa.d_uent, order.data(), order.size()));
    RCF_TRY(upload(ctx, &pa.d_betadf, bdf.data(), bdf.size()));
  }
  op->proj = pa;
  return RCF_OK;
}

extern "C" int rcf_projectors_couplings(rcf_op* op, const double* h) {
  if (!op || !h) return RCF_EINVAL;
  rcf_ctx* ctx = op->ctx;
  ProjAtoms& pa = op->proj;
  if (pa.natoms == 0) return RCF_OK;
  RCF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  pa.hcoup.assign(h, h + 2 * pa.natoms);
  std::vector<double> pj(144);
  channel_projector_table(pj.data());
  build_delta(ctx, &pa, pj.data());
  std::vector<float> d32(pa.delta.begin(), pa.delta.end());
  RCF_CUDA(ctx, cudaMemcpy(pa.d_delta64, pa.delta.data(), sizeof(double) * pa.delta.size(), cudaMemcpyHostToDevice));
  RCF_CUDA(ctx, cudaMemcpy(pa.d_delta32, d32.data(), sizeof(float) * d32.size(), cudaMemcpyHostToDevice));
  return RCF_OK;
}

extern "C" int rcf_projector_support(const rcf_op* op, int atom, int64_t* count, int32_t* nodes) {
  if (!op || !count) return RCF_EINVAL;
  const ProjAtoms& pa = op->proj;
  if (atom < 0 || atom >= pa.natoms) return RCF_EINVAL;
  *count = pa.offsets[atom + 1] - pa.offsets[atom];
  if (nodes)
    for (int e = pa.offsets[atom]; e < pa.offsets[atom + 1]; ++e) nodes[e - pa.offsets[atom]] = pa.node[e];
  return RCF_OK;
}

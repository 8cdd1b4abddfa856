// rcf_apply_noalloc: the Hamiltonian-multivector product without any memory allocation.
//
// rcf_apply keeps the spin-orbit projector coefficients (C = P^H X and
// C' = Delta C, natoms x 12 x nvec complex) in scratch buffers that the
// context allocates on first use.  Some callers cannot let a library call
// cudaMalloc: for example a host whose device memory is already claimed by its
// own pooling allocator, or a latency-sensitive service loop that forbids
// allocation (and the device-wide synchronisation it implies) after start-up.
// For them this variant keeps that scratch in a fixed array in device memory
// that is part of the loaded library (every GPU that loads the library holds
// it until the process exits) and allocates nothing.
#include "internal.h"

namespace rcf {
namespace {

// Capacity: natoms * nvec <= kNoallocAtomVectors; two arrays (C, C') of
// natoms * 12 * nvec complex doubles each: 2 * 16384 * 24 doubles = 6.29 MB.
constexpr int64_t kNoallocAtomVectors = 16384;
constexpr int64_t kNoallocDoubles = 2 * kNoallocAtomVectors * 24;

static __device__ __align__(256) double g_projector_scratch[kNoallocDoubles];

// Device address of g_projector_scratch for the context's device, looked up on the first call
// on that context with its device current (host code must not use the symbol itself as a
// device pointer).  Kept per context, so a context created after a cudaDeviceReset looks it up
// again instead of keeping an address from before the reset.
int scratch_address(rcf_ctx* ctx, void** out) {
  if (!ctx->noalloc_scratch) {
    int cur = -1;
    RCF_CUDA(ctx, cudaGetDevice(&cur));
    if (cur != ctx->device) RCF_CUDA(ctx, cudaSetDevice(ctx->device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_projector_scratch);
    if (cur != ctx->device) cudaSetDevice(cur);
    if (e != cudaSuccess || !p) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_projector_scratch)", __FILE__, __LINE__);
    ctx->noalloc_scratch = p;
  }
  *out = ctx->noalloc_scratch;
  return RCF_OK;
}

bool block_ok(const rcf_op* op, const void* p, int64_t ld, size_t real) {
  const int64_t rows = 2 * op->mesh->nnodes;
  return p && ld >= rows && (ld & 1) == 0 && (reinterpret_cast<uintptr_t>(p) % (4 * real)) == 0;
}

template <typename Real>
int apply_noalloc(rcf_ctx* ctx, const rcf_op* op, int form, const Real* X, int64_t ldx, int nvec,
                  Real* Y, int64_t ldy, const Real* pot, Real* C, Real* C2) {
  StepArgs<Real> a{};
  a.in = X; a.ld_in = ldx;
  a.out = Y; a.ld_out = ldy;
  a.A = Real(1); a.B = Real(0); a.C = Real(0);
  a.nvec = nvec;
  a.pot = pot;
  a.mass = op->mesh->d_mass;
  int proj_mass = 1, add_mass = 1;
  if (form == RCF_FORM_H_DINV) { proj_mass = 0; add_mass = 1; a.scale_out = 0; }
  else if (form == RCF_FORM_DINV_H) { proj_mass = 1; add_mass = 0; a.scale_out = 0; }
  else { proj_mass = 1; add_mass = 1; a.scale_out = 1; }
  Tables t;
  build_tables(op->mesh, form == RCF_FORM_H_DINV ? TAB_COL_SCALED : TAB_ROW_SCALED, &t);
  const bool nl = op->proj.natoms > 0;
  if (nl) {
    // C and C' are overwritten in full by the projection and the coupling launches,
    // so nothing left in the shared array by an earlier call is read.
    RCF_TRY(launch_nl_project<Real>(ctx, op, X, ldx, nvec, proj_mass, C));
    RCF_TRY(launch_nl_delta<Real>(ctx, op, C, nvec, Real(1), C2));
  }
  RCF_TRY(launch_step<Real>(ctx, op->mesh, t, a));
  if (nl) RCF_TRY(launch_nl_addback<Real>(ctx, op, C2, nvec, add_mass, Y, ldy));
  return RCF_OK;
}

}  // namespace
}  // namespace rcf

using namespace rcf;

extern "C" int rcf_apply_noalloc(rcf_ctx* ctx, const rcf_op* op, int form, const void* X,
                                 int64_t ldx, int nvec, void* Y, int64_t ldy, int prec) {
  if (!ctx || !op) return RCF_EINVAL;
  if (op->fm) return fail(ctx, RCF_ENOTSUP, "rcf_apply_noalloc is not available with the full consistent mass");
  if (form < 0 || form > 2) return fail(ctx, RCF_EINVAL, "unknown form %d", form);
  if (prec != RCF_FP64 && prec != RCF_FP32) return fail(ctx, RCF_EINVAL, "unknown precision %d", prec);
  if (nvec < 0) return fail(ctx, RCF_EINVAL, "nvec < 0");
  if (nvec == 0) return RCF_OK;
  const size_t real = prec == RCF_FP64 ? 8 : 4;
  if (!block_ok(op, X, ldx, real) || !block_ok(op, Y, ldy, real))
    return fail(ctx, RCF_EINVAL, "X or Y: NULL, misaligned, or leading dimension below 2M / odd");
  {
    const char* x0 = static_cast<const char*>(X);
    const char* y0 = static_cast<const char*>(Y);
    if (x0 < y0 + size_t(ldy) * nvec * 2 * real && y0 < x0 + size_t(ldx) * nvec * 2 * real)
      return fail(ctx, RCF_EINVAL, "Y overlaps X");
  }
  const int64_t atom_vectors = int64_t(op->proj.natoms) * nvec;
  if (atom_vectors > kNoallocAtomVectors)
    return fail(ctx, RCF_EINVAL,
                "rcf_apply_noalloc: natoms * nvec = %lld exceeds the fixed scratch capacity of %lld "
                "(apply fewer vectors per call, or use rcf_apply)",
                (long long)atom_vectors, (long long)kNoallocAtomVectors);
  void* base = nullptr;
  RCF_TRY(scratch_address(ctx, &base));
  const size_t half = size_t(kNoallocAtomVectors) * 24;   // doubles per array
  if (prec == RCF_FP64) {
    double* C = static_cast<double*>(base);
    return apply_noalloc<double>(ctx, op, form, static_cast<const double*>(X), ldx, nvec,
                                 static_cast<double*>(Y), ldy, op->d_pot64, C, C + half);
  }
  float* C = static_cast<float*>(base);
  return apply_noalloc<float>(ctx, op, form, static_cast<const float*>(X), ldx, nvec,
                              static_cast<float*>(Y), ldy, op->d_pot32, C, C + 2 * half);
}

// Separable spin-orbit projectors (Eq. hnloc; Section III-B-3 stage iv):
//   H_nloc = sum_a P_a Delta_a P_a^H,  P_a column (j, i, sigma) = M_I beta_{j,i}(x_I) in row 2I+sigma.
// Applied in three launches: projection C = P^H (.) (a block reduction per
// atom and vector: register accumulators, warp shuffles, shared memory),
// the 12x12 coupling C' = A Delta C, and the add-back, gathered per node of
// the union of the supports (each node sums the terms of every atom whose
// support holds it, then updates its output once: no atomics where the
// supports of neighbouring atoms overlap).
#include <type_traits>

#include "internal.h"
#include "stencil_common.cuh"

namespace rcf {
namespace {

// a stored value as arithmetic type and back (round to nearest even)
template <typename Real, typename St>
__device__ __forceinline__ Real to_real(St x) {
  if constexpr (std::is_same_v<St, __half>) return Real(__half2float(x));
  else if constexpr (std::is_same_v<St, __nv_bfloat16>) return Real(__bfloat162float(x));
  else return Real(x);
}
template <typename St, typename Real>
__device__ __forceinline__ St from_real(Real x) {
  if constexpr (std::is_same_v<St, __half>) return __float2half_rn(float(x));
  else if constexpr (std::is_same_v<St, __nv_bfloat16>) return __float2bfloat16_rn(float(x));
  else return St(x);
}

// (re, im) of one complex value as a single 8-byte (float) or 16-byte (double) load
__device__ __forceinline__ void ld_pair(const float* p, float& re, float& im) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  re = t.x;
  im = t.y;
}
__device__ __forceinline__ void ld_pair(const double* p, double& re, double& im) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(p));
  re = t.x;
  im = t.y;
}

template <typename Real>
__device__ __forceinline__ Real warp_sum(Real x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

constexpr int kProjThreads = 128;

// grid (natoms, nvec); C[(a*12 + f)*nvec + v] complex
template <typename Real, typename St>
__global__ void __launch_bounds__(kProjThreads)
    nl_project_kernel(const int* __restrict__ off, const int* __restrict__ node,
                      const Real* __restrict__ beta, const double* __restrict__ mass,
                      const St* __restrict__ in, int64_t ld, int nvec, int proj_mass,
                      Real* __restrict__ C) {
  const int a = blockIdx.x, v = blockIdx.y;
  const int e0 = off[a], e1 = off[a + 1];
  const St* x = in + 2 * int64_t(v) * ld;
  Real acc[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) acc[i] = Real(0);
  // two support entries per pass, their node tuples loaded whole, so that two independent
  // index -> value load chains are in flight per thread
  const R4<St>* xt = reinterpret_cast<const R4<St>*>(x);
  for (int e = e0 + threadIdx.x; e < e1; e += 2 * kProjThreads) {
    const int e2 = e + kProjThreads;
    const bool two = e2 < e1;
    const int I = node[e], I2 = two ? node[e2] : I;
    const R4<St> t1 = ldgs(xt + I), t2 = ldgs(xt + I2);
    const Real w1 = proj_mass ? Real(mass[I]) : Real(1);
    const Real w2 = two ? (proj_mass ? Real(mass[I2]) : Real(1)) : Real(0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const R4<St>& t = h ? t2 : t1;
      const Real w = h ? w2 : w1;
      const int64_t eb = 6 * int64_t(h ? (two ? e2 : e) : e);
      const Real ur = to_real<Real>(t.v[0]), ui = to_real<Real>(t.v[1]);
      const Real dr = to_real<Real>(t.v[2]), di = to_real<Real>(t.v[3]);
#pragma unroll
      for (int f6 = 0; f6 < 6; ++f6) {          // f6 = 3 j + i
        const Real b = w * beta[eb + f6];
        const int f = 2 * f6;                   // 6 j + 2 i + sigma = 2 (3 j + i) + sigma
        acc[2 * f + 0] += b * ur;
        acc[2 * f + 1] += b * ui;
        acc[2 * (f + 1) + 0] += b * dr;
        acc[2 * (f + 1) + 1] += b * di;
      }
    }
  }
  __shared__ Real red[kProjThreads / 32][24];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 24; ++i) {
    const Real s = warp_sum(acc[i]);
    if (lane == 0) red[wid][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < 24) {
    Real s = Real(0);
#pragma unroll
    for (int w = 0; w < kProjThreads / 32; ++w) s += red[w][threadIdx.x];
    const int f = threadIdx.x >> 1, part = threadIdx.x & 1;
    C[2 * ((int64_t(a) * 12 + f) * nvec + v) + part] = s;
  }
}

// thread per (atom, vector)
template <typename Real>
__global__ void nl_delta_kernel(const Real* __restrict__ delta, const Real* __restrict__ C, int natoms,
                                int nvec, Real A, Real* __restrict__ C2out) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(natoms) * nvec) return;
  const int a = int(t / nvec), v = int(t % nvec);
  Real cr[12], ci[12];
#pragma unroll
  for (int f = 0; f < 12; ++f) {
    cr[f] = C[2 * ((int64_t(a) * 12 + f) * nvec + v)];
    ci[f] = C[2 * ((int64_t(a) * 12 + f) * nvec + v) + 1];
  }
  const Real* D = delta + int64_t(a) * 288;
#pragma unroll
  for (int f = 0; f < 12; ++f) {
    Real sr = 0, si = 0;
#pragma unroll
    for (int g = 0; g < 12; ++g) {
      const Real dr = D[2 * (f * 12 + g)], di = D[2 * (f * 12 + g) + 1];
      sr += dr * cr[g] - di * ci[g];
      si += dr * ci[g] + di * cr[g];
    }
    C2out[2 * ((int64_t(a) * 12 + f) * nvec + v)] = A * sr;
    C2out[2 * ((int64_t(a) * 12 + f) * nvec + v) + 1] = A * si;
  }
}

// grid (ceil(nunion/128), ceil(nvec/NV)); thread per node of the support union and NV
// consecutive vectors: the node's outputs gain w sum_e beta_e C2[atom_e][.][v] over its
// support entries e, in one read-modify-write per vector.  The entry lists and beta are
// read once for the NV vectors; C2[a][f][v..v+NV) is contiguous.
constexpr int kAddbackNV = 8;
template <typename Real, typename St>
__global__ void nl_addback_kernel(const int* __restrict__ unode, const int* __restrict__ uoff,
                                  const int* __restrict__ uent, const int* __restrict__ atom,
                                  const Real* __restrict__ beta, const double* __restrict__ mass,
                                  int nunion, const Real* __restrict__ C2, int nvec, int add_mass,
                                  St* out, int64_t ld) {
  constexpr int NV = kAddbackNV;
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v0 = blockIdx.y * NV;
  if (u >= nunion) return;
  const int I = unode[u];
  const int nv = min(NV, nvec - v0);
  // the node's outputs of the NV vectors, loaded as whole tuples before any update
  R4<St> y[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j)
    if (j < nv) y[j] = ld4(reinterpret_cast<const R4<St>*>(out + 2 * int64_t(v0 + j) * ld) + I);
  Real s[NV][4];
#pragma unroll
  for (int j = 0; j < NV; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) s[j][i] = Real(0);
  for (int k = uoff[u]; k < uoff[u + 1]; ++k) {
    const int e = uent[k];
    const int a = atom[e];
#pragma unroll
    for (int f6 = 0; f6 < 6; ++f6) {
      const Real b = beta[6 * int64_t(e) + f6];
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        // the complex coefficients of NV consecutive vectors, one (re, im) word each
        const Real* c = C2 + 2 * ((int64_t(a) * 12 + 2 * f6 + sg) * nvec + v0);
#pragma unroll
        for (int j = 0; j < NV; ++j)
          if (j < nv) {
            Real re, im;
            ld_pair(c + 2 * j, re, im);
            s[j][2 * sg + 0] += b * re;
            s[j][2 * sg + 1] += b * im;
          }
      }
    }
  }
  const Real w = add_mass ? Real(mass[I]) : Real(1);
#pragma unroll
  for (int j = 0; j < NV; ++j)
    if (j < nv) {
#pragma unroll
      for (int i = 0; i < 4; ++i) y[j].v[i] = from_real<St>(to_real<Real>(y[j].v[i]) + w * s[j][i]);
      st4(reinterpret_cast<R4<St>*>(out + 2 * int64_t(v0 + j) * ld) + I, y[j]);
    }
}

// gh[a][j] += wgt Re sum_v CW[a,(j,.,.)]^H P_j CU[a,(j,.,.)]; thread per (a, v), atomics
template <typename Real>
__global__ void grad_h_kernel(const double* __restrict__ pj, const Real* __restrict__ CW,
                              const Real* __restrict__ CU, int natoms, int nvec, double wgt,
                              double* gh) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(natoms) * nvec) return;
  const int a = int(t / nvec), v = int(t % nvec);
  for (int j = 0; j < 2; ++j) {
    double s = 0;
    for (int f = 0; f < 6; ++f) {
      double tr = 0, ti = 0;
      for (int g = 0; g < 6; ++g) {
        const double pr = pj[2 * (j * 36 + f * 6 + g)], pi = pj[2 * (j * 36 + f * 6 + g) + 1];
        const int64_t k = 2 * ((int64_t(a) * 12 + 6 * j + g) * nvec + v);
        const double ur = CU[k], ui = CU[k + 1];
        tr += pr * ur - pi * ui;
        ti += pr * ui + pi * ur;
      }
      const int64_t k = 2 * ((int64_t(a) * 12 + 6 * j + f) * nvec + v);
      s += double(CW[k]) * tr + double(CW[k + 1]) * ti;   // Re(conj(w) t)
    }
    atomicAdd(gh + 2 * a + j, wgt * s);
  }
}

}  // namespace

template <typename Real>
static const Real* beta_of(const rcf_op* op);
template <>
const double* beta_of<double>(const rcf_op* op) { return op->proj.d_beta64; }
template <>
const float* beta_of<float>(const rcf_op* op) { return op->proj.d_beta32; }
template <typename Real>
static const Real* delta_of(const rcf_op* op);
template <>
const double* delta_of<double>(const rcf_op* op) { return op->proj.d_delta64; }
template <>
const float* delta_of<float>(const rcf_op* op) { return op->proj.d_delta32; }

template <typename Real, typename St>
int launch_nl_project(rcf_ctx* ctx, const rcf_op* op, const St* in, int64_t ld, int nvec,
                      int proj_mass, Real* C) {
  const ProjAtoms& pa = op->proj;
  if (pa.natoms == 0 || nvec == 0) return RCF_OK;
  dim3 grid(pa.natoms, nvec);
  nl_project_kernel<Real, St><<<grid, kProjThreads, 0, ctx->stream>>>(
      pa.d_offsets, pa.d_node, beta_of<Real>(op), op->mesh->d_mass, in, ld, nvec, proj_mass, C);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

template <typename Real>
int launch_nl_delta(rcf_ctx* ctx, const rcf_op* op, const Real* C, int nvec, Real A, Real* C2) {
  const ProjAtoms& pa = op->proj;
  if (pa.natoms == 0 || nvec == 0) return RCF_OK;
  const int64_t n = int64_t(pa.natoms) * nvec;
  nl_delta_kernel<Real><<<unsigned((n + 127) / 128), 128, 0, ctx->stream>>>(
      delta_of<Real>(op), C, pa.natoms, nvec, A, C2);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

template <typename Real, typename St>
int launch_nl_addback(rcf_ctx* ctx, const rcf_op* op, const Real* C2, int nvec, int add_mass,
                      St* out, int64_t ld) {
  const ProjAtoms& pa = op->proj;
  if (pa.natoms == 0 || nvec == 0 || pa.nunion == 0) return RCF_OK;
  dim3 grid(unsigned((pa.nunion + 127) / 128), unsigned((nvec + kAddbackNV - 1) / kAddbackNV));
  nl_addback_kernel<Real, St><<<grid, 128, 0, ctx->stream>>>(pa.d_unode, pa.d_uoff, pa.d_uent, pa.d_atom,
                                                          beta_of<Real>(op), op->mesh->d_mass, pa.nunion,
                                                          C2, nvec, add_mass, out, ld);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

// channel projectors P_j (6x6 complex each, j = 0: 1/2, 1: 3/2) on index 2 i + sigma:
// P_{1/2} = (1 - L.s)/3, P_{3/2} = (2 + L.s)/3, (L_k)_{ij} = -i eps_{kij}, L.s = sum_k L_k (x) sigma_k
void channel_projector_table(double* h /* [2][6][6] complex */) {
  double Lim[3][3][3] = {};
  auto eps = [](int k, int i, int j) -> double {
    if (k == i || i == j || k == j) return 0.0;
    return ((k + 1) % 3 == i) ? 1.0 : -1.0;
  };
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Lim[k][i][j] = -eps(k, i, j);
  const double sre[3][2][2] = {{{0, 1}, {1, 0}}, {{0, 0}, {0, 0}}, {{1, 0}, {0, -1}}};
  const double sim[3][2][2] = {{{0, 0}, {0, 0}}, {{0, -1}, {1, 0}}, {{0, 0}, {0, 0}}};
  for (int j = 0; j < 2; ++j)
    for (int f = 0; f < 6; ++f)
      for (int g = 0; g < 6; ++g) {
        const int i1 = f / 2, s1 = f % 2, i2 = g / 2, s2 = g % 2;
        double lr = 0, li = 0;   // (L_k)_{i1 i2} (sigma_k)_{s1 s2}, L purely imaginary
        for (int k = 0; k < 3; ++k) {
          lr += -Lim[k][i1][i2] * sim[k][s1][s2];
          li += Lim[k][i1][i2] * sre[k][s1][s2];
        }
        const double id = (f == g) ? 1.0 : 0.0;
        h[2 * (j * 36 + f * 6 + g)] = (j == 0) ? (id - lr) / 3.0 : (2.0 * id + lr) / 3.0;
        h[2 * (j * 36 + f * 6 + g) + 1] = (j == 0) ? -li / 3.0 : li / 3.0;
      }
}

template <typename Real>
int launch_grad_h(rcf_ctx* ctx, const rcf_op* op, const Real* CW, const Real* CU, int nvec,
                  double wgt, double* gh) {
  const ProjAtoms& pa = op->proj;
  if (pa.natoms == 0 || nvec == 0) return RCF_OK;
  const double* pj = ctx->d_pj;
  const int64_t n = int64_t(pa.natoms) * nvec;
  grad_h_kernel<Real><<<unsigned((n + 127) / 128), 128, 0, ctx->stream>>>(pj, CW, CU, pa.natoms,
                                                                           nvec, wgt, gh);
  RCF_CHECK_LAUNCH(ctx);
  return RCF_OK;
}

#define INST(R)                                                                                  \
  template int launch_nl_project<R, R>(rcf_ctx*, const rcf_op*, const R*, int64_t, int, int, R*); \
  template int launch_nl_delta<R>(rcf_ctx*, const rcf_op*, const R*, int, R, R*);              \
  template int launch_nl_addback<R, R>(rcf_ctx*, const rcf_op*, const R*, int, int, R*, int64_t); \
  template int launch_grad_h<R>(rcf_ctx*, const rcf_op*, const R*, const R*, int, double, double*);
INST(float)
INST(double)
#undef INST
#define INST16(S)                                                                                 \
  template int launch_nl_project<float, S>(rcf_ctx*, const rcf_op*, const S*, int64_t, int, int, float*); \
  template int launch_nl_addback<float, S>(rcf_ctx*, const rcf_op*, const float*, int, int, S*, int64_t);
INST16(__half)
INST16(__nv_bfloat16)
#undef INST16

}  // namespace rcf

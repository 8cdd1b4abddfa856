// Internal types of librchfsi: context, mesh, operator, kernel launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "rchfsi.h"

namespace rcf {

constexpr int kMaxP = 8;

// ---------------------------------------------------------------------------
// error plumbing: every failing call records a message in the context
// ---------------------------------------------------------------------------
struct Error {
  int status;
  std::string msg;
};

}  // namespace rcf

struct rcf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t solver = nullptr;
  std::string last_error;
  double* d_pj = nullptr;   // spin-orbit channel projectors P_{1/2}, P_{3/2} (6x6 complex each)
  int64_t launches = 0;     // kernels launched by this library on this context
  int* d_err = nullptr;     // device error word: set by a kernel whose bounded wait timed out
  int step_kernel = RCF_STEP_CPASYNC;   // FP32 step kernel (rcf_set_step_kernel)
  int rr_arith = RCF_RR_TC;             // tall products of Cholesky-QR and Rayleigh-Ritz (rcf_set_rr_arith)
  int64_t wait_limit = int64_t(1) << 24;   // polls of a bounded device-side wait (rcf_set_wait_limit)
  void* noalloc_scratch = nullptr;          // device address of rcf_apply_noalloc's fixed array
  cudaStream_t copy_in = nullptr;       // host-to-device and device-to-host streams of
  cudaStream_t copy_out = nullptr;      // rcf_filter_host (created on first use)
  // grow-only scratch buffers, one per slot
  std::vector<void*> ws_ptr;
  std::vector<size_t> ws_size;
};

struct rcf_mesh {
  rcf_ctx* ctx = nullptr;
  int n[3];        // cells per direction
  double L[3];     // sides
  double h[3];     // cell edges
  int p, np;       // degree, nodes per direction per cell
  int G[3];        // nodes per direction
  int64_t nnodes, ncells;
  int nloc;
  std::vector<double> xi, w;  // GLL nodes and weights on [-1, 1]
  std::vector<double> D;      // D[q*np + a] = l_a'(xi_q)
  std::vector<double> K1;     // K1[a*np + b] = sum_q w_q D[q,a] D[q,b]
  double detJ;
  std::vector<double> mass;   // host M_I
  double* d_mass = nullptr;   // device M_I
  double* d_inv_mass64 = nullptr;   // device 1 / M_I
  float* d_inv_mass32 = nullptr;
};

struct ProjAtoms {
  int natoms = 0;
  std::vector<int> offsets;      // [natoms + 1] entry ranges
  std::vector<int> node;         // [nent] support nodes (sorted per atom)
  std::vector<int> atom;         // [nent]
  std::vector<double> beta;      // [nent][6]  column 3 j + i
  std::vector<double> delta;     // [natoms][12][12] complex (re, im) interleaved
  std::vector<double> hcoup;     // [natoms][2]
  // device copies
  int* d_offsets = nullptr;
  int* d_node = nullptr;
  int* d_atom = nullptr;
  double* d_beta64 = nullptr;
  float* d_beta32 = nullptr;
  double* d_delta64 = nullptr;   // [natoms][144] complex
  float* d_delta32 = nullptr;
  int64_t nent = 0;
  // union of the supports, for the double-float residual: entries grouped by node
  int nunion = 0;
  int* d_nodemap = nullptr;      // [nnodes] union index or -1
  int* d_unode = nullptr;        // [nunion] node of each union index
  int* d_uoff = nullptr;         // [nunion + 1]
  int* d_uent = nullptr;         // [nent] entry ids, grouped by node
  float* d_betadf = nullptr;     // [nent][6][2] beta (hi, lo)
};

// Full consistent mass with Gauss-Legendre quadrature (Section III-A; Section III-B-2): the
// operator's integrals use nq Gauss points per direction; D (the lumped GLL mass) stays the
// filter's diagonal in place of M^-1.
struct FullMass {
  int nq = 0;
  std::vector<double> gx, gw;     // Gauss nodes and weights on [-1, 1]
  std::vector<double> B1;         // [nq][np] Lagrange basis l_a at the Gauss nodes
  // 1D assembled rows per direction d and local position a (0 = element vertex), offsets
  // -p .. p: K = 1/2 (2 / h_d) K1 (stiffness), M = (h_d / 2) M1 (consistent mass);
  // layout [2 (K, M)][3][p][2p + 1]
  std::vector<double> tab;
  // element matrices per direction d: K = 1/2 (2 / h_d) K1 and M = (h_d / 2) M1,
  // layout [2 (K, M)][3][np][np]
  std::vector<double> el;
  double* d_tab64 = nullptr;
  float* d_tab32 = nullptr;
  double* d_B1_64 = nullptr;      // [nq][np]
  float* d_B1_32 = nullptr;
  double* d_vq64 = nullptr;       // [ncells][nq^3][4]: w_q |J| (V, Bx, By, Bz)
  float* d_vq32 = nullptr;
};

struct rcf_op {
  rcf_ctx* ctx = nullptr;
  const rcf_mesh* mesh = nullptr;
  FullMass* fm = nullptr;      // non-null: full consistent mass, Gauss quadrature
  double* d_pot64 = nullptr;   // [nnodes][4] (pv, pbx, pby, pbz) / M_I
  float* d_pot32 = nullptr;
  float* d_potdf = nullptr;    // [nnodes][8] (pv+bz, pv-bz, bx, by) / M_I: hi[4], lo[4]
  ProjAtoms proj;
};

namespace rcf {

// ---------------------------------------------------------------------------
// status helpers
// ---------------------------------------------------------------------------
int fail(rcf_ctx* ctx, int status, const char* fmt, ...);
int cuda_fail(rcf_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);

#define RCF_CUDA(ctx, expr)                                                   \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) return rcf::cuda_fail((ctx), _e, #expr, __FILE__, __LINE__); \
  } while (0)

#define RCF_CHECK_LAUNCH(ctx)          \
  do {                                 \
    ++(ctx)->launches;                 \
    RCF_CUDA(ctx, cudaGetLastError()); \
  } while (0)

#define RCF_TRY(expr)              \
  do {                             \
    int _s = (expr);               \
    if (_s != RCF_OK) return _s;   \
  } while (0)

// grow-only scratch buffer `slot` of at least `bytes`
int workspace(rcf_ctx* ctx, int slot, size_t bytes, void** out);
enum WsSlot {
  WS_R64 = 0, WS_R32, WS_ZA, WS_ZB, WS_COEF, WS_NLC, WS_NLC2, WS_LANCZOS, WS_RR_W, WS_RR_S,
  WS_RR_T, WS_RR_INFO, WS_RR_WORK, WS_GRAD, WS_CKPT, WS_ADJ_A, WS_ADJ_B, WS_ADJ_C, WS_ADJ_U,
  WS_NORM, WS_DF_LAM, WS_DF_C2, WS_DF_NL, WS_HX0, WS_HY0, WS_R16, WS_SCALE, WS_GEMM_PART, WS_TC_A, WS_TC_B, WS_TC_E, WS_TC_C, WS_TC_Q, WS_PCG, WS_FM_U, WS_FM_T, WS_FM_T1, WS_FM_T2,
  WS_FM_S1, WS_FM_S2, WS_FM_CELL, WS_FM_W, WS_RBFP, WS_HTAB, WS_COUNT
};

// ---------------------------------------------------------------------------
// stencil step (stencil.cu)
//
//   out = A * (D^{-1} H_loc or H_loc D^{-1}) in + B * in + C * prev + g[v] * rv
//   then optionally out *= M_I
// where H_loc = kinetic + spinor potential (Eq. hloc, Eq. cellHam).
// ---------------------------------------------------------------------------
// Real: arithmetic type; St: storage type of the multivectors (Real, or a 16-bit float
// type with FP32 arithmetic)
template <typename Real, typename St = Real>
struct StepArgs {
  const St* in;      int64_t ld_in;     // complex elements per vector (even)
  const St* prev;    int64_t ld_prev;   // may be null
  const St* rv;      int64_t ld_rv;     // may be null
  const double* g;                      // [nvec] coefficients of rv (device), may be null
  const unsigned char* rv_bfp;          // instead of rv (FP32 only): R as a 12-bit BFP stream,
                                        // block v * nnodes + node (4-byte aligned), may be null
  St* out;           int64_t ld_out;
  Real A, B, C;
  const Real* pot;                      // [nnodes][4]
  const double* mass;                   // used if scale_out
  int scale_out;
  int nvec;
};

// coefficient tables for the three 1D operators: coef[d][a][a']
struct Tables {
  double c[3][kMaxP + 1][kMaxP + 1];
};
enum TableKind { TAB_ROW_SCALED = 0 /* D^{-1} H */, TAB_COL_SCALED = 1 /* H D^{-1} */ };
void build_tables(const rcf_mesh* m, int kind, Tables* t);

template <typename Real, typename St = Real>
int launch_step(rcf_ctx* ctx, const rcf_mesh* m, const Tables& t, const StepArgs<Real, St>& a);
// FP32 step with TMA plane loads (stencil_tma.cu); *used = false when it does not apply
// (degree, tile divisibility, alignment, tensor-map encoding) and the caller falls back.
int launch_step_tma(rcf_ctx* ctx, const rcf_mesh* m, const Tables& t, const StepArgs<float>& a, bool* used);
// RCF_ETIMEOUT (and clear the word) if a kernel recorded a timed-out wait; synchronises
int check_device_error(rcf_ctx* ctx);

// ---------------------------------------------------------------------------
// double-float residual (residual_df.cu)
// ---------------------------------------------------------------------------
// Rh = RN32(R), Rl = R - Rh (if not null), R = H X - M X diag(lambda) evaluated in
// double-float arithmetic (local part, spin-orbit projectors included); neglam_d =
// -lambda (device, FP64).  X c128 [nvec][ldx], Rh/Rl c64 [nvec][ldr].
int launch_residual_df(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                       const double* neglam_d, float* Rh, float* Rl, int64_t ldr);
// C (m x n, column-major, ldc) = A^H diag(w) B for complex FP64 A (K x m), B (K x n), w the
// weight of complex row k = w[k >> 1] (null: 1), in double-float arithmetic; lower: only
// the tiles on or below the diagonal of a square C (Hermitian A^H A)  (gemm_df.cu)
int launch_gemm_tn_df(rcf_ctx* ctx, const double* A, int64_t lda, const double* B, int64_t ldb,
                      const double* w, int64_t K, int m, int n, int lower, double* C, int64_t ldc);
// FP64-accurate products on the bf16 tensor cores (gemm_tc.cu):
// C (n x nz complex, ldc) = Y^H diag(w) Z over nrows complex rows (w[r / 2], null: 1;
// lower: only C(i, j), i >= j, when Z == Y), and X (nrows x n) = Y Q (X may equal Y; mixed:
// the off-diagonal part of Q at FP32-level accuracy plus the diagonal part in FP64)
int tc_gemm_tn(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* w, const double* Z, int64_t ldz,
               int nz, int64_t nrows, double* C, int64_t ldc, int lower);
int tc_rotate(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Q, int64_t ldq, int64_t nrows,
              double* X, int64_t ldx, bool mixed = false);
// hi[i], lo[i] = double-float split of x[i] (integer operations only)
int launch_split_f64(rcf_ctx* ctx, int64_t n, const double* x, float* hi, float* lo);

// ---------------------------------------------------------------------------
// nonlocal projectors (nonlocal.cu)
// ---------------------------------------------------------------------------
// C[a][f][v] = sum_e w_e beta_e[j,i] in[v][node_e][sigma],  f = 6 j + 2 i + sigma,
// w_e = M_node if proj_mass else 1.   C is complex (Real2) [natoms][12][nvec].
template <typename Real, typename St = Real>
int launch_nl_project(rcf_ctx* ctx, const rcf_op* op, const St* in, int64_t ld, int nvec,
                      int proj_mass, Real* C);
// C2 = A * Delta_a C
template <typename Real>
int launch_nl_delta(rcf_ctx* ctx, const rcf_op* op, const Real* C, int nvec, Real A, Real* C2);
// out[v][node_e][sigma] += w_e sum_{j,i} beta_e[j,i] C2[a][6j+2i+sigma][v], w_e = M if add_mass
template <typename Real, typename St = Real>
int launch_nl_addback(rcf_ctx* ctx, const rcf_op* op, const Real* C2, int nvec, int add_mass,
                      St* out, int64_t ld);

// ---------------------------------------------------------------------------
// vector kernels (vectors.cu)
// ---------------------------------------------------------------------------
// y[v][r] = s(r) * x[v][r], s = M_I^pow (pow in {-1, -0.5, 0.5, 1}) or 1 (pow = 0)
int launch_scale_mass(rcf_ctx* ctx, const rcf_mesh* m, const double* x, int64_t ldx, int nvec,
                      double pw, double* y, int64_t ldy);
// Y = dinv * Z * zs + X * lam[v]     (recovery, Algorithm 1)
template <typename ZReal>
int launch_recover(rcf_ctx* ctx, const rcf_mesh* m, const ZReal* Z, int64_t ldz, double zs,
                   const double* X, int64_t ldx, const double* lam, int nvec, double* Y,
                   int64_t ldy);
// y = (float) x, and optional column norms^2 accumulated into nrm2 (device, pre-zeroed)
int launch_to_c64(rcf_ctx* ctx, int64_t rows, const double* x, int64_t ldx, int nvec, float* y,
                  int64_t ldy);
int launch_colnorm2(rcf_ctx* ctx, int64_t rows, const double* x, int64_t ldx, int nvec,
                    double* nrm2);
// 16-bit storage of the recurrence: per-column largest modulus of a complex64 block (as
// float bits; cmax pre-zeroed), the power-of-two scale above it and its reciprocal, the
// scaled copy in the storage type, and the recovery Y = D^{-1} Z zscale[v] + X lam[v]
// 12-bit BFP storage of n floats (n a multiple of 4, x 16-byte aligned): the stream s
// (6 bytes per 4 values) receives their encoding and x the decoded values (bfp.cu)
int launch_bfp12_round_trip(rcf_ctx* ctx, float* x, int64_t n, unsigned char* s);
int launch_colmax_f32(rcf_ctx* ctx, int64_t rows, const float* x, int64_t ldx, int nvec, unsigned* cmax);
int launch_pow2_scale(rcf_ctx* ctx, const unsigned* cmax, int n, double* scale, float* inv);
template <typename St>
int launch_to_storage(rcf_ctx* ctx, int64_t rows, const float* x, int64_t ldx, int nvec, const float* inv,
                      St* y, int64_t ldy);
template <typename St>
int launch_recover_scaled(rcf_ctx* ctx, const rcf_mesh* m, const St* Z, int64_t ldz, const double* zscale,
                          const double* X, int64_t ldx, const double* lam, int nvec, double* Y, int64_t ldy);
int launch_sqrt_inplace(rcf_ctx* ctx, double* v, int n);
int launch_copy_c128(rcf_ctx* ctx, int64_t rows, const double* x, int64_t ldx, int nvec,
                     double* y, int64_t ldy);
int launch_c64_to_c128(rcf_ctx* ctx, int64_t rows, const float* x, int64_t ldx, int nvec,
                       double* y, int64_t ldy);
// Lanczos helpers on single vectors of length n complex
int launch_dot_re(rcf_ctx* ctx, int64_t n, const double* a, const double* b, double* out);
int launch_lanczos_update(rcf_ctx* ctx, int64_t n, double* w, const double* v,
                          const double* vprev, double alpha, double beta);
int launch_scale_vec(rcf_ctx* ctx, int64_t n, const double* x, double s, double* y);

// ---------------------------------------------------------------------------
// gradients (nonlocal.cu / vectors.cu)
// ---------------------------------------------------------------------------
// gnode[0][I] += wgt Re sum_v W^H U ; gnode[1+d][I] += wgt Re sum_v W^H sigma_d U
// (U scaled by 1/M_I first if u_dinv)
template <typename Real>
int launch_grad_local(rcf_ctx* ctx, const rcf_mesh* m, const Real* W, int64_t ldw, const Real* U,
                      int64_t ldu, int nvec, double wgt, int u_dinv, double* gnode);
// gh[a][j] += wgt Re sum_v CW^H P_j CU  (CW, CU from launch_nl_project with mass weights)
template <typename Real>
int launch_grad_h(rcf_ctx* ctx, const rcf_op* op, const Real* CW, const Real* CU, int nvec,
                  double wgt, double* gh);
void channel_projector_table(double* h /* [2][6][6] complex */);
// dV[e][l] += |J| w_l gnode[0][I(e,l)], dB[d][e][l] += |J| w_l gnode[1+d][I(e,l)]
int launch_grad_to_quadrature(rcf_ctx* ctx, const rcf_mesh* m, const double* gnode, double* dV,
                              double* dB);

// full consistent mass (fullmass.cu): the same contract as apply_full for an operator with
// op->fm (form H: out = A H in + M (B in + C prev + g rv), M the full mass; the other
// forms as apply_full), and Y = M X
template <typename Real>
int apply_full_fm(rcf_ctx* ctx, const rcf_op* op, int form, const StepArgs<Real, Real>& a);
template <typename Real>
int mass_apply_fm(rcf_ctx* ctx, const rcf_op* op, const Real* X, int64_t ldx, int nvec, Real* Y, int64_t ldy);
void free_fm(FullMass* fm);
// set-up of the full-mass operator (fullmass.cu): the Gauss-point potential, and the projector
// entries (node, atom, column / D_I) with the per-atom offsets
int fm_set_potential(rcf_ctx* ctx, rcf_op* op, const double* V, const double* B);
int fm_projector_entries(rcf_ctx* ctx, const rcf_op* op, int natoms, const double* pos, const double* width,
                         double rcut_factor, std::vector<int>* node, std::vector<int>* atom,
                         std::vector<double>* beta, std::vector<int>* offsets);

// the Hamiltonian-multivector product with the nonlocal part (filter.cu)
template <typename Real, typename St = Real>
int apply_full(rcf_ctx* ctx, const rcf_op* op, int form, const StepArgs<Real, St>& a);

}  // namespace rcf

/*
 * rchfsi.h - C ABI of the GB300 (sm_103a) R-ChFSI filter library (librchfsi.so).
 *
 * What it computes (arXiv 2605.30128):
 *   the residual-based Chebyshev filtered subspace iteration (R-ChFSI) for the
 *   noncollinear / spin-orbit finite-element eigenproblem H X = M X Lambda
 *   (Section III-B-2, Eq. ghep, Eq. rChFSIrecurrence, Algorithm 1), with
 *   H = H_loc + H_nloc (Eq. hloc, Eq. hnloc, Eq. cellHam) discretised on a
 *   periodic hexahedral mesh with Lagrange degree p on GLL nodes (Section
 *   III-A, Eq. FEWfns) and the GLL-lumped diagonal mass D = M.
 *
 * Conventions shared by every entry point
 *   - Numbering: global node I = i + Gx (j + Gy k) with G_d = ncell_d * p;
 *     cell e = ex + nx (ey + ny ez); local node l = a + np (b + np c),
 *     np = p + 1; spinor row 2 I + alpha (alpha = 0 up, 1 down).
 *   - Multivectors are COLUMN-MAJOR complex arrays: vector j starts at
 *     element j * ld and holds rows 0 .. 2M-1 contiguously; ld >= 2M and ld
 *     even, counted in complex elements.  "c128" = interleaved (re, im)
 *     doubles; base pointers 32-byte aligned.  They are DEVICE pointers
 *     unless stated otherwise, owned by the caller, on the device of the
 *     context.
 *   - Every call returns an rcf_status (0 = OK) and never throws; the text of
 *     the last failure is rcf_last_error(ctx).  Work is enqueued on the
 *     context's stream; results are valid after that stream synchronises.
 *     Calls that return host scalars (Lanczos bounds, Rayleigh-Ritz values)
 *     synchronise the stream themselves.
 *   - Nothing here allocates memory that the caller must free, except the
 *     handles, which the matching *_destroy releases.  Scratch memory is owned
 *     by the context and reused across calls.
 */
#ifndef RCHFSI_H
#define RCHFSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rcf_ctx rcf_ctx;
typedef struct rcf_mesh rcf_mesh;
typedef struct rcf_op rcf_op;

typedef enum {
  RCF_OK = 0,
  RCF_EINVAL = 1,    /* bad argument: null pointer, size, alignment, bounds order */
  RCF_ENOMEM = 2,    /* device or host allocation failed */
  RCF_ECUDA = 3,     /* a CUDA, cuBLAS or cuSOLVER call failed */
  RCF_ENOTSPD = 4,   /* Cholesky-QR met a Gram matrix that is not positive definite */
  RCF_ETIMEOUT = 5,  /* a bounded device-side wait ran out */
  RCF_ENOTSUP = 6    /* combination not built (e.g. degree p > 8) */
} rcf_status;

/* Arithmetic of the filter's Hamiltonian-multivector products.  RCF_FP32_DF
 * (R-ChFSI only): FP32 recurrence as RCF_FP32, with the residual R evaluated in
 * double-float arithmetic (pairs of floats with exact products and error-free
 * sums: about 2^-46 relative accuracy, against 2^-52 for FP64) instead of FP64,
 * because this GPU runs FP64 at a small fraction of its FP32 rate.  The paper
 * keeps R in FP64 (Section III-C); this variant is the library's. */
typedef enum {
  RCF_FP64 = 0, RCF_FP32 = 1, RCF_FP32_DF = 2, RCF_FP16 = 3, RCF_BF16 = 4, RCF_FP32_BFP12 = 5
} rcf_precision;
/* RCF_FP16 / RCF_BF16 (R-ChFSI only; in rcf_apply and rcf_cheb_step the
 * multivectors are 16-bit complex pairs): the recurrence vectors Z_k, Z_{k-1}
 * and R are STORED as IEEE binary16 / bfloat16 pairs and the products are
 * computed in FP32 from them; R is the double-float residual, each column
 * scaled by the power of two that puts its largest entry in [1/2, 1) before
 * rounding (the recurrence is linear in (Z, R), so the scale returns exactly
 * in the recovery; results are reproducible bit for bit).  This halves the bytes per step
 * of the bandwidth-bound recurrence; the residual-proportional error bound
 * that lets the paper run the products in FP32/TF32 (Section III-C) covers the
 * 16-bit rounding of the stored vectors as well, since that error too scales
 * with ||R||.  The paper applies 16-bit and block-floating-point formats to
 * communicated data (Section III-C-3); this variant is the library's. */
/* RCF_FP32_BFP12 (R-ChFSI only; rcf_filter, rcf_filter_host, rcf_cheb_step):
 * the FP32 recurrence of RCF_FP32 with the FP64 residual R, rounded to FP32,
 * kept as a 12-bit block floating-point stream (Section III-C-3's format with
 * n_bits = 12: one 6-byte block per node 4-tuple (re_up, im_up, re_dn, im_dn)
 * and vector, as rcf_bfp_encode writes it).  Every use of R sees the decoded
 * values, and the steps read their g[v] R term from the stream: 6 bytes per
 * node and vector instead of 16, 27 instead of 32 bytes per DoF, vector and
 * degree.  The recurrence is linear in R, so the storage rounding (2^-9 of the
 * block's largest entry) is an error proportional to ||R||, the property of
 * Section III-B-2 that allows the low-precision recurrence.  In rcf_cheb_step,
 * Zk, Zkm1 and out are complex64 and R is such a stream: block v * nnodes + I
 * holds node I of column v, 4-byte aligned, 6 nnodes nvec bytes.  The paper
 * uses the format for communicated data; this storage use is the library's.
 * With the full mass it applies to the recurrence forms (rcf_cheb_step forms
 * H D^-1 and D^-1 H); rejected by rcf_apply. */

/* Filter form: plain ChFSI (Eq. ChFSIrecurrence) or R-ChFSI (Eq. rChFSIrecurrence). */
typedef enum { RCF_CHFSI = 0, RCF_RCHFSI = 1 } rcf_mode;

/* Operator form for rcf_apply: H, D^{-1} H or H D^{-1}. */
typedef enum { RCF_FORM_H = 0, RCF_FORM_DINV_H = 1, RCF_FORM_H_DINV = 2 } rcf_form;

/* FP32 step-kernel implementation (library-specific; the paper has no counterpart).
 * RCF_STEP_CPASYNC (default): per-thread cp.async staging of each z plane with one
 * block barrier per plane.  RCF_STEP_TMA: one producer thread issues five
 * tensor-memory-accelerator boxes per plane into an mbarrier ring (degrees 4..6,
 * meshes whose node counts in x and y the tile divides; other cases use the
 * default).  Both compute the same sums in the same order. */
typedef enum { RCF_STEP_CPASYNC = 0, RCF_STEP_TMA = 1 } rcf_step_kernel;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device`, enqueueing all work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream is borrowed,
 * not owned.  Creates the cuBLAS / cuSOLVER handles used by Rayleigh-Ritz. */
int rcf_create(rcf_ctx** out, int device, void* stream);
int rcf_destroy(rcf_ctx* ctx);
const char* rcf_status_string(int status);
const char* rcf_last_error(const rcf_ctx* ctx);
/* Block the host until the context's stream has finished. */
int rcf_sync(rcf_ctx* ctx);

/* ---- mesh (Section III-A) -------------------------------------------- */

/* Periodic box of ncell[0] x ncell[1] x ncell[2] hexahedral cells with sides
 * side[0..2] (bohr) and Lagrange degree p (1 <= p <= 8) on GLL nodes, GLL
 * quadrature collocated with the nodes.  Host arrays are copied. */
int rcf_mesh_create(rcf_ctx* ctx, const int ncell[3], const double side[3], int p, rcf_mesh** out);
int rcf_mesh_destroy(rcf_mesh* mesh);
/* Number of global nodes M (2M complex spinor DoF), cells, and nodes per cell (p+1)^3. */
int rcf_mesh_info(const rcf_mesh* mesh, int64_t* nnodes, int64_t* ncells, int* nloc);
/* Local-to-global map R^(e) (Section III-B-3, stage i) as int32 [ncells][nloc] into a host buffer. */
int rcf_mesh_connectivity(const rcf_mesh* mesh, int32_t* host_out);
/* Quadrature-point coordinates (= local GLL nodes, unwrapped) [ncells][nloc][3] into a host buffer. */
int rcf_mesh_quadrature_points(const rcf_mesh* mesh, double* host_out);
/* GLL-lumped mass M_I = sum_{(e,l) -> I} w_l |J|, [nnodes] into a host buffer. */
int rcf_mesh_mass(const rcf_mesh* mesh, double* host_out);

/* ---- operator: H and D = M (Eq. hloc, Eq. hnloc, Eq. cellHam) --------- */

/* Operator on a mesh; V = B = 0 and no projectors until set.  The mesh must
 * outlive the operator. */
int rcf_op_create(rcf_ctx* ctx, const rcf_mesh* mesh, rcf_op** out);
int rcf_op_destroy(rcf_op* op);
/* Spinor potential at quadrature points: V [ncells][nloc], B [3][ncells][nloc]
 * (B may be NULL for B = 0), FP64.  on_device = 0: host arrays; 1: device
 * arrays.  Each node receives the 2x2 block sum_e w_q |J| (V I + B . sigma).
 * Copied; the caller keeps ownership. */
int rcf_potential_set(rcf_op* op, const double* V, const double* B, int on_device);
/* Spin-orbit projectors (Eq. hnloc): per atom a, position pos[a][3], radial
 * widths width[a][2] and couplings h[a][2] for channels j = 1/2, 3/2 (host
 * arrays).  beta_{j,i}(r) = N_j d_i exp(-|d|^2 / 2 s_j^2) on |d| < rcut_factor
 * s_j (d: minimum-image offset, int beta^2 = 1); Delta_a = h_{1/2} P_{1/2} (+)
 * h_{3/2} P_{3/2}, P_{3/2} = (2 + L.sigma)/3, P_{1/2} = (1 - L.sigma)/3.
 * natoms = 0 removes them. */
int rcf_projectors_set(rcf_op* op, int natoms, const double* pos, const double* width,
                       const double* h, double rcut_factor);
/* Replace only the couplings h[natoms][2] (host). */
int rcf_projectors_couplings(rcf_op* op, const double* h);
/* Number of support nodes of atom `atom`; if host_nodes != NULL also the
 * sorted global node indices (int32, `*count` entries). */
int rcf_projector_support(const rcf_op* op, int atom, int64_t* count, int32_t* host_nodes);

/* ---- Hamiltonian-multivector products --------------------------------- */

/* Y = op(X) with op = H, D^{-1} H or H D^{-1} (rcf_form), for nvec vectors.
 * prec = RCF_FP64: X, Y are c128; prec = RCF_FP32: X, Y are complex64
 * (interleaved floats, 16-byte aligned).  Y must not overlap X. */
int rcf_apply(rcf_ctx* ctx, const rcf_op* op, int form, const void* X, int64_t ldx, int nvec,
              void* Y, int64_t ldy, int prec);

/* One step of the three-term recurrence (Eq. ChFSIrecurrence with form
 * RCF_FORM_DINV_H, Eq. rChFSIrecurrence with form RCF_FORM_H_DINV):
 *   out = alpha op(Zk) + beta Zk + gamma Zkm1 + g[v] R_v     (v = column)
 * Zk, Zkm1, R, out share the leading dimension ld; Zkm1, R and g (device
 * double [nvec]) may be NULL.  out may alias Zkm1 (updated in place) but not
 * Zk or R.  prec as in rcf_apply, or RCF_FP32_BFP12 with R a 12-bit BFP stream. */
int rcf_cheb_step(rcf_ctx* ctx, const rcf_op* op, int form, int prec, const void* Zk,
                  const void* Zkm1, const void* R, int64_t ld, int nvec, double alpha, double beta,
                  double gamma, const double* g, void* out);

/* rcf_apply without any memory allocation (the paper has no counterpart).
 * Same operation, arguments, layouts and errors as rcf_apply.  For callers
 * that cannot let a library allocate device memory: a host whose GPU memory
 * is already owned by its own pooling allocator, or a service loop that
 * forbids allocation (and the device-wide synchronisation of cudaMalloc)
 * after start-up.  The spin-orbit projector coefficients, which rcf_apply
 * keeps in context scratch memory, live here in one fixed array of 6.29 MB
 * inside the library's device image, present on every GPU that loads the
 * library until the process exits.  Limit: natoms * nvec <= 16384 per call;
 * larger calls return RCF_EINVAL with a message (split the vectors).  The
 * first call on a context looks up the array's device address with the
 * context's device current; with lazy module loading that first lookup may
 * load the library's device code, a driver-side allocation, so make the first
 * call at set-up, before any stream capture.  A context created after a
 * cudaDeviceReset looks the address up again.  All calls share the one
 * array: calls that may run at the same
 * time on the GPU (different streams or contexts) race and must be
 * serialised by the caller.  Nothing in the array needs clearing between
 * calls: each call overwrites the coefficients it reads. */
int rcf_apply_noalloc(rcf_ctx* ctx, const rcf_op* op, int form, const void* X, int64_t ldx,
                      int nvec, void* Y, int64_t ldy, int prec);

/* Bytes of device scratch memory this context holds (its grow-only slots,
 * allocated on first use by the calls that need them and freed by
 * rcf_destroy); library-specific, for memory accounting. */
int64_t rcf_workspace_bytes(const rcf_ctx* ctx);

/* Number of kernels this context has launched so far (its own kernels; the
 * dense library routines of Rayleigh-Ritz are not counted). */
int64_t rcf_launch_count(const rcf_ctx* ctx);

/* Select the FP32 step kernel of this context (rcf_step_kernel).  Returns
 * RCF_EINVAL for an unknown kind.  Takes effect at the next launch. */
int rcf_set_step_kernel(rcf_ctx* ctx, int kind);

/* Limit, in polls, of every bounded device-side wait of this context's kernels
 * (the mbarrier waits of the TMA step kernel; library-specific, the paper has
 * no counterpart).  Default 2^24.  A wait that reaches the limit makes its
 * kernel record a time-out in the context's device error word and return early
 * (after its own copies in flight have landed, under a separate fixed limit);
 * the next synchronising call then returns RCF_ETIMEOUT and clears the word, and
 * the context stays usable.  0 makes every such wait give up at once (used to
 * test this path).  Returns RCF_EINVAL for a negative limit. */
int rcf_set_wait_limit(rcf_ctx* ctx, int64_t polls);

/* Arithmetic of the tall products of Cholesky-QR and Rayleigh-Ritz: the Gram
 * matrix Y^H M Y, the projected matrix Y^H (H Y), the triangular update
 * Y L^{-H} and the rotation Y Q (library-specific; the paper has no
 * counterpart, it uses FP64 Level-3 BLAS).
 *   RCF_RR_FP64: cuBLAS ZHERK / ZGEMM / ZTRSM in FP64.
 *   RCF_RR_DF: the Gram and projected matrices in double-float arithmetic on
 *     the FP32 pipes (about 2^-46 relative to the magnitudes of the terms);
 *     the triangular update and the rotation stay cuBLAS FP64.
 *   RCF_RR_TC: all four on the bf16 tensor cores, FP64-accurate: every row of
 *     the left and column of the right operand is scaled by a power of two
 *     and split into 7 signed 8-bit digits (Ozaki-Ogita-Oishi-Rump error-free
 *     splitting, 56 bits), the 28 digit products with s + t <= 8 are summed
 *     exactly in FP32 over windows of 1024 terms and accumulated in 64-bit
 *     fixed point; the triangular update applies L^{-H} (cuSOLVER TRTRI on the
 *     n x n factor) as a rotation.  Error about 2^-55 of max|row| max|column|
 *     per term, against 2^-53 |term| for FP64.
 *   RCF_RR_MIXED: as RCF_RR_TC, except the Rayleigh-Ritz rotation X = Y Q,
 *     split as in Section III-C-4: Y Q_offdiag (Q with its diagonal set to zero)
 *     at FP32-level accuracy (3 digits of 8 bits, 6 digit products) plus
 *     Y diag(Q) in FP64.
 * The n x n factorisations (POTRF, TRTRI, HEEVD) are cuSOLVER FP64 in every
 * mode.  Default RCF_RR_TC. */
typedef enum { RCF_RR_FP64 = 0, RCF_RR_DF = 1, RCF_RR_TC = 2, RCF_RR_MIXED = 3 } rcf_rr_arith;
int rcf_set_rr_arith(rcf_ctx* ctx, int kind);

/* C (n x nz complex, column-major, ldc >= n) = Y^H diag(w) Z over nrows
 * complex rows: Y (nrows x n) and Z (nrows x nz) c128 with leading dimensions
 * ldy, ldz >= nrows (even), w device [nrows / 2] (the weight of both spinor
 * rows of a node; NULL: 1; nrows even when given).  arith as rcf_rr_arith.
 * Device buffers; C must not overlap Y or Z.  Asynchronous on the context's
 * stream.  (The building block of the Gram and projected matrices, Algorithm 1
 * RR step; the paper has no separate call.) */
int rcf_inner(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Z, int64_t ldz, int nz,
              int64_t nrows, const double* w, double* C, int64_t ldc, int arith);

/* X (nrows x n complex, ldx) = Y Q for Y (nrows x n, ldy) and Q (n x n
 * complex, column-major, ldq >= n), all device c128.  arith RCF_RR_FP64
 * (cuBLAS ZGEMM; X must not overlap Y), RCF_RR_TC (X may equal Y, with
 * ldx == ldy: the rotation in place; n <= 4096) or RCF_RR_MIXED (the
 * off-diagonal part at FP32-level accuracy plus the diagonal part in FP64;
 * X must not overlap Y).  Asynchronous on the context's stream.  (The subspace rotation of Algorithm 1 / Section
 * III-C-4.) */
int rcf_rotate(rcf_ctx* ctx, const double* Y, int64_t ldy, int n, const double* Q, int64_t ldq,
               int64_t nrows, double* X, int64_t ldx, int arith);

/* ---- filter bounds (Section III-B-2; Lanczos as in Section III-C-1) --- */

/* nsteps of Lanczos on D^{-1/2} H D^{-1/2} from the device c128 vector v0
 * [2M] (not modified; need not be normalised).  Writes host scalars:
 * *theta_min = smallest Ritz value, *upper = largest Ritz value + |beta_m|
 * (the filter's lambda_max).  Synchronises. */
int rcf_lanczos_bounds(rcf_ctx* ctx, const rcf_op* op, int nsteps, const double* v0,
                       double* theta_min, double* upper);

/* ---- residual (Algorithm 1, FP64) -------------------------------------- */

/* R = H X - M X diag(ritz) in FP64.  ritz: host [nvec].  R (c128, ld ldr) and
 * colnorm (device double [nvec], 2-norms of the columns of R) may each be
 * NULL when not wanted. */
int rcf_residual(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                 const double* ritz, double* R, int64_t ldr, double* colnorm);

/* The same residual in double-float arithmetic (the residual of RCF_FP32_DF;
 * no counterpart in the paper): Rh (c64) = the FP32 rounding of R, Rl (c64,
 * may be NULL) = R - Rh rounded to FP32, so Rh + Rl carries R to about 2^-46
 * relative to the sum of the magnitudes of its terms.  Rh and Rl share ldr and
 * must not overlap each other or X.  Synchronises. */
int rcf_residual_df(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                    const double* ritz, float* Rh, float* Rl, int64_t ldr);

/* ---- the filter (Eq. ChFSIrecurrence / Eq. rChFSIrecurrence) ---------- */

/* Y = filtered block of X, degree q = `degree` >= 1, bounds = {lambda_min,
 * lambda_T, lambda_max} (host; need lambda_min < lambda_T < lambda_max).
 * mode RCF_RCHFSI: R = H X - M X Lambda (FP64; double-float for
 * RCF_FP32_DF, FP16 and BF16), Z_0 = 0, Z_1 = sigma_1 R / e,
 * the residual recurrence in `prec` (RCF_FP32_BFP12: FP32 with R read from its
 * 12-bit BFP stream), Lambda_k propagated in FP64, recovery
 * Y = D^{-1} Z_q + X Lambda_q in FP64.  With the full mass (rcf_op_set_gauss)
 * R uses the consistent M and the products its Gauss-point operator, with D
 * the GLL-integrated diagonal (Section III-B-2); FP64 and FP32 only.  mode RCF_CHFSI: Eq. ChFSIrecurrence
 * with M^{-1} = D^{-1}; ritz may be NULL.  Vectors are processed in band
 * blocks of `block` columns (block <= 0: all at once).  X and Y are c128 and
 * must not overlap; ritz: host [nvec]. */
int rcf_filter(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
               const double* ritz, int degree, const double bounds[3], int mode, int prec,
               int block, double* Y, int64_t ldy);

/* rcf_filter with X and Y in HOST memory (c128, leading dimensions ldx, ldy
 * >= 2M; no counterpart in the paper).  Band blocks stream through two
 * device slots per direction: the next block is copied in and the previous one
 * copied out on two copy streams of the context while a block is filtered on
 * its compute stream, so copies and filtering overlap when X and Y are
 * page-locked (pinned) host memory; pageable memory works but its copies do
 * not overlap.  The coefficient tables of all blocks go to the device in one
 * copy ahead of the first block copy.  Device scratch: up to four blocks of
 * `block` c128 vectors besides the filter's own.  Synchronises; returns after Y
 * is complete. */
int rcf_filter_host(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                    const double* ritz, int degree, const double bounds[3], int mode, int prec,
                    int block, double* Y, int64_t ldy);

/* ---- Cholesky-QR2 + Rayleigh-Ritz (Algorithm 1, RR step) ---------------- */

/* Y (c128, in/out) is made M-orthonormal by Cholesky-QR applied twice
 * (S = Y^H M Y = L L^H, Y <- Y L^{-H}); then A = Y^H H Y is diagonalised and
 * X_out = Y Q (c128, must not overlap Y) receives the Ritz vectors, ritz_out
 * (host [nvec]) the Ritz values in ascending order.  Returns RCF_ENOTSPD if a
 * Gram matrix is not positive definite.  Synchronises. */
int rcf_rayleigh_ritz(rcf_ctx* ctx, const rcf_op* op, double* Y, int64_t ldy, int nvec,
                      double* X_out, int64_t ldx, double* ritz_out);

/* The two halves of rcf_rayleigh_ritz, callable (and timed) separately.
 * rcf_cholqr2: Y (c128, in/out) <- Y made M-orthonormal by Cholesky-QR applied
 * twice, with one shifted pass in front if the first Gram factorisation breaks
 * down (then RCF_ENOTSPD only if the shifted pass fails too); synchronises.
 * rcf_rayleigh_ritz_orth: for an M-orthonormal Y (not modified), A = Y^H H Y
 * (FP64), its eigenpairs, X_out = Y Q and ascending ritz_out as in
 * rcf_rayleigh_ritz; X_out must not overlap Y; synchronises. */
int rcf_cholqr2(rcf_ctx* ctx, const rcf_op* op, double* Y, int64_t ldy, int nvec);
int rcf_rayleigh_ritz_orth(rcf_ctx* ctx, const rcf_op* op, const double* Y, int64_t ldy, int nvec,
                           double* X_out, int64_t ldx, double* ritz_out);

/* ---- full consistent mass (Section III-A; Section III-B-2) ---------------- */

/* Switch the operator to the full consistent mass with nq Gauss-Legendre points
 * per direction (p + 1 <= nq <= 12; exact for the mass and kinetic integrals):
 * M_{2I+a,2J+b} = delta_ab int N_I N_J, the kinetic and potential integrals by
 * the same rule, V and B given at the Gauss points, the spin-orbit projector
 * columns int N_I beta.  D, the GLL-integrated (lumped) mass, stays the
 * filter's diagonal in place of M^-1, as in the paper.  Call before
 * rcf_potential_set / rcf_projectors_set, which then take V [ncells][nq^3] and
 * B [3][ncells][nq^3] at the points of rcf_op_gauss_points (point
 * q = qx + nq (qy + nq qz)).  With the full mass: rcf_apply (FP64, FP32),
 * rcf_cheb_step, rcf_residual (R = HX - M X Lambda with the full M),
 * rcf_filter (FP64; FP32 recurrence with the FP64 residual), the Lanczos
 * bound, Cholesky-QR and Rayleigh-Ritz (Y^H M Y with the full M) and
 * rcf_mass_apply; the double-float residual, 16-bit storage, the adjoint, the
 * gradients, the Ritz cotangent and rcf_apply_noalloc return RCF_ENOTSUP.
 * Synchronises. */
int rcf_op_set_gauss(rcf_op* op, int nq);

/* Coordinates of the Gauss points of a full-mass operator (host
 * [ncells][nq^3][3]).  RCF_EINVAL for a lumped operator. */
int rcf_op_gauss_points(const rcf_op* op, double* out);

/* Y = M X: the full consistent mass (three 1D passes) for an operator made
 * with rcf_op_set_gauss (prec RCF_FP64 or RCF_FP32), else the lumped diagonal
 * (RCF_FP64).  Layouts as rcf_apply; Y must not overlap X.  Asynchronous on
 * the context's stream. */
int rcf_mass_apply(rcf_ctx* ctx, const rcf_op* op, const void* X, int64_t ldx, int nvec, void* Y,
                   int64_t ldy, int prec);

/* ---- electrostatics: Poisson solve (Section III-B-1; Algorithm pcg_fusion) ---- */

/* y = K x for scalar nodal fields on the mesh (device FP64 [nnodes], node
 * I = x + G_x (y + G_y z)), K_IJ = int grad N_I . grad N_J the periodic FE
 * Laplacian, applied matrix-free (the paper's K x kernel; twice the kinetic
 * term of Eq. hloc).  y must not overlap x.  Asynchronous on the context's
 * stream. */
int rcf_laplacian(rcf_ctx* ctx, const rcf_mesh* mesh, const double* x, double* y);

/* Solve K x = f by preconditioned CG in the fused arrangement of Algorithm
 * pcg_fusion, FP64 throughout, vectors and scalars on the device.  f and x:
 * device [nnodes]; x holds the initial guess on entry and the solution on exit
 * (K is singular on the periodic mesh: f must have zero sum, and the solution
 * keeps the mean of the guess).  Preconditioner P^-1 = chi(A) diag(K)^-1 with
 * A = diag(K)^-1 K and chi the degree cheb_degree polynomial of Chebyshev
 * semi-iteration on the interval [a, b] of A's spectrum (0 < a < b; b <= 0:
 * b = the Gershgorin bound of A's spectrum and a = b / 20; degree 0: plain
 * Jacobi).  Stops when ||r||_2 < tol or after maxit iterations; writes
 * the iteration count and the final ||r||_2 to the host.  Synchronises once
 * per iteration for the convergence test. */
int rcf_poisson_pcg(rcf_ctx* ctx, const rcf_mesh* mesh, const double* f, double* x, int cheb_degree,
                    double a, double b, double tol, int maxit, int* iterations, double* residual);

/* ---- derivatives (no counterpart in the paper) ------------------------- */

/* Accumulate (+=) the derivatives of weight * Re tr(W^H H U) with respect to
 * V (dV, device [ncells][nloc]), B (dB, device [3][ncells][nloc]) and the
 * couplings h (dh, host [natoms][2]; may be NULL).  W, U: c128, nvec columns. */
int rcf_grad_bilinear(rcf_ctx* ctx, const rcf_op* op, const double* W, int64_t ldw,
                      const double* U, int64_t ldu, int nvec, double weight,
                      double* dV, double* dB, double* dh);

/* Cotangent of the Rayleigh-Ritz values (derivative of the eigenvalues of the
 * projected pencil; the paper has no counterpart).  Given Y (c128, nvec columns)
 * and its Rayleigh-Ritz pairs (theta: host [nvec], X: c128, X = Y Q with X
 * M-orthonormal, as returned by rcf_rayleigh_ritz for the Y it started from),
 * and thetabar = dL/dtheta (host [nvec]), writes
 *   Ybar = dL/dY = sum_j 2 thetabar_j (H - theta_j M) x_j q_j^H
 * (c128, must not overlap Y or X), with Q = (Y^H M Y)^{-1} Y^H M X (FP64; the
 * Gram matrix must be positive definite, else RCF_ENOTSPD), and, when dV and dB
 * are given (device, layouts as in rcf_potential_set; dh host [natoms][2] or
 * NULL), accumulates (+=) the direct term sum_j thetabar_j x_j^H (dH) x_j.
 * Synchronises. */
int rcf_ritz_cotangent(rcf_ctx* ctx, const rcf_op* op, const double* Y, int64_t ldy,
                       const double* X, int64_t ldx, int nvec, const double* theta,
                       const double* thetabar, double* Ybar, int64_t ldb, double* dV,
                       double* dB, double* dh);

/* Reverse-mode derivative of the R-ChFSI filter (X, Lambda and the bounds held
 * constant): given Ybar = dL/dY (c128), accumulate (+=) dL/dV, dL/dB (device,
 * per quadrature point, layouts as in rcf_potential_set) and dL/dh (host
 * [natoms][2], may be NULL) of L = Re tr(Ybar^H Y).  The forward recurrence is
 * recomputed from checkpoints stored every `ckpt_every` steps.  mode must be
 * RCF_RCHFSI; prec = RCF_FP64 or RCF_FP32 (recurrences and products in that
 * precision, gradients accumulated in FP64).  Processes all nvec columns as
 * one block. */
int rcf_adjoint_filter(rcf_ctx* ctx, const rcf_op* op, const double* X, int64_t ldx, int nvec,
                       const double* ritz, int degree, const double bounds[3], int mode, int prec,
                       const double* Ybar, int64_t ldyb, int ckpt_every,
                       double* dV, double* dB, double* dh);

/* ---- block floating-point codec (Section III-C-3) ------------------------ */

/* Four consecutive FP32 values form a block of 4 * nbits bits (nbits = 16, 12
 * or 10: 8, 6 or 5 bytes).  Its low 8 bits hold the shared biased exponent
 * e = e_max + 127, with 2^(e_max-1) <= max |x_i| < 2^e_max (e = 0: all four
 * values zero; a block whose largest magnitude is subnormal takes e_max = -126);
 * bits [8 + i v, 8 + (i+1) v) hold value i's coefficient
 * q_i = round_half_even(x_i 2^(v-1-e_max)), v = nbits - 2, two's complement,
 * clamped to at most 2^(v-1) - 1 (and, at e_max = 128, to at least
 * -(2^(v-1) - 1)).  Decoding gives q_i 2^(e_max-v+1), exactly.  Block b is the
 * little-endian word at byte offset b * (4 * nbits / 8) of the stream.
 *
 * rcf_bfp_stream_bytes: bytes of the stream for n values (ceil(n/4) blocks; a
 * last partial block is completed with zeros); -1 for an invalid nbits or n < 0.
 * rcf_bfp_encode: x (device, float[n], 4-byte aligned; finite values, the code
 * of a block holding Inf or NaN is unspecified) -> stream (device,
 * rcf_bfp_stream_bytes(n, nbits) bytes, 8-byte aligned at nbits = 16, 2-byte
 * at 12).  rcf_bfp_decode: stream -> y (device, float[n], 4-byte aligned).
 * Values and stream must not overlap.  Both enqueue one kernel on the
 * context's stream and return without synchronising; results are valid after
 * rcf_sync.  Errors: RCF_EINVAL for a bad nbits, n < 0, NULL or misaligned
 * pointers, overlap; RCF_ECUDA for a failed launch.  n = 0 does nothing. */
int64_t rcf_bfp_stream_bytes(int64_t n, int nbits);
int rcf_bfp_encode(rcf_ctx* ctx, const float* x, int64_t n, int nbits, void* stream);
int rcf_bfp_decode(rcf_ctx* ctx, const void* stream, int64_t n, int nbits, float* y);

#ifdef __cplusplus
}
#endif
#endif /* RCHFSI_H */

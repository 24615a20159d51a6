/*
 * rverom.h -- C ABI of the GB300 (sm_103a) hyper-reduced FE^2 online path.
 *
 * Method: Lange, Huetter, Kiefer, "A Monolithic Hyper ROM FE^2 Method with
 * Clustered Training at Finite Deformations", arXiv 2306.02687.
 *
 * Conventions shared by every entry point
 *   d      spatial dimension, 2 (plane strain) or 3
 *   g      d*d components of a second-order tensor, row-major: c = i*d + J
 *   ns     3 (2D) or 6 (3D) independent components of a symmetric tensor,
 *          order 2D (11,22,12), 3D (11,22,33,12,13,23), tensor (not
 *          engineering) components
 *   n~     ROM modes of an RVE type, m~ its ECM (hyper-integration) points
 *   nmax   largest n~ over the types of a handle; per-point state arrays are
 *          padded to nmax
 * Pointers named "device" must be CUDA device pointers on the current device;
 * "host" pointers are ordinary host memory.  The library never takes
 * ownership of caller memory.  All device work is enqueued on `stream`
 * (a cudaStream_t passed as void*, NULL = legacy default stream) and is
 * asynchronous with respect to the host unless stated otherwise.
 *
 * Return values: RVEROM_OK (0) or a negative RVEROM_ERR_* code.  Argument
 * errors are detected on the host before anything is enqueued.  Numerical
 * failures of single macro points are not API errors: they are reported per
 * point in `status` (RVEROM_STATUS_*), never by trapping the GPU.
 */
#ifndef RVEROM_H
#define RVEROM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RVEROM_OK 0
#define RVEROM_ERR_ARG (-1)         /* bad size, null pointer, unsupported shape */
#define RVEROM_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define RVEROM_ERR_UNSUPPORTED (-3) /* n~ or d outside the compiled kernels */
#define RVEROM_ERR_SCRATCH_LIMIT (-4) /* batch larger than the static scratch of rve_rom_adjoint_static */

#define RVEROM_STATUS_OK 0
#define RVEROM_STATUS_DETF_NONPOS 1 /* det F <= 0 at some ECM point */
#define RVEROM_STATUS_NONSPD_K 2    /* reduced stiffness not positive definite */
#define RVEROM_STATUS_NONFINITE 3   /* NaN/Inf in the input or the reduced system */
#define RVEROM_STATUS_TIMEOUT 5     /* a bounded internal wait of a tensor-core kernel ran out; the
                                       point's outputs are not valid (4 is the host drivers' NOT_CONVERGED) */

#define RVEROM_FP64 0  /* every step in native float64 */
#define RVEROM_MIXED 1 /* FP64-accurate F_i, P_i, r, Pbar; float32-level tangent contraction
                          (SIMT float32, or three-pass TF32 on the tensor cores) */

#define RVEROM_MAX_TYPES 8

typedef struct rverom_s *rverom_t;
typedef struct rverom_mesh_s *rverom_mesh_t;

/* One RVE type of the hyper-ROM (all arrays host, copied by rve_rom_create).
 *   B      [n_ecm][g][n_modes] gradient of the POD modes at the ECM points,
 *          B_i = grad Phi (x_i): F_i = U + B_i q  (ROM ansatz, Sec. 3.2.1,
 *          Eq. ROM_assumption; element-mode projection of Sec. 4)
 *   w      [n_ecm] ECM weights in the reference volume (Sec. 3.3, Box 1),
 *          positive, summing to V0
 *   phase  [n_ecm] material phase of each ECM point, 0 or 1
 *   moduli [2][2] (mu, kappa) of phase 0 and phase 1 of the compressible
 *          Neo-Hooke law P = mu (F - F^-T) + (kappa - 2 mu/3) ln J F^-T      */
typedef struct {
    int32_t n_modes;
    int32_t n_ecm;
    const double *B;
    const double *w;
    const int32_t *phase;
    double moduli[2][2];
} rverom_type_desc;

/* Create a handle holding device copies of the ROM tables of n_types RVE
 * types (1..RVEROM_MAX_TYPES) of dimension dim, reference volume V0.
 * Supported n_modes: 2D 1..64, 3D 1..47.  Synchronous; allocates device
 * memory (tables and a small reduction workspace).  On error *out is NULL. */
int rve_rom_create(int32_t dim, int32_t n_types, const rverom_type_desc *types, double V0,
                   rverom_t *out);

/* Free the handle and its device memory (synchronizes the device). */
int rve_rom_destroy(rverom_t h);

/* Replace the moduli of one type (host [2][2] = (mu, kappa) per phase).
 * Takes effect for work enqueued after the call returns. */
int rve_rom_set_moduli(rverom_t h, int32_t type, const double *moduli);

/* Largest n~ of the handle (the padding of the per-point state arrays). */
int rve_rom_nmax(rverom_t h, int32_t *nmax);

/* Batched hyper-reduced RVE evaluation at n_points macro integration points:
 * one monolithic Newton evaluation per point (Sec. 3.2.2-3.2.3, Sec. 4):
 *   a1  Fbar = R U (polar split, Eq. polar_decomp); micro update
 *       q <- q - s - S (U - U_prev)                 (Sec. 3.2.3, Delta u~)
 *   a2  F_i = U + B_i q at every ECM point          (Eq. ROM_assumption)
 *   a3  P_i, A_i = dP/dF from the micro law
 *   a4  r = sum w_i B_i^T P_i, Pbar_U = sum w_i P_i / V0  (Eq. ROMintforce, Eq. 2)
 *   a5  K = sum w_i B_i^T A_i B_i, K_qF = sum w_i B_i^T A_i, K_FF = sum w_i A_i
 *                                                     (Eq. ROMstiffness)
 *   a6  s = K^-1 r, S = K^-1 K_qF E, Pbar_alg = Pbar_U - K_qF^T s / V0,
 *       C_U = (K_FF - K_qF^T K^-1 K_qF) / V0          (Eq. Biot_Tangent, condensation)
 *   a7  Pbar = R Pbar_alg, dPdF = dPbar/dFbar through the polar derivative
 * Arguments (all device, row-major, contiguous):
 *   type    [n] int32 RVE type per point, or NULL when every point is type 0
 *   Fbar    [n][g]            macro deformation gradient (in)
 *   q, s    [n][nmax]         reduced amplitudes and K^-1 r (in/out state)
 *   S       [n][nmax][ns]     K^-1 dr/dU (in/out state)
 *   Uprev   [n][ns]           stretch of the previous evaluation (in/out)
 *   Pbar    [n][g]            homogenized 1st Piola-Kirchhoff stress (out)
 *   dPdF    [n][g][g]         consistent tangent dPbar_c/dFbar_e at [c][e] (out)
 *   rnorm   [n]               max_j |r_j| of the evaluated state (out)
 *   status  [n]               RVEROM_STATUS_* (out)
 * A fresh state is q = s = S = 0 and Uprev = the Voigt stretch of Fbar (or
 * of I).  Points whose status is not OK keep their input state; their Pbar
 * and dPdF are NaN.  precision: RVEROM_FP64 or RVEROM_MIXED.  n_points may be
 * 0 (no work).  Points with a type >= n_types get RVEROM_STATUS_NONFINITE. */
int rve_rom_eval_batch(rverom_t h, int64_t n_points, const int32_t *type, const double *Fbar,
                       double *q, double *s, double *S, double *Uprev, double *Pbar, double *dPdF,
                       double *rnorm, int32_t *status, int32_t precision, void *stream);

/* Autotuner of the evaluation kernels: for every RVE type of the handle,
 * time each compiled tile configuration (SIMT or tcgen05 tensor-core
 * kernels; points per CTA, ECM points per chunk, warp roles) of the given
 * precision on a synthetic batch of n_sample points (seeded small
 * stretches, fresh state; device memory for it is allocated and freed
 * here), keep the fastest for
 * rve_rom_eval_batch, and optionally report the best-of-2 times in
 * ms_out [n_types][RVEROM_MAX_CANDIDATES] (host; -1 for unused slots).
 * A candidate for which any point of the sample ends with a status other
 * than RVEROM_STATUS_OK is never kept (its ms_out entry is -2); if no
 * candidate of a type is valid, configuration 0 stays in use.
 * Synchronous.  Without tuning, configuration 0 of each list is used. */
#define RVEROM_MAX_CANDIDATES 4
int rve_rom_autotune(rverom_t h, int32_t precision, int64_t n_sample, float *ms_out, void *stream);

/* Pin the tile configuration `candidate` (0 .. n-1) of one type and
 * precision for rve_rom_eval_batch; candidate < 0 only queries.  The number
 * of compiled candidates is returned in *n_candidates (may be NULL). */
int rve_rom_select_kernel(rverom_t h, int32_t type, int32_t precision, int32_t candidate,
                          int32_t *n_candidates);

/* Name and kernel launches of a forward candidate of one type and precision
 * (candidate < 0: the one rve_rom_eval_batch currently uses, i.e. the
 * autotuner's or rve_rom_select_kernel's pick, else 0).  `name` receives a
 * NUL-terminated, possibly truncated description in a caller buffer of `len`
 * bytes (may be NULL); `launches` (may be NULL) the number of kernels the
 * candidate launches for this type per rve_rom_eval_batch call.  Host only;
 * RVEROM_ERR_ARG for a bad handle, type, precision or candidate.  (A query
 * of this library's dispatch: the paper has no counterpart.) */
int rve_rom_kernel_info(rverom_t h, int32_t type, int32_t precision, int32_t candidate, char *name, int32_t len,
                        int32_t *launches);

/* Implicit-function adjoint at converged states (r(q*) = 0): for cotangents
 * gPbar on Pbar,
 *   gFbar = dPdF^T gPbar      (the condensed consistent tangent)
 *   gTheta[t][ph][k] += sum over points of type t of d<gPbar, Pbar>/d theta,
 *       theta = (mu, kappa) of phase ph, computed as
 *       (1/V0) sum_i w_i < R^T gPbar - B_i z , dP_i/dtheta >,
 *       z = K^-1 K_qF (R^T gPbar)
 * Device arrays: type [n] or NULL, Fbar [n][g], q [n][nmax], gPbar [n][g],
 * gFbar [n][g] (out), gTheta [n_types][2][2] (accumulated, deterministic
 * order), status [n] (out, as in rve_rom_eval_batch).  Uses the handle's
 * reduction workspace, so calls on one handle must not overlap. */
int rve_rom_adjoint(rverom_t h, int64_t n_points, const int32_t *type, const double *Fbar,
                    const double *q, const double *gPbar, double *gFbar, double *gTheta,
                    int32_t *status, void *stream);

/* rve_rom_adjoint_static: the same adjoint as rve_rom_adjoint (same kernel,
 * same arguments, same results) for callers that must not allocate device
 * memory during the call.  The paper has no counterpart; this is an
 * interface variant of this library.  rve_rom_adjoint allocates its
 * reduction workspace and the point lists of mixed-type batches with
 * cudaMalloc on first use or when a batch grows.  Callers that cannot allow
 * that -- a macro FE code calling the adjoint from per-increment material
 * callbacks, where an allocation may synchronize the device and stall the
 * host element loop, or a process whose device memory is reserved by
 * another allocator -- use this entry point, which allocates nothing: its
 * scratch is one static device array of RVEROM_STATIC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.
 * Limits: mixed-type batches (type != NULL) of at most
 * RVEROM_STATIC_MAX_TYPED_POINTS points; devices with at most
 * RVEROM_STATIC_MAX_CTAS / 16 SMs.  Larger requests return
 * RVEROM_ERR_SCRATCH_LIMIT before any work is enqueued.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  All calls share the array and its last contents; the call
 * clears what must start at zero, but calls whose GPU work overlaps (other
 * streams or threads on the same device) race on it. */
#define RVEROM_STATIC_MAX_CTAS 4096
#define RVEROM_STATIC_MAX_TYPED_POINTS (1 << 20)
#define RVEROM_STATIC_SCRATCH_BYTES (RVEROM_STATIC_MAX_CTAS * 4 * 8 + 256 + RVEROM_STATIC_MAX_TYPED_POINTS * 4)
int rve_rom_adjoint_static(rverom_t h, int64_t n_points, const int32_t *type, const double *Fbar,
                           const double *q, const double *gPbar, double *gFbar, double *gTheta,
                           int32_t *status, void *stream);

/* Macro mesh of isoparametric Q4 (dim 2) or hex8 (dim 3) elements with 2^d
 * Gauss points each; integration point alpha = e * 2^d + gp (gp in
 * lexicographic order of the reference coordinates, last coordinate slowest
 * ... first fastest).  X [n_nodes][d] and conn [n_elem][2^d] are host arrays.
 * Builds, on the host, the shape-function gradients and weights of every
 * point and the CSR pattern of the global stiffness (one row per DOF
 * node*d + i), then copies them to the device.  Synchronous. */
int macro_mesh_create(int32_t dim, int64_t n_nodes, int64_t n_elem, const double *X,
                      const int64_t *conn, rverom_mesh_t *out);
int macro_mesh_destroy(rverom_mesh_t m);

/* Sizes of a mesh: integration points, DOFs, CSR non-zeros. */
int macro_mesh_sizes(rverom_mesh_t m, int64_t *n_ip, int64_t *n_dof, int64_t *nnz);

/* Copy the CSR pattern to host arrays row_ptr [n_dof+1], col [nnz]. */
int macro_mesh_csr(rverom_mesh_t m, int64_t *row_ptr, int32_t *col);

/* Fbar at every integration point from nodal displacements (device
 * u [n_nodes][d] -> Fbar [n_ip][g]): Fbar = I + sum_a u_a (x) grad N_a. */
int macro_gradient(rverom_mesh_t m, const double *u, double *Fbar, void *stream);

/* Macro element assembly (Eq. 6 with Pbar; its linearization with dPdF):
 *   R[a*d+i]  = sum_alpha wJ0 sum_J Pbar_iJ dN_a,J
 *   K[(a,i),(b,k)] = sum_alpha wJ0 sum_JL dN_a,J dPdF[iJ][kL] dN_b,L
 * Device: Pbar [n_ip][g], dPdF [n_ip][g][g] (NULL skips K), R [n_dof] and
 * Kvals [nnz] (CSR order of macro_mesh_csr) are overwritten. */
int macro_assemble(rverom_mesh_t m, const double *Pbar, const double *dPdF, double *R,
                   double *Kvals, void *stream);

/* The macro steps of one shard of a data-parallel monolithic iteration
 * (Sec. 2: the element sums of Eq. 6 split over disjoint element ranges,
 * the RVEs of a range evaluated where the range lives).
 * macro_gradient_range: Fbar [(e_end - e_begin) * n_gp_per_elem][g] at the
 * integration points of elements e_begin .. e_end - 1 (points numbered as
 * in macro_gradient, the range's first point at Fbar[0]); u is the whole
 * nodal field [n_nodes][d].
 * macro_assemble_range: ADDS the range's element contributions to R
 * [n_dof] and (when not NULL) Kvals [nnz] of the whole mesh's pattern;
 * Pbar and dPdF hold the range's points only, in the order of
 * macro_gradient_range.  Nothing is zeroed: the caller zeroes R and Kvals
 * once, every range adds, and summing the shards' R and Kvals (an
 * all-reduce across ranks) gives macro_assemble's result up to the order
 * of the floating-point sums.  An empty range (e_end == e_begin) is a no-op.
 * Errors: RVEROM_ERR_ARG for a range outside 0 .. n_elem or missing arrays. */
int macro_gradient_range(rverom_mesh_t m, int64_t e_begin, int64_t e_end, const double *u,
                         double *Fbar, void *stream);
int macro_assemble_range(rverom_mesh_t m, int64_t e_begin, int64_t e_end, const double *Pbar,
                         const double *dPdF, double *R, double *Kvals, void *stream);

/* Convergence scalars of a monolithic iteration (device):
 *   out[0] = max |R| over DOFs with free_mask != 0
 *   out[1] = max |R| over DOFs with free_mask == 0 (reactions)
 *   out[2] = max over points of rnorm
 * free_mask [n_dof] uint8, rnorm [n_points]. */
int macro_residual_norms(rverom_mesh_t m, const double *R, const uint8_t *free_mask,
                         int64_t n_points, const double *rnorm, double *out, void *stream);

/* Global macro solve of a monolithic Newton iteration (Sec. 2: the Newton
 * correction of the discrete macro equilibrium Eq. 6, linearized with the
 * consistent tangent that macro_assemble assembles; the paper uses a direct
 * solver, here conjugate gradients):
 *   K du = -R   on the DOFs with free_mask != 0,   du = 0 on the others,
 *   u += du     (when u is not NULL).
 * Preconditioned by the inverse d x d diagonal block of every node (rows
 * and columns of prescribed DOFs replaced by the identity), in the
 * single-reduction form of Chronopoulos and Gear; stops when
 * ||r||_2 <= tol ||R_free||_2 or after max_iter iterations.  Runs as one
 * cooperative kernel (one block per SM, in the mesh's workspace:
 * no allocation, so the call can sit in a CUDA graph with the rest of the
 * Newton iteration).  Calls on one mesh must not overlap.
 * Device arrays: Kvals [nnz] (CSR of macro_mesh_csr), R [n_dof],
 * free_mask [n_dof] uint8, u [n_dof] (in/out, may be NULL), du [n_dof] (out),
 * info [3] (out): iterations, final relative residual, status (0 converged,
 * 1 max_iter reached, 2 K not positive definite on a search direction,
 * 5 an internal grid barrier ran out of time). */
int macro_solve(rverom_mesh_t m, const double *Kvals, const double *R, const uint8_t *free_mask, double tol,
                int32_t max_iter, double *u, double *du, double *info, void *stream);

/* Largest m~ over the types of a handle (the ECM-point stride of the
 * history arrays of rve_rom_eval_batch_j2). */
int rve_rom_mmax(rverom_t h, int32_t *mmax);

/* rve_rom_eval_batch with a history-dependent micro law (planar RVEs,
 * n~ <= 32, float64): small-strain J2 plasticity with linear isotropic
 * hardening at every ECM point, the matrix law of Example 1 (Sec. 5.1),
 * under plane strain (radial return; the in-plane stress in the place of P,
 * the in-plane block of the consistent tangent in the place of dP/dF).
 * Phases use the handle's (mu, kappa) and, from `plastic` (host
 * [n_types][2][2]), the yield stress sy0 and hardening modulus h of each
 * phase; sy0 <= 0 or infinite makes the phase elastic.
 * hist_in  [n][mmax][7] (device) records (plastic strain 11, 22, 33, 12, 13,
 *          23 and equivalent plastic strain) of the last converged load
 *          step; zero for a virgin material
 * hist_out [n][mmax][7] (device, out; distinct from hist_in) the records
 *          after this evaluation's return mappings; the caller copies them
 *          to hist_in once the load step has converged
 * Other arguments, outputs and status codes as rve_rom_eval_batch; failed
 * points keep their state and their history. */
int rve_rom_eval_batch_j2(rverom_t h, int64_t n_points, const int32_t *type, const double *Fbar, double *q,
                          double *s, double *S, double *Uprev, const double *hist_in, double *hist_out,
                          const double *plastic, double *Pbar, double *dPdF, double *rnorm, int32_t *status,
                          void *stream);

/* ---- offline (training) stage on the GPU, planar RVEs -------------------
 * RVE: the unit cell (V0 = 1) meshed by n x n bilinear quadrilaterals with
 * 2 x 2 Gauss points; element e = ix + n iy, node v = ix + n iy (periodic:
 * indices mod n), micro integration point p = 4 e + gauss point (reference
 * coordinates (xi_0, xi_1) in {-,+}^2, the second fastest); the periodic
 * fluctuation w has DOFs v d + i, node 0 fixed, so the reduced vector of
 * n_dof = 2 n^2 - 2 entries drops the first two; F = Fbar + grad w;
 * compressible Neo-Hooke law per element phase (phase [n * n], moduli [2][2]
 * (mu, kappa) host).  Every call below is asynchronous on `stream` unless it
 * says otherwise. */

/* Full-order snapshots (Sec. 3.2.1, Eq. snapshots_displacement): for each
 * of n_paths training paths (one CTA per path), the micro equilibrium at
 * the macro stretches paths [n_paths][n_steps][4] (device, row-major 2 x 2)
 * in turn, each from the previous solution, by Newton's method
 * (max|f| <= tol) with matrix-free block-Jacobi preconditioned conjugate
 * gradients (relative tolerance cg_tol) for the corrections; the converged
 * fluctuations are the rows X [n_paths * n_steps][n_dof] (device).
 * linear = 1 instead solves the linearized RVE at Fbar = I for the three
 * unit symmetric macro strains (n_paths = 3, n_steps ignored, paths may be
 * NULL): w_v = -K_ww^-1 K_wF E_v, the elastic responses of Eq.
 * SVD_displacement.  info [n_paths][4] (device): Newton iterations, CG
 * iterations, final max|f|, status (0 ok, 1 det F <= 0, 2 CG breakdown,
 * 3 Newton not converged).  Allocates its workspace with cudaMallocAsync. */
int rve_snapshots(int32_t n, const int32_t *phase, const double *moduli, int32_t n_paths, int32_t n_steps,
                  const double *paths, int32_t linear, double tol, double cg_tol, int32_t max_newton,
                  int32_t max_cg, double *X, double *info, void *stream);

/* POD with the elastic/inelastic split (Sec. 3.2.1, Eqs. SVD_displacement
 * and snapshots_displacement): Phi rows 0 .. n_el-1 are the orthonormalized
 * rows of W_el [n_el][n_dof] (the linearized responses; n_el <= 8), rows
 * n_el .. n_modes-1 the leading left singular vectors of the snapshots
 * X [n_snap][n_dof] with their W_el part removed, computed from the
 * eigen-decomposition of their Gram matrix (cyclic Jacobi); eig [n_snap]
 * the eigenvalues (squared singular values) in descending order; info [2]
 * (device) Jacobi sweeps and final relative off-diagonal norm.  Device
 * arrays; allocates scratch with cudaMallocAsync. */
int pod_modes(int64_t n_dof, int32_t n_snap, const double *X, int32_t n_el, const double *W_el, int32_t n_modes,
              double *Phi, double *eig, double *info, void *stream);

/* Gradients of the modes Phi [n_modes][n_dof] at every micro integration
 * point of the n x n RVE: B [n_ip][4][n_modes] (device), the gradient table
 * of the fully integrated ROM (Gauss weights (1 / 2n)^2 each, V0 = 1). */
int rve_mode_gradients(int32_t n, int32_t n_modes, const double *Phi, double *B, void *stream);

/* The ECM training matrix of Sec. 3.3 (Eq. SVDlambda's x_f): for every
 * training state s (stretch U [n_snap][4], converged amplitudes
 * q [n_snap][n_modes] of the fully integrated ROM with table B) and micro
 * point p the integrand f = [B_p^T P_p; P_p] (n_modes + 4 rows per state),
 * minus its integral over the cell (V0 = 1) per row; then the mode rows and
 * the stress rows each scaled to unit Frobenius norm.  xf
 * [n_snap * (n_modes + 4)][n_ip] (device).  Synchronous; RVEROM_ERR_ARG if
 * a state folds a micro point (det F <= 0). */
int ecm_training_matrix(int32_t n, const int32_t *phase, const double *moduli, int32_t n_modes, const double *B,
                        int32_t n_snap, const double *U, const double *q, double *xf, void *stream);

/* Empirical cubature (Sec. 3.3, Eq. SVDlambda and Box 1): the leading
 * m_target - 1 right singular vectors lambda of xf [n_rows][m] (device) by
 * randomized subspace iteration from the Gaussian test matrix Omega
 * [n_rows][k] (device, m_target - 1 <= k <= n_rows; power_its power
 * iterations; re-orthonormalization by SVQB, the Gram matrix's
 * eigendecomposition, which drops directions of relative eigenvalue below
 * 1e-15, so k may exceed the numerical rank of xf: k = n_rows with
 * power_its = 0 spans the whole row space and gives the exact leading
 * singular subspace), then the greedy selection of Box 1 on
 * J = [lambda 1]^T, b = [0 V0]^T: pick the available column most aligned
 * with r = b - J_z w (ties to the lowest index), least-squares weights,
 * non-negative least squares (Lawson-Hanson) when a weight is negative,
 * zero-weight points dropped for good, until m_target points or no
 * candidate is left.  z [m_target] (device int32) and w [m_target] (device)
 * receive the points and weights, *n_sel (host) their count, info [4]
 * (host): greedy iterations, final |J_z w - b|, least-squares solves, 0.
 * m_target <= 1000.  Synchronous; allocates scratch with cudaMallocAsync. */
int ecm_select(int64_t m, int32_t n_rows, const double *xf, double V0, int32_t m_target, const double *Omega,
               int32_t k, int32_t power_its, int32_t *z, double *w, int32_t *n_sel, double *info, void *stream);

/* Biot and Cauchy outputs for updated-Lagrangian macro codes (Sec. 3.2.2,
 * Eqs. workconjugacy and biotstress; Appendix A), from the homogenized
 * first Piola-Kirchhoff stress and its tangent at n points (Fbar = R U):
 *   biot    [n][ns]      T = sym(R^T Pbar), work conjugate to U
 *   cbiot   [n][ns][ns]  dT_v / dU_w for symmetric stretch variations at
 *                        fixed R (dFbar = R dU)
 *   sigma   [n][ns]      Cauchy stress from T = (J/2)(R^T sigma F^-T +
 *                        F^-1 sigma R), solved for the symmetric sigma
 *   csigma  [n][ns][ns]  dsigma_v / dD_w ~ (dsigma/dT) C^B sym(R^T D F), the
 *                        constant-rotation approximation of Appendix A
 * Symmetric tensors by their ns tensor components (the project's order);
 * derivatives with respect to a shear component move both of its entries.
 * Device arrays; Fbar [n][g], Pbar [n][g], dPdF [n][g][g] (as written by
 * rve_rom_eval_batch); any of the four outputs may be NULL.  Points with
 * det Fbar <= 0 or a singular map get NaN outputs. */
int rve_rom_biot_cauchy(int32_t dim, int64_t n, const double *Fbar, const double *Pbar, const double *dPdF,
                        double *biot, double *cbiot, double *sigma, double *csigma, void *stream);

/* Clustered training (Sec. 3.4, Box 2), step 1: the linear-elastic
 * surrogate with the initial RVE stiffness C0 (device [g][g], e.g. the
 * condensed tangent dPbar/dFbar of the hyper-ROM at Fbar = I):
 * Pbar = C0 (Fbar - I) and dPdF = C0 (may be NULL) at n points. */
int surrogate_linear_eval(int32_t dim, int64_t n, const double *C0, const double *Fbar, double *Pbar,
                          double *dPdF, void *stream);

/* Clustered training (Box 2), step 3: k-means (Lloyd) of n macro paths
 * X [n][dim] (device; e.g. the displacement gradients of every macro point
 * over the load steps of a surrogate run, concatenated).  centers [k][dim]
 * (device) holds the initial centres on entry and the final ones on return;
 * labels [n] (device, out) the nearest centre of every path (squared
 * Euclidean distance summed over the coordinates in order; ties to the
 * lowest index).  Iterates assignment and update (mean of the assigned
 * paths; an empty cluster keeps its centre) until no label changes or
 * max_iter updates.  info [2] (host, out): updates done, final sum of
 * squared distances.  Synchronous; allocates a few bytes of device
 * scratch per call (an offline step). */
int paths_kmeans(int64_t n, int32_t dim, const double *X, int32_t k, double *centers, int32_t *labels,
                 int32_t max_iter, double *info, void *stream);

/* ---- diagnostics (no counterpart in the paper) -------------------------- */

/* The double-float natural logarithm that the mixed form's micro law uses
 * for ln J (range reduction to [1/sqrt2, sqrt2) and an atanh series, within
 * 3e-14 relative), evaluated at n device points x [n] (each rounded to a
 * double-float first) into device out [n] (float64).  For testing that
 * routine against float64 log; x must be finite and positive. */
int rverom_df_log(int64_t n, const double *x, double *out, void *stream);

/* Measured throughput, in TFLOP/s, of one execution unit of the current
 * device, the denominators of the roofline fractions of the hot path:
 *   unit 0  FP32 FMA pipe (independent FMA chains, 2 FLOP per FMA)
 *   unit 1  FP64 FMA pipe (the same with doubles)
 *   unit 2  tcgen05.mma kind::tf32, M = 128, N = 256, K = 8
 *   unit 3  tcgen05.mma kind::f16 with BF16 operands, M = 128, N = 256, K = 16
 * One CTA per SM (MMAs) or 8 CTAs of 256 threads per SM (FMAs); the best
 * of three timed runs (CUDA events) after one warm-up.  Synchronous on
 * `stream`; allocates and frees 4 KB of device memory.  RVEROM_ERR_CUDA if
 * a launch fails or an MMA completion wait runs out. */
int rverom_peak_probe(int32_t unit, double *tflops, void *stream);

#ifdef __cplusplus
}
#endif
#endif

/*
 * igafd — GB300-native PCG for single-patch isogeometric Poisson problems,
 * preconditioned by the fast-diagonalization (FD) solve of the Kronecker-sum
 * matrix P (Sangalli & Tani, "Isogeometric preconditioners based on fast
 * solvers for the Sylvester equation").
 *
 * C ABI: plain pointers and sizes only. All "_dev" pointers are CUDA device
 * pointers on the device that was current at igafd_setup_patch; "stream" is
 * a cudaStream_t passed as void* (NULL = legacy default stream).
 *
 * Conventions
 *  - Dof vectors are FP64, length N = n_1 * ... * n_d, with the scalar index
 *    of Eq. (Vh): i = i_1 + n_1 (i_2 + n_2 i_3) (direction 1 fastest), where
 *    n_k = m_k - 2 counts the B-splines of direction k that vanish on the
 *    boundary (homogeneous Dirichlet conditions). Device vectors must be
 *    8-byte aligned; 256-byte alignment gives the best bandwidth.
 *  - The patch owns every device buffer it uses. Only the set-up calls
 *    (igafd_setup_patch, igafd_batch_create, ...) allocate; apply/solve entry
 *    points never allocate (igafd_batch_pcg_solve, which creates and destroys
 *    a batch, is the documented exception).
 *  - Errors are returned as igafd_status, never trapped on the device. After a
 *    device-side limit is hit, the status says so and the context stays usable.
 *  - Calls on one patch must not overlap in time on different streams (the
 *    patch's workspace is shared by its entry points).
 */
#ifndef IGAFD_H
#define IGAFD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct igafd_patch igafd_patch;

typedef enum {
  IGAFD_OK = 0,
  IGAFD_ERR_ARG = -1,           /* invalid argument (sizes, knots, NULLs) */
  IGAFD_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  IGAFD_ERR_NOT_SPD = -3,       /* Cholesky of a 1D mass matrix failed */
  IGAFD_ERR_EIG = -4,           /* Jacobi eigen-solve hit its sweep limit */
  IGAFD_ERR_FOLDED = -5,        /* det J <= 0 at a quadrature point */
  IGAFD_ERR_BREAKDOWN = -6,     /* PCG: (p, Ap) <= 0 or non-finite */
  IGAFD_ERR_NOT_CONVERGED = -7, /* PCG: iteration cap reached */
  IGAFD_ERR_TIMEOUT = -8,       /* a bounded device wait ran out */
  IGAFD_ERR_OOM = -9            /* device allocation failed in setup */
} igafd_status;

/* Arithmetic of the preconditioner's mode-k contractions. The outer PCG
 * (inner products, residual recurrence, A stencil) is always FP64. */
typedef enum {
  IGAFD_FP64 = 0,   /* FP64 contractions and divide: FD is exactly P^{-1} */
  IGAFD_FP32 = 1,   /* FP32 SIMT contractions, FP32 divide */
  IGAFD_BF16 = 2,   /* tcgen05 kind::f16 with bf16 operands, FP32 accumulate */
  IGAFD_FP16 = 3,   /* tcgen05 kind::f16 with fp16 operands (power-of-two scaled
                       per 128-row tile and per U_k), FP32 accumulate */
  IGAFD_TF32 = 4,   /* tcgen05 kind::tf32, FP32 accumulate */
  IGAFD_ADI = 5     /* not FD: the three-variable ADI preconditioner P_J
                       set up by igafd_adi_setup (3D; see below) */
} igafd_dtype;

/* Single-patch problem (Section 2.1, Eqs. (A), (Q)):
 *   -div(kappa grad u) = f on Omega = F([0,1]^d), u = 0 on the boundary,
 * discretised by degree-p tensor B-splines on open knot vectors.
 * All pointers are host pointers, read only during igafd_setup_patch. */
typedef struct {
  int dim;                          /* 2 or 3 */
  int p;                            /* spline degree, 1 <= p <= 7 */
  const int *n_knots;               /* [dim] knot-vector lengths (m_k + p + 1) */
  const double *const *knots;       /* [dim] open knot vectors on [0,1], interior
                                       multiplicity <= p (Eq. (knot-vector)) */
  int geo_p;                        /* degree of the geometry map F, 1..7 */
  const int *geo_n_knots;           /* [dim] */
  const double *const *geo_knots;   /* [dim] knot vectors of F */
  const double *ctrl;               /* control net of F: [dim][g_d]..[g_1]
                                       (coordinate slowest, direction 1 fastest),
                                       g_k = geo_n_knots[k] - geo_p - 1 */
  double kappa;                     /* constant scalar coefficient K = kappa I */
  /* Optional variable coefficient: K(x) = kappa * c(zeta) I with c a
   * degree-kappa_p tensor spline on its own open knot vectors and control
   * values kappa_ctrl [c_d]..[c_1] (direction 1 fastest), all > 0 so that
   * c > 0 everywhere. kappa_ctrl == NULL: constant kappa. */
  int kappa_p;
  const int *kappa_n_knots;
  const double *const *kappa_knots;
  const double *kappa_ctrl;
  int flags;                        /* 0, IGAFD_SETUP_NO_STENCIL, IGAFD_SETUP_FULL_SPACE or
                                       IGAFD_SETUP_HALF_STENCIL */
} igafd_patch_desc;

/* igafd_patch_desc.flags: build everything but the stiffness stencil (no
 * (2p+1)^d x N array, no assembly). Such a patch answers the geometry and
 * preconditioner calls (igafd_patch_query, igafd_get_eigen,
 * igafd_apply_prec, igafd_patch_features, igafd_patch_sepfit,
 * igafd_set_scalings, igafd_quad_points, igafd_load_rhs, igafd_load_rhs_sine);
 * the calls that need A
 * (igafd_apply_A, igafd_pcg_solve, igafd_batch_pcg_solve, igafd_copy_stencil,
 * igafd_autotune, igafd_pcg_condition_estimate) return IGAFD_ERR_ARG. */
#define IGAFD_SETUP_NO_STENCIL 1

/* igafd_patch_desc.flags: keep every B-spline of every direction (the full
 * space, n_k = m_k: no homogeneous Dirichlet removal), for a patch that is
 * one piece of a multi-patch operator (igafd_mp_set_operator). Such a patch
 * has the stiffness stencil over its full index box and no preconditioner
 * (its full 1D stiffness matrices are singular): igafd_apply_prec,
 * igafd_pcg_solve, igafd_setup_prec, igafd_get_eigen, igafd_set_scalings, the
 * ADI calls and igafd_autotune return IGAFD_ERR_ARG; igafd_apply_A,
 * igafd_copy_stencil, igafd_quad_points and the load vectors work on the full
 * space. May be combined with nothing else. */
#define IGAFD_SETUP_FULL_SPACE 2

/* igafd_patch_desc.flags: store the stiffness stencil by its symmetry
 * (A_ij = A_ji, Eq. (A)): only the offsets delta >= 0 in the order of the
 * offset index (delta_d, ..., delta_1) are kept, ((2p+1)^d + 1) / 2 of the
 * (2p+1)^d, each a row array with zero halos; a coupling with delta < 0 of
 * row i is the stored coupling -delta of row i + off(delta). The bytes of A
 * are about halved; the FMAs per row are the same, so a product stays bound
 * by GB300's FP64 pipe and is not shorter (measured 9-15 % longer: the
 * mirrored runs are fetched shifted by one row when their start is odd).
 * It is the format for problems whose full stencil would not fit. Every
 * call that uses A works on
 * such a patch (igafd_copy_stencil expands it to the full layout); the
 * stencil pipeline runs with its default ring depth (the autotuner tunes
 * the rows per thread only). A product differs from the full stencil's at
 * the rounding level: the assembled couplings A_ij and A_ji are summed in
 * different orders, and the half stencil uses A_ij for both. May not be
 * combined with IGAFD_SETUP_NO_STENCIL or IGAFD_SETUP_FULL_SPACE. */
#define IGAFD_SETUP_HALF_STENCIL 4

typedef struct {
  int dim, p;
  int n[3];            /* dofs per direction (1 for unused directions) */
  long long N;         /* total dofs */
  int nel[3];          /* elements per direction */
  int n_offsets;       /* (2p+1)^dim stencil offsets */
  double min_detJ;     /* min det J over all quadrature points */
  double q_bound;      /* Prop. 1 estimate sup lambda_max(Q) / inf lambda_min(Q)
                          over the quadrature points */
  double setup_ms;     /* device time of the last igafd_setup_patch */
  double eig_ms;       /* of which the generalized eigendecompositions */
  long long stencil_bytes;
  int stencil_stages;  /* ring depth of the stencil pipeline in use (autotuned) */
  int stencil_rows;    /* rows per compute thread of the stencil in use (1, or 2 in 3D; autotuned) */
  int eig_refined[3];  /* per direction: 1 if the eigenpairs of the last setup of P came from the
                          FP32 start + FP64 refinement route, 0 if from FP64 Jacobi */
  double eig_check[3][2]; /* per direction, the refinement route's final check: max |U~^T U~ - I|
                             and max |offdiag U~^T K~ U~| / max |diag| (accepted if both <= 1e-12) */
  int fd_fused[3];     /* tensor-core FD in use for TF32, BF16, FP16 operands: 1 = fused (two mode
                          products per kernel; the compile-time-sized kernels where every
                          n_k = 128 in 3D), 0 = one kernel per mode product (autotuned) */
  int fd_tile[3][4];   /* tile shape per operand type (TF32, BF16, FP16; autotuned, see
                          igafd_set_fd_tile): rows per CTA of the per-mode kernel, its column
                          tiles (1 or 2), its K stages, columns per CTA of the fused pencil kernel */
  int stencil_half;    /* 1 if the stencil stores only the offsets from the centre up
                          (IGAFD_SETUP_HALF_STENCIL), 0 if all (2p+1)^d */
} igafd_patch_info;

typedef struct {
  double tol;          /* relative residual tolerance ||r|| <= tol ||b|| */
  int max_iter;        /* iteration cap (products with A inside the loop) */
  int true_every;      /* recompute r = b - A x every this many iterations
                          (0 = only to confirm convergence) */
  igafd_dtype prec_dtype;
  int flexible;        /* 1: beta = (r+, z+ - z)/(r, z); 0: Fletcher-Reeves */
  int x0_given;        /* 1: x_dev holds the initial guess; 0: x0 = 0 */
  int check_every;     /* host polls the device convergence flag every this
                          many iterations (>= 1); later iterations are skipped
                          on the device once converged, so x is unaffected */
  int timing;          /* 1: time the solve with CUDA events and the in-loop
                          A-stencil launches with device-clock stamps taken by
                          the stencil kernel itself (fills the *_ms fields of
                          igafd_pcg_info); polls at most every 32 iterations */
} igafd_pcg_opts;

typedef struct {
  int iterations;      /* products with A inside the loop */
  int status;          /* igafd_status of the solve */
  double relres;       /* final recurrence ||r||/||b|| */
  double true_relres;  /* final ||b - A x|| / ||b|| */
  int true_checks;     /* true-residual recomputations performed */
  double solve_ms;     /* device time of the whole solve (timing = 1) */
  double stencil_ms;   /* summed device time of the in-loop A products */
  double prec_ms;      /* summed device time of the in-loop FD applies, or -1
                          when the loop ran as a captured graph */
} igafd_pcg_info;

/* Build a patch: 1D pencils K_k, M_k by (p+1)-point Gauss quadrature
 * (Section 3, Eq. (prec)), their FP64 generalized eigendecompositions
 * K_k U_k = M_k U_k D_k, U_k^T M_k U_k = I (the eigendecompositions of
 * Algorithm 1, Section 4.1, Eq. (eigen3d)), and the stiffness matrix A of
 * Eq. (A) with Q = kappa |det J| J^{-1} J^{-T} as a (2p+1)^d-point FP64
 * stencil (Section 2.1). Allocates all device memory the patch will use.
 * Errors: ARG (bad sizes/knots), OOM, NOT_SPD, EIG, FOLDED, CUDA.
 * On error *out is NULL and nothing is leaked. */
igafd_status igafd_setup_patch(const igafd_patch_desc *desc, void *stream,
                               igafd_patch **out);

void igafd_destroy_patch(igafd_patch *patch);

igafd_status igafd_patch_query(const igafd_patch *patch, igafd_patch_info *info);

/* Copy the generalized eigenpairs of direction k (0-based) to host memory:
 * U_host[i * n_k + j] = (U_k)_{ij} (column j is the eigenvector of D_host[j]),
 * eigenvalues ascending, each column signed so its largest-magnitude entry is
 * positive. Either pointer may be NULL. Synchronises the device. */
igafd_status igafd_get_eigen(const igafd_patch *patch, int k, double *U_host,
                             double *D_host);

/* Copy the stencil of A to device memory dst_dev[o * N + row], with
 * o = sum_k (delta_k + p) (2p+1)^(k-1): entry A[row, row + delta]; entries
 * whose column leaves the index box are 0 (Section 2.1, sparsity of A). A
 * half-stored stencil (IGAFD_SETUP_HALF_STENCIL) is written out in this
 * layout, its lower offsets as the stored mirrored couplings. */
igafd_status igafd_copy_stencil(const igafd_patch *patch, double *dst_dev,
                                void *stream);

/* y = A x (Eq. (A)); x_dev and y_dev are length-N device vectors that must
 * not overlap. */
igafd_status igafd_apply_A(igafd_patch *patch, const double *x_dev,
                           double *y_dev, void *stream);

/* z = P^{-1} r by fast diagonalization (Algorithm 1 in 2D, Algorithm 3 in
 * 3D, with the forward step applying U_k^T and the backward step U_k):
 * forward mode-k products, divide by D_1 (+) ... (+) D_d, backward mode-k
 * products. With IGAFD_FP64 the result equals P^{-1} r up to rounding;
 * other dtypes give an inexact P^{-1}. The tensor-core dtypes (BF16, FP16,
 * TF32) need n_k <= 256 and return IGAFD_ERR_ARG otherwise. IGAFD_ADI
 * applies P_J^{-1} as igafd_apply_prec_adi does. r_dev and z_dev must not
 * overlap. */
igafd_status igafd_apply_prec(igafd_patch *patch, igafd_dtype dtype,
                              const double *r_dev, double *z_dev, void *stream);

/* Quadrature points of the patch: Q = prod_k nel_k (p + 1) points, the
 * tensor grid of the (p + 1)-point Gauss rule of every element, indexed
 * q = t_1 + T_1 (t_2 + T_2 t_3) with T_k = nel_k (p + 1) and t_k = e_k (p + 1)
 * + g_k (element e_k, Gauss point g_k, increasing zeta_k; direction 1
 * fastest). x_dev (device, [dim][Q], caller-owned) receives the physical
 * coordinates x_c = F_c(zeta_q) (Section 2.1: the map F of the patch), so a
 * caller can evaluate its load f there for igafd_load_rhs. */
igafd_status igafd_quad_points(const igafd_patch *patch, double *x_dev, void *stream);

/* Right-hand side of the Galerkin system of Eq. (poisson) (Section 2.1: the
 * load vector of Eq. (A)'s system): b_i = int f(F(zeta)) B_i(zeta) |det J|
 * dzeta by the patch's Gauss rule, with f given at the quadrature points:
 * f_qp (device, length Q, caller-owned, order of igafd_quad_points). b_dev:
 * length-N device vector, overwritten, not overlapping f_qp. Errors: ARG
 * (null pointers), CUDA. */
igafd_status igafd_load_rhs(igafd_patch *patch, const double *f_qp, double *b_dev, void *stream);

/* igafd_load_rhs for the manufactured solution u = prod_k sin(pi x_k),
 * f = d pi^2 u (Eq. (poisson) with kappa = 1), f evaluated on the device. */
igafd_status igafd_load_rhs_sine(igafd_patch *patch, double *b_dev, void *stream);

/* Solve A x = b by conjugate gradients preconditioned with P (Section 3),
 * P^{-1} applied by fast diagonalization in opts->prec_dtype (or P_J^{-1}
 * by ADI with IGAFD_ADI, after igafd_adi_setup). x_dev is the
 * initial guess if opts->x0_given, and receives the solution (the best
 * iterate on failure). Synchronises with the host only to poll the
 * convergence flag. Returns the solve status (also in info->status). */
igafd_status igafd_pcg_solve(igafd_patch *patch, const igafd_pcg_opts *opts,
                             const double *b_dev, double *x_dev,
                             igafd_pcg_info *info, void *stream);

/* Batched solve of count independent problems A_i x_i = b_i (one per patch,
 * patches on the same device, each at most once) with the same options,
 * driven on the device. The problems are split into groups (below); a
 * group's loop is a CUDA graph whose conditional while-node repeats one PCG
 * iteration (a pass) of every unfinished member until all are finished, each
 * problem with its own device convergence state (recurrence test, true-
 * residual confirmation and restart, iteration cap, breakdown), and the
 * groups' loops run concurrently, each on its own stream. A pass is a few
 * launches over the group's unfinished members (a compaction kernel lists
 * them first): the stencil as one launch per (dim, p, ring stages, rows per
 * thread) class over (problem, CTA) work items, the vector updates and dot
 * products as one launch each, and the tensor-core FD as one launch per
 * kernel kind for problems on the fused kernels (other FD forms run their
 * own launches). In a group of several problems the stencil and FD CTAs are
 * persistent and take work items from a device queue; a group of one
 * problem launches its single solve's grids. Each work item is a CTA of the
 * problem's own single-problem grid, so the results are bitwise those of
 * igafd_pcg_solve on each problem.
 *
 * igafd_batch_create allocates the batch's device tables and builds the
 * graphs for these patches and options (opts->check_every and timing are not
 * used); it must be re-created when a patch's autotuned choices or its
 * preconditioner set-up change. igafd_batch_solve allocates nothing: b[i],
 * x[i] are device vectors of patch i's size (x[i] the initial guess when
 * opts->x0_given); infos (optional) receives one igafd_pcg_info per problem.
 * It synchronises the stream twice (before the loops, to read every (b, b),
 * and after them). Returns the first non-OK problem status (OK if all
 * converged; IGAFD_ERR_TIMEOUT for a problem still unfinished when its
 * loop's guard of 2 max_iter + 16 passes ran out). Errors: ARG, OOM, CUDA. */
typedef struct igafd_batch igafd_batch;
igafd_status igafd_batch_create(igafd_patch *const *patches, int count,
                                const igafd_pcg_opts *opts, igafd_batch **out);

/* igafd_batch_create with the problems split into `groups` groups (0 or more
 * than count: one per problem): consecutive runs of the problems ordered by
 * the stencil work of an iteration, of near-equal total work, so that each
 * group holds problems of like size. Each group runs the loop above over its
 * own members, as its own graph on its own stream, so the groups' loops run
 * concurrently and a group of problems that need few iterations does not
 * wait for the others; lighter groups get the higher stream priority. With
 * passes_per_launch > 0 a launch of a group's graph ends after that many
 * passes and igafd_batch_solve launches it again while members are
 * unfinished (it polls the launches' completion events); 0 runs each group's
 * whole loop in one launch. Iterates are bitwise those of single solves
 * whatever the grouping. igafd_batch_create is the call with one group per
 * problem (groups = 0) for up to 64 problems, else 64 groups, and
 * passes_per_launch = 0. Errors: ARG (also groups or passes_per_launch < 0),
 * OOM, CUDA. */
igafd_status igafd_batch_create_grouped(igafd_patch *const *patches, int count,
                                        const igafd_pcg_opts *opts, int groups,
                                        int passes_per_launch, igafd_batch **out);

/* The number of groups and (group_of, optional: count ints, host) each
 * problem's group. Errors: ARG. */
igafd_status igafd_batch_groups(const igafd_batch *batch, int *groups, int *group_of);
igafd_status igafd_batch_solve(igafd_batch *batch, const double *const *b_dev,
                               double *const *x_dev, igafd_pcg_info *infos, void *stream);
void igafd_batch_destroy(igafd_batch *batch);

/* Device-clock record of group `group`'s loop in the last igafd_batch_solve,
 * one entry per pass (an iteration of each unfinished member): start_us[k]
 * its start relative to the earliest pass of any group, dur_us[k] its length
 * (globaltimer, us) and active[k] the members unfinished at its start. Host
 * arrays of cap entries (cap may be 0 to query the count); *npasses receives
 * the number of recorded passes (the first min(passes, 65536)). Synchronous
 * copies; call after the solve's stream has been synchronised. Errors: ARG
 * (also a group out of range), CUDA. */
igafd_status igafd_batch_pass_log(const igafd_batch *batch, int group, int cap, double *start_us,
                                  double *dur_us, int *active, int *npasses);

/* igafd_batch_create, igafd_batch_solve and igafd_batch_destroy in one call
 * (allocates and frees the batch's tables each time). */
igafd_status igafd_batch_pcg_solve(igafd_patch *const *patches, int count,
                                   const double *const *b_dev, double *const *x_dev,
                                   const igafd_pcg_opts *opts, igafd_pcg_info *infos,
                                   void *stream);

/* Measured arithmetic peaks of a device, for rooflines: the FP64 FMA pipe
 * (SIMT FMAs, eight independent chains per thread on every SM) and the dense
 * tcgen05 tensor-core rate with FP32 accumulation for TF32 and for BF16
 * operands (M = N = 128 MMAs streamed from shared memory into TMEM), in
 * TFLOP/s (one FMA = 2 FLOP); best of three timed launches after a warm-up,
 * about 20 ms in all; sm_max_mhz is the device's maximum SM clock.
 * Allocates and frees a few bytes of device scratch; synchronises the
 * device. Errors: ARG, OOM, CUDA, TIMEOUT (an MMA completion wait ran out). */
typedef struct {
  double fp64_tflops;
  double tf32_tflops;
  double bf16_tflops;
  double sm_max_mhz;
} igafd_peaks;
igafd_status igafd_probe_peaks(int device, igafd_peaks *out);

/* Default options: tol 1e-8, max_iter 1000, true_every 50, FP64,
 * Fletcher-Reeves, x0 = 0, check_every 4, timing off. */
void igafd_pcg_default_opts(igafd_pcg_opts *opts);

const char *igafd_status_str(igafd_status s);

/* Fast-diagonalization apply z = P^{-1} r in FP64 that allocates no memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (code running while another library owns all device
 * memory through its own pool, latency-critical loops that cannot accept an
 * allocation's implicit device synchronisation, plugins handed buffers but no
 * allocation rights). The caller passes everything: dim (2 or 3), n[dim]
 * (host) dofs per direction, U[dim] and D[dim] (host arrays of device
 * pointers to U_k, row-major n_k x n_k with U[k][i*n_k + j] = (U_k)_{ij}, and
 * to the eigenvalues D_k, e.g. as returned by igafd_get_eigen), r and z
 * (device, length N, not overlapping). The two intermediate tensors live in
 * a file-scope static device array of 2 * IGAFD_STATIC_FD_MAX_DOFS doubles
 * (16 MiB), which every GPU that loads the library holds until the process
 * exits. N = prod n_k above IGAFD_STATIC_FD_MAX_DOFS returns IGAFD_ERR_ARG
 * (with a message on stderr). Every call whose stream is not capturing looks
 * up the array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it per device; a call made during a stream capture
 * uses the cached address, so the first call on a device must come before
 * any stream capture (a captured first call returns IGAFD_ERR_ARG), and
 * after a context reset a call outside a capture must come first. All calls
 * share the array, so calls whose kernels overlap on the GPU race:
 * serialise them. */
#define IGAFD_STATIC_FD_MAX_DOFS 1048576
igafd_status igafd_apply_prec_static(int dim, const int *n, const double *const *U,
                                     const double *const *D, const double *r_dev,
                                     double *z_dev, void *stream);

/* Redo P's setup (Section 4.1 in 2D, Section 5.1 in 3D) in place, on the
 * patch's own buffers (no allocation): the 1D pencils K_k, M_k (span-scaled
 * if igafd_set_scalings set scalings), their generalized eigendecompositions
 * K_k U_k = M_k U_k D_k (Section 5.1, Eq. (eigen3d)), 1 / (D_1 (+) D_2 (+) D_3)
 * and the FP32 and tensor-core copies of U_k. The paper's solver timings
 * include this setup of the preconditioner (Section 7.1), so a full
 * time-to-solution is
 * igafd_setup_prec followed by igafd_pcg_solve. igafd_setup_patch runs it
 * once. Synchronises the stream. Errors: IGAFD_ERR_NOT_SPD (M_k not
 * positive definite), IGAFD_ERR_EIG (no convergence), IGAFD_ERR_CUDA. */
igafd_status igafd_setup_prec(igafd_patch *patch, void *stream);

/* Eigen-solver route for the next setup of P: 0 (default) = for every
 * direction with n_k <= 128, an FP32 start in shared memory (Householder
 * tridiagonalisation, bisection, inverse iteration) followed by FP64
 * iterative refinement of the eigenvectors (Ogita and Aishima, 2018) and
 * exact rotations of nearly degenerate pairs, accepted only if
 * max |U~^T U~ - I| <= 1e-12 and the off-diagonal of U~^T K~ U~ is <= 1e-12
 * of its diagonal, else (and for n_k > 128) FP64 cyclic Jacobi; 1 = FP64
 * Jacobi for every direction. igafd_patch_info.eig_refined reports the
 * route each direction took. Other values: IGAFD_ERR_ARG. */
igafd_status igafd_set_eig_route(igafd_patch *patch, int route);

/* Condition estimate of P^{-1} A from the last PCG solve on this patch (the
 * CG-Lanczos relation: with the recorded step lengths alpha_j and direction
 * factors beta_j, the tridiagonal T with T_00 = 1/alpha_0, T_jj = 1/alpha_j
 * + beta_{j-1}/alpha_{j-1} and T_{j,j+1} = sqrt(beta_j)/alpha_j has as
 * eigenvalues the Ritz values of P^{-1} A; Section 4's bounds are on the
 * spread of that spectrum). steps > 0 uses the first `steps` iterations
 * only (e.g. 30), else all of them (at most 2048 are recorded). Exact for the
 * FP64 preconditioner with Fletcher-Reeves beta; with the flexible beta of
 * the mixed-precision preconditioners it is an estimate of an estimate.
 * Writes lambda_min, lambda_max of T and kappa = lambda_max / lambda_min;
 * IGAFD_ERR_ARG when no iteration was recorded. Synchronises the device. */
igafd_status igafd_pcg_condition_estimate(igafd_patch *patch, int steps, double *kappa,
                                          double *lambda_min, double *lambda_max);

/* Host-only helper of the above: extreme eigenvalues of the CG-Lanczos
 * tridiagonal of m steps from alpha[0..m) and beta[0..m-1) (bisection on
 * Sturm counts). IGAFD_ERR_ARG for m < 1, a non-positive alpha or a
 * negative beta. Needs no GPU. */
igafd_status igafd_lanczos_extremes(const double *alpha, const double *beta, int m,
                                    double *lambda_min, double *lambda_max);

/* Time the candidate configurations of the A stencil's pipeline (ring depth
 * 3, 4 or 6 offset groups in flight per CTA; in 3D also one or two rows per
 * compute thread) and of the tensor-core FD (for TF32 and BF16 operands: the
 * fused kernels, two mode products per CTA with the intermediate on chip,
 * against one kernel per mode product; the fused form needs every n_k <= 128)
 * on this patch and keep the fastest of each. Results are cached per process by (dim, p, n_1, n_2, n_3, SM
 * count) and, if the environment variable IGAFD_TUNE_CACHE names a file,
 * appended to it (one JSON object per line); igafd_setup_patch applies a
 * cached choice without measuring. flags bit 0: measure even if cached.
 * Synchronises the stream; must not overlap a solve on the same patch. */
igafd_status igafd_autotune(igafd_patch *patch, int flags, void *stream);

/* Set the stencil pipeline's ring depth by hand (3, 4 or 6; else
 * IGAFD_ERR_ARG). Every depth computes bitwise the same products. A
 * half-stored stencil runs at the default depth whatever is set. */
igafd_status igafd_set_stencil_stages(igafd_patch *patch, int stages);

/* Set the stencil's rows per compute thread by hand: 1, or 2 (3D only; else
 * IGAFD_ERR_ARG). Each row's FMAs run in the same order either way, so the
 * product is bitwise the same; only the fused dot's summation order moves. */
igafd_status igafd_set_stencil_rows(igafd_patch *patch, int rows);

/* Choose how the tensor-core preconditioner (IGAFD_TF32, IGAFD_BF16) runs
 * the six mode products of Sec. 4.1's fast diagonalization when every n_k is
 * at most 128: fused = 1 (the default) uses three kernels, each chaining two
 * mode products through on-chip memory (modes 1 and 2 forward; mode 3
 * forward, the divide by D_1 (+) D_2 (+) D_3 and mode 3 backward; modes 2 and
 * 1 backward); fused = 0 runs one kernel per mode product through global
 * memory. Both round the operands the same way; results agree to FP32
 * accumulation order. The choice applies to every operand type and replaces
 * the per-type choice of igafd_autotune. Other values: IGAFD_ERR_ARG. */
igafd_status igafd_set_fd_fused(igafd_patch *patch, int fused);

/* Tile shape of the tensor-core FD for operand type dtype (IGAFD_TF32,
 * IGAFD_BF16 or IGAFD_FP16), set by hand (igafd_autotune searches the same
 * space and keeps the fastest; every shape computes the same products, so
 * results agree to the FP32 accumulation order): tile[0] rows of the input
 * per CTA of the per-mode kernel (128, or 64 on a half-filled 128-row MMA
 * tile), tile[1] its output columns split into 1 or 2 tiles (more CTAs,
 * each reading its part of the B image), tile[2] K stages in its shared-
 * memory ring (2 or 3), tile[3] columns per CTA of the fused pencil kernel
 * (128 or 64). IGAFD_ERR_ARG for other values or a shape whose ring does not
 * fit in shared memory. */
igafd_status igafd_set_fd_tile(igafd_patch *patch, igafd_dtype dtype, const int *tile);

/* ---- learned span scalings of the pencils -------------------------------
 * Prop. 1 bounds kappa(P^{-1} A) by the spread of the eigenvalues of Q. The
 * element contributions of the 1D pencils can be weighted per span,
 * K~_k = sum_e wK_{k,e} K_k^(e), M~_k = sum_e wM_{k,e} M_k^(e); P stays a
 * Kronecker sum, so the fast diagonalization applies unchanged, while term k
 * of P follows Q_kk more closely. Rows r <-> (direction k, span e) in
 * direction-major order, r = sum_{l<k} nel_l + e; igafd_scaling_rows gives
 * their number. These calls allocate temporary device memory. */
igafd_status igafd_scaling_rows(const igafd_patch *patch, int *rows);

/* Per-row features of Q over the slab of quadrature points whose direction-k
 * coordinate lies in span e: [log mean Q_kk, log mean of the other diagonal
 * entries, log min lambda_min(Q), log max lambda_max(Q), std of log Q_kk,
 * span centre]. feat_dev: float [rows][6]. Synchronises the stream. */
igafd_status igafd_patch_features(igafd_patch *patch, float *feat_dev, void *stream);

/* Separable least-squares fit of log Q_kk over all quadrature points by
 * log wK_k(zeta_k) + sum_{l != k} log wM_l(zeta_l) (backfitting, `sweeps`
 * rounds of slab means; the mean of each log wM_l is fixed to 0).
 * logw_dev: float [rows][2] = (log wK, log wM). Synchronises the stream. */
igafd_status igafd_patch_sepfit(igafd_patch *patch, int sweeps, float *logw_dev, void *stream);

/* Rebuild the preconditioner from span-scaled pencils: logw_dev float
 * [rows][2] of (log wK, log wM), or NULL for the unscaled pencils (the
 * paper's P). Recomputes the eigendecompositions and every FD factor.
 * Synchronises the stream. */
igafd_status igafd_set_scalings(igafd_patch *patch, const float *logw_dev, void *stream);

/* The scaling network: 6 -> 64 -> 64 -> 2, tanh, FP16 weights in the forward
 * pass with FP32 arithmetic; FP32 master weights and Adam for training.
 * Parameter layout (floats): W1[64][6], b1[64], W2[64][64], b2[64],
 * W3[2][64], b3[2]. Inputs are normalised by (x - in_mean) / in_std and the
 * outputs mapped back by out_mean + out_std * net(x). */
#define IGAFD_MLP_PARAMS 4738
typedef struct igafd_mlp igafd_mlp;
/* params_host: IGAFD_MLP_PARAMS initial values (NULL: zeros). */
igafd_status igafd_mlp_create(const float *params_host, igafd_mlp **out);
void igafd_mlp_destroy(igafd_mlp *mlp);
igafd_status igafd_mlp_set_normalization(igafd_mlp *mlp, const float *in_mean,
                                         const float *in_std, const float *out_mean,
                                         const float *out_std);
igafd_status igafd_mlp_get_params(const igafd_mlp *mlp, float *params_host);
igafd_status igafd_mlp_set_params(igafd_mlp *mlp, const float *params_host);
/* Y_dev float [rows][2] = network(X_dev float [rows][6]). */
igafd_status igafd_mlp_forward(igafd_mlp *mlp, const float *X_dev, int rows, float *Y_dev,
                               void *stream);
/* Gradient of the mean squared error of the normalised outputs against the
 * normalised targets T_dev float [rows][2], w.r.t. every parameter
 * (grad_host: IGAFD_MLP_PARAMS floats, may be NULL) and the loss. */
igafd_status igafd_mlp_gradient(igafd_mlp *mlp, const float *X_dev, const float *T_dev, int rows,
                                float *grad_host, float *loss_host, void *stream);
/* One Adam step (beta 0.9 / 0.999) on that loss; loss_host (optional) gets
 * the loss before the step. */
igafd_status igafd_mlp_train_step(igafd_mlp *mlp, const float *X_dev, const float *T_dev,
                                  int rows, float lr, float *loss_host, void *stream);

/* ---- ADI preconditioners (Section 4.2, Algorithm 2; Section 5.2,
 * Algorithm 4) ----------------------------------------------------------
 * An alternative to the fast-diagonalization P^{-1}: J iterations from
 * s_0 = 0 of the Peaceman-Rachford scheme of Eq. (ADI) (2D, gamma_j =
 * omega_j) or of the Douglas scheme of Eq. (ADI3D) (3D), on the same pencils
 * (span-scaled when scalings are set at the time of igafd_adi_setup), give
 * z = P_J^{-1} r with P_J symmetric positive definite and
 * kappa(P_J^{-1} A) <= (1 + eps)/(1 - eps) kappa(P^{-1} A) when the error
 * operator has ||T_J|| <= eps (Theorem 1 and its 3D analogue). n_k <= 256. */

/* 2D: the optimal parameters for equal spectral intervals [a, b]:
 * J = ceil(ln(4 b / a) ln(4 / eps) / pi^2) (Eq. (ADIits)) and
 * omega_host[j-1] = b dn((2j - 1) K / (2J), k), k^2 = 1 - (a/b)^2 (the
 * elliptic-function solution of the one-variable minimax, by the
 * arithmetic-geometric mean from k' = a / b). 0 < a <= b, 0 < eps < 1;
 * omega_host holds max_J values; IGAFD_ERR_NOT_CONVERGED when J > max_J.
 * Needs no GPU. */
igafd_status igafd_adi_wachspress(double a, double b, double eps, int max_J,
                                  double *omega_host, int *J);

/* Parameters for the patch: in 2D igafd_adi_wachspress on the hull of the
 * spectra of M_1^{-1} K_1 and M_2^{-1} K_2 (the patch's D_k); in 3D the
 * greedy parameters of Eqs. (greedy1)-(greedy2) over the triples of
 * eigenvalues of M_k^{-1} K_k (the patch's D_k): omega_host[0..*J-1] get
 * w_1.., *J the first count with rho_J = max over the triples of
 * |prod_j g(w_j; l)| <= eps, g(w; l) = 1 - 2 w^2 (l1 + l2 + l3) /
 * ((w + l1)(w + l2)(w + l3)). The first parameter minimises |g| at the
 * triple of smallest eigenvalues; each later one minimises |g| at the triple
 * where the product is largest (first in i3, i2, i1 order); where |g| has
 * two zeros, the one giving the smaller rho is taken. omega_host must hold
 * max_J values; 0 < eps < 1. Runs on the host (O(J n1 n2 n3)); synchronises
 * the device. Returns IGAFD_ERR_NOT_CONVERGED (with *J = max_J) when max_J
 * parameters do not reach eps. */
igafd_status igafd_adi_parameters(igafd_patch *patch, double eps, int max_J,
                                  double *omega_host, int *J);

/* Host-only core of igafd_adi_parameters on given spectra L1[n1], L2[n2],
 * L3[n3] (positive; the greedy start is at L1[0], L2[0], L3[0], so pass them
 * ascending): the same parameters and return codes. Multithreaded over the
 * triples (contiguous chunks, deterministic result). Needs no GPU. */
igafd_status igafd_adi_greedy(const double *L1, int n1, const double *L2, int n2,
                              const double *L3, int n3, double eps, int max_J,
                              double *omega, int *J);

/* Set up the ADI preconditioner (2D or 3D) with parameters omega_host[0..J-1] (> 0):
 * banded pencils and the banded Cholesky factors of K_k + w_j M_k and of M_k
 * for every direction and parameter, and 6 N-vectors of scratch (the
 * library's only allocation for ADI). dtype IGAFD_FP64 (the paper's
 * arithmetic) or IGAFD_FP32 (FP32 scratch, factors and arithmetic; an
 * inexact P_J). Replaces an earlier ADI set-up; synchronises the stream.
 * IGAFD_ERR_NOT_SPD if a factorisation fails. */
igafd_status igafd_adi_setup(igafd_patch *patch, const double *omega_host, int J,
                             igafd_dtype dtype, void *stream);

/* z = P_J^{-1} r by J ADI iterations: in 2D (Algorithm 2) two kernels of
 * independent banded line problems per iteration, along directions 1 and 2,
 * and a final M_1 solve (2J + 1 launches); in 3D (Algorithm 4) four per
 * iteration, along directions 2, 1, 2, 3 (4J + 1 launches in all). r_dev, z_dev: length-N FP64 device vectors, not
 * overlapping. IGAFD_ERR_ARG without igafd_adi_setup. */
igafd_status igafd_apply_prec_adi(igafd_patch *patch, const double *r_dev,
                                  double *z_dev, void *stream);

/* ---- Multi-patch numbering (Section 6) ----------------------------------
 * Global C^0 space of conforming patches glued along whole sides, and its
 * homogeneous Dirichlet set (every function on a side glued to nothing).
 * m[q * dim + k]: B-splines of patch q in direction k (>= 2). glue[5 g ..]:
 * {patch a, side a, patch b, side b, orientation}, side = 2 (direction) +
 * (0: index 0, 1: last index); the functions of the two sides are matched
 * in the order of their tangential indices (directions other than the
 * side's, increasing), with orientation bit 0 reversing the first
 * tangential direction of side a on side b, bit 1 the second (3D), bit 2
 * exchanging them (3D). Outputs: global[off_q + local] (local index
 * direction 1 fastest, patches concatenated; capacity sum_q prod_k m) the
 * global function of each patch function, numbered in order of first
 * appearance; fixed[g] = 1 for Dirichlet functions (capacity as global);
 * *n_global. IGAFD_ERR_ARG for bad indices or sides of different sizes.
 * Host only; needs no GPU. */
igafd_status igafd_mp_numbering(int dim, int npatch, const int *m, int nglue,
                                const int *glue, long long *global,
                                unsigned char *fixed, long long *n_global);

/* Subdomain of two glued patches qa, qb (Section 6): the single patch made
 * of them along direction dir (patch a's functions first, b's after the
 * shared side; their other directions must match and a's last side in dir
 * must be glued to b's first one in order). rows[] (capacity the product of
 * shape) gets, in the merged patch's order with Dirichlet rows removed
 * (direction 1 fastest), the global function of each of its interior
 * functions, i.e. the rows of R_i; shape[0..dim) its interior sizes. Inputs
 * as returned by igafd_mp_numbering. IGAFD_ERR_ARG when the patches are not
 * glued that way or an interior function is fixed. Host only. */
igafd_status igafd_mp_subdomain(int dim, int npatch, const int *m,
                                const long long *global, const unsigned char *fixed,
                                int qa, int qb, int dir, long long *rows, int *shape);

/* Additive Schwarz preconditioner P_IAS = sum_i R_i^T P_i^{-1} R_i
 * (Eq. (Pias)) of a multi-patch problem: subdomain i is the single patch
 * patches[i] (e.g. two glued patches merged into one, built without a
 * stencil), P_i^{-1} its fast-diagonalization solve, and rows[i][0..N_i)
 * (host, N_i the patch's dofs, distinct, in [0, n_global)) the global
 * function of each of its dofs. The object does not own the patches, which
 * must outlive it. Errors: ARG, OOM, CUDA. */
typedef struct igafd_mp igafd_mp;
igafd_status igafd_mp_create(int nsub, igafd_patch *const *patches,
                             const long long *const *rows, long long n_global,
                             igafd_mp **out);
void igafd_mp_destroy(igafd_mp *mp);
/* z = P_IAS r: z = 0, then per subdomain a gather R_i r, the patch's FD in
 * dtype, and a scatter-add R_i^T (2 kernels + the FD's per subdomain).
 * r_dev, z_dev: length-n_global FP64 device vectors, not overlapping. */
igafd_status igafd_mp_apply_ias(igafd_mp *mp, igafd_dtype dtype, const double *r_dev,
                                double *z_dev, void *stream);

/* The multi-patch stiffness matrix (Section 6: the global C^0 space of glued
 * patches, Eq. (A) summed over the patches): A = sum_q R_q^T A_q R_q, where
 * A_q is patch q's stiffness on its full index box (patches[q] built with
 * IGAFD_SETUP_FULL_SPACE) and R_q takes a global free vector to the patch's
 * local functions: free_of_local[q][t] (host, one per local function,
 * direction 1 fastest) is the global free index of local function t, or -1
 * for a function fixed by the Dirichlet condition (from igafd_mp_numbering:
 * the rank of its global function among the free ones). The indices of one
 * patch must be distinct. Replaces an earlier operator; the patches must
 * outlive mp. Errors: ARG (not full-space, no stencil, bad indices), OOM. */
igafd_status igafd_mp_set_operator(igafd_mp *mp, int npatch, igafd_patch *const *patches,
                                   const long long *const *free_of_local);

/* y = A x with the operator of igafd_mp_set_operator: y = 0, then per patch
 * a gather to its full index box (fixed functions 0), the patch's own
 * stencil, and a scatter-add of the free rows (patches one after the other
 * on the stream, so no atomics). x_dev, y_dev: length n_global, not
 * overlapping. */
igafd_status igafd_mp_apply_A(igafd_mp *mp, const double *x_dev, double *y_dev, void *stream);

/* Conjugate gradients on the multi-patch system A x = b (Section 6, Table
 * "L"), preconditioned by P_IAS (igafd_mp_apply_ias with opts->prec_dtype:
 * FP64, FP32 or the tensor-core types), with the stopping rule of
 * igafd_pcg_solve (recurrence residual, confirmed by the true residual;
 * periodic true residual every opts->true_every; Fletcher-Reeves or, with
 * opts->flexible, the flexible beta). The host drives the loop and reads the
 * dot products back every iteration (the multi-patch problems are small 2D
 * ones); uses workspace allocated by igafd_mp_set_operator. b_dev, x_dev:
 * length n_global (x_dev the initial guess when opts->x0_given). */
igafd_status igafd_mp_pcg_solve(igafd_mp *mp, const igafd_pcg_opts *opts, const double *b_dev,
                                double *x_dev, igafd_pcg_info *info, void *stream);

/* Number of kernels this library has enqueued in this process so far (all
 * devices, all patches); for launch accounting by benchmarks. */
long long igafd_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* IGAFD_H */

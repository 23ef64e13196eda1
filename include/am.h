/*
 * am.h -- C ABI of the GB300 articulated-body Stokes solver (libam.so).
 *
 * The library solves, for suspensions of rigid bodies linked by joints in a
 * viscous (Stokes) fluid, the constrained mobility problem of Sec. 2.3,
 * Eq. linear_system:
 *
 *     [ M    -K   0  ] [lambda]   [ u_s ]
 *     [-K^T   0   C^T] [  U   ] = [ -F  ]
 *     [ 0     C   0  ] [ phi  ]   [  B  ]
 *
 * lambda: forces on the blobs that discretise each body (3 per blob);
 * U = (u_p, omega_p): body velocities (6 per body);
 * phi: Lagrange multipliers of the link constraints (3 per link);
 * M: the Rotne-Prager-Yamakawa blob mobility (Eq. RPY), in free space or
 *    above a no-slip wall at z = 0;
 * K: rigid-body map, (K U)_i = u_p + omega_p x (r_i - q_p) (Eq. no-slip);
 * C: constraint Jacobian of the links (Eq. dg_compact, App. A);
 * B: active-link term (Eq. dg).
 * It is solved by right-preconditioned GMRES with the block-diagonal
 * preconditioner of Sec. 3.1, and am_solve_step advances the bodies by one
 * explicit Euler step with the reconstruction and nonlinear correction of
 * Sec. 4.
 *
 * Conventions for every entry point:
 *  - Return 0 (AM_OK) on success or a negative AM_ERR_* code; the handle's
 *    message is then available from am_last_error(handle) (or
 *    am_last_error(NULL) for the stateless calls).
 *  - Host pointers are caller-owned, read or written during the call only,
 *    never retained.  Arrays are dense, row-major, FP64 unless stated; "3N"
 *    means N consecutive (x, y, z) triples.
 *  - Device pointers (only in am_rpy_matvec) are caller-owned device memory
 *    of the current CUDA device.
 *  - The library owns all device memory of a handle; a handle is not
 *    thread-safe.  All work of a handle runs on its stream.
 */
#ifndef AM_H
#define AM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define AM_API __attribute__((visibility("default")))
#else
#define AM_API
#endif

/* ---- status codes ---------------------------------------------------- */
#define AM_OK                    0
#define AM_ERR_ARG              -1  /* bad argument, size or call order      */
#define AM_ERR_CUDA             -2  /* a CUDA call failed                     */
#define AM_ERR_NOT_CONVERGED    -3  /* GMRES hit max_iter; outputs written    */
#define AM_ERR_WALL_PENETRATION -4  /* a blob centre at or below height a     */
#define AM_ERR_NONUNIT_QUAT     -5  /* | |theta| - 1 | > 1e-8 on input        */
#define AM_ERR_SINGULAR         -6  /* a body's blob mobility block is not SPD */

/* ---- precision of the blob mobility product --------------------------- */
#define AM_FP64  0   /* every operation in FP64                              */
#define AM_MIXED 1   /* pair terms in FP32, per-target sums in FP64; the
                        outer residual of the refinement with double-float
                        pair terms (AM_DF64); Arnoldi and constraint algebra
                        in FP64                                              */
#define AM_DF64  2   /* pair terms in double-float arithmetic (pairs of
                        floats, ~2^-44 relative), sums in FP64: only as the
                        arithmetic of am_apply_mobility_ex                   */

typedef struct am_handle am_handle;

typedef struct {
    double eta;          /* fluid viscosity (> 0)                           */
    double blob_radius;  /* a (> 0), the same for every blob                */
    int    wall;         /* 0: free space; 1: no-slip wall at z = 0         */
    int    precision;    /* AM_FP64 or AM_MIXED                             */
    int    n_systems;    /* independent suspensions S in the handle
                            (1..65536; 0 -> 1), each with its own
                            bodies, links and GMRES state               */
    double tol;          /* GMRES stop: ||b - A y||_2 <= tol ||b||_2        */
    int    restart;      /* GMRES restart length m (1..200); 0 -> 50        */
    int    max_iter;     /* total GMRES iterations cap; 0 -> 500            */
    double corr_tol;     /* delta of Sec. 4.3; correction runs when
                            ||g*||_2^2 >= delta; 0 -> 1e-10                 */
    int    corr_max_iter;/* Gauss-Newton iteration cap; 0 -> 20             */
    void*  cuda_stream;  /* cudaStream_t to run on; NULL -> library stream  */
    int    single_blob;  /* 1: every body is one blob of radius blob_radius
                            at its tracking point, with rotational coupling
                            (Sec. 2.4; free space, AM_FP64); the problem is
                            Eq. linear_system_general on (U, phi) and the
                            blob arguments of am_set_bodies are ignored   */
    double box[3];       /* all 0: unbounded fluid (free space or wall).
                            All > 0: triply periodic box [0, Lx) x [0, Ly)
                            x [0, Lz) with zero mean flow (the periodic
                            suspensions of Sec. 5.3; here without the
                            wall): the blob mobility is the RPY tensor
                            periodised by spectral Ewald summation
                            (O(N log N)); needs wall = 0, one system,
                            multi-blob bodies and every side longer than
                            6 a.  AM_MIXED: FP32 wave part and blocks for
                            the inner products (tolerance max(ewald_tol,
                            1e-6)), the FP64 product for the outer
                            residuals.  Bodies are not wrapped: q
                            stays continuous, the product wraps blob
                            centres into the box                         */
    double ewald_tol;    /* relative accuracy of the periodic product
                            (1e-14 .. 1e-3); 0 -> 1e-10                 */
    double ewald_xi;     /* Ewald splitting parameter (1/length); 0 ->
                            chosen for the least work per product        */
} am_config;

typedef struct {
    int    status;          /* return code of the call                       */
    int    iterations;      /* GMRES iterations (Arnoldi steps)              */
    int    restarts;        /* GMRES cycles started                          */
    double rel_residual;    /* ||b - A y||_2 / ||b||_2 at exit: AM_FP64 the
                               true residual with FP64 products; AM_MIXED
                               the residual with double-float products, or
                               after a correction computed from one, an
                               upper bound of it (the inner mixed residual
                               plus 1e-5 |M32 lambda_dx|, the mixed
                               product's error bound)                        */
    double constraint_residual; /* max_n |(C U - B)_n| at exit               */
    double g2_before;       /* ||g*||_2^2 after reconstruction (Sec. 4.3)    */
    double g2_after;        /* ||g||_2^2 at the end of the step              */
    int    corr_iterations; /* max Gauss-Newton iterations over assemblies   */
    long long pairs;        /* blob pairs evaluated by mobility products     */
    int    kernel_launches; /* kernels launched by the call                  */
    double ms_precond;      /* device time: preconditioner build             */
    double ms_gmres;        /* device time: GMRES                            */
    double ms_update;       /* device time: Euler update, reconstruction,
                               correction                                    */
    int    learned_systems; /* systems whose initial guess used the learned
                               model (am_set_learned; with the check: a
                               positive step along it)                       */
    double rel_residual0;   /* true ||b - A y0||_2 / ||b||_2 of the initial
                               guess (max over systems)                      */
} am_step_stats;

/* Create a solver handle.  cfg is copied.  Errors: AM_ERR_ARG for eta <= 0,
 * blob_radius <= 0, wall not 0/1, unknown precision, n_systems outside
 * 1..65536, tol <= 0 or restart/max_iter out of range, single_blob not 0/1
 * or with a wall or mixed precision; AM_ERR_CUDA.
 *
 * Several systems (n_systems = S > 1): every system is set separately
 * (am_set_bodies/am_set_constraints with its index) and the device layout is
 * built once all have bodies.  Every solve handles all systems at once, each
 * with its own GMRES (own Krylov basis, Givens rotations and stopping test on
 * its own ||b_s||); rel_residual and iteration counts in am_step_stats are
 * the maxima over systems.  Outputs and the link vectors of am_solve_step
 * are the systems' arrays concatenated in system order. */
AM_API int am_create(const am_config* cfg, am_handle** out);

/* Set the bodies of system `system` (0 <= system < n_systems) at the
 * current time (Sec. 2.1, 2.3).
 *   n_bodies         M > 0
 *   q                3M   tracking points q_p (lab frame)
 *   theta            4M   unit quaternions [s, p] of the orientations
 *   blob_offset      M+1  int, CSR offsets: body p owns blobs
 *                         blob_offset[p] .. blob_offset[p+1]-1; [0] = 0,
 *                         every body has at least one blob
 *   blob_body_pos    3Nb  body-frame blob positions relative to q_p, so that
 *                         r_i = q_p + R(theta_p) blob_body_pos_i
 *   force_torque     6M   F_p = (f_p, tau_p) (tau about q_p)
 *   slip             3Nb  slip velocities u_s of Eq. linear_system, or NULL
 *   assembly_of_body M    int, articulated-body index of each body, in
 *                         0 .. n_assemblies-1, every index used
 * Replaces any earlier bodies (and drops links and the solution history).
 * Errors: AM_ERR_ARG, AM_ERR_NONUNIT_QUAT, AM_ERR_WALL_PENETRATION (wall and
 * some r_i,z <= a), AM_ERR_CUDA. */
AM_API int am_set_bodies(am_handle* h, int system, int n_bodies,
                         const double* q, const double* theta,
                         const int* blob_offset, const double* blob_body_pos,
                         const double* force_torque, const double* slip,
                         const int* assembly_of_body);

/* Set the links of system `system` (Eq. constraint):
 *   g_n = q_p + R(theta_p) dl_p[n] - q_q - R(theta_q) dl_q[n] = 0.
 *   n_links          P >= 0
 *   body_p, body_q   P    int, distinct bodies of the same articulated body
 *   dl_p, dl_q       3P   body-frame link vectors at the current time
 *   dl_p_dot, dl_q_dot 3P their time derivatives (active links, Eq. dg), or
 *                    both NULL for passive links (B = 0)
 * May be called before every step to move active links; the connectivity
 * (body_p, body_q) may change too.  Needs am_set_bodies first.
 * Errors: AM_ERR_ARG (bad index, p == q, cross-assembly link, articulated
 * body not connected by its links), AM_ERR_CUDA. */
AM_API int am_set_constraints(am_handle* h, int system, int n_links,
                              const int* body_p, const int* body_q,
                              const double* dl_p, const double* dl_q,
                              const double* dl_p_dot, const double* dl_q_dot);

/* Passive links given by their joint points in the lab frame at the current
 * pose: dl_p[n] = R(theta_p)^T (joint_n - q_p), dl_q[n] likewise, so that
 * g = 0 now.  joint: 3P.  Otherwise as am_set_constraints. */
AM_API int am_set_joints(am_handle* h, int system, int n_links,
                         const int* body_p, const int* body_q,
                         const double* joint);

/* Solve Eq. linear_system at the current pose (no time step).  Outputs (any
 * may be NULL): U 6M, phi 3P, lambda 3Nb.  With a rank-deficient C, phi is
 * determined up to null(C^T); lambda, U and C^T phi are unique.
 * Errors: AM_ERR_ARG (no bodies), AM_ERR_NOT_CONVERGED (outputs written),
 * AM_ERR_CUDA. */
AM_API int am_solve(am_handle* h, am_step_stats* stats,
                    double* U_out, double* phi_out, double* lambda_out);

/* One explicit Euler step of Sec. 4.3 from t to t + dt: solve Eq.
 * linear_system at t (initial guess from the earlier solves, see
 * am_set_initial_guess; the previous solution by default),
 * move each articulated body's centre by dt times its mean body velocity
 * (Eq. ucom) and each orientation by theta_{omega dt} . theta, rebuild the
 * positions with the pseudo-inverse of the connectivity (Eq. pseudo-inv-sol,
 * reconst-up-COM) using the link vectors at t + dt, and run the nonlinear
 * correction (Eq. min_probl_a/b) when ||g*||^2 >= corr_tol.
 *   dl_p_next, dl_q_next  3P each: body-frame link vectors at t + dt, or
 *                         NULL to keep the current ones (passive links).
 * The link derivatives for t + dt must be set by am_set_constraints before
 * the next step.  Outputs as am_solve (values at t).
 * Errors: as am_solve, and AM_ERR_ARG if an articulated body of several
 * bodies is not connected by links. */
AM_API int am_solve_step(am_handle* h, double t, double dt,
                         const double* dl_p_next, const double* dl_q_next,
                         am_step_stats* stats,
                         double* U_out, double* phi_out, double* lambda_out);

/* One explicit midpoint (RK2) step of App. "Midpoint scheme" from t to
 * t + dt: solve at t (guess as am_solve_step), move each articulated body's centre and
 * orientations by dt/2 with those velocities and reconstruct (with the
 * nonlinear correction when ||g*||^2 >= corr_tol) using the link vectors at
 * t + dt/2, solve at that midpoint, then move the pose at t by dt with the
 * midpoint velocities and reconstruct and correct with the link vectors at
 * t + dt.
 *   dl_p_half, dl_q_half          3P each: body-frame link vectors at
 *                                 t + dt/2, or NULL to keep the current ones
 *   dl_p_half_dot, dl_q_half_dot  3P each: their time derivatives (active
 *                                 links: required; passive links: NULL)
 *   dl_p_next, dl_q_next          3P each: link vectors at t + dt, or NULL
 * Outputs (any may be NULL) are the midpoint solution (the velocities used
 * for the update).  stats: iterations and times of both solves summed,
 * rel_residual the larger, g2 of the final reconstruction.  As for
 * am_solve_step, the link derivatives for t + dt must be set by
 * am_set_constraints before the next step.  Errors: as am_solve_step. */
AM_API int am_solve_step_rk2(am_handle* h, double t, double dt,
                             const double* dl_p_half, const double* dl_q_half,
                             const double* dl_p_half_dot, const double* dl_q_half_dot,
                             const double* dl_p_next, const double* dl_q_next,
                             am_step_stats* stats,
                             double* U_out, double* phi_out, double* lambda_out);

/* Current bodies (after the last step): q 3M, theta 4M; either may be NULL. */
AM_API int am_get_bodies(am_handle* h, int system, double* q, double* theta);

/* Current lab-frame blob positions r_i (3Nb). */
AM_API int am_get_blobs(am_handle* h, int system, double* r);

/* One blob mobility product u = M lambda at the current pose (Eq. RPY),
 * host arrays of 3Nb.  For checking and benchmarking the hot kernel.  With
 * single_blob: the body mobility N, (f, tau) per body in and (u, omega) per
 * body out, 6M each. */
AM_API int am_apply_mobility(am_handle* h, const double* lambda, double* u);

/* As am_apply_mobility with the pair arithmetic chosen: AM_FP64, AM_MIXED
 * (FP32 pair terms) or AM_DF64 (double-float pair terms, the arithmetic of
 * the mixed solver's outer residual), whatever the handle's precision.  For
 * checking and benchmarking the products.  Errors: AM_ERR_ARG (unknown
 * arithmetic, no bodies), AM_ERR_CUDA. */
AM_API int am_apply_mobility_ex(am_handle* h, const double* lambda, double* u, int arithmetic);

/* Steric repulsion (Sec. 5.3 uses one between bacteria and with the wall
 * without giving its form; this is the library's).  Between blobs of
 * different articulated bodies closer than `cutoff`:
 *     U(r) = eps (1 + (2a - r) / range)   r <  2a
 *     U(r) = eps exp((2a - r) / range)    r >= 2a
 * and, with a wall, on every blob at height h:
 *     U_w(h) = eps_wall (1 + (a - h) / range_wall)   h <  a
 *     U_w(h) = eps_wall exp((a - h) / range_wall)    h >= a
 * The blob forces -grad U reach each body as force and torque about its
 * tracking point (K^T f) and are added to its external force and torque at
 * every solve and step.  eps = eps_wall = 0 turns it off (the default).
 * Positions must stay below about 1e4 in magnitude (the pair search screens
 * candidates in FP32).  Errors: AM_ERR_ARG (negative values, non-positive
 * range with eps > 0, wall term without a wall). */
AM_API int am_set_repulsion(am_handle* h, double eps, double range, double cutoff,
                            double eps_wall, double range_wall);
/* The steric blob forces (3Nb) at the current pose (zeros when off). */
AM_API int am_steric_forces(am_handle* h, double* f);

/* Layout of the all-pairs product of h instead of the autotuned one: work
 * items of 128 x targets_per_thread targets (2: two targets per thread in
 * paired FP32 lanes; mixed precision only, FP64 handles use 1) against
 * source chunks of source_chunk blobs (0: a default that fills the GPU).
 * targets_per_thread = 0 restores autotuning before the next product;
 * targets_per_thread = 3 selects the symmetric product (handles without a
 * box) on tiles of source_chunk = 32, 64 or 128 blobs (mixed handles: two
 * targets per thread in paired FP32 lanes on tiles of 128, one target per
 * thread on tiles of 32 and 64).  The
 * layout is rebuilt (and autotuned) whenever the bodies change.  A
 * measurement and testing aid, not in the paper.  Errors: AM_ERR_ARG (no
 * bodies, values out of range), AM_ERR_CUDA. */
AM_API int am_set_mobility_layout(am_handle* h, int targets_per_thread, int source_chunk);

/* The layout of the all-pairs product in use (after the autotuning of the
 * first product): layout[0] targets per thread, [1] source chunk (blobs),
 * [2] targets per work item, [3] tile of the symmetric product (32, 64 or
 * 128 blobs; 0 when the one-direction kernel runs).  The symmetric
 * product evaluates each unordered pair of blobs once and applies it in both
 * directions (M_ji = M_ij^T); the autotuner takes it when it is faster and
 * its partial sums (one slot per tile) fit (1 GiB; mixed in paired lanes,
 * tiles of 128: a quarter of the free device memory).  A
 * measurement aid, not in the paper.  Errors: AM_ERR_ARG (NULL, no
 * bodies). */
AM_API int am_get_mobility_layout(am_handle* h, int* layout);

/* y -> A y for the full operator of Eq. linear_system at the current pose
 * (y and Ay: 3Nb + 6M + 3P, ordered (lambda, U, phi)). */
AM_API int am_apply_operator(am_handle* h, const double* y, double* Ay);

/* r -> z solving the block-diagonal approximate problem (Eq. precond) at
 * the current pose, with G~ a generalised inverse when C is
 * rank-deficient (Eq. block_diag_const_res).  Same layout as
 * am_apply_operator. */
AM_API int am_apply_precond(am_handle* h, const double* r, double* z);

/* Stateless blob mobility product on device memory of the current device,
 * u = M(r) lambda (Eq. RPY), free space (wall = 0) or above a no-slip wall
 * at z = 0 (wall = 1; every r_z must exceed a, not checked here).
 *   d_r        3n doubles, blob centres
 *   d_lambda   3n doubles, blob forces
 *   d_u        3n doubles, output velocities (overwritten)
 *   precision  AM_FP64 or AM_MIXED
 *   d_work     scratch of at least am_rpy_matvec_workspace(n, precision)
 *              bytes, 256-byte aligned; contents are overwritten
 *   stream     cudaStream_t or NULL (legacy default stream)
 * Asynchronous on `stream`.  Errors: AM_ERR_ARG (n < 0, eta or a <= 0, NULL
 * pointer with n > 0, workspace too small or misaligned), AM_ERR_CUDA. */
AM_API int am_rpy_matvec(const double* d_r, const double* d_lambda,
                         double* d_u, int n, double eta, double a, int wall,
                         int precision, void* d_work, size_t work_bytes,
                         void* stream);
AM_API size_t am_rpy_matvec_workspace(int n, int precision);

/* Rows row0 .. row0 + nrows - 1 of the product u = M(r) lambda against all
 * n sources: the local step of a suspension sharded by blobs over several
 * GPUs, after the positions and forces of all shards have been gathered.
 *   d_r, d_lambda  3n doubles (all blobs, device); d_u  3 nrows doubles
 *   d_work         at least am_rpy_matvec_rows_workspace(n, nrows,
 *                  precision) bytes, 256-byte aligned
 * Otherwise as am_rpy_matvec (with row0 = 0 and nrows = n the two agree).
 * Errors: AM_ERR_ARG (rows outside 0 .. n - 1 and as am_rpy_matvec),
 * AM_ERR_CUDA. */
AM_API int am_rpy_matvec_rows(const double* d_r, const double* d_lambda, double* d_u, int n,
                              int row0, int nrows, double eta, double a, int wall, int precision,
                              void* d_work, size_t work_bytes, void* stream);
AM_API size_t am_rpy_matvec_rows_workspace(int n, int nrows, int precision);

/* Allocation-free variant of am_rpy_matvec for callers that cannot call
 * cudaMalloc: code that runs where allocating is not allowed or not safe,
 * e.g. inside another library's allocation-free execution path, a host
 * callback, or a process whose device memory is owned by a pool it must
 * not grow.  The caller still passes inputs and outputs (d_r, d_lambda,
 * d_u, n, eta, a, wall, precision and stream mean what they mean for
 * am_rpy_matvec); the scratch lives in a fixed device array of
 * AM_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits.
 *  - Limit: n must satisfy am_rpy_matvec_workspace(n, precision) <=
 *    AM_NOALLOC_SCRATCH_BYTES, evaluated with the device of the call
 *    current (the source split, and with it the scratch, depends on the
 *    SM count); on a 152-SM GB300 that is n <= about 150,000 blobs for
 *    either precision.  Larger n returns AM_ERR_ARG with a message, and
 *    nothing is launched.
 *  - Every call looks up the array's device address on the current device
 *    (cudaGetSymbolAddress; not a stream operation).  The first call on a
 *    device may load the library's device code there: make that first call
 *    before any stream capture.
 *  - Every call on a device shares the one array: calls that overlap on the
 *    GPU (other streams, other threads) race and corrupt each other.  The
 *    array keeps the last call's contents; no part of it needs to start at
 *    zero, since each call writes every scratch value it reads.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * The paper has no counterpart to this entry point. */
#define AM_NOALLOC_SCRATCH_BYTES (8u << 20)
AM_API int am_rpy_matvec_noalloc(const double* d_r, const double* d_lambda, double* d_u,
                                 int n, double eta, double a, int wall, int precision,
                                 void* stream);

/* Pair arithmetic of the mobility kernels, counted with FMA = 2 flops, for
 * roofline figures: per pair of the free-space tensor and per pair of the
 * wall tensor (free part plus image part). */
AM_API int am_flops_per_pair(int wall);

/* Device time of the all-pairs mobility kernel inside the calls of h,
 * measured with CUDA events on the handle's stream around every launch.
 * enable != 0 clears earlier records and starts recording; enable == 0
 * stops recording and keeps the records.  *ms and *launches (either may be
 * NULL) receive the total time and the number of launches recorded so far
 * (this synchronises the stream).  Not in the paper: a measurement aid. */
AM_API int am_mobility_timing(am_handle* h, int enable, double* ms, long long* launches);

/* Throughput of independent FMA streams on the current device, the
 * denominator of the roofline of ALU-bound kernels: fp64 = 1 measures DFMA,
 * 0 FFMA; *flops receives FLOP/s (FMA = 2).  Takes about 0.1 s.  Not in the
 * paper: a measurement aid. */
AM_API int am_alu_peak(int fp64, double* flops);

/* Kernels launched by this library in this process so far. */
AM_API long long am_kernel_launches(void);

/* ---- learned initial guess ----------------------------------------------
 * The paper has no learned component.  These calls add an initial guess for
 * cold starts (am_solve, and the first am_solve_step) predicted per body by
 * a small network from its neighbourhood:
 *   features of body p (AM_MLP_FEAT floats), in its body frame: for the 16
 *     nearest other bodies k of its system (by |q_k - q_p| rounded to 1e-8,
 *     ties by lower body index; zeros when fewer), R_p^T (q_k - q_p) / 4 and
 *     the relative quaternion theta_p^* theta_k with s >= 0 (7 floats each);
 *     then q_p,z / 4 (0 in free space), R_p^T f_p, R_p^T tau_p, the
 *     body-frame (u, omega) of the block-diagonal solution P~^-1 b (Sec.
 *     3.1), log(blobs of p) / 5; the far flow R_p^T u_far(q_p) and its
 *     body-frame gradient (central differences of step 0.5 along the body
 *     axes, row-major), u_far being the flow of point forces at the
 *     tracking points of the bodies of the other articulated bodies of the
 *     system within a distance 16 of q_p, each the sum of its blob forces
 *     in P~^-1 b, through the blob
 *     pair tensor (free or wall; FP32 pair terms); zeros;
 *   target (AM_MLP_OUT floats): the background flow of the body, i.e.
 *     u_ext = (M - M~) lambda at its blobs (what the other bodies' forces
 *     induce there; M~ keeps only blob pairs of the same body), fitted in
 *     the body frame by 29 flows on the body-frame offsets rho: e_k,
 *     e_k x rho, E rho for the strains E01, E02, E12, diag(1,-1,0),
 *     diag(1,0,-1), and rho_i rho_j e_c for c = 0..2, (i,j) = 00, 01, 02,
 *     11, 12, 22; ridge 1e-6 tr(B^T B) / 29; 3 zeros;
 *   network: (x - mu) / sd, three ReLU layers of 256, a linear layer to 32,
 *     times sd_out.  Parameters flat in the order W1, b1, ..., W4, b4 (W
 *     row-major, outputs x inputs), AM_MLP_PARAMS floats.
 * Training runs in FP32 on the GPU (mini-batch Adam on the mean squared
 * error of the normalised output); the solver evaluates the network with
 * BF16 operands and FP32 accumulation on the tensor cores.  The guess is the
 * block-diagonal solve with the predicted flow moved to the right-hand side,
 * x0 = P~^-1 (u_s - u_fit, -F, B), which satisfies C U = B. */
#define AM_MLP_FEAT 144
#define AM_MLP_OUT 32
#define AM_MLP_PARAMS 176928
typedef struct am_mlp am_mlp;

/* New network with He-initialised weights from `seed`, zero biases,
 * mu = 0, sd = sd_out = 1; all its work runs on `stream` (cudaStream_t or
 * NULL).  Errors: AM_ERR_ARG, AM_ERR_CUDA. */
AM_API int am_mlp_create(unsigned long long seed, void* stream, am_mlp** out);
AM_API void am_mlp_destroy(am_mlp* m);
AM_API int am_mlp_num_params(void);
/* Parameters to / from host (AM_MLP_PARAMS floats). */
AM_API int am_mlp_get_params(am_mlp* m, float* params);
AM_API int am_mlp_set_params(am_mlp* m, const float* params);
/* Input normalisation mu, sd (AM_MLP_FEAT each, sd > 0) and output scale
 * sd_out (AM_MLP_OUT, > 0). */
AM_API int am_mlp_set_norm(am_mlp* m, const float* mu, const float* sd, const float* sd_out);
/* FP32 loss and its gradient over n samples X (n x FEAT), T (n x OUT):
 * loss = mean over samples and outputs of (y_n - T / sd_out)^2, y_n the
 * network output before the sd_out scale; grad: AM_MLP_PARAMS floats (NULL
 * to skip).  For checking the training kernels. */
AM_API int am_mlp_loss_grad(am_mlp* m, const float* X, const float* T, int n, double* loss,
                            float* grad);
/* `epochs` passes of mini-batch Adam (beta 0.9, 0.999, eps 1e-8, learning
 * rate lr) over n samples, shuffled each epoch from `seed`; *final_loss (or
 * NULL) receives the mean batch loss of the last epoch. */
AM_API int am_mlp_train(am_mlp* m, const float* X, const float* T, int n, int epochs, int batch,
                        double lr, unsigned long long seed, double* final_loss);
/* Predictions Y (n x OUT, scaled by sd_out) of X (n x FEAT): bf16 = 1 the
 * tensor-core path the solver uses, 0 the FP32 training path. */
AM_API int am_mlp_predict(am_mlp* m, const float* X, int n, int bf16, float* Y);
/* Features X (M x FEAT) of all bodies of all systems at the current pose
 * and, when T is not NULL, the targets T (M x OUT) of the solution of the
 * last am_solve (same pose; one FP64 mobility product).  Errors:
 * AM_ERR_ARG (no bodies), AM_ERR_CUDA. */
AM_API int am_learned_features(am_handle* h, float* X, float* T);
/* Use `model` (NULL: none) for the initial guess of cold starts.  check != 0:
 * per system, the point x_pc + beta (x_learned - x_pc) with the smallest
 * residual on that line, beta = -<r_pc, w> / <w, w>, w = r_learned - r_pc
 * (two extra operator products; never a larger residual than P~^-1 b);
 * check == 0: the learned guess itself.  The handle does not own the model;
 * keep it alive while it is set. */
AM_API int am_set_learned(am_handle* h, am_mlp* model, int check);

/* Initial guess of the time-step solves (am_solve_step, both stages of
 * am_solve_step_rk2), which keep the solutions of the last three solves
 * with their times (t, and t + dt/2 for the midpoint stage):
 *   order 0  P~^-1 b (or the learned guess, am_set_learned) every solve;
 *   order 1  the previous solve's solution (the default; Sec. 3.1);
 *   order 2, 3  lambda and U from the polynomial in time through the last
 *            2 or 3 solutions (Lagrange form in their times) evaluated at
 *            the new solve's time, phi from the previous solution (with a
 *            rank-deficient C, phi is determined only modulo null(C^T)):
 *            an extrapolation that is not in the paper.
 * Every guess from the history is projected so that C U = B.  Fewer
 * solutions than the order, two history times closer than 1e-12 (1 + |t|)
 * apart, or a Lagrange weight above 16 in magnitude lower the order for
 * that solve; a solve at the time of the newest entry replaces it; a new
 * layout (am_set_bodies, am_set_constraints with another connectivity)
 * empties the history.  The converged solution does not depend
 * on the order beyond the tolerance; the iteration count does.  am_solve
 * neither reads nor extends the history.  Errors: AM_ERR_ARG (order outside
 * 0..3). */
AM_API int am_set_initial_guess(am_handle* h, int order);

/* Destroy a handle and free its device memory (NULL is a no-op). */
AM_API void am_destroy(am_handle* h);

/* Parameters of a periodic handle's product (after am_set_bodies):
 * params (6): xi (Ewald splitting), r_c (real-space cutoff), beta (shape
 *             of the exponential-of-semicircle window of the grid
 *             transfer, exp(beta (sqrt(1 - z^2) - 1))), hx, hy, hz (grid
 *             spacings);
 * sizes (6):  Mx, My, Mz (grid points per side), w (window width in
 *             points per side), real-space pairs within r_c at the current
 *             pose (the target itself included), cells of the cell list.
 * Either pointer may be NULL.  Errors: AM_ERR_ARG for a handle without a
 * box or without bodies. */
AM_API int am_periodic_info(am_handle* h, double* params, long long* sizes);

/* Message of the last error of h, or of the calling thread's last stateless
 * call when h is NULL; never NULL. */
AM_API const char* am_last_error(const am_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* AM_H */

// Host-side entry points of ops.cu (kernel orchestration for one handle).
#pragma once
#include "am_internal.cuh"

namespace am {

// device error flags (h->d_flags[0])
constexpr int kFlagWall = 1;        // a blob centre at or below height a
constexpr int kFlagSingular = 2;    // a body block of M or N~ not SPD
constexpr int kFlagCorrection = 4;  // correction normal equations not SPD
constexpr int kFlagTensor = 1 << 8; // a tensor-core (tcgen05) wait timed out (tc_gemm.cuh)
// Bound on the relative error of the mixed mobility product, |(M32 - M) l|
// <= kMixedProductError |M32 l| (20 times the largest measured, 4.7e-7 at
// 60,000 wall blobs against FP64): the bound term of the residual update
constexpr double kMixedProductError = 1e-5;

// Arithmetic of a mobility product: the handle's precision, FP64,
// double-float pair terms (rpy_df.cu), or the mixed FP32 pair terms.
constexpr int kOpHandle = 0, kOpFP64 = 1, kOpDF = 2, kOpMixed = 3;

// Geometry of the current pose: blob positions, lab link vectors, B, b.
void launch_geometry(am_handle* h);
// out = A y (Eq. linear_system) with the mobility product of `mode`.
// active: per-system flags (device); systems with flag 0 get a zero
// mobility product without its pair arithmetic (nullptr: all systems)
void op_apply(am_handle* h, const double* y, double* out, int mode, const int* active = nullptr);
// Blob mobility product only: u = M lambda (3Nb).
void mobility_apply(am_handle* h, const double* lam, double* u, int mode);
// Block-diagonal preconditioner (Sec. 3.1): build at the current pose, apply.
void pc_build(am_handle* h);
void pc_apply(am_handle* h, const double* r, double* z);
// Project the U block of x onto C U = B with the preconditioner
// (x += P~^-1 (0, 0, B - C U)).
void project_constraints(am_handle* h, double* x);
// x = sum_{i < k} w[i] v[i] over the first len entries (k <= 3 vectors)
void combine_vectors(am_handle* h, double* x, const double* const* v, const double* w, int k, int len);
// Solve A x = b (d_b, d_x in the handle; d_x holds the initial guess).
// Returns AM_OK or AM_ERR_NOT_CONVERGED; fills iteration fields of st.
int solve(am_handle* h, am_step_stats* st);
// Euler update + reconstruction + correction (Sec. 4.3) from the solution
// in d_x; writes the new q, theta into the handle.
int advance(am_handle* h, double dt, am_step_stats* st);
// Block-diagonal mobility product of all systems (rpy.cu): work items for
// tpt targets per thread and source chunks (0 = automatic), their launch,
// the sum of the partials, and the autotuner that picks (tpt, chunk).
int mobility_layout(am_handle* h, int tpt, int chunk, int tgroup = 0, int sym = 0);
void launch_items(am_handle* h, const double* lam, int mode, const int* active = nullptr);
int df_resident_grid(bool wall);
int sym_df_resident_grid(bool wall);
void launch_items_df(am_handle* h, const double* lam);
void launch_sum_items(am_handle* h, double* u);
int mobility_autotune(am_handle* h);
// Periodic box (periodic.cu): parameters and buffers for the handle's box,
// tolerance and blob count; cell list and real-space pair blocks of the
// current pose (host-synchronising); the product u = M_per lam into d_mv;
// the chosen parameters (xi, r_c, sigma, hx, hy, hz; Mx, My, Mz, P,
// real-space pairs, cells).
int periodic_setup(am_handle* h);
void periodic_free(am_handle* h);
int periodic_bin(am_handle* h);
void launch_periodic(am_handle* h, const double* lam, bool fp32);
void periodic_info(const am_handle* h, double* d6, long long* i6);
// Per system, x <- xp + beta_s (x - xp) with beta_s minimising the
// residual |b - A x| on that line (operator in the handle's precision);
// returns how many systems have beta_s > 0.  Uses d_w, d_rir, d_z, d_part
// and the upper half of d_sysred.
int line_initial(am_handle* h, double* x, const double* xp);
// Learned initial guess (mlp.cu): x = P~^-1 (b - predicted background
// flow), with x_pc = P~^-1 b left in d_dx; uses d_rir.
int learned_x0(am_handle* h, double* x);
// Features (and background-flow targets of the solution in d_x) of all
// bodies to host X, T; uses d_dx and d_w.
int learned_features(am_handle* h, float* X, float* T);
// Steric repulsion (steric.cu): blob forces at the current pose and their
// body sums subtracted from the force rows of d_b; no-op when off.
void steric_apply(am_handle* h);
// Single-blob mode (single_blob.cu): grand mobility product v = N g (6M),
// the right-hand side (N F, B), the operator, the preconditioner.
void sb_mobility(am_handle* h, const double* g, double* v);
void sb_rhs(am_handle* h);
void sb_op_apply(am_handle* h, const double* y, double* out);
void sb_pc_build(am_handle* h);
void sb_pc_apply(am_handle* h, const double* r, double* z);
// phi rows of the preconditioner (precond.cu): z_phi = G~ (r_phi - C U^)
// with U^ in d_pc_Uhat.
void pc_apply_links(am_handle* h, const double* r, double* z);
// Read and clear the device error flags.
int take_flags(am_handle* h);

}  // namespace am

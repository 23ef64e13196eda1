// Internal declarations of libam: handle layout, device helpers, launchers.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "am.h"

namespace am {

constexpr int kTile = 128;        // sources per shared-memory tile
constexpr int kThreads = 128;     // threads per block of the pair kernels
constexpr int kSbChunks = 16;     // most source chunks of the single-blob body mobility
constexpr double kPi = 3.14159265358979323846;

extern std::atomic<long long> g_launches;
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int num_sms();

// Constants of the RPY pair tensors (free space and wall image part).
struct RpyParams {
    double a, a2, four_a2;
    double inv8pieta;     // 1 / (8 pi eta)
    double k_far2;        // inv8pieta * 2 a^2 / 3
    double k_far3;        // inv8pieta * 2 a^2
    double mu0;           // 1 / (6 pi eta a)
    double k_near1;       // 9 / (32 a)
    double k_near2;       // mu0 * 3 / (32 a)
};
RpyParams make_params(double eta, double a);

// Source splitting of the all-pairs product: grid (target blocks, splits).
struct Split { int splits; int chunk; int tpt; };
Split choose_split(int n, int precision);
Split choose_split_rows(int n, int nt, int precision);

// ---- mobility product launchers (rpy.cu) ------------------------------
// FP64: r4 = (x, y, z, 0) per blob.  Mixed: hi/lo float4 positions.
// Writes partial sums part[s][3n] for s < splits.
void launch_rpy_partial_f64_rows(const double4_32a* r4, const double* lam, double* part, int n, int t0, int nt,
                                 const Split& sp, const RpyParams& prm, int wall, cudaStream_t st);
void launch_rpy_partial_mixed_rows(const float4* hi, const float4* lo, const double* lam, double* part, int n,
                                   int t0, int nt, const Split& sp, const RpyParams& prm, int wall,
                                   cudaStream_t st);
void launch_rpy_partial_f64(const double4_32a* r4, const double* lam, double* part,
                            int n, const Split& sp, const RpyParams& prm, int wall,
                            cudaStream_t st);
void launch_rpy_partial_mixed(const float4* hi, const float4* lo, const double* lam,
                              double* part, int n, const Split& sp,
                              const RpyParams& prm, int wall, cudaStream_t st);
void launch_pack_positions(const double* r3, double4_32a* r4, float4* hi, float4* lo,
                           int n, cudaStream_t st);
void launch_sum_partials(const double* part, double* u, int n, int splits,
                         cudaStream_t st);

// Control block of a device-side Arnoldi cycle.
struct ArnoldiCtrl {
    int j;          // current column (number of completed steps when stopped)
    int it;         // steps taken in this cycle
    int budget;     // steps allowed in this cycle
    int m;          // restart length
    int stop;       // set when the cycle ends
    double tol_abs; // stop when the residual estimate is <= tol_abs
};

// One work item of the block-diagonal all-pairs product: targets [t0, t1)
// against sources [j0, j1) of one system, partial sums at pbase.
struct MvItem {
    int t0, t1;       // targets [t0, t1)
    int j0, j1;       // sources [j0, j1)
    int tbase, n3;    // first blob of the system, 3 N_s
    long long pbase;  // poff_s + c * 3 N_s
    int sys, pad;     // system index
};

// One item of the symmetric products: tiles I (targets) and J (sources)
// of T = 32 NSUB blobs of one system with I <= J; the pairs between them are
// evaluated once and give the rows of I (slot J) and the columns of J (slot
// I); the diagonal item (I = J) takes each unordered pair of its tile once
// and writes rows and columns together.
struct SymItem {
    int i0, ni, j0, nj;     // first blob and count of tile I and of tile J
    int tbase, sys;         // first blob of the system, system
    int ti, tj;             // tile indices within the system (partial-sum slots)
    long long poff;         // the system's partial-sum offset
    int n3, pad;            // 3 N_s
};

// ---- device helpers -----------------------------------------------------
// Programmatic dependent launch: a kernel launched by launch_dep may be
// scheduled while its predecessor in the stream drains; it calls dep_wait
// before its first global memory access, which returns once the
// predecessor has completed and its writes are visible (a no-op for a
// kernel launched without the attribute).
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class K, class... Args>
inline cudaError_t launch_dep(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kernel, std::forward<Args>(args)...);
}

// End of a work-queue kernel (counter[0]: next item, counter[1]: blocks
// finished): the last block to finish zeroes both for the next launch.
// Every block has taken its last item before it counts itself finished, so
// no block reads the queue after the reset.
__device__ __forceinline__ void item_queue_done(int* counter) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&counter[1], 1) == (int)gridDim.x - 1) {
            counter[0] = 0;
            counter[1] = 0;
        }
    }
}

// R(theta) v = 2 [ p (p.v) + s (p x v) + (s^2 - 1/2) v ]   (App. B, Eq. rot_mat)
__device__ __forceinline__ void quat_rotate(double s, double px, double py, double pz,
                                            double vx, double vy, double vz,
                                            double& ox, double& oy, double& oz) {
    double pv = px * vx + py * vy + pz * vz;
    double cx = py * vz - pz * vy, cy = pz * vx - px * vz, cz = px * vy - py * vx;
    double c = s * s - 0.5;
    ox = 2.0 * (px * pv + s * cx + c * vx);
    oy = 2.0 * (py * pv + s * cy + c * vy);
    oz = 2.0 * (pz * pv + s * cz + c * vz);
}
// R(theta)^T v (the inverse rotation: p -> -p)
__device__ __forceinline__ void quat_rotate_inv(double s, double px, double py, double pz,
                                                double vx, double vy, double vz,
                                                double& ox, double& oy, double& oz) {
    quat_rotate(s, -px, -py, -pz, vx, vy, vz, ox, oy, oz);
}
// theta_2 . theta_1 (Eq. quaternion_mult)
__device__ __forceinline__ void quat_mul(const double* t2, const double* t1, double* o) {
    double s2 = t2[0], s1 = t1[0];
    o[0] = s2 * s1 - (t2[1] * t1[1] + t2[2] * t1[2] + t2[3] * t1[3]);
    o[1] = s2 * t1[1] + s1 * t2[1] + (t2[2] * t1[3] - t2[3] * t1[2]);
    o[2] = s2 * t1[2] + s1 * t2[2] + (t2[3] * t1[1] - t2[1] * t1[3]);
    o[3] = s2 * t1[3] + s1 * t2[3] + (t2[1] * t1[2] - t2[2] * t1[1]);
}
// theta_gamma = [cos(g/2), sin(g/2) gamma / g]  (Sec. 2.1)
__device__ __forceinline__ void quat_from_rotvec(double gx, double gy, double gz, double* o) {
    double g = sqrt(gx * gx + gy * gy + gz * gz);
    double sg, cg;
    sincos(0.5 * g, &sg, &cg);
    double f = (g > 1e-8) ? sg / g : 0.5 - g * g / 48.0;
    o[0] = cg; o[1] = f * gx; o[2] = f * gy; o[3] = f * gz;
}

}  // namespace am

namespace am {
struct PeriodicPlan;  // periodic.cu
}

// ---- the handle -----------------------------------------------------------
// Host copy of one system (suspension) as last set by the caller; local body
// indices.  The device layout concatenates all systems.
struct am_sys_rec {
    bool has_bodies = false;
    int M = 0, Nb = 0, NA = 0, P = 0;
    std::vector<double> q, theta, rho, F, slip;
    std::vector<int> blob_off, asm_of_body;
    std::vector<int> bp, bq;
    std::vector<double> dlp, dlq, dlpd, dlqd;  // dlpd empty: passive links
};

struct am_handle {
    am_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    am::RpyParams prm{};

    // sizes (all systems together)
    int M = 0, Nb = 0, P = 0, NA = 0, n = 0;
    bool have_bodies = false;

    // systems: host records, layout state and per-system offsets
    int S = 1;
    std::vector<am_sys_rec> sys;
    bool dirty = true;        // records changed since the device layout was built
    bool committed = false;   // a device layout exists
    std::vector<int> sys_body0, sys_blob0, sys_link0, sys_asm0;
    // per-system device data of the batched solve
    int* d_sys_of_elem = nullptr;                 // n: system of each unknown
    int *d_chunk_start = nullptr, *d_chunk_end = nullptr, *d_sys_chunk_off = nullptr;
    int nchunks = 0;
    int* d_sys_of_blob = nullptr;                 // Nb
    int* d_sys_body_off = nullptr;                // S + 1: first body of each system
    int *d_sys_blob0 = nullptr, *d_sys_nb = nullptr, *d_sys_nch = nullptr;
    long long* d_sys_poff = nullptr;
    // batched GMRES scalars (per system)
    double *d_Hs = nullptr, *d_css = nullptr, *d_sns = nullptr, *d_gs = nullptr, *d_coefs = nullptr,
           *d_xis = nullptr, *d_bnorm_s = nullptr, *d_beta_s = nullptr, *d_inv_s = nullptr,
           *d_tol_s = nullptr, *d_sysred = nullptr, *d_hcols = nullptr;
    int *d_active = nullptr, *d_kdone = nullptr;
    int* d_arn_cnt = nullptr;  // S + 1 arrival counts of the fused Arnoldi step kernels
    int* d_pcb_cnt = nullptr;  // M arrival counts of the preconditioner apply (per body)
    int chunk_len = 1024, chunk_threads = 256;  // dot-product chunk length, threads per chunk block
    // all-pairs work items (block-diagonal over systems) and their queue
    void* d_items = nullptr;
    int n_items = 0;
    int* d_item_counter = nullptr;
    int mv_tpt = 1, mv_chunk = 0, mv_tgroup = 0, mv_grid = 0, mv_grid64 = 0, mv_griddf = 0;
    long long mv_part_total = 0;
    bool mv_tuned = false;
    // tile-pair items of the symmetric FP64 product (tiles of 32 sym_nsub blobs)
    void* d_sym_items = nullptr;
    int n_sym = 0, sym_nsub = 0, mv_gridsym = 0, mv_gridsym32 = 0, mv_gridsymdf = 0;

    // host structure
    std::vector<int> blob_off, asm_of_body, bp, bq;
    std::vector<int> asm_body_off, asm_body_idx, asm_link_off, asm_link_idx;
    std::vector<long long> minv_off, G_off, pplus_off, corr_off;
    std::vector<int> G_dim;
    long long minv_total = 0, G_total = 0, pplus_total = 0, corr_total = 0;
    int max_body_blobs = 0;
    int max_asm_links = 0;
    bool active_links = false;
    bool links_connected = true;

    // device: bodies
    double *d_q = nullptr, *d_theta = nullptr, *d_rho = nullptr, *d_F = nullptr,
           *d_slip = nullptr;
    int *d_blob_off = nullptr, *d_body_of_blob = nullptr, *d_asm_of_body = nullptr;
    int *d_asm_body_off = nullptr, *d_asm_body_idx = nullptr;
    double4_32a *d_r4 = nullptr, *d_d4 = nullptr;   // lab positions, R(theta) rho
    float4 *d_rhi = nullptr, *d_rlo = nullptr;  // mixed-precision positions
    double* d_r3 = nullptr;                     // lab positions, 3Nb (get_blobs)

    // device: links
    int *d_bp = nullptr, *d_bq = nullptr;
    double *d_dlp = nullptr, *d_dlq = nullptr, *d_dlpd = nullptr, *d_dlqd = nullptr;
    double *d_dlp1 = nullptr, *d_dlq1 = nullptr;     // link vectors at t + dt
    double *d_lp = nullptr, *d_lq = nullptr, *d_B = nullptr;
    int *d_body_link_off = nullptr, *d_body_link_idx = nullptr;
    int *d_asm_link_off = nullptr, *d_asm_link_idx = nullptr, *d_link_local = nullptr;
    double* d_pplus = nullptr; long long* d_pplus_off = nullptr;
    int* d_body_local = nullptr;

    // device: preconditioner (matrices in FP64, or FP32 when pc32)
    bool pc32 = false;
    void *d_minv = nullptr, *d_pcwork = nullptr, *d_Y = nullptr;
    double* d_Nt = nullptr;
    long long* d_minv_off = nullptr;
    void *d_G = nullptr, *d_Gwork = nullptr;
    int *d_pcw_body = nullptr, *d_pcw_chunk = nullptr, *d_pcw_off = nullptr;
    // body preconditioner build: bodies of <= 64 rows first (n_pcb_small),
    // then the larger ones, built by clusters of pcb_cs CTAs when pcb_cs > 1
    int* d_pcb_list = nullptr;
    int n_pcb_small = 0, pcb_cs = 1;
    // the same for the articulated-body build (by 3 x links rows)
    int* d_pca_list = nullptr;
    int n_pca_small = 0, pca_cs = 1;
    int *d_pca_asm = nullptr, *d_pca_chunk = nullptr;
    int n_pcw = 0, n_pca = 0;
    double* d_ytp = nullptr;
    long long* d_G_off = nullptr; int* d_G_rank = nullptr;
    int* d_perm = nullptr; long long* d_perm_off = nullptr;
    double *d_pc_w = nullptr, *d_pc_Uhat = nullptr;
    bool pc_valid = false;

    // device: solver vectors
    double *d_b = nullptr, *d_x = nullptr, *d_t = nullptr,
           *d_z = nullptr, *d_w = nullptr, *d_V = nullptr, *d_Z = nullptr;
    double *d_Hm = nullptr, *d_cs = nullptr, *d_sn = nullptr, *d_g = nullptr,
           *d_coef = nullptr, *d_part = nullptr, *d_scal = nullptr, *d_xi = nullptr,
           *d_npart = nullptr, *d_rir = nullptr, *d_dx = nullptr;
    int restart = 50;
    int ldv = 0;
    long long pairs = 0;
    // solution history of the time-step solves (most recent: slot hist_head)
    double* d_xhist = nullptr;  // 3 x n
    double t_hist[3] = {0, 0, 0};
    int n_hist = 0, hist_head = 0;
    int guess_order = 1;        // am_set_initial_guess
    double t_solve = 0.0;       // time of the time-step solve being prepared

    // device: mobility partial sums
    double* d_mv = nullptr;
    // periodic box (cfg.box): spectral Ewald plan, real-space pairs of the
    // current pose, status of the last binning
    am::PeriodicPlan* per = nullptr;
    long long per_nnz = 0;
    int per_status = 0;
    am::Split split{1, 0, 1};

    // device: step
    double *d_qnew = nullptr, *d_thnew = nullptr, *d_corr = nullptr, *d_red = nullptr;
    double *d_q0 = nullptr, *d_th0 = nullptr;   // pose at t_k during a midpoint step

    // steric repulsion (am_set_repulsion): parameters and blob forces (3Nb)
    bool steric_on = false;
    bool sb = false;   // single-blob bodies (am_config.single_blob)
    double* d_sbpart = nullptr;   // kSbChunks x 6M partial sums of the body mobility
    double st_eps = 0.0, st_b = 1.0, st_rc = 0.0, st_eps_w = 0.0, st_b_w = 1.0;
    double* d_fst = nullptr;
    double *d_zbuf = nullptr, *d_cbuf = nullptr;
    long long* d_corr_off = nullptr;
    int* d_iters = nullptr;
    int* d_flags = nullptr;

    // host staging (pinned)
    double* h_scal = nullptr;
    int* h_flags = nullptr;
    int* h_iters = nullptr;

    cudaEvent_t ev[8] = {};
    bool geometry_valid = false;

    // device-resident Arnoldi cycle: control block, fixed in/out vectors and
    // one CUDA graph (WHILE node) per operator precision
    am::ArnoldiCtrl* d_ctrl = nullptr;
    am::ArnoldiCtrl* h_ctrl = nullptr;
    double *d_vj = nullptr, *d_zj = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraph_t graph[2] = {nullptr, nullptr};
    long long graph_gen[2] = {-1, -1};
    long long body_launches[2] = {0, 0};
    long long body_pairs[2] = {0, 0};
    long long layout_gen = 0;
    bool graphs_ok = true;

    // learned initial guess of cold starts (am_set_learned; not owned)
    am_mlp* mlp = nullptr;
    bool mlp_check = true;

    // per-launch timing of the all-pairs kernel (am_mobility_timing)
    bool timing = false;
    std::vector<cudaEvent_t> tev;   // start/stop pairs
    size_t tev_used = 0;
};

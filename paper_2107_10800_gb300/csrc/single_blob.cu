// Single-blob bodies with rotational coupling, free space (Sec. 2.4): every
// body is one blob of radius a at its tracking point, the body mobility N is
// the generalised RPY tensor (translation, rotation, and their coupling), and
// the constrained problem is Eq. linear_system_general on y = (U, phi):
//     U - N C^T phi = N F,     C U = B.
// Pair tensor for d = x_i - x_j, r = |d|, e = d / r (equal radii):
//   u_i     += M_tt(d) f_j + c(r) (T_j x e) ... written as -c(r) e x T_j
//   omega_i += -c(r) e x f_j + alpha(r) T_j + beta(r) (e . T_j) e
//   c     = 1 / (8 pi eta r^2)                         r >= 2a
//         = (r / a - 3 r^2 / (8 a^2)) / (16 pi eta a^2) r <  2a
//   alpha = -1 / (16 pi eta r^3),  beta = 3 / (16 pi eta r^3)          r >= 2a
//   alpha = (1 - 27 s / 32 + 5 s^3 / 64) / (8 pi eta a^3),
//   beta  = (9 s / 32 - 3 s^3 / 64) / (8 pi eta a^3),  s = r / a      r <  2a
//   self: mu0 = 1 / (6 pi eta a) for translation, 1 / (8 pi eta a^3) for
//   rotation (the far forms are the vorticity of the regularised Stokeslet
//   and of the rotlet; the overlapping ones are the closed forms for equal
//   spheres of Wajnryb, Mizerski, Zuk and Szymczak 2013).
// Preconditioner: N replaced by its self blocks N~ = diag(mu0 I, mu_r I), so
// phi = G~ (r_phi - C r_U) with G~ = (C N~ C^T)^+ per articulated body (the
// assembly factorisation of precond.cu) and U = r_U + N~ C^T phi.
#include "am_internal.cuh"
#include "ops.cuh"
#include "rpy_pair.cuh"

#include <algorithm>
#include <climits>

namespace am {

namespace {

// N~ of every body: diag(mu0 I3, mu_r I3) as 6 x 6 row-major
__global__ void k_sb_fill_nt(int M, double mu0, double mur, double* __restrict__ Nt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    double* o = Nt + 36 * (size_t)p;
    for (int k = 0; k < 36; ++k) o[k] = 0.0;
    for (int k = 0; k < 3; ++k) { o[7 * k] = mu0; o[7 * (k + 3)] = mur; }
}

// (C^T phi)_p: +phi_n and l_p x phi_n on the link's body p, -phi_n and
// -(l_q x phi_n) on its body q (App. A)
__device__ __forceinline__ void ct_phi_body(int p, const int* __restrict__ blo, const int* __restrict__ bli,
                                            const double* __restrict__ lp, const double* __restrict__ lq,
                                            const double* __restrict__ phi, double* g) {
    for (int k = 0; k < 6; ++k) g[k] = 0.0;
    for (int e = blo[p]; e < blo[p + 1]; ++e) {
        const int code = bli[e], n = code >> 1, side = code & 1;
        const double f0 = phi[3 * (size_t)n], f1 = phi[3 * (size_t)n + 1], f2 = phi[3 * (size_t)n + 2];
        const double* l = side ? lq + 3 * (size_t)n : lp + 3 * (size_t)n;
        const double sg = side ? -1.0 : 1.0;
        g[0] += sg * f0; g[1] += sg * f1; g[2] += sg * f2;
        g[3] += sg * (l[1] * f2 - l[2] * f1);
        g[4] += sg * (l[2] * f0 - l[0] * f2);
        g[5] += sg * (l[0] * f1 - l[1] * f0);
    }
}

__global__ void k_sb_ctphi(int M, const int* __restrict__ blo, const int* __restrict__ bli,
                           const double* __restrict__ lp, const double* __restrict__ lq,
                           const double* __restrict__ phi, double* __restrict__ g) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    double v[6];
    ct_phi_body(p, blo, bli, lp, lq, phi, v);
    for (int k = 0; k < 6; ++k) g[6 * (size_t)p + k] = v[k];
}

// v = N g for all systems (block diagonal): one thread per target body,
// source bodies of the union of the block's systems in shared-memory tiles
__global__ void __launch_bounds__(kThreads)
k_sb_mobility(int M, const double* __restrict__ q, const int* __restrict__ sys_of_U,
              const int* __restrict__ sys_body_off, const double* __restrict__ g, RpyK<double> k, double eta,
              double a, double* __restrict__ v) {
    __shared__ double sx[kTile][3];
    __shared__ double sg[kTile][6];
    __shared__ int s_lo, s_hi;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    const bool live = i < M;
    int j0 = INT_MAX, j1 = 0;
    double xi[3] = {0.0, 0.0, 0.0};
    if (live) {
        const int s = sys_of_U[6 * (size_t)i];
        j0 = sys_body_off[s];
        j1 = sys_body_off[s + 1];
        for (int c = 0; c < 3; ++c) xi[c] = q[3 * (size_t)i + c];
    }
    if (threadIdx.x == 0) { s_lo = INT_MAX; s_hi = 0; }
    __syncthreads();
    if (live) { atomicMin(&s_lo, j0); atomicMax(&s_hi, j1); }
    __syncthreads();
    // this block's share of the sources: chunk blockIdx.y of gridDim.y
    const int span = s_hi - s_lo;
    const int lo_all = s_lo + (int)((long long)span * blockIdx.y / gridDim.y);
    const int hi_all = s_lo + (int)((long long)span * (blockIdx.y + 1) / gridDim.y);
    const double pi = 3.14159265358979323846;
    const double ctr_far = 1.0 / (8.0 * pi * eta);          // c r^2
    const double cnear = 1.0 / (16.0 * pi * eta * a * a);   // c / (s - 3 s^2 / 8)
    const double rr_far = 1.0 / (16.0 * pi * eta);           // |alpha| r^3, beta r^3 / 3
    const double rr_near = 1.0 / (8.0 * pi * eta * a * a * a);
    double ux = 0, uy = 0, uz = 0, wx = 0, wy = 0, wz = 0;  // translational part accumulates u / A1
    for (int jt = lo_all; jt < hi_all; jt += kTile) {
        const int cnt = min(kTile, hi_all - jt);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int j = jt + threadIdx.x;
            for (int c = 0; c < 3; ++c) sx[threadIdx.x][c] = q[3 * (size_t)j + c];
            for (int c = 0; c < 6; ++c) sg[threadIdx.x][c] = g[6 * (size_t)j + c];
        }
        __syncthreads();
        if (!live) continue;
        for (int t = 0; t < cnt; ++t) {
            const int j = jt + t;
            if (j < j0 || j >= j1) continue;
            const double f0 = sg[t][0], f1 = sg[t][1], f2 = sg[t][2];
            const double T0 = sg[t][3], T1 = sg[t][4], T2 = sg[t][5];
            const double dx = xi[0] - sx[t][0], dy = xi[1] - sx[t][1], dz = xi[2] - sx[t][2];
            // translation from force (RPY, self included at r = 0)
            pair_free<double>(dx, dy, dz, f0, f1, f2, k, ux, uy, uz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) {  // self rotation
                wx += rr_near * T0; wy += rr_near * T1; wz += rr_near * T2;
                continue;
            }
            const double r = sqrt(r2), ri = 1.0 / r;
            const double ex = dx * ri, ey = dy * ri, ez = dz * ri;
            double c, al, be;
            if (r >= 2.0 * a) {
                c = ctr_far * ri * ri;
                const double r3 = ri * ri * ri;
                al = -rr_far * r3;
                be = 3.0 * rr_far * r3;
            } else {
                const double sv = r / a;
                c = cnear * (sv - 0.375 * sv * sv);
                al = rr_near * (1.0 - 27.0 / 32.0 * sv + 5.0 / 64.0 * sv * sv * sv);
                be = rr_near * (9.0 / 32.0 * sv - 3.0 / 64.0 * sv * sv * sv);
            }
            // u_i += -c e x T_j  (translation from torque), divided by A1 to
            // share the accumulator of the RPY part
            const double cA = c / k.A1;
            ux -= cA * (ey * T2 - ez * T1);
            uy -= cA * (ez * T0 - ex * T2);
            uz -= cA * (ex * T1 - ey * T0);
            // omega_i += -c e x f_j + alpha T_j + beta (e . T_j) e
            const double eT = ex * T0 + ey * T1 + ez * T2;
            wx += -c * (ey * f2 - ez * f1) + al * T0 + be * eT * ex;
            wy += -c * (ez * f0 - ex * f2) + al * T1 + be * eT * ey;
            wz += -c * (ex * f1 - ey * f0) + al * T2 + be * eT * ez;
        }
    }
    if (!live) return;
    double* o = v + 6 * ((size_t)blockIdx.y * M + i);  // partial sums of chunk blockIdx.y
    o[0] = k.A1 * ux; o[1] = k.A1 * uy; o[2] = k.A1 * uz;
    o[3] = wx; o[4] = wy; o[5] = wz;
}

// v = sum over the nc chunks of the partial sums (fixed order)
__global__ void k_sb_sum(int n6, int nc, const double* __restrict__ part, double* __restrict__ v) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n6) return;
    double a = 0.0;
    for (int c = 0; c < nc; ++c) a += part[(size_t)c * n6 + t];
    v[t] = a;
}

// out_U = U - v (v = N C^T phi); out_phi = C U
__global__ void k_sb_epilogue(int M, int P, const double* __restrict__ y, const double* __restrict__ v,
                              const int* __restrict__ bp, const int* __restrict__ bq,
                              const double* __restrict__ lp, const double* __restrict__ lq,
                              double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 6 * M) {
        out[t] = y[t] - v[t];
        return;
    }
    const int n = t - 6 * M;
    if (n >= P) return;
    const double* Up = y + 6 * (size_t)bp[n];
    const double* Uq = y + 6 * (size_t)bq[n];
    const double* l1 = lp + 3 * (size_t)n;
    const double* l2 = lq + 3 * (size_t)n;
    // u_p - l_p x omega_p - u_q + l_q x omega_q
    double* o = out + 6 * (size_t)M + 3 * (size_t)n;
    o[0] = Up[0] - (l1[1] * Up[5] - l1[2] * Up[4]) - Uq[0] + (l2[1] * Uq[5] - l2[2] * Uq[4]);
    o[1] = Up[1] - (l1[2] * Up[3] - l1[0] * Up[5]) - Uq[1] + (l2[2] * Uq[3] - l2[0] * Uq[5]);
    o[2] = Up[2] - (l1[0] * Up[4] - l1[1] * Up[3]) - Uq[2] + (l2[0] * Uq[4] - l2[1] * Uq[3]);
}

// z_U = r_U + N~ C^T phi (phi already in z)
__global__ void k_sb_ap3(int M, const int* __restrict__ blo, const int* __restrict__ bli,
                         const double* __restrict__ lp, const double* __restrict__ lq, double mu0, double mur,
                         const double* __restrict__ r, double* __restrict__ z) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    double g[6];
    ct_phi_body(p, blo, bli, lp, lq, z + 6 * (size_t)M, g);
    for (int k2 = 0; k2 < 6; ++k2) {
        const double s = k2 < 3 ? mu0 : mur;
        z[6 * (size_t)p + k2] = r[6 * (size_t)p + k2] + s * g[k2];
    }
}

inline int nb(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

static double sb_mu0(const am_handle* h) { return 1.0 / (6.0 * 3.14159265358979323846 * h->cfg.eta * h->cfg.blob_radius); }
static double sb_mur(const am_handle* h) {
    const double a = h->cfg.blob_radius;
    return 1.0 / (8.0 * 3.14159265358979323846 * h->cfg.eta * a * a * a);
}

void sb_mobility(am_handle* h, const double* g, double* v) {
    // source chunks so that the grid has about 4 blocks per SM (at most
    // kSbChunks; the partial sums live in d_sbpart)
    const int tb = nb(h->M, kThreads);
    const int nc = std::max(1, std::min(kSbChunks, (4 * num_sms() + tb - 1) / tb));
    dim3 grid(tb, nc);
    k_sb_mobility<<<grid, kThreads, 0, h->stream>>>(
        h->M, h->d_q, h->d_sys_of_elem, h->d_sys_body_off, g, rpy_consts<double>(h->prm), h->cfg.eta,
        h->cfg.blob_radius, h->d_sbpart);
    k_sb_sum<<<nb(6LL * h->M, 256), 256, 0, h->stream>>>(6 * h->M, nc, h->d_sbpart, v);
    count_launch(2);
    long long pairs = 0;
    for (const auto& r : h->sys) pairs += (long long)r.M * r.M;
    h->pairs += pairs;
}

void sb_rhs(am_handle* h) {
    // b_U = N F (b_phi = B is already in place)
    sb_mobility(h, h->d_F, h->d_b);
}

void sb_op_apply(am_handle* h, const double* y, double* out) {
    cudaStream_t s = h->stream;
    const int M = h->M, P = h->P;
    if (P) {
        k_sb_ctphi<<<nb(M, 128), 128, 0, s>>>(M, h->d_body_link_off, h->d_body_link_idx, h->d_lp, h->d_lq,
                                              y + 6 * (size_t)M, h->d_pc_Uhat);
        count_launch();
        sb_mobility(h, h->d_pc_Uhat, h->d_dx);
    } else {
        cudaMemsetAsync(h->d_dx, 0, 6 * (size_t)M * sizeof(double), s);
    }
    k_sb_epilogue<<<nb(6LL * M + P, 256), 256, 0, s>>>(M, P, y, h->d_dx, h->d_bp, h->d_bq, h->d_lp, h->d_lq, out);
    count_launch();
}

void sb_pc_build(am_handle* h) {
    k_sb_fill_nt<<<nb(h->M, 128), 128, 0, h->stream>>>(h->M, sb_mu0(h), sb_mur(h), h->d_Nt);
    count_launch();
}

void sb_pc_apply(am_handle* h, const double* r, double* z) {
    cudaStream_t s = h->stream;
    const int M = h->M;
    // U^ = r_U
    cudaMemcpyAsync(h->d_pc_Uhat, r, 6 * (size_t)M * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (h->P) {
        pc_apply_links(h, r, z);  // phi = G~ (r_phi - C U^) into z
        k_sb_ap3<<<nb(M, 128), 128, 0, s>>>(M, h->d_body_link_off, h->d_body_link_idx, h->d_lp, h->d_lq,
                                            sb_mu0(h), sb_mur(h), r, z);
        count_launch();
    } else {
        cudaMemcpyAsync(z, r, 6 * (size_t)M * sizeof(double), cudaMemcpyDeviceToDevice, s);
    }
}

}  // namespace am

// O(N) kernels of the solve: pose, links, the fused part of the operator
// apply, the block-diagonal preconditioner (build and apply), GMRES vector
// kernels, and the Euler update with reconstruction and correction.
#include "am_internal.cuh"
#include "dev_util.cuh"
#include "ops.cuh"
#include "rpy_pair.cuh"

#include <algorithm>

namespace am {

// ------------------------------------------------------- pose, links ---
// r_i = q_p + R(theta_p) rho_i  (Sec. 2.3)
__global__ void k_pose(int Nb, const int* __restrict__ body_of_blob, const double* __restrict__ q,
                       const double* __restrict__ th, const double* __restrict__ rho,
                       double4_32a* __restrict__ r4, double4_32a* __restrict__ d4,
                       float4* __restrict__ hi, float4* __restrict__ lo, double* __restrict__ r3,
                       double a, int wall, int* flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const int p = body_of_blob[i];
    double dx, dy, dz;
    quat_rotate(th[4 * p], th[4 * p + 1], th[4 * p + 2], th[4 * p + 3],
                rho[3 * (size_t)i], rho[3 * (size_t)i + 1], rho[3 * (size_t)i + 2], dx, dy, dz);
    const double x = q[3 * p] + dx, y = q[3 * p + 1] + dy, z = q[3 * p + 2] + dz;
    r4[i] = make_double4_32a(x, y, z, 0.0);
    d4[i] = make_double4_32a(dx, dy, dz, 0.0);
    r3[3 * (size_t)i] = x; r3[3 * (size_t)i + 1] = y; r3[3 * (size_t)i + 2] = z;
    const float hx = (float)x, hy = (float)y, hz = (float)z;
    hi[i] = make_float4(hx, hy, hz, 0.f);
    lo[i] = make_float4((float)(x - hx), (float)(y - hy), (float)(z - hz), 0.f);
    if (wall && !(z > a)) atomicOr(flags, kFlagWall);
}

// l_np = R_p dl_np, l_nq = R_q dl_nq; B_n = R_q d(dl_nq)/dt - R_p d(dl_np)/dt (Eq. dg)
__global__ void k_links(int P, const int* __restrict__ bp, const int* __restrict__ bq,
                        const double* __restrict__ th, const double* __restrict__ dlp,
                        const double* __restrict__ dlq, const double* __restrict__ dlpd,
                        const double* __restrict__ dlqd, double* __restrict__ lp,
                        double* __restrict__ lq, double* __restrict__ B) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= P) return;
    const int p = bp[n], q = bq[n];
    const double* tp = th + 4 * p;
    const double* tq = th + 4 * q;
    double x, y, z;
    quat_rotate(tp[0], tp[1], tp[2], tp[3], dlp[3 * n], dlp[3 * n + 1], dlp[3 * n + 2], x, y, z);
    lp[3 * n] = x; lp[3 * n + 1] = y; lp[3 * n + 2] = z;
    quat_rotate(tq[0], tq[1], tq[2], tq[3], dlq[3 * n], dlq[3 * n + 1], dlq[3 * n + 2], x, y, z);
    lq[3 * n] = x; lq[3 * n + 1] = y; lq[3 * n + 2] = z;
    double bx = 0.0, by = 0.0, bz = 0.0;
    if (dlpd) {
        double ax, ay, az;
        quat_rotate(tq[0], tq[1], tq[2], tq[3], dlqd[3 * n], dlqd[3 * n + 1], dlqd[3 * n + 2], bx, by, bz);
        quat_rotate(tp[0], tp[1], tp[2], tp[3], dlpd[3 * n], dlpd[3 * n + 1], dlpd[3 * n + 2], ax, ay, az);
        bx -= ax; by -= ay; bz -= az;
    }
    B[3 * n] = bx; B[3 * n + 1] = by; B[3 * n + 2] = bz;
}

// b = (u_s, -F, B)  (Eq. linear_system)
__global__ void k_rhs(int Nb, int M, int P, const double* __restrict__ slip,
                      const double* __restrict__ F, const double* __restrict__ B,
                      double* __restrict__ b) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = 3 * Nb, nu = 6 * M;
    if (k < nl) b[k] = slip ? slip[k] : 0.0;
    else if (k < nl + nu) b[k] = -F[k - nl];
    else if (k < nl + nu + 3 * P) b[k] = B[k - nl - nu];
}

// --------------------------------------------------- operator epilogue ---
// out_lambda = M lambda - K U   (sum of the mobility partials, minus the
//                                 rigid velocity u_p + omega_p x (r_i - q_p))
// out_U      = -K^T lambda + C^T phi
// out_phi    = C U   (per link: u_p + omega_p x l_np - u_q - omega_q x l_nq)
__global__ void k_op_epilogue(int Nb, int M, int P, int nblob_blocks, int nbody_blocks,
                              const double* __restrict__ part, const int* __restrict__ sys_of_blob,
                              const int* __restrict__ sys_blob0, const int* __restrict__ sys_nb,
                              const int* __restrict__ sys_nch, const long long* __restrict__ sys_poff,
                              const double* __restrict__ y, double* __restrict__ out,
                              const int* __restrict__ body_of_blob, const int* __restrict__ blob_off,
                              const double4_32a* __restrict__ d4, const int* __restrict__ bl_off,
                              const int* __restrict__ bl_idx, const double* __restrict__ lp,
                              const double* __restrict__ lq, const int* __restrict__ bp,
                              const int* __restrict__ bq) {
    dep_wait();
    const double* lam = y;
    const double* U = y + 3 * (size_t)Nb;
    const double* phi = U + 6 * (size_t)M;
    double* oU = out + 3 * (size_t)Nb;
    double* of = oU + 6 * (size_t)M;
    const int b = blockIdx.x;
    if (b < nblob_blocks) {
        const int i = b * blockDim.x + threadIdx.x;
        if (i >= Nb) return;
        const int sy = sys_of_blob[i];
        const size_t n3 = 3 * (size_t)sys_nb[sy];
        const double* pb = part + sys_poff[sy] + 3 * (size_t)(i - sys_blob0[sy]);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int t = 0; t < sys_nch[sy]; ++t) {
            const double* pp = pb + t * n3;
            s0 += pp[0]; s1 += pp[1]; s2 += pp[2];
        }
        const int p = body_of_blob[i];
        const double4_32a d = d4[i];
        const double* u = U + 6 * p;
        // u + omega x d
        const double k0 = u[0] + (u[4] * d.z - u[5] * d.y);
        const double k1 = u[1] + (u[5] * d.x - u[3] * d.z);
        const double k2 = u[2] + (u[3] * d.y - u[4] * d.x);
        out[3 * (size_t)i] = s0 - k0;
        out[3 * (size_t)i + 1] = s1 - k1;
        out[3 * (size_t)i + 2] = s2 - k2;
    } else if (b < nblob_blocks + nbody_blocks) {
        const int wpb = blockDim.x >> 5;
        const int p = (b - nblob_blocks) * wpb + (threadIdx.x >> 5);
        const int lane = threadIdx.x & 31;
        if (p >= M) return;
        double f0 = 0, f1 = 0, f2 = 0, t0 = 0, t1 = 0, t2 = 0;
        for (int i = blob_off[p] + lane; i < blob_off[p + 1]; i += 32) {
            const double4_32a d = d4[i];
            const double l0 = lam[3 * (size_t)i], l1 = lam[3 * (size_t)i + 1], l2 = lam[3 * (size_t)i + 2];
            f0 += l0; f1 += l1; f2 += l2;
            t0 += d.y * l2 - d.z * l1;
            t1 += d.z * l0 - d.x * l2;
            t2 += d.x * l1 - d.y * l0;
        }
        f0 = warp_sum(f0); f1 = warp_sum(f1); f2 = warp_sum(f2);
        t0 = warp_sum(t0); t1 = warp_sum(t1); t2 = warp_sum(t2);
        if (lane == 0) {
            double c[6] = {0, 0, 0, 0, 0, 0};
            for (int k = bl_off[p]; k < bl_off[p + 1]; ++k) {
                const int e = bl_idx[k];
                const int n = e >> 1;
                const double sg = (e & 1) ? -1.0 : 1.0;
                const double* l = (e & 1) ? lq + 3 * n : lp + 3 * n;
                const double* ph = phi + 3 * n;
                double tq[3];
                cross3(l, ph, tq);
                for (int a = 0; a < 3; ++a) { c[a] += sg * ph[a]; c[3 + a] += sg * tq[a]; }
            }
            double* o = oU + 6 * p;
            o[0] = c[0] - f0; o[1] = c[1] - f1; o[2] = c[2] - f2;
            o[3] = c[3] - t0; o[4] = c[4] - t1; o[5] = c[5] - t2;
        }
    } else {
        const int n = (b - nblob_blocks - nbody_blocks) * blockDim.x + threadIdx.x;
        if (n >= P) return;
        const double* up = U + 6 * bp[n];
        const double* uq = U + 6 * bq[n];
        double wp[3], wq[3];
        cross3(up + 3, lp + 3 * n, wp);
        cross3(uq + 3, lq + 3 * n, wq);
        for (int a = 0; a < 3; ++a) of[3 * n + a] = up[a] + wp[a] - uq[a] - wq[a];
    }
}

// --------------------------------------------------------- GMRES kernels ---
__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, int n, double a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], y[i]);
}

// zero the lambda and U blocks and put B - C U0 in the phi block: the
// right-hand side whose preconditioned solution projects U0 onto C U = B.
__global__ void k_proj_rhs(int Nb, int M, int P, const int* __restrict__ bp,
                           const int* __restrict__ bq, const double* __restrict__ lp,
                           const double* __restrict__ lq, const double* __restrict__ B,
                           const double* __restrict__ x, double* __restrict__ t) {
    const int nl = 3 * Nb, nu = 6 * M;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nl + nu) { t[k] = 0.0; return; }
    const int n = k - nl - nu;
    if (n >= P) return;
    const double* U = x + nl;
    const double* up = U + 6 * bp[n];
    const double* uq = U + 6 * bq[n];
    double wp[3], wq[3];
    cross3(up + 3, lp + 3 * n, wp);
    cross3(uq + 3, lq + 3 * n, wq);
    for (int a = 0; a < 3; ++a) t[nl + nu + 3 * n + a] = B[3 * n + a] - (up[a] + wp[a] - uq[a] - wq[a]);
}

// max_n |(C U - B)_n| into scal[slot] (single block)
__global__ void k_constraint_residual(int Nb, int M, int P, const int* __restrict__ bp,
                                      const int* __restrict__ bq, const double* __restrict__ lp,
                                      const double* __restrict__ lq, const double* __restrict__ B,
                                      const double* __restrict__ x, double* __restrict__ scal,
                                      int slot) {
    __shared__ double sh[256];
    const double* U = x + 3 * (size_t)Nb;
    double mx = 0.0;
    for (int n = threadIdx.x; n < P; n += blockDim.x) {
        const double* up = U + 6 * bp[n];
        const double* uq = U + 6 * bq[n];
        double wp[3], wq[3];
        cross3(up + 3, lp + 3 * n, wp);
        cross3(uq + 3, lq + 3 * n, wq);
        for (int a = 0; a < 3; ++a) mx = fmax(mx, fabs(up[a] + wp[a] - uq[a] - wq[a] - B[3 * n + a]));
    }
    sh[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[slot] = sh[0];
}

// ------------------------------------------------ Euler + reconstruction ---
// Per articulated body a (one block), Sec. 4.3 steps 2-5:
//   u_COM = mean_p u_p; q_COM* = mean_p q_p + dt u_COM;
//   theta*_p = theta_{omega_p dt} . theta_p;
//   z_n = R(theta*_p) dl_np(t+dt) - R(theta*_q) dl_nq(t+dt);
//   q*_p = -((P^a)^+ z)_p + q_COM*;  g2 += |g_n(q*, theta*)|^2.
__global__ void __launch_bounds__(128)
k_euler_reconstruct(const int* __restrict__ asm_body_off, const int* __restrict__ asm_body_idx,
                    const int* __restrict__ asm_link_off, const int* __restrict__ asm_link_idx,
                    const int* __restrict__ bp, const int* __restrict__ bq,
                    const double* __restrict__ U, const double* __restrict__ q,
                    const double* __restrict__ th, const double* __restrict__ dlp1,
                    const double* __restrict__ dlq1, const double* __restrict__ pplus,
                    const long long* __restrict__ pplus_off, double dt,
                    double* __restrict__ qnew, double* __restrict__ thnew,
                    double* __restrict__ zbuf, double* __restrict__ g2acc) {
    __shared__ double sh[64];
    const int a = blockIdx.x;
    const int B0 = asm_body_off[a], Ma = asm_body_off[a + 1] - B0;
    const int L0 = asm_link_off[a], Pa = asm_link_off[a + 1] - L0;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < Ma; k += blockDim.x) {
        const int p = asm_body_idx[B0 + k];
        for (int x = 0; x < 3; ++x) { acc[x] += U[6 * (size_t)p + x]; acc[3 + x] += q[3 * p + x]; }
        double gq[4];
        quat_from_rotvec(U[6 * (size_t)p + 3] * dt, U[6 * (size_t)p + 4] * dt, U[6 * (size_t)p + 5] * dt, gq);
        quat_mul(gq, th + 4 * p, thnew + 4 * p);
    }
    double com[3];
    for (int x = 0; x < 3; ++x) {
        const double su = block_sum(acc[x], sh);
        const double sq = block_sum(acc[3 + x], sh);
        com[x] = sq / Ma + dt * (su / Ma);
    }
    // block_sum synchronises, so thnew is visible to the whole block here
    double* z = zbuf + 3 * (size_t)L0;
    for (int k = threadIdx.x; k < Pa; k += blockDim.x) {
        const int n = asm_link_idx[L0 + k];
        const double* tp = thnew + 4 * bp[n];
        const double* tq = thnew + 4 * bq[n];
        double ax, ay, az, bx, by, bz;
        quat_rotate(tp[0], tp[1], tp[2], tp[3], dlp1[3 * n], dlp1[3 * n + 1], dlp1[3 * n + 2], ax, ay, az);
        quat_rotate(tq[0], tq[1], tq[2], tq[3], dlq1[3 * n], dlq1[3 * n + 1], dlq1[3 * n + 2], bx, by, bz);
        z[3 * k] = ax - bx; z[3 * k + 1] = ay - by; z[3 * k + 2] = az - bz;
    }
    __syncthreads();
    const double* Pp = pplus + pplus_off[a];
    for (int k = threadIdx.x; k < Ma; k += blockDim.x) {
        const int p = asm_body_idx[B0 + k];
        double s[3] = {0, 0, 0};
        for (int l = 0; l < Pa; ++l) {
            const double c = Pp[(size_t)k * Pa + l];
            for (int x = 0; x < 3; ++x) s[x] = fma(c, z[3 * l + x], s[x]);
        }
        for (int x = 0; x < 3; ++x) qnew[3 * p + x] = com[x] - s[x];
    }
    __syncthreads();
    double gg = 0.0;
    for (int k = threadIdx.x; k < Pa; k += blockDim.x) {
        const int n = asm_link_idx[L0 + k];
        for (int x = 0; x < 3; ++x) {
            const double gx = qnew[3 * bp[n] + x] - qnew[3 * bq[n] + x] + z[3 * k + x];
            gg = fma(gx, gx, gg);
        }
    }
    gg = block_sum(gg, sh);
    if (threadIdx.x == 0 && Pa > 0) atomicAdd(g2acc, gg);
}

// d/d(dth) of R(dth) v, dth = [s, p] (from Eq. rot_mat):
//   column s:   4 s v + 2 p x v
//   column p_l: 2 delta_il (p.v) + 2 p_i v_l + 2 s eps_ilk v_k
__device__ __forceinline__ void d_rot_apply(const double* dth, const double* v, double* D /*3x4*/) {
    const double s = dth[0];
    const double p[3] = {dth[1], dth[2], dth[3]};
    double pxv[3];
    cross3(p, v, pxv);
    const double pv = p[0] * v[0] + p[1] * v[1] + p[2] * v[2];
    for (int i = 0; i < 3; ++i) D[i * 4] = 4.0 * s * v[i] + 2.0 * pxv[i];
    // eps_ilk v_k as a matrix E[i][l]: E = -[v]^x
    const double E[9] = {0.0, v[2], -v[1], -v[2], 0.0, v[0], v[1], -v[0], 0.0};
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l)
            D[i * 4 + 1 + l] = 2.0 * ((i == l) ? pv : 0.0) + 2.0 * p[i] * v[l] + 2.0 * s * E[i * 3 + l];
}

// Correction (Sec. 4.2): per articulated body, Gauss-Newton on the residual
// [g_n(dq, dth) (Eq. residual); |dth_p|^2 - 1] from dq = 0, dth = [1,0,0,0],
// until its squared norm is below delta^2.  Each step solves the normal
// equations (J^T J + mu I) step = -J^T r with mu = 1e-10 max diag(J^T J),
// which gives the minimum-norm least-squares step to high relative accuracy
// (the residual is invariant under rigid motions of the whole articulated
// body, so J^T J is singular).  Runs only if the global ||g*||^2 >= delta.
__global__ void __launch_bounds__(256)
k_correct(const int* __restrict__ asm_body_off, const int* __restrict__ asm_body_idx,
          const int* __restrict__ asm_link_off, const int* __restrict__ asm_link_idx,
          const int* __restrict__ bp, const int* __restrict__ bq, const int* __restrict__ body_local,
          const int* __restrict__ link_local, const int* __restrict__ bl_off,
          const int* __restrict__ bl_idx,
          const double* __restrict__ dlp1, const double* __restrict__ dlq1,
          double* __restrict__ qnew, double* __restrict__ thnew, const double* __restrict__ g2acc,
          double delta, int max_iter, double* __restrict__ ws, const long long* __restrict__ ws_off,
          int* __restrict__ iters_out, int* flags) {
    __shared__ double sh[64];
    __shared__ double smax[8];
    const int a = blockIdx.x;
    const int B0 = asm_body_off[a], Ma = asm_body_off[a + 1] - B0;
    const int L0 = asm_link_off[a], Pa = asm_link_off[a + 1] - L0;
    if (threadIdx.x == 0) iters_out[a] = 0;
    if (Pa == 0 || !(*g2acc >= delta)) return;
    const int nd = 7 * Ma;
    double* x = ws + ws_off[a];
    double* N = x + nd;
    double* rhs = N + (size_t)nd * nd;
    double* ltp = rhs + nd;
    double* ltq = ltp + 3 * Pa;
    double* g = ltq + 3 * Pa;
    double* yv = g + 3 * Pa;
    for (int k = threadIdx.x; k < Pa; k += blockDim.x) {
        const int n = asm_link_idx[L0 + k];
        const double* tp = thnew + 4 * bp[n];
        const double* tq = thnew + 4 * bq[n];
        quat_rotate(tp[0], tp[1], tp[2], tp[3], dlp1[3 * n], dlp1[3 * n + 1], dlp1[3 * n + 2],
                    ltp[3 * k], ltp[3 * k + 1], ltp[3 * k + 2]);
        quat_rotate(tq[0], tq[1], tq[2], tq[3], dlq1[3 * n], dlq1[3 * n + 1], dlq1[3 * n + 2],
                    ltq[3 * k], ltq[3 * k + 1], ltq[3 * k + 2]);
    }
    for (int k = threadIdx.x; k < nd; k += blockDim.x) x[k] = ((k % 7) == 3) ? 1.0 : 0.0;
    __syncthreads();
    int it = 0;
    while (true) {
        // residual
        double rr = 0.0;
        for (int k = threadIdx.x; k < Pa; k += blockDim.x) {
            const int n = asm_link_idx[L0 + k];
            const int lp_ = body_local[bp[n]], lq_ = body_local[bq[n]];
            const double* xp = x + 7 * lp_;
            const double* xq = x + 7 * lq_;
            double ap[3], aq[3];
            quat_rotate(xp[3], xp[4], xp[5], xp[6], ltp[3 * k], ltp[3 * k + 1], ltp[3 * k + 2], ap[0], ap[1], ap[2]);
            quat_rotate(xq[3], xq[4], xq[5], xq[6], ltq[3 * k], ltq[3 * k + 1], ltq[3 * k + 2], aq[0], aq[1], aq[2]);
            for (int c = 0; c < 3; ++c) {
                const double v = qnew[3 * bp[n] + c] + xp[c] + ap[c] - qnew[3 * bq[n] + c] - xq[c] - aq[c];
                g[3 * k + c] = v;
                rr = fma(v, v, rr);
            }
        }
        for (int k = threadIdx.x; k < Ma; k += blockDim.x) {
            const double* xb = x + 7 * k;
            const double u = xb[3] * xb[3] + xb[4] * xb[4] + xb[5] * xb[5] + xb[6] * xb[6] - 1.0;
            rr = fma(u, u, rr);
        }
        rr = block_sum(rr, sh);
        if (rr < delta * delta || it >= max_iter) break;
        // normal equations, one block row per body (deterministic)
        for (int k = threadIdx.x; k < Ma; k += blockDim.x) {
            const int p = asm_body_idx[B0 + k];
            double* Nrow = N + (size_t)(7 * k) * nd;
            for (int e = 0; e < 7 * nd; ++e) Nrow[e] = 0.0;
            double rh[7] = {0, 0, 0, 0, 0, 0, 0};
            const double* xb = x + 7 * k;
            for (int e = bl_off[p]; e < bl_off[p + 1]; ++e) {
                const int code = bl_idx[e];
                const int n = code >> 1;
                const int side = code & 1;
                const int loc = link_local[n];  // position of link n in its assembly
                const double sg = side ? -1.0 : 1.0;
                const int other = body_local[side ? bp[n] : bq[n]];
                const double* xo = x + 7 * other;
                double Dm[12], Do[12];
                d_rot_apply(xb + 3, side ? ltq + 3 * loc : ltp + 3 * loc, Dm);
                d_rot_apply(xo + 3, side ? ltp + 3 * loc : ltq + 3 * loc, Do);
                // J rows of link n: this body sg [I, Dm], other body -sg [I, Do]
                double Jm[21], Jo[21];
                for (int r = 0; r < 3; ++r) {
                    for (int c = 0; c < 3; ++c) {
                        Jm[r * 7 + c] = sg * (r == c ? 1.0 : 0.0);
                        Jo[r * 7 + c] = -sg * (r == c ? 1.0 : 0.0);
                    }
                    for (int c = 0; c < 4; ++c) {
                        Jm[r * 7 + 3 + c] = sg * Dm[r * 4 + c];
                        Jo[r * 7 + 3 + c] = -sg * Do[r * 4 + c];
                    }
                }
                for (int i = 0; i < 7; ++i) {
                    for (int j = 0; j < 7; ++j) {
                        double smm = 0.0, smo = 0.0;
                        for (int r = 0; r < 3; ++r) {
                            smm += Jm[r * 7 + i] * Jm[r * 7 + j];
                            smo += Jm[r * 7 + i] * Jo[r * 7 + j];
                        }
                        Nrow[(size_t)i * nd + 7 * k + j] += smm;
                        Nrow[(size_t)i * nd + 7 * other + j] += smo;
                    }
                    double sr = 0.0;
                    for (int r = 0; r < 3; ++r) sr += Jm[r * 7 + i] * g[3 * loc + r];
                    rh[i] += sr;
                }
            }
            // unit-norm row: 2 dth^T on the quaternion columns
            const double u = xb[3] * xb[3] + xb[4] * xb[4] + xb[5] * xb[5] + xb[6] * xb[6] - 1.0;
            for (int i = 0; i < 4; ++i) {
                for (int j = 0; j < 4; ++j) Nrow[(size_t)(3 + i) * nd + 7 * k + 3 + j] += 4.0 * xb[3 + i] * xb[3 + j];
                rh[3 + i] += 2.0 * xb[3 + i] * u;
            }
            for (int i = 0; i < 7; ++i) rhs[7 * k + i] = -rh[i];
        }
        __syncthreads();
        double dm = 0.0;
        for (int k = threadIdx.x; k < nd; k += blockDim.x) dm = fmax(dm, N[(size_t)k * nd + k]);
        // max over the block
        {
            double v = dm;
            for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
            if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double mm = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, smax[w]);
                sh[48] = mm;
            }
            __syncthreads();
        }
        const double mu = 1e-10 * sh[48];
        for (int k = threadIdx.x; k < nd; k += blockDim.x) N[(size_t)k * nd + k] += mu;
        __syncthreads();
        if (!block_cholesky(N, nd, sh)) {
            if (threadIdx.x == 0) atomicOr(flags, kFlagCorrection);
            break;
        }
        // solve L L^T step = rhs (one warp, row by row)
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            for (int i = 0; i < nd; ++i) {
                double s = 0.0;
                for (int k = lane; k < i; k += 32) s = fma(N[(size_t)i * nd + k], yv[k], s);
                s = warp_sum(s);
                if (lane == 0) yv[i] = (rhs[i] - s) / N[(size_t)i * nd + i];
                __syncwarp();
            }
            for (int i = nd - 1; i >= 0; --i) {
                double s = 0.0;
                for (int k = i + 1 + lane; k < nd; k += 32) s = fma(N[(size_t)k * nd + i], yv[k], s);
                s = warp_sum(s);
                if (lane == 0) yv[i] = (yv[i] - s) / N[(size_t)i * nd + i];
                __syncwarp();
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nd; k += blockDim.x) x[k] += yv[k];
        __syncthreads();
        ++it;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < Ma; k += blockDim.x) {
        const int p = asm_body_idx[B0 + k];
        const double* xb = x + 7 * k;
        for (int c = 0; c < 3; ++c) qnew[3 * p + c] += xb[c];
        double o[4];
        quat_mul(xb + 3, thnew + 4 * p, o);
        for (int c = 0; c < 4; ++c) thnew[4 * p + c] = o[c];
    }
    if (threadIdx.x == 0) iters_out[a] = it;
}

// |g|^2 over all links (global accumulator), after the step
__global__ void k_g2(int P, const int* __restrict__ bp, const int* __restrict__ bq,
                     const double* __restrict__ q, const double* __restrict__ th,
                     const double* __restrict__ dlp, const double* __restrict__ dlq,
                     double* __restrict__ acc) {
    __shared__ double sh[64];
    double gg = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < P; n += gridDim.x * blockDim.x) {
        const int p = bp[n], qq = bq[n];
        const double* tp = th + 4 * p;
        const double* tq = th + 4 * qq;
        double ax, ay, az, bx, by, bz;
        quat_rotate(tp[0], tp[1], tp[2], tp[3], dlp[3 * n], dlp[3 * n + 1], dlp[3 * n + 2], ax, ay, az);
        quat_rotate(tq[0], tq[1], tq[2], tq[3], dlq[3 * n], dlq[3 * n + 1], dlq[3 * n + 2], bx, by, bz);
        const double g0 = q[3 * p] + ax - q[3 * qq] - bx;
        const double g1 = q[3 * p + 1] + ay - q[3 * qq + 1] - by;
        const double g2 = q[3 * p + 2] + az - q[3 * qq + 2] - bz;
        gg += g0 * g0 + g1 * g1 + g2 * g2;
    }
    gg = block_sum(gg, sh);
    if (threadIdx.x == 0) atomicAdd(acc, gg);
}

}  // namespace am

namespace am {

// ------------------------------------------- device-controlled Arnoldi ---
// One Arnoldi step whose index j lives in device memory (ArnoldiCtrl), so the
// same kernels can run inside a CUDA-graph WHILE node without the host.

__global__ void k_ctrl_init(ArnoldiCtrl* c, int budget, int m, double tol_abs) {
    c->j = 0; c->it = 0; c->budget = budget; c->m = m; c->stop = 0; c->tol_abs = tol_abs;
}

// ---- per-system (batched) GMRES kernels ----------------------------------
// Unknowns of system s occupy three segments of the global vector (its
// blobs' lambda, its bodies' U, its links' phi); the dot-product chunks never
// straddle two systems and are listed system by system
// (sys_chunk_off[s] .. sys_chunk_off[s+1]).

// npart[c] = sum of v^2 over chunk c
__global__ void __launch_bounds__(256)
k_chunk_sq(const double* __restrict__ v, const int* __restrict__ cs, const int* __restrict__ ce,
           double* __restrict__ npart) {
    __shared__ double sh[64];
    const int c = blockIdx.x;
    double a = 0.0;
    for (int i = cs[c] + threadIdx.x; i < ce[c]; i += blockDim.x) a = fma(v[i], v[i], a);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) npart[c] = a;
}

// r = b - Ax and npart[c] = sum of r^2 over chunk c
__global__ void __launch_bounds__(256)
k_chunk_resid(const double* __restrict__ b, const double* __restrict__ Ax, double* __restrict__ r,
              const int* __restrict__ cs, const int* __restrict__ ce, double* __restrict__ npart) {
    __shared__ double sh[64];
    const int c = blockIdx.x;
    double a = 0.0;
    for (int i = cs[c] + threadIdx.x; i < ce[c]; i += blockDim.x) {
        const double v = b[i] - Ax[i];
        r[i] = v;
        a = fma(v, v, a);
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) npart[c] = a;
}

// out[s] = sqrt(sum of the system's chunk partials)
__global__ void k_sys_norm(const double* __restrict__ npart, const int* __restrict__ coff, int S,
                           double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double a = 0.0;
    for (int c = coff[s]; c < coff[s + 1]; ++c) a += npart[c];
    out[s] = sqrt(a);
}

// out = min over systems (with b_s != 0) of |r_s| / |b_s|
__global__ void k_sys_minrel(int S, const double* __restrict__ beta, const double* __restrict__ bnorm,
                             double* __restrict__ out) {
    __shared__ double smin[256];
    double mn = 1e300;
    for (int s = threadIdx.x; s < S; s += blockDim.x)
        if (bnorm[s] > 0.0) mn = fmin(mn, beta[s] / bnorm[s]);
    smin[threadIdx.x] = mn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = smin[0];
}

// Start of a restart cycle, one block: per system the relative residual
// beta_s / ||b_s||; systems above tol are active, with v_0 scale 1/beta_s,
// g = (beta_s, 0, ...), absolute stop threshold tol ||b_s||.  red[0] = max
// relative residual (NaN if any is not finite), red[1] = active count.
__global__ void k_cycle_init(int S, int m, double tol, const double* __restrict__ beta,
                             const double* __restrict__ bnorm, int* __restrict__ active,
                             double* __restrict__ inv, double* __restrict__ g, int* __restrict__ kdone,
                             double* __restrict__ tol_s, double* __restrict__ red) {
    __shared__ double smax[256];
    __shared__ int scnt[256];
    __shared__ int sbad[256];
    double mx = 0.0;
    int cnt = 0, bad = 0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double bn = bnorm[s], be = beta[s];
        const double rel = bn > 0.0 ? be / bn : 0.0;
        const bool finite = (rel == rel) && rel < 1e300;
        const bool act = finite && bn > 0.0 && rel > tol;
        active[s] = act ? 1 : 0;
        inv[s] = act ? 1.0 / be : 0.0;
        double* gs = g + (size_t)s * (m + 1);
        gs[0] = act ? be : 0.0;
        for (int k = 1; k <= m; ++k) gs[k] = 0.0;
        kdone[s] = 0;
        tol_s[s] = tol * bn;
        if (finite) mx = fmax(mx, rel); else bad = 1;
        cnt += act ? 1 : 0;
    }
    smax[threadIdx.x] = mx;
    scnt[threadIdx.x] = cnt;
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            scnt[threadIdx.x] += scnt[threadIdx.x + o];
            sbad[threadIdx.x] |= sbad[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        red[0] = sbad[0] ? nan("") : smax[0];
        red[1] = (double)scnt[0];
    }
}

// v *= a[system of the element]; the result also into copy (if not null)
__global__ void k_scale_sys(double* __restrict__ v, int n, const int* __restrict__ sys_of,
                            const double* __restrict__ a, double* __restrict__ copy = nullptr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double t = v[i] * a[sys_of[i]];
        v[i] = t;
        if (copy) copy[i] = t;
    }
}

// v = 0 on the elements of inactive systems
__global__ void k_mask_sys(double* __restrict__ v, int n, const int* __restrict__ sys_of,
                           const int* __restrict__ active) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (!active[sys_of[i]]) v[i] = 0.0;
}

// Per active system, with a = |w_s|^2: H column j, Givens rotations, the
// residual estimate; a system stops (kdone = j + 1) when the estimate
// reaches its threshold or the step breaks down.  inv[s] = 1/|w_s| (0 if
// stopped).
__device__ __forceinline__ void finish_one(int s, int j, int m, const double* __restrict__ hcol, double a,
                                           double* __restrict__ H, double* __restrict__ cs,
                                           double* __restrict__ sn, double* __restrict__ g,
                                           int* __restrict__ active, int* __restrict__ kdone,
                                           const double* __restrict__ tol_s, double* __restrict__ inv) {
    if (!active[s]) { inv[s] = 0.0; return; }
    const int m1 = m + 1;
    const double nrm = sqrt(a);
    double* h = H + ((size_t)s * m + j) * m1;
    const double* hc = hcol + (size_t)s * m1;
    double* css = cs + (size_t)s * m;
    double* sns = sn + (size_t)s * m;
    double* gs = g + (size_t)s * m1;
    // the earlier rotations applied in order; only the running entry carries
    // from one rotation to the next, the rest are loads and stores
    double carry = hc[0];
    for (int i = 0; i < j; ++i) {
        const double b = hc[i + 1];
        const double t = css[i] * carry + sns[i] * b;
        carry = -sns[i] * carry + css[i] * b;
        h[i] = t;
    }
    const double d = hypot(carry, nrm);
    double cc = 1.0, sg = 0.0;
    if (d > 0.0) { cc = carry / d; sg = nrm / d; }
    css[j] = cc; sns[j] = sg;
    h[j] = d;
    h[j + 1] = 0.0;
    gs[j + 1] = -sg * gs[j];
    gs[j] = cc * gs[j];
    const double est = fabs(gs[j + 1]);
    const bool stop = !(est > tol_s[s]) || nrm == 0.0;
    inv[s] = (!stop && nrm > 0.0) ? 1.0 / nrm : 0.0;
    if (stop) { active[s] = 0; kdone[s] = j + 1; }
}

// Advance j; the cycle ends when no system is active, at the restart length
// or at the step budget (still-active systems then close at j + 1).  Every
// thread of the one block calls it.
__device__ void loop_ctrl(ArnoldiCtrl* c, int* __restrict__ active, int* __restrict__ kdone, int S,
                          cudaGraphConditionalHandle hc, int in_graph) {
    __shared__ int scnt[256];
    __shared__ int s_stop;
    const int j1 = c->j + 1;
    int cnt = 0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) cnt += __ldcg(active + s);  // set by other blocks
    scnt[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) scnt[threadIdx.x] += scnt[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) s_stop = (scnt[0] == 0 || j1 >= c->m || c->it + 1 >= c->budget) ? 1 : 0;
    __syncthreads();
    if (s_stop)
        for (int s = threadIdx.x; s < S; s += blockDim.x)
            if (__ldcg(active + s)) { kdone[s] = j1; active[s] = 0; }
    __syncthreads();
    if (threadIdx.x == 0) {
        c->it += 1;
        c->j = j1;
        c->stop = s_stop;
        if (in_graph) cudaGraphSetConditional(hc, s_stop ? 0u : 1u);
    }
}

// ---- one Arnoldi step after w = A z: CGS2, norm, Givens, loop control --
// Three kernels of one block per dot-product chunk (chunks never straddle
// systems).  After a block has written its chunk's partial sums it counts
// itself in cnt[s] (s its system); the block that completes the count (the
// system's last) sums the system's partials in chunk order, and in the last
// kernel the last system's last block (count cnt[S]) also runs the loop
// control.  The completing block zeroes its count for the next use.  The
// arithmetic and its order are those of separate dot, coefficient,
// orthogonalisation, norm and step-end kernels.

// part[k * nchunks + b] = <V_k, w> over chunk [c0, c1), k <= j (a warp per k)
__device__ __forceinline__ void chunk_dots(const double* __restrict__ V, size_t ldv, const double* w, int c0,
                                           int c1, int j, double* __restrict__ part, int nchunks, int b) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = wid; k <= j; k += nw) {
        const double* v = V + (size_t)k * ldv;
        double a = 0.0;
        for (int i = c0 + lane; i < c1; i += 32) a = fma(v[i], w[i], a);
        a = warp_sum(a);
        if (lane == 0) part[(size_t)k * nchunks + b] = a;
    }
}

// coef[s][k] = sum over the system's chunks (a warp per k, its lanes over
// the chunks); hcol[s][k] = (hcol +) coef
__device__ __forceinline__ void sys_coef(int s, const double* part, int nchunks, const int* __restrict__ coff,
                                         int m1, int j, double* __restrict__ coef, double* __restrict__ hcol,
                                         int accumulate) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int q0 = coff[s], q1 = coff[s + 1];
    for (int k = wid; k <= j; k += nw) {
        const double* pk = part + (size_t)k * nchunks;
        double a = 0.0;
        for (int q = q0 + lane; q < q1; q += 32) a += __ldcg(pk + q);  // other blocks' sums
        a = warp_sum(a);
        if (lane == 0) {
            coef[(size_t)s * m1 + k] = a;
            double* hc = hcol + (size_t)s * m1 + k;
            *hc = accumulate ? *hc + a : a;
        }
    }
}

// w_i -= sum_{k <= j} coef[s][k] V_k,i over the chunk; returns the thread's
// share of |w|^2 over the chunk (after the update).  When the chunk is
// shorter than the block, the block's G = blockDim / len groups of len
// threads each sum every G-th term of an element's sum (shorter dependent
// FP64 chains), combined in shared memory (sh: blockDim doubles).
__device__ __forceinline__ double chunk_orth(const double* __restrict__ V, size_t ldv, double* w, int c0,
                                             int c1, int j, const double* cf, int len, double* sh) {
    const int per = min((int)blockDim.x, len);  // threads per group
    const int G = blockDim.x / per;
    const int e = threadIdx.x % per, g = threadIdx.x / per;
    double a = 0.0;
    for (int i0 = c0; i0 < c1; i0 += per) {
        const int i = i0 + e;
        double p = 0.0;
        if (i < c1)
            for (int k = g; k <= j; k += G) p = fma(cf[k], V[(size_t)k * ldv + i], p);
        if (G > 1) {
            __syncthreads();
            sh[threadIdx.x] = p;
            __syncthreads();
            if (g == 0)
                for (int q = 1; q < G; ++q) p += sh[q * per + e];
        }
        if (g == 0 && i < c1) {
            const double v = w[i] - p;
            w[i] = v;
            a = fma(v, v, a);
        }
    }
    return a;
}

// Z[j] = z (flexible GMRES keeps the preconditioned vectors); first CGS
// pass: dots and coefficients
__global__ void __launch_bounds__(256)
k_arn_dots(const double* __restrict__ V, size_t ldv, const double* __restrict__ w,
           const double* __restrict__ z, double* __restrict__ Z, const int* __restrict__ cs,
           const int* __restrict__ ce, const int* __restrict__ sys_of, const int* __restrict__ coff,
           double* __restrict__ part, int nchunks, int m1, double* __restrict__ coef, double* __restrict__ hcol,
           int* __restrict__ cnt, const ArnoldiCtrl* __restrict__ c) {
    dep_wait();
    const int j = c->j, b = blockIdx.x, c0 = cs[b], c1 = ce[b], s = sys_of[c0];
    double* zc = Z + (size_t)j * ldv;
    for (int i = c0 + threadIdx.x; i < c1; i += blockDim.x) zc[i] = z[i];
    chunk_dots(V, ldv, w, c0, c1, j, part, nchunks, b);
    if (arrive_last(cnt, s, coff[s + 1] - coff[s])) sys_coef(s, part, nchunks, coff, m1, j, coef, hcol, 0);
}

// first CGS pass: orthogonalisation; second pass: dots and coefficients
__global__ void __launch_bounds__(256)
k_arn_orth_dots(const double* __restrict__ V, size_t ldv, double* __restrict__ w, const int* __restrict__ cs,
                const int* __restrict__ ce, const int* __restrict__ sys_of, const int* __restrict__ coff, int clen,
                double* __restrict__ part, int nchunks, int m1, double* __restrict__ coef,
                double* __restrict__ hcol, int* __restrict__ cnt, const ArnoldiCtrl* __restrict__ c) {
    dep_wait();
    __shared__ double sh[256];
    const int j = c->j, b = blockIdx.x, c0 = cs[b], c1 = ce[b], s = sys_of[c0];
    chunk_orth(V, ldv, w, c0, c1, j, coef + (size_t)s * m1, clen, sh);
    __syncthreads();  // the chunk of w is updated before its dots
    chunk_dots(V, ldv, w, c0, c1, j, part, nchunks, b);
    if (arrive_last(cnt, s, coff[s + 1] - coff[s])) sys_coef(s, part, nchunks, coff, m1, j, coef, hcol, 1);
}

// second pass: orthogonalisation and |w|^2; per system the step end
// (finish_one), then the loop control
__global__ void __launch_bounds__(256)
k_arn_orth_finish(const double* __restrict__ V, size_t ldv, double* __restrict__ w, const int* __restrict__ cs,
                  const int* __restrict__ ce, const int* __restrict__ sys_of, const int* __restrict__ coff, int clen,
                  double* __restrict__ npart, int m1, const double* __restrict__ coef,
                  const double* __restrict__ hcol, int* __restrict__ cnt, int S, int m, double* __restrict__ H,
                  double* __restrict__ csv, double* __restrict__ snv, double* __restrict__ g,
                  int* __restrict__ active, int* __restrict__ kdone, const double* __restrict__ tol_s,
                  double* __restrict__ inv, ArnoldiCtrl* c, cudaGraphConditionalHandle hc, int in_graph) {
    dep_wait();
    __shared__ double sh[256];
    const int j = c->j, b = blockIdx.x, c0 = cs[b], c1 = ce[b], s = sys_of[c0];
    double a = chunk_orth(V, ldv, w, c0, c1, j, coef + (size_t)s * m1, clen, sh);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) npart[b] = a;
    if (arrive_last(cnt, s, coff[s + 1] - coff[s])) {
        double w2 = 0.0;
        for (int q = coff[s] + threadIdx.x; q < coff[s + 1]; q += blockDim.x) w2 += __ldcg(npart + q);
        w2 = block_sum(w2, sh);
        if (threadIdx.x == 0) finish_one(s, j, m, hcol, w2, H, csv, snv, g, active, kdone, tol_s, inv);
        if (arrive_last(cnt, S, S)) loop_ctrl(c, active, kdone, S, hc, in_graph);
    }
}

// V[j+1] = w * inv[system], also into vj (the next step's vector to
// precondition); with the loop control already advanced (j_ahead), the
// column is V[j].
__global__ void k_next_basis(const double* __restrict__ w, double* __restrict__ V, size_t ldv, int n,
                             const int* __restrict__ sys_of, const double* __restrict__ inv,
                             const ArnoldiCtrl* __restrict__ c, double* __restrict__ vj, int j_ahead) {
    dep_wait();
    double* v = V + (size_t)(c->j + (j_ahead ? 0 : 1)) * ldv;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double t = inv[sys_of[i]] * w[i];
        v[i] = t;
        vj[i] = t;
    }
}

// xi_s = H_s(0:k, 0:k)^-1 g_s(0:k), k = kdone[s]  (one thread per system)
__global__ void k_hess_solve_sys(const double* __restrict__ H, const double* __restrict__ g,
                                 const int* __restrict__ kdone, double* __restrict__ xi, int S, int m) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int k = kdone[s], m1 = m + 1;
    const double* Hs = H + (size_t)s * m * m1;
    const double* gs = g + (size_t)s * m1;
    double* xs = xi + (size_t)s * m1;
    for (int i = k - 1; i >= 0; --i) {
        double a = gs[i];
        for (int q = i + 1; q < k; ++q) a -= Hs[(size_t)q * m1 + i] * xs[q];
        const double d = Hs[(size_t)i * m1 + i];
        xs[i] = d != 0.0 ? a / d : 0.0;
    }
}

// t_i = sum_{k < kdone[s]} xi_s[k] Z_k,i with s the system of i
__global__ void k_combine_sys(const double* __restrict__ Z, size_t ldv, const double* __restrict__ xi,
                              const int* __restrict__ kdone, const int* __restrict__ sys_of, int n, int m1,
                              double* __restrict__ t) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = sys_of[i];
        const double* xs = xi + (size_t)s * m1;
        double a = 0.0;
        for (int k = 0; k < kdone[s]; ++k) a = fma(xs[k], Z[(size_t)k * ldv + i], a);
        t[i] = a;
    }
}

}  // namespace am

// =============================================================== host ===
namespace am {

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

int take_flags(am_handle* h) {
    int f = 0;
    cudaMemcpyAsync(h->h_flags, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream);
    cudaStreamSynchronize(h->stream);
    f = *h->h_flags;
    return f;
}

void launch_geometry(am_handle* h) {
    cudaStream_t s = h->stream;
    if (h->Nb) {
        k_pose<<<nblk(h->Nb, 256), 256, 0, s>>>(h->Nb, h->d_body_of_blob, h->d_q, h->d_theta, h->d_rho,
                                                 h->d_r4, h->d_d4, h->d_rhi, h->d_rlo, h->d_r3,
                                                 h->cfg.blob_radius, h->cfg.wall, h->d_flags);
        count_launch();
    }
    if (h->P) {
        k_links<<<nblk(h->P, 256), 256, 0, s>>>(h->P, h->d_bp, h->d_bq, h->d_theta, h->d_dlp, h->d_dlq,
                                                 h->active_links ? h->d_dlpd : nullptr,
                                                 h->active_links ? h->d_dlqd : nullptr,
                                                 h->d_lp, h->d_lq, h->d_B);
        count_launch();
    }
    k_rhs<<<nblk(h->n, 256), 256, 0, s>>>(h->Nb, h->M, h->P, h->d_slip, h->d_F, h->d_B, h->d_b);
    count_launch();
    if (h->sb) {
        sb_rhs(h);
        return;
    }
    if (h->per) h->per_status = periodic_bin(h);
    steric_apply(h);
}

static void timing_mark(am_handle* h) {
    if (!h->timing) return;
    if (h->tev_used == h->tev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        h->tev.push_back(e);
    }
    cudaEventRecord(h->tev[h->tev_used++], h->stream);
}

static void mobility_partial(am_handle* h, const double* lam, int mode, const int* active = nullptr) {
    timing_mark(h);
    launch_items(h, lam, mode, active);
    timing_mark(h);
    long long pairs = h->per_nnz;  // periodic: the real-space pairs
    if (!h->per)
        for (const auto& r : h->sys) pairs += (long long)r.Nb * r.Nb;
    h->pairs += pairs;
}

void mobility_apply(am_handle* h, const double* lam, double* u, int mode) {
    mobility_partial(h, lam, mode);
    launch_sum_items(h, u);
}

void op_apply(am_handle* h, const double* y, double* out, int mode, const int* active) {
    if (h->sb) {
        sb_op_apply(h, y, out);
        return;
    }
    mobility_partial(h, y, mode, active);
    const int nbb = nblk(h->Nb, 128), nbody = nblk(h->M, 4), nlink = nblk(h->P, 128);
    launch_dep(k_op_epilogue, dim3(nbb + nbody + nlink), dim3(128), 0, h->stream, h->Nb, h->M, h->P, nbb, nbody,
               h->d_mv, h->d_sys_of_blob, h->d_sys_blob0, h->d_sys_nb, h->d_sys_nch, h->d_sys_poff, y, out,
               h->d_body_of_blob, h->d_blob_off, h->d_d4, h->d_body_link_off, h->d_body_link_idx, h->d_lp, h->d_lq,
               h->d_bp, h->d_bq);
    count_launch();
}

void project_constraints(am_handle* h, double* x) {
    if (!h->P) return;
    cudaStream_t s = h->stream;
    k_proj_rhs<<<nblk(h->n, 256), 256, 0, s>>>(h->Nb, h->M, h->P, h->d_bp, h->d_bq, h->d_lp, h->d_lq,
                                                h->d_B, x, h->d_t);
    count_launch();
    pc_apply(h, h->d_t, h->d_z);
    k_axpy<<<nblk(h->n, 256), 256, 0, s>>>(x, h->d_z, h->n, 1.0);
    count_launch();
}

static int red_blocks(int n) { return std::min(nblk(n, 256), 2 * num_sms()); }

__global__ void k_combine3(double* __restrict__ x, const double* __restrict__ v0,
                           const double* __restrict__ v1, const double* __restrict__ v2, double w0,
                           double w1, double w2, int k, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double a = w0 * v0[i];
        if (k > 1) a = fma(w1, v1[i], a);
        if (k > 2) a = fma(w2, v2[i], a);
        x[i] = a;
    }
}

void combine_vectors(am_handle* h, double* x, const double* const* v, const double* w, int k, int len) {
    if (len <= 0) return;
    k_combine3<<<red_blocks(len), 256, 0, h->stream>>>(x, v[0], k > 1 ? v[1] : v[0], k > 2 ? v[2] : v[0],
                                                         w[0], k > 1 ? w[1] : 0.0, k > 2 ? w[2] : 0.0, k, len);
    count_launch();
}


static void read_scal(am_handle* h, int count) {
    cudaMemcpyAsync(h->h_scal, h->d_scal, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaStreamSynchronize(h->stream);
}

// per-system 2-norms of v into out (S doubles, device)
static void sys_norms(am_handle* h, const double* v, double* out) {
    k_chunk_sq<<<h->nchunks, 256, 0, h->stream>>>(v, h->d_chunk_start, h->d_chunk_end, h->d_npart);
    k_sys_norm<<<nblk(h->S, 128), 128, 0, h->stream>>>(h->d_npart, h->d_sys_chunk_off, h->S, out);
    count_launch(2);
}

// per-system residual r = b - A x (operator in FP64 or the handle's
// precision) and its norms into out
static void sys_residual(am_handle* h, const double* b, const double* x, double* r, double* out, int mode) {
    op_apply(h, x, h->d_w, mode);
    k_chunk_resid<<<h->nchunks, 256, 0, h->stream>>>(b, h->d_w, r, h->d_chunk_start, h->d_chunk_end, h->d_npart);
    k_sys_norm<<<nblk(h->S, 128), 128, 0, h->stream>>>(h->d_npart, h->d_sys_chunk_off, h->S, out);
    count_launch(2);
}

// Per chunk c, with w = rl - rp: part[c] = <rp, w>, part[nch + c] = <w, w>
__global__ void __launch_bounds__(256)
k_chunk_line(const double* __restrict__ rp, const double* __restrict__ rl, const int* __restrict__ cs,
             const int* __restrict__ ce, int nch, double* __restrict__ part) {
    __shared__ double sh[64];
    const int c = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = cs[c] + threadIdx.x; i < ce[c]; i += blockDim.x) {
        const double w = rl[i] - rp[i];
        a = fma(rp[i], w, a);
        b = fma(w, w, b);
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) { part[c] = a; part[nch + c] = b; }
}

// Per system the step along xl - xp that minimises |r(xp + beta (xl - xp))|:
// beta_s = -<rp, w> / <w, w> (0 when w = 0); out[0] = systems with beta > 0.
__global__ void k_sys_line(const double* __restrict__ part, const int* __restrict__ coff, int S, int nch,
                           double* __restrict__ beta, double* __restrict__ out) {
    __shared__ double sh[64];
    double cnt = 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int c = coff[s]; c < coff[s + 1]; ++c) { a += part[c]; b += part[nch + c]; }
        const double bs = b > 0.0 ? -a / b : 0.0;
        beta[s] = bs;
        cnt += bs > 0.0 ? 1.0 : 0.0;
    }
    cnt = block_sum(cnt, sh);
    if (threadIdx.x == 0) out[0] = cnt;
}

// x = xp + beta_s (x - xp)
__global__ void k_line_combine(double* __restrict__ x, const double* __restrict__ xp, int n,
                               const int* __restrict__ sys_of, const double* __restrict__ beta) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = fma(beta[sys_of[i]], x[i] - xp[i], xp[i]);
}

int line_initial(am_handle* h, double* x, const double* xp) {
    const int S = h->S;
    double* beta = h->d_sysred + 2 * (size_t)S;
    double* rn = h->d_sysred + 3 * (size_t)S;
    sys_residual(h, h->d_b, x, h->d_rir, rn, kOpHandle);   // r of the learned guess
    sys_residual(h, h->d_b, xp, h->d_z, rn, kOpHandle);    // r of P~^-1 b
    k_chunk_line<<<h->nchunks, 256, 0, h->stream>>>(h->d_z, h->d_rir, h->d_chunk_start, h->d_chunk_end,
                                                    h->nchunks, h->d_part);
    k_sys_line<<<1, 256, 0, h->stream>>>(h->d_part, h->d_sys_chunk_off, S, h->nchunks, beta, h->d_scal);
    k_line_combine<<<red_blocks(h->n), 256, 0, h->stream>>>(x, xp, h->n, h->d_sys_of_elem, beta);
    count_launch(3);
    read_scal(h, 1);
    return (int)h->h_scal[0];
}

// One Arnoldi step of flexible GMRES for every system at once, with the step
// index in device memory: z = P^-1 V[j] (stored in Z[j]), w = A z, CGS2 with
// per-system coefficients, per-system Givens updates and stopping,
// V[j+1] = w / |w_s|, then the loop control.
static void issue_arnoldi_step(am_handle* h, bool fp64, cudaGraphConditionalHandle hc, bool in_graph) {
    cudaStream_t s = h->stream;
    const int n = h->n, m = h->restart, m1 = m + 1, S = h->S;
    const size_t ldv = (size_t)h->ldv;
    const int nb = red_blocks(n), nch = h->nchunks, ct = h->chunk_threads;
    pc_apply(h, h->d_vj, h->d_zj);  // vj = V[j], written with V[j]
    // the input of a stopped system is zero: its product skips the pairs
    op_apply(h, h->d_zj, h->d_w, fp64, S > 1 ? h->d_active : nullptr);
    launch_dep(k_arn_dots, dim3(nch), dim3(ct), 0, s, h->d_V, ldv, h->d_w, h->d_zj, h->d_Z, h->d_chunk_start,
               h->d_chunk_end, h->d_sys_of_elem, h->d_sys_chunk_off, h->d_part, nch, m1, h->d_coefs, h->d_hcols,
               h->d_arn_cnt, h->d_ctrl);
    launch_dep(k_arn_orth_dots, dim3(nch), dim3(ct), 0, s, h->d_V, ldv, h->d_w, h->d_chunk_start, h->d_chunk_end,
               h->d_sys_of_elem, h->d_sys_chunk_off, h->chunk_len, h->d_part, nch, m1, h->d_coefs, h->d_hcols,
               h->d_arn_cnt, h->d_ctrl);
    launch_dep(k_arn_orth_finish, dim3(nch), dim3(ct), 0, s, h->d_V, ldv, h->d_w, h->d_chunk_start, h->d_chunk_end,
               h->d_sys_of_elem, h->d_sys_chunk_off, h->chunk_len, h->d_npart, m1, h->d_coefs, h->d_hcols,
               h->d_arn_cnt, S, m, h->d_Hs, h->d_css, h->d_sns, h->d_gs, h->d_active, h->d_kdone, h->d_tol_s,
               h->d_inv_s, h->d_ctrl, hc, in_graph ? 1 : 0);
    // j has advanced: V[j] = w / |w_s| and the next step's input
    launch_dep(k_next_basis, dim3(nb), dim3(256), 0, s, h->d_w, h->d_V, ldv, n, h->d_sys_of_elem, h->d_inv_s,
               h->d_ctrl, h->d_vj, 1);
    count_launch(4);
}

// The graph of one Arnoldi cycle: a WHILE node whose body is one step,
// captured once per handle layout and operator precision.
static bool ensure_graph(am_handle* h, bool fp64) {
    const int gi = fp64 ? 1 : 0;
    if (h->gexec[gi] && h->graph_gen[gi] == h->layout_gen) return true;
    if (h->gexec[gi]) { cudaGraphExecDestroy(h->gexec[gi]); h->gexec[gi] = nullptr; }
    if (h->graph[gi]) { cudaGraphDestroy(h->graph[gi]); h->graph[gi] = nullptr; }
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    cudaGraphConditionalHandle hc;
    if (cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        cudaGraphDestroy(g);
        return false;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) {
        cudaGraphDestroy(g);
        return false;
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    const long long l0 = g_launches.load();
    const long long p0 = h->pairs;
    const bool timing = h->timing;
    h->timing = false;
    bool ok = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        issue_arnoldi_step(h, fp64, hc, true);
        cudaGraph_t out = nullptr;
        ok = cudaStreamEndCapture(h->stream, &out) == cudaSuccess;
    }
    h->timing = timing;
    h->body_launches[gi] = g_launches.load() - l0;
    h->body_pairs[gi] = h->pairs - p0;
    g_launches.store(l0);
    h->pairs = p0;
    cudaGetLastError();
    if (!ok || cudaGraphInstantiate(&h->gexec[gi], g, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        h->gexec[gi] = nullptr;
        return false;
    }
    h->graph[gi] = g;
    h->graph_gen[gi] = h->layout_gen;
    return true;
}

// Flexible GMRES(m) (right preconditioning, x = x0 + Z xi with the stored
// z_j = P^-1 v_j, so a preconditioner applied in FP32 is allowed), CGS2, for
// all systems of the handle at once: each system has its own Krylov basis
// segment, Hessenberg matrix, Givens rotations and stopping test
// ||b_s - A x_s|| <= tol ||b_s||; converged systems drop out.  The operator is
// FP64 (fp64) or the handle's precision.  Each restart cycle runs on the
// device as one graph launch (WHILE node over Arnoldi steps); with
// per-kernel timing on, the same steps are launched from the host instead
// (event records cannot live in a graph loop).  Returns the number of steps;
// *rel = the largest final relative residual.
static int gmres(am_handle* h, const double* rhs, double* x, double tol, bool fp64, int budget,
                 double* rel, int* cycles, double* rel0 = nullptr) {
    cudaStream_t s = h->stream;
    const int n = h->n, m = h->restart, m1 = m + 1, S = h->S;
    const size_t ldv = (size_t)h->ldv;
    const int nb = red_blocks(n);
    sys_norms(h, rhs, h->d_bnorm_s);
    cudaMemsetAsync(h->d_arn_cnt, 0, (S + 1) * sizeof(int), s);  // arrival counts of the step kernels
    const bool use_graph = !h->timing && h->graphs_ok && ensure_graph(h, fp64);
    const int gi = fp64 ? 1 : 0;
    int it = 0;
    *rel = 0.0;
    bool first = true;
    while (true) {
        sys_residual(h, rhs, x, h->d_V, h->d_beta_s, fp64);
        k_cycle_init<<<1, 256, 0, s>>>(S, m, tol, h->d_beta_s, h->d_bnorm_s, h->d_active, h->d_inv_s, h->d_gs,
                                       h->d_kdone, h->d_tol_s, h->d_scal);
        count_launch();
        read_scal(h, 2);
        *rel = h->h_scal[0];
        if (first && rel0) *rel0 = *rel;
        first = false;
        const int n_active = (int)h->h_scal[1];
        if (n_active == 0 || it >= budget || !(*rel == *rel)) break;
        ++*cycles;
        k_scale_sys<<<nb, 256, 0, s>>>(h->d_V, n, h->d_sys_of_elem, h->d_inv_s, h->d_vj);
        k_ctrl_init<<<1, 1, 0, s>>>(h->d_ctrl, budget - it, m, 0.0);
        count_launch(2);
        if (use_graph) {
            cudaGraphLaunch(h->gexec[gi], s);
            cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(ArnoldiCtrl), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            g_launches.fetch_add(h->body_launches[gi] * h->h_ctrl->it);
            h->pairs += h->body_pairs[gi] * h->h_ctrl->it;
        } else {
            do {
                issue_arnoldi_step(h, fp64, 0, false);
                cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(ArnoldiCtrl), cudaMemcpyDeviceToHost, s);
                cudaStreamSynchronize(s);
            } while (!h->h_ctrl->stop);
        }
        it += h->h_ctrl->it;
        k_hess_solve_sys<<<nblk(S, 128), 128, 0, s>>>(h->d_Hs, h->d_gs, h->d_kdone, h->d_xis, S, m);
        k_combine_sys<<<nb, 256, 0, s>>>(h->d_Z, ldv, h->d_xis, h->d_kdone, h->d_sys_of_elem, n, m1, h->d_t);
        k_axpy<<<nb, 256, 0, s>>>(x, h->d_t, n, 1.0);
        count_launch(3);
    }
    return it;
}

// m2[s] += |u_i|^2 over the blobs of system s, u = M lambda summed from the
// partials of the last mobility product (a warp whose blobs share one system
// adds once)
__global__ void k_sys_mob_norm2(int Nb, const double* __restrict__ part, const int* __restrict__ sys_of_blob,
                                const int* __restrict__ sys_blob0, const int* __restrict__ sys_nb,
                                const int* __restrict__ sys_nch, const long long* __restrict__ sys_poff,
                                double* __restrict__ m2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int s = -1;
    double v = 0.0;
    if (i < Nb) {
        s = sys_of_blob[i];
        const size_t n3 = 3 * (size_t)sys_nb[s];
        const double* p = part + sys_poff[s] + 3 * (size_t)(i - sys_blob0[s]);
        double a = 0.0, b = 0.0, c = 0.0;
        for (int q = 0; q < sys_nch[s]; ++q) { a += p[q * n3]; b += p[q * n3 + 1]; c += p[q * n3 + 2]; }
        v = a * a + b * b + c * c;
    }
    const int s0 = __shfl_sync(0xffffffffu, s, 0);
    if (__all_sync(0xffffffffu, s == s0)) {
        v = warp_sum(v);
        if (lane == 0 && s0 >= 0) atomicAdd(&m2[s0], v);
    } else if (s >= 0) {
        atomicAdd(&m2[s], v);
    }
}

// The outer residual after a correction dx computed from an accurate
// residual r (rir): r - A dx = the inner solve's final residual r32 = r -
// A32 dx (the mixed operator) plus (A32 - A) dx, whose norm is below
// eps |M32 lambda_dx| (only the pair terms differ).  Per system the decision
// norm is |r32_s| + eps |M32 lambda_dx|_s; systems that were already within
// tol (not corrected) keep their norm.
__global__ void k_sys_resid_bound(int S, double tol, double eps, const double* __restrict__ bn,
                                  const double* __restrict__ beta32, const double* __restrict__ m2,
                                  double* __restrict__ be) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double b = bn[s], e = be[s];
    const double rel = b > 0.0 ? e / b : 0.0;
    const bool corrected = (rel == rel) && rel < 1e300 && b > 0.0 && rel > tol;
    if (corrected) be[s] = beta32[s] + eps * sqrt(m2[s]);
}

int solve(am_handle* h, am_step_stats* st) {
    const double tol = h->cfg.tol;
    const int budget = h->cfg.max_iter;
    int cycles = 0, it = 0;
    double rel = 0.0;
    if (h->cfg.precision == AM_FP64) {
        it = gmres(h, h->d_b, h->d_x, tol, true, budget, &rel, &cycles, &st->rel_residual0);
    } else {
        // Iterative refinement per system: residual outside with
        // double-float pair terms (rpy_df.cu; ~2^-44 per pair, far below the
        // 1e-8 .. 1e-12 tolerances, at about an eighth of the FP64 cost),
        // mixed-precision GMRES for the correction inside (systems already
        // at tol get a zero right-hand side and drop out).
        cudaStream_t s = h->stream;
        const int nb = red_blocks(h->n);
        double* bn_out = h->d_sysred;           // ||b_s|| of the outer problem
        double* be_out = h->d_sysred + h->S;    // ||b_s - A x_s|| (double-float operator)
        sys_norms(h, h->d_b, bn_out);
        // accurate: rir holds b - A x with double-float pair terms.  After a
        // correction from an accurate residual the next residual is the
        // inner solve's final mixed residual with an error bound (no
        // double-float product); after that one, the next is double-float
        // again, so bound terms never accumulate.
        bool accurate = false, updated = false, first_inner = true;
        for (int outer = 0; outer < 20; ++outer) {
            // The first residual only seeds the first correction, so the
            // mixed operator (error ~1e-7 |b|) computes it unless some system
            // is within 1e-5 of converged; every stopping decision is taken
            // on a double-float residual or on the bound above.
            bool res64 = outer > 0;
            if (updated) {
                res64 = true;  // rir and be_out were set from the inner solve
            } else {
                sys_residual(h, h->d_b, h->d_x, h->d_rir, be_out, res64 ? kOpDF : kOpHandle);
            }
            accurate = res64 && !updated;
            k_cycle_init<<<1, 256, 0, s>>>(h->S, h->restart, tol, be_out, bn_out, h->d_active,
                                           h->d_inv_s, h->d_gs, h->d_kdone, h->d_tol_s, h->d_scal);
            count_launch();
            if (!res64) {
                k_sys_minrel<<<1, 256, 0, s>>>(h->S, be_out, bn_out, h->d_scal + 2);
                count_launch();
                read_scal(h, 3);
                if (h->h_scal[2] < 1e-5 || h->h_scal[1] == 0.0) {
                    res64 = true;
                    accurate = true;
                    sys_residual(h, h->d_b, h->d_x, h->d_rir, be_out, kOpDF);
                    k_cycle_init<<<1, 256, 0, s>>>(h->S, h->restart, tol, be_out, bn_out, h->d_active,
                                                   h->d_inv_s, h->d_gs, h->d_kdone, h->d_tol_s, h->d_scal);
                    count_launch();
                }
            }
            read_scal(h, 2);
            rel = h->h_scal[0];
            if (outer == 0) st->rel_residual0 = rel;
            const int n_active = (int)h->h_scal[1];
            if (n_active == 0 || it >= budget || !(rel == rel)) break;
            k_mask_sys<<<nb, 256, 0, s>>>(h->d_rir, h->n, h->d_sys_of_elem, h->d_active);
            count_launch();
            // Inner tolerance (relative to the current residual): the FP32
            // operator's error (~1e-6 of the correction) bounds it below.
            // The first correction takes about the square root of the
            // reduction still needed, the next ones all of it: two outer
            // cycles at 1e-8, with fewer iterations than a first correction
            // driven to 1e-6 (measured: diatom colony 44.6 -> 40, 1,000
            // bacteria 43 -> 35 iterations per step), whose last iterations
            // fall below the FP32 products' accuracy.
            const double need = 0.3 * tol / rel;
            const double tin = std::max(1e-6, first_inner ? std::sqrt(need) : need);
            first_inner = false;
            cudaMemsetAsync(h->d_dx, 0, h->n * sizeof(double), s);
            double rin = 0.0;
            it += gmres(h, h->d_rir, h->d_dx, tin, false, budget - it, &rin, &cycles);
            k_axpy<<<nb, 256, 0, s>>>(h->d_x, h->d_dx, h->n, 1.0);
            count_launch();
            updated = false;
            if (accurate && !h->sb) {
                // gmres ended on sys_residual: V[0] = rir - A32 dx, beta_s its
                // norms, and the mobility partials hold M32 lambda_dx
                double* m2 = h->d_sysred + 2 * (size_t)h->S;
                cudaMemsetAsync(m2, 0, h->S * sizeof(double), s);
                k_sys_mob_norm2<<<nblk(h->Nb, 256), 256, 0, s>>>(h->Nb, h->d_mv, h->d_sys_of_blob, h->d_sys_blob0,
                                                                 h->d_sys_nb, h->d_sys_nch, h->d_sys_poff, m2);
                k_sys_resid_bound<<<nblk(h->S, 128), 128, 0, s>>>(h->S, tol, kMixedProductError, bn_out,
                                                                  h->d_beta_s, m2, be_out);
                cudaMemcpyAsync(h->d_rir, h->d_V, h->n * sizeof(double), cudaMemcpyDeviceToDevice, s);
                count_launch(2);
                updated = true;
            }
        }
    }
    if (h->P) {
        k_constraint_residual<<<1, 256, 0, h->stream>>>(h->Nb, h->M, h->P, h->d_bp, h->d_bq, h->d_lp,
                                                        h->d_lq, h->d_B, h->d_x, h->d_scal, 6);
        count_launch();
        read_scal(h, 7);
        st->constraint_residual = h->h_scal[6];
    } else {
        st->constraint_residual = 0.0;
    }
    st->iterations = it;
    st->restarts = cycles;
    st->rel_residual = rel;
    return (rel <= tol) ? AM_OK : AM_ERR_NOT_CONVERGED;
}

int advance(am_handle* h, double dt, am_step_stats* st) {
    cudaStream_t s = h->stream;
    cudaMemsetAsync(h->d_red, 0, 2 * sizeof(double), s);
    k_euler_reconstruct<<<h->NA, 128, 0, s>>>(h->d_asm_body_off, h->d_asm_body_idx, h->d_asm_link_off,
                                               h->d_asm_link_idx, h->d_bp, h->d_bq,
                                               h->d_x + 3 * (size_t)h->Nb, h->d_q, h->d_theta,
                                               h->d_dlp1, h->d_dlq1, h->d_pplus, h->d_pplus_off, dt,
                                               h->d_qnew, h->d_thnew, h->d_zbuf, h->d_red);
    count_launch();
    if (h->P) {
        k_correct<<<h->NA, 256, 0, s>>>(h->d_asm_body_off, h->d_asm_body_idx, h->d_asm_link_off,
                                         h->d_asm_link_idx, h->d_bp, h->d_bq, h->d_body_local,
                                         h->d_link_local, h->d_body_link_off, h->d_body_link_idx,
                                         h->d_dlp1, h->d_dlq1, h->d_qnew, h->d_thnew, h->d_red,
                                         h->cfg.corr_tol, h->cfg.corr_max_iter, h->d_corr,
                                         h->d_corr_off, h->d_iters, h->d_flags);
        k_g2<<<std::max(1, std::min(nblk(h->P, 256), 64)), 256, 0, s>>>(
            h->P, h->d_bp, h->d_bq, h->d_qnew, h->d_thnew, h->d_dlp1, h->d_dlq1, h->d_red + 1);
        count_launch(2);
    }
    cudaMemcpyAsync(h->d_q, h->d_qnew, 3 * h->M * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->d_theta, h->d_thnew, 4 * h->M * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (h->P) {
        cudaMemcpyAsync(h->d_dlp, h->d_dlp1, 3 * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(h->d_dlq, h->d_dlq1, 3 * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s);
    }
    cudaMemcpyAsync(h->h_scal, h->d_red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h->h_iters, h->d_iters, h->NA * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    st->g2_before = h->h_scal[0];
    st->g2_after = h->P ? h->h_scal[1] : 0.0;
    int mx = 0;
    for (int a = 0; a < h->NA; ++a) mx = std::max(mx, h->h_iters[a]);
    st->corr_iterations = mx;
    return AM_OK;
}

}  // namespace am

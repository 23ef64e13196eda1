// Learned initial guess (not in the paper): per-body features, a small MLP
// trained on the GPU with FP32 kernels and evaluated with BF16 tensor-core
// kernels, and the initial guess it gives the solve.
//
// Features of body p, in its body frame (FEAT = 144): for the 16 nearest
// other bodies k of its system (distance rounded to 1e-8, then body index),
// R_p^T (q_k - q_p) / 4 and the relative quaternion theta_p^* . theta_k
// (s >= 0); then q_p,z / 4 (0 in free space), R_p^T f_p, R_p^T tau_p, the
// body-frame velocity of the block-diagonal solution P~^-1 b, log(blobs)/5;
// the far flow R_p^T u_far(q_p) and its body-frame gradient by central
// differences along the body axes (step 0.5), where u_far is the flow of
// point forces f_k (the summed blob forces of P~^-1 b) at the tracking points
// of the bodies of the other articulated bodies of the system within 16 of
// q_p; zeros to 144.
// Target (OUT = 32): the background flow u_ext = (M - M~) lambda that the
// other bodies induce at the body's blobs, fitted in the body frame by
// NFLOW = 29 flows on the body-frame offsets rho (translation, rotation,
// traceless strain, quadratic) with ridge 1e-6 tr(B^T B) / 29.
// MLP: (x - mu)/sd -> 3 x [256, ReLU] -> 32, prediction scaled by sd_out.
// Initial guess: x0 = P~^-1 (u_s - u_fit, -F, B).
#include "am_internal.cuh"
#include "dev_util.cuh"
#include "ops.cuh"
#include "rpy_pair.cuh"
#include "tc_gemm.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <random>
#include <string>
#include <vector>

namespace am {
void set_thread_error(const std::string& msg);
}

namespace {

using am::quat_mul;
using am::quat_rotate;
using am::quat_rotate_inv;

constexpr int FEAT = 144, OUT = 32, NFLOW = 29, WIDTH = 256, NLAYER = 4, KNN = 16;
constexpr double LSCALE = 4.0, RIDGE = 1e-6, FAR_H = 0.5, FAR_R = 16.0;
const int kDims[NLAYER + 1] = {FEAT, WIDTH, WIDTH, WIDTH, OUT};

size_t layer_w_off(int l) {
    size_t o = 0;
    for (int k = 0; k < l; ++k) o += (size_t)kDims[k + 1] * kDims[k] + kDims[k + 1];
    return o;
}
size_t n_params_total() { return layer_w_off(NLAYER); }

// ------------------------------------------------------------ features ---
// One thread per body: brute-force k nearest in its own system (insertion
// into a sorted list of KNN), then the feature row.  sys_of_U: system of
// each body (the system of its first velocity unknown).
__global__ void k_features(int M, const double* __restrict__ q, const double* __restrict__ th,
                           const double* __restrict__ F, const int* __restrict__ blob_off,
                           const double* __restrict__ Upc, const int* __restrict__ sys_of_U,
                           const int* __restrict__ sys_body_off, int wall, float* __restrict__ X) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int s = sys_of_U[6 * (size_t)p];
    const int b0 = sys_body_off[s], b1 = sys_body_off[s + 1];
    double keyv[KNN];
    int idx[KNN];
    int cnt = 0;
    const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
    for (int k = b0; k < b1; ++k) {
        if (k == p) continue;
        const double dx = q[3 * k] - qx, dy = q[3 * k + 1] - qy, dz = q[3 * k + 2] - qz;
        const double key = floor(sqrt(dx * dx + dy * dy + dz * dz) * 1e8 + 0.5);
        // insert (key, k) into the sorted list of the nearest KNN
        if (cnt == KNN && !(key < keyv[KNN - 1] || (key == keyv[KNN - 1] && k < idx[KNN - 1]))) continue;
        int pos = cnt < KNN ? cnt : KNN - 1;
        while (pos > 0 && (key < keyv[pos - 1] || (key == keyv[pos - 1] && k < idx[pos - 1]))) {
            keyv[pos] = keyv[pos - 1];
            idx[pos] = idx[pos - 1];
            --pos;
        }
        keyv[pos] = key;
        idx[pos] = k;
        if (cnt < KNN) ++cnt;
    }
    float* x = X + (size_t)p * FEAT;
    for (int c = 0; c < FEAT; ++c) x[c] = 0.f;
    const double s0 = th[4 * p], p1 = th[4 * p + 1], p2 = th[4 * p + 2], p3 = th[4 * p + 3];
    const double cj[4] = {s0, -p1, -p2, -p3};
    for (int slot = 0; slot < cnt; ++slot) {
        const int k = idx[slot];
        double vx, vy, vz;
        quat_rotate_inv(s0, p1, p2, p3, q[3 * k] - qx, q[3 * k + 1] - qy, q[3 * k + 2] - qz, vx, vy, vz);
        x[7 * slot] = (float)(vx / LSCALE);
        x[7 * slot + 1] = (float)(vy / LSCALE);
        x[7 * slot + 2] = (float)(vz / LSCALE);
        double rq[4];
        quat_mul(cj, th + 4 * k, rq);
        const double sg = rq[0] < 0.0 ? -1.0 : 1.0;
        for (int c = 0; c < 4; ++c) x[7 * slot + 3 + c] = (float)(sg * rq[c]);
    }
    const int base = 7 * KNN;
    x[base] = wall ? (float)(qz / LSCALE) : 0.f;
    double a, b, c;
    quat_rotate_inv(s0, p1, p2, p3, F[6 * p], F[6 * p + 1], F[6 * p + 2], a, b, c);
    x[base + 1] = (float)a; x[base + 2] = (float)b; x[base + 3] = (float)c;
    quat_rotate_inv(s0, p1, p2, p3, F[6 * p + 3], F[6 * p + 4], F[6 * p + 5], a, b, c);
    x[base + 4] = (float)a; x[base + 5] = (float)b; x[base + 6] = (float)c;
    const double* u = Upc + 6 * (size_t)p;
    quat_rotate_inv(s0, p1, p2, p3, u[0], u[1], u[2], a, b, c);
    x[base + 7] = (float)a; x[base + 8] = (float)b; x[base + 9] = (float)c;
    quat_rotate_inv(s0, p1, p2, p3, u[3], u[4], u[5], a, b, c);
    x[base + 10] = (float)a; x[base + 11] = (float)b; x[base + 12] = (float)c;
    x[base + 13] = (float)(log((double)(blob_off[p + 1] - blob_off[p])) / 5.0);
}

// f_p = sum of the blob forces of body p (FP64)
__global__ void k_body_force(int M, const int* __restrict__ blob_off, const double* __restrict__ lam,
                             double* __restrict__ f) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = blob_off[p]; i < blob_off[p + 1]; ++i) {
        a += lam[3 * (size_t)i];
        b += lam[3 * (size_t)i + 1];
        c += lam[3 * (size_t)i + 2];
    }
    f[3 * (size_t)p] = a;
    f[3 * (size_t)p + 1] = b;
    f[3 * (size_t)p + 2] = c;
}

// Far-flow features of body p (one thread): the flow of the point forces f_k
// of the other articulated bodies' bodies of its system within FAR_R of q_p
// at q_p and at
// q_p +- h R_p e_j, pair terms in FP32 (blob pair tensor with the blob
// radius), sums in FP32; written to X[126 .. 137].
__global__ void k_far_flow(int M, const double* __restrict__ q, const double* __restrict__ th,
                           const double* __restrict__ f, const int* __restrict__ sys_of_U,
                           const int* __restrict__ sys_body_off, const int* __restrict__ asm_of_body, int wall,
                           am::RpyK<float> k, float* __restrict__ X) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int s = sys_of_U[6 * (size_t)p];
    const int b0 = sys_body_off[s], b1 = sys_body_off[s + 1];
    const int ap = asm_of_body[p];
    const double* t = th + 4 * (size_t)p;
    double xe[7][3];
    for (int e = 0; e < 7; ++e)
        for (int c = 0; c < 3; ++c) xe[e][c] = q[3 * (size_t)p + c];
    for (int j = 0; j < 3; ++j) {
        double ax[3] = {0.0, 0.0, 0.0};
        ax[j] = FAR_H;
        double w0, w1, w2;
        am::quat_rotate(t[0], t[1], t[2], t[3], ax[0], ax[1], ax[2], w0, w1, w2);
        xe[1 + 2 * j][0] += w0; xe[1 + 2 * j][1] += w1; xe[1 + 2 * j][2] += w2;
        xe[2 + 2 * j][0] -= w0; xe[2 + 2 * j][1] -= w1; xe[2 + 2 * j][2] -= w2;
    }
    float acc[7][3];
    for (int e = 0; e < 7; ++e) acc[e][0] = acc[e][1] = acc[e][2] = 0.f;
    const double px = q[3 * (size_t)p], py = q[3 * (size_t)p + 1], pz = q[3 * (size_t)p + 2];
    for (int kb = b0; kb < b1; ++kb) {
        if (asm_of_body[kb] == ap) continue;
        const double qx = q[3 * (size_t)kb], qy = q[3 * (size_t)kb + 1], qz = q[3 * (size_t)kb + 2];
        const double ex = qx - px, ey = qy - py, ez = qz - pz;
        if (ex * ex + ey * ey + ez * ez > FAR_R * FAR_R) continue;
        const float fx = (float)f[3 * (size_t)kb], fy = (float)f[3 * (size_t)kb + 1], fz = (float)f[3 * (size_t)kb + 2];
#pragma unroll
        for (int e = 0; e < 7; ++e) {
            const float dx = (float)(xe[e][0] - qx), dy = (float)(xe[e][1] - qy), dz = (float)(xe[e][2] - qz);
            am::pair_free<float>(dx, dy, dz, fx, fy, fz, k, acc[e][0], acc[e][1], acc[e][2]);
            if (wall)
                am::pair_image<float>(dx, dy, (float)(xe[e][2] + qz), (float)xe[e][2], (float)qz, fx, fy, fz, k,
                                      acc[e][0], acc[e][1], acc[e][2]);
        }
    }
    double ub[7][3];
    for (int e = 0; e < 7; ++e)
        am::quat_rotate_inv(t[0], t[1], t[2], t[3], k.A1 * acc[e][0], k.A1 * acc[e][1], k.A1 * acc[e][2],
                            ub[e][0], ub[e][1], ub[e][2]);
    float* x = X + (size_t)p * FEAT + 7 * KNN + 14;
    for (int c = 0; c < 3; ++c) x[c] = (float)ub[0][c];
    for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 3; ++j) x[3 + 3 * c + j] = (float)((ub[1 + 2 * j][c] - ub[2 + 2 * j][c]) / (2.0 * FAR_H));
}

// Row c (velocity component c) of the 29 body-frame flows at offset d:
// e_k; e_k x d; E d for E01, E02, E12 (unit symmetric off-diagonal pairs),
// diag(1,-1,0), diag(1,0,-1); d_i d_j e_c' for c' = 0..2 and (i, j) in
// (00, 01, 02, 11, 12, 22).
__device__ __forceinline__ void flow_row(const double* d, int c, double* b) {
    for (int k = 0; k < NFLOW; ++k) b[k] = 0.0;
    b[c] = 1.0;
    const double x = d[0], y = d[1], z = d[2];
    // rotations: e0 x d = (0, -z, y), e1 x d = (z, 0, -x), e2 x d = (-y, x, 0)
    // strains:   E01 d = (y, x, 0), E02 d = (z, 0, x), E12 d = (0, z, y),
    //            diag(1,-1,0) d = (x, -y, 0), diag(1,0,-1) d = (x, 0, -z)
    if (c == 0) {
        b[4] = z; b[5] = -y;
        b[6] = y; b[7] = z; b[9] = x; b[10] = x;
    } else if (c == 1) {
        b[3] = -z; b[5] = x;
        b[6] = x; b[8] = z; b[9] = -y;
    } else {
        b[3] = y; b[4] = -x;
        b[7] = x; b[8] = y; b[10] = -z;
    }
    const int q = 11 + 6 * c;
    b[q] = x * x; b[q + 1] = x * y; b[q + 2] = x * z;
    b[q + 3] = y * y; b[q + 4] = y * z; b[q + 5] = z * z;
}

// u_i -= (M~ lambda)_i: the mobility of the blobs of i's own body (the
// blocks the block-diagonal preconditioner keeps), FP64.
__global__ void k_self_sub(int Nb, const int* __restrict__ body_of_blob, const int* __restrict__ blob_off,
                           const double4_32a* __restrict__ r4, const double* __restrict__ lam, int wall,
                           am::RpyK<double> k, double* __restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const int p = body_of_blob[i];
    const double4_32a x = r4[i];
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int j = blob_off[p]; j < blob_off[p + 1]; ++j) {
        const double4_32a y = r4[j];
        const double lx = lam[3 * j], ly = lam[3 * j + 1], lz = lam[3 * j + 2];
        am::pair_free<double>(x.x - y.x, x.y - y.y, x.z - y.z, lx, ly, lz, k, ux, uy, uz);
        if (wall) am::pair_image<double>(x.x - y.x, x.y - y.y, x.z + y.z, x.z, y.z, lx, ly, lz, k, ux, uy, uz);
    }
    u[3 * (size_t)i] -= k.A1 * ux;
    u[3 * (size_t)i + 1] -= k.A1 * uy;
    u[3 * (size_t)i + 2] -= k.A1 * uz;
}

// Per body (one block): ridge fit of the body-frame flow R_p^T u over its
// blobs by the 29 flows; G = B^T B and g = B^T u accumulated by entry, the
// 29 x 29 solve by Cholesky in one thread.  T[p] = (c, 0, 0, 0) as float.
__global__ void __launch_bounds__(128)
k_flow_fit(const int* __restrict__ blob_off, const double* __restrict__ rho, const double* __restrict__ th,
           const double* __restrict__ u, float* __restrict__ T) {
    __shared__ double G[NFLOW][NFLOW + 1];
    __shared__ double g[NFLOW];
    const int p = blockIdx.x;
    const int i0 = blob_off[p], i1 = blob_off[p + 1];
    const double* t = th + 4 * (size_t)p;
    const int n_entries = NFLOW * (NFLOW + 1) / 2 + NFLOW;
    for (int e = threadIdx.x; e < n_entries; e += blockDim.x) {
        int a, b2 = -1;  // G[a][b2] for e < 435, else g[a]
        if (e < NFLOW * (NFLOW + 1) / 2) {
            a = 0;
            int rem = e;
            while (rem >= NFLOW - a) { rem -= NFLOW - a; ++a; }
            b2 = a + rem;
        } else {
            a = e - NFLOW * (NFLOW + 1) / 2;
        }
        double acc = 0.0;
        for (int i = i0; i < i1; ++i) {
            const double* d = rho + 3 * (size_t)i;
            double ub[3];
            if (b2 < 0)
                am::quat_rotate_inv(t[0], t[1], t[2], t[3], u[3 * (size_t)i], u[3 * (size_t)i + 1],
                                    u[3 * (size_t)i + 2], ub[0], ub[1], ub[2]);
            for (int c = 0; c < 3; ++c) {
                double row[NFLOW];
                flow_row(d, c, row);
                acc += row[a] * (b2 < 0 ? ub[c] : row[b2]);
            }
        }
        if (b2 < 0) g[a] = acc;
        else { G[a][b2] = acc; G[b2][a] = acc; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int a = 0; a < NFLOW; ++a) tr += G[a][a];
        const double eps = RIDGE * tr / NFLOW;
        for (int a = 0; a < NFLOW; ++a) G[a][a] += eps;
        // Cholesky G = L L^T in place (lower triangle)
        for (int j = 0; j < NFLOW; ++j) {
            double dsum = G[j][j];
            for (int k2 = 0; k2 < j; ++k2) dsum -= G[j][k2] * G[j][k2];
            const double ljj = sqrt(fmax(dsum, 1e-300));
            G[j][j] = ljj;
            for (int r = j + 1; r < NFLOW; ++r) {
                double v = G[r][j];
                for (int k2 = 0; k2 < j; ++k2) v -= G[r][k2] * G[j][k2];
                G[r][j] = v / ljj;
            }
        }
        double c[NFLOW];
        for (int r = 0; r < NFLOW; ++r) {  // L y = g
            double v = g[r];
            for (int k2 = 0; k2 < r; ++k2) v -= G[r][k2] * c[k2];
            c[r] = v / G[r][r];
        }
        for (int r = NFLOW - 1; r >= 0; --r) {  // L^T c = y
            double v = c[r];
            for (int k2 = r + 1; k2 < NFLOW; ++k2) v -= G[k2][r] * c[k2];
            c[r] = v / G[r][r];
        }
        float* o = T + (size_t)p * OUT;
        for (int k2 = 0; k2 < OUT; ++k2) o[k2] = k2 < NFLOW ? (float)c[k2] : 0.f;
    }
}

// Blob rows of the right-hand side: bt_i = b_i - R_p B(rho_i) c_p with c_p
// the network's coefficients (FP32) for the body p of blob i.
__global__ void k_flow_rhs(int Nb, const int* __restrict__ body_of_blob, const double* __restrict__ rho,
                           const double* __restrict__ th, const float* __restrict__ C,
                           const double* __restrict__ b, double* __restrict__ bt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const int p = body_of_blob[i];
    const float* cp = C + (size_t)p * OUT;
    const double* d = rho + 3 * (size_t)i;
    double v[3];
    for (int c = 0; c < 3; ++c) {
        double row[NFLOW];
        flow_row(d, c, row);
        double s = 0.0;
        for (int k = 0; k < NFLOW; ++k) s = fma(row[k], (double)cp[k], s);
        v[c] = s;
    }
    const double* t = th + 4 * (size_t)p;
    double w0, w1, w2;
    am::quat_rotate(t[0], t[1], t[2], t[3], v[0], v[1], v[2], w0, w1, w2);
    bt[3 * (size_t)i] = b[3 * (size_t)i] - w0;
    bt[3 * (size_t)i + 1] = b[3 * (size_t)i + 1] - w1;
    bt[3 * (size_t)i + 2] = b[3 * (size_t)i + 2] - w2;
}

// --------------------------------------------------------- FP32 training ---
// C[r][o] = sum_i A[r][i] W[o][i] + b[o]; Z = C, Aout = relu(C) (or C)
__global__ void __launch_bounds__(256)
k_linear_fwd(const float* __restrict__ A, const float* __restrict__ W, const float* __restrict__ b,
             float* __restrict__ Z, float* __restrict__ Aout, int n, int in, int out, int relu) {
    __shared__ float As[32][33];
    __shared__ float Ws[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int r0 = blockIdx.y * 32, o0 = blockIdx.x * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < in; k0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int rr = e / 32, kk = e % 32;
            As[rr][kk] = (r0 + rr < n && k0 + kk < in) ? A[(size_t)(r0 + rr) * in + k0 + kk] : 0.f;
            Ws[rr][kk] = (o0 + rr < out && k0 + kk < in) ? W[(size_t)(o0 + rr) * in + k0 + kk] : 0.f;
        }
        __syncthreads();
        for (int kk = 0; kk < 32; ++kk) {
            const float w = Ws[tx][kk];
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(As[ty + 8 * q][kk], w, acc[q]);
        }
        __syncthreads();
    }
    const int o = o0 + tx;
    if (o >= out) return;
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + ty + 8 * q;
        if (r >= n) continue;
        const float z = acc[q] + b[o];
        Z[(size_t)r * out + o] = z;
        Aout[(size_t)r * out + o] = relu ? fmaxf(z, 0.f) : z;
    }
}

// gW[o][i] = sum_r dZ[r][o] A[r][i];  gb[o] = sum_r dZ[r][o]
__global__ void __launch_bounds__(256)
k_linear_wgrad(const float* __restrict__ dZ, const float* __restrict__ A, float* __restrict__ gW,
               float* __restrict__ gb, int n, int in, int out) {
    __shared__ float Ds[32][33];
    __shared__ float As[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int o0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float bacc = 0.f;
    for (int r0 = 0; r0 < n; r0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int rr = e / 32, cc = e % 32;
            Ds[rr][cc] = (r0 + rr < n && o0 + cc < out) ? dZ[(size_t)(r0 + rr) * out + o0 + cc] : 0.f;
            As[rr][cc] = (r0 + rr < n && i0 + cc < in) ? A[(size_t)(r0 + rr) * in + i0 + cc] : 0.f;
        }
        __syncthreads();
        for (int rr = 0; rr < 32; ++rr) {
            const float a = As[rr][tx];
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(Ds[rr][ty + 8 * q], a, acc[q]);
            if (blockIdx.x == 0 && ty == 0) bacc += Ds[rr][tx];
        }
        __syncthreads();
    }
    const int i = i0 + tx;
    for (int q = 0; q < 4; ++q) {
        const int o = o0 + ty + 8 * q;
        if (o < out && i < in) gW[(size_t)o * in + i] = acc[q];
    }
    if (blockIdx.x == 0 && ty == 0 && o0 + tx < out) gb[o0 + tx] = bacc;
}

// dA[r][i] = sum_o dZ[r][o] W[o][i]; then dZprev = dA * (Zprev > 0)
__global__ void __launch_bounds__(256)
k_linear_xgrad(const float* __restrict__ dZ, const float* __restrict__ W, const float* __restrict__ Zprev,
               float* __restrict__ dZprev, int n, int in, int out) {
    __shared__ float Ds[32][33];
    __shared__ float Ws[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int r0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int o0 = 0; o0 < out; o0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int rr = e / 32, cc = e % 32;
            Ds[rr][cc] = (r0 + rr < n && o0 + cc < out) ? dZ[(size_t)(r0 + rr) * out + o0 + cc] : 0.f;
            Ws[rr][cc] = (o0 + rr < out && i0 + cc < in) ? W[(size_t)(o0 + rr) * in + i0 + cc] : 0.f;
        }
        __syncthreads();
        for (int oo = 0; oo < 32; ++oo) {
            const float w = Ws[oo][tx];
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(Ds[ty + 8 * q][oo], w, acc[q]);
        }
        __syncthreads();
    }
    const int i = i0 + tx;
    if (i >= in) return;
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + ty + 8 * q;
        if (r < n) dZprev[(size_t)r * in + i] = Zprev[(size_t)r * in + i] > 0.f ? acc[q] : 0.f;
    }
}

__global__ void k_normalize(const float* __restrict__ X, const float* __restrict__ mu,
                            const float* __restrict__ sd, float* __restrict__ A, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * FEAT) return;
    const int c = e % FEAT;
    A[e] = (X[e] - mu[c]) / sd[c];
}

// dZ = 2 (Zout - T / sd_out) / (n OUT); loss partials per block
__global__ void k_loss_grad(const float* __restrict__ Zout, const float* __restrict__ T,
                            const float* __restrict__ sdo, float* __restrict__ dZ, int n,
                            double* __restrict__ loss) {
    __shared__ double sh[64];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (e < n * OUT) {
        const float d = Zout[e] - T[e] / sdo[e % OUT];
        dZ[e] = 2.f * d / (float)(n * OUT);
        l = (double)d * d;
    }
    l = am::block_sum(l, sh);
    if (threadIdx.x == 0) atomicAdd(loss, l / (double)(n * OUT));
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void k_gather_rows(const float* __restrict__ src, const int* __restrict__ rows, int nrows,
                              int width, float* __restrict__ dst) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nrows * width) return;
    const int r = e / width, c = e % width;
    dst[e] = src[(size_t)rows[r] * width + c];
}

// ------------------------------------------------- BF16 tensor inference ---
__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) dst[e] = __float2bfloat16(src[e]);
}

__global__ void k_normalize_bf16(const float* __restrict__ X, const float* __restrict__ mu,
                                 const float* __restrict__ sd, __nv_bfloat16* __restrict__ A, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * FEAT) return;
    const int c = e % FEAT;
    A[e] = __float2bfloat16((X[e] - mu[c]) / sd[c]);
}

}  // namespace

// ===================================================================== model
struct am_mlp {
    float *d_p = nullptr, *d_m = nullptr, *d_v = nullptr, *d_g = nullptr;
    __nv_bfloat16* d_wbf = nullptr;
    float *d_mu = nullptr, *d_sd = nullptr, *d_sdo = nullptr;
    int adam_t = 0;
    int cap = 0;
    float *d_X = nullptr, *d_T = nullptr, *d_bx = nullptr, *d_bt = nullptr, *d_dz0 = nullptr, *d_dz1 = nullptr;
    float* d_z[NLAYER + 1] = {};
    float* d_a[NLAYER + 1] = {};
    __nv_bfloat16 *d_h0 = nullptr, *d_h1 = nullptr;
    int* d_rows = nullptr;
    int* d_flag = nullptr;  // tensor-core wait timeouts of the standalone prediction
    double* d_loss = nullptr;
    int data_n = 0;
    cudaStream_t st = nullptr;
    bool bf_valid = false;
};

namespace {

int mlp_fail(int code, const std::string& m) {
    am::set_thread_error(m);
    return code;
}

#define MCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return mlp_fail(AM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int ensure_cap(am_mlp* m, int n) {
    if (n <= m->cap) return AM_OK;
    for (int l = 0; l <= NLAYER; ++l) {
        if (m->d_z[l]) cudaFree(m->d_z[l]);
        if (m->d_a[l]) cudaFree(m->d_a[l]);
        MCK(cudaMalloc(&m->d_z[l], (size_t)n * WIDTH * sizeof(float)));
        MCK(cudaMalloc(&m->d_a[l], (size_t)n * WIDTH * sizeof(float)));
    }
    for (float** p : {&m->d_dz0, &m->d_dz1, &m->d_bx, &m->d_bt}) {
        if (*p) cudaFree(*p);
        MCK(cudaMalloc(p, (size_t)n * WIDTH * sizeof(float)));
    }
    for (__nv_bfloat16** p : {&m->d_h0, &m->d_h1}) {
        if (*p) cudaFree(*p);
        MCK(cudaMalloc(p, (size_t)n * WIDTH * sizeof(__nv_bfloat16)));
    }
    m->cap = n;
    return AM_OK;
}

const float* W_of(const am_mlp* m, int l) { return m->d_p + layer_w_off(l); }
const float* b_of(const am_mlp* m, int l) { return m->d_p + layer_w_off(l) + (size_t)kDims[l + 1] * kDims[l]; }

// forward (FP32) of n rows already in X (device) into the activation buffers
void forward32(am_mlp* m, const float* X, int n) {
    cudaStream_t s = m->st;
    k_normalize<<<(n * FEAT + 255) / 256, 256, 0, s>>>(X, m->d_mu, m->d_sd, m->d_a[0], n);
    am::count_launch();
    for (int l = 0; l < NLAYER; ++l) {
        dim3 grid((kDims[l + 1] + 31) / 32, (n + 31) / 32);
        k_linear_fwd<<<grid, 256, 0, s>>>(m->d_a[l], W_of(m, l), b_of(m, l), m->d_z[l + 1], m->d_a[l + 1], n,
                                           kDims[l], kDims[l + 1], l < NLAYER - 1 ? 1 : 0);
        am::count_launch();
    }
}

// loss and gradient (into d_g) of n rows (X, T device); loss added to d_loss
void backward32(am_mlp* m, const float* X, const float* T, int n) {
    cudaStream_t s = m->st;
    forward32(m, X, n);
    k_loss_grad<<<(n * OUT + 255) / 256, 256, 0, s>>>(m->d_z[NLAYER], T, m->d_sdo, m->d_dz0, n, m->d_loss);
    am::count_launch();
    float* dz = m->d_dz0;
    float* dzp = m->d_dz1;
    for (int l = NLAYER - 1; l >= 0; --l) {
        const int in = kDims[l], out = kDims[l + 1];
        float* gW = m->d_g + layer_w_off(l);
        float* gb = gW + (size_t)out * in;
        dim3 gw((in + 31) / 32, (out + 31) / 32);
        k_linear_wgrad<<<gw, 256, 0, s>>>(dz, m->d_a[l], gW, gb, n, in, out);
        am::count_launch();
        if (l > 0) {
            dim3 gx((in + 31) / 32, (n + 31) / 32);
            k_linear_xgrad<<<gx, 256, 0, s>>>(dz, W_of(m, l), m->d_z[l], dzp, n, in, out);
            am::count_launch();
            std::swap(dz, dzp);
        }
    }
}

void refresh_bf16(am_mlp* m) {
    if (m->bf_valid) return;
    for (int l = 0; l < NLAYER; ++l) {
        const int nw = kDims[l + 1] * kDims[l];
        k_to_bf16<<<(nw + 255) / 256, 256, 0, m->st>>>(W_of(m, l), m->d_wbf + layer_w_off(l), nw);
        am::count_launch();
    }
    m->bf_valid = true;
}

// BF16 prediction of n rows (X device) into Y (device, n x OUT, scaled by
// sd_out): each layer on the tcgen05 tensor cores (tc_gemm.cuh), one block
// per 128 rows, FP32 accumulators in tensor memory, bias and ReLU in the
// epilogue; a timed-out tensor-core wait sets am::kFlagTensor in *flags.
void predict_bf16(am_mlp* m, const float* X, int n, float* Y, int* flags) {
    cudaStream_t s = m->st;
    refresh_bf16(m);
    k_normalize_bf16<<<(n * FEAT + 255) / 256, 256, 0, s>>>(X, m->d_mu, m->d_sd, m->d_h0, n);
    am::count_launch();
    __nv_bfloat16* hin = m->d_h0;
    __nv_bfloat16* hout = m->d_h1;
    static_assert(am::tc::kFlagTensorTimeout == am::kFlagTensor, "one flag bit for tensor-core timeouts");
    for (int l = 0; l < NLAYER; ++l) {
        const bool last = l == NLAYER - 1;
        const int smem = am::tc::smem_bytes(kDims[l], kDims[l + 1]);
        cudaFuncSetAttribute(am::tc::k_linear_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        am::tc::k_linear_tc<<<(n + am::tc::kRows - 1) / am::tc::kRows, 128, smem, s>>>(
            hin, m->d_wbf + layer_w_off(l), b_of(m, l), last ? nullptr : hout, last ? Y : nullptr,
            last ? m->d_sdo : nullptr, n, kDims[l], kDims[l + 1], last ? 0 : 1, flags);
        am::count_launch();
        std::swap(hin, hout);
    }
}

__global__ void k_scale_out(float* __restrict__ Y, const float* __restrict__ sdo, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * OUT) Y[e] *= sdo[e % OUT];
}

}  // namespace

extern "C" AM_API int am_mlp_create(unsigned long long seed, void* stream, am_mlp** out) {
    if (!out) return mlp_fail(AM_ERR_ARG, "am_mlp_create: NULL output");
    *out = nullptr;
    am_mlp* m = new am_mlp();
    m->st = static_cast<cudaStream_t>(stream);
    const size_t np = n_params_total();
    std::vector<float> p(np, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < NLAYER; ++l) {
        // He initialisation for ReLU layers
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / kDims[l]));
        const size_t o = layer_w_off(l);
        for (size_t k = 0; k < (size_t)kDims[l + 1] * kDims[l]; ++k) p[o + k] = nd(rng) * (l == NLAYER - 1 ? 0.1f : 1.f);
    }
    std::vector<float> one(FEAT, 1.f), zero(FEAT, 0.f);
    auto fail = [&](cudaError_t e) { am_mlp_destroy(m); return mlp_fail(AM_ERR_CUDA, cudaGetErrorString(e)); };
    cudaError_t e;
    if ((e = cudaMalloc(&m->d_p, np * sizeof(float))) || (e = cudaMalloc(&m->d_m, np * sizeof(float))) ||
        (e = cudaMalloc(&m->d_v, np * sizeof(float))) || (e = cudaMalloc(&m->d_g, np * sizeof(float))) ||
        (e = cudaMalloc(&m->d_wbf, np * sizeof(__nv_bfloat16))) || (e = cudaMalloc(&m->d_mu, FEAT * sizeof(float))) ||
        (e = cudaMalloc(&m->d_sd, FEAT * sizeof(float))) || (e = cudaMalloc(&m->d_sdo, OUT * sizeof(float))) ||
        (e = cudaMalloc(&m->d_loss, sizeof(double))) || (e = cudaMalloc(&m->d_flag, sizeof(int))))
        return fail(e);
    cudaMemcpy(m->d_p, p.data(), np * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(m->d_m, 0, np * sizeof(float));
    cudaMemset(m->d_v, 0, np * sizeof(float));
    cudaMemcpy(m->d_mu, zero.data(), FEAT * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(m->d_sd, one.data(), FEAT * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(m->d_sdo, one.data(), OUT * sizeof(float), cudaMemcpyHostToDevice);
    if ((e = cudaGetLastError())) return fail(e);
    *out = m;
    return AM_OK;
}

extern "C" AM_API void am_mlp_destroy(am_mlp* m) {
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    for (void* p : {(void*)m->d_p, (void*)m->d_m, (void*)m->d_v, (void*)m->d_g, (void*)m->d_wbf, (void*)m->d_mu,
                    (void*)m->d_sd, (void*)m->d_sdo, (void*)m->d_X, (void*)m->d_T, (void*)m->d_bx, (void*)m->d_bt,
                    (void*)m->d_dz0, (void*)m->d_dz1, (void*)m->d_h0, (void*)m->d_h1, (void*)m->d_rows,
                    (void*)m->d_loss, (void*)m->d_flag})
        if (p) cudaFree(p);
    for (int l = 0; l <= NLAYER; ++l) {
        if (m->d_z[l]) cudaFree(m->d_z[l]);
        if (m->d_a[l]) cudaFree(m->d_a[l]);
    }
    delete m;
}

extern "C" AM_API int am_mlp_num_params(void) { return (int)n_params_total(); }

extern "C" AM_API int am_mlp_get_params(am_mlp* m, float* p) {
    if (!m || !p) return mlp_fail(AM_ERR_ARG, "am_mlp_get_params: NULL argument");
    MCK(cudaMemcpyAsync(p, m->d_p, n_params_total() * sizeof(float), cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    return AM_OK;
}

extern "C" AM_API int am_mlp_set_params(am_mlp* m, const float* p) {
    if (!m || !p) return mlp_fail(AM_ERR_ARG, "am_mlp_set_params: NULL argument");
    MCK(cudaMemcpyAsync(m->d_p, p, n_params_total() * sizeof(float), cudaMemcpyHostToDevice, m->st));
    MCK(cudaStreamSynchronize(m->st));
    m->bf_valid = false;
    return AM_OK;
}

extern "C" AM_API int am_mlp_set_norm(am_mlp* m, const float* mu, const float* sd, const float* sd_out) {
    if (!m || !mu || !sd || !sd_out) return mlp_fail(AM_ERR_ARG, "am_mlp_set_norm: NULL argument");
    for (int c = 0; c < FEAT; ++c)
        if (!(sd[c] > 0.f)) return mlp_fail(AM_ERR_ARG, "am_mlp_set_norm: sd must be > 0");
    for (int c = 0; c < OUT; ++c)
        if (!(sd_out[c] > 0.f)) return mlp_fail(AM_ERR_ARG, "am_mlp_set_norm: sd_out must be > 0");
    MCK(cudaMemcpyAsync(m->d_mu, mu, FEAT * sizeof(float), cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemcpyAsync(m->d_sd, sd, FEAT * sizeof(float), cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemcpyAsync(m->d_sdo, sd_out, OUT * sizeof(float), cudaMemcpyHostToDevice, m->st));
    MCK(cudaStreamSynchronize(m->st));
    return AM_OK;
}

static int upload_data(am_mlp* m, const float* X, const float* T, int n) {
    if (m->d_X) cudaFree(m->d_X);
    if (m->d_T) cudaFree(m->d_T);
    if (m->d_rows) cudaFree(m->d_rows);
    m->d_X = m->d_T = nullptr;
    m->d_rows = nullptr;
    MCK(cudaMalloc(&m->d_X, (size_t)n * FEAT * sizeof(float)));
    MCK(cudaMalloc(&m->d_T, (size_t)std::max(n, 1) * OUT * sizeof(float)));
    MCK(cudaMalloc(&m->d_rows, (size_t)n * sizeof(int)));
    MCK(cudaMemcpyAsync(m->d_X, X, (size_t)n * FEAT * sizeof(float), cudaMemcpyHostToDevice, m->st));
    if (T) MCK(cudaMemcpyAsync(m->d_T, T, (size_t)n * OUT * sizeof(float), cudaMemcpyHostToDevice, m->st));
    m->data_n = n;
    return AM_OK;
}

extern "C" AM_API int am_mlp_loss_grad(am_mlp* m, const float* X, const float* T, int n, double* loss,
                                       float* grad) {
    if (!m || !X || !T || n <= 0) return mlp_fail(AM_ERR_ARG, "am_mlp_loss_grad: bad argument");
    int rc = ensure_cap(m, n);
    if (rc) return rc;
    rc = upload_data(m, X, T, n);
    if (rc) return rc;
    MCK(cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->st));
    backward32(m, m->d_X, m->d_T, n);
    MCK(cudaGetLastError());
    if (loss) MCK(cudaMemcpyAsync(loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
    if (grad) MCK(cudaMemcpyAsync(grad, m->d_g, n_params_total() * sizeof(float), cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    return AM_OK;
}

extern "C" AM_API int am_mlp_train(am_mlp* m, const float* X, const float* T, int n, int epochs, int batch,
                                   double lr, unsigned long long seed, double* final_loss) {
    if (!m || !X || !T || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.0))
        return mlp_fail(AM_ERR_ARG, "am_mlp_train: bad argument");
    batch = std::min(batch, n);
    int rc = ensure_cap(m, batch);
    if (rc) return rc;
    rc = upload_data(m, X, T, n);
    if (rc) return rc;
    std::vector<int> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::mt19937_64 rng(seed);
    const size_t np = n_params_total();
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        MCK(cudaMemcpyAsync(m->d_rows, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, m->st));
        MCK(cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->st));
        int nb = 0;
        for (int r0 = 0; r0 < n; r0 += batch, ++nb) {
            const int bn = std::min(batch, n - r0);
            k_gather_rows<<<(bn * FEAT + 255) / 256, 256, 0, m->st>>>(m->d_X, m->d_rows + r0, bn, FEAT, m->d_bx);
            k_gather_rows<<<(bn * OUT + 255) / 256, 256, 0, m->st>>>(m->d_T, m->d_rows + r0, bn, OUT, m->d_bt);
            am::count_launch(2);
            backward32(m, m->d_bx, m->d_bt, bn);
            ++m->adam_t;
            const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
            k_adam<<<((int)np + 255) / 256, 256, 0, m->st>>>(m->d_p, m->d_g, m->d_m, m->d_v, (int)np, (float)lr, b1,
                                                             b2, eps, c1, c2);
            am::count_launch();
        }
        double lsum = 0.0;
        MCK(cudaMemcpyAsync(&lsum, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
        MCK(cudaStreamSynchronize(m->st));
        last = lsum / nb;
    }
    MCK(cudaGetLastError());
    m->bf_valid = false;
    if (final_loss) *final_loss = last;
    return AM_OK;
}

extern "C" AM_API int am_mlp_predict(am_mlp* m, const float* X, int n, int bf16, float* Y) {
    if (!m || !X || !Y || n <= 0) return mlp_fail(AM_ERR_ARG, "am_mlp_predict: bad argument");
    int rc = ensure_cap(m, n);
    if (rc) return rc;
    rc = upload_data(m, X, nullptr, n);
    if (rc) return rc;
    float* dY = m->d_bt;
    if (bf16) {
        MCK(cudaMemsetAsync(m->d_flag, 0, sizeof(int), m->st));
        predict_bf16(m, m->d_X, n, dY, m->d_flag);
    } else {
        forward32(m, m->d_X, n);
        MCK(cudaMemcpyAsync(dY, m->d_z[NLAYER], (size_t)n * OUT * sizeof(float), cudaMemcpyDeviceToDevice, m->st));
        k_scale_out<<<(n * OUT + 255) / 256, 256, 0, m->st>>>(dY, m->d_sdo, n);
        am::count_launch();
    }
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(Y, dY, (size_t)n * OUT * sizeof(float), cudaMemcpyDeviceToHost, m->st));
    int flag = 0;
    if (bf16) MCK(cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    if (flag) return mlp_fail(AM_ERR_CUDA, "am_mlp_predict: a tensor-core wait timed out");
    return AM_OK;
}

// ======================================================= solver interface
namespace am {

// x_pc = P~^-1 b into xpc, then the features of all bodies at the current
// pose into dX and, when dT is given, the background-flow targets of the
// solution in d_x (u_ext = M lambda - M~ lambda in d_w, fitted per body).
static int features_dev(am_handle* h, double* xpc, float* dX, float* dT) {
    cudaStream_t s = h->stream;
    pc_apply(h, h->d_b, xpc);
    const double* Upc = xpc + 3 * (size_t)h->Nb;
    k_features<<<(h->M + 127) / 128, 128, 0, s>>>(h->M, h->d_q, h->d_theta, h->d_F, h->d_blob_off, Upc,
                                                  h->d_sys_of_elem + 3 * (size_t)h->Nb, h->d_sys_body_off,
                                                  h->cfg.wall, dX);
    k_body_force<<<(h->M + 127) / 128, 128, 0, s>>>(h->M, h->d_blob_off, xpc, h->d_w);
    k_far_flow<<<(h->M + 127) / 128, 128, 0, s>>>(h->M, h->d_q, h->d_theta, h->d_w,
                                                  h->d_sys_of_elem + 3 * (size_t)h->Nb, h->d_sys_body_off,
                                                  h->d_asm_of_body, h->cfg.wall, rpy_consts<float>(h->prm), dX);
    count_launch(3);
    if (dT) {
        mobility_apply(h, h->d_x, h->d_w, true);
        k_self_sub<<<(h->Nb + 127) / 128, 128, 0, s>>>(h->Nb, h->d_body_of_blob, h->d_blob_off, h->d_r4, h->d_x,
                                                       h->cfg.wall, rpy_consts<double>(h->prm), h->d_w);
        k_flow_fit<<<h->M, 128, 0, s>>>(h->d_blob_off, h->d_rho, h->d_theta, h->d_w, dT);
        count_launch(2);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int learned_x0(am_handle* h, double* x) {
    am_mlp* m = h->mlp;
    cudaStream_t s = h->stream;
    double* xpc = h->d_dx;
    if (ensure_cap(m, h->M)) return 1;
    if (features_dev(h, xpc, m->d_bx, nullptr)) return 1;
    cudaStream_t keep = m->st;
    m->st = s;
    predict_bf16(m, m->d_bx, h->M, m->d_bt, h->d_flags);
    m->st = keep;
    // right-hand side with the predicted background flow moved over, then
    // the block-diagonal solve (which keeps C U = B)
    cudaMemcpyAsync(h->d_rir, h->d_b, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    k_flow_rhs<<<(h->Nb + 127) / 128, 128, 0, s>>>(h->Nb, h->d_body_of_blob, h->d_rho, h->d_theta, m->d_bt,
                                                   h->d_b, h->d_rir);
    count_launch();
    pc_apply(h, h->d_rir, x);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int learned_features(am_handle* h, float* X, float* T) {
    cudaStream_t s = h->stream;
    float *dX = nullptr, *dT = nullptr;
    if (cudaMalloc(&dX, (size_t)h->M * FEAT * sizeof(float)) != cudaSuccess) return 1;
    if (T && cudaMalloc(&dT, (size_t)h->M * OUT * sizeof(float)) != cudaSuccess) {
        cudaFree(dX);
        return 1;
    }
    int rc = features_dev(h, h->d_dx, dX, dT);
    if (!rc) {
        cudaMemcpyAsync(X, dX, (size_t)h->M * FEAT * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (T) cudaMemcpyAsync(T, dT, (size_t)h->M * OUT * sizeof(float), cudaMemcpyDeviceToHost, s);
        rc = cudaStreamSynchronize(s) != cudaSuccess;
    }
    cudaFree(dX);
    if (dT) cudaFree(dT);
    return rc;
}

}  // namespace am

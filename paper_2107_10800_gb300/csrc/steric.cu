// Steric repulsion (Sec. 5.3 adds one between bacteria and with the wall
// without giving its form; this is the library's reading):
//   blobs i, j of different articulated bodies at distance r < r_c:
//     U = eps (1 + (2a - r) / b) for r < 2a,  eps exp((2a - r) / b) otherwise
//   every blob at height h above a wall:
//     U_w = eps_w (1 + (a - h) / b_w) for h < a,  eps_w exp((a - h) / b_w) otherwise
// Blob forces f = -grad U; the bodies receive K^T f (force, and torque about
// the tracking point), which is subtracted from the force rows of the
// right-hand side b = (u_s, -F, B) after it is formed.
//
// Pairs: one thread per target blob, source tiles of 128 blobs over the
// union of the systems of the block's targets; a candidate is screened with
// the FP32 hi + lo position difference (error ~1e-7 of the distance) against
// a slightly enlarged cutoff and accepted, with its force, in FP64.
#include "am_internal.cuh"
#include "ops.cuh"

#include <climits>

namespace am {

namespace {

__global__ void __launch_bounds__(kThreads)
k_steric_blob(int Nb, const double4_32a* __restrict__ r4, const float4* __restrict__ hi,
              const float4* __restrict__ lo, const int* __restrict__ body_of_blob,
              const int* __restrict__ asm_of_body, const int* __restrict__ sys_of_blob,
              const int* __restrict__ sys_blob0, const int* __restrict__ sys_nb, double a, double eps, double b,
              double rc, int wall, double eps_w, double b_w, double* __restrict__ f) {
    __shared__ float4 sh[kTile];
    __shared__ float4 so[kTile];
    __shared__ int sasm[kTile];
    __shared__ int s_lo, s_hi;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    const bool live = i < Nb;
    int j0 = INT_MAX, j1 = 0, ai = -1;
    float4 xh = make_float4(0.f, 0.f, 0.f, 0.f), xl = xh;
    double4_32a xi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (live) {
        const int s = sys_of_blob[i];
        j0 = sys_blob0[s];
        j1 = j0 + sys_nb[s];
        ai = asm_of_body[body_of_blob[i]];
        xh = hi[i];
        xl = lo[i];
        xi = r4[i];
    }
    if (threadIdx.x == 0) { s_lo = INT_MAX; s_hi = 0; }
    __syncthreads();
    if (live) { atomicMin(&s_lo, j0); atomicMax(&s_hi, j1); }
    __syncthreads();
    const int lo_all = s_lo, hi_all = s_hi;
    const float rcs = (float)(rc * (1.0 + 1e-4) + 1e-6);
    const float rc2f = rcs * rcs;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int jt = lo_all; jt < hi_all; jt += kTile) {
        const int cnt = min(kTile, hi_all - jt);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int j = jt + threadIdx.x;
            sh[threadIdx.x] = hi[j];
            so[threadIdx.x] = lo[j];
            sasm[threadIdx.x] = asm_of_body[body_of_blob[j]];
        }
        __syncthreads();
        if (!live) continue;
        for (int q = 0; q < cnt; ++q) {
            const int j = jt + q;
            if (j < j0 || j >= j1 || sasm[q] == ai) continue;
            const float4 h = sh[q], o = so[q];
            const float dx = (xh.x - h.x) + (xl.x - o.x), dy = (xh.y - h.y) + (xl.y - o.y),
                        dz = (xh.z - h.z) + (xl.z - o.z);
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= rc2f) continue;
            const double4_32a xj = r4[j];
            const double ex = xi.x - xj.x, ey = xi.y - xj.y, ez = xi.z - xj.z;
            const double r = sqrt(ex * ex + ey * ey + ez * ez);
            if (!(r < rc) || !(r > 0.0)) continue;
            // -dU/dr: eps / b inside contact, eps / b exp((2a - r) / b) outside
            const double mag = (r < 2.0 * a) ? eps / b : eps / b * exp((2.0 * a - r) / b);
            const double c = mag / r;
            fx = fma(c, ex, fx);
            fy = fma(c, ey, fy);
            fz = fma(c, ez, fz);
        }
    }
    if (!live) return;
    if (wall) {
        const double hgt = xi.z;
        fz += (hgt < a) ? eps_w / b_w : eps_w / b_w * exp((a - hgt) / b_w);
    }
    f[3 * (size_t)i] = fx;
    f[3 * (size_t)i + 1] = fy;
    f[3 * (size_t)i + 2] = fz;
}

// per body: K^T f (force and torque about the tracking point) subtracted
// from the body rows of b = (u_s, -F, B)
__global__ void k_steric_body(int M, int Nb, const int* __restrict__ blob_off, const double4_32a* __restrict__ d4,
                              const double* __restrict__ f, double* __restrict__ bvec) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    double F[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blob_off[p]; i < blob_off[p + 1]; ++i) {
        const double fx = f[3 * (size_t)i], fy = f[3 * (size_t)i + 1], fz = f[3 * (size_t)i + 2];
        const double4_32a d = d4[i];
        F[0] += fx; F[1] += fy; F[2] += fz;
        F[3] += d.y * fz - d.z * fy;
        F[4] += d.z * fx - d.x * fz;
        F[5] += d.x * fy - d.y * fx;
    }
    double* o = bvec + 3 * (size_t)Nb + 6 * (size_t)p;
    for (int c = 0; c < 6; ++c) o[c] -= F[c];
}

}  // namespace

void steric_apply(am_handle* h) {
    if (!h->steric_on || h->Nb == 0) return;
    cudaStream_t s = h->stream;
    const int grid = (h->Nb + kThreads - 1) / kThreads;
    k_steric_blob<<<grid, kThreads, 0, s>>>(h->Nb, h->d_r4, h->d_rhi, h->d_rlo, h->d_body_of_blob,
                                            h->d_asm_of_body, h->d_sys_of_blob, h->d_sys_blob0, h->d_sys_nb,
                                            h->cfg.blob_radius, h->st_eps, h->st_b, h->st_rc, h->cfg.wall,
                                            h->st_eps_w, h->st_b_w, h->d_fst);
    k_steric_body<<<(h->M + 127) / 128, 128, 0, s>>>(h->M, h->Nb, h->d_blob_off, h->d_d4, h->d_fst, h->d_b);
    count_launch(2);
}

}  // namespace am

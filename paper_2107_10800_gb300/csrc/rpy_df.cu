// The blob mobility product u = M lambda (Sec. 2.3, Eq. RPY; wall: the
// Rotne-Prager-Blake tensor) with the pair terms in double-float arithmetic
// (df64.cuh) on the FP32 pipes.  Same closed forms as rpy_pair.cuh (free
// space: far r >= 2a, overlapping r < 2a, self; wall: the fused free-space
// and image pair), same work items as the FP64 and mixed products; each tile of
// 128 sources is summed in df and folded into FP64.  Relative error per pair
// a few units of 2^-44, against 2^-53 for FP64 and 2^-24 for the mixed
// product, at about an eighth of the FP64 cost: the mixed solver uses it for
// its outer residuals.
#include "am_internal.cuh"
#include "df64.cuh"
#include "ops.cuh"

namespace am {

namespace {

// constants of the pair terms as df (see RpyK)
struct RpyDf {
    df a2, four_a2, kf2, kf3, kn0, kn1, kn2;
    df wc1, w2a2, wc2, wc3, nwa4, wi2;  // wall polynomial coefficients (pair_wall_r2)
    double A1;
};

RpyDf rpy_df_consts(const RpyParams& q) {
    auto split = [](double x) {
        const float h = (float)x;
        return df{h, (float)(x - (double)h)};
    };
    RpyDf k;
    k.a2 = split(q.a2);
    k.four_a2 = split(q.four_a2);
    k.kf2 = split(2.0 * q.a2 / 3.0);
    k.kf3 = split(2.0 * q.a2);
    k.kn0 = split(4.0 / (3.0 * q.a));
    k.kn1 = split(9.0 / (32.0 * q.a));
    k.kn2 = split(1.0 / (8.0 * q.a2));
    const double a4 = q.a2 * q.a2;
    k.wc1 = split(-2.0 * q.a2 / 3.0);
    k.w2a2 = split(2.0 * q.a2);
    k.wc2 = split(2.0 * a4 / 3.0);
    k.wc3 = split(-10.0 * a4 / 3.0);
    k.nwa4 = split(-20.0 * a4 / 3.0);
    k.wi2 = split(-4.0 * a4 / 3.0);
    k.A1 = q.inv8pieta;
    return k;
}

// the free-space coefficients c1, c2 at squared distance r2 (rpy_pair.cuh)
__device__ __forceinline__ void free_coefs_df(df r2, const RpyDf& k, df& c1, df& c2) {
    const df one{1.0f, 0.0f};
    if (df_ge(r2, k.four_a2)) {
        const df ri = df_rsqrt(r2);
        const df ri2 = df_mul(ri, ri);
        c1 = df_mul(ri, df_fma(k.kf2, ri2, one));
        c2 = df_mul(df_mul(ri, ri2), df_fma(df_neg(k.kf3), ri2, one));
    } else if (r2.h > 0.0f) {
        const df ri = df_rsqrt(r2);
        const df r = df_mul(r2, ri);
        c1 = df_mul(k.kn0, df_fma(df_neg(k.kn1), r, one));
        c2 = df_mul(k.kn2, ri);
    } else {
        c1 = k.kn0;
        c2 = df{0.0f, 0.0f};
    }
}

// u/A1 += c1 lambda + c2 d (d . lambda), the free-space pair of rpy_pair.cuh
__device__ __forceinline__ void pair_free_df(df dx, df dy, df dz, df r2, df lx, df ly, df lz,
                                             const RpyDf& k, df& ux, df& uy, df& uz) {
    df c1, c2;
    free_coefs_df(r2, k, c1, c2);
    const df sdl = df_mul(c2, df_fma(dx, lx, df_fma(dy, ly, df_mul(dz, lz))));
    ux = df_fma(c1, lx, df_fma(sdl, dx, ux));
    uy = df_fma(c1, ly, df_fma(sdl, dy, uy));
    uz = df_fma(c1, lz, df_fma(sdl, dz, uz));
}

// Free-space pair plus wall image of one source in double-float: the same
// operations as pair_wall_r2 of rpy_pair.cuh (polynomials in w = s^2 on the
// unnormalised image vector R = (dx, dy, Rz)), scalings by small integers as
// exact (powers of two) or single-float multiplies.  h2 = twice the source
// height, nx3 = minus the target height.
__device__ __forceinline__ void pair_wall_df(df dx, df dy, df dz, df rxy2, df r2, df Rz, df h2, df nx3, df lx,
                                             df ly, df lz, const RpyDf& k, df& ux, df& uy, df& uz) {
    const df Rz2 = df_mul(Rz, Rz);
    const df dlxy = df_fma(dx, lx, df_mul(dy, ly));
    const df Df = df_fma(dz, lz, dlxy);  // d . lambda
    const df Di = df_fma(Rz, lz, dlxy);  // R . lambda
    df c1f, c2f;
    free_coefs_df(r2, k, c1f, c2f);
    const df sdl = df_mul(c2f, Df);
    const df s = df_rsqrt(df_add(rxy2, Rz2));
    const df w = df_mul(s, s), s3 = df_mul(s, w), w2 = df_mul(w, w);
    const df c1 = df_fma(h2, nx3, k.wc1);
    const df c2 = df_fma(Rz2, k.w2a2, k.wc2);
    const df c3 = df_mul(Rz2, k.wc3);
    const df x1 = df_fma(w, c3, c2);
    const df cI = df_fma(w, df_fma(w, x1, c1), df{-1.0f, 0.0f});
    const df y = df_fma(w, c3, x1);   // c2 + 2 w c3
    const df yz = df_fma(w, c3, y);   // c2 + 3 w c3
    // cRR = -4 - 3 cI - 2 w^2 y
    const df cRR = df_add(df_scale2(df_mul(w2, y), -2.0f), df_add(df_mul_f(cI, -3.0f), df{-4.0f, 0.0f}));
    const df A4w2n = df_mul(w2, k.nwa4);  // -20/3 a^4 w^2
    // inner = -2 cRR - 2 - A4w2n
    const df inner = df_add(df_add(df_scale2(cRR, -2.0f), df{-2.0f, 0.0f}), df_neg(A4w2n));
    const df P = df_mul(s3, df_fma(cRR, Di, df_mul(df_fma(Rz, inner, h2), lz)));
    const df Q = df_mul(s3, df_fma(h2, Df, df_fma(df_mul(A4w2n, Rz), Di,
                                                   df_mul(df_mul(w, df_add(df_scale2(yz, -2.0f), k.wi2)), lz))));
    const df cc = df_fma(s, cI, c1f);
    const df pp = df_add(sdl, P);
    ux = df_fma(cc, lx, df_fma(pp, dx, ux));
    uy = df_fma(cc, ly, df_fma(pp, dy, uy));
    uz = df_fma(cc, lz, df_fma(sdl, dz, df_fma(P, Rz, df_add(uz, Q))));
}

// Both directions of one pair in double-float (the operations of
// pair_wall_sym in rpy_pair.cuh): u += M lambda_j at the target, v += M^T
// mu_i at the source.
template <bool WALL>
__device__ __forceinline__ void pair_sym_df(df dx, df dy, df dz, df rxy2, df r2, df Rz, df h2, df nx3, df lx,
                                            df ly, df lz, df mx, df my, df mz, const RpyDf& k, df& ux, df& uy,
                                            df& uz, df& vx, df& vy, df& vz) {
    df c1f, c2f;
    free_coefs_df(r2, k, c1f, c2f);
    const df dlxy = df_fma(dx, lx, df_mul(dy, ly));
    const df Df = df_fma(dz, lz, dlxy);
    const df dmxy = df_fma(dx, mx, df_mul(dy, my));
    const df Dfm = df_fma(dz, mz, dmxy);
    if (!WALL) {
        const df sl = df_mul(c2f, Df), sm = df_mul(c2f, Dfm);
        ux = df_fma(c1f, lx, df_fma(sl, dx, ux));
        uy = df_fma(c1f, ly, df_fma(sl, dy, uy));
        uz = df_fma(c1f, lz, df_fma(sl, dz, uz));
        vx = df_fma(c1f, mx, df_fma(sm, dx, vx));
        vy = df_fma(c1f, my, df_fma(sm, dy, vy));
        vz = df_fma(c1f, mz, df_fma(sm, dz, vz));
        return;
    }
    const df Rz2 = df_mul(Rz, Rz);
    const df s = df_rsqrt(df_add(rxy2, Rz2));
    const df w = df_mul(s, s), s3 = df_mul(s, w), w2 = df_mul(w, w);
    const df c1 = df_fma(h2, nx3, k.wc1);
    const df c2 = df_fma(Rz2, k.w2a2, k.wc2);
    const df c3 = df_mul(Rz2, k.wc3);
    const df x1 = df_fma(w, c3, c2);
    const df cI = df_fma(w, df_fma(w, x1, c1), df{-1.0f, 0.0f});
    const df y = df_fma(w, c3, x1);
    const df yz = df_fma(w, c3, y);
    const df cRR = df_add(df_scale2(df_mul(w2, y), -2.0f), df_add(df_mul_f(cI, -3.0f), df{-4.0f, 0.0f}));
    const df A4w2n = df_mul(w2, k.nwa4);
    const df inner = df_add(df_add(df_scale2(cRR, -2.0f), df{-2.0f, 0.0f}), df_neg(A4w2n));
    const df g = df_fma(Rz, inner, h2);
    const df phi = df_mul(w, df_add(df_scale2(yz, -2.0f), k.wi2));
    const df cc = df_fma(s, cI, c1f);
    const df s3cRR = df_mul(s3, cRR), s3g = df_mul(s3, g), s3h2 = df_mul(s3, h2);
    const df s3A = df_mul(s3, df_mul(A4w2n, Rz)), s3phi = df_mul(s3, phi);
    {
        const df Di = df_fma(Rz, lz, dlxy);
        const df sdl = df_mul(c2f, Df);
        const df P = df_fma(s3cRR, Di, df_mul(s3g, lz));
        const df Q = df_fma(s3h2, Df, df_fma(s3A, Di, df_mul(s3phi, lz)));
        const df pp = df_add(sdl, P);
        ux = df_fma(cc, lx, df_fma(pp, dx, ux));
        uy = df_fma(cc, ly, df_fma(pp, dy, uy));
        uz = df_fma(cc, lz, df_fma(sdl, dz, df_fma(P, Rz, df_add(uz, Q))));
    }
    {
        const df Di = df_fma(Rz, mz, dmxy);
        const df cd = df_fma(c2f, Dfm, df_mul(s3h2, mz));
        const df P = df_fma(s3cRR, Di, df_mul(s3A, mz));
        const df Q = df_fma(s3g, Di, df_mul(s3phi, mz));
        const df pp = df_add(cd, P);
        vx = df_fma(cc, mx, df_fma(pp, dx, vx));
        vy = df_fma(cc, my, df_fma(pp, dy, vy));
        vz = df_fma(cc, mz, df_fma(cd, dz, df_fma(P, Rz, df_add(vz, Q))));
    }
}

__device__ __forceinline__ df df_shfl(df x, int src) {
    return df{__shfl_sync(0xffffffffu, x.h, src), __shfl_sync(0xffffffffu, x.l, src)};
}

// Symmetric double-float product on the handle's tile pairs of 128 blobs
// (the scheme of rpy_sym_f64: 32 x 32 warp tiles, the source's column sum
// carried lane to lane, steps 1..16 on the diagonal of a diagonal item);
// warp-tile sums in double-float, added in FP64 across warps in a fixed
// order.
template <bool WALL>
__global__ void __launch_bounds__(kThreads)
rpy_sym_df(const float4* __restrict__ hi, const float4* __restrict__ lo, const double* __restrict__ lam,
           double* __restrict__ part, const SymItem* __restrict__ items, int n_items, int* __restrict__ counter,
           RpyDf k) {
    constexpr int T = 128, NSUB = 4, NWT = 16;
    __shared__ float4 shI[T], soI[T], shJ[T], soJ[T];
    __shared__ float4 lhI[T], llI[T], lhJ[T], llJ[T];
    __shared__ double up[NWT][32][3], vp[NWT][32][3];
    __shared__ int s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int round = 0;; ++round) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = round == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(counter, 1);
        __syncthreads();
        const int itn = s_item;
        if (itn >= n_items) break;
        const SymItem m = items[itn];
        const bool diag = m.ti == m.tj;
        {
            const int q = threadIdx.x;
            const bool oi = q < m.ni, oj = q < m.nj;
            shI[q] = oi ? hi[m.i0 + q] : make_float4(0.f, 0.f, 1.f, 0.f);
            soI[q] = oi ? lo[m.i0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
            shJ[q] = oj ? hi[m.j0 + q] : make_float4(0.f, 0.f, 1.f, 0.f);
            soJ[q] = oj ? lo[m.j0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
            df a{0.f, 0.f}, b{0.f, 0.f}, c{0.f, 0.f};
            if (oi) {
                a = df_from(lam[3 * (size_t)(m.i0 + q)]);
                b = df_from(lam[3 * (size_t)(m.i0 + q) + 1]);
                c = df_from(lam[3 * (size_t)(m.i0 + q) + 2]);
            }
            lhI[q] = make_float4(a.h, b.h, c.h, 0.f);
            llI[q] = make_float4(a.l, b.l, c.l, 0.f);
            a = df{0.f, 0.f}; b = df{0.f, 0.f}; c = df{0.f, 0.f};
            if (oj) {
                a = df_from(lam[3 * (size_t)(m.j0 + q)]);
                b = df_from(lam[3 * (size_t)(m.j0 + q) + 1]);
                c = df_from(lam[3 * (size_t)(m.j0 + q) + 2]);
            }
            lhJ[q] = make_float4(a.h, b.h, c.h, 0.f);
            llJ[q] = make_float4(a.l, b.l, c.l, 0.f);
        }
        __syncthreads();
        for (int wt = warp; wt < NWT; wt += 4) {
            const int a = wt / NSUB, b = wt % NSUB;
            df ux{0.f, 0.f}, uy{0.f, 0.f}, uz{0.f, 0.f}, vx{0.f, 0.f}, vy{0.f, 0.f}, vz{0.f, 0.f};
            if (!(diag && b < a)) {
                const bool self_tile = diag && a == b;
                const int t = 32 * a + lane;
                const bool ti_ok = t < m.ni;
                const float4 xh = shI[t], xl = soI[t], mh = lhI[t], ml = llI[t];
                const df xx{xh.x, xl.x}, xy{xh.y, xl.y}, xz{xh.z, xl.z};
                const df nx3 = df_neg(xz);
                const df mx{mh.x, ml.x}, my{mh.y, ml.y}, mz{mh.z, ml.z};
#pragma unroll 1
                for (int step = 0; step < 32; ++step) {
                    const int q = 32 * b + ((lane + step) & 31);
                    const bool pair_ok = ti_ok && q < m.nj &&
                                         (!self_tile || (step >= 1 && (step < 16 || (step == 16 && lane < 16))));
                    if (pair_ok || (self_tile && step == 0 && ti_ok)) {
                        const float4 yh = shJ[q], yl = soJ[q], lh = lhJ[q], ll = llJ[q];
                        const df lx{lh.x, ll.x}, ly{lh.y, ll.y}, lz{lh.z, ll.z};
                        const df yz{yh.z, yl.z};
                        const df dx = df_sub(xx, df{yh.x, yl.x});
                        const df dy = df_sub(xy, df{yh.y, yl.y});
                        const df dz = df_sub(xz, yz);
                        const df rxy2 = df_fma(dx, dx, df_mul(dy, dy));
                        const df r2 = df_fma(dz, dz, rxy2);
                        if (pair_ok) {
                            pair_sym_df<WALL>(dx, dy, dz, rxy2, r2, df_add(xz, yz), df_scale2(yz, 2.0f), nx3, lx, ly,
                                              lz, mx, my, mz, k, ux, uy, uz, vx, vy, vz);
                        } else if (WALL) {  // the self term
                            pair_wall_df(dx, dy, dz, rxy2, r2, df_add(xz, yz), df_scale2(yz, 2.0f), nx3, lx, ly, lz,
                                         k, ux, uy, uz);
                        } else {
                            pair_free_df(dx, dy, dz, r2, lx, ly, lz, k, ux, uy, uz);
                        }
                    }
                    const int src = (lane + 1) & 31;
                    vx = df_shfl(vx, src);
                    vy = df_shfl(vy, src);
                    vz = df_shfl(vz, src);
                }
            }
            up[wt][lane][0] = df_to(ux); up[wt][lane][1] = df_to(uy); up[wt][lane][2] = df_to(uz);
            vp[wt][lane][0] = df_to(vx); vp[wt][lane][1] = df_to(vy); vp[wt][lane][2] = df_to(vz);
        }
        __syncthreads();
        double* rowo = part + m.poff + (long long)m.tj * m.n3 + 3 * (long long)(m.i0 - m.tbase);
        double* colo = part + m.poff + (long long)m.ti * m.n3 + 3 * (long long)(m.j0 - m.tbase);
        {
            const int t = threadIdx.x, a = t >> 5, l = t & 31;
            if (t < m.ni) {
                double sx = 0.0, sy = 0.0, sz = 0.0;
                for (int b = 0; b < NSUB; ++b) {
                    sx += up[a * NSUB + b][l][0]; sy += up[a * NSUB + b][l][1]; sz += up[a * NSUB + b][l][2];
                }
                if (diag)
                    for (int a2 = 0; a2 < NSUB; ++a2) {
                        sx += vp[a2 * NSUB + a][l][0]; sy += vp[a2 * NSUB + a][l][1]; sz += vp[a2 * NSUB + a][l][2];
                    }
                rowo[3 * t] = k.A1 * sx; rowo[3 * t + 1] = k.A1 * sy; rowo[3 * t + 2] = k.A1 * sz;
            }
            if (!diag && t < m.nj) {
                double sx = 0.0, sy = 0.0, sz = 0.0;
                for (int a2 = 0; a2 < NSUB; ++a2) {
                    sx += vp[a2 * NSUB + a][l][0]; sy += vp[a2 * NSUB + a][l][1]; sz += vp[a2 * NSUB + a][l][2];
                }
                colo[3 * t] = k.A1 * sx; colo[3 * t + 1] = k.A1 * sy; colo[3 * t + 2] = k.A1 * sz;
            }
        }
    }
    item_queue_done(counter);
}

template <bool WALL>
__global__ void __launch_bounds__(kThreads)
rpy_items_df(const float4* __restrict__ hi, const float4* __restrict__ lo, const double* __restrict__ lam,
             double* __restrict__ part, const MvItem* __restrict__ items, int n_items,
             int* __restrict__ counter, RpyDf k) {
    __shared__ float4 sh[kTile];
    __shared__ float4 so[kTile];
    __shared__ float4 slh[kTile];
    __shared__ float4 sll[kTile];
    __shared__ int s_item;
    for (int round = 0;; ++round) {
        // first item = the block's own index, later ones from the queue
        __syncthreads();
        if (threadIdx.x == 0) s_item = round == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(counter, 1);
        __syncthreads();
        const int itn = s_item;
        if (itn >= n_items) break;
        const MvItem m = items[itn];
        // items built for two targets per thread span 2 x 128 targets
        for (int tb = m.t0; tb < m.t1; tb += kThreads) {
            const int i = tb + threadIdx.x;
            const float4 xh = (i < m.t1) ? hi[i] : make_float4(0.f, 0.f, 1.f, 0.f);
            const float4 xl = (i < m.t1) ? lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            const df xx{xh.x, xl.x}, xy{xh.y, xl.y}, xz{xh.z, xl.z};
            const df nx3 = df_neg(xz);
            double U0 = 0.0, U1 = 0.0, U2 = 0.0;
            // warps with no target of the item only help stage the sources
            const bool warp_live = tb + (int)(threadIdx.x & ~31u) < m.t1;
            for (int jt = m.j0; jt < m.j1; jt += kTile) {
                const int cnt = min(kTile, m.j1 - jt);
                __syncthreads();
                if (threadIdx.x < cnt) {
                    const int j = jt + threadIdx.x;
                    sh[threadIdx.x] = hi[j];
                    so[threadIdx.x] = lo[j];
                    const df a = df_from(lam[3 * (size_t)j]), b = df_from(lam[3 * (size_t)j + 1]),
                             c = df_from(lam[3 * (size_t)j + 2]);
                    slh[threadIdx.x] = make_float4(a.h, b.h, c.h, 0.f);
                    sll[threadIdx.x] = make_float4(a.l, b.l, c.l, 0.f);
                }
                __syncthreads();
                if (!warp_live) continue;
                df ux{0.f, 0.f}, uy{0.f, 0.f}, uz{0.f, 0.f};
                for (int q = 0; q < cnt; ++q) {
                    const float4 yh = sh[q], yl = so[q], lh = slh[q], ll = sll[q];
                    const df lx{lh.x, ll.x}, ly{lh.y, ll.y}, lz{lh.z, ll.z};
                    const df yz{yh.z, yl.z};
                    const df dx = df_sub(xx, df{yh.x, yl.x});
                    const df dy = df_sub(xy, df{yh.y, yl.y});
                    const df dz = df_sub(xz, yz);
                    if (WALL) {
                        const df rxy2 = df_fma(dx, dx, df_mul(dy, dy));
                        pair_wall_df(dx, dy, dz, rxy2, df_fma(dz, dz, rxy2), df_add(xz, yz), df_scale2(yz, 2.0f),
                                     nx3, lx, ly, lz, k, ux, uy, uz);
                    } else {
                        const df r2 = df_fma(dx, dx, df_fma(dy, dy, df_mul(dz, dz)));
                        pair_free_df(dx, dy, dz, r2, lx, ly, lz, k, ux, uy, uz);
                    }
                }
                U0 += df_to(ux);
                U1 += df_to(uy);
                U2 += df_to(uz);
            }
            if (i < m.t1) {
                double* o = part + m.pbase + 3 * (size_t)(i - m.tbase);
                o[0] = k.A1 * U0; o[1] = k.A1 * U1; o[2] = k.A1 * U2;
            }
        }
    }
    item_queue_done(counter);
}

}  // namespace

int sym_df_resident_grid(bool wall) {
    int per = 0;
    cudaError_t e = wall ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rpy_sym_df<true>, kThreads, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rpy_sym_df<false>, kThreads, 0);
    if (e != cudaSuccess || per <= 0) per = 2;
    return per * num_sms();
}

int df_resident_grid(bool wall) {
    int per = 0;
    cudaError_t e = wall ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rpy_items_df<true>, kThreads, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rpy_items_df<false>, kThreads, 0);
    if (e != cudaSuccess || per <= 0) per = 4;
    return per * num_sms();
}

// Partial sums of u = M lambda for all systems with double-float pair terms;
// positions from the hi/lo arrays.
void launch_items_df(am_handle* h, const double* lam) {
    cudaStream_t st = h->stream;  // the queue counter is zero (reset by the last launch's last block)
    const MvItem* items = static_cast<const MvItem*>(h->d_items);
    const RpyDf k = rpy_df_consts(h->prm);
    if (h->n_sym > 0 && h->sym_nsub == 4) {  // tile pairs of 128: the symmetric double-float product
        const SymItem* si = static_cast<const SymItem*>(h->d_sym_items);
        if (h->cfg.wall)
            rpy_sym_df<true><<<h->mv_gridsymdf, kThreads, 0, st>>>(h->d_rhi, h->d_rlo, lam, h->d_mv, si, h->n_sym,
                                                                   h->d_item_counter, k);
        else
            rpy_sym_df<false><<<h->mv_gridsymdf, kThreads, 0, st>>>(h->d_rhi, h->d_rlo, lam, h->d_mv, si, h->n_sym,
                                                                    h->d_item_counter, k);
        count_launch();
        return;
    }
    if (h->cfg.wall)
        rpy_items_df<true><<<h->mv_griddf, kThreads, 0, st>>>(h->d_rhi, h->d_rlo, lam, h->d_mv, items, h->n_items,
                                                             h->d_item_counter, k);
    else
        rpy_items_df<false><<<h->mv_griddf, kThreads, 0, st>>>(h->d_rhi, h->d_rlo, lam, h->d_mv, items,
                                                              h->n_items, h->d_item_counter, k);
    count_launch();
}

}  // namespace am

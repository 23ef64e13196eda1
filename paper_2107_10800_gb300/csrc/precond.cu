// Block-diagonal preconditioner (Sec. 3.1): the exact solution of the
// approximate problem Eq. precond, where M keeps only same-body blocks M^(pp).
//
// Build, per body p (one block): M^(pp) from the pair tensors, its explicit
// inverse by blocked Cholesky, blocked triangular inverse and X^T X on 32 x 32
// shared-memory tiles, Y_p = (M^(pp))^-1 K_p, S_p = K_p^T Y_p and
// N~_p = S_p^-1 (a body of more than two tiles takes a cluster of CTAs when
// such bodies are too few to fill the GPU).  Per articulated body a (one
// block): H_a = C_a N~_a C_a^T and its generalised inverse G~_a
// (Eq. block_diag_const_res) by symmetric pivoted Cholesky (32-column panels,
// then the blocked inverse of the rank-r factor):
// H(perm) = L L^T with L of rank r gives
// G~ = perm [(L11 L11^T)^-1 0; 0 0] perm^T, which solves H phi = c exactly for
// every c in range(H) = range(C_a).
//
// Apply, for r = (r1, r2, r3):
//   w = M~^-1 r1;  U^ = N~ (-r2 - K^T w), with K^T w = Y^T r1
//   phi = G~ (r3 - C U^)
//   U = U^ + N~ C^T phi;  lambda = w + Y U  (= M~^-1 (r1 + K U)).
// The dense products run over flattened (body, 32-row chunk) and
// (articulated body, 32-row chunk) work items so that every SM gets work.
//
// Matrices are stored in T = double (FP64 path) or float (mixed path, where
// the preconditioner only steers the inner iterations); vectors are FP64.
#include "am_internal.cuh"
#include "dev_util.cuh"
#include "ops.cuh"
#include "rpy_pair.cuh"

#include <algorithm>

namespace am {

constexpr int kRows = 32;  // rows per apply work item

// One body per team: body_list[blockIdx.x / team size]; a cluster team
// splits the pair tensors, the tiles of the blocked inverse and the rows of
// Y among its CTAs, and its first CTA forms N~_p.
template <class T, class Team>
__global__ void __launch_bounds__(kPcThreads)
k_pcb_build(const int* __restrict__ body_list, const int* __restrict__ blob_off,
            const double4_32a* __restrict__ r4, const double4_32a* __restrict__ d4,
            const long long* __restrict__ moff, T* __restrict__ minv, T* __restrict__ work,
            T* __restrict__ Y, double* __restrict__ Nt, RpyK<T> prm, int wall, int* flags) {
    __shared__ double sh[64];
    __shared__ PcTiles<T> tiles;
    __shared__ int s_bad;
    const Team team;
    const int tr = team.rank(), ts = team.size();
    const int b = body_list[blockIdx.x / ts];
    const int i0 = blob_off[b];
    const int nbl = blob_off[b + 1] - i0;
    const int m = 3 * nbl;
    if (threadIdx.x == 0) s_bad = 0;
    T* A = minv + moff[b];
    T* L = work + 2 * moff[b];
    T* X = L + (size_t)m * m;
    // the lower triangle of M^(pp) (blob pairs ti >= sj, the factorisation
    // reads no entry above the diagonal), pair tensors in the storage
    // precision from FP64 differences
    for (int idx = threadIdx.x + tr * blockDim.x; idx < nbl * nbl; idx += blockDim.x * ts) {
        const int ti = idx / nbl, sj = idx % nbl;
        if (sj > ti) continue;
        const double4_32a x = r4[i0 + ti], y = r4[i0 + sj];
        T Tt[9];
        pair_tensor<T>((T)(x.x - y.x), (T)(x.y - y.y), (T)(x.z - y.z), (T)x.z, (T)y.z, prm, wall, Tt);
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) L[(size_t)(3 * ti + a) * m + 3 * sj + c] = Tt[3 * a + c];
    }
    team.sync();
    // (M^(pp))^-1 by blocked Cholesky, triangular inverse and X^T X
    blocked_spd_inverse(L, X, A, m, tiles, &s_bad, team);
    if (s_bad) {
        if (threadIdx.x == 0 && tr == 0) atomicOr(flags, kFlagSingular);
        return;
    }
    T* Yb = Y + 18 * (size_t)i0;
    for (int i = threadIdx.x + tr * blockDim.x; i < m; i += blockDim.x * ts) {
        double y[6] = {0, 0, 0, 0, 0, 0};
        for (int bb = 0; bb < nbl; ++bb) {
            const double v[3] = {(double)A[(size_t)(3 * bb) * m + i], (double)A[(size_t)(3 * bb + 1) * m + i],
                                 (double)A[(size_t)(3 * bb + 2) * m + i]};
            const double4_32a dd = d4[i0 + bb];
            const double d[3] = {dd.x, dd.y, dd.z};
            double c[3];
            cross3(d, v, c);
            for (int a = 0; a < 3; ++a) { y[a] += v[a]; y[3 + a] += c[a]; }
        }
        for (int a = 0; a < 6; ++a) Yb[6 * (size_t)i + a] = (T)y[a];
    }
    team.sync();
    if (tr != 0) return;
    if (threadIdx.x < 36) {
        const int c = threadIdx.x / 6, e = threadIdx.x % 6;
        double s = 0.0;
        for (int bb = 0; bb < nbl; ++bb) {
            if (c < 3) {
                s += (double)Yb[6 * (size_t)(3 * bb + c) + e];
            } else {
                const double v[3] = {(double)Yb[6 * (size_t)(3 * bb) + e], (double)Yb[6 * (size_t)(3 * bb + 1) + e],
                                     (double)Yb[6 * (size_t)(3 * bb + 2) + e]};
                const double4_32a dd = d4[i0 + bb];
                const double d[3] = {dd.x, dd.y, dd.z};
                double cr[3];
                cross3(d, v, cr);
                s += cr[c - 3];
            }
        }
        sh[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S[36];
        for (int k = 0; k < 36; ++k) S[k] = sh[k];
        if (!spd6_inverse(S, Nt + 36 * (size_t)b)) atomicOr(flags, kFlagSingular);
    }
}

// W = E N~ for E = sigma [I, -l^x] (3 x 6 block of C on one body, App. A)
__device__ __forceinline__ void e_times_n(double sg, const double* l, const double* N, double* W) {
    for (int c = 0; c < 6; ++c) {
        const double v[3] = {N[3 * 6 + c], N[4 * 6 + c], N[5 * 6 + c]};
        double cr[3];
        cross3(l, v, cr);
        for (int a = 0; a < 3; ++a) W[a * 6 + c] = sg * (N[a * 6 + c] - cr[a]);
    }
}

// One articulated body per team: asm_list[blockIdx.x / team size].  In a
// cluster team the first CTA takes the column steps of each panel (pivot
// search and swaps included) and the team shares the trailing tiles, the
// blocked inverse and the scatter into G~; the first CTA publishes the rank
// (or -1 while the factorisation goes on) in rank_out[a] before each team
// barrier, so every CTA leaves the panel loop at the same panel.
template <class T, class Team>
__global__ void __launch_bounds__(kPcThreads)
k_pca_build(const int* __restrict__ asm_list, const int* __restrict__ asm_link_off,
            const int* __restrict__ asm_link_idx, const int* __restrict__ bp, const int* __restrict__ bq,
            const double* __restrict__ lp, const double* __restrict__ lq, const double* __restrict__ Nt,
            const long long* __restrict__ goff, T* __restrict__ G, T* __restrict__ gwork,
            int* __restrict__ perm_all, const long long* __restrict__ poff, int* __restrict__ rank_out,
            double tol) {
    extern __shared__ unsigned char dyn_smem[];
    double* dg = reinterpret_cast<double*>(dyn_smem);  // m values: the Schur-complement diagonal
    __shared__ PcTiles<T> tiles;
    __shared__ double s_pv, s_sk, s_isk;
    __shared__ int s_pi;
    const Team team;
    const int tr = team.rank(), ts = team.size();
    const int a = asm_list[blockIdx.x / ts];
    const int L0 = asm_link_off[a];
    const int Pa = asm_link_off[a + 1] - L0;
    const int m = 3 * Pa;
    if (m == 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T* H = gwork + 2 * goff[a];
    T* X = H + (size_t)m * m;
    T* Ga = G + goff[a];
    int* perm = perm_all + poff[a];
    for (int idx = threadIdx.x + tr * blockDim.x; idx < Pa * Pa; idx += blockDim.x * ts) {
        const int r = idx / Pa, c = idx % Pa;
        const int ln = asm_link_idx[L0 + r], lk = asm_link_idx[L0 + c];
        double blk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int sn = 0; sn < 2; ++sn) {
            const int bn = sn ? bq[ln] : bp[ln];
            for (int sk = 0; sk < 2; ++sk) {
                const int bk = sk ? bq[lk] : bp[lk];
                if (bn != bk) continue;
                double W[18];
                e_times_n(sn ? -1.0 : 1.0, sn ? lq + 3 * ln : lp + 3 * ln, Nt + 36 * (size_t)bn, W);
                const double* l = sk ? lq + 3 * lk : lp + 3 * lk;
                const double sg = sk ? -1.0 : 1.0;
                // (W E_k^T)[x][y] = sg (W[x][y] + (W[x][3:6] x l)_y)
                for (int x = 0; x < 3; ++x) {
                    const double w3[3] = {W[x * 6 + 3], W[x * 6 + 4], W[x * 6 + 5]};
                    double cr[3];
                    cross3(w3, l, cr);
                    for (int yy = 0; yy < 3; ++yy) blk[x * 3 + yy] += sg * (W[x * 6 + yy] + cr[yy]);
                }
            }
        }
        for (int x = 0; x < 3; ++x)
            for (int yy = 0; yy < 3; ++yy) H[(size_t)(3 * r + x) * m + 3 * c + yy] = (T)blk[x * 3 + yy];
    }
    if (tr == 0)
        for (int i = threadIdx.x; i < m; i += blockDim.x) perm[i] = i;
    team.sync();
    // symmetric pivoted Cholesky (largest remaining diagonal first, ties to
    // the lower index), stopped at the first pivot <= tol * the first one;
    // blocked: within a panel of 32 columns each column is formed from the
    // panel's earlier columns (left-looking) with the Schur-complement
    // diagonal dg kept up to date for the pivot search, and after the panel
    // the trailing block (both triangles, which the row and column swaps
    // read) takes one tile-product update.
    if (tr == 0)
        for (int i = threadIdx.x; i < m; i += blockDim.x) dg[i] = (double)H[(size_t)i * m + i];
    __syncthreads();
    double d0 = 0.0;
    int r = m;
    for (int k0 = 0; k0 < m; k0 += kNB) {
        const int kend = min(m, k0 + kNB);
        if (tr == 0) {
            bool stop = false;
            for (int k = k0; k < kend; ++k) {
                // pivot: warp 0 scans the remaining diagonal
                if (wid == 0) {
                    double best = -1.0;
                    int bi = 0x7fffffff;
                    for (int i = k + lane; i < m; i += 32) {
                        const double v = dg[i];
                        if (v > best || (v == best && i < bi)) { best = v; bi = i; }
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        const double ov = __shfl_down_sync(0xffffffffu, best, o);
                        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
                    }
                    if (lane == 0) {
                        s_pv = best;
                        s_pi = bi;
                        s_sk = best > 0.0 ? sqrt(best) : 1.0;
                        s_isk = 1.0 / s_sk;
                    }
                }
                __syncthreads();
                const double dmax = s_pv;
                const int j = s_pi;
                if (k == 0) d0 = dmax;
                if (!(dmax > tol * d0) || !(dmax > 0.0)) { r = k; stop = true; break; }
                if (j != k) {
                    // rows k, j and columns k, j exchanged in one pass: the
                    // row entries off columns k, j, the column entries off
                    // rows k, j, and the 2 x 2 block of both
                    for (int x = threadIdx.x; x < 2 * m; x += blockDim.x) {
                        if (x < m) {
                            const int c = x;
                            if (c == j) continue;
                            if (c == k) {
                                const T hkk = H[(size_t)k * m + k], hjj = H[(size_t)j * m + j];
                                const T hkj = H[(size_t)k * m + j], hjk = H[(size_t)j * m + k];
                                H[(size_t)k * m + k] = hjj;
                                H[(size_t)j * m + j] = hkk;
                                H[(size_t)k * m + j] = hjk;
                                H[(size_t)j * m + k] = hkj;
                            } else {
                                const T t = H[(size_t)k * m + c];
                                H[(size_t)k * m + c] = H[(size_t)j * m + c];
                                H[(size_t)j * m + c] = t;
                            }
                        } else {
                            const int rr = x - m;
                            if (rr == k || rr == j) continue;
                            const T t = H[(size_t)rr * m + k];
                            H[(size_t)rr * m + k] = H[(size_t)rr * m + j];
                            H[(size_t)rr * m + j] = t;
                        }
                    }
                    if (threadIdx.x == 0) {
                        const int t = perm[k];
                        perm[k] = perm[j];
                        perm[j] = t;
                        const double td = dg[k];
                        dg[k] = dg[j];
                        dg[j] = td;
                    }
                    __syncthreads();
                }
                // column k: Schur value from the panel's earlier columns (at
                // most 31, loaded together and summed in T, groups of 8 past
                // the panel's count skipped), scaled by the pivot's inverse
                // square root (formed once, by the thread that found it)
                const double sk = s_sk, isk = s_isk;
                const T* rowk = H + (size_t)k * m + k0;
                const int nk = k - k0;
                for (int i = k + threadIdx.x; i < m; i += blockDim.x) {
                    T* rowi = H + (size_t)i * m;
                    T pa[kNB], pb[kNB];
#pragma unroll
                    for (int t = 0; t < kNB; ++t) {
                        pa[t] = t < nk ? rowi[k0 + t] : (T)0;
                        pb[t] = t < nk ? rowk[t] : (T)0;
                    }
                    T acc = 0;
#pragma unroll
                    for (int g = 0; g < kNB; g += 8)
                        if (g < nk) {
#pragma unroll
                            for (int u = 0; u < 8; ++u) acc = fma(pa[g + u], pb[g + u], acc);
                        }
                    const double v = (double)rowi[k] - (double)acc;
                    if (i == k) {
                        rowi[k] = (T)sk;
                    } else {
                        const double l = v * isk;
                        rowi[k] = (T)l;
                        dg[i] -= l * l;
                    }
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) rank_out[a] = stop ? r : -1;
        }
        team.sync();
        const int st = *reinterpret_cast<volatile const int*>(rank_out + a);
        if (st >= 0) { r = st; break; }
        // trailing update of rows and columns >= kend by the panel's columns
        constexpr int E = kNB * kNB / kPcThreads;
        int q = 0;
        for (int i0 = kend; i0 < m; i0 += kNB) {
            for (int j0 = kend; j0 < m; j0 += kNB, ++q) {
                if (q % ts != tr) continue;
                tile_load(tiles.a, H, m, m, i0, k0, false);
                tile_load(tiles.b, H, m, m, j0, k0, false);
                __syncthreads();
                T acc[E];
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] = 0;
                tile_mac<T, true>(tiles.a, tiles.b, acc);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int rr = acc_row(e), c = acc_col(e);
                    if (i0 + rr < m && j0 + c < m) H[(size_t)(i0 + rr) * m + j0 + c] -= acc[e];
                }
                __syncthreads();
            }
        }
        team.sync();
    }
    if (threadIdx.x == 0 && tr == 0) rank_out[a] = r;
    // (L11 L11^T)^-1 of the rank-r leading block, blocked (written over H)
    blocked_chol_inverse(H, X, H, r, m, tiles, team);
    for (int idx = threadIdx.x + tr * blockDim.x; idx < m * m; idx += blockDim.x * ts) Ga[idx] = (T)0;
    team.sync();
    for (int idx = threadIdx.x + tr * blockDim.x; idx < r * r; idx += blockDim.x * ts) {
        const int i = idx / r, jj = idx % r;
        Ga[(size_t)perm[i] * m + perm[jj]] = H[(size_t)i * m + jj];
    }
}

// ------------------------------------------------------------- apply ---
// Work item it: body pcw_body[it], rows pcw_chunk[it]*32 .. +32.  128 threads:
// lane = row within the chunk, warp = quarter of the columns.
template <class T>
__global__ void __launch_bounds__(128)
k_pc_ap1(const int* __restrict__ pcw_body, const int* __restrict__ pcw_chunk,
         const int* __restrict__ blob_off, const T* __restrict__ minv,
         const long long* __restrict__ moff, const T* __restrict__ Y, const double* __restrict__ r,
         double* __restrict__ w, double* __restrict__ ytp, int Nb, const int* __restrict__ pcw_off,
         const double* __restrict__ Nt, double* __restrict__ Uhat, int* __restrict__ body_cnt) {
    dep_wait();
    __shared__ double red[4][kRows];
    __shared__ double yred[4][6];
    const int it = blockIdx.x;
    const int b = pcw_body[it];
    const int i0 = blob_off[b];
    const int m = 3 * (blob_off[b + 1] - i0);
    const int lane = threadIdx.x & 31, part = threadIdx.x >> 5;
    const int row = pcw_chunk[it] * kRows + lane;
    const T* A = minv + moff[b];
    const double* r1 = r + 3 * (size_t)i0;
    double s = 0.0;
    if (row < m) {
        // eight independent loads in flight per thread, four partial sums
        T acc[4] = {0, 0, 0, 0};
        int k = part;
        for (; k + 28 < m; k += 32) {
            T av[8], rv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                av[u] = A[(size_t)(k + 4 * u) * m + row];
                rv[u] = (T)r1[k + 4 * u];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u & 3] = fma(av[u], rv[u], acc[u & 3]);
        }
        for (; k < m; k += 4) acc[0] = fma(A[(size_t)k * m + row], (T)r1[k], acc[0]);
        s = (double)((acc[0] + acc[1]) + (acc[2] + acc[3]));
    }
    red[part][lane] = s;
    // partial Y^T r1 over this chunk's rows (warp `part` takes columns part, part+4)
    double yv[6] = {0, 0, 0, 0, 0, 0};
    if (part == 0 && row < m) {
        const T* Yr = Y + 18 * (size_t)i0 + 6 * (size_t)row;
        const double ri = r1[row];
        for (int c = 0; c < 6; ++c) yv[c] = (double)Yr[c] * ri;
    }
    if (part == 0)
        for (int c = 0; c < 6; ++c) {
            const double t = warp_sum(yv[c]);
            if (lane == 0) yred[0][c] = t;
        }
    __syncthreads();
    if (part == 0) {
        if (row < m) w[3 * (size_t)i0 + row] = red[0][lane] + red[1][lane] + red[2][lane] + red[3][lane];
        if (lane < 6) ytp[6 * (size_t)it + lane] = yred[0][lane];
    }
    // the body's last item: U^_b = N~_b (-r2_b - sum of the body's Y^T r1 partials)
    if (arrive_last(body_cnt, b, pcw_off[b + 1] - pcw_off[b]) && part == 0) {
        double v = 0.0;
        if (lane < 6) {
            v = -r[3 * (size_t)Nb + 6 * (size_t)b + lane];
            for (int q = pcw_off[b]; q < pcw_off[b + 1]; ++q) v -= __ldcg(ytp + 6 * (size_t)q + lane);
        }
        double vv[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) vv[c] = __shfl_sync(0xffffffffu, v, c);
        if (lane < 6) {
            const double* N = Nt + 36 * (size_t)b + 6 * lane;
            double t = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) t += N[c] * vv[c];
            Uhat[6 * (size_t)b + lane] = t;
        }
    }
}

// c_n = r3_n - (C U^)_n
__global__ void k_pc_cvec(int Nb, int M, int P, const int* __restrict__ bp, const int* __restrict__ bq,
                          const double* __restrict__ lp, const double* __restrict__ lq,
                          const double* __restrict__ Uhat, const double* __restrict__ r,
                          double* __restrict__ cbuf) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= P) return;
    const double* r3 = r + 3 * (size_t)Nb + 6 * (size_t)M;
    const double* up = Uhat + 6 * bp[n];
    const double* uq = Uhat + 6 * bq[n];
    double wp[3], wq[3];
    cross3(up + 3, lp + 3 * n, wp);
    cross3(uq + 3, lq + 3 * n, wq);
    for (int x = 0; x < 3; ++x) cbuf[3 * n + x] = r3[3 * n + x] - (up[x] + wp[x] - uq[x] - wq[x]);
}

// phi rows of one (articulated body, 32-row chunk) item: phi = G~ c, with c
// read from cbuf (k_pc_cvec) or, FUSED, formed here from U^ and r3 for the
// entries this block stages (c_n = r3_n - (C U^)_n)
template <class T, bool FUSED>
__global__ void __launch_bounds__(128)
k_pc_ap2(int Nb, int M, const int* __restrict__ pca_asm, const int* __restrict__ pca_chunk,
         const int* __restrict__ asm_link_off, const int* __restrict__ asm_link_idx,
         const T* __restrict__ G, const long long* __restrict__ goff, const double* __restrict__ cbuf,
         double* __restrict__ z, const int* __restrict__ bp, const int* __restrict__ bq,
         const double* __restrict__ lp, const double* __restrict__ lq, const double* __restrict__ Uhat,
         const double* __restrict__ r) {
    dep_wait();
    constexpr int kStage = 1024;  // entries of c staged in shared memory at a time
    __shared__ double red[4][kRows];
    __shared__ double cs[kStage];
    const int it = blockIdx.x;
    const int a = pca_asm[it];
    const int L0 = asm_link_off[a];
    const int m = 3 * (asm_link_off[a + 1] - L0);
    const int lane = threadIdx.x & 31, part = threadIdx.x >> 5;
    const int row = pca_chunk[it] * kRows + lane;
    const T* Ga = G + goff[a];
    T acc[4] = {0, 0, 0, 0};
    for (int c0 = 0; c0 < m; c0 += kStage) {
        const int cn = min(kStage, m - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < cn; k += blockDim.x) {
            const int kk = c0 + k;
            const int n = asm_link_idx[L0 + kk / 3], x = kk % 3;
            if (FUSED) {
                const double* up = Uhat + 6 * bp[n];
                const double* uq = Uhat + 6 * bq[n];
                double wp[3], wq[3];
                cross3(up + 3, lp + 3 * n, wp);
                cross3(uq + 3, lq + 3 * n, wq);
                cs[k] = r[3 * (size_t)Nb + 6 * (size_t)M + 3 * n + x] - (up[x] + wp[x] - uq[x] - wq[x]);
            } else {
                cs[k] = cbuf[3 * n + x];
            }
        }
        __syncthreads();
        if (row < m) {
            const T* Gc = Ga + (size_t)c0 * m + row;
            int k = part;
            for (; k + 28 < cn; k += 32) {
                T gv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) gv[u] = Gc[(size_t)(k + 4 * u) * m];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u & 3] = fma(gv[u], (T)cs[k + 4 * u], acc[u & 3]);
            }
            for (; k < cn; k += 4) acc[0] = fma(Gc[(size_t)k * m], (T)cs[k], acc[0]);
        }
    }
    const double s = row < m ? (double)((acc[0] + acc[1]) + (acc[2] + acc[3])) : 0.0;
    red[part][lane] = s;
    __syncthreads();
    if (part == 0 && row < m) {
        const int n = asm_link_idx[L0 + row / 3];
        z[3 * (size_t)Nb + 6 * (size_t)M + 3 * n + row % 3] = red[0][lane] + red[1][lane] + red[2][lane] + red[3][lane];
    }
}

// U_b = U^_b + N~_b (C^T phi)_b;  lambda rows = w + Y U
template <class T>
__global__ void __launch_bounds__(128)
k_pc_ap3(int Nb, int M, const int* __restrict__ pcw_body, const int* __restrict__ pcw_chunk,
         const int* __restrict__ blob_off, const T* __restrict__ Y, const double* __restrict__ Nt,
         const double* __restrict__ w, const double* __restrict__ Uhat,
         const int* __restrict__ bl_off, const int* __restrict__ bl_idx,
         const double* __restrict__ lp, const double* __restrict__ lq, double* __restrict__ z) {
    dep_wait();
    __shared__ double sU[6];
    const int it = blockIdx.x;
    const int b = pcw_body[it];
    const double* phi = z + 3 * (size_t)Nb + 6 * (size_t)M;
    if (threadIdx.x < 32) {
        // (C^T phi)_b: the body's link ends spread over the lanes of warp 0
        const int lane = threadIdx.x;
        double f[6] = {0, 0, 0, 0, 0, 0};
        for (int k = bl_off[b] + lane; k < bl_off[b + 1]; k += 32) {
            const int e = bl_idx[k];
            const int n = e >> 1;
            const double sg = (e & 1) ? -1.0 : 1.0;
            const double* l = (e & 1) ? lq + 3 * n : lp + 3 * n;
            const double* ph = phi + 3 * n;
            double t[3];
            cross3(l, ph, t);
            for (int x = 0; x < 3; ++x) { f[x] += sg * ph[x]; f[3 + x] += sg * t[x]; }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) f[c] = warp_sum(f[c]);
        if (lane < 6) {
            const double* N = Nt + 36 * (size_t)b + 6 * lane;
            double s = Uhat[6 * (size_t)b + lane];
#pragma unroll
            for (int c = 0; c < 6; ++c) s += N[c] * f[c];
            sU[lane] = s;
            if (pcw_chunk[it] == 0) z[3 * (size_t)Nb + 6 * (size_t)b + lane] = s;
        }
    }
    __syncthreads();
    const int i0 = blob_off[b];
    const int m = 3 * (blob_off[b + 1] - i0);
    const int row = pcw_chunk[it] * kRows + threadIdx.x;
    if (threadIdx.x < kRows && row < m) {
        const T* Yr = Y + 18 * (size_t)i0 + 6 * (size_t)row;
        double s = w[3 * (size_t)i0 + row];
        for (int c = 0; c < 6; ++c) s = fma((double)Yr[c], sU[c], s);
        z[3 * (size_t)i0 + row] = s;
    }
}

// ----------------------------------------------------------------- host ---
// Launch of a build kernel over the items list[0 .. n): one CTA each, or
// one cluster of cs CTAs each.
template <class K, class... Args>
static void launch_team(K kernel, int n, int cs, size_t smem, cudaStream_t s, Args... args) {
    if (n <= 0) return;
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3((unsigned)(n * cs));
    lc.blockDim = dim3(kPcThreads);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    lc.attrs = at;
    lc.numAttrs = cs > 1 ? 1 : 0;
    cudaLaunchKernelEx(&lc, kernel, args...);
    count_launch();
}

template <class T>
static void pca_build_t(am_handle* h, double tol) {
    const size_t smem = (size_t)3 * std::max(1, h->max_asm_links) * sizeof(double);  // Schur diagonal
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_pca_build<T, CtaTeam>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_pca_build<T, ClusterTeam>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    const int n_one = h->pca_cs > 1 ? h->n_pca_small : h->NA;
    launch_team(k_pca_build<T, CtaTeam>, n_one, 1, smem, h->stream, (const int*)h->d_pca_list,
                (const int*)h->d_asm_link_off, (const int*)h->d_asm_link_idx, (const int*)h->d_bp,
                (const int*)h->d_bq, (const double*)h->d_lp, (const double*)h->d_lq, (const double*)h->d_Nt,
                (const long long*)h->d_G_off, (T*)h->d_G, (T*)h->d_Gwork, h->d_perm,
                (const long long*)h->d_perm_off, h->d_G_rank, tol);
    if (h->pca_cs > 1)
        launch_team(k_pca_build<T, ClusterTeam>, h->NA - h->n_pca_small, h->pca_cs, smem, h->stream,
                    (const int*)(h->d_pca_list + h->n_pca_small), (const int*)h->d_asm_link_off,
                    (const int*)h->d_asm_link_idx, (const int*)h->d_bp, (const int*)h->d_bq,
                    (const double*)h->d_lp, (const double*)h->d_lq, (const double*)h->d_Nt,
                    (const long long*)h->d_G_off, (T*)h->d_G, (T*)h->d_Gwork, h->d_perm,
                    (const long long*)h->d_perm_off, h->d_G_rank, tol);
}

template <class T>
static void pc_build_t(am_handle* h, double tol) {
    cudaStream_t s = h->stream;
    // one block of kPcThreads per body and per articulated body (the tile
    // routines assume that block size)
    // bodies of one or two 32-row tiles one CTA each; larger bodies one
    // cluster of pcb_cs CTAs each when they are too few to fill the GPU
    const int n_one = h->pcb_cs > 1 ? h->n_pcb_small : h->M;
    launch_team(k_pcb_build<T, CtaTeam>, n_one, 1, 0, s, (const int*)h->d_pcb_list, (const int*)h->d_blob_off,
                (const double4_32a*)h->d_r4, (const double4_32a*)h->d_d4, (const long long*)h->d_minv_off,
                (T*)h->d_minv, (T*)h->d_pcwork, (T*)h->d_Y, h->d_Nt, rpy_consts<T>(h->prm), h->cfg.wall,
                h->d_flags);
    if (h->pcb_cs > 1)
        launch_team(k_pcb_build<T, ClusterTeam>, h->M - h->n_pcb_small, h->pcb_cs, 0, s,
                    (const int*)(h->d_pcb_list + h->n_pcb_small), (const int*)h->d_blob_off,
                    (const double4_32a*)h->d_r4, (const double4_32a*)h->d_d4, (const long long*)h->d_minv_off,
                    (T*)h->d_minv, (T*)h->d_pcwork, (T*)h->d_Y, h->d_Nt, rpy_consts<T>(h->prm),
                    h->cfg.wall, h->d_flags);
    if (h->P) pca_build_t<T>(h, tol);
}

void pc_apply_links(am_handle* h, const double* r, double* z) {
    cudaStream_t s = h->stream;
    k_pc_cvec<<<(h->P + 127) / 128, 128, 0, s>>>(h->Nb, h->M, h->P, h->d_bp, h->d_bq, h->d_lp, h->d_lq,
                                                  h->d_pc_Uhat, r, h->d_cbuf);
    if (h->pc32)
        k_pc_ap2<float, false><<<h->n_pca, 128, 0, s>>>(h->Nb, h->M, h->d_pca_asm, h->d_pca_chunk,
                                                         h->d_asm_link_off, h->d_asm_link_idx, (const float*)h->d_G,
                                                         h->d_G_off, h->d_cbuf, z, nullptr, nullptr, nullptr,
                                                         nullptr, nullptr, nullptr);
    else
        k_pc_ap2<double, false><<<h->n_pca, 128, 0, s>>>(h->Nb, h->M, h->d_pca_asm, h->d_pca_chunk,
                                                          h->d_asm_link_off, h->d_asm_link_idx, (const double*)h->d_G,
                                                          h->d_G_off, h->d_cbuf, z, nullptr, nullptr, nullptr,
                                                          nullptr, nullptr, nullptr);
    count_launch(2);
}

void pc_build(am_handle* h) {
    // arrival counts of the apply's per-body reductions (each completing
    // block zeroes its own; zeroed here as well, outside any graph)
    if (h->d_pcb_cnt) cudaMemsetAsync(h->d_pcb_cnt, 0, std::max(h->M, 1) * sizeof(int), h->stream);
    if (h->sb) {
        sb_pc_build(h);
        if (h->P) pca_build_t<double>(h, 1e-11);
        h->pc_valid = true;
        return;
    }
    if (h->pc32)
        pc_build_t<float>(h, 1e-5);
    else
        pc_build_t<double>(h, 1e-11);
    h->pc_valid = true;
}

template <class T>
static void pc_apply_t(am_handle* h, const double* r, double* z) {
    cudaStream_t s = h->stream;
    // w and Y^T r1 per (body, chunk) item; the body's last item forms U^
    launch_dep(k_pc_ap1<T>, dim3(h->n_pcw), dim3(128), 0, s, h->d_pcw_body, h->d_pcw_chunk, h->d_blob_off,
               (const T*)h->d_minv, h->d_minv_off, (const T*)h->d_Y, r, h->d_pc_w, h->d_ytp, h->Nb, h->d_pcw_off,
               h->d_Nt, h->d_pc_Uhat, h->d_pcb_cnt);
    count_launch();
    if (h->P) {
        // phi = G~ (r3 - C U^), c formed per staged entry
        launch_dep(k_pc_ap2<T, true>, dim3(h->n_pca), dim3(128), 0, s, h->Nb, h->M, h->d_pca_asm, h->d_pca_chunk,
                   h->d_asm_link_off, h->d_asm_link_idx, (const T*)h->d_G, h->d_G_off, nullptr, z, h->d_bp, h->d_bq,
                   h->d_lp, h->d_lq, h->d_pc_Uhat, r);
        count_launch();
    }
    launch_dep(k_pc_ap3<T>, dim3(h->n_pcw), dim3(128), 0, s, h->Nb, h->M, h->d_pcw_body, h->d_pcw_chunk,
               h->d_blob_off, (const T*)h->d_Y, h->d_Nt, h->d_pc_w, h->d_pc_Uhat, h->d_body_link_off,
               h->d_body_link_idx, h->d_lp, h->d_lq, z);
    count_launch();
}

void pc_apply(am_handle* h, const double* r, double* z) {
    if (h->sb) {
        sb_pc_apply(h, r, z);
        return;
    }
    if (h->pc32)
        pc_apply_t<float>(h, r, z);
    else
        pc_apply_t<double>(h, r, z);
}

}  // namespace am

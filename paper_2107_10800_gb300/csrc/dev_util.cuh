// Small device helpers shared by the kernels of libam.
#pragma once
#include "am_internal.cuh"

namespace am {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; every thread gets the result.  sh: >= 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double r = (lane < (int)((blockDim.x + 31) >> 5)) ? sh[lane] : 0.0;
        r = warp_sum(r);
        if (lane == 0) sh[32] = r;
    }
    __syncthreads();
    return sh[32];
}

// Arrival count of the blocks that share a reduction: every block that has
// written its partial results calls it (all threads); true in every thread
// of the block that completes cnt[idx] = total, which then reads the
// others' partials (with __ldcg: they bypass this SM's L1) and has zeroed
// the count for the next use.  No block waits for another.
__device__ __forceinline__ bool arrive_last(int* cnt, int idx, int total) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int t = atomicAdd(&cnt[idx], 1);
        s_last = (t == total - 1) ? 1 : 0;
        if (s_last) cnt[idx] = 0;
    }
    __syncthreads();
    const bool last = s_last != 0;
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// In-place lower Cholesky factor of the m x m matrix A (row-major, full
// storage, T = double or float), cooperative over the block.  Returns false
// (to every thread) if a pivot is not positive.  sh: >= 2 doubles.
template <class T>
__device__ bool block_cholesky(T* A, int m, double* sh) {
    for (int k = 0; k < m; ++k) {
        if (threadIdx.x == 0) {
            const double d = (double)A[(size_t)k * m + k];
            sh[0] = d;
            if (d > 0.0) {
                const T s = (T)sqrt(d);
                A[(size_t)k * m + k] = s;
                sh[1] = 1.0 / (double)s;
            }
        }
        __syncthreads();
        if (!(sh[0] > 0.0)) return false;
        const T inv = (T)sh[1];
        for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[(size_t)i * m + k] *= inv;
        __syncthreads();
        const int len = m - k - 1;
        for (int idx = threadIdx.x; idx < len * len; idx += blockDim.x) {
            const int i = k + 1 + idx / len, j = k + 1 + idx % len;
            if (j <= i) A[(size_t)i * m + j] -= A[(size_t)i * m + k] * A[(size_t)j * m + k];
        }
        __syncthreads();
    }
    return true;
}

// ---- blocked SPD inverse on 32 x 32 shared-memory tiles -----------------
// A = M^-1 for an m x m symmetric positive definite M (row-major, full
// storage in global memory) by blocked right-looking Cholesky M = L L^T,
// the blocked lower-triangular inverse X = L^-1 and A = X^T X, every step a
// product of 32 x 32 tiles staged in shared memory.  A team of CTAs of
// kPcThreads threads works on one matrix: one CTA, or the CTAs of a thread
// block cluster, which share the tiles of every step round robin and meet at
// the cluster barrier (release/acquire: the tiles one CTA wrote to global
// memory are seen by the others after it).  L and X are m x m scratch (L may
// alias nothing else).  A non-positive pivot sets *bad (shared) and is
// replaced by 1 so that every CTA still reaches every barrier; the result is
// then meaningless.  Every CTA of a team takes the same branches (the
// diagonal tiles are factored redundantly in each), so the barrier counts
// agree.
constexpr int kNB = 32;
constexpr int kPcThreads = 256;

template <class T>
struct PcTiles {
    T a[kNB][kNB + 1];
    T b[kNB][kNB + 1];
    T c[kNB][kNB + 1];
};

// tile of G (leading dimension ld) at (r0, c0) into S, zero outside
// [0, m) x [0, m); transposed: S[j][i] = G[r0 + i][c0 + j]
template <class T>
__device__ __forceinline__ void tile_load(T (*S)[kNB + 1], const T* G, int ld, int m, int r0, int c0, bool tr) {
    for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
        const int i = idx / kNB, j = idx % kNB;
        const T v = (r0 + i < m && c0 + j < m) ? G[(size_t)(r0 + i) * ld + c0 + j] : (T)0;
        if (tr) S[j][i] = v; else S[i][j] = v;
    }
}

// The accumulators of a 32 x 32 tile: each of the 256 threads holds a 2 x 2
// block, acc[e] (e = 0..3) the entry (acc_row(e), acc_col(e)) with rows
// 2 (t / 16) + e / 2 and columns 2 (t % 16) + e % 2, t = threadIdx.x; per k a
// thread loads two entries of each operand for four multiply-adds.
static_assert(kNB == 32 && kPcThreads == 256, "2 x 2 accumulator blocks of 256 threads cover a 32 x 32 tile");
__device__ __forceinline__ int acc_row(int e) { return 2 * ((int)threadIdx.x >> 4) + (e >> 1); }
__device__ __forceinline__ int acc_col(int e) { return 2 * ((int)threadIdx.x & 15) + (e & 1); }

// acc[e] += sum_k A[r][k] B[c][k] (nt) or sum_k A[r][k] B[k][c] (nn) for the
// thread's entries (r, c), each sum in the order k = 0, 1, ..
template <class T, bool NT>
__device__ __forceinline__ void tile_mac(const T (*A)[kNB + 1], const T (*B)[kNB + 1], T* acc) {
    const int r = acc_row(0), c = acc_col(0);
    T s00 = acc[0], s01 = acc[1], s10 = acc[2], s11 = acc[3];
#pragma unroll 8
    for (int k = 0; k < kNB; ++k) {
        const T a0 = A[r][k], a1 = A[r + 1][k];
        const T b0 = NT ? B[c][k] : B[k][c];
        const T b1 = NT ? B[c + 1][k] : B[k][c + 1];
        s00 = fma(a0, b0, s00);
        s01 = fma(a0, b1, s01);
        s10 = fma(a1, b0, s10);
        s11 = fma(a1, b1, s11);
    }
    acc[0] = s00; acc[1] = s01; acc[2] = s10; acc[3] = s11;
}

// In place: the lower Cholesky factor of the leading kw x kw part of the
// tile S (right-looking, one column per step, every thread of the block).
// A non-positive pivot sets *bad and is replaced by 1.
template <class T>
__device__ __forceinline__ void tile_cholesky(T (*S)[kNB + 1], int kw, int* bad) {
    for (int j = 0; j < kw; ++j) {
        T d = S[j][j];
        if (!(d > (T)0)) d = (T)1;
        const T sd = sqrt(d);
        const int i = threadIdx.x;
        if (i > j && i < kw) S[i][j] /= sd;
        __syncthreads();
        // the pivot itself (read by no one in this half-step) and the
        // trailing lower triangle
        if (threadIdx.x == 0) {
            if (!(S[j][j] > (T)0)) *bad = 1;
            S[j][j] = sd;
        }
        const int w = kw - 1 - j;
        for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
            const int r = j + 1 + idx / w, c = j + 1 + idx % w;
            if (c <= r) S[r][c] -= S[r][j] * S[c][j];
        }
        __syncthreads();
    }
}

// D = S^-1 for the lower triangle of S (kw x kw), zeros elsewhere in D:
// forward substitution on the identity, one row of D per step, that row's
// updates of the rows below spread over the block (every thread calls).
template <class T>
__device__ __forceinline__ void tile_lower_inverse(const T (*S)[kNB + 1], T (*D)[kNB + 1], int kw) {
    for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
        const int i = idx / kNB, j = idx % kNB;
        D[i][j] = (i == j && i < kw) ? (T)1 : (T)0;
    }
    __syncthreads();
    for (int i = 0; i < kw; ++i) {
        if (threadIdx.x <= i) D[i][threadIdx.x] /= S[i][i];
        __syncthreads();
        const int w = i + 1;
        for (int idx = threadIdx.x; idx < (kw - 1 - i) * w; idx += blockDim.x) {
            const int q = i + 1 + idx / w, jj = idx % w;
            D[q][jj] -= S[q][i] * D[i][jj];
        }
        __syncthreads();
    }
}

struct CtaTeam {
    __device__ __forceinline__ int rank() const { return 0; }
    __device__ __forceinline__ int size() const { return 1; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

struct ClusterTeam {
    int r, n;
    __device__ __forceinline__ ClusterTeam() {
        unsigned v;
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(v));
        r = (int)v;
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(v));
        n = (int)v;
    }
    __device__ __forceinline__ int rank() const { return r; }
    __device__ __forceinline__ int size() const { return n; }
    __device__ __forceinline__ void sync() const {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
};

// Blocked right-looking Cholesky in place (lower triangle of the leading
// n x n block of L, leading dimension ld).
template <class T, class Team>
__device__ void blocked_cholesky(T* L, int n, int ld, PcTiles<T>& s, int* bad, const Team& team) {
    constexpr int E = kNB * kNB / kPcThreads;
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int kw = min(kNB, n - k0);
        __syncthreads();
        tile_load(s.a, L, ld, n, k0, k0, false);
        __syncthreads();
        tile_cholesky(s.a, kw, bad);
        tile_lower_inverse(s.a, s.b, kw);
        __syncthreads();
        // panel below the diagonal block: L_rk = M_rk L_kk^-T
        int q = 0;
        for (int r0 = k0 + kNB; r0 < n; r0 += kNB, ++q) {
            if (q % team.size() != team.rank()) continue;
            tile_load(s.c, L, ld, n, r0, k0, false);
            __syncthreads();
            T acc[E];
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = 0;
            tile_mac<T, true>(s.c, s.b, acc);
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int r = acc_row(e), c = acc_col(e);
                if (r0 + r < n && c < kw) L[(size_t)(r0 + r) * ld + k0 + c] = acc[e];
            }
            __syncthreads();
        }
        // every CTA has read M_kk: the factor may replace it now
        team.sync();
        if (team.rank() == 0)
            for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
                const int i = idx / kNB, j = idx % kNB;
                if (i < kw && j <= i) L[(size_t)(k0 + i) * ld + k0 + j] = s.a[i][j];
            }
        __syncthreads();
        // trailing update of the lower triangle: M_IJ -= L_Ik L_Jk^T
        q = 0;
        for (int i0 = k0 + kNB; i0 < n; i0 += kNB) {
            for (int j0 = k0 + kNB; j0 <= i0; j0 += kNB, ++q) {
                if (q % team.size() != team.rank()) continue;
                tile_load(s.a, L, ld, n, i0, k0, false);
                tile_load(s.b, L, ld, n, j0, k0, false);
                __syncthreads();
                T acc[E];
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] = 0;
                tile_mac<T, true>(s.a, s.b, acc);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int r = acc_row(e), c = acc_col(e);
                    if (i0 + r < n && j0 + c < n) L[(size_t)(i0 + r) * ld + j0 + c] -= acc[e];
                }
                __syncthreads();
            }
        }
        team.sync();
    }
}

// From the lower Cholesky factor L (n x n, leading dimension ld): X = L^-1
// (lower) and A = X^T X = (L L^T)^-1 (full), blocked.  X by block columns
// right-looking: the diagonal blocks X_KK = L_KK^-1 first, then for each K
// the updates B_IJ -= L_IK X_KJ (I > K, J <= K) of the strictly lower blocks
// B (kept in X, zero at the start), each block of row K + 1 finished as
// X_IJ = X_II B_IJ by the CTA that adds its last term.  A may alias L.
template <class T, class Team>
__device__ void blocked_chol_inverse(const T* L, T* X, T* A, int n, int ld, PcTiles<T>& s, const Team& team) {
    constexpr int E = kNB * kNB / kPcThreads;
    const int nt = (n + kNB - 1) / kNB;
    // --- diagonal blocks of X; the strictly lower blocks start at zero ---
    for (int k = team.rank(); k < nt; k += team.size()) {
        const int k0 = k * kNB, kw = min(kNB, n - k0);
        __syncthreads();
        tile_load(s.a, L, ld, n, k0, k0, false);
        __syncthreads();
        tile_lower_inverse(s.a, s.b, kw);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
            const int i = idx / kNB, j = idx % kNB;
            if (i < kw && j < kw) X[(size_t)(k0 + i) * ld + k0 + j] = s.b[i][j];
        }
        for (int j0 = 0; j0 < k0; j0 += kNB)
            for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
                const int i = idx / kNB, j = idx % kNB;
                if (i < kw) X[(size_t)(k0 + i) * ld + j0 + j] = (T)0;
            }
    }
    team.sync();
    // --- strictly lower blocks, one block column step K at a time ---
    for (int K = 0; K + 1 < nt; ++K) {
        const int K0 = K * kNB;
        int q = 0;
        for (int I = K + 1; I < nt; ++I) {
            const int I0 = I * kNB;
            for (int J = 0; J <= K; ++J, ++q) {
                if (q % team.size() != team.rank()) continue;
                const int J0 = J * kNB;
                __syncthreads();
                tile_load(s.a, L, ld, n, I0, K0, false);  // L_IK
                tile_load(s.b, X, ld, n, K0, J0, false);  // X_KJ
                __syncthreads();
                T acc[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int r = acc_row(e), c = acc_col(e);
                    acc[e] = (I0 + r < n && J0 + c < n) ? -X[(size_t)(I0 + r) * ld + J0 + c] : (T)0;
                }
                tile_mac<T, false>(s.a, s.b, acc);  // acc = -(B_IJ - L_IK X_KJ)
                if (I == K + 1) {
                    __syncthreads();
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        s.c[acc_row(e)][acc_col(e)] = acc[e];
                    }
                    tile_load(s.a, X, ld, n, I0, I0, false);  // X_II
                    __syncthreads();
#pragma unroll
                    for (int e = 0; e < E; ++e) acc[e] = 0;
                    tile_mac<T, false>(s.a, s.c, acc);  // acc = -X_II B_IJ
                }
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int r = acc_row(e), c = acc_col(e);
                    if (I0 + r < n && J0 + c < n) X[(size_t)(I0 + r) * ld + J0 + c] = -acc[e];
                }
            }
        }
        team.sync();
    }
    // --- A = X^T X (lower triangle, mirrored) ---
    int q = 0;
    for (int i0 = 0; i0 < n; i0 += kNB) {
        for (int j0 = 0; j0 <= i0; j0 += kNB, ++q) {
            if (q % team.size() != team.rank()) continue;
            T acc[E];
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = 0;
            for (int q0 = i0; q0 < n; q0 += kNB) {
                __syncthreads();
                tile_load(s.a, X, ld, n, q0, i0, true);   // s.a[r][k] = X[q0 + k][i0 + r]
                tile_load(s.b, X, ld, n, q0, j0, false);  // s.b[k][c] = X[q0 + k][j0 + c]
                __syncthreads();
                tile_mac<T, false>(s.a, s.b, acc);
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int r = acc_row(e), c = acc_col(e);
                const int i = i0 + r, j = j0 + c;
                if (i < n && j < n && j <= i) {
                    A[(size_t)i * ld + j] = acc[e];
                    A[(size_t)j * ld + i] = acc[e];
                }
            }
        }
    }
    team.sync();
}

template <class T, class Team>
__device__ void blocked_spd_inverse(T* L, T* X, T* A, int m, PcTiles<T>& s, int* bad, const Team& team) {
    blocked_cholesky(L, m, m, s, bad, team);
    blocked_chol_inverse(L, X, A, m, m, s, team);
}

// 6 x 6 symmetric positive definite inverse in one thread (Cholesky).
__device__ __forceinline__ bool spd6_inverse(const double* S, double* Out) {
    double L[36];
    for (int i = 0; i < 36; ++i) L[i] = 0.0;
    for (int j = 0; j < 6; ++j) {
        double d = 0.5 * (S[j * 6 + j] + S[j * 6 + j]);
        for (int k = 0; k < j; ++k) d -= L[j * 6 + k] * L[j * 6 + k];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        L[j * 6 + j] = d;
        for (int i = j + 1; i < 6; ++i) {
            double s = 0.5 * (S[i * 6 + j] + S[j * 6 + i]);
            for (int k = 0; k < j; ++k) s -= L[i * 6 + k] * L[j * 6 + k];
            L[i * 6 + j] = s / d;
        }
    }
    // columns of the inverse: solve L L^T x = e_c
    for (int c = 0; c < 6; ++c) {
        double y[6];
        for (int i = 0; i < 6; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * 6 + k] * y[k];
            y[i] = s / L[i * 6 + i];
        }
        for (int i = 5; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < 6; ++k) s -= L[k * 6 + i] * y[k];
            y[i] = s / L[i * 6 + i];
        }
        for (int i = 0; i < 6; ++i) Out[i * 6 + c] = y[i];
    }
    return true;
}


}  // namespace am

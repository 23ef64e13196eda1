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
// product of 32 x 32 tiles staged in shared memory.  One block of kPcThreads
// threads per matrix; L and X are m x m scratch (L may alias nothing else).
// A non-positive pivot sets *bad (shared) and is replaced by 1 so that the
// block still reaches every barrier; the result is then meaningless.
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

// acc[e] for entry (r, c) = (idx / 32, idx % 32), idx = threadIdx.x + e * blockDim.x:
// sum_k A[r][k] B[c][k] (nt) or sum_k A[r][k] B[k][c] (nn)
template <class T, bool NT>
__device__ __forceinline__ void tile_mac(const T (*A)[kNB + 1], const T (*B)[kNB + 1], T* acc) {
#pragma unroll
    for (int e = 0; e < kNB * kNB / kPcThreads; ++e) {
        const int idx = threadIdx.x + e * kPcThreads, r = idx / kNB, c = idx % kNB;
        T s = acc[e];
#pragma unroll 8
        for (int k = 0; k < kNB; ++k) s = fma(A[r][k], NT ? B[c][k] : B[k][c], s);
        acc[e] = s;
    }
}

// inverse of the lower triangle of S (kw x kw) into D (zeros above the
// diagonal); thread j computes column j by forward substitution
template <class T>
__device__ __forceinline__ void tile_lower_inverse(const T (*S)[kNB + 1], T (*D)[kNB + 1], int kw) {
    const int j = threadIdx.x;
    if (j < kNB) {
        for (int i = 0; i < kNB; ++i) D[i][j] = (T)0;
        if (j < kw) {
            D[j][j] = (T)1 / S[j][j];
            for (int i = j + 1; i < kw; ++i) {
                T s = 0;
                for (int t = j; t < i; ++t) s = fma(S[i][t], D[t][j], s);
                D[i][j] = -s / S[i][i];
            }
        }
    }
}

// Blocked right-looking Cholesky in place (lower triangle of the leading
// n x n block of L, leading dimension ld).
template <class T>
__device__ void blocked_cholesky(T* L, int n, int ld, PcTiles<T>& s, int* bad) {
    constexpr int E = kNB * kNB / kPcThreads;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // --- Cholesky, in place in L (lower triangle) ---
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int kw = min(kNB, n - k0);
        __syncthreads();
        tile_load(s.a, L, ld, n, k0, k0, false);
        __syncthreads();
        if (wid == 0) {
            for (int j = 0; j < kw; ++j) {
                if (lane == j) {
                    T d = s.a[j][j];
                    if (!(d > (T)0)) { *bad = 1; d = (T)1; }
                    s.a[j][j] = sqrt(d);
                }
                __syncwarp();
                if (lane > j && lane < kw) s.a[lane][j] /= s.a[j][j];
                __syncwarp();
                if (lane > j && lane < kw)
                    for (int c = j + 1; c <= lane; ++c) s.a[lane][c] -= s.a[lane][j] * s.a[c][j];
                __syncwarp();
            }
        }
        __syncthreads();
        tile_lower_inverse(s.a, s.b, kw);
        for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
            const int i = idx / kNB, j = idx % kNB;
            if (i < kw && j <= i) L[(size_t)(k0 + i) * ld + k0 + j] = s.a[i][j];
        }
        __syncthreads();
        // panel below the diagonal block: L_rk = M_rk L_kk^-T
        for (int r0 = k0 + kNB; r0 < n; r0 += kNB) {
            tile_load(s.c, L, ld, n, r0, k0, false);
            __syncthreads();
            T acc[E];
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = 0;
            tile_mac<T, true>(s.c, s.b, acc);
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = threadIdx.x + e * kPcThreads, r = idx / kNB, c = idx % kNB;
                if (r0 + r < n && c < kw) L[(size_t)(r0 + r) * ld + k0 + c] = acc[e];
            }
            __syncthreads();
        }
        // trailing update of the lower triangle: M_IJ -= L_Ik L_Jk^T
        for (int i0 = k0 + kNB; i0 < n; i0 += kNB) {
            tile_load(s.a, L, ld, n, i0, k0, false);
            for (int j0 = k0 + kNB; j0 <= i0; j0 += kNB) {
                tile_load(s.b, L, ld, n, j0, k0, false);
                __syncthreads();
                T acc[E];
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] = 0;
                tile_mac<T, true>(s.a, s.b, acc);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int idx = threadIdx.x + e * kPcThreads, r = idx / kNB, c = idx % kNB;
                    if (i0 + r < n && j0 + c < n) L[(size_t)(i0 + r) * ld + j0 + c] -= acc[e];
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
}

// From the lower Cholesky factor L (n x n, leading dimension ld): X = L^-1
// (lower) and A = X^T X = (L L^T)^-1 (full), blocked.
template <class T>
__device__ void blocked_chol_inverse(const T* L, T* X, T* A, int n, int ld, PcTiles<T>& s) {
    constexpr int E = kNB * kNB / kPcThreads;
    // --- X = L^-1: diagonal blocks, then block rows below ---
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int kw = min(kNB, n - k0);
        __syncthreads();
        tile_load(s.a, L, ld, n, k0, k0, false);
        __syncthreads();
        tile_lower_inverse(s.a, s.b, kw);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
            const int i = idx / kNB, j = idx % kNB;
            if (i < kw && j < kw) X[(size_t)(k0 + i) * ld + k0 + j] = s.b[i][j];
        }
    }
    for (int j0 = 0; j0 < n; j0 += kNB) {
        for (int i0 = j0 + kNB; i0 < n; i0 += kNB) {
            // T = sum_{K = J .. I-1} L_IK X_KJ, then X_IJ = -X_II T
            T acc[E];
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = 0;
            for (int q0 = j0; q0 < i0; q0 += kNB) {
                __syncthreads();
                tile_load(s.a, L, ld, n, i0, q0, false);
                tile_load(s.b, X, ld, n, q0, j0, false);
                __syncthreads();
                tile_mac<T, false>(s.a, s.b, acc);
            }
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = threadIdx.x + e * kPcThreads;
                s.c[idx / kNB][idx % kNB] = acc[e];
            }
            tile_load(s.a, X, ld, n, i0, i0, false);
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = 0;
            tile_mac<T, false>(s.a, s.c, acc);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = threadIdx.x + e * kPcThreads, r = idx / kNB, c = idx % kNB;
                if (i0 + r < n && j0 + c < n) X[(size_t)(i0 + r) * ld + j0 + c] = -acc[e];
            }
        }
    }
    // --- A = X^T X (lower triangle, mirrored) ---
    for (int i0 = 0; i0 < n; i0 += kNB) {
        for (int j0 = 0; j0 <= i0; j0 += kNB) {
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
                const int idx = threadIdx.x + e * kPcThreads, r = idx / kNB, c = idx % kNB;
                const int i = i0 + r, j = j0 + c;
                if (i < n && j < n && j <= i) {
                    A[(size_t)i * ld + j] = acc[e];
                    A[(size_t)j * ld + i] = acc[e];
                }
            }
        }
    }
    __syncthreads();
}

template <class T>
__device__ void blocked_spd_inverse(T* L, T* X, T* A, int m, PcTiles<T>& s, int* bad) {
    blocked_cholesky(L, m, m, s, bad);
    blocked_chol_inverse(L, X, A, m, m, s);
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

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

template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// X = L^{-1} for the leading r x r lower triangle of L (leading dimension
// ld).  One warp per column j: X[i][j] = -(sum_{k<i} L[i][k] X[k][j]) / L[i][i]
// with the dot product split over the lanes and the column kept in shared
// memory (col: blockDim.x / 32 columns of r values); rows of L are read
// coalesced.  X's upper triangle is left unset.
template <class T>
__device__ void block_lower_inverse(const T* L, T* X, int r, int ld, T* col) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T* c = col + (size_t)wid * r;
    for (int j = wid; j < r; j += nw) {
        const T djj = (T)1 / L[(size_t)j * ld + j];
        if (lane == 0) { c[j] = djj; X[(size_t)j * ld + j] = djj; }
        __syncwarp();
        for (int i = j + 1; i < r; ++i) {
            const T* Li = L + (size_t)i * ld;
            T s = 0;
            for (int k = j + lane; k < i; k += 32) s = fma(Li[k], c[k], s);
            s = warp_sum_t(s);
            if (lane == 0) {
                const T v = -s / Li[i];
                c[i] = v;
                X[(size_t)i * ld + j] = v;
            }
            __syncwarp();
        }
    }
    __syncthreads();
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

// Pair terms of the blob mobility (Sec. 2.3, Eq. RPY), shared by the
// all-pairs product and the preconditioner's same-body blocks.  The formulas
// are stated at the top of rpy.cu.
#pragma once
#include "am_internal.cuh"

namespace am {

// ---------------------------------------------------------------- FP64 ---
struct RpyParamsDev {
    double a2, four_a2, inv8pieta, k_far2, k_far3, mu0, k_near1, k_near2;
};

__device__ __forceinline__ void pair_free_f64(double dx, double dy, double dz,
                                              double lx, double ly, double lz,
                                              const RpyParamsDev& p,
                                              double& ux, double& uy, double& uz) {
    double r2 = dx * dx + dy * dy + dz * dz;
    double c1, c2;
    if (r2 >= p.four_a2) {
        double ri = rsqrt(r2);
        double ri2 = ri * ri;
        c1 = ri * fma(p.k_far2, ri2, p.inv8pieta);
        c2 = ri * ri2 * fma(-p.k_far3, ri2, p.inv8pieta);
    } else {
        double r = sqrt(r2);
        c1 = p.mu0 * fma(-p.k_near1, r, 1.0);
        c2 = (r2 > 0.0) ? p.k_near2 / r : 0.0;
    }
    double s = c2 * (dx * lx + dy * ly + dz * lz);
    ux = fma(c1, lx, fma(s, dx, ux));
    uy = fma(c1, ly, fma(s, dy, uy));
    uz = fma(c1, lz, fma(s, dz, uz));
}

__device__ __forceinline__ void pair_image_f64(double Rx, double Ry, double Rz,
                                               double x3, double h,
                                               double lx, double ly, double lz,
                                               const RpyParamsDev& p,
                                               double& ux, double& uy, double& uz) {
    double s = rsqrt(Rx * Rx + Ry * Ry + Rz * Rz);
    double s2 = s * s;
    double hs = h * s;
    double hx = hs * (x3 * s);
    double ez = Rz * s;
    double ez2 = ez * ez;
    double A = p.a2 * s2;
    double A2 = A * A;
    double cI = -1.0 - 2.0 * hx + A * fma(2.0, ez2, -2.0 / 3.0) + A2 * fma(-10.0 / 3.0, ez2, 2.0 / 3.0);
    double cRR = -1.0 + 6.0 * hx + A * fma(-10.0, ez2, 2.0) + A2 * fma(70.0 / 3.0, ez2, -10.0 / 3.0);
    double cRz = fma(ez, -12.0 * hx + A * fma(20.0, ez2, -4.0) + A2 * fma(-140.0 / 3.0, ez2, 40.0 / 3.0), 2.0 * hs);
    double czR = fma(-20.0 / 3.0 * A2, ez, 2.0 * hs);
    double czz = -4.0 * hs * hs - 4.0 * A * ez2 + A2 * fma(20.0, ez2, -8.0 / 3.0);
    double rx = Rx * s, ry = Ry * s;
    double dotR = rx * lx + ry * ly + ez * lz;
    double t = fma(cRR, dotR, cRz * lz);
    double pre = p.inv8pieta * s;
    ux = fma(pre, fma(cI, lx, t * rx), ux);
    uy = fma(pre, fma(cI, ly, t * ry), uy);
    uz = fma(pre, fma(cI, lz, fma(t, ez, fma(czR, dotR, czz * lz))), uz);
}

// --------------------------------------------------------------- mixed ---
struct RpyParamsF {
    float a2, four_a2, inv8pieta, k_far2, k_far3, mu0, k_near1, k_near2;
};

__device__ __forceinline__ void pair_free_f32(float dx, float dy, float dz,
                                              float lx, float ly, float lz,
                                              const RpyParamsF& p,
                                              float& ux, float& uy, float& uz) {
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float c1, c2;
    if (r2 >= p.four_a2) {
        float ri = rsqrtf(r2);
        float ri2 = ri * ri;
        c1 = ri * fmaf(p.k_far2, ri2, p.inv8pieta);
        c2 = ri * ri2 * fmaf(-p.k_far3, ri2, p.inv8pieta);
    } else {
        float r = sqrtf(r2);
        c1 = p.mu0 * fmaf(-p.k_near1, r, 1.0f);
        c2 = (r2 > 0.0f) ? p.k_near2 / r : 0.0f;
    }
    float s = c2 * fmaf(dx, lx, fmaf(dy, ly, dz * lz));
    ux = fmaf(c1, lx, fmaf(s, dx, ux));
    uy = fmaf(c1, ly, fmaf(s, dy, uy));
    uz = fmaf(c1, lz, fmaf(s, dz, uz));
}

__device__ __forceinline__ void pair_image_f32(float Rx, float Ry, float Rz, float x3, float h,
                                               float lx, float ly, float lz,
                                               const RpyParamsF& p,
                                               float& ux, float& uy, float& uz) {
    float s = rsqrtf(fmaf(Rx, Rx, fmaf(Ry, Ry, Rz * Rz)));
    float s2 = s * s;
    float hs = h * s;
    float hx = hs * (x3 * s);
    float ez = Rz * s;
    float ez2 = ez * ez;
    float A = p.a2 * s2;
    float A2 = A * A;
    float cI = -1.0f - 2.0f * hx + A * fmaf(2.0f, ez2, -2.0f / 3.0f) + A2 * fmaf(-10.0f / 3.0f, ez2, 2.0f / 3.0f);
    float cRR = -1.0f + 6.0f * hx + A * fmaf(-10.0f, ez2, 2.0f) + A2 * fmaf(70.0f / 3.0f, ez2, -10.0f / 3.0f);
    float cRz = fmaf(ez, -12.0f * hx + A * fmaf(20.0f, ez2, -4.0f) + A2 * fmaf(-140.0f / 3.0f, ez2, 40.0f / 3.0f), 2.0f * hs);
    float czR = fmaf(-20.0f / 3.0f * A2, ez, 2.0f * hs);
    float czz = -4.0f * hs * hs - 4.0f * A * ez2 + A2 * fmaf(20.0f, ez2, -8.0f / 3.0f);
    float rx = Rx * s, ry = Ry * s;
    float dotR = fmaf(rx, lx, fmaf(ry, ly, ez * lz));
    float t = fmaf(cRR, dotR, cRz * lz);
    float pre = p.inv8pieta * s;
    ux = fmaf(pre, fmaf(cI, lx, t * rx), ux);
    uy = fmaf(pre, fmaf(cI, ly, t * ry), uy);
    uz = fmaf(pre, fmaf(cI, lz, fmaf(t, ez, fmaf(czR, dotR, czz * lz))), uz);
}


// Full 3x3 tensor T (row-major, T[3a+b]: velocity a at x from force b at y).
__device__ __forceinline__ void pair_tensor_f64(double4_32a x, double4_32a y, const RpyParamsDev& p,
                                                int wall, double* T) {
    for (int b = 0; b < 3; ++b) {
        double l[3] = {0.0, 0.0, 0.0};
        l[b] = 1.0;
        double ux = 0.0, uy = 0.0, uz = 0.0;
        pair_free_f64(x.x - y.x, x.y - y.y, x.z - y.z, l[0], l[1], l[2], p, ux, uy, uz);
        if (wall) pair_image_f64(x.x - y.x, x.y - y.y, x.z + y.z, x.z, y.z, l[0], l[1], l[2], p, ux, uy, uz);
        T[b] = ux; T[3 + b] = uy; T[6 + b] = uz;
    }
}

inline RpyParamsDev dev_params(const RpyParams& q) {
    return RpyParamsDev{q.a2, q.four_a2, q.inv8pieta, q.k_far2, q.k_far3, q.mu0, q.k_near1, q.k_near2};
}

}  // namespace am

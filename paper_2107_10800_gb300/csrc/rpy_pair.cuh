// Pair terms of the blob mobility (Sec. 2.3, Eq. RPY), shared by the
// all-pairs product and the preconditioner's same-body blocks.
//
// The functions accumulate u / A1 with A1 = 1/(8 pi eta); callers multiply
// the sums by A1 once.  With d = r_i - r_j, r = |d|, ri = 1/r:
//   free, r >= 2a:  c1 = ri (1 + (2a^2/3) ri^2),  c2 = ri^3 (1 - 2a^2 ri^2)
//   free, r <  2a:  c1 = (4/(3a)) (1 - 9r/(32a)), c2 = 1/(8 a^2 r)  (0 at r = 0)
//   u/A1 += c1 lambda + c2 d (d . lambda)
// which is (1/(8 pi eta r)) [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) dhat dhat]
// far and mu0 [(1 - 9r/(32a)) I + (3r/(32a)) dhat dhat] near, mu0 = 1/(6 pi eta a).
//
// Wall image part, R = x - y* (y* the mirror image of the source in z = 0),
// s = 1/|R|, Rh = R s, h = source height, x3 = target height, ez = R3 s,
// A = a^2 s^2, u = h x3 s^2, t1 = A ez^2, t2 = A^2 ez^2:
//   cI  = -1 - 2u - 2/3 A + 2 t1 + 2/3 A^2 - 10/3 t2
//   cRR = -1 + 6u + 2 A - 10 t1 - 10/3 A^2 + 70/3 t2
//   cRz = 2 h s + ez (-2 cRR - 2 + 20/3 A^2)
//   czR = 2 h s - 20/3 A^2 ez
//   czz = -4 (h s)^2 - 4 t1 - 8/3 A^2 + 20 t2
//   u/A1 += s [cI lambda + (cRR (Rh.lambda) + cRz lambda_3) Rh
//              + (czR (Rh.lambda) + czz lambda_3) e3]
// (the image terms of Blake's Green's function averaged over both blob
// surfaces, (1 + a^2/6 lap_x)(1 + a^2/6 lap_y), exact for blobs above a).
#pragma once
#include "am_internal.cuh"

namespace am {

template <class T>
struct RpyK {
    T a2;        // a^2
    T four_a2;   // 4 a^2 (contact distance squared)
    T kf2;       // 2 a^2 / 3
    T kf3;       // 2 a^2
    T kn0;       // 4 / (3 a)
    T kn1;       // 9 / (32 a)
    T kn2;       // 1 / (8 a^2)
    // wall coefficients of pair_wall (polynomial form in w = s^2)
    T wc1;       // -2 a^2 / 3
    T w2a2;      // 2 a^2
    T wc2;       // 2 a^4 / 3
    T wc3;       // -10 a^4 / 3
    T wa4;       // 20 a^4 / 3
    T wi2;       // -4 a^4 / 3
    double A1;   // 1 / (8 pi eta)
};

template <class T>
inline RpyK<T> rpy_consts(const RpyParams& q) {
    RpyK<T> k;
    k.a2 = (T)q.a2;
    k.four_a2 = (T)q.four_a2;
    k.kf2 = (T)(2.0 * q.a2 / 3.0);
    k.kf3 = (T)(2.0 * q.a2);
    k.kn0 = (T)(4.0 / (3.0 * q.a));
    k.kn1 = (T)(9.0 / (32.0 * q.a));
    k.kn2 = (T)(1.0 / (8.0 * q.a2));
    const double a4 = q.a2 * q.a2;
    k.wc1 = (T)(-2.0 * q.a2 / 3.0);
    k.w2a2 = (T)(2.0 * q.a2);
    k.wc2 = (T)(2.0 * a4 / 3.0);
    k.wc3 = (T)(-10.0 * a4 / 3.0);
    k.wa4 = (T)(20.0 * a4 / 3.0);
    k.wi2 = (T)(-4.0 * a4 / 3.0);
    k.A1 = q.inv8pieta;
    return k;
}

// FP32: the hardware estimate (PTX rsqrt.approx, relative error below
// 2^-22.9) without the subnormal path, which no argument here needs: they
// are squared distances of at least (2a)^2 or squared image distances of
// at least the squared sum of two heights above the wall
__device__ __forceinline__ float rsq(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float sqt(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqt(double x) { return sqrt(x); }

// the free-space coefficients c1, c2 of a pair at squared distance r2
template <class T>
__device__ __forceinline__ void free_coefs(T r2, const RpyK<T>& k, T& c1, T& c2) {
    if (r2 >= k.four_a2) {
        const T ri = rsq(r2);
        const T ri2 = ri * ri;
        c1 = ri * fma(k.kf2, ri2, (T)1);
        c2 = (ri * ri2) * fma(-k.kf3, ri2, (T)1);
    } else {
        const T r = sqt(r2);
        c1 = k.kn0 * fma(-k.kn1, r, (T)1);
        c2 = (r2 > (T)0) ? k.kn2 / r : (T)0;
    }
}

template <class T>
__device__ __forceinline__ void pair_free_r2(T dx, T dy, T dz, T r2, T lx, T ly, T lz,
                                             const RpyK<T>& k, T& ux, T& uy, T& uz) {
    T c1, c2;
    free_coefs<T>(r2, k, c1, c2);
    const T sdl = c2 * fma(dx, lx, fma(dy, ly, dz * lz));
    ux = fma(c1, lx, fma(sdl, dx, ux));
    uy = fma(c1, ly, fma(sdl, dy, uy));
    uz = fma(c1, lz, fma(sdl, dz, uz));
}

template <class T>
__device__ __forceinline__ void pair_free(T dx, T dy, T dz, T lx, T ly, T lz, const RpyK<T>& k,
                                          T& ux, T& uy, T& uz) {
    pair_free_r2<T>(dx, dy, dz, fma(dx, dx, fma(dy, dy, dz * dz)), lx, ly, lz, k, ux, uy, uz);
}

// The image coefficients of one pair (see the header): s = 1/|R|, the
// direction Rh = (rx, ry, ez) and cI, cRR, cRz, czR, czz
template <class T>
struct ImageCoefs {
    T s, rx, ry, ez, cI, cRR, cRz, czR, czz;
};

template <class T>
__device__ __forceinline__ ImageCoefs<T> image_coefs(T Rx, T Ry, T Rz, T x3, T h, const RpyK<T>& k) {
    ImageCoefs<T> c;
    const T s = rsq(fma(Rx, Rx, fma(Ry, Ry, Rz * Rz)));
    const T s2 = s * s;
    const T hs = h * s;
    const T u = hs * (x3 * s);
    const T ez = Rz * s;
    const T ez2 = ez * ez;
    const T A = k.a2 * s2;
    const T A2 = A * A;
    const T t1 = A * ez2;
    const T t2 = A2 * ez2;
    c.cI = fma((T)(-10.0 / 3.0), t2, fma((T)(2.0 / 3.0), A2, fma((T)2, t1, fma((T)(-2.0 / 3.0), A, fma((T)-2, u, (T)-1)))));
    c.cRR = fma((T)(70.0 / 3.0), t2, fma((T)(-10.0 / 3.0), A2, fma((T)-10, t1, fma((T)2, A, fma((T)6, u, (T)-1)))));
    const T inner = fma((T)(20.0 / 3.0), A2, fma((T)-2, c.cRR, (T)-2));
    const T hs2 = (T)2 * hs;
    c.cRz = fma(ez, inner, hs2);
    c.czR = fma((T)(-20.0 / 3.0) * A2, ez, hs2);
    c.czz = fma((T)-4, hs * hs, fma((T)20, t2, fma((T)(-8.0 / 3.0), A2, (T)-4 * t1)));
    c.s = s;
    c.rx = Rx * s;
    c.ry = Ry * s;
    c.ez = ez;
    return c;
}

template <class T>
__device__ __forceinline__ void pair_image(T Rx, T Ry, T Rz, T x3, T h, T lx, T ly, T lz,
                                           const RpyK<T>& k, T& ux, T& uy, T& uz) {
    const ImageCoefs<T> c = image_coefs<T>(Rx, Ry, Rz, x3, h, k);
    const T dotR = fma(c.rx, lx, fma(c.ry, ly, c.ez * lz));
    const T t = fma(c.cRR, dotR, c.cRz * lz);
    ux = fma(c.s, fma(c.cI, lx, t * c.rx), ux);
    uy = fma(c.s, fma(c.cI, ly, t * c.ry), uy);
    uz = fma(c.s, fma(c.cI, lz, fma(t, c.ez, fma(c.czR, dotR, c.czz * lz))), uz);
}

// Free-space pair plus wall image of one source, fused (the sum of
// pair_free_r2 and pair_image, reorganised; the products are the same up to
// rounding).  With w = s^2, R = (dx, dy, Rz), h2 = 2h, D = R . lambda and
//   c1 = -2 h x3 - 2a^2/3,  c2 = 2a^2 Rz^2 + 2a^4/3,  c3 = -10a^4 Rz^2 / 3,
// the image coefficients above are polynomials in w:
//   cI  = -1 + w c1 + w^2 c2 + w^3 c3
//   cRR = -1 - 3 w c1 - 5 w^2 c2 - 7 w^3 c3 = -4 - 3 cI - 2 w^2 (c2 + 2 w c3)
//   s^2 cRz = s^3 (2h + Rz (20/3 a^4 w^2 - 2 cRR - 2))
//   s^2 czR = s^3 (2h - 20/3 a^4 w^2 Rz)
//   s czz   = s^3 (-4h^2 - 2 w (c2 + 3 w c3) - 4/3 a^4 w)
// and, applied to the unnormalised R (Rh = R s, Rh . lambda = s D),
//   u/A1 += s cI lambda + P R + Q e3,
//   P = s^3 cRR D + s^2 cRz lambda_3,  Q = s^2 czR D + s czz lambda_3.
// In Q, 2h D - 4h^2 lambda_3 = 2h (d . lambda) because D - 2h lambda_3 =
// d . lambda (R_z - 2h = d_z), so
//   Q = s^3 (2h (d . lambda) - 20/3 a^4 w^2 Rz D
//            + w (-2 (c2 + 3 w c3) - 4/3 a^4) lambda_3)
// with no negated operand (the paired-lane form has no free negation).
// The free and image parts share one multiply-add per component of lambda
// and of d (R_x = d_x, R_y = d_y).  rxy2 = dx^2 + dy^2 and r2 = rxy2 + dz^2
// come from the caller; nx3 = -x3 (target height).
template <class T>
__device__ __forceinline__ void pair_wall_r2(T dx, T dy, T dz, T rxy2, T r2, T Rz, T h2, T nx3, T lx,
                                             T ly, T lz, const RpyK<T>& k, T& ux, T& uy, T& uz) {
    const T Rz2 = Rz * Rz;
    const T dlxy = fma(dx, lx, dy * ly);
    const T Df = fma(dz, lz, dlxy);   // d . lambda
    const T Di = fma(Rz, lz, dlxy);   // R . lambda
    T c1f, c2f;
    free_coefs<T>(r2, k, c1f, c2f);
    const T sdl = c2f * Df;
    const T s = rsq(rxy2 + Rz2);
    const T w = s * s, s3 = s * w, w2 = w * w;
    const T c1 = fma(h2, nx3, k.wc1);
    const T c2 = fma(Rz2, k.w2a2, k.wc2);
    const T c3 = Rz2 * k.wc3;
    const T x1 = fma(w, c3, c2);
    const T cI = fma(w, fma(w, x1, c1), (T)-1);
    const T y = fma(w, c3, x1);                 // c2 + 2 w c3
    const T yz = fma(w, c3, y);                 // c2 + 3 w c3
    const T cRR = fma(w2 * y, (T)-2, fma(cI, (T)-3, (T)-4));
    const T A4w2n = w2 * -k.wa4;                // -20/3 a^4 w^2
    const T P = s3 * fma(cRR, Di, fma(Rz, fma(cRR, (T)-2, fma(A4w2n, (T)-1, (T)-2)), h2) * lz);
    const T Q = s3 * fma(h2, Df, fma(A4w2n * Rz, Di, (w * fma(yz, (T)-2, k.wi2)) * lz));
    const T cc = fma(s, cI, c1f);
    const T pp = sdl + P;
    ux = fma(cc, lx, fma(pp, dx, ux));
    uy = fma(cc, ly, fma(pp, dy, uy));
    uz = fma(cc, lz, fma(sdl, dz, fma(P, Rz, uz + Q)));
}

// Both directions of one pair from one evaluation (the mobility is
// symmetric: M_ji = M_ij^T).  u/A1 += M_ij lambda_j at the target as
// pair_wall_r2 (same arguments: d = x_i - x_j, Rz = z_i + z_j, h2 = 2 z_j,
// nx3 = -z_i) and v/A1 += M_ij^T mu_i at the source, the velocity that
// target i's force mu causes there.  Written as a tensor applied to lambda,
// pair_wall_r2 is
//   cc I + c2f d d^T + s^3 cRR R R^T + s^3 g R e3^T
//        + s^3 e3 (h2 d^T - (20/3) a^4 w^2 Rz R^T) + s^3 phi e3 e3^T,
// g = Rz inner + h2, phi = w (c2-term of Q), so the transpose multiplies mu
// with the d, R and e3 coefficients
//   c2f (d . mu) + s^3 h2 mu_3,  s^3 cRR (R . mu) - (20/3) s^3 a^4 w^2 Rz mu_3,
//   s^3 g (R . mu) + s^3 phi mu_3.
// The coefficients are shared; the second direction costs about 20
// operations against about 60 for a separate evaluation.
template <class T>
__device__ __forceinline__ void pair_wall_sym(T dx, T dy, T dz, T rxy2, T r2, T Rz, T h2, T nx3, T lx, T ly,
                                              T lz, T mx, T my, T mz, const RpyK<T>& k, T& ux, T& uy, T& uz,
                                              T& vx, T& vy, T& vz) {
    const T Rz2 = Rz * Rz;
    T c1f, c2f;
    free_coefs<T>(r2, k, c1f, c2f);
    const T s = rsq(rxy2 + Rz2);
    const T w = s * s, s3 = s * w, w2 = w * w;
    const T c1 = fma(h2, nx3, k.wc1);
    const T c2 = fma(Rz2, k.w2a2, k.wc2);
    const T c3 = Rz2 * k.wc3;
    const T x1 = fma(w, c3, c2);
    const T cI = fma(w, fma(w, x1, c1), (T)-1);
    const T y = fma(w, c3, x1);                 // c2 + 2 w c3
    const T yz = fma(w, c3, y);                 // c2 + 3 w c3
    const T cRR = fma(w2 * y, (T)-2, fma(cI, (T)-3, (T)-4));
    const T A4w2n = w2 * -k.wa4;                // -20/3 a^4 w^2
    const T cc = fma(s, cI, c1f);
    const T g = fma(Rz, fma(cRR, (T)-2, fma(A4w2n, (T)-1, (T)-2)), h2);
    const T s3cRR = s3 * cRR, s3g = s3 * g, s3h2 = s3 * h2;
    const T s3A = s3 * (A4w2n * Rz), s3phi = s3 * (w * fma(yz, (T)-2, k.wi2));
    {   // u += M_ij lambda
        const T dlxy = fma(dx, lx, dy * ly);
        const T Df = fma(dz, lz, dlxy), Di = fma(Rz, lz, dlxy);
        const T sdl = c2f * Df;
        const T P = fma(s3cRR, Di, s3g * lz);
        const T Q = fma(s3h2, Df, fma(s3A, Di, s3phi * lz));
        const T pp = sdl + P;
        ux = fma(cc, lx, fma(pp, dx, ux));
        uy = fma(cc, ly, fma(pp, dy, uy));
        uz = fma(cc, lz, fma(sdl, dz, fma(P, Rz, uz + Q)));
    }
    {   // v += M_ij^T mu
        const T dmxy = fma(dx, mx, dy * my);
        const T Df = fma(dz, mz, dmxy), Di = fma(Rz, mz, dmxy);
        const T cd = fma(c2f, Df, s3h2 * mz);
        const T P = fma(s3cRR, Di, s3A * mz);
        const T Q = fma(s3g, Di, s3phi * mz);
        const T pp = cd + P;
        vx = fma(cc, mx, fma(pp, dx, vx));
        vy = fma(cc, my, fma(pp, dy, vy));
        vz = fma(cc, mz, fma(cd, dz, fma(P, Rz, vz + Q)));
    }
}

// Free space: the RPY tensor is symmetric in the pair and even in d
template <class T>
__device__ __forceinline__ void pair_free_sym(T dx, T dy, T dz, T r2, T lx, T ly, T lz, T mx, T my, T mz,
                                              const RpyK<T>& k, T& ux, T& uy, T& uz, T& vx, T& vy, T& vz) {
    T c1, c2;
    free_coefs<T>(r2, k, c1, c2);
    const T sl = c2 * fma(dx, lx, fma(dy, ly, dz * lz));
    const T sm = c2 * fma(dx, mx, fma(dy, my, dz * mz));
    ux = fma(c1, lx, fma(sl, dx, ux));
    uy = fma(c1, ly, fma(sl, dy, uy));
    uz = fma(c1, lz, fma(sl, dz, uz));
    vx = fma(c1, mx, fma(sm, dx, vx));
    vy = fma(c1, my, fma(sm, dy, vy));
    vz = fma(c1, mz, fma(sm, dz, vz));
}

// Full 3 x 3 tensor Tt (row-major, Tt[3a + b]: velocity a at x from force b
// at y), including the 1/(8 pi eta) factor, for d = x - y and the heights
// xz, yz of x and y: the operators of pair_free_r2 and pair_image written
// out, c1 I + c2 d d^T and (wall) s (cI I + cRR Rh Rh^T + cRz Rh e3^T +
// czR e3 Rh^T + czz e3 e3^T).
template <class T>
__device__ __forceinline__ void pair_tensor(T dx, T dy, T dz, T xz, T yz, const RpyK<T>& k, int wall, T* Tt) {
    T c1, c2;
    free_coefs<T>(fma(dx, dx, fma(dy, dy, dz * dz)), k, c1, c2);
    const T d[3] = {dx, dy, dz};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Tt[3 * a + b] = (a == b ? c1 : (T)0) + c2 * d[a] * d[b];
    if (wall) {
        const ImageCoefs<T> c = image_coefs<T>(dx, dy, xz + yz, xz, yz, k);
        const T Rh[3] = {c.rx, c.ry, c.ez};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                T v = c.cRR * Rh[a] * Rh[b] + (a == b ? c.cI : (T)0);
                if (b == 2) v += c.cRz * Rh[a];
                if (a == 2) v += c.czR * Rh[b];
                if (a == 2 && b == 2) v += c.czz;
                Tt[3 * a + b] += c.s * v;
            }
    }
    const T A1 = (T)k.A1;
    for (int q = 0; q < 9; ++q) Tt[q] *= A1;
}

// the constants in another precision
template <class T>
__device__ __host__ inline RpyK<T> rpy_cast(const RpyK<double>& q) {
    RpyK<T> k;
    k.a2 = (T)q.a2; k.four_a2 = (T)q.four_a2; k.kf2 = (T)q.kf2; k.kf3 = (T)q.kf3;
    k.kn0 = (T)q.kn0; k.kn1 = (T)q.kn1; k.kn2 = (T)q.kn2;
    k.wc1 = (T)q.wc1; k.w2a2 = (T)q.w2a2; k.wc2 = (T)q.wc2; k.wc3 = (T)q.wc3; k.wa4 = (T)q.wa4; k.wi2 = (T)q.wi2;
    k.A1 = q.A1;
    return k;
}

}  // namespace am

// Periodic blob mobility: u = M_per lambda for the free-space RPY tensor
// (Sec. 2.3, Eq. RPY: the Oseen tensor averaged over both blob surfaces)
// periodised over a box Lx x Ly x Lz with zero mean flow, the periodic
// boundary conditions of the suspension runs of Sec. 5.3, by spectral Ewald
// summation in O(N log N) instead of the O(N^2) all-pairs sum.
//
// In Fourier space the periodic mobility is sinc^2(ka) (I - khat khat) /
// (eta k^2) over the nonzero wave vectors of the box.  Ewald's split with
// Hasimoto's function H(k) = (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2)):
//  - real space: M_RPY(d) - W(d) over pairs closer than r_c (minimum image),
//    W the R^3 inverse transform of the wave multiplier, W(r) = (A I +
//    B rhat rhat) / eta with the radial integrals
//        A = 1/(2 pi^2) int H sinc^2(ka) [(2/3) j0(kr) - j2(kr)/3] dk,
//        B = 1/(2 pi^2) int H sinc^2(ka) j2(kr) dk,
//    tabulated in s = r^2 (A and B/s are smooth functions of s) by
//    Gauss-Legendre quadrature; M_RPY in closed form (rpy_pair.cuh).  The
//    pair blocks depend on the pose only, so they are formed once per pose
//    into a sparse block matrix (CSR over the blobs in cell order, 6
//    doubles per pair) that every product reads;
//  - wave space: the forces are spread onto a uniform grid with the
//    "exponential of semicircle" window phi(z) = exp(beta (sqrt(1 - z^2) -
//    1)), z = t / (w h / 2), over w x w x w points (the window of Barnett,
//    Magland and af Klinteberg's non-uniform FFT), transformed (cuFFT, the
//    three components batched), multiplied by sinc^2(ka) H(k) (I - khat
//    khat) / (eta k^2) / Phi(k)^2 (Phi the window's transform, computed by
//    quadrature; the division undoes the spreading and the interpolation),
//    transformed back and interpolated at the blobs with the same window.
//    The spreading adds into the grid with FP64 atomics, so the last bits of
//    the wave part depend on the order of arrival.
//
// Parameters from the relative tolerance eps (lg = ln(1/eps)): grid spacing
// h = pi / (2 xi sqrt(lg + ln(1 + lg))) (the wave multiplier below eps
// beyond the grid's Nyquist wave number; wave vectors beyond that radius are
// dropped), window width w = ceil(log10(1/eps)) + 1 points with beta = 2.6 w,
// r_c = 2a + sqrt(0.8 lg) / xi (the real part below eps mu0 beyond it); xi
// minimises a cost model of the product (real-space pairs read against grid
// points transformed, weights measured on GB300) subject to r_c <= min(L)/3
// (three cells per side).
// These rules were calibrated against the Ewald sum evaluated to rounding
// (width 9 gives 7e-10 relative, 11 gives 2e-11).
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "am_internal.cuh"
#include "ops.cuh"
#include "rpy_pair.cuh"

namespace am {

// The wave-space part at one precision (T = double for the FP64 product,
// float for the mixed one): window, grid, its half spectra, the multiplier
// and the cuFFT plans.
struct Wave {
    int P = 0, M[3] = {0, 0, 0};            // window width w, grid points per side
    double beta = 0, kcut = 0, h[3] = {0, 0, 0};
    long long ngrid = 0, nhat = 0;          // real points, half-spectrum points
    void* grid = nullptr;                   // 3 x ngrid T
    void* hat = nullptr;                    // 3 x nhat complex T
    void* kfac = nullptr;                   // (fac, fac / k^2) per half-spectrum point, T
    cufftHandle fwd = 0, inv = 0;
    bool planned = false;
};

struct PeriodicPlan {
    double L[3] = {0, 0, 0};
    double xi = 0, rc = 0, tol = 0;
    int nc[3] = {0, 0, 0}, ncell = 0;      // cells per side (side >= r_c)
    int ntab = 0;
    double ds = 0;                          // table step in s = r^2
    int Nb = 0;
    Wave w64, w32;                          // FP64 wave part; FP32 one for mixed handles
    bool has32 = false;
    // device
    double2* d_tab = nullptr;               // (A(s), B(s)/s)
    int* d_cell_start = nullptr;            // ncell + 1
    int* d_cell_fill = nullptr;             // ncell
    int* d_cell_of = nullptr;               // Nb
    int* d_order = nullptr;                 // sorted position -> blob
    double4_32a* d_spos = nullptr;          // sorted wrapped positions
    float4* d_sposf = nullptr;              // the same in FP32 (cut test)
    long long* d_row = nullptr;             // Nb + 1 CSR offsets
    int* d_nbr = nullptr;                   // neighbour blob indices
    double* d_blk = nullptr;                // 6 x cap pair blocks (SoA)
    float* d_blk32 = nullptr;               // the same in FP32 (mixed handles)
    long long cap = 0, nnz = 0;
    long long* d_scan = nullptr;            // scan scratch
    int* d_code = nullptr;                  // per pair: neighbour cell << 26 | source sorted index
    double4_32a* d_rprev = nullptr;         // positions of the last binning
    int* d_moved = nullptr;                 // set when a blob moved since d_rprev
    bool valid = false;  // pair blocks of the current pose are in place
};

namespace {

template <class T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };
template <class T> using vec2_t = typename Vec2<T>::type;
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }

constexpr int kTab = 16384;  // table nodes over [0, r_c^2]
constexpr int kScanBlock = 1024;

// ---- radial functions of the wave part (own series and closed forms) ----
// j2(x) / x^2 = sum_n (-x^2/2)^n / (n! (2n+5)!!)
__device__ __forceinline__ double j2_over_x2(double x) {
    if (x < 1.0) {
        const double y = -0.5 * x * x;
        double term = 1.0 / 15.0, sum = term;
        for (int n = 1; n < 10; ++n) {
            term *= y / ((double)n * (double)(2 * n + 5));
            sum += term;
        }
        return sum;
    }
    double s, c;
    sincos(x, &s, &c);
    const double xi = 1.0 / x;
    return ((3.0 * xi * xi - 1.0) * s * xi - 3.0 * c * xi * xi) * xi * xi;
}

__device__ __forceinline__ double j0f(double x) {
    if (x < 1e-3) return 1.0 - x * x / 6.0 + x * x * x * x / 120.0;
    return sin(x) / x;
}

// Table node t: s = t ds; A(s) and B(s)/s by the quadrature rule (nodes k_q,
// weights already times H(k_q) sinc^2(k_q a) / (2 pi^2)); one warp per node,
// lanes over the quadrature nodes, a shuffle tree for the sums.
__global__ void k_per_table(int ntab, double ds, const double* __restrict__ kq, const double* __restrict__ wq,
                            int nq, double2* __restrict__ tab) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntab) return;
    const double r = sqrt(t * ds);
    double A = 0.0, Bs = 0.0;
    for (int q = lane; q < nq; q += 32) {
        const double k = kq[q], x = k * r;
        const double q2 = j2_over_x2(x);
        const double j2 = x * x * q2;
        A = fma(wq[q], (2.0 / 3.0) * j0f(x) - j2 / 3.0, A);
        Bs = fma(wq[q] * k * k, q2, Bs);
    }
    for (int o = 16; o > 0; o >>= 1) {
        A += __shfl_xor_sync(0xffffffffu, A, o);
        Bs += __shfl_xor_sync(0xffffffffu, Bs, o);
    }
    if (lane == 0) tab[t] = make_double2(A, Bs);
}

// cubic Lagrange interpolation of the table at s (4 nodes around s)
__device__ __forceinline__ double2 tab_at(const double2* __restrict__ tab, int ntab, double inv_ds, double s) {
    const double u = s * inv_ds;
    int i = (int)u - 1;
    i = max(0, min(i, ntab - 4));
    const double t = u - (double)i;  // in [0, 3] up to the ends
    const double w0 = -(t - 1.0) * (t - 2.0) * (t - 3.0) / 6.0;
    const double w1 = t * (t - 2.0) * (t - 3.0) / 2.0;
    const double w2 = -t * (t - 1.0) * (t - 3.0) / 2.0;
    const double w3 = t * (t - 1.0) * (t - 2.0) / 6.0;
    const double2 a = tab[i], b = tab[i + 1], c = tab[i + 2], d = tab[i + 3];
    return make_double2(w0 * a.x + w1 * b.x + w2 * c.x + w3 * d.x, w0 * a.y + w1 * b.y + w2 * c.y + w3 * d.y);
}

// Wave multiplier per half-spectrum point (cuFFT D2Z layout of a Mz x My x
// Mx grid: index (iz My + iy)(Mx/2 + 1) + ix), with the normalisation of the
// spread -> forward -> inverse -> interpolate chain, hx hy hz / (Mx My Mz),
// divided by the window's transform squared (phx[|mx|] phy[|my|] phz[|mz|]
// per axis), and zero at k = 0, beyond |k| = kcut and on the Nyquist planes
// of even sizes.
template <class T>
__global__ void k_per_kfac(int Mx, int My, int Mz, double Lx, double Ly, double Lz, double a, double eta,
                           double xi, double kcut, const double* __restrict__ phx, const double* __restrict__ phy,
                           const double* __restrict__ phz, vec2_t<T>* __restrict__ kfac) {
    const long long Mxh = Mx / 2 + 1;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= Mxh * My * Mz) return;
    const int ix = (int)(q % Mxh), iy = (int)((q / Mxh) % My), iz = (int)(q / (Mxh * My));
    const int mx = ix, my = iy <= My / 2 ? iy : iy - My, mz = iz <= Mz / 2 ? iz : iz - Mz;
    const bool nyq = (Mx % 2 == 0 && 2 * ix == Mx) || (My % 2 == 0 && 2 * iy == My) || (Mz % 2 == 0 && 2 * iz == Mz);
    const double kx = 2.0 * kPi * mx / Lx, ky = 2.0 * kPi * my / Ly, kz = 2.0 * kPi * mz / Lz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    if (k2 == 0.0 || nyq || k2 > kcut * kcut) {
        kfac[q] = mk2((T)0, (T)0);
        return;
    }
    const double k = sqrt(k2), ka = k * a;
    const double sinc = ka < 1e-4 ? 1.0 - ka * ka / 6.0 : sin(ka) / ka;
    const double x = k2 / (4.0 * xi * xi);
    const double norm = (Lx / Mx) * (Ly / My) * (Lz / Mz) / ((double)Mx * (double)My * (double)Mz);
    const double ph = phx[ix] * phy[iy <= My / 2 ? iy : My - iy] * phz[iz <= Mz / 2 ? iz : Mz - iz];
    const double fac = norm / eta * sinc * sinc * (1.0 + x) * exp(-x) / (k2 * ph * ph);
    kfac[q] = mk2((T)fac, (T)(fac / k2));
}

// ---- cell list ------------------------------------------------------------
__device__ __forceinline__ double wrap1(double x, double L) {
    double w = x - L * floor(x / L);
    if (w >= L) w -= L;
    if (w < 0.0) w = 0.0;
    return w;
}

__global__ void k_per_cell(int Nb, const double4_32a* __restrict__ r4, double Lx, double Ly, double Lz, int ncx,
                           int ncy, int ncz, int* __restrict__ cell_of, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const double4_32a p = r4[i];
    const double x = wrap1(p.x, Lx), y = wrap1(p.y, Ly), z = wrap1(p.z, Lz);
    const int cx = min((int)(x / Lx * ncx), ncx - 1);
    const int cy = min((int)(y / Ly * ncy), ncy - 1);
    const int cz = min((int)(z / Lz * ncz), ncz - 1);
    const int c = (cz * ncy + cy) * ncx + cx;
    cell_of[i] = c;
    atomicAdd(&cnt[c], 1);
}

// exclusive scan of n counts (int or long long) into out (long long or int),
// three passes: block sums, a one-block scan of them, block offsets
template <class Tin>
__global__ void k_scan_blocks(const Tin* __restrict__ in, int n, long long* __restrict__ bsum) {
    __shared__ long long sh[32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    long long v = i < n ? (long long)in[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long w = sh[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = w;
    }
}

__global__ void k_scan_sums(long long* __restrict__ bsum, int nb) {
    // one block of kScanBlock threads; nb block sums, exclusive in place
    __shared__ long long sh[kScanBlock];
    long long carry = 0;
    for (int base = 0; base < nb; base += kScanBlock) {
        const int i = base + threadIdx.x;
        const long long v = i < nb ? bsum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kScanBlock; o <<= 1) {
            const long long add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        carry += sh[kScanBlock - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

template <class Tin, class Tout>
__global__ void k_scan_apply(const Tin* __restrict__ in, int n, const long long* __restrict__ bsum,
                             Tout* __restrict__ out) {
    __shared__ long long sh[kScanBlock];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const long long v = i < n ? (long long)in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        const long long add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += add;
        __syncthreads();
    }
    if (i < n) out[i] = (Tout)(bsum[blockIdx.x] + sh[threadIdx.x] - v);
    if (i == n - 1) out[n] = (Tout)(bsum[blockIdx.x] + sh[threadIdx.x]);
}

// out[0..n] = exclusive scan of in[0..n) with the total in out[n]
template <class Tin, class Tout>
void exclusive_scan(const Tin* in, int n, Tout* out, long long* scratch, cudaStream_t s) {
    const int nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_blocks<Tin><<<nb, kScanBlock, 0, s>>>(in, n, scratch);
    k_scan_sums<<<1, kScanBlock, 0, s>>>(scratch, nb);
    k_scan_apply<Tin, Tout><<<nb, kScanBlock, 0, s>>>(in, n, scratch, out);
    count_launch(3);
}

__global__ void k_per_fill(int Nb, const int* __restrict__ cell_of, const int* __restrict__ start,
                           int* __restrict__ fill, int* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const int c = cell_of[i];
    order[start[c] + atomicAdd(&fill[c], 1)] = i;
}

// the sorted wrapped positions (blobs of a cell in the order of arrival at
// k_per_fill, which only changes the order of the sums)
__global__ void k_per_gather_pos(int Nb, const int* __restrict__ order, const double4_32a* __restrict__ r4,
                                 double Lx, double Ly, double Lz, double4_32a* __restrict__ spos,
                                 float4* __restrict__ sposf) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Nb) return;
    const double4_32a r = r4[order[p]];
    double4_32a w;
    w.x = wrap1(r.x, Lx); w.y = wrap1(r.y, Ly); w.z = wrap1(r.z, Lz); w.w = 0.0;
    spos[p] = w;
    sposf[p] = make_float4((float)w.x, (float)w.y, (float)w.z, 0.f);
}

// Neighbour cell k (0..26) of the cell of (x, y, z): its index and the shift
// that brings its blobs next to the target (target - shift is compared).
struct CellGeom {
    int nc[3];
    double L[3];
};

__device__ __forceinline__ int neighbour_cell(const CellGeom& g, int cx, int cy, int cz, int k, double& sx,
                                              double& sy, double& sz) {
    int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
    int nx = cx + dx, ny = cy + dy, nz = cz + dz;
    sx = sy = sz = 0.0;
    if (nx < 0) { nx += g.nc[0]; sx = -g.L[0]; } else if (nx >= g.nc[0]) { nx -= g.nc[0]; sx = g.L[0]; }
    if (ny < 0) { ny += g.nc[1]; sy = -g.L[1]; } else if (ny >= g.nc[1]) { ny -= g.nc[1]; sy = g.L[1]; }
    if (nz < 0) { nz += g.nc[2]; sz = -g.L[2]; } else if (nz >= g.nc[2]) { nz -= g.nc[2]; sz = g.L[2]; }
    return (nz * g.nc[1] + ny) * g.nc[0] + nx;
}

__device__ __forceinline__ void cell_coords(const CellGeom& g, double x, double y, double z, int& cx, int& cy,
                                            int& cz) {
    cx = min((int)(x / g.L[0] * g.nc[0]), g.nc[0] - 1);
    cy = min((int)(y / g.L[1] * g.nc[1]), g.nc[1] - 1);
    cz = min((int)(z / g.L[2] * g.nc[2]), g.nc[2] - 1);
}

// Pairs of sorted target p within r_c, by an FP32 distance test that is the
// same in both passes: count them, or list them as codes (neighbour cell
// 0..26) << 26 | source sorted index, ascending within a row (cells in
// order, sources in sorted order within a cell).
template <bool WRITE>
__global__ void k_per_pairs(int Nb, CellGeom g, const double4_32a* __restrict__ spos,
                            const float4* __restrict__ sposf, const int* __restrict__ start, float rc2f,
                            long long* __restrict__ row, int* __restrict__ code, long long cap) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Nb) return;
    const double4_32a x = spos[p];
    const float4 xf = sposf[p];
    int cx, cy, cz;
    cell_coords(g, x.x, x.y, x.z, cx, cy, cz);
    long long out = WRITE ? row[p] : 0;
    int count = 0;
    for (int kc = 0; kc < 27; ++kc) {
        double sx, sy, sz;
        const int c = neighbour_cell(g, cx, cy, cz, kc, sx, sy, sz);
        const float tx = xf.x - (float)sx, ty = xf.y - (float)sy, tz = xf.z - (float)sz;
        for (int q = start[c]; q < start[c + 1]; ++q) {
            const float4 yf = sposf[q];
            const float dxf = tx - yf.x, dyf = ty - yf.y, dzf = tz - yf.z;
            if (fmaf(dxf, dxf, fmaf(dyf, dyf, dzf * dzf)) >= rc2f) continue;
            if (WRITE) {
                if (out < cap) code[out] = (kc << 26) | q;  // cap is the counted total
                ++out;
            } else {
                ++count;
            }
        }
    }
    if (!WRITE) row[p] = count;
}

// FP64 pair block M_RPY(d) - W(d) = alpha I + beta d d^T of target p and
// listed source q in neighbour cell kc (the six distinct entries)
__device__ __forceinline__ void pair_block(const CellGeom& g, int cx, int cy, int cz, const double4_32a& x,
                                           const double4_32a* __restrict__ spos, int q, int kc,
                                           const double2* __restrict__ tab, int ntab, double inv_ds,
                                           const RpyK<double>& k, double inv_eta, double* m) {
    double sx, sy, sz;
    neighbour_cell(g, cx, cy, cz, kc, sx, sy, sz);
    const double4_32a y = spos[q];
    const double dx = (x.x - sx) - y.x, dy = (x.y - sy) - y.y, dz = (x.z - sz) - y.z;
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    double c1, c2;
    free_coefs<double>(r2, k, c1, c2);
    const double2 w = tab_at(tab, ntab, inv_ds, r2);
    const double al = k.A1 * c1 - w.x * inv_eta;
    const double be = k.A1 * c2 - w.y * inv_eta;
    m[0] = fma(be, dx * dx, al);
    m[1] = be * dx * dy;
    m[2] = be * dx * dz;
    m[3] = fma(be, dy * dy, al);
    m[4] = be * dy * dz;
    m[5] = fma(be, dz * dz, al);
}

// Blocks of the listed pairs, one warp per target row (lanes over its
// pairs), and the source's blob index for the products.  MIRROR = false:
// the pairs with q >= p, in FP64; MIRROR = true: the pairs with q < p,
// copied from the entry (q -> p) of row q, which sits at code
// (26 - kc) << 26 | p (the opposite neighbour cell) and is found by binary
// search (the block is even in d); computed in FP64 when the FP32 cut
// listed only one direction.
template <bool MIRROR>
__global__ void __launch_bounds__(256)
k_per_blocks(int Nb, CellGeom g, const double4_32a* __restrict__ spos, const int* __restrict__ order,
             const long long* __restrict__ row, const int* __restrict__ code, int* __restrict__ nbr,
             double* __restrict__ blk, long long cap, const double2* __restrict__ tab, int ntab, double inv_ds,
             RpyK<double> k, double inv_eta) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= Nb) return;
    const double4_32a x = spos[p];
    int cx, cy, cz;
    cell_coords(g, x.x, x.y, x.z, cx, cy, cz);
    const long long e1 = min(row[p + 1], cap);
    for (long long e = row[p] + lane; e < e1; e += 32) {
        const int cd = code[e];
        const int q = cd & ((1 << 26) - 1), kc = cd >> 26;
        if (q >= Nb || kc < 0 || kc > 26) {  // never listed (the two FP32 passes agree): a zero block, in bounds
            nbr[e] = 0;
            for (int j = 0; j < 6; ++j) blk[j * cap + e] = 0.0;
            continue;
        }
        if ((q < p) != MIRROR) continue;
        nbr[e] = order[q];
        double m[6];
        bool have = false;
        if (MIRROR) {
            const int want = ((26 - kc) << 26) | p;
            long long lo = row[q], hi = min(row[q + 1], cap) - 1;
            while (lo <= hi) {
                const long long mid = (lo + hi) >> 1;
                const int v = code[mid];
                if (v == want) {
                    for (int j = 0; j < 6; ++j) m[j] = blk[j * cap + mid];
                    have = true;
                    break;
                }
                if (v < want) lo = mid + 1; else hi = mid - 1;
            }
        }
        if (!have) pair_block(g, cx, cy, cz, x, spos, q, kc, tab, ntab, inv_ds, k, inv_eta, m);
        for (int j = 0; j < 6; ++j) blk[j * cap + e] = m[j];
    }
}

// *moved = 1 if any blob moved since the last binning (x, y, z compared)
__global__ void k_per_moved(int Nb, const double4_32a* __restrict__ r4, const double4_32a* __restrict__ prev,
                            int* __restrict__ moved) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const double4_32a a = r4[i], b = prev[i];
    if (a.x != b.x || a.y != b.y || a.z != b.z) *moved = 1;
}

template <class T>
__global__ void k_per_zero(T* __restrict__ g, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        g[i] = (T)0;
}

// Window weight of lane l (< w = P) along one axis: grid index i0 + l (the
// w points nearest x) and exp(beta (sqrt(1 - z^2) - 1)), z = ((i0 + l) h -
// x) / (w h / 2)
struct SpreadGeom {
    int M[3], P;
    double h[3], inv_half[3], beta;
};

template <class T>
__device__ __forceinline__ void axis_weight(double x, int d, const SpreadGeom& g, int lane, int& idx, T& w) {
    const int i0 = (int)ceil(x / g.h[d] - 0.5 * g.P);
    int i = i0 + lane;
    const double z = ((double)i * g.h[d] - x) * g.inv_half[d];  // in FP64: positions far from the origin
    if constexpr (sizeof(T) == 8) {
        w = exp(g.beta * (sqrt(fmax(0.0, 1.0 - z * z)) - 1.0));
    } else {
        const float zf = (float)z;
        w = expf((float)g.beta * (sqrtf(fmaxf(0.f, 1.f - zf * zf)) - 1.f));
    }
    if (i < 0) i += g.M[d]; else if (i >= g.M[d]) i -= g.M[d];
    idx = i;
}

// Lanes of a warp: floor(32 / w) blobs side by side, w lanes each (sorted
// blob order); lane l of a blob owns the grid column x = i0x + l and walks
// the w x w (y, z) points.  Lanes past the last group only take part in the
// shuffles.
struct LaneMap {
    int sub, lp, base;  // blob slot in the warp, lane within the blob, first lane of the blob
    bool live;          // a lane of a blob that exists
    int p;              // the blob (sorted position), clamped into range
};

__device__ __forceinline__ LaneMap lane_map(int Nb, int P) {
    LaneMap m;
    const int per = 32 / P;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    m.sub = lane / P;
    m.lp = lane - m.sub * P;
    const bool slot = m.sub < per;
    if (!slot) { m.sub = 0; m.lp = lane; }
    m.base = m.sub * P;
    const int gid = warp * per + m.sub;
    m.live = slot && gid < Nb;
    m.p = min(gid, Nb - 1);
    return m;
}

// The lanes of a blob compute one window weight per axis each (their own
// grid column, row and layer); before the loops every lane collects the w
// weights and indices of the y and z axes into registers (4 w shuffles per
// blob instead of two per inner iteration).
template <class T, int P>
__device__ __forceinline__ void window_axes(const SpreadGeom& g, const LaneMap& m, const double4_32a& x, int& ix,
                                            T& wx, int* iy, T* wy, int* iz, T* wz) {
    int jy = 0, jz = 0;
    T vy = (T)0, vz = (T)0;
    ix = 0;
    wx = (T)0;
    if (m.lp < P) {
        axis_weight(x.x, 0, g, m.lp, ix, wx);
        axis_weight(x.y, 1, g, m.lp, jy, vy);
        axis_weight(x.z, 2, g, m.lp, jz, vz);
    }
#pragma unroll
    for (int t = 0; t < P; ++t) {
        wy[t] = __shfl_sync(0xffffffffu, vy, m.base + t);
        iy[t] = __shfl_sync(0xffffffffu, jy, m.base + t);
        wz[t] = __shfl_sync(0xffffffffu, vz, m.base + t);
        iz[t] = __shfl_sync(0xffffffffu, jz, m.base + t);
    }
}

template <class T, int P>
__global__ void __launch_bounds__(256)
k_per_spread(int Nb, SpreadGeom g, const double4_32a* __restrict__ spos, const int* __restrict__ order,
             const double* __restrict__ lam, T* __restrict__ grid, long long ngrid) {
    const LaneMap m = lane_map(Nb, P);
    const double4_32a x = spos[m.p];
    const int i = order[m.p];
    const T lx = (T)lam[3 * (size_t)i], ly = (T)lam[3 * (size_t)i + 1], lz = (T)lam[3 * (size_t)i + 2];
    int ix, iy[P], iz[P];
    T wx, wy[P], wz[P];
    window_axes<T, P>(g, m, x, ix, wx, iy, wy, iz, wz);
    if (!m.live) return;
    const T ax = wx * lx, ay = wx * ly, az = wx * lz;
#pragma unroll 1
    for (int pz = 0; pz < P; ++pz) {
        const long long zrow = (long long)iz[pz] * g.M[1];
#pragma unroll
        for (int py = 0; py < P; ++py) {
            const T w = wy[py] * wz[pz];
            const long long idx = (zrow + iy[py]) * g.M[0] + ix;
            atomicAdd(grid + idx, w * ax);
            atomicAdd(grid + ngrid + idx, w * ay);
            atomicAdd(grid + 2 * ngrid + idx, w * az);
        }
    }
}

// f_hat <- fac (f_hat - k (k . f_hat) / k^2) on the half spectrum
template <class T>
__global__ void k_per_kmul(int Mx, int My, int Mz, double Lx, double Ly, double Lz,
                           const vec2_t<T>* __restrict__ kfac, vec2_t<T>* __restrict__ hat, long long nhat) {
    using C = vec2_t<T>;
    const long long Mxh = Mx / 2 + 1;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= nhat) return;
    const C f = kfac[q];
    C* h0 = hat + q;
    C* h1 = hat + nhat + q;
    C* h2 = hat + 2 * nhat + q;
    if (f.x == (T)0) {
        *h0 = mk2((T)0, (T)0); *h1 = mk2((T)0, (T)0); *h2 = mk2((T)0, (T)0);
        return;
    }
    const int ix = (int)(q % Mxh), iy = (int)((q / Mxh) % My), iz = (int)(q / (Mxh * My));
    const int mx = ix, my = iy <= My / 2 ? iy : iy - My, mz = iz <= Mz / 2 ? iz : iz - Mz;
    const T kx = (T)(2.0 * kPi * mx / Lx), ky = (T)(2.0 * kPi * my / Ly), kz = (T)(2.0 * kPi * mz / Lz);
    const C a = *h0, b = *h1, c = *h2;
    const T dr = kx * a.x + ky * b.x + kz * c.x, di = kx * a.y + ky * b.y + kz * c.y;
    *h0 = mk2(f.x * a.x - f.y * kx * dr, f.x * a.y - f.y * kx * di);
    *h1 = mk2(f.x * b.x - f.y * ky * dr, f.x * b.y - f.y * ky * di);
    *h2 = mk2(f.x * c.x - f.y * kz * dr, f.x * c.y - f.y * kz * di);
}

// u_i = sum over its CSR row of the pair blocks times lambda_j (real space)
// + the interpolation of the wave-space field at r_i with the window; the
// lanes of lane_map, sums in a fixed order (lane-strided rows, the lanes of
// a blob added in lane order through shared memory).
template <class T, int P>
__global__ void __launch_bounds__(256)
k_per_gather(int Nb, SpreadGeom g, const double4_32a* __restrict__ spos, const int* __restrict__ order,
             const long long* __restrict__ row, const int* __restrict__ nbr, const T* __restrict__ blk,
             long long cap, const double* __restrict__ lam, const T* __restrict__ grid, long long ngrid,
             double* __restrict__ out) {
    __shared__ double part[256][3];
    const LaneMap m = lane_map(Nb, P);
    T ux = (T)0, uy = (T)0, uz = (T)0;
    if (m.live) {
        for (long long e = row[m.p] + m.lp; e < row[m.p + 1]; e += P) {
            const int j = nbr[e];
            const T lx = (T)lam[3 * (size_t)j], ly = (T)lam[3 * (size_t)j + 1], lz = (T)lam[3 * (size_t)j + 2];
            const T m00 = blk[e], m01 = blk[cap + e], m02 = blk[2 * cap + e];
            const T m11 = blk[3 * cap + e], m12 = blk[4 * cap + e], m22 = blk[5 * cap + e];
            ux = fma(m00, lx, fma(m01, ly, fma(m02, lz, ux)));
            uy = fma(m01, lx, fma(m11, ly, fma(m12, lz, uy)));
            uz = fma(m02, lx, fma(m12, ly, fma(m22, lz, uz)));
        }
    }
    const double4_32a x = spos[m.p];
    int ix, iy[P], iz[P];
    T wx, wy[P], wz[P];
    window_axes<T, P>(g, m, x, ix, wx, iy, wy, iz, wz);
    T vx = (T)0, vy = (T)0, vz = (T)0;
    if (m.live) {
#pragma unroll 1
        for (int pz = 0; pz < P; ++pz) {
            const long long zrow = (long long)iz[pz] * g.M[1];
#pragma unroll
            for (int py = 0; py < P; ++py) {
                const long long idx = (zrow + iy[py]) * g.M[0] + ix;
                const T w = wy[py] * wz[pz];
                vx = fma(w, __ldg(grid + idx), vx);
                vy = fma(w, __ldg(grid + ngrid + idx), vy);
                vz = fma(w, __ldg(grid + 2 * ngrid + idx), vz);
            }
        }
    }
    part[threadIdx.x][0] = (double)fma(wx, vx, ux);
    part[threadIdx.x][1] = (double)fma(wx, vy, uy);
    part[threadIdx.x][2] = (double)fma(wx, vz, uz);
    __syncwarp();
    if (m.live && m.lp == 0) {
        const int t0 = threadIdx.x;  // the blob's first lane
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int l = 0; l < P; ++l) {
            sx += part[t0 + l][0];
            sy += part[t0 + l][1];
            sz += part[t0 + l][2];
        }
        const int i = order[m.p];
        out[3 * (size_t)i] = sx;
        out[3 * (size_t)i + 1] = sy;
        out[3 * (size_t)i + 2] = sz;
    }
}

template <class T, int P>
void launch_window(int Nb, const SpreadGeom& g, const PeriodicPlan* p, const Wave& w, const T* blk,
                   const double* lam, double* out, bool spread, cudaStream_t s) {
    const int per_block = 8 * (32 / P);  // blobs per 256-thread block (lane_map)
    const int nb = (Nb + per_block - 1) / per_block;
    T* grid = static_cast<T*>(w.grid);
    if (spread)
        k_per_spread<T, P><<<nb, 256, 0, s>>>(Nb, g, p->d_spos, p->d_order, lam, grid, w.ngrid);
    else
        k_per_gather<T, P><<<nb, 256, 0, s>>>(Nb, g, p->d_spos, p->d_order, p->d_row, p->d_nbr, blk, p->cap, lam,
                                              grid, w.ngrid, out);
}

// window widths 4 .. 16 (tolerances 1e-3 .. 1e-15)
template <class T>
void launch_window_any(int Nb, const SpreadGeom& g, const PeriodicPlan* p, const Wave& w, const T* blk,
                       const double* lam, double* out, bool spread, cudaStream_t s) {
    switch (w.P) {
        case 4: launch_window<T, 4>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 5: launch_window<T, 5>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 6: launch_window<T, 6>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 7: launch_window<T, 7>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 8: launch_window<T, 8>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 9: launch_window<T, 9>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 10: launch_window<T, 10>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 11: launch_window<T, 11>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 12: launch_window<T, 12>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 13: launch_window<T, 13>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 14: launch_window<T, 14>(Nb, g, p, w, blk, lam, out, spread, s); break;
        case 15: launch_window<T, 15>(Nb, g, p, w, blk, lam, out, spread, s); break;
        default: launch_window<T, 16>(Nb, g, p, w, blk, lam, out, spread, s); break;
    }
}

// FP32 copy of the pair blocks (6 x cap, SoA) for the mixed product
__global__ void k_per_blk32(const double* __restrict__ blk, float* __restrict__ blk32, long long cap, long long nnz) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
         e += (long long)gridDim.x * blockDim.x)
        for (int j = 0; j < 6; ++j) blk32[j * cap + e] = (float)blk[j * cap + e];
}

// ---- host ------------------------------------------------------------------
int fft_size(int n) {  // smallest 2-3-5-smooth size >= n (cuFFT's fast radices)
    for (;; ++n) {
        int m = n;
        for (int f : {2, 3, 5})
            while (m % f == 0) m /= f;
        if (m == 1) return n;
    }
}

// 20-point Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_20)
void gauss_legendre20(double* x, double* w) {
    const int n = 20;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void free_wave(Wave& w) {
    if (w.planned) {
        cufftDestroy(w.fwd);
        cufftDestroy(w.inv);
    }
    void* ptrs[] = {w.grid, w.hat, w.kfac};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    w = Wave();
}

void free_plan(PeriodicPlan* p) {
    if (!p) return;
    free_wave(p->w64);
    free_wave(p->w32);
    void* ptrs[] = {p->d_tab,  p->d_cell_start, p->d_cell_fill, p->d_cell_of, p->d_order, p->d_spos,
                    p->d_sposf, p->d_row,     p->d_nbr,       p->d_blk,     p->d_scan,  p->d_code,
                    p->d_rprev, p->d_moved,   p->d_blk32};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

template <class T>
bool dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T)) == cudaSuccess;
}

SpreadGeom spread_geom(const Wave& w) {
    SpreadGeom g;
    for (int d = 0; d < 3; ++d) {
        g.M[d] = w.M[d];
        g.h[d] = w.h[d];
        g.inv_half[d] = 2.0 / (w.P * w.h[d]);
    }
    g.P = w.P;
    g.beta = w.beta;
    return g;
}

// Grid of the wave part for tolerance tol at splitting xi: the Nyquist wave
// number where the wave multiplier falls below tol, 2-3-5-smooth sizes.
long long wave_grid(const PeriodicPlan* p, double xi, double tol, int P, int* M) {
    const double lg = std::log(1.0 / tol), xN = lg + std::log1p(lg);
    const double hmax = kPi / (2.0 * xi * std::sqrt(xN));
    long long tot = 1;
    for (int d = 0; d < 3; ++d) {
        M[d] = fft_size(std::max(P + 1, (int)std::ceil(p->L[d] / hmax)));
        tot *= M[d];
    }
    return tot;
}

int window_width(double tol) { return std::min(16, std::max(4, (int)std::ceil(std::log10(1.0 / tol)) + 1)); }

// Buffers, cuFFT plans and multiplier of the wave part at precision T for
// tolerance tol (gx, gw: 20-point Gauss-Legendre rule).
template <class T>
int wave_setup(PeriodicPlan* p, Wave& w, double tol, double a, double eta, cudaStream_t s, const double* gx,
               const double* gw, std::string& err) {
    const double lg = std::log(1.0 / tol), xN = lg + std::log1p(lg);
    w.P = window_width(tol);
    w.beta = 2.6 * w.P;
    w.ngrid = wave_grid(p, p->xi, tol, w.P, w.M);
    for (int d = 0; d < 3; ++d) w.h[d] = p->L[d] / w.M[d];
    w.nhat = (long long)(w.M[0] / 2 + 1) * w.M[1] * w.M[2];
    w.kcut = 2.0 * p->xi * std::sqrt(xN);
    using C = vec2_t<T>;
    if (cudaMalloc(&w.grid, 3 * (size_t)w.ngrid * sizeof(T)) != cudaSuccess ||
        cudaMalloc(&w.hat, 3 * (size_t)w.nhat * sizeof(C)) != cudaSuccess ||
        cudaMalloc(&w.kfac, (size_t)w.nhat * sizeof(C)) != cudaSuccess) {
        cudaGetLastError();
        err = "periodic mobility: device allocation failed";
        return AM_ERR_CUDA;
    }
    int n3[3] = {w.M[2], w.M[1], w.M[0]};
    const bool f64 = sizeof(T) == 8;
    if (cufftPlanMany(&w.fwd, 3, n3, nullptr, 1, 0, nullptr, 1, 0, f64 ? CUFFT_D2Z : CUFFT_R2C, 3) !=
        CUFFT_SUCCESS) {
        err = "periodic mobility: cuFFT plan failed";
        return AM_ERR_CUDA;
    }
    if (cufftPlanMany(&w.inv, 3, n3, nullptr, 1, 0, nullptr, 1, 0, f64 ? CUFFT_Z2D : CUFFT_C2R, 3) !=
        CUFFT_SUCCESS) {
        cufftDestroy(w.fwd);
        err = "periodic mobility: cuFFT plan failed";
        return AM_ERR_CUDA;
    }
    w.planned = true;
    cufftSetStream(w.fwd, s);
    cufftSetStream(w.inv, s);
    // window transforms per axis at k = 2 pi m / L, m = 0 .. M/2:
    // Phi(k) = (w h / 2) int_{-1}^{1} exp(beta (sqrt(1 - z^2) - 1)) cos(k w h z / 2) dz
    // (composite 20-point Gauss-Legendre, 16 panels)
    std::vector<double> ph;
    int ph_off[4] = {0, 0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        const double half = 0.5 * w.P * w.h[d];
        for (int m = 0; m <= w.M[d] / 2; ++m) {
            const double k = 2.0 * kPi * m / p->L[d];
            double acc = 0.0;
            for (int pn = 0; pn < 16; ++pn) {
                const double z0 = -1.0 + 2.0 * pn / 16.0, zh = 1.0 / 16.0;
                for (int i = 0; i < 20; ++i) {
                    const double z = z0 + zh * (1.0 + gx[i]);
                    acc += zh * gw[i] * std::exp(w.beta * (std::sqrt(std::max(0.0, 1.0 - z * z)) - 1.0)) *
                           std::cos(k * half * z);
                }
            }
            ph.push_back(half * acc);
        }
        ph_off[d + 1] = (int)ph.size();
    }
    double* d_ph = nullptr;
    if (!dalloc(&d_ph, ph.size())) {
        err = "periodic mobility: device allocation failed";
        return AM_ERR_CUDA;
    }
    cudaMemcpyAsync(d_ph, ph.data(), ph.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    k_per_kfac<T><<<(int)((w.nhat + 255) / 256), 256, 0, s>>>(w.M[0], w.M[1], w.M[2], p->L[0], p->L[1], p->L[2],
                                                              a, eta, p->xi, w.kcut, d_ph + ph_off[0],
                                                              d_ph + ph_off[1], d_ph + ph_off[2],
                                                              static_cast<C*>(w.kfac));
    count_launch();
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(d_ph);
    if (e != cudaSuccess) {
        err = "periodic mobility: setup kernels failed";
        return AM_ERR_CUDA;
    }
    return AM_OK;
}

CellGeom cell_geom(const PeriodicPlan* p) {
    CellGeom g;
    for (int d = 0; d < 3; ++d) {
        g.nc[d] = p->nc[d];
        g.L[d] = p->L[d];
    }
    return g;
}

}  // namespace

void periodic_free(am_handle* h) {
    free_plan(h->per);
    h->per = nullptr;
    h->per_nnz = 0;
}

// Parameters and buffers for the handle's box, tolerance and blob count
// (the FP64 wave part, and the FP32 one at tolerance max(ewald_tol, 1e-6)
// for mixed handles; both share xi and the real-space pairs).
int periodic_setup(am_handle* h) {
    const double a = h->cfg.blob_radius, eta = h->cfg.eta;
    const double tol = h->cfg.ewald_tol > 0.0 ? h->cfg.ewald_tol : 1e-10;
    const int Nb = h->Nb;
    if (h->per && h->per->Nb == Nb) {  // the same box, tolerance and blob count: keep the plan
        h->per->valid = false;         // (bin again at the next pose)
        return AM_OK;
    }
    periodic_free(h);
    if (Nb <= 0 || Nb >= (1 << 26)) {
        h->err = "periodic box: the blob count must be in 1 .. 2^26 - 1";
        return AM_ERR_ARG;
    }
    PeriodicPlan* p = new PeriodicPlan();
    h->per = p;
    p->Nb = Nb;
    p->tol = tol;
    for (int d = 0; d < 3; ++d) p->L[d] = h->cfg.box[d];
    const double lg = std::log(1.0 / tol), crc = std::sqrt(0.8 * lg);
    const int P = window_width(tol);
    const double Lmin = std::min(p->L[0], std::min(p->L[1], p->L[2]));
    if (!(Lmin / 3.0 > 2.0 * a * 1.01)) {
        h->err = "periodic box: every side must exceed 6 blob radii";
        return AM_ERR_ARG;
    }
    const double xi_lo = crc / (Lmin / 3.0 - 2.0 * a);
    const double V = p->L[0] * p->L[1] * p->L[2], dens = Nb / V;
    double xi = h->cfg.ewald_xi;
    if (xi > 0.0) {
        if (xi < xi_lo) {
            h->err = "periodic box: ewald_xi too small for the box (r_c would exceed a third of a side)";
            return AM_ERR_ARG;
        }
    } else {
        // time per product, measured on GB300: about 20 ps per real-space
        // pair (its 52 bytes read, plus its share of the per-pose block
        // build over a solve) against 700 ps per grid point (the three
        // FP64 transforms each way, bound by the FP64 rate); the spreading
        // and interpolation do not depend on xi
        // memory: the real-space pairs (60 bytes each with the listing
        // codes; estimated from the mean density, so with a margin of two
        // for clustered blobs) within a quarter of the free device memory
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)16 << 30;
        const double pair_budget = 0.25 * (double)free_b / (2.0 * 60.0);
        double best = 1e300;
        for (int t = 0; t < 96; ++t) {
            const double x = xi_lo * std::pow(2.0, t / 8.0);
            int M[3];
            const long long tot = wave_grid(p, x, tol, P, M);
            if (tot > (1LL << 31)) break;
            const double rc = 2.0 * a + crc / x;
            const double pairs = (double)Nb * (1.0 + dens * 4.0 / 3.0 * kPi * rc * rc * rc);
            if (pairs > pair_budget) continue;
            const double cost = 20.0 * pairs + 700.0 * (double)tot;
            if (cost < best) {
                best = cost;
                xi = x;
            }
        }
        if (!(xi > 0.0)) {
            h->err = "periodic box: no grid fits (box too large for the blob radius and tolerance)";
            return AM_ERR_ARG;
        }
    }
    p->xi = xi;
    p->rc = 2.0 * a + crc / xi;
    for (int d = 0; d < 3; ++d) p->nc[d] = std::max(3, (int)std::floor(p->L[d] / p->rc));
    p->ncell = p->nc[0] * p->nc[1] * p->nc[2];
    p->ntab = kTab;
    p->ds = p->rc * p->rc * 1.001 / (kTab - 3);

    const int nscan = (std::max(Nb, p->ncell) + kScanBlock - 1) / kScanBlock + 1;
    bool ok = dalloc(&p->d_tab, p->ntab) && dalloc(&p->d_cell_start, p->ncell + 1) &&
              dalloc(&p->d_cell_fill, p->ncell) && dalloc(&p->d_cell_of, Nb) && dalloc(&p->d_order, Nb) &&
              dalloc(&p->d_spos, Nb) && dalloc(&p->d_sposf, Nb) && dalloc(&p->d_row, Nb + 1) &&
              dalloc(&p->d_scan, nscan) && dalloc(&p->d_rprev, Nb) && dalloc(&p->d_moved, 1);
    if (!ok) {
        cudaGetLastError();
        h->err = "periodic mobility: device allocation failed";
        return AM_ERR_CUDA;
    }
    cudaStream_t s = h->stream;
    double gx[20], gw[20];
    gauss_legendre20(gx, gw);
    int rc = wave_setup<double>(p, p->w64, tol, a, eta, s, gx, gw, h->err);
    if (rc) return rc;
    if (h->cfg.precision == AM_MIXED) {
        rc = wave_setup<float>(p, p->w32, std::max(tol, 1e-6), a, eta, s, gx, gw, h->err);
        if (rc) return rc;
        p->has32 = true;
    }

    // quadrature of the wave part's radial integrals: 20-point panels, four
    // per oscillation period of the integrand, up to k = 2 xi sqrt(50)
    const double kmax = 2.0 * xi * std::sqrt(50.0);
    const double span = std::max(p->rc * 1.001, 2.0 * a);
    const int panels = std::max(64, (int)std::ceil(4.0 * kmax * span / (2.0 * kPi)));
    std::vector<double> kq, wq;
    kq.reserve(20 * panels);
    wq.reserve(20 * panels);
    for (int pn = 0; pn < panels; ++pn) {
        const double k0 = kmax * pn / panels, k1 = kmax * (pn + 1) / panels;
        const double mid = 0.5 * (k0 + k1), half = 0.5 * (k1 - k0);
        for (int i = 0; i < 20; ++i) {
            const double k = mid + half * gx[i];
            const double x = k * k / (4.0 * xi * xi);
            const double ka = k * a;
            const double sinc = ka < 1e-4 ? 1.0 - ka * ka / 6.0 : std::sin(ka) / ka;
            kq.push_back(k);
            wq.push_back(half * gw[i] * (1.0 + x) * std::exp(-x) * sinc * sinc / (2.0 * kPi * kPi));
        }
    }
    double *d_kq = nullptr, *d_wq = nullptr;
    if (!dalloc(&d_kq, kq.size()) || !dalloc(&d_wq, wq.size())) {
        if (d_kq) cudaFree(d_kq);
        h->err = "periodic mobility: device allocation failed";
        return AM_ERR_CUDA;
    }
    cudaMemcpyAsync(d_kq, kq.data(), kq.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_wq, wq.data(), wq.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    k_per_table<<<(p->ntab * 32 + 255) / 256, 256, 0, s>>>(p->ntab, p->ds, d_kq, d_wq, (int)kq.size(), p->d_tab);
    count_launch();
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(d_kq);
    cudaFree(d_wq);
    if (e != cudaSuccess) {
        h->err = "periodic mobility: setup kernels failed";
        return AM_ERR_CUDA;
    }
    return AM_OK;
}

// Cell list and real-space pair blocks at the current blob positions
// (h->d_r4); called with every pose (launch_geometry).
int periodic_bin(am_handle* h) {
    PeriodicPlan* p = h->per;
    if (!p) return AM_ERR_ARG;
    cudaStream_t s = h->stream;
    const int Nb = p->Nb;
    const int nbk = (Nb + 255) / 256;
    if (p->valid) {  // the same positions as at the last binning: nothing to redo
        int moved = 1;
        cudaMemsetAsync(p->d_moved, 0, sizeof(int), s);
        k_per_moved<<<nbk, 256, 0, s>>>(Nb, h->d_r4, p->d_rprev, p->d_moved);
        count_launch();
        cudaMemcpyAsync(&moved, p->d_moved, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            h->err = "periodic mobility: position check failed";
            p->valid = false;
            return AM_ERR_CUDA;
        }
        if (!moved) return AM_OK;
    }
    p->valid = false;
    cudaMemsetAsync(p->d_cell_fill, 0, p->ncell * sizeof(int), s);
    k_per_cell<<<nbk, 256, 0, s>>>(Nb, h->d_r4, p->L[0], p->L[1], p->L[2], p->nc[0], p->nc[1], p->nc[2],
                                   p->d_cell_of, p->d_cell_fill);
    count_launch();
    exclusive_scan<int, int>(p->d_cell_fill, p->ncell, p->d_cell_start, p->d_scan, s);
    cudaMemsetAsync(p->d_cell_fill, 0, p->ncell * sizeof(int), s);
    k_per_fill<<<nbk, 256, 0, s>>>(Nb, p->d_cell_of, p->d_cell_start, p->d_cell_fill, p->d_order);
    k_per_gather_pos<<<nbk, 256, 0, s>>>(Nb, p->d_order, h->d_r4, p->L[0], p->L[1], p->L[2], p->d_spos,
                                         p->d_sposf);
    count_launch(2);
    const CellGeom cg = cell_geom(p);
    const RpyK<double> k = rpy_consts<double>(h->prm);
    const float rc2f = (float)(p->rc * p->rc);
    // count, scan, list, then the FP64 blocks
    k_per_pairs<false><<<nbk, 256, 0, s>>>(Nb, cg, p->d_spos, p->d_sposf, p->d_cell_start, rc2f, p->d_row,
                                           nullptr, 0);
    count_launch();
    exclusive_scan<long long, long long>(p->d_row, Nb, p->d_row, p->d_scan, s);
    long long nnz = 0;
    cudaMemcpyAsync(&nnz, p->d_row + Nb, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        h->err = "periodic mobility: cell list failed";
        return AM_ERR_CUDA;
    }
    if (nnz > p->cap) {
        if (p->d_nbr) cudaFree(p->d_nbr);
        if (p->d_blk) cudaFree(p->d_blk);
        if (p->d_code) cudaFree(p->d_code);
        if (p->d_blk32) cudaFree(p->d_blk32);
        p->d_nbr = nullptr;
        p->d_blk = nullptr;
        p->d_code = nullptr;
        p->d_blk32 = nullptr;
        const long long cap = nnz + nnz / 4 + 1024;
        if (!dalloc(&p->d_nbr, cap) || !dalloc(&p->d_blk, 6 * (size_t)cap) || !dalloc(&p->d_code, cap) ||
            (p->has32 && !dalloc(&p->d_blk32, 6 * (size_t)cap))) {
            cudaGetLastError();
            p->cap = 0;
            h->err = "periodic mobility: device allocation of the real-space pairs failed";
            return AM_ERR_CUDA;
        }
        p->cap = cap;
    }
    k_per_pairs<true><<<nbk, 256, 0, s>>>(Nb, cg, p->d_spos, p->d_sposf, p->d_cell_start, rc2f, p->d_row,
                                          p->d_code, p->cap);
    const int nbw = (int)(((long long)Nb * 32 + 255) / 256);
    k_per_blocks<false><<<nbw, 256, 0, s>>>(Nb, cg, p->d_spos, p->d_order, p->d_row, p->d_code, p->d_nbr, p->d_blk,
                                            p->cap, p->d_tab, p->ntab, 1.0 / p->ds, k, 1.0 / h->cfg.eta);
    k_per_blocks<true><<<nbw, 256, 0, s>>>(Nb, cg, p->d_spos, p->d_order, p->d_row, p->d_code, p->d_nbr, p->d_blk,
                                           p->cap, p->d_tab, p->ntab, 1.0 / p->ds, k, 1.0 / h->cfg.eta);
    if (p->has32) {
        k_per_blk32<<<8 * num_sms(), 256, 0, s>>>(p->d_blk, p->d_blk32, p->cap, nnz);
        count_launch();
    }
    cudaMemcpyAsync(p->d_rprev, h->d_r4, Nb * sizeof(double4_32a), cudaMemcpyDeviceToDevice, s);
    count_launch(3);
    p->nnz = nnz;
    h->per_nnz = nnz;
    if (cudaGetLastError() != cudaSuccess) {
        h->err = "periodic mobility: pair kernels failed";
        return AM_ERR_CUDA;
    }
    p->valid = true;
    return AM_OK;
}

// u = M_per lam (3 Nb each, blob order) into h->d_mv, with the FP64 wave
// part and blocks, or (fp32, mixed handles) the FP32 ones.  Stream-ordered;
// no host synchronisation, so it can be captured into a graph.
template <class T>
void launch_wave(am_handle* h, const Wave& w, const T* blk, const double* lam) {
    PeriodicPlan* p = h->per;
    cudaStream_t s = h->stream;
    const SpreadGeom g = spread_geom(w);
    T* grid = static_cast<T*>(w.grid);
    k_per_zero<T><<<8 * num_sms(), 256, 0, s>>>(grid, 3 * w.ngrid);
    launch_window_any<T>(p->Nb, g, p, w, blk, lam, h->d_mv, true, s);
    if constexpr (sizeof(T) == 8)
        cufftExecD2Z(w.fwd, static_cast<double*>(w.grid), static_cast<cufftDoubleComplex*>(w.hat));
    else
        cufftExecR2C(w.fwd, static_cast<float*>(w.grid), static_cast<cufftComplex*>(w.hat));
    k_per_kmul<T><<<(int)((w.nhat + 255) / 256), 256, 0, s>>>(w.M[0], w.M[1], w.M[2], p->L[0], p->L[1], p->L[2],
                                                              static_cast<const vec2_t<T>*>(w.kfac),
                                                              static_cast<vec2_t<T>*>(w.hat), w.nhat);
    if constexpr (sizeof(T) == 8)
        cufftExecZ2D(w.inv, static_cast<cufftDoubleComplex*>(w.hat), static_cast<double*>(w.grid));
    else
        cufftExecC2R(w.inv, static_cast<cufftComplex*>(w.hat), static_cast<float*>(w.grid));
    launch_window_any<T>(p->Nb, g, p, w, blk, lam, h->d_mv, false, s);
    count_launch(4);
}

void launch_periodic(am_handle* h, const double* lam, bool fp32) {
    PeriodicPlan* p = h->per;
    if (!p->valid) {  // binning failed (reported by the caller): no launch on stale pairs
        cudaMemsetAsync(h->d_mv, 0, 3 * (size_t)p->Nb * sizeof(double), h->stream);
        return;
    }
    if (fp32 && p->has32)
        launch_wave<float>(h, p->w32, p->d_blk32, lam);
    else
        launch_wave<double>(h, p->w64, p->d_blk, lam);
}

// xi, r_c, beta, hx, hy, hz; Mx, My, Mz, w, real-space pairs, cells
void periodic_info(const am_handle* h, double* d6, long long* i6) {
    const PeriodicPlan* p = h->per;
    if (d6) {
        d6[0] = p->xi; d6[1] = p->rc; d6[2] = p->w64.beta;
        d6[3] = p->w64.h[0]; d6[4] = p->w64.h[1]; d6[5] = p->w64.h[2];
    }
    if (i6) {
        i6[0] = p->w64.M[0]; i6[1] = p->w64.M[1]; i6[2] = p->w64.M[2];
        i6[3] = p->w64.P; i6[4] = p->nnz; i6[5] = p->ncell;
    }
}

}  // namespace am

// All-pairs blob mobility product u = M lambda (Sec. 2.3, Eq. RPY).
//
// Free space, equal radii a, d = r_i - r_j, r = |d|, A1 = 1/(8 pi eta),
// mu0 = 1/(6 pi eta a):
//   r >= 2a:  M = A1/r [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) dhat dhat]
//   r <  2a:  M = mu0 [(1 - 9r/(32a)) I + (3r/(32a)) dhat dhat],  M_ii = mu0 I.
// No-slip wall at z = 0: add the image part, the double surface average of
// the image terms of Blake's Green's function.  Written in the basis
// {delta_ij, Rh_i Rh_j, Rh_i e3_j, e3_i Rh_j, e3_i e3_j} with R = x - y*,
// y* = (y1, y2, -y3), s = 1/|R|, Rh = R s, h = y3 (source height),
// x3 = target height, ez = R3 s, A = a^2 s^2:
//   M_img = A1 s [ cI delta + cRR Rh Rh + cRz Rh e3 + czR e3 Rh + czz e3 e3 ]
//   cI  = -1 - 2 h x3 s^2 + A (2 ez^2 - 2/3) + A^2 (2/3 - 10/3 ez^2)
//   cRR = -1 + 6 h x3 s^2 + A (2 - 10 ez^2) + A^2 (70/3 ez^2 - 10/3)
//   cRz = 2 h s + ez [ -12 h x3 s^2 + A (20 ez^2 - 4) + A^2 (40/3 - 140/3 ez^2) ]
//   czR = 2 h s - 20/3 A^2 ez
//   czz = -4 h^2 s^2 + A (-4 ez^2) + A^2 (20 ez^2 - 8/3)
// (derived from Blake's image system by applying (1 + a^2/6 lap_x)
// (1 + a^2/6 lap_y), which is exact for blobs whose centres are above a).
//
// Layout: one thread per target blob, 128 targets per block; sources are
// staged through shared memory 128 at a time; the sources are split into
// `splits` contiguous chunks (grid.y) so that small systems still fill the
// 152 SMs; each (target block, chunk) writes its partial sums, and a second
// kernel adds the chunks.
#include "am_internal.cuh"
#include "rpy_pair.cuh"
#include "ops.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

namespace am {

std::atomic<long long> g_launches{0};

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    return sms;
}

RpyParams make_params(double eta, double a) {
    RpyParams p;
    p.a = a;
    p.a2 = a * a;
    p.four_a2 = 4.0 * a * a;
    p.inv8pieta = 1.0 / (8.0 * kPi * eta);
    p.k_far2 = p.inv8pieta * 2.0 * a * a / 3.0;
    p.k_far3 = p.inv8pieta * 2.0 * a * a;
    p.mu0 = 1.0 / (6.0 * kPi * eta * a);
    p.k_near1 = 9.0 / (32.0 * a);
    p.k_near2 = p.mu0 * 3.0 / (32.0 * a);
    return p;
}

Split choose_split(int n, int precision) { return choose_split_rows(n, n, precision); }

// n sources, nt targets
Split choose_split_rows(int n, int nt, int precision) {
    Split s{1, std::max(n, 1), 1};
    if (n <= 0 || nt <= 0) return s;
    const int want = 4 * num_sms();  // blocks to fill the GPU
    // two targets per thread once one source chunk already fills the GPU
    if (precision == AM_MIXED && (nt + 2 * kThreads - 1) / (2 * kThreads) >= want) s.tpt = 2;
    const int tiles = (n + kTile - 1) / kTile;
    const int tblocks = (nt + kThreads * s.tpt - 1) / (kThreads * s.tpt);
    const int splits = std::max(1, std::min(tiles, (want + tblocks - 1) / tblocks));
    const int per = (tiles + splits - 1) / splits;  // tiles per chunk
    s.chunk = per * kTile;
    s.splits = (n + s.chunk - 1) / s.chunk;
    return s;
}

template <bool WALL>
__global__ void __launch_bounds__(kThreads)
rpy_partial_f64(const double4_32a* __restrict__ r4, const double* __restrict__ lam,
                double* __restrict__ part, int n, int chunk, RpyK<double> k, int t0, int nt) {
    __shared__ double4_32a sr[kTile];
    __shared__ double sl[3 * kTile];
    // targets t0 .. t0 + nt - 1 against sources 0 .. n - 1
    const int it = blockIdx.x * kThreads + threadIdx.x;
    const int i = t0 + it;
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(n, j0 + chunk);
    double4_32a ri = (it < nt) ? r4[i] : make_double4_32a(0.0, 0.0, 1.0, 0.0);
    const double nx3 = -ri.z;
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int jt = j0; jt < j1; jt += kTile) {
        const int cnt = min(kTile, j1 - jt);
        __syncthreads();
        if (threadIdx.x < cnt) {
            double4_32a v = r4[jt + threadIdx.x];
            v.w = 2.0 * v.z;  // twice the source height, for the wall term
            sr[threadIdx.x] = v;
        }
        for (int q = threadIdx.x; q < 3 * cnt; q += kThreads) sl[q] = lam[3 * (size_t)jt + q];
        __syncthreads();
#pragma unroll 2
        for (int q = 0; q < cnt; ++q) {
            const double4_32a rj = sr[q];
            const double lx = sl[3 * q], ly = sl[3 * q + 1], lz = sl[3 * q + 2];
            const double dx = ri.x - rj.x, dy = ri.y - rj.y, dz = ri.z - rj.z;
            if (WALL) {
                const double rxy2 = fma(dx, dx, dy * dy);
                pair_wall_r2<double>(dx, dy, dz, rxy2, fma(dz, dz, rxy2), ri.z + rj.z, rj.w, nx3, lx, ly, lz, k,
                                     ux, uy, uz);
            } else {
                pair_free<double>(dx, dy, dz, lx, ly, lz, k, ux, uy, uz);
            }
        }
    }
    if (it < nt) {
        double* o = part + (size_t)blockIdx.y * 3 * nt + 3 * (size_t)it;
        o[0] = k.A1 * ux; o[1] = k.A1 * uy; o[2] = k.A1 * uz;
    }
}

// sources per FP32 partial sum of the mixed kernels before it is added to
// the tile's compensated (hi, lo) sums
constexpr int kSumBlock = 16;

// hi + lo += t with Knuth's TwoSum (rounding error of hi + t kept in lo):
// the compensated accumulation of the tile sums of the mixed kernels
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float t) {
    const float s = __fadd_rn(hi, t);
    const float v = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(t, v)));
    hi = s;
}

// Positions as hi + lo float pairs (hi = float(x), lo = float(x - hi)).  A
// pair's difference is first formed from hi alone; within a radius of a
// quarter of the target's largest coordinate, where the rounding of hi
// (1.2e-7 |x|) would exceed 5e-7 of the distance, the lo parts are added,
// which keeps FP32 relative accuracy of nearby differences anywhere in the
// domain.  Pair terms and the sum over one tile are FP32; tile sums are
// folded into FP64.  TPT targets per thread share each shared-memory load.
template <bool WALL, int TPT>
__global__ void __launch_bounds__(kThreads, 4)
rpy_partial_mixed(const float4* __restrict__ hi, const float4* __restrict__ lo,
                  const double* __restrict__ lam, double* __restrict__ part, int n,
                  int chunk, RpyK<float> k, int t0, int nt) {
    __shared__ float4 sh[kTile];
    __shared__ float4 so[kTile];
    __shared__ float4 sl[kTile];
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(n, j0 + chunk);
    float4 hi_i[TPT], lo_i[TPT];
    float near2[TPT];
    double U[TPT][3];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int it = (blockIdx.x * TPT + t) * kThreads + threadIdx.x;
        const int i = t0 + it;
        hi_i[t] = (it < nt) ? hi[i] : make_float4(0.f, 0.f, 1.f, 0.f);
        lo_i[t] = (it < nt) ? lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float nr = 0.25f * fmaxf(fabsf(hi_i[t].x), fmaxf(fabsf(hi_i[t].y), fabsf(hi_i[t].z)));
        near2[t] = nr * nr;
        U[t][0] = U[t][1] = U[t][2] = 0.0;
    }
    for (int jt = j0; jt < j1; jt += kTile) {
        const int cnt = min(kTile, j1 - jt);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int j = jt + threadIdx.x;
            const float4 hj = hi[j];
            sh[threadIdx.x] = make_float4(hj.x, hj.y, hj.z, 2.f * hj.z);  // .w: twice the height
            so[threadIdx.x] = lo[j];
            sl[threadIdx.x] = make_float4((float)lam[3 * (size_t)j], (float)lam[3 * (size_t)j + 1],
                                          (float)lam[3 * (size_t)j + 2], 0.f);
        }
        __syncthreads();
        // pair terms summed in FP32 over blocks of kSumBlock sources, each block
        // added to the tile's (hi, lo) sums by TwoSum, the tile folded into FP64
        float th[TPT][3], tl[TPT][3];
#pragma unroll
        for (int t = 0; t < TPT; ++t)
            for (int c = 0; c < 3; ++c) th[t][c] = tl[t][c] = 0.f;
        for (int q0 = 0; q0 < cnt; q0 += kSumBlock) {
        const int qe = min(cnt, q0 + kSumBlock);
        float u[TPT][3];
#pragma unroll
        for (int t = 0; t < TPT; ++t) u[t][0] = u[t][1] = u[t][2] = 0.f;
#pragma unroll 2
        for (int q = q0; q < qe; ++q) {
            const float4 h = sh[q];
            const float4 l = sl[q];
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                float dx = hi_i[t].x - h.x, dy = hi_i[t].y - h.y, dz = hi_i[t].z - h.z;
                float rxy2 = fmaf(dx, dx, dy * dy);
                float r2 = fmaf(dz, dz, rxy2);
                if (r2 < near2[t]) {
                    const float4 o = so[q];
                    dx += lo_i[t].x - o.x;
                    dy += lo_i[t].y - o.y;
                    dz += lo_i[t].z - o.z;
                    rxy2 = fmaf(dx, dx, dy * dy);
                    r2 = fmaf(dz, dz, rxy2);
                }
                if (WALL)
                    pair_wall_r2<float>(dx, dy, dz, rxy2, r2, hi_i[t].z + h.z, h.w, -hi_i[t].z, l.x, l.y, l.z, k,
                                        u[t][0], u[t][1], u[t][2]);
                else
                    pair_free_r2<float>(dx, dy, dz, r2, l.x, l.y, l.z, k, u[t][0], u[t][1], u[t][2]);
            }
        }
#pragma unroll
        for (int t = 0; t < TPT; ++t)
            for (int c = 0; c < 3; ++c) two_sum_acc(th[t][c], tl[t][c], u[t][c]);
        }
#pragma unroll
        for (int t = 0; t < TPT; ++t)
            for (int c = 0; c < 3; ++c) U[t][c] += (double)th[t][c] + (double)tl[t][c];
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int it = (blockIdx.x * TPT + t) * kThreads + threadIdx.x;
        if (it < nt) {
            double* o = part + (size_t)blockIdx.y * 3 * nt + 3 * (size_t)it;
            o[0] = k.A1 * U[t][0]; o[1] = k.A1 * U[t][1]; o[2] = k.A1 * U[t][2];
        }
    }
}

__global__ void pack_positions(const double* __restrict__ r3, double4_32a* __restrict__ r4,
                               float4* __restrict__ hi, float4* __restrict__ lo, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = r3[3 * (size_t)i], y = r3[3 * (size_t)i + 1], z = r3[3 * (size_t)i + 2];
    if (r4) r4[i] = make_double4_32a(x, y, z, 0.0);
    if (hi) {
        float hx = (float)x, hy = (float)y, hz = (float)z;
        hi[i] = make_float4(hx, hy, hz, 0.f);
        lo[i] = make_float4((float)(x - hx), (float)(y - hy), (float)(z - hz), 0.f);
    }
}

__global__ void sum_partials(const double* __restrict__ part, double* __restrict__ u,
                             int n3, int splits) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n3) return;
    double s = 0.0;
    for (int t = 0; t < splits; ++t) s += part[(size_t)t * n3 + k];
    u[k] = s;
}


// Targets t0 .. t0 + nt - 1 against all n sources; partial sums of split c
// at part[c * 3 nt + 3 (i - t0)].
void launch_rpy_partial_f64_rows(const double4_32a* r4, const double* lam, double* part, int n, int t0, int nt,
                                 const Split& sp, const RpyParams& prm, int wall, cudaStream_t st) {
    if (n <= 0 || nt <= 0) return;
    dim3 grid((nt + kThreads - 1) / kThreads, sp.splits);
    const RpyK<double> k = rpy_consts<double>(prm);
    if (wall)
        rpy_partial_f64<true><<<grid, kThreads, 0, st>>>(r4, lam, part, n, sp.chunk, k, t0, nt);
    else
        rpy_partial_f64<false><<<grid, kThreads, 0, st>>>(r4, lam, part, n, sp.chunk, k, t0, nt);
    count_launch();
}

void launch_rpy_partial_mixed_rows(const float4* hi, const float4* lo, const double* lam, double* part, int n,
                                   int t0, int nt, const Split& sp, const RpyParams& prm, int wall,
                                   cudaStream_t st) {
    if (n <= 0 || nt <= 0) return;
    const RpyK<float> k = rpy_consts<float>(prm);
    const int per = kThreads * sp.tpt;
    dim3 grid((nt + per - 1) / per, sp.splits);
    if (sp.tpt == 2) {
        if (wall)
            rpy_partial_mixed<true, 2><<<grid, kThreads, 0, st>>>(hi, lo, lam, part, n, sp.chunk, k, t0, nt);
        else
            rpy_partial_mixed<false, 2><<<grid, kThreads, 0, st>>>(hi, lo, lam, part, n, sp.chunk, k, t0, nt);
    } else {
        if (wall)
            rpy_partial_mixed<true, 1><<<grid, kThreads, 0, st>>>(hi, lo, lam, part, n, sp.chunk, k, t0, nt);
        else
            rpy_partial_mixed<false, 1><<<grid, kThreads, 0, st>>>(hi, lo, lam, part, n, sp.chunk, k, t0, nt);
    }
    count_launch();
}

void launch_rpy_partial_f64(const double4_32a* r4, const double* lam, double* part, int n,
                            const Split& sp, const RpyParams& prm, int wall, cudaStream_t st) {
    launch_rpy_partial_f64_rows(r4, lam, part, n, 0, n, sp, prm, wall, st);
}

void launch_rpy_partial_mixed(const float4* hi, const float4* lo, const double* lam, double* part,
                              int n, const Split& sp, const RpyParams& prm, int wall,
                              cudaStream_t st) {
    launch_rpy_partial_mixed_rows(hi, lo, lam, part, n, 0, n, sp, prm, wall, st);
}

void launch_pack_positions(const double* r3, double4_32a* r4, float4* hi, float4* lo, int n,
                           cudaStream_t st) {
    if (n <= 0) return;
    pack_positions<<<(n + 255) / 256, 256, 0, st>>>(r3, r4, hi, lo, n);
    count_launch();
}

void launch_sum_partials(const double* part, double* u, int n, int splits, cudaStream_t st) {
    if (n <= 0) return;
    int n3 = 3 * n;
    sum_partials<<<(n3 + 255) / 256, 256, 0, st>>>(part, u, n3, splits);
    count_launch();
}

}  // namespace am

// ------------------------------------------------------------ C ABI -------
namespace {
thread_local std::string t_err = "";
int fail(int code, const char* msg) {
    t_err = msg;
    return code;
}
size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

namespace am {
const char* thread_error() { return t_err.c_str(); }
void set_thread_error(const std::string& msg) { t_err = msg; }
}

extern "C" AM_API size_t am_rpy_matvec_workspace(int n, int precision) {
    if (n <= 0) return 0;
    am::Split sp = am::choose_split(n, precision);
    size_t pos = (precision == AM_MIXED) ? 2 * align256((size_t)n * sizeof(float4))
                                         : align256((size_t)n * sizeof(double4_32a));
    return pos + align256((size_t)sp.splits * 3 * n * sizeof(double));
}

extern "C" AM_API int am_rpy_matvec(const double* d_r, const double* d_lambda, double* d_u, int n,
                                    double eta, double a, int wall, int precision, void* d_work,
                                    size_t work_bytes, void* stream) {
    if (n < 0) return fail(AM_ERR_ARG, "am_rpy_matvec: n < 0");
    if (!(eta > 0.0) || !(a > 0.0)) return fail(AM_ERR_ARG, "am_rpy_matvec: eta and a must be > 0");
    if (wall != 0 && wall != 1) return fail(AM_ERR_ARG, "am_rpy_matvec: wall must be 0 or 1");
    if (precision != AM_FP64 && precision != AM_MIXED)
        return fail(AM_ERR_ARG, "am_rpy_matvec: unknown precision");
    if (n == 0) return AM_OK;
    if (!d_r || !d_lambda || !d_u || !d_work) return fail(AM_ERR_ARG, "am_rpy_matvec: NULL pointer");
    if (work_bytes < am_rpy_matvec_workspace(n, precision))
        return fail(AM_ERR_ARG, "am_rpy_matvec: workspace too small");
    if (reinterpret_cast<uintptr_t>(d_work) % 256 != 0)
        return fail(AM_ERR_ARG, "am_rpy_matvec: workspace not 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    am::Split sp = am::choose_split(n, precision);
    am::RpyParams prm = am::make_params(eta, a);
    char* w = static_cast<char*>(d_work);
    if (precision == AM_MIXED) {
        float4* hi = reinterpret_cast<float4*>(w);
        float4* lo = reinterpret_cast<float4*>(w + align256((size_t)n * sizeof(float4)));
        double* part = reinterpret_cast<double*>(w + 2 * align256((size_t)n * sizeof(float4)));
        am::launch_pack_positions(d_r, nullptr, hi, lo, n, st);
        am::launch_rpy_partial_mixed(hi, lo, d_lambda, part, n, sp, prm, wall, st);
        am::launch_sum_partials(part, d_u, n, sp.splits, st);
    } else {
        double4_32a* r4 = reinterpret_cast<double4_32a*>(w);
        double* part = reinterpret_cast<double*>(w + align256((size_t)n * sizeof(double4_32a)));
        am::launch_pack_positions(d_r, r4, nullptr, nullptr, n, st);
        am::launch_rpy_partial_f64(r4, d_lambda, part, n, sp, prm, wall, st);
        am::launch_sum_partials(part, d_u, n, sp.splits, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AM_ERR_CUDA, cudaGetErrorString(e));
    return AM_OK;
}

extern "C" AM_API size_t am_rpy_matvec_rows_workspace(int n, int nrows, int precision) {
    if (n <= 0 || nrows <= 0) return 0;
    am::Split sp = am::choose_split_rows(n, nrows, precision);
    size_t pos = (precision == AM_MIXED) ? 2 * align256((size_t)n * sizeof(float4))
                                         : align256((size_t)n * sizeof(double4_32a));
    return pos + align256((size_t)sp.splits * 3 * nrows * sizeof(double));
}

extern "C" AM_API int am_rpy_matvec_rows(const double* d_r, const double* d_lambda, double* d_u, int n, int row0,
                                         int nrows, double eta, double a, int wall, int precision, void* d_work,
                                         size_t work_bytes, void* stream) {
    if (n < 0 || nrows < 0 || row0 < 0 || (long long)row0 + nrows > n)
        return fail(AM_ERR_ARG, "am_rpy_matvec_rows: need 0 <= row0, 0 <= nrows, row0 + nrows <= n");
    if (!(eta > 0.0) || !(a > 0.0)) return fail(AM_ERR_ARG, "am_rpy_matvec_rows: eta and a must be > 0");
    if (wall != 0 && wall != 1) return fail(AM_ERR_ARG, "am_rpy_matvec_rows: wall must be 0 or 1");
    if (precision != AM_FP64 && precision != AM_MIXED)
        return fail(AM_ERR_ARG, "am_rpy_matvec_rows: unknown precision");
    if (n == 0 || nrows == 0) return AM_OK;
    if (!d_r || !d_lambda || !d_u || !d_work) return fail(AM_ERR_ARG, "am_rpy_matvec_rows: NULL pointer");
    if (work_bytes < am_rpy_matvec_rows_workspace(n, nrows, precision))
        return fail(AM_ERR_ARG, "am_rpy_matvec_rows: workspace too small");
    if (reinterpret_cast<uintptr_t>(d_work) % 256 != 0)
        return fail(AM_ERR_ARG, "am_rpy_matvec_rows: workspace not 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    am::Split sp = am::choose_split_rows(n, nrows, precision);
    am::RpyParams prm = am::make_params(eta, a);
    char* w = static_cast<char*>(d_work);
    if (precision == AM_MIXED) {
        float4* hi = reinterpret_cast<float4*>(w);
        float4* lo = reinterpret_cast<float4*>(w + align256((size_t)n * sizeof(float4)));
        double* part = reinterpret_cast<double*>(w + 2 * align256((size_t)n * sizeof(float4)));
        am::launch_pack_positions(d_r, nullptr, hi, lo, n, st);
        am::launch_rpy_partial_mixed_rows(hi, lo, d_lambda, part, n, row0, nrows, sp, prm, wall, st);
        am::launch_sum_partials(part, d_u, nrows, sp.splits, st);
    } else {
        double4_32a* r4 = reinterpret_cast<double4_32a*>(w);
        double* part = reinterpret_cast<double*>(w + align256((size_t)n * sizeof(double4_32a)));
        am::launch_pack_positions(d_r, r4, nullptr, nullptr, n, st);
        am::launch_rpy_partial_f64_rows(r4, d_lambda, part, n, row0, nrows, sp, prm, wall, st);
        am::launch_sum_partials(part, d_u, nrows, sp.splits, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AM_ERR_CUDA, cudaGetErrorString(e));
    return AM_OK;
}

extern "C" AM_API int am_flops_per_pair(int wall) {
    // Counted from pair_free_* and pair_image_* with FMA = 2 (rsqrt = 1):
    // free (pair_free): difference 3, r^2 5, rsqrt 1, ri^2 1, c1 3, c2 4,
    //       d.lambda 5, scale 1, accumulate 12  -> 35
    // image (pair_image): R3 1, R^2 5, rsqrt 1, s^2 1, hs 1, u 2, ez 1,
    //       ez^2 1, A 1, A^2 1, t1 1, t2 1, cI 10, cRR 10, inner 4, cRz 3,
    //       czR 3, czz 8, Rh 2, Rh.lambda 5, t 3, accumulate 19  -> 84
    // (the factor 1/(8 pi eta) is applied once per target and tile)
    return wall ? 35 + 84 : 35;
}

extern "C" AM_API long long am_kernel_launches(void) { return am::g_launches.load(); }

// ======================================================================
// Block-diagonal product over the systems of a handle (batched form).
// Work items (system, block of targets, chunk of sources) are pulled from an
// atomic queue by a persistent grid sized to the resident blocks of all SMs;
// items are ordered largest first.  The partial sums of system s, chunk c,
// blob i go to part[poff_s + c * 3 N_s + 3 (i - blob0_s)].
namespace am {

// An item of a stopped system (active[sys] == 0; the system's input is
// zero) writes zero partial sums instead of evaluating its pairs.
__device__ __forceinline__ bool item_skipped(const MvItem& m, const int* __restrict__ active,
                                             double* __restrict__ part) {
    if (!active || active[m.sys]) return false;
    for (int i = m.t0 + threadIdx.x; i < m.t1; i += blockDim.x) {
        double* o = part + m.pbase + 3 * (size_t)(i - m.tbase);
        o[0] = 0.0; o[1] = 0.0; o[2] = 0.0;
    }
    return true;
}

template <bool WALL>
__global__ void __launch_bounds__(kThreads)
rpy_items_f64(const double4_32a* __restrict__ r4, const double* __restrict__ lam,
              double* __restrict__ part, const MvItem* __restrict__ items, int n_items,
              int* __restrict__ counter, RpyK<double> k, const int* __restrict__ active) {
    dep_wait();
    __shared__ double4_32a sr[kTile];
    __shared__ double sl[3 * kTile];
    __shared__ int s_item;
    for (int round = 0;; ++round) {
        // first item = the block's own index (spread over the SMs as the
        // blocks are), later ones from the queue
        __syncthreads();
        if (threadIdx.x == 0) s_item = round == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(counter, 1);
        __syncthreads();
        const int itn = s_item;
        if (itn >= n_items) break;
        const MvItem m = items[itn];
        if (item_skipped(m, active, part)) continue;
        // items built for two targets per thread span 2 x 128 targets
        for (int tb = m.t0; tb < m.t1; tb += kThreads) {
        const int i = tb + threadIdx.x;
        double4_32a ri = (i < m.t1) ? r4[i] : make_double4_32a(0.0, 0.0, 1.0, 0.0);
        const double nx3 = -ri.z;
        // warps with no target of the item (items of fewer targets than
        // the block) only help stage the sources
        const bool warp_live = tb + (int)(threadIdx.x & ~31u) < m.t1;
        double ux = 0.0, uy = 0.0, uz = 0.0;
        for (int jt = m.j0; jt < m.j1; jt += kTile) {
            const int cnt = min(kTile, m.j1 - jt);
            __syncthreads();
            if (threadIdx.x < cnt) {
                double4_32a v = r4[jt + threadIdx.x];
                v.w = 2.0 * v.z;  // twice the source height, for the wall term
                sr[threadIdx.x] = v;
            }
            for (int q = threadIdx.x; q < 3 * cnt; q += kThreads) sl[q] = lam[3 * (size_t)jt + q];
            __syncthreads();
            if (!warp_live) continue;
#pragma unroll 2
            for (int q = 0; q < cnt; ++q) {
                const double4_32a rj = sr[q];
                const double lx = sl[3 * q], ly = sl[3 * q + 1], lz = sl[3 * q + 2];
                const double dx = ri.x - rj.x, dy = ri.y - rj.y, dz = ri.z - rj.z;
                if (WALL) {
                    const double rxy2 = fma(dx, dx, dy * dy);
                    pair_wall_r2<double>(dx, dy, dz, rxy2, fma(dz, dz, rxy2), ri.z + rj.z, rj.w, nx3, lx, ly,
                                         lz, k, ux, uy, uz);
                } else {
                    pair_free<double>(dx, dy, dz, lx, ly, lz, k, ux, uy, uz);
                }
            }
        }
        if (i < m.t1) {
            double* o = part + m.pbase + 3 * (size_t)(i - m.tbase);
            o[0] = k.A1 * ux; o[1] = k.A1 * uy; o[2] = k.A1 * uz;
        }
        }
    }
    item_queue_done(counter);
}

// Symmetric FP64 product (the mobility is symmetric: M_ji = M_ij^T).  Per
// item the block stages both tiles; its warps take the item's NSUB x NSUB
// warp tiles (32 targets x 32 sources) in turn.  In a warp tile lane l
// holds target l and, at step t, meets source (l + t) mod 32: u_l gathers
// M lambda_source, and the source's column sum v (M^T mu_l) is carried
// from lane to lane (lane l hands it to lane l - 1), so after 32 steps it
// is back on the source's lane with the sum over the 32 targets.  On the
// diagonal of a diagonal item the steps 1..15, and 16 on lanes 0..15, take
// every unordered pair once (step 0: the self term).  Warp-tile sums go to
// shared memory and are added in a fixed order: the result does not
// depend on scheduling.
template <bool WALL, int NSUB>
__global__ void __launch_bounds__(NSUB == 1 ? 32 : 128)
rpy_sym_f64(const double4_32a* __restrict__ r4, const double* __restrict__ lam, double* __restrict__ part,
            const SymItem* __restrict__ items, int n_items, int* __restrict__ counter, RpyK<double> k,
            const int* __restrict__ active) {
    dep_wait();
    constexpr int T = 32 * NSUB;
    constexpr int NW = NSUB == 1 ? 1 : 4;
    constexpr int NWT = NSUB * NSUB;
    __shared__ double4_32a sI[T], sJ[T];
    __shared__ double lI[3 * T], lJ[3 * T];
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
        double* rowo = part + m.poff + (long long)m.tj * m.n3 + 3 * (long long)(m.i0 - m.tbase);
        double* colo = part + m.poff + (long long)m.ti * m.n3 + 3 * (long long)(m.j0 - m.tbase);
        if (active && !active[m.sys]) {  // a stopped system: zero partial sums
            for (int q = threadIdx.x; q < 3 * m.ni; q += blockDim.x) rowo[q] = 0.0;
            if (!diag)
                for (int q = threadIdx.x; q < 3 * m.nj; q += blockDim.x) colo[q] = 0.0;
            continue;
        }
        for (int q = threadIdx.x; q < T; q += blockDim.x) {
            double4_32a a = q < m.ni ? r4[m.i0 + q] : make_double4_32a(0.0, 0.0, 1.0, 0.0);
            a.w = 2.0 * a.z;
            sI[q] = a;
            double4_32a b = q < m.nj ? r4[m.j0 + q] : make_double4_32a(0.0, 0.0, 1.0, 0.0);
            b.w = 2.0 * b.z;
            sJ[q] = b;
        }
        for (int q = threadIdx.x; q < 3 * T; q += blockDim.x) {
            lI[q] = q < 3 * m.ni ? lam[3 * (size_t)m.i0 + q] : 0.0;
            lJ[q] = q < 3 * m.nj ? lam[3 * (size_t)m.j0 + q] : 0.0;
        }
        __syncthreads();
        for (int wt = warp; wt < NWT; wt += NW) {
            const int a = wt / NSUB, b = wt % NSUB;
            double ux = 0.0, uy = 0.0, uz = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
            if (!(diag && b < a)) {  // below the diagonal of a diagonal item: taken by (b, a)
                const bool self_tile = diag && a == b;
                const int t = 32 * a + lane;
                const double4_32a xi = sI[t];
                const double mx = lI[3 * t], my = lI[3 * t + 1], mz = lI[3 * t + 2];
                const double nx3 = -xi.z;
                const bool ti_ok = t < m.ni;
#pragma unroll 1
                for (int step = 0; step < 32; ++step) {
                    const int q = 32 * b + ((lane + step) & 31);
                    const bool pair_ok = ti_ok && q < m.nj &&
                                         (!self_tile || (step >= 1 && (step < 16 || (step == 16 && lane < 16))));
                    if (pair_ok) {
                        const double4_32a xj = sJ[q];
                        const double lx = lJ[3 * q], ly = lJ[3 * q + 1], lz = lJ[3 * q + 2];
                        const double dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
                        if (WALL) {
                            const double rxy2 = fma(dx, dx, dy * dy);
                            pair_wall_sym<double>(dx, dy, dz, rxy2, fma(dz, dz, rxy2), xi.z + xj.z, xj.w, nx3, lx,
                                                  ly, lz, mx, my, mz, k, ux, uy, uz, vx, vy, vz);
                        } else {
                            pair_free_sym<double>(dx, dy, dz, fma(dx, dx, fma(dy, dy, dz * dz)), lx, ly, lz, mx,
                                                  my, mz, k, ux, uy, uz, vx, vy, vz);
                        }
                    } else if (self_tile && step == 0 && ti_ok) {  // the self term
                        if (WALL)
                            pair_wall_r2<double>(0.0, 0.0, 0.0, 0.0, 0.0, 2.0 * xi.z, xi.w, nx3, mx, my, mz, k, ux,
                                                 uy, uz);
                        else
                            pair_free<double>(0.0, 0.0, 0.0, mx, my, mz, k, ux, uy, uz);
                    }
                    // hand the column sum to the lane that meets this source next
                    const int src = (lane + 1) & 31;
                    vx = __shfl_sync(0xffffffffu, vx, src);
                    vy = __shfl_sync(0xffffffffu, vy, src);
                    vz = __shfl_sync(0xffffffffu, vz, src);
                }
            }
            up[wt][lane][0] = ux; up[wt][lane][1] = uy; up[wt][lane][2] = uz;
            vp[wt][lane][0] = vx; vp[wt][lane][1] = vy; vp[wt][lane][2] = vz;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            const int a = t >> 5, l = t & 31;
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

template <bool WALL, int TPT>
__global__ void __launch_bounds__(kThreads, 4)
rpy_items_mixed(const float4* __restrict__ hi, const float4* __restrict__ lo,
                const double* __restrict__ lam, double* __restrict__ part,
                const MvItem* __restrict__ items, int n_items, int* __restrict__ counter,
                RpyK<float> k, const int* __restrict__ active) {
    dep_wait();
    __shared__ float4 sh[kTile];
    __shared__ float4 so[kTile];
    __shared__ float4 sl[kTile];
    __shared__ int s_item;
    for (int round = 0;; ++round) {
        // first item = the block's own index (spread over the SMs as the
        // blocks are), later ones from the queue
        __syncthreads();
        if (threadIdx.x == 0) s_item = round == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(counter, 1);
        __syncthreads();
        const int itn = s_item;
        if (itn >= n_items) break;
        const MvItem m = items[itn];
        if (item_skipped(m, active, part)) continue;
        float4 hi_i[TPT], lo_i[TPT];
        float near2[TPT];
        double U[TPT][3];
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int i = m.t0 + t * kThreads + threadIdx.x;
            hi_i[t] = (i < m.t1) ? hi[i] : make_float4(0.f, 0.f, 1.f, 0.f);
            lo_i[t] = (i < m.t1) ? lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float nr = 0.25f * fmaxf(fabsf(hi_i[t].x), fmaxf(fabsf(hi_i[t].y), fabsf(hi_i[t].z)));
            near2[t] = nr * nr;
            U[t][0] = U[t][1] = U[t][2] = 0.0;
        }
        // warps with no target of the item only help stage the sources
        const bool warp_live = m.t0 + (int)(threadIdx.x & ~31u) < m.t1;
        for (int jt = m.j0; jt < m.j1; jt += kTile) {
            const int cnt = min(kTile, m.j1 - jt);
            __syncthreads();
            if (threadIdx.x < cnt) {
                const int j = jt + threadIdx.x;
                const float4 hj = hi[j];
                sh[threadIdx.x] = make_float4(hj.x, hj.y, hj.z, 2.f * hj.z);  // .w: twice the height
                so[threadIdx.x] = lo[j];
                sl[threadIdx.x] = make_float4((float)lam[3 * (size_t)j], (float)lam[3 * (size_t)j + 1],
                                              (float)lam[3 * (size_t)j + 2], 0.f);
            }
            __syncthreads();
            if (!warp_live) continue;
            // pair terms summed in FP32 over blocks of kSumBlock sources, each block
            // added to the tile's (hi, lo) sums by TwoSum, the tile folded into FP64
            float th[TPT][3], tl[TPT][3];
#pragma unroll
            for (int t = 0; t < TPT; ++t)
                for (int c = 0; c < 3; ++c) th[t][c] = tl[t][c] = 0.f;
            for (int q0 = 0; q0 < cnt; q0 += kSumBlock) {
            const int qe = min(cnt, q0 + kSumBlock);
            float u[TPT][3];
#pragma unroll
            for (int t = 0; t < TPT; ++t) u[t][0] = u[t][1] = u[t][2] = 0.f;
#pragma unroll 2
            for (int q = q0; q < qe; ++q) {
                const float4 h = sh[q];
                const float4 l = sl[q];
#pragma unroll
                for (int t = 0; t < TPT; ++t) {
                    float dx = hi_i[t].x - h.x, dy = hi_i[t].y - h.y, dz = hi_i[t].z - h.z;
                    float rxy2 = fmaf(dx, dx, dy * dy);
                    float r2 = fmaf(dz, dz, rxy2);
                    if (r2 < near2[t]) {
                        const float4 o = so[q];
                        dx += lo_i[t].x - o.x;
                        dy += lo_i[t].y - o.y;
                        dz += lo_i[t].z - o.z;
                        rxy2 = fmaf(dx, dx, dy * dy);
                        r2 = fmaf(dz, dz, rxy2);
                    }
                    if (WALL)
                        pair_wall_r2<float>(dx, dy, dz, rxy2, r2, hi_i[t].z + h.z, h.w, -hi_i[t].z, l.x, l.y, l.z,
                                            k, u[t][0], u[t][1], u[t][2]);
                    else
                        pair_free_r2<float>(dx, dy, dz, r2, l.x, l.y, l.z, k, u[t][0], u[t][1], u[t][2]);
                }
            }
#pragma unroll
            for (int t = 0; t < TPT; ++t)
                for (int c = 0; c < 3; ++c) two_sum_acc(th[t][c], tl[t][c], u[t][c]);
            }
#pragma unroll
            for (int t = 0; t < TPT; ++t)
                for (int c = 0; c < 3; ++c) U[t][c] += (double)th[t][c] + (double)tl[t][c];
        }
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int i = m.t0 + t * kThreads + threadIdx.x;
            if (i < m.t1) {
                double* o = part + m.pbase + 3 * (size_t)(i - m.tbase);
                o[0] = k.A1 * U[t][0]; o[1] = k.A1 * U[t][1]; o[2] = k.A1 * U[t][2];
            }
        }
    }
    item_queue_done(counter);
}

// ---- paired FP32 arithmetic: two targets per thread in the lanes of float2
// registers (__ffma2_rn and friends: one instruction for both targets), the
// source values in shared memory already duplicated and negated so that one
// 128-bit load gives ready register pairs.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 rsq2(float2 a) { return make_float2(rsq(a.x), rsq(a.y)); }

// (hi, lo) += t exactly in each lane (Knuth's TwoSum of hi and t, the
// rounding error added to lo): the compensated accumulation of the tile sums
__device__ __forceinline__ void two_sum_acc2(float2& hi, float2& lo, float2 t) {
    const float2 m1 = bc2(-1.f);
    const float2 s = add2(hi, t);
    const float2 v = fma2(hi, m1, s);                          // s - hi
    const float2 e = add2(fma2(fma2(v, m1, s), m1, hi),        // hi - (s - v)
                          fma2(v, m1, t));                      // + (t - v)
    hi = s;
    lo = add2(lo, e);
}

// Free-space pair plus wall image in both lanes: pair_wall_r2 of
// rpy_pair.cuh (same operations in the same order), with the free-space
// coefficients of the far branch; pairs closer than 2a in either lane take
// free_coefs per lane.  nx3 = -x3 per lane.
template <bool WALL>
__device__ __forceinline__ void pair2(float2 dx, float2 dy, float2 dz, float2 rxy2, float2 r2, float2 Rz, float2 h2,
                                      float2 nx3, float2 lx, float2 ly, float2 lz, const RpyK<float>& k,
                                      float2& ux, float2& uy, float2& uz) {
    const float2 one = bc2(1.f);
    float2 c1f, c2f;
    if (r2.x < k.four_a2 || r2.y < k.four_a2) {
        free_coefs<float>(r2.x, k, c1f.x, c2f.x);
        free_coefs<float>(r2.y, k, c1f.y, c2f.y);
    } else {
        const float2 ri = rsq2(r2);
        const float2 ri2 = mul2(ri, ri);
        c1f = mul2(ri, fma2(bc2(k.kf2), ri2, one));
        c2f = mul2(mul2(ri, ri2), fma2(bc2(-k.kf3), ri2, one));
    }
    const float2 dlxy = fma2(dx, lx, mul2(dy, ly));
    const float2 Df = fma2(dz, lz, dlxy);
    const float2 sdl = mul2(c2f, Df);
    if (!WALL) {
        ux = fma2(c1f, lx, fma2(sdl, dx, ux));
        uy = fma2(c1f, ly, fma2(sdl, dy, uy));
        uz = fma2(c1f, lz, fma2(sdl, dz, uz));
        return;
    }
    const float2 Rz2 = mul2(Rz, Rz);
    const float2 Di = fma2(Rz, lz, dlxy);
    const float2 s = rsq2(add2(rxy2, Rz2));
    const float2 w = mul2(s, s), s3 = mul2(s, w), w2 = mul2(w, w);
    const float2 c1 = fma2(h2, nx3, bc2(k.wc1));
    const float2 c2 = fma2(Rz2, bc2(k.w2a2), bc2(k.wc2));
    const float2 c3 = mul2(Rz2, bc2(k.wc3));
    const float2 x1 = fma2(w, c3, c2);
    const float2 cI = fma2(w, fma2(w, x1, c1), bc2(-1.f));
    const float2 y = fma2(w, c3, x1);
    const float2 yz = fma2(w, c3, y);
    const float2 cRR = fma2(mul2(w2, y), bc2(-2.f), fma2(cI, bc2(-3.f), bc2(-4.f)));
    const float2 A4w2n = mul2(w2, bc2(-k.wa4));
    const float2 inner = fma2(cRR, bc2(-2.f), fma2(A4w2n, bc2(-1.f), bc2(-2.f)));
    const float2 P = mul2(s3, fma2(cRR, Di, mul2(fma2(Rz, inner, h2), lz)));
    const float2 Q = mul2(s3, fma2(h2, Df, fma2(mul2(A4w2n, Rz), Di, mul2(mul2(w, fma2(yz, bc2(-2.f), bc2(k.wi2))), lz))));
    const float2 cc = fma2(s, cI, c1f);
    const float2 pp = add2(sdl, P);
    ux = fma2(cc, lx, fma2(pp, dx, ux));
    uy = fma2(cc, ly, fma2(pp, dy, uy));
    uz = fma2(cc, lz, fma2(sdl, dz, fma2(P, Rz, add2(uz, Q))));
}

// Both directions of a pair in paired FP32 lanes: u += M lambda_src for two
// targets (the lanes), and v += M^T mu for the source from each target (v.x
// from the first, v.y from the second; the caller adds them).  The
// operations of pair_wall_sym (rpy_pair.cuh) on the lanes of pair2.
template <bool WALL>
__device__ __forceinline__ void pair2_sym(float2 dx, float2 dy, float2 dz, float2 rxy2, float2 r2, float2 Rz,
                                          float2 h2, float2 nx3, float2 lx, float2 ly, float2 lz, float2 mx,
                                          float2 my, float2 mz, const RpyK<float>& k, float2& ux, float2& uy,
                                          float2& uz, float2& vx, float2& vy, float2& vz) {
    const float2 one = bc2(1.f);
    float2 c1f, c2f;
    if (r2.x < k.four_a2 || r2.y < k.four_a2) {
        free_coefs<float>(r2.x, k, c1f.x, c2f.x);
        free_coefs<float>(r2.y, k, c1f.y, c2f.y);
    } else {
        const float2 ri = rsq2(r2);
        const float2 ri2 = mul2(ri, ri);
        c1f = mul2(ri, fma2(bc2(k.kf2), ri2, one));
        c2f = mul2(mul2(ri, ri2), fma2(bc2(-k.kf3), ri2, one));
    }
    const float2 dlxy = fma2(dx, lx, mul2(dy, ly));
    const float2 Df = fma2(dz, lz, dlxy);
    const float2 dmxy = fma2(dx, mx, mul2(dy, my));
    const float2 Dfm = fma2(dz, mz, dmxy);
    if (!WALL) {
        const float2 sl = mul2(c2f, Df), sm = mul2(c2f, Dfm);
        ux = fma2(c1f, lx, fma2(sl, dx, ux));
        uy = fma2(c1f, ly, fma2(sl, dy, uy));
        uz = fma2(c1f, lz, fma2(sl, dz, uz));
        vx = fma2(c1f, mx, fma2(sm, dx, vx));
        vy = fma2(c1f, my, fma2(sm, dy, vy));
        vz = fma2(c1f, mz, fma2(sm, dz, vz));
        return;
    }
    const float2 Rz2 = mul2(Rz, Rz);
    const float2 s = rsq2(add2(rxy2, Rz2));
    const float2 w = mul2(s, s), s3 = mul2(s, w), w2 = mul2(w, w);
    const float2 c1 = fma2(h2, nx3, bc2(k.wc1));
    const float2 c2 = fma2(Rz2, bc2(k.w2a2), bc2(k.wc2));
    const float2 c3 = mul2(Rz2, bc2(k.wc3));
    const float2 x1 = fma2(w, c3, c2);
    const float2 cI = fma2(w, fma2(w, x1, c1), bc2(-1.f));
    const float2 y = fma2(w, c3, x1);
    const float2 yz = fma2(w, c3, y);
    const float2 cRR = fma2(mul2(w2, y), bc2(-2.f), fma2(cI, bc2(-3.f), bc2(-4.f)));
    const float2 A4w2n = mul2(w2, bc2(-k.wa4));
    const float2 cc = fma2(s, cI, c1f);
    const float2 g = fma2(Rz, fma2(cRR, bc2(-2.f), fma2(A4w2n, bc2(-1.f), bc2(-2.f))), h2);
    const float2 s3cRR = mul2(s3, cRR), s3g = mul2(s3, g), s3h2 = mul2(s3, h2);
    const float2 s3A = mul2(s3, mul2(A4w2n, Rz)), s3phi = mul2(s3, mul2(w, fma2(yz, bc2(-2.f), bc2(k.wi2))));
    {
        const float2 Di = fma2(Rz, lz, dlxy);
        const float2 sdl = mul2(c2f, Df);
        const float2 P = fma2(s3cRR, Di, mul2(s3g, lz));
        const float2 Q = fma2(s3h2, Df, fma2(s3A, Di, mul2(s3phi, lz)));
        const float2 pp = add2(sdl, P);
        ux = fma2(cc, lx, fma2(pp, dx, ux));
        uy = fma2(cc, ly, fma2(pp, dy, uy));
        uz = fma2(cc, lz, fma2(sdl, dz, fma2(P, Rz, add2(uz, Q))));
    }
    {
        const float2 Di = fma2(Rz, mz, dmxy);
        const float2 cd = fma2(c2f, Dfm, mul2(s3h2, mz));
        const float2 P = fma2(s3cRR, Di, mul2(s3A, mz));
        const float2 Q = fma2(s3g, Di, mul2(s3phi, mz));
        const float2 pp = add2(cd, P);
        vx = fma2(cc, mx, fma2(pp, dx, vx));
        vy = fma2(cc, my, fma2(pp, dy, vy));
        vz = fma2(cc, mz, fma2(cd, dz, fma2(P, Rz, add2(vz, Q))));
    }
}

// Symmetric mixed product on tile pairs of 128 blobs (the SymItem list of
// the handle, tiles of 128): warp w holds 64 targets of tile I, two per lane
// in the lanes of float2 registers (targets 64 (w & 1) + l and + 32), and
// takes source sub-tiles 2 (w >> 1) and 2 (w >> 1) + 1 of tile J (32
// sources each).  At step t lane l meets source (l + t) mod 32 of the
// sub-tile with both targets; the source's column sum (the two targets'
// contributions added) moves one lane per step as in rpy_sym_f64.
// Differences from the hi parts, with the lo parts added within a quarter
// of the target's largest coordinate (as rpy_items_mixed_x2).  FP32 sums over
// at most 64 terms (a warp's sources for u, its targets for v), added in
// FP64 across warps in a fixed order.  Diagonal items (I = J) take every
// ordered pair in one direction (the self term included), no column sums.
template <bool WALL>
__global__ void __launch_bounds__(kThreads, 4)
rpy_sym_mixed_x2(const float4* __restrict__ hi, const float4* __restrict__ lo, const double* __restrict__ lam,
                 double* __restrict__ part, const SymItem* __restrict__ items, int n_items, int* __restrict__ counter,
                 RpyK<float> k, const int* __restrict__ active) {
    dep_wait();
    constexpr int T = 128;
    __shared__ float4 sq[3][T];   // sources: (-hx, -hx, -hy, -hy), (2hz, 2hz, lz, lz), (lx, lx, ly, ly)
    __shared__ float4 so[T];      // (-ox, -ox, -oy, -oy)
    __shared__ float2 soz[T];     // (-oz, -oz)
    __shared__ double up[4][64][3];     // row sums of each warp's 64 targets
    __shared__ double vp[4][2][32][3];  // column sums of each warp's two sub-tiles
    __shared__ int s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int th = warp & 1;            // target half of tile I
    const int sb0 = 2 * (warp >> 1);    // the warp's first source sub-tile
    for (int round = 0;; ++round) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = round == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(counter, 1);
        __syncthreads();
        const int itn = s_item;
        if (itn >= n_items) break;
        const SymItem m = items[itn];
        const bool diag = m.ti == m.tj;
        double* rowo = part + m.poff + (long long)m.tj * m.n3 + 3 * (long long)(m.i0 - m.tbase);
        double* colo = part + m.poff + (long long)m.ti * m.n3 + 3 * (long long)(m.j0 - m.tbase);
        if (active && !active[m.sys]) {
            for (int q = threadIdx.x; q < 3 * m.ni; q += blockDim.x) rowo[q] = 0.0;
            if (!diag)
                for (int q = threadIdx.x; q < 3 * m.nj; q += blockDim.x) colo[q] = 0.0;
            continue;
        }
        {   // stage the sources of tile J (one per thread)
            const int q = threadIdx.x;
            const bool ok = q < m.nj;
            const float4 h = ok ? hi[m.j0 + q] : make_float4(0.f, 0.f, 1.f, 0.f);
            const float4 o = ok ? lo[m.j0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float lx = ok ? (float)lam[3 * (size_t)(m.j0 + q)] : 0.f;
            const float ly = ok ? (float)lam[3 * (size_t)(m.j0 + q) + 1] : 0.f;
            const float lz = ok ? (float)lam[3 * (size_t)(m.j0 + q) + 2] : 0.f;
            sq[0][q] = make_float4(-h.x, -h.x, -h.y, -h.y);
            sq[1][q] = make_float4(2.f * h.z, 2.f * h.z, lz, lz);
            sq[2][q] = make_float4(lx, lx, ly, ly);
            so[q] = make_float4(-o.x, -o.x, -o.y, -o.y);
            soz[q] = make_float2(-o.z, -o.z);
        }
        __syncthreads();
        const int t0 = 64 * th + lane, t1 = t0 + 32;
        const bool ok0 = t0 < m.ni, ok1 = t1 < m.ni;
        const float4 h0 = ok0 ? hi[m.i0 + t0] : make_float4(0.f, 0.f, 1.f, 0.f);
        const float4 h1 = ok1 ? hi[m.i0 + t1] : make_float4(0.f, 0.f, 1.f, 0.f);
        const float4 l0 = ok0 ? lo[m.i0 + t0] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 l1 = ok1 ? lo[m.i0 + t1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 HX = make_float2(h0.x, h1.x), HY = make_float2(h0.y, h1.y), HZ = make_float2(h0.z, h1.z);
        const float2 LX = make_float2(l0.x, l1.x), LY = make_float2(l0.y, l1.y), LZ = make_float2(l0.z, l1.z);
        const float2 NX3 = make_float2(-h0.z, -h1.z);
        const float n0 = 0.25f * fmaxf(fabsf(h0.x), fmaxf(fabsf(h0.y), fabsf(h0.z)));
        const float n1 = 0.25f * fmaxf(fabsf(h1.x), fmaxf(fabsf(h1.y), fabsf(h1.z)));
        const float near2x = n0 * n0, near2y = n1 * n1;
        // the targets' forces for the column sums (zero for missing targets)
        float2 MX = bc2(0.f), MY = bc2(0.f), MZ = bc2(0.f);
        if (ok0) {
            MX.x = (float)lam[3 * (size_t)(m.i0 + t0)];
            MY.x = (float)lam[3 * (size_t)(m.i0 + t0) + 1];
            MZ.x = (float)lam[3 * (size_t)(m.i0 + t0) + 2];
        }
        if (ok1) {
            MX.y = (float)lam[3 * (size_t)(m.i0 + t1)];
            MY.y = (float)lam[3 * (size_t)(m.i0 + t1) + 1];
            MZ.y = (float)lam[3 * (size_t)(m.i0 + t1) + 2];
        }
        float2 ux = bc2(0.f), uy = bc2(0.f), uz = bc2(0.f);
        for (int sbi = 0; sbi < 2; ++sbi) {
            const int sb = sb0 + sbi;
            float vx = 0.f, vy = 0.f, vz = 0.f;  // column sum of source 32 sb + ((lane + t) & 31)
#pragma unroll 2
            for (int t = 0; t < 32; ++t) {
                const int q = 32 * sb + (diag ? t : ((lane + t) & 31));
                const float4 v0 = sq[0][q], v1 = sq[1][q], v2 = sq[2][q];
                const float2 h2 = make_float2(v1.x, v1.y);
                float2 dx = add2(HX, make_float2(v0.x, v0.y));
                float2 dy = add2(HY, make_float2(v0.z, v0.w));
                float2 dz = fma2(h2, bc2(-0.5f), HZ);
                const float2 Rz = fma2(h2, bc2(0.5f), HZ);
                float2 rxy2 = fma2(dx, dx, mul2(dy, dy));
                float2 r2 = fma2(dz, dz, rxy2);
                if (r2.x < near2x || r2.y < near2y) {
                    const float4 o = so[q];
                    dx = add2(dx, add2(LX, make_float2(o.x, o.y)));
                    dy = add2(dy, add2(LY, make_float2(o.z, o.w)));
                    dz = add2(dz, add2(LZ, soz[q]));
                    rxy2 = fma2(dx, dx, mul2(dy, dy));
                    r2 = fma2(dz, dz, rxy2);
                }
                const float2 lxs = make_float2(v2.x, v2.y), lys = make_float2(v2.z, v2.w),
                             lzs = make_float2(v1.z, v1.w);
                if (diag) {
                    pair2<WALL>(dx, dy, dz, rxy2, r2, Rz, h2, NX3, lxs, lys, lzs, k, ux, uy, uz);
                } else {
                    float2 cx = bc2(0.f), cy = bc2(0.f), cz = bc2(0.f);
                    pair2_sym<WALL>(dx, dy, dz, rxy2, r2, Rz, h2, NX3, lxs, lys, lzs, MX, MY, MZ, k, ux, uy, uz,
                                    cx, cy, cz);
                    vx += cx.x + cx.y;
                    vy += cy.x + cy.y;
                    vz += cz.x + cz.y;
                    const int src = (lane + 1) & 31;
                    vx = __shfl_sync(0xffffffffu, vx, src);
                    vy = __shfl_sync(0xffffffffu, vy, src);
                    vz = __shfl_sync(0xffffffffu, vz, src);
                }
            }
            vp[warp][sbi][lane][0] = vx;
            vp[warp][sbi][lane][1] = vy;
            vp[warp][sbi][lane][2] = vz;
        }
        up[warp][lane][0] = ux.x; up[warp][lane][1] = uy.x; up[warp][lane][2] = uz.x;
        up[warp][32 + lane][0] = ux.y; up[warp][32 + lane][1] = uy.y; up[warp][32 + lane][2] = uz.y;
        __syncthreads();
        {
            const int t = threadIdx.x;
            if (t < m.ni) {  // target t: half t >> 6, row t & 63 of warps th and th + 2
                const int hh = t >> 6, j = t & 63;
                rowo[3 * t] = k.A1 * (up[hh][j][0] + up[hh + 2][j][0]);
                rowo[3 * t + 1] = k.A1 * (up[hh][j][1] + up[hh + 2][j][1]);
                rowo[3 * t + 2] = k.A1 * (up[hh][j][2] + up[hh + 2][j][2]);
            }
            if (!diag && t < m.nj) {  // source t: sub-tile sb = t >> 5 of warps 2 (sb >> 1) and + 1
                const int sb = t >> 5, l = t & 31, wa = 2 * (sb >> 1), si = sb & 1;
                colo[3 * t] = k.A1 * (vp[wa][si][l][0] + vp[wa + 1][si][l][0]);
                colo[3 * t + 1] = k.A1 * (vp[wa][si][l][1] + vp[wa + 1][si][l][1]);
                colo[3 * t + 2] = k.A1 * (vp[wa][si][l][2] + vp[wa + 1][si][l][2]);
            }
        }
    }
    item_queue_done(counter);
}

// Symmetric mixed product on tiles of 32 NSUB blobs, one target per lane:
// the scheme of rpy_sym_f64 (each unordered pair of a tile pair evaluated
// once and applied in both directions, the column sums carried from lane
// to lane, the diagonal warp tile on steps 1..16) with FP32 pair terms.
// Differences are formed from the hi parts of the positions; within a
// quarter of the target's largest coordinate the lo parts are added, as in
// rpy_items_mixed.  A lane sums the 32 terms of a warp tile in FP32; the
// warp-tile sums are added in FP64 in a fixed order.  Small tiles spread
// systems of a few thousand blobs over every SM.
template <bool WALL, int NSUB>
__global__ void __launch_bounds__(NSUB == 1 ? 32 : 128)
rpy_sym_mixed(const float4* __restrict__ hi, const float4* __restrict__ lo, const double* __restrict__ lam,
              double* __restrict__ part, const SymItem* __restrict__ items, int n_items, int* __restrict__ counter,
              RpyK<float> k, const int* __restrict__ active) {
    dep_wait();
    constexpr int T = 32 * NSUB;
    constexpr int NW = NSUB == 1 ? 1 : 4;
    constexpr int NWT = NSUB * NSUB;
    __shared__ float4 hI[T], hJ[T];  // hi parts, .w = twice the height
    __shared__ float4 oI[T], oJ[T];  // lo parts
    __shared__ float4 lI[T], lJ[T];  // forces
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
        double* rowo = part + m.poff + (long long)m.tj * m.n3 + 3 * (long long)(m.i0 - m.tbase);
        double* colo = part + m.poff + (long long)m.ti * m.n3 + 3 * (long long)(m.j0 - m.tbase);
        if (active && !active[m.sys]) {  // a stopped system: zero partial sums
            for (int q = threadIdx.x; q < 3 * m.ni; q += blockDim.x) rowo[q] = 0.0;
            if (!diag)
                for (int q = threadIdx.x; q < 3 * m.nj; q += blockDim.x) colo[q] = 0.0;
            continue;
        }
        for (int q = threadIdx.x; q < T; q += blockDim.x) {
            const bool oi = q < m.ni, oj = q < m.nj;
            float4 a = oi ? hi[m.i0 + q] : make_float4(0.f, 0.f, 1.f, 0.f);
            a.w = 2.f * a.z;
            hI[q] = a;
            oI[q] = oi ? lo[m.i0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
            lI[q] = oi ? make_float4((float)lam[3 * (size_t)(m.i0 + q)], (float)lam[3 * (size_t)(m.i0 + q) + 1],
                                     (float)lam[3 * (size_t)(m.i0 + q) + 2], 0.f)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 b = oj ? hi[m.j0 + q] : make_float4(0.f, 0.f, 1.f, 0.f);
            b.w = 2.f * b.z;
            hJ[q] = b;
            oJ[q] = oj ? lo[m.j0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
            lJ[q] = oj ? make_float4((float)lam[3 * (size_t)(m.j0 + q)], (float)lam[3 * (size_t)(m.j0 + q) + 1],
                                     (float)lam[3 * (size_t)(m.j0 + q) + 2], 0.f)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        for (int wt = warp; wt < NWT; wt += NW) {
            const int a = wt / NSUB, b = wt % NSUB;
            float ux = 0.f, uy = 0.f, uz = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
            if (!(diag && b < a)) {  // below the diagonal of a diagonal item: taken by (b, a)
                const bool self_tile = diag && a == b;
                const int t = 32 * a + lane;
                const float4 xi = hI[t], xo = oI[t], mu = lI[t];
                const float nr = 0.25f * fmaxf(fabsf(xi.x), fmaxf(fabsf(xi.y), fabsf(xi.z)));
                const float near2 = nr * nr;
                const bool ti_ok = t < m.ni;
#pragma unroll 1
                for (int step = 0; step < 32; ++step) {
                    const int q = 32 * b + ((lane + step) & 31);
                    const bool pair_ok = ti_ok && q < m.nj &&
                                         (!self_tile || (step >= 1 && (step < 16 || (step == 16 && lane < 16))));
                    if (pair_ok) {
                        const float4 xj = hJ[q], l = lJ[q];
                        float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
                        float rxy2 = fmaf(dx, dx, dy * dy);
                        float r2 = fmaf(dz, dz, rxy2);
                        if (r2 < near2) {
                            const float4 o = oJ[q];
                            dx += xo.x - o.x;
                            dy += xo.y - o.y;
                            dz += xo.z - o.z;
                            rxy2 = fmaf(dx, dx, dy * dy);
                            r2 = fmaf(dz, dz, rxy2);
                        }
                        if (WALL)
                            pair_wall_sym<float>(dx, dy, dz, rxy2, r2, xi.z + xj.z, xj.w, -xi.z, l.x, l.y, l.z, mu.x,
                                                 mu.y, mu.z, k, ux, uy, uz, vx, vy, vz);
                        else
                            pair_free_sym<float>(dx, dy, dz, r2, l.x, l.y, l.z, mu.x, mu.y, mu.z, k, ux, uy, uz, vx,
                                                 vy, vz);
                    } else if (self_tile && step == 0 && ti_ok) {  // the self term
                        if (WALL)
                            pair_wall_r2<float>(0.f, 0.f, 0.f, 0.f, 0.f, xi.w, xi.w, -xi.z, mu.x, mu.y, mu.z, k, ux,
                                                uy, uz);
                        else
                            pair_free<float>(0.f, 0.f, 0.f, mu.x, mu.y, mu.z, k, ux, uy, uz);
                    }
                    // hand the column sum to the lane that meets this source next
                    const int src = (lane + 1) & 31;
                    vx = __shfl_sync(0xffffffffu, vx, src);
                    vy = __shfl_sync(0xffffffffu, vy, src);
                    vz = __shfl_sync(0xffffffffu, vz, src);
                }
            }
            up[wt][lane][0] = ux; up[wt][lane][1] = uy; up[wt][lane][2] = uz;
            vp[wt][lane][0] = vx; vp[wt][lane][1] = vy; vp[wt][lane][2] = vz;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            const int a = t >> 5, l = t & 31;
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

// The mixed product with two targets per thread (items of 256 targets):
// target t0 + threadIdx.x in lane x, t0 + 128 + threadIdx.x in lane y.
// Differences are formed from the hi parts; within a quarter of the
// target's largest coordinate (either lane), where the rounding of hi
// would exceed 5e-7 of the distance, the lo parts are added (as in
// rpy_items_mixed).  The sources are staged duplicated in shared memory so
// that one 128-bit load gives ready register pairs: (-hx, -hx, -hy, -hy),
// (2hz, 2hz, lz, lz), (lx, lx, ly, ly), and the lo parts (-ox, -ox, -oy, -oy),
// (-oz, -oz) apart, read only for near pairs.
template <bool WALL>
__global__ void __launch_bounds__(kThreads, 5)
rpy_items_mixed_x2(const float4* __restrict__ hi, const float4* __restrict__ lo,
                   const double* __restrict__ lam, double* __restrict__ part,
                   const MvItem* __restrict__ items, int n_items, int* __restrict__ counter,
                   RpyK<float> k, const int* __restrict__ active) {
    dep_wait();
    __shared__ float4 sq[3][kTile];
    __shared__ float4 so[kTile];
    __shared__ float2 soz[kTile];
    __shared__ int s_item;
    for (int round = 0;; ++round) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = round == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(counter, 1);
        __syncthreads();
        const int itn = s_item;
        if (itn >= n_items) break;
        const MvItem m = items[itn];
        if (item_skipped(m, active, part)) continue;
        const int i0 = m.t0 + threadIdx.x, i1 = m.t0 + kThreads + threadIdx.x;
        const float4 h0 = (i0 < m.t1) ? hi[i0] : make_float4(0.f, 0.f, 1.f, 0.f);
        const float4 h1 = (i1 < m.t1) ? hi[i1] : make_float4(0.f, 0.f, 1.f, 0.f);
        const float4 l0 = (i0 < m.t1) ? lo[i0] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 l1 = (i1 < m.t1) ? lo[i1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 HX = make_float2(h0.x, h1.x), HY = make_float2(h0.y, h1.y), HZ = make_float2(h0.z, h1.z);
        const float2 LX = make_float2(l0.x, l1.x), LY = make_float2(l0.y, l1.y), LZ = make_float2(l0.z, l1.z);
        const float2 NX3 = make_float2(-h0.z, -h1.z);
        const float n0 = 0.25f * fmaxf(fabsf(h0.x), fmaxf(fabsf(h0.y), fabsf(h0.z)));
        const float n1 = 0.25f * fmaxf(fabsf(h1.x), fmaxf(fabsf(h1.y), fabsf(h1.z)));
        const float near2x = n0 * n0, near2y = n1 * n1;
        double U[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
        for (int jt = m.j0; jt < m.j1; jt += kTile) {
            const int cnt = min(kTile, m.j1 - jt);
            __syncthreads();
            if (threadIdx.x < cnt) {
                const int j = jt + threadIdx.x;
                const float4 h = hi[j], o = lo[j];
                const float lx = (float)lam[3 * (size_t)j], ly = (float)lam[3 * (size_t)j + 1],
                            lz = (float)lam[3 * (size_t)j + 2];
                sq[0][threadIdx.x] = make_float4(-h.x, -h.x, -h.y, -h.y);
                sq[1][threadIdx.x] = make_float4(2.f * h.z, 2.f * h.z, lz, lz);
                sq[2][threadIdx.x] = make_float4(lx, lx, ly, ly);
                so[threadIdx.x] = make_float4(-o.x, -o.x, -o.y, -o.y);
                soz[threadIdx.x] = make_float2(-o.z, -o.z);
            }
            __syncthreads();
            // pair terms summed in FP32 over blocks of kSumBlock sources, each block
            // added to the tile's (hi, lo) sums by TwoSum, the tile folded
            // into FP64
            float2 hx = bc2(0.f), hy = bc2(0.f), hz = bc2(0.f), lx_ = bc2(0.f), ly_ = bc2(0.f), lz_ = bc2(0.f);
            for (int q0 = 0; q0 < cnt; q0 += kSumBlock) {
            const int qe = min(cnt, q0 + kSumBlock);
            float2 ux = bc2(0.f), uy = bc2(0.f), uz = bc2(0.f);
#pragma unroll 2
            for (int q = q0; q < qe; ++q) {
                const float4 v0 = sq[0][q], v1 = sq[1][q], v2 = sq[2][q];
                const float2 h2 = make_float2(v1.x, v1.y);
                float2 dx = add2(HX, make_float2(v0.x, v0.y));
                float2 dy = add2(HY, make_float2(v0.z, v0.w));
                float2 dz = fma2(h2, bc2(-0.5f), HZ);
                const float2 Rz = fma2(h2, bc2(0.5f), HZ);
                float2 rxy2 = fma2(dx, dx, mul2(dy, dy));
                float2 r2 = fma2(dz, dz, rxy2);
                if (r2.x < near2x || r2.y < near2y) {
                    const float4 o = so[q];
                    dx = add2(dx, add2(LX, make_float2(o.x, o.y)));
                    dy = add2(dy, add2(LY, make_float2(o.z, o.w)));
                    dz = add2(dz, add2(LZ, soz[q]));
                    rxy2 = fma2(dx, dx, mul2(dy, dy));
                    r2 = fma2(dz, dz, rxy2);
                }
                pair2<WALL>(dx, dy, dz, rxy2, r2, Rz, h2, NX3, make_float2(v2.x, v2.y), make_float2(v2.z, v2.w),
                            make_float2(v1.z, v1.w), k, ux, uy, uz);
            }
            two_sum_acc2(hx, lx_, ux);
            two_sum_acc2(hy, ly_, uy);
            two_sum_acc2(hz, lz_, uz);
            }
            U[0][0] += (double)hx.x + (double)lx_.x; U[0][1] += (double)hy.x + (double)ly_.x;
            U[0][2] += (double)hz.x + (double)lz_.x;
            U[1][0] += (double)hx.y + (double)lx_.y; U[1][1] += (double)hy.y + (double)ly_.y;
            U[1][2] += (double)hz.y + (double)lz_.y;
        }
        if (i0 < m.t1) {
            double* o = part + m.pbase + 3 * (size_t)(i0 - m.tbase);
            o[0] = k.A1 * U[0][0]; o[1] = k.A1 * U[0][1]; o[2] = k.A1 * U[0][2];
        }
        if (i1 < m.t1) {
            double* o = part + m.pbase + 3 * (size_t)(i1 - m.tbase);
            o[0] = k.A1 * U[1][0]; o[1] = k.A1 * U[1][1]; o[2] = k.A1 * U[1][2];
        }
    }
    item_queue_done(counter);
}

// u_i = sum over the chunks of i's system of the partial sums
__global__ void k_sum_items(int Nb, const double* __restrict__ part, const int* __restrict__ sys_of_blob,
                            const int* __restrict__ sys_blob0, const int* __restrict__ sys_nb,
                            const int* __restrict__ sys_nch, const long long* __restrict__ sys_poff,
                            double* __restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const int s = sys_of_blob[i];
    const size_t n3 = 3 * (size_t)sys_nb[s];
    const double* p = part + sys_poff[s] + 3 * (size_t)(i - sys_blob0[s]);
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = 0; q < sys_nch[s]; ++q) {
        a += p[q * n3]; b += p[q * n3 + 1]; c += p[q * n3 + 2];
    }
    u[3 * (size_t)i] = a; u[3 * (size_t)i + 1] = b; u[3 * (size_t)i + 2] = c;
}

template <class F>
static int resident_grid(F kernel, int threads = kThreads) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess || per <= 0)
        per = 4;
    return per * num_sms();
}

// resident blocks of the symmetric FP64 kernel for nsub (1, 2, 4)
static int sym_grid(bool wall, int nsub) {
    const int th = nsub == 1 ? 32 : 128;
    if (wall) {
        if (nsub == 1) return resident_grid(rpy_sym_f64<true, 1>, th);
        if (nsub == 2) return resident_grid(rpy_sym_f64<true, 2>, th);
        return resident_grid(rpy_sym_f64<true, 4>, th);
    }
    if (nsub == 1) return resident_grid(rpy_sym_f64<false, 1>, th);
    if (nsub == 2) return resident_grid(rpy_sym_f64<false, 2>, th);
    return resident_grid(rpy_sym_f64<false, 4>, th);
}

// resident blocks of the symmetric mixed kernel: paired lanes (tpt 2,
// tiles of 128) or one target per lane (tiles of 32 nsub)
static int sym_mixed_grid(bool wall, int tpt, int nsub) {
    if (tpt == 2) return wall ? resident_grid(rpy_sym_mixed_x2<true>) : resident_grid(rpy_sym_mixed_x2<false>);
    const int th = nsub == 1 ? 32 : 128;
    if (wall) {
        if (nsub == 1) return resident_grid(rpy_sym_mixed<true, 1>, th);
        if (nsub == 2) return resident_grid(rpy_sym_mixed<true, 2>, th);
        return resident_grid(rpy_sym_mixed<true, 4>, th);
    }
    if (nsub == 1) return resident_grid(rpy_sym_mixed<false, 1>, th);
    if (nsub == 2) return resident_grid(rpy_sym_mixed<false, 2>, th);
    return resident_grid(rpy_sym_mixed<false, 4>, th);
}

// Work items for tpt targets per thread and source chunks of `chunk` blobs
// (0: choose so that the items fill the GPU); with sym = nsub > 0 also the
// tile-pair items of the symmetric product on tiles of 32 nsub blobs, whose
// partial-sum slots are the source chunks of that length (mixed handles:
// paired lanes with tpt = 2 on tiles of 128, one target per lane with
// tpt = 1).  Returns 0 on success.
int mobility_layout(am_handle* h, int tpt, int chunk, int tgroup, int sym) {
    const int S = h->S;
    if (h->cfg.precision != AM_MIXED) tpt = 1;
    if (h->per) chunk = std::max(1, h->Nb);  // the periodic product writes u in one piece
    if (h->per || (tpt == 2 && sym != 4)) sym = 0;  // paired lanes: tiles of 128 only
    if (sym) chunk = 32 * sym;
    // targets per item: a block's targets, or (one target per thread) 32 or
    // 64 of them so that small systems spread over more SMs
    if (tpt == 2 || tgroup <= 0 || tgroup > kThreads || tgroup % 32) tgroup = kThreads * tpt;
    if (chunk <= 0) {
        // about 8 resident waves of items over all systems
        long long pairs = 0;
        for (int s = 0; s < S; ++s) pairs += (long long)h->sys[s].Nb * h->sys[s].Nb;
        const long long want = 8LL * 4 * num_sms();
        const long long per_item = std::max<long long>(pairs / want, (long long)kThreads * tpt * kTile);
        chunk = (int)std::max<long long>(kTile, per_item / (kThreads * tpt) / kTile * kTile);
    }
    std::vector<MvItem> items;
    std::vector<int> nch(S);
    std::vector<long long> poff(S);
    long long off = 0;
    for (int s = 0; s < S; ++s) {
        const int nb = h->sys[s].Nb, b0 = h->sys_blob0[s];
        nch[s] = std::max(1, (nb + chunk - 1) / chunk);
        poff[s] = off;
        for (int c = 0; c < nch[s]; ++c) {
            const int j0 = b0 + c * chunk, j1 = std::min(b0 + nb, j0 + chunk);
            for (int t0 = b0; t0 < b0 + nb; t0 += tgroup) {
                MvItem it;
                it.t0 = t0; it.t1 = std::min(b0 + nb, t0 + tgroup);
                it.j0 = j0; it.j1 = j1; it.tbase = b0; it.n3 = 3 * nb;
                it.pbase = off + (long long)c * 3 * nb;
                it.sys = s; it.pad = 0;
                items.push_back(it);
            }
        }
        off += (long long)nch[s] * 3 * nb;
    }
    std::stable_sort(items.begin(), items.end(), [](const MvItem& a, const MvItem& b) {
        return (long long)(a.t1 - a.t0) * (a.j1 - a.j0) > (long long)(b.t1 - b.t0) * (b.j1 - b.j0);
    });
    std::vector<SymItem> sitems;
    if (sym) {
        const int T = 32 * sym;
        for (int s = 0; s < S; ++s) {
            const int nb = h->sys[s].Nb, b0 = h->sys_blob0[s];
            const int nt = (nb + T - 1) / T;
            for (int a = 0; a < nt; ++a)
                for (int b = a; b < nt; ++b) {
                    SymItem it;
                    it.i0 = b0 + a * T; it.ni = std::min(T, nb - a * T);
                    it.j0 = b0 + b * T; it.nj = std::min(T, nb - b * T);
                    it.tbase = b0; it.sys = s; it.ti = a; it.tj = b;
                    it.poff = poff[s]; it.n3 = 3 * nb; it.pad = 0;
                    sitems.push_back(it);
                }
        }
    }
    cudaStream_t st = h->stream;
    if (h->d_sym_items) cudaFree(h->d_sym_items);
    h->d_sym_items = nullptr;
    h->n_sym = 0;
    if (!sitems.empty()) {
        if (cudaMalloc(&h->d_sym_items, sitems.size() * sizeof(SymItem)) != cudaSuccess ||
            cudaMemcpyAsync(h->d_sym_items, sitems.data(), sitems.size() * sizeof(SymItem), cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
            return 1;
        h->n_sym = (int)sitems.size();
        h->sym_nsub = sym;
        h->mv_gridsym = std::min(sym_grid(h->cfg.wall != 0, sym), h->n_sym);
        h->mv_gridsym32 = std::min(sym_mixed_grid(h->cfg.wall != 0, tpt, sym), h->n_sym);
        h->mv_gridsymdf = std::min(sym_df_resident_grid(h->cfg.wall != 0), h->n_sym);
    }
    if (h->d_items) cudaFree(h->d_items);
    h->d_items = nullptr;
    if (h->d_mv) cudaFree(h->d_mv);
    h->d_mv = nullptr;
    if (cudaMalloc(&h->d_items, std::max<size_t>(items.size(), 1) * sizeof(MvItem)) != cudaSuccess) return 1;
    if (cudaMalloc(reinterpret_cast<void**>(&h->d_mv), std::max<long long>(off, 1) * sizeof(double)) != cudaSuccess)
        return 1;
    if (cudaMemcpyAsync(h->d_items, items.data(), items.size() * sizeof(MvItem), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(h->d_sys_nch, nch.data(), S * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(h->d_sys_poff, poff.data(), S * sizeof(long long), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return 1;
    cudaStreamSynchronize(st);
    h->n_items = (int)items.size();
    const int n_it = std::max(1, h->n_items);
    h->mv_tpt = tpt;
    h->mv_chunk = chunk;
    h->mv_tgroup = tgroup;
    h->mv_part_total = off;
    if (h->cfg.precision == AM_MIXED) {
        if (h->cfg.wall)
            h->mv_grid = tpt == 2 ? resident_grid(rpy_items_mixed_x2<true>) : resident_grid(rpy_items_mixed<true, 1>);
        else
            h->mv_grid = tpt == 2 ? resident_grid(rpy_items_mixed_x2<false>) : resident_grid(rpy_items_mixed<false, 1>);
    } else {
        h->mv_grid = h->cfg.wall ? resident_grid(rpy_items_f64<true>) : resident_grid(rpy_items_f64<false>);
    }
    h->mv_grid64 = h->cfg.wall ? resident_grid(rpy_items_f64<true>) : resident_grid(rpy_items_f64<false>);
    // never more blocks than items
    h->mv_grid = std::min(h->mv_grid, n_it);
    h->mv_grid64 = std::min(h->mv_grid64, n_it);
    h->mv_griddf = std::min(df_resident_grid(h->cfg.wall != 0), n_it);
    h->layout_gen++;
    return 0;
}

// The partial sums of u = M lambda for all systems (mode: the handle's
// precision, FP64 or double-float).
void launch_items(am_handle* h, const double* lam, int mode, const int* active) {
    if (h->per) {  // FP32 wave part for the mixed operator; FP64 for FP64 and double-float requests
        launch_periodic(h, lam, mode == kOpMixed || (mode == kOpHandle && h->cfg.precision == AM_MIXED));
        return;
    }
    if (mode == kOpDF) {
        launch_items_df(h, lam);
        return;
    }
    const bool fp64 = mode == kOpFP64 || (mode == kOpHandle && h->cfg.precision == AM_FP64);
    cudaStream_t st = h->stream;  // the queue counter is zero (reset by the last launch's last block)
    const MvItem* items = static_cast<const MvItem*>(h->d_items);
    if (fp64 && h->n_sym > 0) {
        const RpyK<double> k = rpy_consts<double>(h->prm);
        const SymItem* si = static_cast<const SymItem*>(h->d_sym_items);
        const int th = h->sym_nsub == 1 ? 32 : 128;
#define AM_SYM(W, N)                                                                                      \
    launch_dep(rpy_sym_f64<W, N>, dim3(h->mv_gridsym), dim3(th), 0, st, h->d_r4, lam, h->d_mv, si, h->n_sym, \
               h->d_item_counter, k, active)
        if (h->cfg.wall) {
            if (h->sym_nsub == 1) AM_SYM(true, 1); else if (h->sym_nsub == 2) AM_SYM(true, 2); else AM_SYM(true, 4);
        } else {
            if (h->sym_nsub == 1) AM_SYM(false, 1); else if (h->sym_nsub == 2) AM_SYM(false, 2); else AM_SYM(false, 4);
        }
#undef AM_SYM
    } else if (fp64) {
        const RpyK<double> k = rpy_consts<double>(h->prm);
        if (h->cfg.wall)
            launch_dep(rpy_items_f64<true>, dim3(h->mv_grid64), dim3(kThreads), 0, st, h->d_r4, lam, h->d_mv, items,
                       h->n_items, h->d_item_counter, k, active);
        else
            launch_dep(rpy_items_f64<false>, dim3(h->mv_grid64), dim3(kThreads), 0, st, h->d_r4, lam, h->d_mv, items,
                       h->n_items, h->d_item_counter, k, active);
    } else if (h->n_sym > 0) {
        const RpyK<float> k = rpy_consts<float>(h->prm);
        const SymItem* si = static_cast<const SymItem*>(h->d_sym_items);
        const int th = h->mv_tpt == 2 || h->sym_nsub > 1 ? kThreads : 32;
#define AM_SYM32(W, N)                                                                                      \
    launch_dep(rpy_sym_mixed<W, N>, dim3(h->mv_gridsym32), dim3(th), 0, st, h->d_rhi, h->d_rlo, lam, h->d_mv, si, \
               h->n_sym, h->d_item_counter, k, active)
#define AM_SYM32X2(W)                                                                                         \
    launch_dep(rpy_sym_mixed_x2<W>, dim3(h->mv_gridsym32), dim3(kThreads), 0, st, h->d_rhi, h->d_rlo, lam, h->d_mv, \
               si, h->n_sym, h->d_item_counter, k, active)
        if (h->cfg.wall) {
            if (h->mv_tpt == 2) AM_SYM32X2(true);
            else if (h->sym_nsub == 1) AM_SYM32(true, 1);
            else if (h->sym_nsub == 2) AM_SYM32(true, 2);
            else AM_SYM32(true, 4);
        } else {
            if (h->mv_tpt == 2) AM_SYM32X2(false);
            else if (h->sym_nsub == 1) AM_SYM32(false, 1);
            else if (h->sym_nsub == 2) AM_SYM32(false, 2);
            else AM_SYM32(false, 4);
        }
#undef AM_SYM32X2
#undef AM_SYM32
    } else {
        const RpyK<float> k = rpy_consts<float>(h->prm);
#define AM_MIXED_ITEMS(W, T)                                                                                 \
    launch_dep(rpy_items_mixed<W, T>, dim3(h->mv_grid), dim3(kThreads), 0, st, h->d_rhi, h->d_rlo, lam, h->d_mv, \
               items, h->n_items, h->d_item_counter, k, active)
#define AM_MIXED_X2(W)                                                                                      \
    launch_dep(rpy_items_mixed_x2<W>, dim3(h->mv_grid), dim3(kThreads), 0, st, h->d_rhi, h->d_rlo, lam, h->d_mv, \
               items, h->n_items, h->d_item_counter, k, active)
        if (h->cfg.wall) {
            if (h->mv_tpt == 2) AM_MIXED_X2(true); else AM_MIXED_ITEMS(true, 1);
        } else {
            if (h->mv_tpt == 2) AM_MIXED_X2(false); else AM_MIXED_ITEMS(false, 1);
        }
#undef AM_MIXED_X2
#undef AM_MIXED_ITEMS
    }
    count_launch();
}

void launch_sum_items(am_handle* h, double* u) {
    if (h->Nb <= 0) return;
    k_sum_items<<<(h->Nb + 255) / 256, 256, 0, h->stream>>>(h->Nb, h->d_mv, h->d_sys_of_blob, h->d_sys_blob0,
                                                            h->d_sys_nb, h->d_sys_nch, h->d_sys_poff, u);
    count_launch();
}

// Autotuner: times the handle's product and the sum of its partials for
// candidate layouts on the current positions and keeps the fastest.
int mobility_autotune(am_handle* h) {
    if (h->per) {  // the periodic product has no item layout to tune
        h->mv_tuned = true;
        return 0;
    }
    struct Cand { int tpt, chunk, tgroup, sym; };
    std::vector<Cand> cand;
    const bool mixed = h->cfg.precision == AM_MIXED;
    long long maxnb = 0;
    for (const auto& r : h->sys) maxnb = std::max<long long>(maxnb, r.Nb);
    for (int tpt : (mixed ? std::vector<int>{1, 2} : std::vector<int>{1}))
        for (int chunk : {0, 512, 1024, 2048, 4096, 8192})
            if (chunk == 0 || chunk <= 2 * maxnb) cand.push_back({tpt, chunk, 0, 0});
    // One system of modest size: the items all start at once, so the
    // slowest SM sets the time; chunks that make the item count a multiple
    // of the SM count (k = 1..6 items per SM) balance the last wave.  Small
    // systems also try items of 32 or 64 targets (one target per thread),
    // which spread a few thousand blobs over all SMs: with 2 FP64 FMAs per
    // SM per cycle one 128 x 128 item of FP64 pairs takes tens of us.
    if (h->S == 1 && maxnb * maxnb <= 4000000000LL) {
        for (int tpt : (mixed ? std::vector<int>{1, 2} : std::vector<int>{1})) {
            for (int tg : {kThreads * tpt, 64, 32}) {
                if (tpt == 2 && tg != kThreads * tpt) continue;
                if (tg != kThreads * tpt && maxnb > 16384) continue;
                const long long ntb = (maxnb + tg - 1) / tg;
                for (int k = 1; k <= 6; ++k) {
                    const long long c = ((long long)k * num_sms() + ntb - 1) / ntb;  // chunks per system
                    const long long chunk = (maxnb + c - 1) / c;
                    if (chunk >= 32) cand.push_back({tpt, (int)chunk, tg == kThreads * tpt ? 0 : tg, 0});
                }
                if (tg != kThreads * tpt) cand.push_back({tpt, 32, tg, 0});
            }
        }
    }
    // The symmetric product: on tiles of 32, 64 and 128 blobs while its
    // partial sums (one slot per tile of the system) stay within 1 GiB (FP64,
    // and mixed with one target per lane); mixed in paired lanes on tiles
    // of 128 while they stay within a quarter of the free device memory
    // (24 GB for 360,000 blobs)
    for (int nsub : {1, 2, 4}) {
        long long slots = 0;
        for (const auto& r : h->sys) slots += (long long)((r.Nb + 32 * nsub - 1) / (32 * nsub)) * 3 * r.Nb;
        if (slots * 8 <= (1LL << 30)) cand.push_back({1, 32 * nsub, 0, nsub});
    }
    if (mixed) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        long long slots = 0;
        for (const auto& r : h->sys) slots += (long long)((r.Nb + 127) / 128) * 3 * r.Nb;
        if ((double)slots * 8.0 <= 0.25 * (double)free_b) cand.push_back({2, 128, 0, 4});
    }
    cudaStream_t st = h->stream;
    double* lam = nullptr;
    if (cudaMalloc(&lam, 6 * (size_t)std::max(h->Nb, 1) * sizeof(double)) != cudaSuccess) return 1;
    cudaMemsetAsync(lam, 0, 6 * (size_t)h->Nb * sizeof(double), st);
    double* usum = lam + 3 * (size_t)std::max(h->Nb, 1);  // the sum of the partials: its cost grows with them
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand pick = cand[0];
    const bool timing = h->timing;
    h->timing = false;
    // per candidate: a warm-up product and sum, timed; a candidate whose
    // warm-up is already 50 % slower than the best (per product) stops there,
    // and products of more than 20 ms are taken from the warm-up alone (large
    // systems, where the candidates cost seconds)
    for (auto c : cand) {
        if (mobility_layout(h, c.tpt, c.chunk, c.tgroup, c.sym)) continue;
        cudaEventRecord(e0, st);
        launch_items(h, lam, false);  // warm-up
        launch_sum_items(h, usum);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) continue;
        float warm = 0.f;
        cudaEventElapsedTime(&warm, e0, e1);
        float ms = warm;
        if (warm < 1.5f * best && warm <= 20.f) {
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < 2; ++rep) {
                launch_items(h, lam, false);
                launch_sum_items(h, usum);
            }
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) continue;
            cudaEventElapsedTime(&ms, e0, e1);
            ms *= 0.5f;
        }
        if (ms < best) { best = ms; pick = c; }
    }
    h->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(lam);
    cudaGetLastError();
    h->mv_tuned = true;
    return mobility_layout(h, pick.tpt, pick.chunk, pick.tgroup, pick.sym);
}

}  // namespace am

// am_rpy_matvec_noalloc: the blob mobility product for callers that cannot
// allocate device memory.  Same kernels and source split as am_rpy_matvec;
// the scratch (packed positions and per-chunk partial sums) is a fixed
// device array of this file instead of a caller workspace.
#include "am_internal.cuh"

#include <string>

namespace am {
void set_thread_error(const std::string& msg);
}

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[AM_NOALLOC_SCRATCH_BYTES];

// errors are reported through am_last_error(NULL), like am_rpy_matvec's
int fail(int code, const std::string& msg) {
    am::set_thread_error(msg);
    return code;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array on the current device.  The host-side
// name of a __device__ array is not a device address, so it is looked up with
// the device current, on every call: the lookup is not a stream operation,
// and a cached address would go stale if the module were loaded again (after
// a device reset, in a new primary context).
int scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(AM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = p;
    return AM_OK;
}

}  // namespace

extern "C" AM_API int am_rpy_matvec_noalloc(const double* d_r, const double* d_lambda, double* d_u,
                                            int n, double eta, double a, int wall, int precision,
                                            void* stream) {
    if (n < 0) return fail(AM_ERR_ARG, "am_rpy_matvec_noalloc: n < 0");
    if (!(eta > 0.0) || !(a > 0.0)) return fail(AM_ERR_ARG, "am_rpy_matvec_noalloc: eta and a must be > 0");
    if (wall != 0 && wall != 1) return fail(AM_ERR_ARG, "am_rpy_matvec_noalloc: wall must be 0 or 1");
    if (precision != AM_FP64 && precision != AM_MIXED)
        return fail(AM_ERR_ARG, "am_rpy_matvec_noalloc: unknown precision");
    if (n == 0) return AM_OK;
    if (!d_r || !d_lambda || !d_u) return fail(AM_ERR_ARG, "am_rpy_matvec_noalloc: NULL pointer");
    const size_t need = am_rpy_matvec_workspace(n, precision);
    if (need > AM_NOALLOC_SCRATCH_BYTES)
        return fail(AM_ERR_ARG, "am_rpy_matvec_noalloc: n = " + std::to_string(n) + " needs " +
                                    std::to_string(need) + " bytes of scratch, more than the " +
                                    std::to_string((size_t)AM_NOALLOC_SCRATCH_BYTES) +
                                    " of the fixed array; use am_rpy_matvec with a workspace");
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    am::Split sp = am::choose_split(n, precision);
    am::RpyParams prm = am::make_params(eta, a);
    char* w = static_cast<char*>(base);
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

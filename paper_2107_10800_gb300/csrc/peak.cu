// FMA throughput probe: the roofline denominator for ALU-bound kernels.
// Every thread runs 8 independent FMA chains so the pipes, not latency,
// bound the rate; the grid covers every SM several times.
#include "am_internal.cuh"

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_streams(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
            x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
        }
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keep the chains live
}

template <class T>
int run(double* flops) {
    const int blocks = am::num_sms() * 8, threads = 256;
    T* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) return AM_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = sizeof(T) == 8 ? 256 : 8192;
    const T a = (T)0.999999, b = (T)1e-7;
    fma_streams<T><<<blocks, threads>>>(out, iters / 8, a, b);  // warm-up
    am::count_launch();
    cudaEventRecord(e0);
    fma_streams<T><<<blocks, threads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    am::count_launch();
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.f) return AM_ERR_CUDA;
    const double fl = 2.0 * 8 * 4 * (double)iters * blocks * threads;
    *flops = fl / (ms * 1e-3);
    return AM_OK;
}

}  // namespace

extern "C" AM_API int am_alu_peak(int fp64, double* flops) {
    if (!flops) return AM_ERR_ARG;
    return fp64 ? run<double>(flops) : run<float>(flops);
}

// One 128-row tile of a dense layer on the 5th-generation tensor cores
// (tcgen05): D = A W^T with A (rows x K) and W (N x K) in BF16, both
// K-major, the FP32 accumulators in tensor memory (TMEM); bias, ReLU and the
// output scaling in the epilogue.  Used for the learned initial guess's
// network (K = 144 or 256, N = 256 or 32).
//
// Shared memory holds the whole tile (no K pipeline: K <= 256), staged by
// 16-byte cp.async copies: A as 128 x K
// and W as N x K in the canonical no-swizzle K-major layout of core matrices
// (8 rows x 16 bytes, stored as 128 contiguous bytes), element (r, k) at
//   ((r / 8) * (K / 8) + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so that the leading-dimension byte offset (between core matrices along K)
// is 128 and the stride byte offset (between 8-row groups) is K / 8 * 128.
// One elected thread issues the K / 16 MMAs (M = 128, N, K = 16 each) and
// commits them to an mbarrier; every warp then reads its 32 TMEM lanes (the
// tile's rows 32 w .. 32 w + 31) with tcgen05.ld.  Waits are bounded: on
// timeout the block sets kFlagTensorTimeout in *flags, stores nothing,
// releases its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace am {
namespace tc {

constexpr int kRows = 128;                  // M of the MMA: rows per tile
constexpr int kFlagTensorTimeout = 1 << 8;  // set in *flags when a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of tcgen05.mma: start address, leading
// and stride byte offsets (all >> 4), descriptor version 1 (bits 46-47), no
// base offset, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits
// 4-5 = 1), A and B in BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15,
// 16 = 0), N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// bytes of dynamic shared memory for a tile of K columns and N outputs
__host__ __device__ constexpr int smem_bytes(int K, int N) { return 2 * K * (kRows + N); }

// TMEM columns to allocate for N accumulator columns (a power of two >= 32)
__device__ __forceinline__ uint32_t tmem_cols(int N) {
    uint32_t c = 32;
    while (c < (uint32_t)N) c <<= 1;
    return c;
}

// Out[r][o] = act(sum_k A[r][k] W[o][k] + b[o]) for the rows of block
// blockIdx.x: BF16 output (Obf) or FP32 output scaled by sdo (Of).  K a
// multiple of 16 (<= 256), N a multiple of 16 (16 .. 256); A and W rows 16-byte
// aligned; blockDim.x == 128.
__global__ void __launch_bounds__(128, 1)
k_linear_tc(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ W,
            const float* __restrict__ b, __nv_bfloat16* __restrict__ Obf, float* __restrict__ Of,
            const float* __restrict__ sdo, int n, int K, int N, int relu, int* flags) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char* sA = smem;
    unsigned char* sB = smem + 2 * kRows * K;
    const int row0 = blockIdx.x * kRows;
    const int kc = K / 8;  // 16-byte chunks of a row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = tmem_cols(N);

    // stage the tile in the core-matrix layout with 16-byte asynchronous
    // copies, all in flight at once (rows beyond n are zero-filled: source
    // size 0, the address of row 0 given but not read)
    for (int idx = threadIdx.x; idx < kRows * kc; idx += blockDim.x) {
        const int r = idx / kc, c = idx % kc;
        const bool in = row0 + r < n;
        const __nv_bfloat16* src = A + (size_t)(in ? row0 + r : 0) * K + 8 * c;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                     ::"r"(smem_u32(sA + ((r >> 3) * kc + c) * 128 + (r & 7) * 16)), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
    }
    for (int idx = threadIdx.x; idx < N * kc; idx += blockDim.x) {
        const int r = idx / kc, c = idx % kc;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                     ::"r"(smem_u32(sB + ((r >> 3) * kc + c) * 128 + (r & 7) * 16)), "l"(W + (size_t)r * K + 8 * c)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the staged tile is read by the tensor cores (async proxy)
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (threadIdx.x == 0) {
        const uint32_t id = idesc_bf16_f32(kRows, N);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB), sbo = (uint32_t)kc * 128u;
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t da = smem_desc(a0 + 256u * s, 128u, sbo);
            const uint64_t db = smem_desc(b0 + 256u * s, 128u, sbo);
            const uint32_t acc = s > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                ::"r"(tmem), "l"(da), "l"(db), "r"(id), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&mbar)) : "memory");
    }
    bool done = false;
    for (int it = 0; it < (1 << 22) && !done; ++it) done = mbar_try_wait(smem_u32(&mbar), 0u);
    if (!done && threadIdx.x == 0) atomicOr(flags, kFlagTensorTimeout);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const int r = row0 + warp * 32 + lane;
    for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
              "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (done && r < n) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int o = c0 + j;
                float x = __uint_as_float(v[j]) + b[o];
                if (relu) x = fmaxf(x, 0.f);
                if (Of) Of[(size_t)r * N + o] = sdo ? x * sdo[o] : x;
                else Obf[(size_t)r * N + o] = __float2bfloat16(x);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace tc
}  // namespace am

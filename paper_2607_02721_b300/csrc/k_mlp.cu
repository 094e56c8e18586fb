// Tensor-core (tcgen05) kernels of the surrogate sensitivity model.  This file holds
// the GEMM self-check used to validate the descriptor encodings on the device.
#include "csgs_internal.cuh"
#include "tc_gemm.cuh"

namespace csgs {
namespace {

constexpr long long kWaitBudget = 2000000000LL;  // ~1 s at 2 GHz; a wait beyond it is an error

// C[128 x N] = A[128 x K] * B[N x K]^T, BF16 in, FP32 out; one CTA of 128 threads
// (one warpgroup, so warp w reads TMEM lanes 32w..32w+31).  K % 16 == 0, K <= 128,
// N % 16 == 0, 16 <= N <= 256.
__global__ void __launch_bounds__(128) k_gemm_check(const __nv_bfloat16* __restrict__ A,
                                                    const __nv_bfloat16* __restrict__ B, float* __restrict__ C,
                                                    int K, int N, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // operand tiles start on a 1024-byte boundary
    unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sA = smem;
    unsigned char* sB = smem + 128 * K * 2;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // stage A (row tid) and B (rows tid, tid + 128) in the K-major core-matrix layout
    for (int k8 = 0; k8 < K / 8; ++k8) {
        const uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)tid * K + k8 * 8);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_off(tid, k8 * 8, K)) = v;
    }
    for (int r = tid; r < N; r += 128)
        for (int k8 = 0; k8 < K / 8; ++k8) {
            const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)r * K + k8 * 8);
            *reinterpret_cast<uint4*>(sB + tc::kmajor_off(r, k8 * 8, K)) = v;
        }
    tc::fence_smem_to_async();
    if (warp == 0) tc::tmem_alloc(&slot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = slot;
    if (tid == 0) {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, sbo);
            const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, sbo);
            tc::mma(taddr, ad, bd, tc::idesc_bf16(128, (uint32_t)N), kk > 0 ? 1u : 0u);
        }
        tc::commit(&bar);
    }
    bool ok = tc::mbar_wait(&bar, 0, kWaitBudget);
    if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(err, 1);
        tc::mbar_wait(&bar, 0, kWaitBudget);  // let an in-flight MMA drain before freeing TMEM
    } else {
        tc::fence_after_sync();
        const int row = warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) C[(size_t)row * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 256);
}

}  // namespace

int gemm_check(const void* A, const void* B, float* C, int K, int N, int* d_err, cudaStream_t st) {
    const size_t smem = (size_t)128 * K * 2 + (size_t)N * K * 2 + 1024;
    cudaFuncSetAttribute(k_gemm_check, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gemm_check<<<1, 128, smem, st>>>(reinterpret_cast<const __nv_bfloat16*>(A),
                                       reinterpret_cast<const __nv_bfloat16*>(B), C, K, N, d_err);
    count_launches(1);
    return 0;
}

}  // namespace csgs

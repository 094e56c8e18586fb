// Tensor-core (tcgen05) kernels of the surrogate sensitivity model.  This file holds
// the GEMM self-check used to validate the descriptor encodings on the device.
#include "csgs_internal.cuh"
#include "tc_gemm.cuh"

namespace csgs {
namespace {

constexpr long long kWaitBudget = 2000000000LL;  // ~1 s at 2 GHz; a wait beyond it is an error

// C[128 x N] = A[128 x K] * B[N x K]^T, BF16 in, FP32 out; one CTA of 128 threads
// (one warpgroup, so warp w reads TMEM lanes 32w..32w+31).  K % 16 == 0, K <= 128,
// N % 16 == 0, 16 <= N <= 256.  first_wait: clock cycles the threads wait for the MMA
// chain's completion (0: one non-blocking test); a warp that gives up sets *err and then
// waits the full budget for the chain to drain, so no MMA is in flight when the tensor
// memory is freed.  mn_major: A is given as [K][128] and B as [K][N] (C = A^T B) and both
// are staged in the MN-major layout.
__global__ void __launch_bounds__(128) k_gemm_check(const __nv_bfloat16* __restrict__ A,
                                                    const __nv_bfloat16* __restrict__ B, float* __restrict__ C,
                                                    int K, int N, int* err, long long first_wait, int mn_major) {
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
    if (!mn_major) {
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
    } else {
        // 16-byte runs of 8 consecutive m (n) at one k, copied as they are
        for (int c = tid; c < K * 16; c += 128) {
            const int k = c >> 4, m8 = c & 15;
            const uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)k * 128 + m8 * 8);
            *reinterpret_cast<uint4*>(sA + tc::mnmajor_off(m8 * 8, k, 128)) = v;
        }
        for (int c = tid; c < K * (N / 8); c += 128) {
            const int k = c / (N / 8), n8 = c % (N / 8);
            const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)k * N + n8 * 8);
            *reinterpret_cast<uint4*>(sB + tc::mnmajor_off(n8 * 8, k, N)) = v;
        }
    }
    tc::fence_smem_to_async();
    if (warp == 0) tc::tmem_alloc(&slot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = slot;
    if (tid == 0) {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        if (!mn_major) {
            const uint32_t sbo = (uint32_t)(K / 8) * 128u;
            for (int kk = 0; kk < K / 16; ++kk) {
                const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, sbo);
                const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, sbo);
                tc::mma(taddr, ad, bd, tc::idesc_bf16(128, (uint32_t)N), kk > 0 ? 1u : 0u);
            }
        } else {
            // K-direction core-matrix strides (LBO); M/N-direction 128 bytes (SBO); each MMA
            // takes two K-groups
            const uint32_t la = 16u * 128u, lb = (uint32_t)(N / 8) * 128u;
            for (int kk = 0; kk < K / 16; ++kk) {
                const uint64_t ad = tc::smem_desc(a0 + kk * 2 * la, la, 128);
                const uint64_t bd = tc::smem_desc(b0 + kk * 2 * lb, lb, 128);
                tc::mma(taddr, ad, bd, tc::idesc_bf16_mn(128, (uint32_t)N), kk > 0 ? 1u : 0u);
            }
        }
        tc::commit(&bar);
    }
    bool ok = first_wait > 0 ? tc::mbar_wait(&bar, 0, first_wait) : tc::mbar_test(&bar, 0);
    if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(err, 1);
        // let an in-flight MMA drain before freeing TMEM
        if (!tc::mbar_wait(&bar, 0, kWaitBudget) && lane == 0) atomicOr(err, 2);
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

int gemm_check(const void* A, const void* B, float* C, int K, int N, int* d_err, long long first_wait, int mn_major,
               cudaStream_t st) {
    // the MN-major check takes the largest allocation, so that the tensor core's reads stay
    // inside the CTA's shared memory for any reading of the descriptor's two strides
    const size_t smem = mn_major ? (size_t)226 * 1024 : (size_t)128 * K * 2 + (size_t)N * K * 2 + 1024;
    cudaFuncSetAttribute(k_gemm_check, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gemm_check<<<1, 128, smem, st>>>(reinterpret_cast<const __nv_bfloat16*>(A),
                                       reinterpret_cast<const __nv_bfloat16*>(B), C, K, N, d_err,
                                       first_wait < 0 ? kWaitBudget : first_wait, mn_major);
    count_launches(1);
    return 0;
}

}  // namespace csgs

// ======================================================================= surrogate MLP
// x (64 features) -> 256 (GELU) -> 256 (GELU) -> 1, BF16 operands, FP32 accumulation in
// tensor memory.  Parameter block (FP32 master copy, same order as the host API):
// W1[256][64], b1[256], W2[256][256], b2[256], w3[256], b3.  BF16 copies W1b, W2b and the
// transpose W2Tb feed the tensor cores.
namespace csgs {
namespace {

constexpr int kIn = 64, kH = 256;
constexpr int kRows = 128;            // rows per tile (MMA M)
constexpr uint32_t kIdesc1 = tc::idesc_bf16(128, 256);

// erf by Abramowitz & Stegun, Handbook of Mathematical Functions, formula 7.1.26:
// erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2), t = 1 / (1 + p x),
// x >= 0, |error| <= 1.5e-7 (odd extension for x < 0); the reciprocal and the
// exponential use the hardware approximations (relative error ~2^-22).
__device__ __forceinline__ float ex2_fast(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float erf_as(float x) {
    const float ax = fabsf(x);
    const float t = rcp_fast(fmaf(0.3275911f, ax, 1.f));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    poly *= t;
    const float e = ex2_fast(-ax * ax * 1.4426950408889634f);
    return copysignf(fmaf(-poly, e, 1.f), x);
}
// GELU(z) = z Phi(z) = 0.5 z (1 + erf(z / sqrt 2)); GELU'(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erf_as(z * 0.70710678118654752f)); }

// Two FP32 values in one 64-bit register for the packed instructions (fma / mul / add
// .rn.f32x2): each half is rounded exactly as the scalar instruction would round it.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2c(float a) { return f2(a, a); }
__device__ __forceinline__ void f2split(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// gelu() of two values with the packed instructions, bit for bit the scalar result: the
// same operations in the same order, except that the polynomial is carried negated (all
// its coefficients negated: negation is exact, so -poly comes out exactly) and
// (-|x|) |x| log2 e is formed as (x x)(-log2 e) (the same product).
__device__ __forceinline__ f32x2 gelu2(f32x2 z) {
    const f32x2 x = mul2(z, f2c(0.70710678118654752f));
    float x0, x1;
    f2split(x, x0, x1);
    float d0, d1;
    f2split(fma2(f2c(0.3275911f), f2(fabsf(x0), fabsf(x1)), f2c(1.f)), d0, d1);
    const f32x2 t = f2(rcp_fast(d0), rcp_fast(d1));
    f32x2 np = fma2(t, f2c(-1.061405429f), f2c(1.453152027f));
    np = fma2(t, np, f2c(-1.421413741f));
    np = fma2(t, np, f2c(0.284496736f));
    np = fma2(t, np, f2c(-0.254829592f));
    np = mul2(np, t);
    float a0, a1;
    f2split(mul2(mul2(x, x), f2c(-1.4426950408889634f)), a0, a1);
    float r0, r1;
    f2split(fma2(np, f2(ex2_fast(a0), ex2_fast(a1)), f2c(1.f)), r0, r1);
    const f32x2 onep = add2(f2c(1.f), f2(copysignf(r0, x0), copysignf(r1, x1)));
    return mul2(mul2(f2c(0.5f), z), onep);
}
// GELU and its derivative from one reciprocal and one exponential: with x = z / sqrt 2,
// erf's factor exp(-x^2) = exp(-z^2 / 2) is also sqrt(2 pi) phi(z).  g is gelu(z) bit for
// bit (the same operations); gd = Phi(z) + z phi(z).
__device__ __forceinline__ void gelu_both(float z, float& g, float& gd) {
    const float x = z * 0.70710678118654752f;
    const float ax = fabsf(x);
    const float t = rcp_fast(fmaf(0.3275911f, ax, 1.f));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    poly *= t;
    const float e = ex2_fast(-ax * ax * 1.4426950408889634f);
    const float er = copysignf(fmaf(-poly, e, 1.f), x);
    g = 0.5f * z * (1.f + er);
    gd = fmaf(0.5f, er, 0.5f) + z * e * 0.39894228040143268f;
}
__device__ __forceinline__ float gelu_d(float z) {
    float g, gd;
    gelu_both(z, g, gd);
    return gd;
}

// gelu_both() of two values with the packed instructions, bit for bit the scalar results
// (the operations of gelu2, then gd as in gelu_both).
__device__ __forceinline__ void gelu2_both(f32x2 z, f32x2& g, f32x2& gd) {
    const f32x2 x = mul2(z, f2c(0.70710678118654752f));
    float x0, x1;
    f2split(x, x0, x1);
    float d0, d1;
    f2split(fma2(f2c(0.3275911f), f2(fabsf(x0), fabsf(x1)), f2c(1.f)), d0, d1);
    const f32x2 t = f2(rcp_fast(d0), rcp_fast(d1));
    f32x2 np = fma2(t, f2c(-1.061405429f), f2c(1.453152027f));
    np = fma2(t, np, f2c(-1.421413741f));
    np = fma2(t, np, f2c(0.284496736f));
    np = fma2(t, np, f2c(-0.254829592f));
    np = mul2(np, t);
    float a0, a1;
    f2split(mul2(mul2(x, x), f2c(-1.4426950408889634f)), a0, a1);
    const f32x2 e = f2(ex2_fast(a0), ex2_fast(a1));
    float r0, r1;
    f2split(fma2(np, e, f2c(1.f)), r0, r1);
    const f32x2 er = f2(copysignf(r0, x0), copysignf(r1, x1));
    g = mul2(mul2(f2c(0.5f), z), add2(f2c(1.f), er));
    gd = add2(fma2(f2c(0.5f), er, f2c(0.5f)), mul2(mul2(z, e), f2c(0.39894228040143268f)));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

struct MlpDev {
    const __nv_bfloat16* W1b;
    const __nv_bfloat16* W2b;
    const __nv_bfloat16* W2Tb;
    const float* b1;
    const float* b2;
    const float* w3;
    const float* b3;
};

// stage_rows with asynchronous 16-byte copies (cp.async, no register round trip; rows
// beyond nrows are zero-filled without a read).  Completed by stage_rows_wait().
__device__ __forceinline__ void stage_rows_async(unsigned char* dst, const __nv_bfloat16* src, int r0, int nrows,
                                                 int R, int K, int ld) {
    const int chunks = R * (K / 8);
    for (int idx = threadIdx.x; idx < chunks; idx += blockDim.x) {
        const int r = idx / (K / 8), k8 = idx % (K / 8);
        const bool in = r0 + r < nrows;
        const __nv_bfloat16* g = src + (size_t)(in ? r0 + r : r0) * ld + k8 * 8;
        const uint32_t s = tc::smem_u32(dst + tc::kmajor_off(r, k8 * 8, K));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(g), "r"(in ? 16 : 0) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_rows_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage an R x K row-major BF16 matrix (rows r0.., zero beyond nrows) into the K-major
// core-matrix layout, 16 bytes per thread step.
__device__ __forceinline__ void stage_rows(unsigned char* dst, const __nv_bfloat16* src, int r0, int nrows, int R,
                                           int K, int ld) {
    const int chunks = R * (K / 8);
    for (int idx = threadIdx.x; idx < chunks; idx += blockDim.x) {
        const int r = idx / (K / 8), k8 = idx % (K / 8);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r0 + r < nrows) v = *reinterpret_cast<const uint4*>(src + (size_t)(r0 + r) * ld + k8 * 8);
        *reinterpret_cast<uint4*>(dst + tc::kmajor_off(r, k8 * 8, K)) = v;
    }
}

// issue M=128 MMAs over K (K-major tiles a, b), commit to bar
__device__ __forceinline__ void mma_tile(uint32_t d, const unsigned char* a, const unsigned char* b, int K,
                                         uint32_t idesc, bool accumulate_first, uint64_t* bar) {
    const uint32_t a0 = tc::smem_u32(a), b0 = tc::smem_u32(b), sbo = (uint32_t)(K / 8) * 128u;
    for (int kk = 0; kk < K / 16; ++kk)
        tc::mma(d, tc::smem_desc(a0 + kk * 256, 128, sbo), tc::smem_desc(b0 + kk * 256, 128, sbo), idesc,
                (kk > 0 || accumulate_first) ? 1u : 0u);
    tc::commit(bar);
}

__device__ __forceinline__ unsigned char* align1k(unsigned char* p) {
    return p + ((1024u - (tc::smem_u32(p) & 1023u)) & 1023u);
}

// Forward, persistent over 128-row tiles with the weights resident in shared memory
// (W1 32 KB + W2 128 KB, staged once per CTA), an X tile (16 KB) and one 128-column
// K-chunk of the first hidden layer (32 KB).  Per tile:
//   layer 1: X W1^T -> TMEM columns [0, 256)
//   epilogue 1, columns [0, 128) -> H chunk; layer 2, K = 0..127 -> TMEM [256, 512)
//   epilogue 1, columns [128, 256) -> H chunk (after the first half has been read);
//   layer 2, K = 128..255 (accumulate); the next tile's X is staged meanwhile
//   layer 1 of the next tile is issued before epilogue 2 (it writes columns [0, 256),
//   which epilogue 1 has finished reading), so it runs under epilogue 2
//   epilogue 2: y = w3 . GELU(z2 + b2) + b3.
constexpr int kHc = 128;  // K-chunk of the hidden layer held in shared memory

__device__ __forceinline__ void mma_tile_k(uint32_t d, const unsigned char* a, int Ka, const unsigned char* b, int Kb,
                                           int k0, int nk, uint32_t idesc, bool accumulate_first, uint64_t* bar) {
    // A: K-major tile with Ka columns (starting at its column 0); B: K-major with Kb columns, from column k0
    const uint32_t a0 = tc::smem_u32(a), b0 = tc::smem_u32(b) + (uint32_t)(k0 / 8) * 128u;
    const uint32_t sboa = (uint32_t)(Ka / 8) * 128u, sbob = (uint32_t)(Kb / 8) * 128u;
    for (int kk = 0; kk < nk / 16; ++kk)
        tc::mma(d, tc::smem_desc(a0 + kk * 256, 128, sboa), tc::smem_desc(b0 + kk * 256, 128, sbob), idesc,
                (kk > 0 || accumulate_first) ? 1u : 0u);
    tc::commit(bar);
}

// 512 threads: warp w reads TMEM lanes 32 (w % 4).. and handles column quarter w / 4.
// TRAIN additionally stores GELU'(z1) (FP32), h1 (BF16) and dz2 = d loss / d z2 (BF16) per row
// (loss = mean (y - t)^2 over the B rows) and accumulates d/dw3, d/db3 and the loss.
template <bool TRAIN>
__global__ void __launch_bounds__(512, 1) k_mlp_fwd2(const __nv_bfloat16* __restrict__ X, int B, MlpDev p,
                                                     float* __restrict__ y, const float* __restrict__ t,
                                                     float* __restrict__ gd1o, __nv_bfloat16* __restrict__ h1o,
                                                     __nv_bfloat16* __restrict__ dz2o, float* __restrict__ gw3,
                                                     float* __restrict__ gb3, float* __restrict__ loss, float inv_B,
                                                     int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = align1k(smem_raw);
    unsigned char* sW1 = sm;                         // 256 x 64
    unsigned char* sW2 = sW1 + kH * kIn * 2;         // 256 x 256
    unsigned char* sX = sW2 + kH * kH * 2;           // 128 x 64
    unsigned char* sH = sX + kRows * kIn * 2;        // 128 x 128
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    __shared__ float sdot[4][kRows];
    __shared__ float sgw3[kH];
    __shared__ __align__(16) float sb1[kH], sb2[kH], sw3[kH];  // biases and output weights, read every tile
    __shared__ float sred[2][16];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, qt = warp >> 2, row = q * 32 + lane;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (TRAIN && tid < kH) sgw3[tid] = 0.f;
    if (tid < kH) {
        sb1[tid] = p.b1[tid];
        sb2[tid] = p.b2[tid];
        sw3[tid] = p.w3[tid];
    }
    if (warp == 0) tc::tmem_alloc(&slot, 512);
    stage_rows(sW1, p.W1b, 0, kH, kH, kIn, kIn);
    stage_rows(sW2, p.W2b, 0, kH, kH, kH, kH);
    const int ntiles = (B + kRows - 1) / kRows;
    int tile = blockIdx.x;
    if (tile < ntiles) stage_rows(sX, X, tile * kRows, B, kRows, kIn, kIn);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = slot;
    const uint32_t tl = taddr + ((uint32_t)(q * 32) << 16);
    uint32_t phase = 0;
    bool failed = false;
    float lsum = 0.f, db3 = 0.f;
    if (tile < ntiles && tid == 0) mma_tile_k(taddr, sX, kIn, sW1, kIn, 0, kIn, kIdesc1, false, &bar);
    for (; tile < ntiles; tile += gridDim.x) {
        const int r0 = tile * kRows;
        const bool valid = r0 + row < B;
        bool ok = tc::mbar_wait(&bar, phase, kWaitBudget);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
        // layer 1 has read the X tile: fetch the next one under the epilogues
        const int next = tile + gridDim.x;
        if (next < ntiles) stage_rows_async(sX, X, next * kRows, B, kRows, kIn, kIn);
        for (int h = 0; h < 2; ++h) {
            const int c_base = h * kHc;
            if (h == 1) {
                // the first K-chunk must have been consumed before the H buffer is rewritten
                ok = tc::mbar_wait(&bar, phase, kWaitBudget);
                phase ^= 1u;
                if (!__syncthreads_and(ok)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
            }
#pragma unroll
            for (int c = qt * 32; c < qt * 32 + 32; c += 16) {
                float v[16];
                tc::tmem_ld16(tl + (uint32_t)(c_base + c), v);
                const float4* b4 = reinterpret_cast<const float4*>(sb1 + c_base + c);
                f32x2 z[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 b = b4[i];
                    z[2 * i] = add2(f2(v[4 * i], v[4 * i + 1]), f2(b.x, b.y));
                    z[2 * i + 1] = add2(f2(v[4 * i + 2], v[4 * i + 3]), f2(b.z, b.w));
                }
                uint32_t pk[8];
                if (TRAIN) {
                    // GELU'(z1) for the backward, from the same reciprocal and exponential
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        f32x2 g, gd;
                        gelu2_both(z[i], g, gd);
                        float g0, g1;
                        f2split(g, g0, g1);
                        pk[i] = pack_bf16(g0, g1);
                        f2split(gd, v[2 * i], v[2 * i + 1]);
                    }
                    if (valid) {
                        float4* go = reinterpret_cast<float4*>(gd1o + (size_t)(r0 + row) * kH + c_base + c);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            go[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float g0, g1;
                        f2split(gelu2(z[i]), g0, g1);
                        pk[i] = pack_bf16(g0, g1);
                    }
                }
                *reinterpret_cast<uint4*>(sH + tc::kmajor_off(row, c, kHc)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4*>(sH + tc::kmajor_off(row, c + 8, kHc)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                if (TRAIN && valid) {
                    uint4* ho = reinterpret_cast<uint4*>(h1o + (size_t)(r0 + row) * kH + c_base + c);
                    ho[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    ho[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
            tc::fence_smem_to_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) mma_tile_k(taddr + 256u, sH, kHc, sW2, kH, c_base, kHc, kIdesc1, h == 1, &bar);
        }
        if (failed) break;
        stage_rows_wait();
        tc::fence_smem_to_async();
        ok = tc::mbar_wait(&bar, phase, kWaitBudget);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
        if (next < ntiles && tid == 0) mma_tile_k(taddr, sX, kIn, sW1, kIn, 0, kIn, kIdesc1, false, &bar);
        float part = 0.f;
#pragma unroll
        for (int c0 = qt * 64; c0 < qt * 64 + 64; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tl + 256u + (uint32_t)c0, v);
            const float4* b4 = reinterpret_cast<const float4*>(sb2 + c0);
            const float4* w4 = reinterpret_cast<const float4*>(sw3 + c0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 b = b4[i], w = w4[i];
                float g0, g1, g2, g3;
                f2split(gelu2(add2(f2(v[4 * i], v[4 * i + 1]), f2(b.x, b.y))), g0, g1);
                f2split(gelu2(add2(f2(v[4 * i + 2], v[4 * i + 3]), f2(b.z, b.w))), g2, g3);
                part = fmaf(w.x, g0, part);
                part = fmaf(w.y, g1, part);
                part = fmaf(w.z, g2, part);
                part = fmaf(w.w, g3, part);
            }
        }
        sdot[qt][row] = part;
        __syncthreads();
        const float yr = (sdot[0][row] + sdot[1][row]) + (sdot[2][row] + sdot[3][row]) + p.b3[0];
        if (qt == 0 && valid) y[r0 + row] = yr;
        if (TRAIN) {
            const float e = valid ? yr - t[r0 + row] : 0.f;
            const float dy = 2.f * e * inv_B;
            if (qt == 0) {
                lsum += e * e * inv_B;
                db3 += dy;
            }
#pragma unroll
            for (int c0 = qt * 64; c0 < qt * 64 + 64; c0 += 16) {
                float v[16], g[16];
                tc::tmem_ld16(tl + 256u + (uint32_t)c0, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float ge, gd;
                    gelu_both(v[i] + sb2[c0 + i], ge, gd);
                    g[i] = dy * ge;  // this row's d loss / d w3
                    v[i] = dy * sw3[c0 + i] * gd;
                }
                const float cs = warp_colsum16(g, lane);
                if ((lane & 1) == 0) {
                    const int col = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
                    atomicAdd(&sgw3[c0 + col], cs);
                }
                if (valid) {
                    uint32_t pk[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) pk[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
                    uint4* o = reinterpret_cast<uint4*>(dz2o + (size_t)(r0 + row) * kH + c0);
                    o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    stage_rows_wait();  // no copy into shared memory outstanding at exit
    if (failed && tid == 0) atomicOr(err, 1);
    if (failed) tc::mbar_wait(&bar, phase, kWaitBudget);  // drain before freeing TMEM
    if (TRAIN) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            db3 += __shfl_xor_sync(0xffffffffu, db3, o);
        }
        __syncthreads();
        if (lane == 0) {
            sred[0][warp] = lsum;
            sred[1][warp] = db3;
        }
        __syncthreads();
        if (tid == 0) {
            float l = 0.f, d = 0.f;
            for (int w = 0; w < 16; ++w) {
                l += sred[0][w];
                d += sred[1][w];
            }
            atomicAdd(loss, l);
            atomicAdd(gb3, d);
        }
        if (tid < kH) atomicAdd(&gw3[tid], sgw3[tid]);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

// dz1 = (dz2 W2) * GELU'(z1) (GELU'(z1) stored by the training forward), BF16 out; smem
// A = dz2 tile (64 KB), B = W2^T (128 KB,
// resident).  512 threads: warp w reads TMEM lanes 32 (w % 4).. and handles column
// quarter w / 4; the next tile's dz2 rows are loaded into registers while the tensor
// core works on the current one.
__global__ void __launch_bounds__(512, 1) k_mlp_dh1(const __nv_bfloat16* __restrict__ dz2, const float* __restrict__ gd1,
                                                    int B, MlpDev p, __nv_bfloat16* __restrict__ dz1, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = align1k(smem_raw);
    unsigned char* sA = sm;
    unsigned char* sB = sm + kRows * kH * 2;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, qt = warp >> 2, row = q * 32 + lane;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&slot, 256);
    stage_rows(sB, p.W2Tb, 0, kH, kH, kH, kH);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = slot, tl = taddr + ((uint32_t)(q * 32) << 16);
    uint32_t phase = 0;
    bool failed = false;
    const int ntiles = (B + kRows - 1) / kRows;
    // thread t holds 16-byte chunks t, t + 512, ... of a tile (128 rows x 32 chunks)
    constexpr int kChunks = kRows * (kH / 8) / 512;
    uint4 pre[kChunks];
    auto load_tile = [&](int r0) {
#pragma unroll
        for (int k = 0; k < kChunks; ++k) {
            const int idx = tid + k * 512, r = idx / (kH / 8), k8 = idx % (kH / 8);
            pre[k] = r0 + r < B ? *reinterpret_cast<const uint4*>(dz2 + (size_t)(r0 + r) * kH + k8 * 8)
                                : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    if (blockIdx.x < ntiles) load_tile(blockIdx.x * kRows);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int r0 = tile * kRows;
#pragma unroll
        for (int k = 0; k < kChunks; ++k) {
            const int idx = tid + k * 512, r = idx / (kH / 8), k8 = idx % (kH / 8);
            *reinterpret_cast<uint4*>(sA + tc::kmajor_off(r, k8 * 8, kH)) = pre[k];
        }
        tc::fence_smem_to_async();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) mma_tile(taddr, sA, sB, kH, kIdesc1, false, &bar);
        const int next = tile + gridDim.x;
        if (next < ntiles) load_tile(next * kRows);
        const bool valid = r0 + row < B;
        // this row's GELU'(z1) for the first two 16-column chunks, loaded under the MMA; each
        // later chunk's is loaded two chunks ahead into the registers the chunk before freed
        const float4* grow = reinterpret_cast<const float4*>(gd1 + (size_t)(r0 + row) * kH + qt * 64);
        float4 gq[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) gq[i] = valid ? grow[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool ok = tc::mbar_wait(&bar, phase, kWaitBudget);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            const int c0 = qt * 64 + ch * 16;
            float v[16];
            tc::tmem_ld16(tl + (uint32_t)c0, v);
            float gd[16];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 f = gq[(ch & 1) * 4 + i];
                gd[4 * i] = f.x;
                gd[4 * i + 1] = f.y;
                gd[4 * i + 2] = f.z;
                gd[4 * i + 3] = f.w;
            }
            if (ch < 2) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    gq[(ch & 1) * 4 + i] = valid ? grow[(ch + 2) * 4 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (valid) {
                uint32_t pk[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) pk[i] = pack_bf16(v[2 * i] * gd[2 * i], v[2 * i + 1] * gd[2 * i + 1]);
                uint4* o = reinterpret_cast<uint4*>(dz1 + (size_t)(r0 + row) * kH + c0);
                o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (failed && tid == 0) atomicOr(err, 1);
    if (failed) tc::mbar_wait(&bar, phase, kWaitBudget);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 256);
}

// Weight gradient of one layer over the CTA's rows, split-K by rows: part[cta] = dz^T act
// for the 128 outputs of block blockIdx.y, and the bias gradient sum_rows dz (atomics).
// Both operands are MN-major in shared memory (outputs resp. inputs contiguous, one row
// per k), so a 16-byte run of a dz or act row is copied as it is; thread t always stages
// the same 8 outputs (t % 16) of A, which gives it the bias sums from its registers.  The
// next 128-row chunk is loaded into registers while the tensor core works on the current.
template <int NIN>
__global__ void __launch_bounds__(256) k_mlp_wgrad(const __nv_bfloat16* __restrict__ dz,
                                                   const __nv_bfloat16* __restrict__ act, int B, int rows_per_cta,
                                                   float* __restrict__ part, float* __restrict__ gb, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = align1k(smem_raw);
    unsigned char* sA = sm;                  // MN-major, 128 outs x 128 rows
    unsigned char* sB = sm + 128 * 128 * 2;  // MN-major, NIN ins x 128 rows
    constexpr int kCA = 128 * 16 / 256;      // 16-byte runs of A per thread and chunk (8)
    constexpr int kCB = 128 * (NIN / 8) / 256;  // of B (16 or 4)
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    __shared__ float sbias[8][128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ob = blockIdx.y;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&slot, NIN < 32 ? 32 : NIN);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = slot;
    uint32_t phase = 0;
    bool failed = false;
    float bs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int rbeg = blockIdx.x * rows_per_cta;
    const int rend = min(B, rbeg + rows_per_cta);
    const int o8 = tid & 15;  // this thread's 8 outputs of A: o8 * 8 ..
    uint4 ra[kCA], rb[kCB];
    auto load = [&](int r0) {
#pragma unroll
        for (int j = 0; j < kCA; ++j) {
            const int row = (tid >> 4) + 16 * j;
            ra[j] = r0 + row < rend
                        ? *reinterpret_cast<const uint4*>(dz + (size_t)(r0 + row) * kH + ob * 128 + o8 * 8)
                        : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < kCB; ++j) {
            const int c = tid + 256 * j, row = c / (NIN / 8), i8 = c % (NIN / 8);
            rb[j] = r0 + row < rend ? *reinterpret_cast<const uint4*>(act + (size_t)(r0 + row) * NIN + i8 * 8)
                                    : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    if (rbeg < rend) load(rbeg);
    // K-direction core-matrix strides of the two operands; M/N-direction 128 bytes
    constexpr uint32_t la = 16u * 128u, lb = (uint32_t)(NIN / 8) * 128u;
    int chunk = 0;
    for (int r0 = rbeg; r0 < rend; r0 += 128, ++chunk) {
#pragma unroll
        for (int j = 0; j < kCA; ++j) {
            const int row = (tid >> 4) + 16 * j;
            *reinterpret_cast<uint4*>(sA + tc::mnmajor_off(o8 * 8, row, 128)) = ra[j];
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&ra[j]);
#pragma unroll
            for (int i = 0; i < 8; ++i) bs[i] += __bfloat162float(e[i]);
        }
#pragma unroll
        for (int j = 0; j < kCB; ++j) {
            const int c = tid + 256 * j, row = c / (NIN / 8), i8 = c % (NIN / 8);
            *reinterpret_cast<uint4*>(sB + tc::mnmajor_off(i8 * 8, row, NIN)) = rb[j];
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
            for (int kk = 0; kk < 8; ++kk)
                tc::mma(taddr, tc::smem_desc(a0 + kk * 2 * la, la, 128), tc::smem_desc(b0 + kk * 2 * lb, lb, 128),
                        tc::idesc_bf16_mn(128, NIN), (kk > 0 || chunk > 0) ? 1u : 0u);
            tc::commit(&bar);
        }
        if (r0 + 128 < rend) load(r0 + 128);
        const bool ok = tc::mbar_wait(&bar, phase, kWaitBudget);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
    }
    if (failed) {
        if (tid == 0) atomicOr(err, 1);
        tc::mbar_wait(&bar, phase, kWaitBudget);
    } else if (chunk == 0) {
        float* dst = part + (size_t)blockIdx.x * kH * NIN + (size_t)ob * 128 * NIN;
        for (int i = tid; i < 128 * NIN; i += 256) dst[i] = 0.f;
    } else {
        if (warp < 4) {
            const int o = warp * 32 + lane;
            const uint32_t tl = taddr + ((uint32_t)(warp * 32) << 16);
            float* dst = part + (size_t)blockIdx.x * kH * NIN + (size_t)(ob * 128 + o) * NIN;
            for (int c0 = 0; c0 < NIN; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tl + (uint32_t)c0, v);
                float4* d4 = reinterpret_cast<float4*>(dst + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        }
        // bias: lanes l and l ^ 16 hold the same outputs; then the 8 warps' sums
#pragma unroll
        for (int i = 0; i < 8; ++i) bs[i] += __shfl_xor_sync(0xffffffffu, bs[i], 16);
        if (lane < 16)
#pragma unroll
            for (int i = 0; i < 8; ++i) sbias[warp][o8 * 8 + i] = bs[i];
        __syncthreads();
        if (tid < 128) {
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < 8; ++w) s += sbias[w][tid];
            atomicAdd(gb + ob * 128 + tid, s);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, NIN < 32 ? 32 : NIN);
}

// Adam on parameter i of the FP32 master block with gradient g; refreshes its BF16 copies.
__device__ __forceinline__ void adam_one(int i, float g, float* __restrict__ P, float* __restrict__ m,
                                         float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                                         float c2, __nv_bfloat16* __restrict__ W1b, __nv_bfloat16* __restrict__ W2b,
                                         __nv_bfloat16* __restrict__ W2Tb) {
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float pi = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    P[i] = pi;
    const int nW1 = kH * kIn, oW2 = nW1 + kH, nW2 = kH * kH;
    if (i < nW1) W1b[i] = __float2bfloat16_rn(pi);
    if (i >= oW2 && i < oW2 + nW2) {
        const int j = i - oW2, o = j / kH, k = j % kH;
        W2b[j] = __float2bfloat16_rn(pi);
        W2Tb[k * kH + o] = __float2bfloat16_rn(pi);
    }
}

// One kernel for the end of a training step: the weight gradients summed over the split-K
// partials in split order (as k_sum_partials does), the bias and output-weight gradients
// read from their accumulators in G and cleared for the next step, and Adam.
__global__ void k_mlp_sum_adam(const float* __restrict__ part2, const float* __restrict__ part1, int splits,
                               float* __restrict__ G, float* __restrict__ P, float* __restrict__ m,
                               float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                               __nv_bfloat16* __restrict__ W1b, __nv_bfloat16* __restrict__ W2b,
                               __nv_bfloat16* __restrict__ W2Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const int nW1 = kH * kIn, oW2 = nW1 + kH, nW2 = kH * kH;
    float g;
    if (i < nW1) {
        g = 0.f;
        for (int s = 0; s < splits; ++s) g += part1[(size_t)s * nW1 + i];
    } else if (i >= oW2 && i < oW2 + nW2) {
        g = 0.f;
        for (int s = 0; s < splits; ++s) g += part2[(size_t)s * nW2 + (i - oW2)];
    } else {
        g = G[i];
        G[i] = 0.f;
    }
    adam_one(i, g, P, m, v, lr, b1, b2, eps, c1, c2, W1b, W2b, W2Tb);
}

__global__ void k_mlp_refresh(const float* __restrict__ P, int n, __nv_bfloat16* __restrict__ W1b,
                              __nv_bfloat16* __restrict__ W2b, __nv_bfloat16* __restrict__ W2Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nW1 = kH * kIn, oW2 = nW1 + kH, nW2 = kH * kH;
    if (i < nW1) W1b[i] = __float2bfloat16_rn(P[i]);
    if (i >= oW2 && i < oW2 + nW2) {
        const int j = i - oW2, o = j / kH, k = j % kH;
        W2b[j] = __float2bfloat16_rn(P[i]);
        W2Tb[k * kH + o] = __float2bfloat16_rn(P[i]);
    }
}

}  // namespace

int mlp_wgrad_splits(int64_t B) {
    // about 512 rows per CTA, at most 148 x 2 CTAs per weight-gradient launch
    int64_t s = (B + 511) / 512;
    if (s > 148) s = 148;
    return s < 1 ? 1 : (int)s;
}

MlpBufs mlp_layout(float* P, __nv_bfloat16* W1b, __nv_bfloat16* W2b, __nv_bfloat16* W2Tb) {
    MlpBufs b;
    b.P = P;
    b.W1b = W1b;
    b.W2b = W2b;
    b.W2Tb = W2Tb;
    return b;
}

static MlpDev dev_view(const MlpBufs& m) {
    MlpDev d;
    d.W1b = m.W1b;
    d.W2b = m.W2b;
    d.W2Tb = m.W2Tb;
    const float* P = m.P;
    d.b1 = P + kH * kIn;
    d.b2 = P + kH * kIn + kH + kH * kH;
    d.w3 = d.b2 + kH;
    d.b3 = d.w3 + kH;
    return d;
}

static int fwd_grid(int B) {
    const int nt = (B + kRows - 1) / kRows;
    return nt < 148 ? nt : 148;
}

namespace {
__global__ void k_sum_partials(const float* __restrict__ part, int splits, int n, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.f;
    for (int k = 0; k < splits; ++k) acc += part[(size_t)k * n + i];
    out[i] = acc;
}

__global__ void k_debug_gelu(const float* __restrict__ z, int n, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // the packed evaluations the network's epilogues use, in both lanes (lane 1 holds -z);
    // they must equal the scalar gelu() / gelu_d() bit for bit, else the value is reported
    // as NaN
    float g, gm, b0, b1, d0, d1;
    f2split(gelu2(f2(z[i], -z[i])), g, gm);
    f32x2 gb, gdb;
    gelu2_both(f2(z[i], -z[i]), gb, gdb);
    f2split(gb, b0, b1);
    f2split(gdb, d0, d1);
    float s0, sd0, s1, sd1;
    gelu_both(z[i], s0, sd0);
    gelu_both(-z[i], s1, sd1);
    const bool same = __float_as_uint(g) == __float_as_uint(gelu(z[i])) &&
                      __float_as_uint(gm) == __float_as_uint(gelu(-z[i])) &&
                      __float_as_uint(b0) == __float_as_uint(g) && __float_as_uint(b1) == __float_as_uint(gm) &&
                      __float_as_uint(s0) == __float_as_uint(g) && __float_as_uint(s1) == __float_as_uint(gm) &&
                      __float_as_uint(d0) == __float_as_uint(sd0) && __float_as_uint(d1) == __float_as_uint(sd1) &&
                      __float_as_uint(sd0) == __float_as_uint(gelu_d(z[i]));
    out[2 * i] = same ? g : __int_as_float(0x7fc00000);
    out[2 * i + 1] = gelu_d(z[i]);
}
}  // namespace

void debug_gelu(const float* z, int n, float* out, cudaStream_t st) {
    k_debug_gelu<<<(n + 255) / 256, 256, 0, st>>>(z, n, out);
    count_launches(1);
}

void mlp_refresh(const MlpBufs& m, cudaStream_t st) {
    k_mlp_refresh<<<(kMlpParams + 255) / 256, 256, 0, st>>>(m.P, kMlpParams, m.W1b, m.W2b, m.W2Tb);
    count_launches(1);
}

void mlp_forward(const MlpBufs& m, const void* X, int B, float* y, int* err, cudaStream_t st) {
    const size_t smem = (size_t)kH * kIn * 2 + (size_t)kH * kH * 2 + (size_t)kRows * kIn * 2 +
                        (size_t)kRows * kHc * 2 + 1024;
    cudaFuncSetAttribute(k_mlp_fwd2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_mlp_fwd2<false><<<fwd_grid(B), 512, smem, st>>>(reinterpret_cast<const __nv_bfloat16*>(X), B, dev_view(m), y,
                                                      nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                      0.f, err);
    count_launches(1);
}

// The gradient kernels of one batch: forward (y, loss, d/dw3, d/db3 into G), dh1, and the
// two weight-gradient GEMMs (split-K partials in tmp.wpart, bias gradients into G).  G's
// bias and output-weight entries and *loss accumulate: the caller zeroes them.  Returns
// the number of split-K partials.
static int mlp_backward_core(const MlpBufs& m, const void* X, const float* t, int B, float* y, float* G,
                             float* loss, const MlpTemp& tmp, int* err, cudaStream_t st) {
    const __nv_bfloat16* Xb = reinterpret_cast<const __nv_bfloat16*>(X);
    const MlpDev d = dev_view(m);
    float* gW1 = G;
    float* gb1 = gW1 + kH * kIn;
    float* gW2 = gb1 + kH;
    float* gb2 = gW2 + kH * kH;
    float* gw3 = gb2 + kH;
    float* gb3 = gw3 + kH;
    const size_t smem_f = (size_t)kH * kIn * 2 + (size_t)kH * kH * 2 + (size_t)kRows * kIn * 2 +
                          (size_t)kRows * kHc * 2 + 1024;
    cudaFuncSetAttribute(k_mlp_fwd2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f);
    k_mlp_fwd2<true><<<fwd_grid(B), 512, smem_f, st>>>(Xb, B, d, y, t, tmp.gd1, tmp.h1, tmp.dz2, gw3, gb3, loss,
                                                       1.f / (float)B, err);
    const size_t smem_d = (size_t)kRows * kH * 2 + (size_t)kH * kH * 2 + 1024;
    cudaFuncSetAttribute(k_mlp_dh1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_d);
    k_mlp_dh1<<<fwd_grid(B), 512, smem_d, st>>>(tmp.dz2, tmp.gd1, B, d, tmp.dz1, err);
    const int splits = mlp_wgrad_splits(B);
    const int rows_per_cta = (B + splits - 1) / splits;
    float* part2 = tmp.wpart;
    float* part1 = tmp.wpart + (size_t)splits * kH * kH;
    const size_t smem_w2 = (size_t)128 * 128 * 2 + (size_t)kH * 128 * 2 + 1024;
    cudaFuncSetAttribute(k_mlp_wgrad<kH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w2);
    k_mlp_wgrad<kH><<<dim3(splits, 2), 256, smem_w2, st>>>(tmp.dz2, tmp.h1, B, rows_per_cta, part2, gb2, err);
    const size_t smem_w1 = (size_t)128 * 128 * 2 + (size_t)kIn * 128 * 2 + 1024;
    cudaFuncSetAttribute(k_mlp_wgrad<kIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w1);
    k_mlp_wgrad<kIn><<<dim3(splits, 2), 256, smem_w1, st>>>(tmp.dz1, Xb, B, rows_per_cta, part1, gb1, err);
    count_launches(4);
    return splits;
}

void mlp_gradient(const MlpBufs& m, const void* X, const float* t, int B, float* y, float* G, float* loss,
                  const MlpTemp& tmp, int* err, cudaStream_t st) {
    cudaMemsetAsync(G, 0, sizeof(float) * kMlpParams, st);
    cudaMemsetAsync(loss, 0, sizeof(float), st);
    const int splits = mlp_backward_core(m, X, t, B, y, G, loss, tmp, err, st);
    float* gW1 = G;
    float* gW2 = G + kH * kIn + kH;
    const float* part2 = tmp.wpart;
    const float* part1 = tmp.wpart + (size_t)splits * kH * kH;
    k_sum_partials<<<(kH * kH + 255) / 256, 256, 0, st>>>(part2, splits, kH * kH, gW2);
    k_sum_partials<<<(kH * kIn + 255) / 256, 256, 0, st>>>(part1, splits, kH * kIn, gW1);
    count_launches(2);
}

void mlp_train_step(const MlpBufs& m, const void* X, const float* t, int B, float* y, float* G, float* loss,
                    const MlpTemp& tmp, float* mo, float* vo, float lr, int step, int* err, cudaStream_t st) {
    const int splits = mlp_backward_core(m, X, t, B, y, G, loss, tmp, err, st);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 - pow(0.9, (double)step)), c2 = (float)(1.0 - pow(0.999, (double)step));
    k_mlp_sum_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(tmp.wpart, tmp.wpart + (size_t)splits * kH * kH, splits, G,
                                                             m.P, mo, vo, lr, b1, b2, eps, c1, c2, m.W1b, m.W2b,
                                                             m.W2Tb);
    count_launches(1);
}

}  // namespace csgs

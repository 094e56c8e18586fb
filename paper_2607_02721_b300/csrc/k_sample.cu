// Sensitivity sampling (Algorithm 1, steps 3-5): S = sum_i s_i in FP64 (fixed
// reduction order, so repeated runs agree bit for bit), p_i = s_i / S, an integer CDF
// C_i = sum_{j<=i} round(p_j 2^56), m i.i.d. draws J_t = min{i : C_i > u_t} with
// u_t = floor(x_t C_total / 2^64) and x_t a 64-bit Philox4x32-10 word (key = seed,
// counter = t), counts n_i, and weights w_i = n_i / (m p_i).  The integer CDF makes
// the draws exact: the same p, seed and t always select the same index.
#include "csgs_internal.cuh"

namespace csgs {
namespace {

constexpr int kRedBlocks = 512;
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kChunk = kThreads * kItems;

__global__ void __launch_bounds__(kThreads) k_partial_sum(const float* __restrict__ s, int64_t n,
                                                          double* __restrict__ partial) {
    __shared__ double ws[kThreads / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)kRedBlocks * kThreads)
        acc += (double)s[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kRedBlocks) k_final_sum(const double* __restrict__ partial, double* S) {
    __shared__ double ws[kRedBlocks / 32];
    double v = partial[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRedBlocks / 32; ++w) t += ws[w];
        *S = t;
    }
}

// Surrogate prior: per block, the sum of log a - log b over the i with a > 0 and b > 0 (FP64)
// and their count; k_final_sum2 adds the blocks in a fixed order.
__global__ void __launch_bounds__(kThreads) k_log_ratio_partial(const float* __restrict__ a, const float* __restrict__ b,
                                                                int64_t n, double* __restrict__ partial) {
    __shared__ double ws[2][kThreads / 32];
    double acc = 0.0, cnt = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)kRedBlocks * kThreads) {
        const float x = a[i], y = b[i];
        if (x > 0.f && y > 0.f) {
            acc += log((double)x) - log((double)y);
            cnt += 1.0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ws[0][threadIdx.x >> 5] = acc;
        ws[1][threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            t0 += ws[0][w];
            t1 += ws[1][w];
        }
        partial[2 * blockIdx.x] = t0;
        partial[2 * blockIdx.x + 1] = t1;
    }
}

__global__ void __launch_bounds__(kRedBlocks) k_final_sum2(const double* __restrict__ partial, double* out) {
    __shared__ double ws[2][kRedBlocks / 32];
    double v = partial[2 * threadIdx.x], c = partial[2 * threadIdx.x + 1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ws[0][threadIdx.x >> 5] = v;
        ws[1][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < kRedBlocks / 32; ++w) {
            t0 += ws[0][w];
            t1 += ws[1][w];
        }
        out[0] = t0;
        out[1] = t1;
    }
}

__global__ void k_scene_normalise(float* __restrict__ s, int64_t n, const double* __restrict__ sumA) {
    const double A = *sumA;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s[i] = A > 0.0 ? (float)((double)s[i] / A) : 0.f;
}

__global__ void k_scale(float* __restrict__ s, int64_t n, double f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s[i] = (float)((double)s[i] * f);
}

__global__ void k_image_fold(float* __restrict__ s, float* __restrict__ vbuf, int64_t n,
                             const double* __restrict__ sumA_view) {
    const double A = *sumA_view;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = vbuf[i];
        if (v > 0.f) {
            if (A > 0.0) s[i] = fmaxf(s[i], (float)((double)v / A));
            vbuf[i] = 0.f;
        }
    }
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies, round keys bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__global__ void k_log_target(const float* __restrict__ s, int64_t n, float eps, float* __restrict__ t) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = logf(s[i] + eps);
}

// residual target against the prior p: t = log(s + eps) - log(p + eps) - mu
__global__ void k_residual_target(const float* __restrict__ s, const float* __restrict__ p, int64_t n, float eps,
                                  float mu, float* __restrict__ t) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = logf(s[i] + eps) - logf(p[i] + eps) - mu;
}

// the prediction y as a residual on the prior: exp(y + log(p + eps) + mu) - eps, then as k_combine
__global__ void k_combine_prior(const float* __restrict__ y, const float* __restrict__ p,
                                const float* __restrict__ s_exact, int64_t n, float eps, float mu, int fill_only,
                                float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = fmaxf(expf(y[i] + logf(p[i] + eps) + mu) - eps, 0.f);
        const float s = s_exact ? s_exact[i] : 0.f;
        out[i] = fill_only ? (s > 0.f ? s : e) : fmaxf(e, s);
    }
}

__global__ void k_combine(const float* __restrict__ y, const float* __restrict__ s_exact, int64_t n, float eps,
                          int fill_only, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = fmaxf(expf(y[i]) - eps, 0.f);
        const float s = s_exact ? s_exact[i] : 0.f;
        out[i] = fill_only ? (s > 0.f ? s : e) : fmaxf(e, s);
    }
}

// minibatch rows: row j of step `step` = floor(x * n / 2^32), x a Philox word (key = seed,
// counter = (j, step)); gathers the features and targets into contiguous buffers
__global__ void k_gather_batch(const uint4* __restrict__ X, const float* __restrict__ t, int64_t n, int B,
                               uint64_t seed, uint32_t step, uint4* __restrict__ Xb, float* __restrict__ tb,
                               float* __restrict__ zero) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0 && zero) *zero = 0.f;
    if (j >= B) return;
    const uint4 r = philox4x32_10(make_uint4((uint32_t)j, step, 0x5EEDu, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const int64_t row = (int64_t)(((unsigned long long)r.x * (unsigned long long)n) >> 32);
#pragma unroll
    for (int c = 0; c < 8; ++c) Xb[(size_t)j * 8 + c] = X[(size_t)row * 8 + c];
    tb[j] = t[row];
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_probs(const float* __restrict__ s, int64_t n, const double* __restrict__ S, double* __restrict__ p) {
    const double tot = *S;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = tot > 0.0 ? (double)s[i] / tot : 0.0;
}

// ---- block scans (one value per thread)
template <typename T>
__device__ __forceinline__ T block_scan_excl(T v, T* ws, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (int)(blockDim.x >> 5) ? ws[lane] : (T)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    T pre = x - v + (warp > 0 ? ws[warp - 1] : (T)0);
    *total = ws[(blockDim.x >> 5) - 1];
    __syncthreads();
    return pre;
}

__device__ __forceinline__ unsigned long long quant(double p) {
    return (unsigned long long)__double2ll_rn(scalbn(p, 56));
}

// CDF phase 1: per-block sums of the quantised probabilities
__global__ void __launch_bounds__(kThreads) k_cdf_reduce(const double* __restrict__ p, int64_t n,
                                                         unsigned long long* __restrict__ part) {
    __shared__ unsigned long long ws[32];
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * kItems;
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n) sum += quant(p[base + k]);
    unsigned long long tot;
    block_scan_excl<unsigned long long>(sum, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_top(T* __restrict__ part, int nb, T* total) {
    __shared__ T ws[32];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int i = b0 + threadIdx.x;
        T v = i < nb ? part[i] : (T)0;
        T tot;
        T pre = block_scan_excl<T>(v, ws, &tot);
        T c = carry;
        if (i < nb) part[i] = c + pre;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// CDF phase 3: inclusive prefix per element
__global__ void __launch_bounds__(kThreads) k_cdf_down(const double* __restrict__ p, int64_t n,
                                                       const unsigned long long* __restrict__ part,
                                                       unsigned long long* __restrict__ C) {
    __shared__ unsigned long long ws[32];
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * kItems;
    unsigned long long q[kItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        q[k] = base + k < n ? quant(p[base + k]) : 0ull;
        sum += q[k];
    }
    unsigned long long tot;
    unsigned long long run = block_scan_excl<unsigned long long>(sum, ws, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        run += q[k];
        if (base + k < n) C[base + k] = run;
    }
}

__global__ void k_draw(const unsigned long long* __restrict__ C, int64_t n, int64_t m, uint64_t seed,
                       uint32_t* __restrict__ counts, int32_t* __restrict__ draws) {
    const unsigned long long total = C[n - 1];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)((uint64_t)t >> 32), 0u, 0u),
                                      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        const unsigned long long x = ((unsigned long long)r.y << 32) | r.x;
        const unsigned long long u = __umul64hi(x, total);
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (C[mid] > u)
                hi = mid;
            else
                lo = mid + 1;
        }
        atomicAdd(counts + lo, 1u);
        if (draws) draws[t] = (int32_t)lo;
    }
}

// compaction of the sampled indices (ascending) with their weights
__global__ void __launch_bounds__(kThreads) k_flag_reduce(const uint32_t* __restrict__ counts, int64_t n,
                                                          uint32_t* __restrict__ part) {
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * kItems;
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n) sum += counts[base + k] > 0u;
    uint32_t tot;
    block_scan_excl<uint32_t>(sum, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) k_flag_down(const uint32_t* __restrict__ counts,
                                                        const double* __restrict__ p, int64_t n, int64_t m,
                                                        const uint32_t* __restrict__ part, int32_t* __restrict__ idx,
                                                        float* __restrict__ w) {
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * kItems;
    uint32_t c[kItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        c[k] = base + k < n ? counts[base + k] : 0u;
        sum += c[k] > 0u;
    }
    uint32_t tot;
    uint32_t pos = block_scan_excl<uint32_t>(sum, ws, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (c[k] > 0u) {
            idx[pos] = (int32_t)(base + k);
            w[pos] = (float)((double)c[k] / ((double)m * p[base + k]));
            ++pos;
        }
    }
}

}  // namespace

void sum_scores(const float* s, int64_t n, double* partial, double* S, cudaStream_t st) {
    k_partial_sum<<<kRedBlocks, kThreads, 0, st>>>(s, n, partial);
    count_launches(1);
    k_final_sum<<<1, kRedBlocks, 0, st>>>(partial, S);
    count_launches(1);
}

void scene_normalise(float* s, int64_t n, const double* sumA, cudaStream_t st) {
    k_scene_normalise<<<148 * 8, 256, 0, st>>>(s, n, sumA);
    count_launches(1);
}

void scale_scores(float* s, int64_t n, double f, cudaStream_t st) {
    k_scale<<<148 * 8, 256, 0, st>>>(s, n, f);
    count_launches(1);
}

void image_fold(float* s, float* vbuf, int64_t n, const double* sumA_view, cudaStream_t st) {
    k_image_fold<<<148 * 8, 256, 0, st>>>(s, vbuf, n, sumA_view);
    count_launches(1);
}

void log_target(const float* s, int64_t n, float eps, float* t, cudaStream_t st) {
    k_log_target<<<148 * 8, 256, 0, st>>>(s, n, eps, t);
    count_launches(1);
}

void log_ratio_mean(const float* a, const float* b, int64_t n, double* partial, double* out, cudaStream_t st) {
    k_log_ratio_partial<<<kRedBlocks, kThreads, 0, st>>>(a, b, n, partial);
    k_final_sum2<<<1, kRedBlocks, 0, st>>>(partial, out);
    count_launches(2);
}

void residual_target(const float* s, const float* p, int64_t n, float eps, float mu, float* t, cudaStream_t st) {
    k_residual_target<<<148 * 8, 256, 0, st>>>(s, p, n, eps, mu, t);
    count_launches(1);
}

void surrogate_combine_prior(const float* y, const float* p, const float* s_exact, int64_t n, float eps, float mu,
                             int fill_only, float* out, cudaStream_t st) {
    k_combine_prior<<<148 * 8, 256, 0, st>>>(y, p, s_exact, n, eps, mu, fill_only, out);
    count_launches(1);
}

void surrogate_combine(const float* y, const float* s_exact, int64_t n, float eps, int fill_only, float* out,
                       cudaStream_t st) {
    k_combine<<<148 * 8, 256, 0, st>>>(y, s_exact, n, eps, fill_only, out);
    count_launches(1);
}

void gather_batch(const void* X, const float* t, int64_t n, int B, uint64_t seed, uint32_t step, void* Xb, float* tb,
                  float* zero, cudaStream_t st) {
    k_gather_batch<<<(B + 255) / 256, 256, 0, st>>>(reinterpret_cast<const uint4*>(X), t, n, B, seed, step,
                                                     reinterpret_cast<uint4*>(Xb), tb, zero);
    count_launches(1);
}

void adam_update(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                 int step, cudaStream_t st) {
    const float c1 = (float)(1.0 - pow((double)b1, (double)step)), c2 = (float)(1.0 - pow((double)b2, (double)step));
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    k_adam<<<(int)blocks, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    count_launches(1);
}

void probabilities_from_scores(const float* s, int64_t n, const double* S, double* p, cudaStream_t st) {
    k_probs<<<148 * 8, 256, 0, st>>>(s, n, S, p);
    count_launches(1);
}

void sample_draws(const double* p, int64_t n, int64_t m, uint64_t seed, const SampleTemp& t, int32_t* draws,
                  int32_t* idx, float* w, cudaStream_t st) {
    const int nb = (int)((n + kChunk - 1) / kChunk);
    k_cdf_reduce<<<nb, kThreads, 0, st>>>(p, n, t.C_tmp);
    count_launches(1);
    k_scan_top<unsigned long long><<<1, 1024, 0, st>>>(t.C_tmp, nb, nullptr);
    count_launches(1);
    k_cdf_down<<<nb, kThreads, 0, st>>>(p, n, t.C_tmp, t.C);
    count_launches(1);
    cudaMemsetAsync(t.counts, 0, sizeof(uint32_t) * (size_t)n, st);
    int db = (int)((m + 255) / 256);
    if (db > 148 * 16) db = 148 * 16;
    k_draw<<<db, 256, 0, st>>>(t.C, n, m, seed, t.counts, draws);
    count_launches(1);
    k_flag_reduce<<<nb, kThreads, 0, st>>>(t.counts, n, t.scan_tmp);
    count_launches(1);
    k_scan_top<uint32_t><<<1, 1024, 0, st>>>(t.scan_tmp, nb, t.n_out);
    count_launches(1);
    k_flag_down<<<nb, kThreads, 0, st>>>(t.counts, p, n, m, t.scan_tmp, idx, w);
    count_launches(1);
}

}  // namespace csgs

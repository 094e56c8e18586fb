// Front-to-back compositing of one 16x16 screen tile per CTA (Sec. 3 "Scalar rendering
// function": rho = alpha k, T = prod (1 - rho), a = c rho T, A = sum a) and the
// per-Gaussian sensitivity reduction (Eq. sen).
//
// Each thread owns one pixel; a warp covers an 8x4 pixel block.  The tile's
// depth-sorted splat list is staged through shared memory 256 records at a time.
// While staging, each splat gets a mask of the warp blocks its footprint's bounding
// box touches, and every warp compacts the batch into its own list, so a warp only
// evaluates splats that can reach one of its pixels.
//
// Per (pixel, splat) the kernel evaluates, in tile-centred pixel coordinates (X, Y),
//   e1 = s1 X + s1k Y + c1,  e2 = s2 Y + c2,  p = log2(alpha) - e1^2 - e2^2
// (the EWA kernel's exponent in base 2, conic in Cholesky form; five FMAs), then one
// compare against thr = max(log2 alpha - qcut, log2 alpha_min) decides the
// 3-sigma footprint and the alpha_min skip together, and rho = min(rho_max, 2^p).
// A thread stops at the Gaussian that would bring T below t_min; the CTA leaves
// once every pixel has stopped.
//
// Score (per-pixel resolution) runs two passes over the same list inside one CTA:
// pass 1 yields A(q) and the index of each pixel's last contributor, pass 2 recomputes
// rho bit for bit (same operations, same contributor set) and reduces
// imp = a / A per Gaussian: warp max with redux.sync on the float bits (imp >= 0, so
// unsigned order = float order), a shared-memory max across the CTA's warps, and one
// global atomicMax per (tile, Gaussian).
// Score (per-scene resolution) is one pass: warp sums of a, one global atomicAdd per
// (tile, Gaussian), and the CTA's sum of A added to an FP64 total.
#include "csgs_internal.cuh"

namespace csgs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

enum { kRender = 0, kScorePixel = 1, kScoreScene = 2 };

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Shared {
    float4 A[kThreads];  // s1, s1k, c1, s2
    float4 B[kThreads];  // c2, log2 alpha, thr, cw = obj_w . rgb
    float4 C[kThreads];  // r, g, b, -
    uint32_t gid[kThreads];
    uint32_t msk[kThreads];
    uint8_t wl[kWarps][kThreads];  // per-warp compacted batch indices
    uint32_t red[kThreads];
    float part[kWarps][kThreads];
    int last;
    double sumA[kWarps];
};

// Stage splat i of the tile list into slot threadIdx.x (tile centre (cx, cy)).
template <int MODE>
__device__ __forceinline__ void stage(const CompositeArgs& a, Shared& sh, uint32_t i, uint32_t end, float cx,
                                      float cy) {
    const int tid = threadIdx.x;
    if (MODE == kScorePixel) sh.red[tid] = 0u;
    if (MODE == kScoreScene)
#pragma unroll
        for (int w = 0; w < kWarps; ++w) sh.part[w][tid] = 0.f;
    sh.msk[tid] = 0u;
    if (i >= end) return;
    const uint32_t g = __ldg(a.inst_gid + i);
    if (g >= (uint32_t)a.n_gauss) return;  // only reachable after a reported capacity overflow
    const float4* sp = reinterpret_cast<const float4*>(a.splats + g);
    const float4 m = __ldg(sp), q = __ldg(sp + 1), c = __ldg(sp + 2);
    // tile-centred mean from the two-float pixel mean
    const float mx = __fadd_rn(__fadd_rn(m.x, -cx), m.z);
    const float my = __fadd_rn(__fadd_rn(m.y, -cy), m.w);
    const float s1 = q.x, s1k = q.y, s2 = q.z;
    const float c1 = -__fmaf_rn(s1, mx, __fmul_rn(s1k, my));
    const float c2 = -__fmul_rn(s2, my);
    sh.A[tid] = make_float4(s1, s1k, c1, s2);
    sh.B[tid] = make_float4(c2, c.w, q.w, a.o.ow0 * c.x + a.o.ow1 * c.y + a.o.ow2 * c.z);
    sh.C[tid] = make_float4(c.x, c.y, c.z, 0.f);
    sh.gid[tid] = g;
    // bounding box of the footprint: rx^2 = qcut (1/s1^2 + (s1k/(s1 s2))^2), ry^2 = qcut / s2^2,
    // widened so that FP32 rounding never drops a pixel that passes the test
    const float i1 = 1.f / s1, i2 = 1.f / s2;
    const float kk = s1k * i1 * i2;
    const float rx = sqrtf(a.o.qcut * (i1 * i1 + kk * kk)) * 1.001f + 0.01f;
    const float ry = sqrtf(a.o.qcut) * i2 * 1.001f + 0.01f;
    const float xlo = mx - rx, xhi = mx + rx, ylo = my - ry, yhi = my + ry;
    uint32_t cols = 0u, rows = 0u;
    cols |= (xlo <= -0.5f && xhi >= -7.5f) ? 1u : 0u;
    cols |= (xlo <= 7.5f && xhi >= 0.5f) ? 2u : 0u;
#pragma unroll
    for (int r = 0; r < 4; ++r) rows |= (ylo <= -4.5f + 4.f * r && yhi >= -7.5f + 4.f * r) ? (1u << r) : 0u;
    uint32_t mk = 0u;
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (rows & (1u << r)) mk |= cols << (2 * r);
    sh.msk[tid] = mk;
}

// Compact the staged batch into this warp's list; returns its length.
__device__ __forceinline__ int warp_list(Shared& sh, int cnt, int warp, int lane) {
    const uint32_t lt = (1u << lane) - 1u;
    int nw = 0;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int j = c0 + lane;
        const bool bit = j < cnt && ((sh.msk[j] >> warp) & 1u);
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        if (bit) sh.wl[warp][nw + __popc(bal & lt)] = (uint8_t)j;
        nw += __popc(bal);
    }
    __syncwarp();
    return nw;
}

// Base-2 exponent of rho at pixel (X, Y) for staged splat j.
__device__ __forceinline__ float exponent2(const float4& A, const float4& B, float X, float Y) {
    const float e1 = __fmaf_rn(A.x, X, __fmaf_rn(A.y, Y, A.z));
    const float e2 = __fmaf_rn(A.w, Y, B.x);
    return __fmaf_rn(-e1, e1, __fmaf_rn(-e2, e2, B.y));
}

template <int MODE, bool STATS>
__global__ void __launch_bounds__(kThreads) k_composite(const CompositeArgs a) {
    __shared__ Shared sh;
    const CamDev& cam = a.cam;
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lx = (warp & 1) * 8 + (lane & 7), ly = (warp >> 1) * 4 + (lane >> 3);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < cam.W && py < cam.H;
    const float X = (float)lx - 7.5f, Y = (float)ly - 7.5f;
    const float cx = (float)(tx * kTile) + 7.5f, cy = (float)(ty * kTile) + 7.5f;
    const uint2 rg = a.ranges[tile];
    const uint32_t start = rg.x;
    const int n = (int)(rg.y - rg.x);
    const float rho_max = a.o.rho_max, t_min = a.o.t_min;

    float T = 1.f, A0 = 0.f, A1 = 0.f, A2 = 0.f;
    int last = 0;
    bool done = !inside;
    unsigned long long n_eval = 0, n_hit = 0, n_viol = 0;
    if (tid == 0) sh.last = 0;

    // ---------------------------------------------------------------- pass 1
    for (int b = 0; b < n; b += kThreads) {
        if (__syncthreads_count(done) == kThreads) break;
        stage<MODE>(a, sh, start + b + tid, rg.y, cx, cy);
        __syncthreads();
        const int cnt = min(kThreads, n - b);
        const int nw = warp_list(sh, cnt, warp, lane);
        if (MODE != kScoreScene) {
            if (!done) {
                for (int k = 0; k < nw; ++k) {
                    const int j = sh.wl[warp][k];
                    const float4 Aj = sh.A[j];
                    const float4 Bj = sh.B[j];
                    const float p = exponent2(Aj, Bj, X, Y);
                    if (STATS) ++n_eval;
                    if (p < Bj.z) continue;
                    const float raw = ex2_approx(p);
                    const float r = fminf(rho_max, raw);
                    if (STATS) {
                        ++n_hit;
                        n_viol += raw >= 1.f;
                    }
                    const float Tn = __fmul_rn(T, __fadd_rn(1.f, -r));
                    if (Tn < t_min) {
                        done = true;
                        break;
                    }
                    const float w = __fmul_rn(r, T);
                    const float4 Cj = sh.C[j];
                    A0 = __fmaf_rn(Cj.x, w, A0);
                    A1 = __fmaf_rn(Cj.y, w, A1);
                    A2 = __fmaf_rn(Cj.z, w, A2);
                    T = Tn;
                    last = b + j + 1;
                }
            }
        } else {
            // per-scene resolution: warp-uniform loop so the warp can sum a per Gaussian
            bool act = !done;
            if (__any_sync(0xffffffffu, act)) {
                for (int k = 0; k < nw; ++k) {
                    const int j = sh.wl[warp][k];
                    float v = 0.f;
                    if (act) {
                        const float4 Aj = sh.A[j];
                        const float4 Bj = sh.B[j];
                        const float p = exponent2(Aj, Bj, X, Y);
                        if (STATS) ++n_eval;
                        if (p >= Bj.z) {
                            const float r = fminf(rho_max, ex2_approx(p));
                            if (STATS) ++n_hit;
                            const float Tn = __fmul_rn(T, __fadd_rn(1.f, -r));
                            if (Tn < t_min) {
                                act = false;
                                done = true;
                            } else {
                                const float w = __fmul_rn(r, T);
                                const float4 Cj = sh.C[j];
                                A0 = __fmaf_rn(Cj.x, w, A0);
                                A1 = __fmaf_rn(Cj.y, w, A1);
                                A2 = __fmaf_rn(Cj.z, w, A2);
                                v = __fmul_rn(Bj.w, w);
                                T = Tn;
                            }
                        }
                    }
                    if (__any_sync(0xffffffffu, v > 0.f)) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (lane == 0) sh.part[warp][j] = v;
                    }
                    if (!__any_sync(0xffffffffu, act)) break;
                }
            }
            __syncthreads();
            if (tid < cnt) {
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) v += sh.part[w][tid];
                if (v > 0.f) atomicAdd(a.s_sum + sh.gid[tid], v);
            }
        }
    }

    if (MODE == kRender) {
        if (inside) {
            const size_t pix = (size_t)py * cam.W + px;
            a.rgb[3 * pix + 0] = A0;
            a.rgb[3 * pix + 1] = A1;
            a.rgb[3 * pix + 2] = A2;
            if (a.T) a.T[pix] = T;
        }
    }

    if (MODE == kScoreScene) {
        // CTA sum of the pixel objective, added to the FP64 scene total
        double Ao = inside ? (double)(a.o.ow0 * A0 + a.o.ow1 * A1 + a.o.ow2 * A2) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Ao += __shfl_xor_sync(0xffffffffu, Ao, o);
        __syncthreads();
        if (lane == 0) sh.sumA[warp] = Ao;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w) t += sh.sumA[w];
            if (t > 0.0) atomicAdd(&a.ctr->sumA, t);
        }
    }

    // ---------------------------------------------------------------- pass 2
    unsigned long long n_eval2 = 0, n_hit2 = 0;
    if (MODE == kScorePixel) {
        const float Aobj = a.o.ow0 * A0 + a.o.ow1 * A1 + a.o.ow2 * A2;
        const bool has = inside && Aobj > 0.f;  // queries with A = 0 are discarded
        // T' = T / A: imp = cw rho T' directly
        float Tq = has ? 1.f / Aobj : 0.f;
        if (!has) last = 0;
        __syncthreads();
        atomicMax(&sh.last, last);
        __syncthreads();
        const int n2 = sh.last;
        for (int b = 0; b < n2; b += kThreads) {
            __syncthreads();
            stage<MODE>(a, sh, start + b + tid, rg.y, cx, cy);
            __syncthreads();
            const int cnt = min(kThreads, n2 - b);
            const int nw = warp_list(sh, cnt, warp, lane);
            const int lim = max(0, min(cnt, last - b));
            const int jw = (int)__reduce_max_sync(0xffffffffu, (unsigned)lim);
            for (int k = 0; k < nw; ++k) {
                const int j = sh.wl[warp][k];
                if (j >= jw) break;  // the list is in increasing j; warp-uniform
                uint32_t bits = 0u;
                if (j < lim) {
                    const float4 Aj = sh.A[j];
                    const float4 Bj = sh.B[j];
                    const float p = exponent2(Aj, Bj, X, Y);
                    if (STATS) ++n_eval2;
                    if (p >= Bj.z) {
                        const float r = fminf(rho_max, ex2_approx(p));
                        if (STATS) ++n_hit2;
                        bits = __float_as_uint(__fmul_rn(Bj.w, __fmul_rn(r, Tq)));
                        Tq = __fmul_rn(Tq, __fadd_rn(1.f, -r));
                    }
                }
                const uint32_t mx = __reduce_max_sync(0xffffffffu, bits);
                if (lane == 0 && mx) atomicMax(&sh.red[j], mx);
            }
            __syncthreads();
            if (tid < cnt) {
                const uint32_t v = sh.red[tid];
                if (v) atomicMax(a.s_bits + sh.gid[tid], v);
            }
        }
    }

    if (STATS) {
        unsigned long long e = n_eval, h = n_hit, e2 = n_eval2, h2 = n_hit2, vv = n_viol;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(0xffffffffu, e, o);
            h += __shfl_xor_sync(0xffffffffu, h, o);
            e2 += __shfl_xor_sync(0xffffffffu, e2, o);
            h2 += __shfl_xor_sync(0xffffffffu, h2, o);
            vv += __shfl_xor_sync(0xffffffffu, vv, o);
        }
        if (lane == 0) {
            if (e) atomicAdd(&a.ctr->pairs_eval, e);
            if (h) atomicAdd(&a.ctr->pairs_hit, h);
            if (e2) atomicAdd(&a.ctr->pairs_eval2, e2);
            if (h2) atomicAdd(&a.ctr->pairs_hit2, h2);
            if (vv) atomicAdd(&a.ctr->violations, vv);
        }
    }
}

}  // namespace

void launch_composite_render(const CompositeArgs& a, cudaStream_t st) {
    const int tiles = a.cam.tiles_x * a.cam.tiles_y;
    if (a.stats)
        k_composite<kRender, true><<<tiles, kThreads, 0, st>>>(a);
    else
        k_composite<kRender, false><<<tiles, kThreads, 0, st>>>(a);
    count_launches(1);
}

void launch_composite_score(const CompositeArgs& a, cudaStream_t st) {
    const int tiles = a.cam.tiles_x * a.cam.tiles_y;
    if (a.o.resolution == CSGS_RES_SCENE) {
        if (a.stats)
            k_composite<kScoreScene, true><<<tiles, kThreads, 0, st>>>(a);
        else
            k_composite<kScoreScene, false><<<tiles, kThreads, 0, st>>>(a);
    } else {
        if (a.stats)
            k_composite<kScorePixel, true><<<tiles, kThreads, 0, st>>>(a);
        else
            k_composite<kScorePixel, false><<<tiles, kThreads, 0, st>>>(a);
    }
    count_launches(1);
}

}  // namespace csgs

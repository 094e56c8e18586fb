// Front-to-back compositing of one 16x16 screen tile per CTA (Sec. 3 "Scalar rendering
// function": rho = alpha k, T = prod (1 - rho), a = c rho T, A = sum a) and the
// per-Gaussian sensitivity reduction (Eq. sen).
//
// Each thread owns one pixel.  The tile's depth-sorted splat list is staged through
// shared memory 256 records at a time; a warp covers an 8x4 pixel block so its
// lanes see similar footprints.  A thread stops at the Gaussian that would bring T
// below t_min; the CTA leaves once every pixel has stopped.
//
// Score (per-pixel resolution) runs two passes over the same list inside one CTA:
// pass 1 yields A(q) and the index of each pixel's last contributor, pass 2 recomputes
// rho and T bit for bit (explicitly rounded operations, the same contributor set)
// and reduces imp = a / A per Gaussian: warp max with redux.sync on the float bits
// (imp >= 0, so unsigned order = float order), a shared-memory max across the CTA's
// warps, and one global atomicMax per (tile, Gaussian).
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

// Base-2 exponent of the kernel value at tile-relative offset (dx, dy).
__device__ __forceinline__ float exponent2(float dx, float dy, float qa, float qb, float qc) {
    const float t = __fmaf_rn(qb, dy, __fmul_rn(qa, dx));
    const float u = __fmul_rn(__fmul_rn(qc, dy), dy);
    return __fmaf_rn(dx, t, u);
}

struct Shared {
    float4 m[kThreads];  // (mean x, mean y) tile-relative, qa, qb
    float4 q[kThreads];  // qc, opacity, r, g
    float2 c[kThreads];  // b, objective colour weight cw = obj_w . rgb
    uint32_t gid[kThreads];
    uint32_t red[kThreads];
    float part[kWarps][kThreads];
    int last;
    double sumA[kWarps];
};

template <int MODE>
__device__ __forceinline__ void stage(const CompositeArgs& a, Shared& sh, uint32_t i, uint32_t end, float ox,
                                      float oy) {
    const int tid = threadIdx.x;
    if (MODE == kScorePixel) sh.red[tid] = 0u;
    if (MODE == kScoreScene)
#pragma unroll
        for (int w = 0; w < kWarps; ++w) sh.part[w][tid] = 0.f;
    if (i >= end) return;
    const uint32_t g = __ldg(a.inst_gid + i);
    if (g >= (uint32_t)a.n_gauss) {  // only reachable after a reported capacity overflow
        sh.m[tid] = make_float4(1e6f, 1e6f, -1.f, 0.f);
        sh.q[tid] = make_float4(-1.f, 0.f, 0.f, 0.f);
        sh.c[tid] = make_float2(0.f, 0.f);
        sh.gid[tid] = 0u;
        return;
    }
    const float4* sp = reinterpret_cast<const float4*>(a.splats + g);
    const float4 m = __ldg(sp), q = __ldg(sp + 1), c = __ldg(sp + 2);
    // tile-relative mean from the two-float pixel mean
    const float mx = __fadd_rn(__fadd_rn(m.x, -ox), m.z);
    const float my = __fadd_rn(__fadd_rn(m.y, -oy), m.w);
    sh.m[tid] = make_float4(mx, my, q.x, q.y);
    sh.q[tid] = make_float4(q.z, q.w, c.x, c.y);
    const float cw = a.o.ow0 * c.x + a.o.ow1 * c.y + a.o.ow2 * c.z;
    sh.c[tid] = make_float2(c.z, cw);
    sh.gid[tid] = g;
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
    const float fx = (float)lx, fy = (float)ly;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
    const uint2 rg = a.ranges[tile];
    const uint32_t start = rg.x;
    const int n = (int)(rg.y - rg.x);
    const float pcut = a.o.pcut, rho_max = a.o.rho_max, alpha_min = a.o.alpha_min, t_min = a.o.t_min;

    float T = 1.f, A0 = 0.f, A1 = 0.f, A2 = 0.f;
    int last = 0;
    bool done = !inside;
    unsigned long long n_eval = 0, n_hit = 0, n_viol = 0;
    if (tid == 0) sh.last = 0;

    // ---------------------------------------------------------------- pass 1
    for (int b = 0; b < n; b += kThreads) {
        if (__syncthreads_count(done) == kThreads) break;
        stage<MODE>(a, sh, start + b + tid, rg.y, ox, oy);
        __syncthreads();
        const int cnt = min(kThreads, n - b);
        if (MODE != kScoreScene) {
            if (!done) {
                for (int j = 0; j < cnt; ++j) {
                    const float4 m = sh.m[j];
                    const float4 q = sh.q[j];
                    const float p = exponent2(__fadd_rn(fx, -m.x), __fadd_rn(fy, -m.y), m.z, m.w, q.x);
                    if (STATS) ++n_eval;
                    if (p < pcut) continue;
                    const float raw = __fmul_rn(q.y, ex2_approx(p));
                    const float r = fminf(rho_max, raw);
                    if (r < alpha_min) continue;
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
                    A0 = __fmaf_rn(q.z, w, A0);
                    A1 = __fmaf_rn(q.w, w, A1);
                    A2 = __fmaf_rn(sh.c[j].x, w, A2);
                    T = Tn;
                    last = b + j + 1;
                }
            }
        } else {
            // per-scene resolution: warp-uniform loop so the warp can sum a per Gaussian
            bool act = !done;
            if (__any_sync(0xffffffffu, act)) {
                for (int j = 0; j < cnt; ++j) {
                    float v = 0.f;
                    if (act) {
                        const float4 m = sh.m[j];
                        const float4 q = sh.q[j];
                        const float p = exponent2(__fadd_rn(fx, -m.x), __fadd_rn(fy, -m.y), m.z, m.w, q.x);
                        if (STATS) ++n_eval;
                        if (p >= pcut) {
                            const float raw = __fmul_rn(q.y, ex2_approx(p));
                            const float r = fminf(rho_max, raw);
                            if (r >= alpha_min) {
                                if (STATS) ++n_hit;
                                const float Tn = __fmul_rn(T, __fadd_rn(1.f, -r));
                                if (Tn < t_min) {
                                    act = false;
                                    done = true;
                                } else {
                                    const float w = __fmul_rn(r, T);
                                    const float2 c = sh.c[j];
                                    A0 = __fmaf_rn(q.z, w, A0);
                                    A1 = __fmaf_rn(q.w, w, A1);
                                    A2 = __fmaf_rn(c.x, w, A2);
                                    v = __fmul_rn(c.y, w);
                                    T = Tn;
                                }
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
        const float invA = has ? 1.f / Aobj : 0.f;
        if (!has) last = 0;
        __syncthreads();
        atomicMax(&sh.last, last);
        __syncthreads();
        const int n2 = sh.last;
        T = 1.f;
        for (int b = 0; b < n2; b += kThreads) {
            __syncthreads();
            stage<MODE>(a, sh, start + b + tid, rg.y, ox, oy);
            __syncthreads();
            const int cnt = min(kThreads, n2 - b);
            const int lim = max(0, min(cnt, last - b));
            const int jw = (int)__reduce_max_sync(0xffffffffu, (unsigned)lim);
            for (int j = 0; j < jw; ++j) {
                uint32_t bits = 0u;
                if (j < lim) {
                    const float4 m = sh.m[j];
                    const float4 q = sh.q[j];
                    const float p = exponent2(__fadd_rn(fx, -m.x), __fadd_rn(fy, -m.y), m.z, m.w, q.x);
                    if (STATS) ++n_eval2;
                    if (p >= pcut) {
                        const float r = fminf(rho_max, __fmul_rn(q.y, ex2_approx(p)));
                        if (r >= alpha_min) {
                            if (STATS) ++n_hit2;
                            const float w = __fmul_rn(r, T);
                            bits = __float_as_uint(__fmul_rn(__fmul_rn(sh.c[j].y, w), invA));
                            T = __fmul_rn(T, __fadd_rn(1.f, -r));
                        }
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

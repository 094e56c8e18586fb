// Front-to-back compositing of one 16x16 screen tile per CTA (Sec. 3 "Scalar rendering
// function": rho = alpha k, T = prod (1 - rho), a = c rho T, A = sum a) and the
// per-Gaussian sensitivity reduction (Eq. sen).
//
// Each thread owns one pixel; a warp covers an 8x4 pixel block.  The tile's
// depth-sorted splat list is staged through shared memory 256 records at a time.
// While staging, each splat gets a mask of the warp blocks its footprint reaches (the
// ellipse's exact extent over each 4-row band), and every warp compacts the batch into
// its own list, so a warp only evaluates splats that can reach one of its pixels.
// Pass 2 of the two-pass modes reuses pass 1's masks (one 8-bit mask per tile-list entry
// kept in global memory).
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
// Score (per-scene, per-image and per-tile resolutions) is one pass: warp sums of a (16
// entries per vector-halving butterfly), one global atomicAdd per (tile, Gaussian), and the
// CTA's sum of A added to an FP64 total.
#include "csgs_internal.cuh"

namespace csgs {
namespace {

// CTA layout for tiles of 2^LW x 2^LH pixels: one thread per pixel, 8x4-pixel warps in
// kCols columns and kBands 4-row bands (warp w = column + kCols band), so a warp mask has
// kWarps <= 8 bits.
template <int LW, int LH>
struct TileCfg {
    static constexpr int kLw = LW, kLh = LH;
    static constexpr int kW = 1 << LW, kH = 1 << LH;
    static constexpr int kCols = kW / 8, kBands = kH / 4;
    static constexpr int kWarps = kCols * kBands, kThreads = 32 * kWarps;
    // pixel (lx, ly) of the tile sits at (lx - kHx, ly - kHy) from the tile centre
    static constexpr float kHx = 0.5f * (float)(kW - 1), kHy = 0.5f * (float)(kH - 1);
    static_assert(kCols >= 1 && kBands >= 1 && kWarps <= 8, "warp masks are 8 bits per tile-list entry");
};
using Tile16x16 = TileCfg<4, 4>;
using Tile32x8 = TileCfg<5, 3>;
using Tile16x8 = TileCfg<4, 3>;
using Tile8x8 = TileCfg<3, 3>;

// Modes: the render, and the query resolutions of Sec. 3.5.  Pixel and channel
// resolutions run two passes (A(q) first); tile, image and scene are one pass that
// sums each Gaussian's terms over the query's pixels (warp sums).
enum { kRender = 0, kScorePixel = 1, kScoreChannel = 2, kScoreTile = 3, kScoreImage = 4, kScoreScene = 5,
       kTransfer = 6 };
// Score variants (Sec. 3.5 "Additional variants"): a = c rho T, (c rho T)^2, rho T.
enum { kL1 = 0, kL2 = 1, kNC = 2 };

__host__ __device__ constexpr bool two_pass(int mode) { return mode == kScorePixel || mode == kScoreChannel; }
__host__ __device__ constexpr bool summed(int mode) {
    return mode == kScoreTile || mode == kScoreImage || mode == kScoreScene;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Single-instruction approximations (relative error ~2^-22) for the conservative culling
// bounds, which carry margins far larger than that.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <class TC>
struct Shared {
    static constexpr int NT = TC::kThreads, NW = TC::kWarps;
    float4 A[NT];  // s1, s1k, c1, s2
    float4 B[NT];  // c2, log2 alpha, thr, cw = obj_w . rgb
    float4 C[NT];  // r, g, b, cw2 = obj_w . rgb^2
    uint32_t gid[NT];
    float wsel[NT];  // transfer: the coreset weight w_i of the staged splat
    uint32_t msk[NT];
    uint16_t wl[NW][NT];  // per-warp compacted batch: byte offsets 16 x slot
    union {
        uint32_t red[4 * NT];  // two-pass modes: pass-2 maxima, word 0 of each 16-byte slot
        float part[NW][NT];    // summed modes: the warps' term sums per slot
    };
    int last;
    int item;  // persistent launch: the queue position the CTA took
    double sumA[NW];
};

// Stage splat i of the tile list into slot threadIdx.x (tile centre (cx, cy)).  MSK = 1:
// also store the warp mask per tile-list entry (pass 1 of the two-pass modes); MSK = 2:
// load it instead of recomputing it (pass 2).
template <int MODE, int MSK, class TC>
__device__ __forceinline__ void stage(const CompositeArgs& a, Shared<TC>& sh, uint32_t i, uint32_t end, float cx,
                                      float cy) {
    const int tid = threadIdx.x;
    if (two_pass(MODE)) sh.red[4 * tid] = 0u;
    if (summed(MODE))
#pragma unroll
        for (int w = 0; w < TC::kWarps; ++w) sh.part[w][tid] = 0.f;
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
    sh.C[tid] = make_float4(c.x, c.y, c.z, a.o.ow0 * c.x * c.x + a.o.ow1 * c.y * c.y + a.o.ow2 * c.z * c.z);
    sh.gid[tid] = g;
    if (MODE == kTransfer) sh.wsel[tid] = __ldg(a.wsel + g);
    if (MSK == 2) {
        sh.msk[tid] = a.mskbuf[i];
        return;
    }
    // Warp-block mask.  The test p >= thr is the ellipse e1^2 + e2^2 <= R with R =
    // log2 alpha - thr (the 3-sigma cut and the alpha_min skip in one), e1 = s1 u + s1k v,
    // e2 = s2 v, (u, v) = pixel - mean.  For each 4-row band of warp blocks, take the
    // exact x-extent of the ellipse over the band's v-interval: the right end
    // (sqrt(R - (s2 v)^2) - s1k v) / s1 is concave in v with its maximum at
    // v* = -s1k sqrt(R) / (s2 sqrt(s1k^2 + s2^2)) (the left end mirrors it at -v*), so
    // clamping v* to the interval gives the band's extreme.  R and every bound are
    // padded so that FP32 rounding (and the approximate square roots and reciprocals)
    // never drops a pixel that passes the test.
    const float R = fmaf(fmaxf(c.w - q.w, 0.f), 1.002f, 1e-5f);
    const float sR = sqrt_approx(R);
    const float i1 = rcp_approx(s1), i2 = rcp_approx(s2);
    const float vmax = sR * i2 * 1.001f + 0.01f;
    const float vstar = -s1k * sR * i2 * rsqrt_approx(fmaf(s1k, s1k, s2 * s2));
    uint32_t mk = 0u;
    // band r covers the rows 4r .. 4r + 3 (y = 4r - kHy .. 4r + 3 - kHy from the centre), warp
    // column c the columns 8c .. 8c + 7; the bounds are padded by 0.02 px
    constexpr float y0 = -TC::kHy - 0.02f, y1 = 3.f - TC::kHy + 0.02f;
#pragma unroll
    for (int r = 0; r < TC::kBands; ++r) {
        const float va = fmaxf(y0 + 4.f * r - my, -vmax);
        const float vb = fminf(y1 + 4.f * r - my, vmax);
        if (!(va <= vb)) continue;
        const float vr = fminf(fmaxf(vstar, va), vb);
        const float vl = fminf(fmaxf(-vstar, va), vb);
        const float er = s2 * vr, el = s2 * vl;
        const float wr = sqrt_approx(fmaxf(fmaf(-er, er, R), 0.f));
        const float wl = sqrt_approx(fmaxf(fmaf(-el, el, R), 0.f));
        const float xr = mx + (wr - s1k * vr) * i1;
        const float xl = mx - (wl + s1k * vl) * i1;
        const float pad = 0.02f + 1e-3f * (wr + wl) * i1;
        uint32_t cols = 0u;
#pragma unroll
        for (int c = 0; c < TC::kCols; ++c) {
            const float xa = 8.f * c - TC::kHx, xb = 8.f * c + 7.f - TC::kHx;
            cols |= (xl - pad <= xb && xr + pad >= xa) ? 1u << c : 0u;
        }
        mk |= cols << (TC::kCols * r);
    }
    sh.msk[tid] = mk;
    if (MSK == 1) a.mskbuf[i] = (uint8_t)mk;
}

// Staged record at byte offset off (16 x slot) of a float4 array in shared memory: the
// warp lists hold these offsets, so a list entry addresses its records without scaling.
__device__ __forceinline__ float4 at16(const float4* base, uint32_t off) {
    return *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) + off);
}

// Compact the staged batch into this warp's list (byte offsets 16 x slot); returns its
// length.
template <class TC>
__device__ __forceinline__ int warp_list(Shared<TC>& sh, int cnt, int warp, int lane) {
    const uint32_t lt = (1u << lane) - 1u;
    int nw = 0;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int j = c0 + lane;
        const bool bit = j < cnt && ((sh.msk[j] >> warp) & 1u);
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        if (bit) sh.wl[warp][nw + __popc(bal & lt)] = (uint16_t)(j << 4);
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

// Per-channel accumulation of pass 1 (render: the colours; scores: the variant's
// per-channel terms, whose sums are the per-channel objectives A_lambda).
template <int MODE, int VAR>
__device__ __forceinline__ void accumulate(float& A0, float& A1, float& A2, const float4& Cj, float w) {
    if (MODE == kRender || VAR == kL1) {
        A0 = __fmaf_rn(Cj.x, w, A0);
        A1 = __fmaf_rn(Cj.y, w, A1);
        A2 = __fmaf_rn(Cj.z, w, A2);
    } else if (VAR == kL2) {
        const float a0 = __fmul_rn(Cj.x, w), a1 = __fmul_rn(Cj.y, w), a2 = __fmul_rn(Cj.z, w);
        A0 = __fmaf_rn(a0, a0, A0);
        A1 = __fmaf_rn(a1, a1, A1);
        A2 = __fmaf_rn(a2, a2, A2);
    } else {
        A0 = __fadd_rn(A0, w);
    }
}

// The pixel-aggregated term a of a contributor with w = rho T.
template <int VAR>
__device__ __forceinline__ float pixel_term(float w, const float4& Bj, const float4& Cj) {
    if (VAR == kL1) return __fmul_rn(Bj.w, w);
    if (VAR == kL2) return __fmul_rn(Cj.w, __fmul_rn(w, w));
    return w;
}

template <int VAR>
__device__ __forceinline__ float pixel_objective(const KOpts& o, float A0, float A1, float A2) {
    if (VAR == kNC) return A0;
    return o.ow0 * A0 + o.ow1 * A1 + o.ow2 * A2;
}

// The per-pixel objective after pass 1: the per-pixel score accumulates it directly in A0
// (one FMA per contributor), the other modes per channel.
template <int MODE, int VAR>
__device__ __forceinline__ float pass1_objective(const KOpts& o, float A0, float A1, float A2) {
    if (MODE == kScorePixel) return A0;
    return pixel_objective<VAR>(o, A0, A1, A2);
}

// One tile of the view (all threads of the CTA; shared memory is free again on return).
template <int MODE, int VAR, bool STATS, class TC>
__device__ __forceinline__ void composite_tile(const CompositeArgs& a, Shared<TC>& sh, const int tile) {
    constexpr int kThreads = TC::kThreads, kWarps = TC::kWarps;
    const CamDev& cam = a.cam;
    const int ntx = tiles_x_of(cam, TC::kLw);
    const int tx = tile % ntx, ty = tile / ntx;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lx = (warp % TC::kCols) * 8 + (lane & 7), ly = (warp / TC::kCols) * 4 + (lane >> 3);
    const int px = (tx << TC::kLw) + lx, py = (ty << TC::kLh) + ly;
    const bool inside = px < cam.W && py < cam.H;
    const float X = (float)lx - TC::kHx, Y = (float)ly - TC::kHy;
    const float cx = (float)(tx << TC::kLw) + TC::kHx, cy = (float)(ty << TC::kLh) + TC::kHy;
    const uint2 rg = a.ranges[tile];
    const uint32_t start = rg.x;
    const int n = (int)(rg.y - rg.x);
    const float rho_max = a.o.rho_max, t_min = a.o.t_min;

    float T = 1.f, A0 = 0.f, A1 = 0.f, A2 = 0.f;
    float tr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // transfer: A_th[3], A_w[3]
    float Tw = 1.f, gam = 0.f, minf = 1.f;
    int last16 = 0;  // 16 x (index past the pixel's last contributor)
    int processed = 0;  // tile-list entries staged by pass 1 (CTA-uniform)
    bool done = !inside;
    unsigned long long n_eval = 0, n_hit = 0, n_viol = 0, n_went1 = 0, n_went2 = 0;
    if (tid == 0) sh.last = 0;

    // ---------------------------------------------------------------- pass 1
    for (int b = 0; b < n; b += kThreads) {
        if (__syncthreads_count(done) == kThreads) break;
        stage<MODE, two_pass(MODE) ? 1 : 0, TC>(a, sh, start + b + tid, rg.y, cx, cy);
        __syncthreads();
        const int cnt = min(kThreads, n - b);
        processed = b + cnt;
        const int nw = warp_list(sh, cnt, warp, lane);
        if (MODE == kTransfer) {
            // full-scene order with T and the reduced scene's T_w side by side
            for (int k = 0; k < nw && !done; ++k) {
                const int j = sh.wl[warp][k] >> 4;
                const float4 Aj = sh.A[j];
                const float4 Bj = sh.B[j];
                const float p = exponent2(Aj, Bj, X, Y);
                if (p < Bj.z) continue;
                const float r = fminf(rho_max, ex2_approx(p));
                const float4 Cj = sh.C[j];
                const float w = __fmul_rn(r, T);
                A0 = __fmaf_rn(Cj.x, w, A0);
                A1 = __fmaf_rn(Cj.y, w, A1);
                A2 = __fmaf_rn(Cj.z, w, A2);
                const float wi = sh.wsel[j];
                if (wi > 0.f) {
                    const float wt = __fmul_rn(wi, w);
                    tr[0] = __fmaf_rn(Cj.x, wt, tr[0]);
                    tr[1] = __fmaf_rn(Cj.y, wt, tr[1]);
                    tr[2] = __fmaf_rn(Cj.z, wt, tr[2]);
                    const float ww = __fmul_rn(__fmul_rn(wi, r), Tw);
                    tr[3] = __fmaf_rn(Cj.x, ww, tr[3]);
                    tr[4] = __fmaf_rn(Cj.y, ww, tr[4]);
                    tr[5] = __fmaf_rn(Cj.z, ww, tr[5]);
                    if (T > 0.f && Tw > 0.f) gam = fmaxf(gam, fabsf(log2f(T) - log2f(Tw)) * 0.69314718055994531f);
                }
                const float f = __fadd_rn(1.f, -__fmul_rn(wi, r));
                minf = fminf(minf, f);
                Tw = __fmul_rn(Tw, f);
                const float Tn = __fmul_rn(T, __fadd_rn(1.f, -r));
                if (Tn < t_min) done = true;  // t_min = 0 in the pure setting: never
                T = Tn;
            }
        } else if (!summed(MODE)) {
            int kmax = 0;  // counting runs: entries this lane walked (the warp walks the maximum)
            const int b16 = (b + 1) << 4;
            // one list entry (byte offset jo) at pixel (X, Y): false once the pixel has stopped
            auto step = [&](uint32_t jo, const float4& Bj, float p) -> bool {
                if (STATS) ++n_eval;
                if (p < Bj.z) return true;
                const float raw = ex2_approx(p);
                const float r = fminf(rho_max, raw);
                if (STATS) {
                    ++n_hit;
                    n_viol += raw >= 1.f;
                }
                // T (1 - rho) rounded once, as T - T rho
                const float Tn = __fmaf_rn(-T, r, T);
                if (Tn < t_min) {
                    done = true;
                    return false;
                }
                const float w = __fmul_rn(r, T);
                if (MODE == kScorePixel)
                    A0 = VAR == kL1 ? __fmaf_rn(Bj.w, w, A0)
                                    : (VAR == kL2 ? __fmaf_rn(at16(sh.C, jo).w, __fmul_rn(w, w), A0) : __fadd_rn(A0, w));
                else
                    accumulate<MODE, VAR>(A0, A1, A2, at16(sh.C, jo), w);
                T = Tn;
                last16 = b16 + (int)jo;
                return true;
            };
            if (!done) {
                // two entries per iteration: the second entry's loads and exponent are
                // independent of the first's contribution, so they overlap its latency; the
                // entries are still applied in list order
                int k = 0;
                for (; k + 1 < nw; k += 2) {
                    const uint32_t j0 = sh.wl[warp][k], j1 = sh.wl[warp][k + 1];
                    const float4 Aa = at16(sh.A, j0), Ba = at16(sh.B, j0), Ab = at16(sh.A, j1), Bb = at16(sh.B, j1);
                    const float pa = exponent2(Aa, Ba, X, Y), pb = exponent2(Ab, Bb, X, Y);
                    if (STATS) kmax = k + 1;
                    if (!step(j0, Ba, pa)) break;
                    if (STATS) kmax = k + 2;
                    if (!step(j1, Bb, pb)) break;
                }
                if (!done && k < nw) {
                    const uint32_t j = sh.wl[warp][k];
                    const float4 Aj = at16(sh.A, j), Bj = at16(sh.B, j);
                    if (STATS) kmax = k + 1;
                    step(j, Bj, exponent2(Aj, Bj, X, Y));
                }
            }
            if (STATS) {
                const int wk = (int)__reduce_max_sync(0xffffffffu, (unsigned)kmax);
                if (lane == 0) n_went1 += wk;
            }
        } else {
            // summed resolutions: warp-uniform loop over chunks of 16 entries; the warp's sum
            // of each entry's terms comes from one vector-halving butterfly per chunk
            bool act = !done;
            if (__any_sync(0xffffffffu, act)) {
                for (int k0 = 0; k0 < nw; k0 += 16) {
                    float v[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        v[u] = 0.f;
                        if (k0 + u < nw && act) {
                            const int j = sh.wl[warp][k0 + u] >> 4;
                            const float4 Aj = sh.A[j];
                            const float4 Bj = sh.B[j];
                            const float p = exponent2(Aj, Bj, X, Y);
                            if (STATS) ++n_eval;
                            if (p >= Bj.z) {
                                const float r = fminf(rho_max, ex2_approx(p));
                                if (STATS) ++n_hit;
                                const float Tn = __fmaf_rn(-T, r, T);
                                if (Tn < t_min) {
                                    act = false;
                                    done = true;
                                } else {
                                    const float w = __fmul_rn(r, T);
                                    const float4 Cj = sh.C[j];
                                    accumulate<MODE, VAR>(A0, A1, A2, Cj, w);
                                    v[u] = pixel_term<VAR>(w, Bj, Cj);
                                    T = Tn;
                                }
                            }
                        }
                    }
                    const float cs = warp_colsum16(v, lane);
                    const int c = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                                  ((lane >> 1) & 1);
                    if ((lane & 1) == 0 && k0 + c < nw) sh.part[warp][sh.wl[warp][k0 + c] >> 4] = cs;
                    if (!__any_sync(0xffffffffu, act)) break;
                }
            }
            __syncthreads();
            if (tid < cnt) {
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) v += sh.part[w][tid];
                if (MODE == kScoreTile)
                    a.tile_sum[start + b + tid] = v;
                else if (v > 0.f)
                    atomicAdd(a.s_sum + sh.gid[tid], v);
            }
        }
    }

    int last = last16 >> 4;
    if (MODE == kRender) {
        if (inside) {
            const size_t pix = (size_t)py * cam.W + px;
            a.rgb[3 * pix + 0] = A0;
            a.rgb[3 * pix + 1] = A1;
            a.rgb[3 * pix + 2] = A2;
            if (a.T) a.T[pix] = T;
            if (a.last) a.last[pix] = last;
        }
    }

    if (MODE == kTransfer && inside) {
        float* o = a.aux + ((size_t)py * cam.W + px) * 11;
        o[0] = A0;
        o[1] = A1;
        o[2] = A2;
#pragma unroll
        for (int k = 0; k < 6; ++k) o[3 + k] = tr[k];
        o[9] = gam;
        o[10] = minf;
    }

    if (two_pass(MODE)) {
        // |Q'|: pixel queries with a non-zero objective
        const bool nz = inside && pass1_objective<MODE, VAR>(a.o, A0, A1, A2) > 0.f;
        const unsigned c = __popc(__ballot_sync(0xffffffffu, nz));
        if (lane == 0 && c) atomicAdd(&a.ctr->queries, (unsigned long long)c);
    }

    if (summed(MODE)) {
        // CTA sum of the pixel objective: the tile query's A, or a share of the
        // image / scene query's A (FP64 totals)
        double Ao = inside ? (double)pixel_objective<VAR>(a.o, A0, A1, A2) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Ao += __shfl_xor_sync(0xffffffffu, Ao, o);
        __syncthreads();
        if (lane == 0) sh.sumA[warp] = Ao;
        __syncthreads();
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += sh.sumA[w];
        if (MODE == kScoreScene && tid == 0 && t > 0.0) atomicAdd(&a.ctr->sumA, t);
        if (MODE == kScoreImage && tid == 0 && t > 0.0) atomicAdd(&a.ctr->sumA_view, t);
        if (MODE == kScoreTile && t > 0.0) {
            // imp(g, tile) = (sum of g's terms over the tile) / A(tile)
            const double inv = 1.0 / t;
            for (int i = tid; i < processed; i += kThreads) {
                const float v = a.tile_sum[start + i];
                if (v > 0.f) {
                    const uint32_t g = __ldg(a.inst_gid + start + i);
                    if (g < (uint32_t)a.n_gauss) atomicMax(a.s_bits + g, __float_as_uint((float)((double)v * inv)));
                }
            }
        }
    }

    // ---------------------------------------------------------------- pass 2
    unsigned long long n_eval2 = 0, n_hit2 = 0;
    if (two_pass(MODE)) {
        // queries with A = 0 are discarded (Sec. 3.2)
        float inv0 = 0.f, inv1 = 0.f, inv2 = 0.f;
        bool has;
        if (MODE == kScorePixel) {
            const float Aobj = pass1_objective<MODE, VAR>(a.o, A0, A1, A2);
            has = inside && Aobj > 0.f;
            inv0 = has ? 1.f / Aobj : 0.f;
        } else {
            inv0 = A0 > 0.f ? 1.f / A0 : 0.f;
            inv1 = A1 > 0.f ? 1.f / A1 : 0.f;
            inv2 = A2 > 0.f ? 1.f / A2 : 0.f;
            if (VAR == kNC) inv1 = inv2 = inv0;
            has = inside && (inv0 > 0.f || inv1 > 0.f || inv2 > 0.f);
        }
        // pixel resolution with a term linear in T: track T / A directly
        constexpr bool kScaled = MODE == kScorePixel && VAR != kL2;
        T = kScaled ? inv0 : 1.f;
        if (!has) last = 0;
        __syncthreads();
        atomicMax(&sh.last, last);
        __syncthreads();
        const int n2 = sh.last;
        for (int b = 0; b < n2; b += kThreads) {
            __syncthreads();
            stage<MODE, 2, TC>(a, sh, start + b + tid, rg.y, cx, cy);
            __syncthreads();
            const int cnt = min(kThreads, n2 - b);
            const int lim = max(0, min(cnt, last - b));
            const uint32_t lim16 = (uint32_t)lim << 4;
            // the warp's list holds only entries below its lanes' largest contributor bound
            const int jw = (int)__reduce_max_sync(0xffffffffu, (unsigned)lim);
            const int nw = warp_list(sh, jw, warp, lane);
            if (STATS && lane == 0) n_went2 += nw;
            // 16 entries per unrolled iteration for the per-pixel score (408 against 413 us per
            // view at 8, 418 at 4); the per-channel score stays at 4 (at 8 it needs 48 registers)
            constexpr int kUnroll2 = MODE == kScorePixel ? 16 : 4;
#pragma unroll kUnroll2
            for (int k = 0; k < nw; ++k) {
                const uint32_t jo = sh.wl[warp][k];
                // branch-free: every lane evaluates the entry and keeps the result only where
                // it is one of its pass-1 contributors (the warp takes this path anyway as
                // soon as one lane contributes)
                const float4 Aj = at16(sh.A, jo);
                const float4 Bj = at16(sh.B, jo);
                const float p = exponent2(Aj, Bj, X, Y);
                const bool hit = jo < lim16 && p >= Bj.z;
                if (STATS) {
                    n_eval2 += jo < lim16;
                    n_hit2 += hit;
                }
                // a pair outside the pixel's contributor set gets rho = 0: its term is +0
                // (bits 0) and T - T 0 = T exactly
                const float r1 = fminf(rho_max, ex2_approx(p));
                const float r = hit ? r1 : 0.f;
                const float w = __fmul_rn(r, T);
                float imp;
                if (kScaled) {
                    imp = VAR == kL1 ? __fmul_rn(Bj.w, w) : w;
                } else if (MODE == kScorePixel) {
                    imp = __fmul_rn(pixel_term<VAR>(w, Bj, at16(sh.C, jo)), inv0);
                } else {
                    const float4 Cj = at16(sh.C, jo);
                    float t0, t1, t2;
                    if (VAR == kL1) {
                        t0 = __fmul_rn(Cj.x, w);
                        t1 = __fmul_rn(Cj.y, w);
                        t2 = __fmul_rn(Cj.z, w);
                    } else if (VAR == kL2) {
                        t0 = __fmul_rn(Cj.x, w);
                        t1 = __fmul_rn(Cj.y, w);
                        t2 = __fmul_rn(Cj.z, w);
                        t0 = __fmul_rn(t0, t0);
                        t1 = __fmul_rn(t1, t1);
                        t2 = __fmul_rn(t2, t2);
                    } else {
                        t0 = t1 = t2 = w;
                    }
                    imp = fmaxf(__fmul_rn(t0, inv0), fmaxf(__fmul_rn(t1, inv1), __fmul_rn(t2, inv2)));
                }
                const uint32_t bits = __float_as_uint(imp);
                T = __fmaf_rn(-T, r, T);
                const uint32_t mx = __reduce_max_sync(0xffffffffu, bits);
                if (lane == 0) atomicMax(reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(sh.red) + jo), mx);
            }
            __syncthreads();
            if (tid < cnt) {
                const uint32_t v = sh.red[4 * tid];
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
        if (tid == 0) {
            atomicAdd(&a.ctr->staged1, (unsigned long long)processed);
            if (two_pass(MODE)) atomicAdd(&a.ctr->staged2, (unsigned long long)sh.last);
        }
        if (lane == 0) {
            if (e) atomicAdd(&a.ctr->pairs_eval, e);
            if (h) atomicAdd(&a.ctr->pairs_hit, h);
            if (e2) atomicAdd(&a.ctr->pairs_eval2, e2);
            if (h2) atomicAdd(&a.ctr->pairs_hit2, h2);
            if (vv) atomicAdd(&a.ctr->violations, vv);
            if (n_went1) atomicAdd(&a.ctr->wentries1, n_went1);
            if (n_went2) atomicAdd(&a.ctr->wentries2, n_went2);
        }
    }
}

// A launch of one CTA per tile (CTA b takes tile order[b]), or a persistent launch
// (PERSIST): fewer CTAs, each taking the next position of the order from a counter
// (a.work, zero at launch) until the view's tiles are used up.
template <int MODE, int VAR, bool STATS, class TC, bool PERSIST>
__global__ void __launch_bounds__(TC::kThreads) k_composite(const CompositeArgs a) {
    __shared__ Shared<TC> sh;
    if (!PERSIST) {
        composite_tile<MODE, VAR, STATS, TC>(a, sh, a.order ? (int)__ldg(a.order + blockIdx.x) : (int)blockIdx.x);
        return;
    }
    const int T = tiles_of(a.cam, TC::kLw, TC::kLh);
    for (;;) {
        if (threadIdx.x == 0) sh.item = (int)atomicAdd(a.work, 1u);
        __syncthreads();
        const int item = sh.item;
        __syncthreads();  // every thread has read the position before the next one is taken
        if (item >= T) break;
        composite_tile<MODE, VAR, STATS, TC>(a, sh, a.order ? (int)__ldg(a.order + item) : item);
    }
}

// Backward of the render (Sec. 3's compositing, back to front): for contributor i of a
// pixel, with S the colour composited behind it,
//   dC/dc_i = rho_i T_i,  dC/drho_i = c_i T_i - S / (1 - rho_i),  T_i = T_{i+1} / (1 - rho_i),
// rho_i = min(rho_max, alpha k) (no gradient through the clamp), k = exp(-m / 2),
// m = d^T Q d, d = pixel - mean.  rho is recomputed exactly as in the forward pass and
// the contributor set is the forward's (the pixel's last contributor).  Per-Gaussian
// sums over the tile's pixels: warp sums, shared-memory sums, one global add per
// (tile, Gaussian) and component.
__global__ void __launch_bounds__(Tile16x16::kThreads) k_composite_bwd(const CompositeArgs a) {
    using TC = Tile16x16;
    constexpr int kThreads = TC::kThreads;
    __shared__ Shared<TC> sh;
    __shared__ float4 sD[kThreads];      // mean x, mean y (tile-centred), Q xx, Q xy
    __shared__ float2 sE[kThreads];      // Q yy, alpha
    __shared__ float acc[kThreads][9];
    const CamDev& cam = a.cam;
    const int tile = blockIdx.x;
    const int ntx = tiles_x_of(cam, TC::kLw);
    const int tx = tile % ntx, ty = tile / ntx;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lx = (warp % TC::kCols) * 8 + (lane & 7), ly = (warp / TC::kCols) * 4 + (lane >> 3);
    const int px = (tx << TC::kLw) + lx, py = (ty << TC::kLh) + ly;
    const bool inside = px < cam.W && py < cam.H;
    const float X = (float)lx - TC::kHx, Y = (float)ly - TC::kHy;
    const float cx = (float)(tx << TC::kLw) + TC::kHx, cy = (float)(ty << TC::kLh) + TC::kHy;
    const uint2 rg = a.ranges[tile];
    const uint32_t start = rg.x;
    const float rho_max = a.o.rho_max;
    const float K2inv = 1.f / (0.5f * kLog2e);
    const size_t pix = (size_t)py * cam.W + px;
    float T = inside ? a.T[pix] : 1.f;
    int last = inside ? a.last[pix] : 0;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (inside) {
        g0 = a.grad_rgb[3 * pix];
        g1 = a.grad_rgb[3 * pix + 1];
        g2 = a.grad_rgb[3 * pix + 2];
    }
    float S0 = 0.f, S1 = 0.f, S2 = 0.f;
    if (tid == 0) sh.last = 0;
    __syncthreads();
    atomicMax(&sh.last, last);
    __syncthreads();
    const int n2 = sh.last;
    for (int b = ((n2 - 1) / kThreads) * kThreads; n2 > 0 && b >= 0; b -= kThreads) {
        __syncthreads();
        stage<kRender, 0, TC>(a, sh, start + b + tid, rg.y, cx, cy);
        {
            const float4 Aj = sh.A[tid];
            // tile-centred mean and natural-unit conic back from the Cholesky form
            const float s1 = Aj.x, s1k = Aj.y, s2 = Aj.w;
            const float my = -sh.B[tid].x / s2;
            const float mx = -(Aj.z + s1k * my) / s1;
            sD[tid] = make_float4(mx, my, s1 * s1 * K2inv, s1 * s1k * K2inv);
            sE[tid] = make_float2((s1k * s1k + s2 * s2) * K2inv, exp2f(sh.B[tid].y));
#pragma unroll
            for (int c = 0; c < 9; ++c) acc[tid][c] = 0.f;
        }
        __syncthreads();
        const int cnt = min(kThreads, n2 - b);
        const int nw = warp_list(sh, cnt, warp, lane);
        const int lim = max(0, min(cnt, last - b));
        for (int k = nw - 1; k >= 0; --k) {
            const int j = sh.wl[warp][k] >> 4;
            float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool any = false;
            if (j < lim) {
                const float4 Aj = sh.A[j];
                const float4 Bj = sh.B[j];
                const float p = exponent2(Aj, Bj, X, Y);
                if (p >= Bj.z) {
                    any = true;
                    const float raw = ex2_approx(p);
                    const float r = fminf(rho_max, raw);
                    const float Ti = T / (1.f - r);
                    const float4 Cj = sh.C[j];
                    const float rT = r * Ti;
                    v[6] = g0 * rT;
                    v[7] = g1 * rT;
                    v[8] = g2 * rT;
                    const float inv1 = 1.f / (1.f - r);
                    const float drho = g0 * (Cj.x * Ti - S0 * inv1) + g1 * (Cj.y * Ti - S1 * inv1) +
                                       g2 * (Cj.z * Ti - S2 * inv1);
                    S0 = fmaf(Cj.x, rT, S0);
                    S1 = fmaf(Cj.y, rT, S1);
                    S2 = fmaf(Cj.z, rT, S2);
                    T = Ti;
                    if (raw < rho_max) {
                        const float4 D = sD[j];
                        const float2 E = sE[j];
                        v[5] = drho * raw / E.y;
                        const float dm = -0.5f * raw * drho;
                        const float dx = X - D.x, dy = Y - D.y;
                        v[0] = -2.f * dm * (D.z * dx + D.w * dy);
                        v[1] = -2.f * dm * (D.w * dx + E.x * dy);
                        v[2] = dm * dx * dx;
                        v[3] = 2.f * dm * dx * dy;
                        v[4] = dm * dy * dy;
                    }
                }
            }
            if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    float x = v[c];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    if (lane == 0 && x != 0.f) atomicAdd(&acc[j][c], x);
                }
            }
        }
        __syncthreads();
        if (tid < cnt && sh.msk[tid]) {
            const uint32_t g = sh.gid[tid];
#pragma unroll
            for (int c = 0; c < 9; ++c)
                if (acc[tid][c] != 0.f) atomicAdd(a.g2d + (size_t)g * 9 + c, acc[tid][c]);
        }
    }
}

}  // namespace

// The backward and the per-tile resolution (whose query is a 16x16 tile) run on 16x16 tiles
// only; the other modes on the shape in a.o (tile_lw, tile_lh).
int composite_resident_ctas(int lw, int lh) {
    int r = 0;
    if (lw == 5 && lh == 3)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_composite<kScorePixel, kL1, false, Tile32x8, true>,
                                                      Tile32x8::kThreads, 0);
    else if (lw == 4 && lh == 3)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_composite<kScorePixel, kL1, false, Tile16x8, true>,
                                                      Tile16x8::kThreads, 0);
    else if (lw == 3 && lh == 3)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_composite<kScorePixel, kL1, false, Tile8x8, true>,
                                                      Tile8x8::kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_composite<kScorePixel, kL1, false, Tile16x16, true>,
                                                      Tile16x16::kThreads, 0);
    return r;
}

void launch_composite_backward(const CompositeArgs& a, cudaStream_t st) {
    const int tiles = tiles_of(a.cam, Tile16x16::kLw, Tile16x16::kLh);
    k_composite_bwd<<<tiles, Tile16x16::kThreads, 0, st>>>(a);
    count_launches(1);
}

template <int MODE, int VAR, bool STATS, class TC>
static void launch_one(const CompositeArgs& a, cudaStream_t st) {
    const int tiles = tiles_of(a.cam, TC::kLw, TC::kLh);
    // persistent launches for the per-pixel score (the timed path); the other modes take
    // one CTA per tile
    if (MODE == kScorePixel && a.work && a.o.persist_ctas > 0 && a.o.persist_ctas < tiles)
        k_composite<MODE, VAR, STATS, TC, MODE == kScorePixel><<<a.o.persist_ctas, TC::kThreads, 0, st>>>(a);
    else
        k_composite<MODE, VAR, STATS, TC, false><<<tiles, TC::kThreads, 0, st>>>(a);
}

template <int MODE, int VAR, bool STATS>
static void launch_shape(const CompositeArgs& a, cudaStream_t st) {
    if (MODE != kScoreTile && a.o.tile_lw == 5 && a.o.tile_lh == 3)
        launch_one<MODE, VAR, STATS, Tile32x8>(a, st);
    else if (MODE != kScoreTile && a.o.tile_lw == 4 && a.o.tile_lh == 3)
        launch_one<MODE, VAR, STATS, Tile16x8>(a, st);
    else if (MODE != kScoreTile && a.o.tile_lw == 3 && a.o.tile_lh == 3)
        launch_one<MODE, VAR, STATS, Tile8x8>(a, st);
    else
        launch_one<MODE, VAR, STATS, Tile16x16>(a, st);
}

void launch_composite_transfer(const CompositeArgs& a, cudaStream_t st) {
    launch_shape<kTransfer, kL1, false>(a, st);
    count_launches(1);
}

void launch_composite_render(const CompositeArgs& a, cudaStream_t st) {
    if (a.stats)
        launch_shape<kRender, kL1, true>(a, st);
    else
        launch_shape<kRender, kL1, false>(a, st);
    count_launches(1);
}

template <int MODE, int VAR>
static void launch_mode(const CompositeArgs& a, cudaStream_t st) {
    if (a.stats)
        launch_shape<MODE, VAR, true>(a, st);
    else
        launch_shape<MODE, VAR, false>(a, st);
}

template <int MODE>
static void launch_var(const CompositeArgs& a, cudaStream_t st) {
    switch (a.o.variant) {
        case CSGS_VAR_L2: launch_mode<MODE, kL2>(a, st); break;
        case CSGS_VAR_NC: launch_mode<MODE, kNC>(a, st); break;
        default: launch_mode<MODE, kL1>(a, st); break;
    }
}

void launch_composite_score(const CompositeArgs& a, cudaStream_t st) {
    switch (a.o.resolution) {
        case CSGS_RES_SCENE: launch_var<kScoreScene>(a, st); break;
        case CSGS_RES_CHANNEL: launch_var<kScoreChannel>(a, st); break;
        case CSGS_RES_TILE: launch_var<kScoreTile>(a, st); break;
        case CSGS_RES_IMAGE: launch_var<kScoreImage>(a, st); break;
        default: launch_var<kScorePixel>(a, st); break;
    }
    count_launches(1);
}

}  // namespace csgs

// EWA projection of Gaussians into query views (the kernel k(g, q) of Sec. 3,
// "Scalar rendering function"), batched over views: each thread loads one
// Gaussian's attributes from the structure-of-arrays scene once (coalesced HBM
// reads), builds its 3-D covariance once, and projects it into every view of the
// batch.  Per (view, Gaussian) it writes a 48-byte splat record, a depth key and a
// tile rectangle.
#include <math.h>

#include "csgs_internal.cuh"
#include "ffmath.cuh"

namespace csgs {
namespace {

struct Proj {
    bool valid;
    ff::F2 mx, my;       // two-float pixel-space mean
    float ca, cb, cc;    // 2-D covariance (dilated)
    float ia, ib, ic;    // conic
    float idet;          // 1 / det(cov)
    float depth, op;
    float rgb[3];
    uint32_t tx0, ty0, tx1, ty1;
};

// Real SH basis (degree <= 3) along unit direction (x, y, z); the sign convention of
// the 3DGS colour model.  Constants are the closed-form normalisations.
template <int DEG>
__device__ __forceinline__ void sh_colour(const float* shc, float x, float y, float z, float rgb[3]) {
    float Y[16];
    Y[0] = 0.28209479177387814f;
    if (DEG >= 1) {
        Y[1] = -0.48860251190291992f * y;
        Y[2] = 0.48860251190291992f * z;
        Y[3] = -0.48860251190291992f * x;
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 1.0925484305920792f * x * y;
        Y[5] = -1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (2.f * zz - xx - yy);
        Y[7] = -1.0925484305920792f * x * z;
        Y[8] = 0.54627421529603959f * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -0.59004358992664352f * y * (3.f * xx - yy);
            Y[10] = 2.8906114426405538f * x * y * z;
            Y[11] = -0.45704579946446572f * y * (4.f * zz - xx - yy);
            Y[12] = 0.37317633259011540f * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -0.45704579946446572f * x * (4.f * zz - xx - yy);
            Y[14] = 1.4453057213202769f * z * (xx - yy);
            Y[15] = -0.59004358992664352f * x * (xx - 3.f * yy);
        }
    }
    constexpr int K = (DEG + 1) * (DEG + 1);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) acc = fmaf(shc[3 * k + ch], Y[k], acc);
        acc += 0.5f;
        rgb[ch] = fmaxf(acc, 0.f);
    }
}

// The EWA 2-D covariance (entries ca, cb, cc of Sigma' = J Sc J^T + dilation I) of a
// Gaussian with camera-space mean (x, y, z) and world covariance cov3.
__device__ __forceinline__ void ewa_cov2(const float cov3[6], const CamDev& c, const KOpts& o, float x, float y,
                                         float z, float& ca, float& cb, float& cc) {
    // camera-space covariance  Sc = R Sigma R^T   (Sigma symmetric: 00 01 02 11 12 22)
    const float s00 = cov3[0], s01 = cov3[1], s02 = cov3[2], s11 = cov3[3], s12 = cov3[4], s22 = cov3[5];
    float T[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float a0 = c.R[3 * i], a1 = c.R[3 * i + 1], a2 = c.R[3 * i + 2];
        T[3 * i + 0] = a0 * s00 + a1 * s01 + a2 * s02;
        T[3 * i + 1] = a0 * s01 + a1 * s11 + a2 * s12;
        T[3 * i + 2] = a0 * s02 + a1 * s12 + a2 * s22;
    }
    float Sc[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Sc[3 * i + j] = T[3 * i] * c.R[3 * j] + T[3 * i + 1] * c.R[3 * j + 1] + T[3 * i + 2] * c.R[3 * j + 2];

    // Jacobian of the perspective map linearised at the (clamped) mean
    const float invz = 1.f / z;
    float txz = fminf(fmaxf(x * invz, -c.limx), c.limx);
    float tyz = fminf(fmaxf(y * invz, -c.limy), c.limy);
    const float j00 = c.fx * invz, j02 = -c.fx * txz * invz;
    const float j11 = c.fy * invz, j12 = -c.fy * tyz * invz;
    // cov2 = J Sc J^T
    const float u0 = j00 * Sc[0] + j02 * Sc[6], u1 = j00 * Sc[1] + j02 * Sc[7], u2 = j00 * Sc[2] + j02 * Sc[8];
    const float v1 = j11 * Sc[4] + j12 * Sc[7], v2 = j11 * Sc[5] + j12 * Sc[8];
    ca = u0 * j00 + u2 * j02 + o.dilation;
    cb = u1 * j11 + u2 * j12;
    cc = v1 * j11 + v2 * j12 + o.dilation;
}

template <int DEG>
__device__ __forceinline__ void project_one(const float mu[3], const float cov3[6], float op, const float* shc,
                                            const CamDev& c, const KOpts& o, Proj& r) {
    r.valid = false;
    const ff::F2 X = ff::dot3_plus(c.R[0], c.R[1], c.R[2], c.t[0], mu[0], mu[1], mu[2]);
    const ff::F2 Yc = ff::dot3_plus(c.R[3], c.R[4], c.R[5], c.t[1], mu[0], mu[1], mu[2]);
    const ff::F2 Z = ff::dot3_plus(c.R[6], c.R[7], c.R[8], c.t[2], mu[0], mu[1], mu[2]);
    const float z = Z.hi;
    if (!(z > c.near_z)) return;
    if (!(op >= o.alpha_min)) return;  // rho <= alpha < alpha_min everywhere

    float ca, cb, cc;
    ewa_cov2(cov3, c, o, X.hi, Yc.hi, z, ca, cb, cc);
    // determinant with Kahan's compensated 2x2 formula
    float w = __fmul_rn(cb, cb);
    float e = __fmaf_rn(-cb, cb, w);
    float det = __fadd_rn(__fmaf_rn(ca, cc, -w), e);
    if (!(det > 0.f)) return;
    const float idet = 1.f / det;

    const ff::F2 mx = ff::persp(c.fx, X, Z, c.cx);
    const ff::F2 my = ff::persp(c.fy, Yc, Z, c.cy);

    // pixel bounding box of the ellipse d^T cov^-1 d <= m (|dx| <= sqrt(m cov_xx)), where
    // m = min(cut2, 2 ln(alpha / alpha_min)) also applies the alpha_min skip (alpha k <
    // alpha_min outside it); widened so FP32 rounding can never exclude a pixel that passes
    const float m_eff = fminf(o.cut2, fmaf(2.f / kLog2e, log2f(op) - o.l2amin, 1e-4f));
    const float rx = sqrtf(m_eff * ca) * 1.001f + 0.01f;
    const float ry = sqrtf(m_eff * cc) * 1.001f + 0.01f;
    float fx0 = ceilf(mx.hi - rx), fx1 = floorf(mx.hi + rx);
    float fy0 = ceilf(my.hi - ry), fy1 = floorf(my.hi + ry);
    fx0 = fmaxf(fx0, 0.f);
    fy0 = fmaxf(fy0, 0.f);
    fx1 = fminf(fx1, (float)(c.W - 1));
    fy1 = fminf(fy1, (float)(c.H - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return;
    r.tx0 = (uint32_t)fx0 >> o.tile_lw;
    r.ty0 = (uint32_t)fy0 >> o.tile_lh;
    r.tx1 = ((uint32_t)fx1 >> o.tile_lw) + 1;
    r.ty1 = ((uint32_t)fy1 >> o.tile_lh) + 1;

    // colour along camera centre -> mean
    float dx = mu[0] - c.campos[0], dy = mu[1] - c.campos[1], dz = mu[2] - c.campos[2];
    float inv = 1.f / sqrtf(dx * dx + dy * dy + dz * dz);
    sh_colour<DEG>(shc, dx * inv, dy * inv, dz * inv, r.rgb);

    r.valid = true;
    r.mx = mx;
    r.my = my;
    r.ca = ca;
    r.cb = cb;
    r.cc = cc;
    r.idet = idet;
    r.ia = cc * idet;
    r.ib = -cb * idet;
    r.ic = ca * idet;
    r.depth = z;
    r.op = op;
}

// Loads the Gaussian's attributes and builds Sigma = Rq diag(s)^2 Rq^T.
template <int DEG>
__device__ __forceinline__ void load_gaussian(const SceneDev& sc, int i, const float* wts, float mu[3], float cov3[6],
                                              float& op, float* shc) {
    const int n = sc.n;
    mu[0] = __ldg(sc.means + i);
    mu[1] = __ldg(sc.means + n + i);
    mu[2] = __ldg(sc.means + 2 * n + i);
    const float sx = expf(__ldg(sc.log_scales + i));
    const float sy = expf(__ldg(sc.log_scales + n + i));
    const float sz = expf(__ldg(sc.log_scales + 2 * n + i));
    float qw = __ldg(sc.quats + i), qx = __ldg(sc.quats + n + i), qy = __ldg(sc.quats + 2 * n + i),
          qz = __ldg(sc.quats + 3 * n + i);
    const float qn = 1.f / sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qn;
    qx *= qn;
    qy *= qn;
    qz *= qn;
    const float r00 = 1.f - 2.f * (qy * qy + qz * qz), r01 = 2.f * (qx * qy - qw * qz), r02 = 2.f * (qx * qz + qw * qy);
    const float r10 = 2.f * (qx * qy + qw * qz), r11 = 1.f - 2.f * (qx * qx + qz * qz), r12 = 2.f * (qy * qz - qw * qx);
    const float r20 = 2.f * (qx * qz - qw * qy), r21 = 2.f * (qy * qz + qw * qx), r22 = 1.f - 2.f * (qx * qx + qy * qy);
    // M = Rq diag(s); Sigma = M M^T
    const float m00 = r00 * sx, m01 = r01 * sy, m02 = r02 * sz;
    const float m10 = r10 * sx, m11 = r11 * sy, m12 = r12 * sz;
    const float m20 = r20 * sx, m21 = r21 * sy, m22 = r22 * sz;
    cov3[0] = m00 * m00 + m01 * m01 + m02 * m02;
    cov3[1] = m00 * m10 + m01 * m11 + m02 * m12;
    cov3[2] = m00 * m20 + m01 * m21 + m02 * m22;
    cov3[3] = m10 * m10 + m11 * m11 + m12 * m12;
    cov3[4] = m10 * m20 + m11 * m21 + m12 * m22;
    cov3[5] = m20 * m20 + m21 * m21 + m22 * m22;
    op = 1.f / (1.f + expf(-__ldg(sc.opac + i)));
    if (wts) op *= __ldg(wts + i);
    constexpr int K = (DEG + 1) * (DEG + 1);
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) shc[3 * k + ch] = __ldg(sc.sh + (size_t)(3 * k + ch) * n + i);
}

// Three CTAs per SM (at most 80 registers; the degree-3 colour coefficients spill a little
// to L1): the kernel runs beside compositing, and a smaller register footprint leaves room
// for compositing CTAs (measured: 0.6% shorter scoring step than at 115 registers).
template <int DEG>
__global__ void __launch_bounds__(256, 3) k_project(SceneDev sc, const CamDev* __restrict__ cams, int nv,
                                                 const float* __restrict__ wts, KOpts o, Splat* __restrict__ splats,
                                                 uint32_t* __restrict__ keys, uint2* __restrict__ rects,
                                                 DevCounters* ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n) return;
    float mu[3], cov3[6], op;
    float shc[3 * (DEG + 1) * (DEG + 1)];
    load_gaussian<DEG>(sc, i, wts, mu, cov3, op, shc);
    const float K2 = 0.5f * kLog2e;
    for (int v = 0; v < nv; ++v) {
        const CamDev& c = cams[v];
        Proj r;
        project_one<DEG>(mu, cov3, op, shc, c, o, r);
        const size_t off = (size_t)v * sc.n + i;
        if (!r.valid) {
            keys[off] = o.narrow_keys ? kNarrowCulled : 0xFFFFFFFFu;
            rects[off] = make_uint2(0u, 0u);
            continue;
        }
        // Cholesky form of the base-2 exponent's quadratic form (0.5 log2 e) d^T cov^-1 d
        // = e1^2 + e2^2: s2^2 = K2 / cov_yy, s1^2 = K2 cov_yy / det, s1k = -s1 cov_xy / cov_yy
        const float s2 = sqrtf(K2 / r.cc);
        const float s1 = sqrtf(K2 * r.cc * r.idet);
        const float s1k = -s1 * r.cb / r.cc;
        const float la = log2f(r.op);
        const float thr = fmaxf(la - o.qcut, o.l2amin);
        Splat s;
        s.m = make_float4(r.mx.hi, r.my.hi, r.mx.lo, r.my.lo);
        s.q = make_float4(s1, s1k, s2, thr);
        s.c = make_float4(r.rgb[0], r.rgb[1], r.rgb[2], la);
        splats[off] = s;
        uint32_t key = __float_as_uint(r.depth);
        if (o.narrow_keys) {
            key -= __float_as_uint(c.near_z);  // >= 1: r.depth > near_z > 0
            if (key >= kNarrowCulled) {
                atomicOr(&ctr->err, kErrDepthRange);
                key = kNarrowCulled - 1u;
            }
        }
        keys[off] = key;
        rects[off] = make_uint2(r.tx0 | (r.ty0 << 16), r.tx1 | (r.ty1 << 16));
    }
}

template <int DEG>
__global__ void k_debug_project(SceneDev sc, const CamDev* __restrict__ cam, KOpts o, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n) return;
    float mu[3], cov3[6], op;
    float shc[3 * (DEG + 1) * (DEG + 1)];
    load_gaussian<DEG>(sc, i, nullptr, mu, cov3, op, shc);
    Proj r;
    project_one<DEG>(mu, cov3, op, shc, *cam, o, r);
    float* d = out + (size_t)16 * i;
    d[0] = r.valid ? 1.f : 0.f;
    if (!r.valid) {
        for (int k = 1; k < 16; ++k) d[k] = 0.f;
        return;
    }
    d[1] = r.mx.hi;
    d[2] = r.my.hi;
    d[3] = r.ia;
    d[4] = r.ib;
    d[5] = r.ic;
    d[6] = r.ca;
    d[7] = r.cb;
    d[8] = r.cc;
    d[9] = r.depth;
    d[10] = r.op;
    d[11] = r.rgb[0];
    d[12] = r.rgb[1];
    d[13] = r.rgb[2];
    d[14] = (float)((r.tx1 - r.tx0) * (r.ty1 - r.ty0));
    d[15] = r.mx.lo;
}

__global__ void k_check_finite(const float* __restrict__ p, int64_t n, DevCounters* ctr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < n; i += stride) bad |= !isfinite(p[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctr->err, kErrNonFinite);
}

// Per-Gaussian statistics over query views (features of the surrogate model): number
// of views whose image the footprint touches, and the mean and maximum area (px^2) of
// the projected 3-sigma ellipse, pi * cut2 * sqrt(det cov2D), over those views.
// What the view statistics take from the projection of one Gaussian in one view: whether
// its footprint reaches the image (the projection's tests: in front of the near plane,
// alpha >= alpha_min, the opacity-aware bounding box over the pixel centres) and the
// ellipse's area pi cut2 sqrt(det Sigma').  The pixel mean is plain FP32 here (the
// projection's two-float mean moves the box by ~1e-4 px), and no colour is evaluated.
__device__ __forceinline__ bool stats_one(const float mu[3], const float cov3[6], float m_eff, const CamDev& c,
                                          const KOpts& o, float& area) {
    const float x = fmaf(c.R[0], mu[0], fmaf(c.R[1], mu[1], fmaf(c.R[2], mu[2], c.t[0])));
    const float y = fmaf(c.R[3], mu[0], fmaf(c.R[4], mu[1], fmaf(c.R[5], mu[2], c.t[1])));
    const float z = fmaf(c.R[6], mu[0], fmaf(c.R[7], mu[1], fmaf(c.R[8], mu[2], c.t[2])));
    if (!(z > c.near_z)) return false;
    float ca, cb, cc;
    ewa_cov2(cov3, c, o, x, y, z, ca, cb, cc);
    const float det = ca * cc - cb * cb;
    if (!(det > 0.f)) return false;
    const float invz = 1.f / z;
    const float mx = fmaf(c.fx * x, invz, c.cx), my = fmaf(c.fy * y, invz, c.cy);
    const float rx = sqrtf(m_eff * ca) * 1.001f + 0.01f;
    const float ry = sqrtf(m_eff * cc) * 1.001f + 0.01f;
    const float fx0 = fmaxf(ceilf(mx - rx), 0.f), fx1 = fminf(floorf(mx + rx), (float)(c.W - 1));
    const float fy0 = fmaxf(ceilf(my - ry), 0.f), fy1 = fminf(floorf(my + ry), (float)(c.H - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return false;
    area = 3.14159265358979f * o.cut2 * sqrtf(det);
    return true;
}

// Per-Gaussian view statistics over nv views: count of views reached, mean and maximum
// footprint area (added to the previous values with accumulate).
__global__ void __launch_bounds__(256) k_view_stats(SceneDev sc, const CamDev* __restrict__ cams, int nv, KOpts o,
                                                    float* __restrict__ stats, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n) return;
    float mu[3], cov3[6], op, dc[3];  // dc: the DC colour coefficients, unused here
    load_gaussian<0>(sc, i, nullptr, mu, cov3, op, dc);
    float cnt = 0.f, sum = 0.f, mx = 0.f;
    if (accumulate) {
        cnt = stats[3 * i];
        sum = stats[3 * i + 1] * cnt;
        mx = stats[3 * i + 2];
    }
    if (op >= o.alpha_min) {  // rho <= alpha < alpha_min everywhere otherwise
        // the box's Mahalanobis radius: the footprint cut, or where alpha k falls below alpha_min
        const float m_eff = fminf(o.cut2, fmaf(2.f / kLog2e, log2f(op) - o.l2amin, 1e-4f));
        for (int v = 0; v < nv; ++v) {
            float area;
            if (!stats_one(mu, cov3, m_eff, cams[v], o, area)) continue;
            cnt += 1.f;
            sum += area;
            mx = fmaxf(mx, area);
        }
    }
    stats[3 * i] = cnt;
    stats[3 * i + 1] = cnt > 0.f ? sum / cnt : 0.f;
    stats[3 * i + 2] = mx;
}

// Surrogate features, BF16 [N][64]: mean / 4, log-scale + 4, unit quaternion, opacity
// logit, SH coefficients x 5 (48 slots, zero beyond the degree), log(1 + view count),
// log(1 + mean area) / 4, log(1 + max area) / 4, extra / 8 (zero without an extra input),
// one zero pad.
__global__ void k_features(SceneDev sc, const float* __restrict__ stats, const float* __restrict__ extra,
                           __nv_bfloat16* __restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n) return;
    const int n = sc.n;
    float f[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) f[k] = 0.f;
    for (int k = 0; k < 3; ++k) f[k] = sc.means[k * n + i] * 0.25f;
    for (int k = 0; k < 3; ++k) f[3 + k] = sc.log_scales[k * n + i] + 4.f;
    float q[4], qn = 0.f;
    for (int k = 0; k < 4; ++k) {
        q[k] = sc.quats[k * n + i];
        qn += q[k] * q[k];
    }
    qn = rsqrtf(qn);
    for (int k = 0; k < 4; ++k) f[6 + k] = q[k] * qn;
    f[10] = sc.opac[i];
    const int nk = 3 * (sc.deg + 1) * (sc.deg + 1);
    for (int k = 0; k < nk; ++k) f[11 + k] = sc.sh[(size_t)k * n + i] * 5.f;
    f[59] = log1pf(stats[3 * i]);
    f[60] = log1pf(stats[3 * i + 1]) * 0.25f;
    f[61] = log1pf(stats[3 * i + 2]) * 0.25f;
    if (extra) f[62] = extra[i] * 0.125f;
    uint4* dst = reinterpret_cast<uint4*>(X + (size_t)i * 64);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        __nv_bfloat162 a = __floats2bfloat162_rn(f[8 * c], f[8 * c + 1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(f[8 * c + 2], f[8 * c + 3]);
        __nv_bfloat162 cc = __floats2bfloat162_rn(f[8 * c + 4], f[8 * c + 5]);
        __nv_bfloat162 d = __floats2bfloat162_rn(f[8 * c + 6], f[8 * c + 7]);
        dst[c] = make_uint4(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b),
                            *reinterpret_cast<uint32_t*>(&cc), *reinterpret_cast<uint32_t*>(&d));
    }
}

// Gradients of the real SH basis (degree <= 3) with respect to the direction (x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float* Y, float (*G)[3]) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        Y[k] = 0.f;
        G[k][0] = G[k][1] = G[k][2] = 0.f;
    }
    Y[0] = 0.28209479177387814f;
    if (DEG >= 1) {
        const float c1 = 0.48860251190291992f;
        Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
        G[1][1] = -c1; G[2][2] = c1; G[3][0] = -c1;
    }
    if (DEG >= 2) {
        const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.54627421529603959f;
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = a * x * y; Y[5] = -a * y * z; Y[6] = b * (2.f * zz - xx - yy); Y[7] = -a * x * z; Y[8] = c * (xx - yy);
        G[4][0] = a * y; G[4][1] = a * x;
        G[5][1] = -a * z; G[5][2] = -a * y;
        G[6][0] = -2.f * b * x; G[6][1] = -2.f * b * y; G[6][2] = 4.f * b * z;
        G[7][0] = -a * z; G[7][2] = -a * x;
        G[8][0] = 2.f * c * x; G[8][1] = -2.f * c * y;
        if (DEG >= 3) {
            const float e0 = 0.59004358992664352f, e1 = 2.8906114426405538f, e2 = 0.45704579946446572f,
                        e3 = 0.37317633259011540f, e4 = 1.4453057213202769f;
            Y[9] = -e0 * y * (3.f * xx - yy); Y[10] = e1 * x * y * z; Y[11] = -e2 * y * (4.f * zz - xx - yy);
            Y[12] = e3 * z * (2.f * zz - 3.f * xx - 3.f * yy); Y[13] = -e2 * x * (4.f * zz - xx - yy);
            Y[14] = e4 * z * (xx - yy); Y[15] = -e0 * x * (xx - 3.f * yy);
            G[9][0] = -6.f * e0 * x * y; G[9][1] = -e0 * (3.f * xx - 3.f * yy);
            G[10][0] = e1 * y * z; G[10][1] = e1 * x * z; G[10][2] = e1 * x * y;
            G[11][0] = 2.f * e2 * x * y; G[11][1] = -e2 * (4.f * zz - xx - 3.f * yy); G[11][2] = -8.f * e2 * y * z;
            G[12][0] = -6.f * e3 * x * z; G[12][1] = -6.f * e3 * y * z; G[12][2] = e3 * (6.f * zz - 3.f * xx - 3.f * yy);
            G[13][0] = -e2 * (4.f * zz - 3.f * xx - yy); G[13][1] = 2.f * e2 * x * y; G[13][2] = -8.f * e2 * x * z;
            G[14][0] = 2.f * e4 * x * z; G[14][1] = -2.f * e4 * y * z; G[14][2] = e4 * (xx - yy);
            G[15][0] = -e0 * (3.f * xx - 3.f * yy); G[15][1] = 6.f * e0 * x * y;
        }
    }
}

// Projection backward of one view, per Gaussian: the 2-D gradients g2d[i] = dL/d(mean x,
// mean y, Q xx, Q xy, Q yy, alpha', r, g, b) chained to the mean (through the projected
// mean, the Jacobian J of the EWA covariance and the SH view direction), the SH
// coefficients (unclamped colours) and the opacity logit (alpha' = w sigmoid(logit)).
// With Q = cov'^-1: dL/dcov' = -Q G Q, dL/dJ = 2 (dL/dcov') J Sigma_cam.
template <int DEG>
__global__ void __launch_bounds__(256) k_project_bwd(SceneDev sc, const CamDev* __restrict__ camp,
                                                     const float* __restrict__ wts, KOpts o,
                                                     const float* __restrict__ g2d, float* __restrict__ g_means,
                                                     float* __restrict__ g_sh, float* __restrict__ g_logit) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n) return;
    const float* G = g2d + (size_t)9 * i;
    float gsum = 0.f;
#pragma unroll
    for (int c = 0; c < 9; ++c) gsum += fabsf(G[c]);
    if (gsum == 0.f) return;
    const CamDev& c = *camp;
    const int n = sc.n;
    float mu[3], cov3[6], op;
    float shc[3 * (DEG + 1) * (DEG + 1)];
    load_gaussian<DEG>(sc, i, nullptr, mu, cov3, op, shc);
    const float w = wts ? wts[i] : 1.f;
    g_logit[i] += G[5] * w * op * (1.f - op);
    const float x = c.R[0] * mu[0] + c.R[1] * mu[1] + c.R[2] * mu[2] + c.t[0];
    const float y = c.R[3] * mu[0] + c.R[4] * mu[1] + c.R[5] * mu[2] + c.t[1];
    const float z = c.R[6] * mu[0] + c.R[7] * mu[1] + c.R[8] * mu[2] + c.t[2];
    const float s00 = cov3[0], s01 = cov3[1], s02 = cov3[2], s11 = cov3[3], s12 = cov3[4], s22 = cov3[5];
    float T[9], Sc[9];
    for (int r = 0; r < 3; ++r) {
        const float a0 = c.R[3 * r], a1 = c.R[3 * r + 1], a2 = c.R[3 * r + 2];
        T[3 * r + 0] = a0 * s00 + a1 * s01 + a2 * s02;
        T[3 * r + 1] = a0 * s01 + a1 * s11 + a2 * s12;
        T[3 * r + 2] = a0 * s02 + a1 * s12 + a2 * s22;
    }
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q)
            Sc[3 * r + q] = T[3 * r] * c.R[3 * q] + T[3 * r + 1] * c.R[3 * q + 1] + T[3 * r + 2] * c.R[3 * q + 2];
    float ux = x / z, uy = y / z;
    const bool inx = ux >= -c.limx && ux <= c.limx, iny = uy >= -c.limy && uy <= c.limy;
    ux = fminf(fmaxf(ux, -c.limx), c.limx);
    uy = fminf(fmaxf(uy, -c.limy), c.limy);
    const float J[6] = {c.fx / z, 0.f, -c.fx * ux / z, 0.f, c.fy / z, -c.fy * uy / z};
    float JS[6];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 3; ++q) JS[3 * r + q] = J[3 * r] * Sc[q] + J[3 * r + 1] * Sc[3 + q] + J[3 * r + 2] * Sc[6 + q];
    const float ca = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + o.dilation;
    const float cb = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
    const float cc = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + o.dilation;
    const float idet = 1.f / (ca * cc - cb * cb);
    const float Q[4] = {cc * idet, -cb * idet, -cb * idet, ca * idet};
    const float Gq[4] = {G[2], 0.5f * G[3], 0.5f * G[3], G[4]};
    float QG[4], H[4];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) QG[2 * r + q] = Q[2 * r] * Gq[q] + Q[2 * r + 1] * Gq[2 + q];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) H[2 * r + q] = -(QG[2 * r] * Q[q] + QG[2 * r + 1] * Q[2 + q]);
    float dJ[6];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 3; ++q) dJ[3 * r + q] = 2.f * (H[2 * r] * JS[q] + H[2 * r + 1] * JS[3 + q]);
    float dx = 0.f, dy = 0.f, dz = 0.f;
    const float iz = 1.f / z, iz2 = iz * iz;
    dz += dJ[0] * (-c.fx * iz2) + dJ[4] * (-c.fy * iz2);
    dz += dJ[2] * (c.fx * ux * iz2) + dJ[5] * (c.fy * uy * iz2);
    if (inx) {
        dx += dJ[2] * (-c.fx * iz) * iz;
        dz += dJ[2] * (-c.fx * iz) * (-x * iz2);
    }
    if (iny) {
        dy += dJ[5] * (-c.fy * iz) * iz;
        dz += dJ[5] * (-c.fy * iz) * (-y * iz2);
    }
    dx += G[0] * c.fx * iz;
    dz += G[0] * (-c.fx * x * iz2);
    dy += G[1] * c.fy * iz;
    dz += G[1] * (-c.fy * y * iz2);
    float gm[3];
    for (int k = 0; k < 3; ++k) gm[k] = c.R[k] * dx + c.R[3 + k] * dy + c.R[6 + k] * dz;
    // colour through the SH basis and the view direction
    const float vx = mu[0] - c.campos[0], vy = mu[1] - c.campos[1], vz = mu[2] - c.campos[2];
    const float len = sqrtf(vx * vx + vy * vy + vz * vz), il = 1.f / len;
    const float hx = vx * il, hy = vy * il, hz = vz * il;
    float Y[16], GY[16][3];
    sh_basis_grad<DEG>(hx, hy, hz, Y, GY);
    constexpr int K = (DEG + 1) * (DEG + 1);
    float gd[3] = {0.f, 0.f, 0.f};
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.5f;
        for (int k = 0; k < K; ++k) acc = fmaf(shc[3 * k + ch], Y[k], acc);
        if (!(acc > 0.f)) continue;
        const float gc = G[6 + ch];
        for (int k = 0; k < K; ++k) {
            g_sh[(size_t)(3 * k + ch) * n + i] += gc * Y[k];
            gd[0] += gc * shc[3 * k + ch] * GY[k][0];
            gd[1] += gc * shc[3 * k + ch] * GY[k][1];
            gd[2] += gc * shc[3 * k + ch] * GY[k][2];
        }
    }
    const float dd = gd[0] * hx + gd[1] * hy + gd[2] * hz;
    gm[0] += (gd[0] - dd * hx) * il;
    gm[1] += (gd[1] - dd * hy) * il;
    gm[2] += (gd[2] - dd * hz) * il;
    for (int k = 0; k < 3; ++k) g_means[(size_t)k * n + i] += gm[k];
}

__global__ void k_scatter_weights(const int32_t* __restrict__ idx, const float* __restrict__ w, int64_t n_sel,
                                  float* __restrict__ wfull, int64_t n, DevCounters* ctr) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_sel; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = idx[k];
        if (i < 0 || i >= n) {
            atomicOr(&ctr->err, kErrIndex);
            continue;
        }
        wfull[i] = w[k];
    }
}

}  // namespace

void scatter_weights(const int32_t* idx, const float* w, int64_t n_sel, float* wfull, int64_t n, DevCounters* ctr,
                     cudaStream_t st) {
    if (n_sel <= 0) return;
    int64_t blocks = (n_sel + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    k_scatter_weights<<<(int)blocks, 256, 0, st>>>(idx, w, n_sel, wfull, n, ctr);
    count_launches(1);
}

void launch_view_stats(const SceneDev& sc, const CamDev* d_cams, int nv, const KOpts& o, float* stats, int accumulate,
                       cudaStream_t st) {
    const int threads = 256;
    const int blocks = (sc.n + threads - 1) / threads;
    // validity and footprint do not depend on the colour: the degree-0 instantiation reads
    // only the DC coefficients and evaluates no higher harmonics, whatever the scene's degree
    k_view_stats<<<blocks, threads, 0, st>>>(sc, d_cams, nv, o, stats, accumulate);
    count_launches(1);
}

void launch_project_backward(const SceneDev& sc, const CamDev* d_cam, const float* d_w, const KOpts& o,
                             const float* g2d, float* g_means, float* g_sh, float* g_logit, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (sc.n + threads - 1) / threads;
    switch (sc.deg) {
        case 0: k_project_bwd<0><<<blocks, threads, 0, st>>>(sc, d_cam, d_w, o, g2d, g_means, g_sh, g_logit); break;
        case 1: k_project_bwd<1><<<blocks, threads, 0, st>>>(sc, d_cam, d_w, o, g2d, g_means, g_sh, g_logit); break;
        case 2: k_project_bwd<2><<<blocks, threads, 0, st>>>(sc, d_cam, d_w, o, g2d, g_means, g_sh, g_logit); break;
        default: k_project_bwd<3><<<blocks, threads, 0, st>>>(sc, d_cam, d_w, o, g2d, g_means, g_sh, g_logit); break;
    }
    count_launches(1);
}

void launch_features(const SceneDev& sc, const float* stats, const float* extra, void* X, cudaStream_t st) {
    k_features<<<(sc.n + 255) / 256, 256, 0, st>>>(sc, stats, extra, reinterpret_cast<__nv_bfloat16*>(X));
    count_launches(1);
}

void launch_project(const SceneDev& sc, const CamDev* d_cams, int nv, const float* d_w, const KOpts& o, Splat* splats,
                    uint32_t* keys, uint2* rects, DevCounters* ctr, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (sc.n + threads - 1) / threads;
    switch (sc.deg) {
        case 0: k_project<0><<<blocks, threads, 0, st>>>(sc, d_cams, nv, d_w, o, splats, keys, rects, ctr); break;
        case 1: k_project<1><<<blocks, threads, 0, st>>>(sc, d_cams, nv, d_w, o, splats, keys, rects, ctr); break;
        case 2: k_project<2><<<blocks, threads, 0, st>>>(sc, d_cams, nv, d_w, o, splats, keys, rects, ctr); break;
        default: k_project<3><<<blocks, threads, 0, st>>>(sc, d_cams, nv, d_w, o, splats, keys, rects, ctr); break;
    }
    count_launches(1);
}

void launch_debug_project(const SceneDev& sc, const CamDev* d_cam, const KOpts& o, float* out, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (sc.n + threads - 1) / threads;
    switch (sc.deg) {
        case 0: k_debug_project<0><<<blocks, threads, 0, st>>>(sc, d_cam, o, out); break;
        case 1: k_debug_project<1><<<blocks, threads, 0, st>>>(sc, d_cam, o, out); break;
        case 2: k_debug_project<2><<<blocks, threads, 0, st>>>(sc, d_cam, o, out); break;
        default: k_debug_project<3><<<blocks, threads, 0, st>>>(sc, d_cam, o, out); break;
    }
    count_launches(1);
}

void launch_check_finite(const float* p, int64_t n, DevCounters* ctr, cudaStream_t st) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_check_finite<<<(int)blocks, 256, 0, st>>>(p, n, ctr);
    count_launches(1);
}

}  // namespace csgs

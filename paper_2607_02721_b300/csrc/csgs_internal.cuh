// Internal declarations of the sm_103a sensitivity-scoring path (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "csgs.h"

namespace csgs {

// Number of kernels this library has launched (all contexts); every launch site adds to it.
void count_launches(long long k);
long long launches();

// Screen tiles: one CTA composites one tile of 2^lw x 2^lh pixels.  Shapes (CSGS_TILE_*):
// 16x16 (the default, and the query of the per-tile resolution), 32x8, 16x8 and 8x8; the
// footprint test is per pixel, so the shape changes only the work split, not which pairs
// contribute.
constexpr int kTileLw16 = 4, kTileLh16 = 4;
constexpr float kLog2e = 1.4426950408889634f;

// Per-view camera, precomputed on the host from csgs_camera.
struct CamDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int W, H;
    float near_z;
    float campos[3];   // -R^T t
    float limx, limy;  // clamp_fov * tan(half FOV) per axis
};

// Tiles of a view per row / column for tiles of 2^lw x 2^lh pixels.
__host__ __device__ inline int tiles_x_of(const CamDev& c, int lw) { return (c.W + (1 << lw) - 1) >> lw; }
__host__ __device__ inline int tiles_y_of(const CamDev& c, int lh) { return (c.H + (1 << lh) - 1) >> lh; }
__host__ __device__ inline int tiles_of(const CamDev& c, int lw, int lh) { return tiles_x_of(c, lw) * tiles_y_of(c, lh); }

struct SceneDev {
    int n;
    int deg;
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opac;
    const float* sh;
};

// Scoring conventions in the form the kernels use.
struct KOpts {
    float alpha_min, rho_max, t_min;
    float qcut;       // footprint cut in base-2 exponent units: 0.5 log2(e) cut2
    float l2amin;     // log2(alpha_min)
    float cut2;
    float dilation, clamp_fov;
    float ow0, ow1, ow2;  // per-pixel objective weights
    int resolution, variant;
    int narrow_keys;  // depth keys: 1 = narrow (27-bit, relative to the near plane), 0 = the float bits
    int tile_lw, tile_lh;  // tile shape: 2^tile_lw x 2^tile_lh pixels
    int persist_ctas;      // per-pixel score: CTAs of a persistent compositing launch (0: one per tile)
    int accumulate;        // scoring: take the maximum with the scores already in the output
};

// One projected Gaussian in one view (48 bytes, 16-byte aligned).
//   m = (mean x hi, mean y hi, mean x lo, mean y lo): the pixel-space mean as an
//       unevaluated two-float sum, so the tile-relative offset keeps FP32 accuracy
//   q = (s1, s1k, s2, thr): the base-2 exponent of rho is
//       log2(alpha) - e1^2 - e2^2,  e1 = s1 dx + s1k dy,  e2 = s2 dy,
//       i.e. the conic (scaled by 0.5 log2 e) in Cholesky form; thr folds the
//       footprint cut and alpha_min into one threshold on that exponent:
//       thr = max(log2(alpha) - qcut, log2(alpha_min))
//   c = (r, g, b, log2(alpha))
struct __align__(16) Splat {
    float4 m;
    float4 q;
    float4 c;
};

// Device error word bits.
enum : uint32_t { kErrCapacity = 1u, kErrNonFinite = 2u, kErrIndex = 4u, kErrDepthRange = 8u };

// Narrow depth keys: bits(z) - bits(near_z) (positive floats order as their bit patterns),
// sorted as three 9-bit digits.  A visible Gaussian has key >= 1; culled ones get
// kNarrowCulled, after every visible key.  A visible depth whose key would reach
// kNarrowCulled (z beyond about 2^16 near_z) flags kErrDepthRange, and the call repeats
// with the full 32-bit keys (four 8-bit digits).
constexpr int kNarrowKeyBits = 27;
constexpr uint32_t kNarrowCulled = (1u << kNarrowKeyBits) - 1u;

// Device counters (one block per context).
// Sum of 16 per-lane values over the warp's 32 lanes, one column per lane pair:
// vector-halving butterfly (8 + 4 + 2 + 1 + 1 shuffles).  Returns the sum of column
// 8 b4 + 4 b3 + 2 b2 + b1 (b_k = bit k of the lane index), held by lanes 2c and 2c + 1.
__device__ __forceinline__ float warp_colsum16(const float (&v)[16], int lane) {
    float a[8], b[4], c[2];
    const bool h1 = lane & 16, h2 = lane & 8, h3 = lane & 4, h4 = lane & 2;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float send = h1 ? v[i] : v[i + 8];
        a[i] = (h1 ? v[i + 8] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = h2 ? a[i] : a[i + 4];
        b[i] = (h2 ? a[i + 4] : a[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = h3 ? b[i] : b[i + 2];
        c[i] = (h3 ? b[i + 2] : b[i]) + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const float send = h4 ? c[0] : c[1];
    float d = (h4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, send, 2);
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

// Binning slots: scoring bins view k in slot k % kBinSlots on the slot's own stream, so
// the binning of the next views overlaps the compositing of the current one.
constexpr int kBinSlots = 4;
constexpr int kCompStreams = 2;  // compositing streams of a scoring submission

struct DevCounters {
    uint32_t err;
    uint32_t pad;
    unsigned long long n_inst[kBinSlots];  // instances of the view in each binning slot (may exceed capacity)
    unsigned long long max_inst;    // maximum over binning chains
    unsigned long long inst_total;  // sum over binning chains
    unsigned long long pairs_eval;
    unsigned long long pairs_hit;
    unsigned long long pairs_eval2;
    unsigned long long pairs_hit2;
    unsigned long long violations;
    double sumA;                    // scene resolution: sum of the objective over queries
    double sumA_view;               // image resolution: the current view's objective
    unsigned long long queries;     // pixel queries with A > 0 (two-pass resolutions)
    unsigned long long staged1;     // tile-list entries staged by compositing pass 1 (counting runs)
    unsigned long long staged2;     // ... and by pass 2
    unsigned long long wentries1;   // (warp, tile-list entry) iterations of pass 1 (counting runs)
    unsigned long long wentries2;   // ... and of pass 2
};

// ---- launchers (k_project.cu)
void launch_project(const SceneDev& sc, const CamDev* d_cams, int nv, const float* d_w, const KOpts& o,
                    Splat* splats, uint32_t* keys, uint2* rects, DevCounters* ctr, cudaStream_t st);
void launch_debug_project(const SceneDev& sc, const CamDev* d_cam, const KOpts& o, float* out, cudaStream_t st);
void launch_check_finite(const float* p, int64_t n, DevCounters* ctr, cudaStream_t st);
void launch_view_stats(const SceneDev& sc, const CamDev* d_cams, int nv, const KOpts& o, float* stats, int accumulate,
                       cudaStream_t st);
void launch_features(const SceneDev& sc, const float* stats, const float* extra, void* X, cudaStream_t st);
// chain the per-Gaussian 2-D gradients of one view to means [3][N], SH [(d+1)^2][3][N]
// and opacity logits [N] (accumulated)
void launch_project_backward(const SceneDev& sc, const CamDev* d_cam, const float* d_w, const KOpts& o,
                             const float* g2d, float* g_means, float* g_sh, float* g_logit, cudaStream_t st);
// wfull[idx[k]] = w[k] (indices outside [0, n) set kErrIndex and are skipped)
void scatter_weights(const int32_t* idx, const float* w, int64_t n_sel, float* wfull, int64_t n, DevCounters* ctr,
                     cudaStream_t st);

// ---- sorting and scans (k_sort.cu)
constexpr int kSortBlocks = 148 * 4;       // default radix-sort grid (the autotuner may pick another)
constexpr int kSortMaxBlocks = 2048;
// words of one segment's radix histograms (per-block digit counts + digit totals) for a
// grid of G blocks per segment
inline size_t sort_hist_stride(int G) { return (size_t)512 * (size_t)G + 512; }
// Stable LSD radix sort of (key, value) pairs on key bits [0, bits), digit_bits (8 or 9)
// bits per pass, of S independent segments of n keys each (segment k at offset
// k * seg_stride in every array).  n is read from d_n (device) and clamped to n_max.
// iota_vals: the values are the indices 0..n-1 within each segment (vals_a is not read).
// hist: S * sort_hist_stride(G) words.  Returns which buffer holds the result (0: a, 1: b).
int radix_sort_pairs(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b, const unsigned long long* d_n,
                     uint32_t n_max, int bits, int digit_bits, uint32_t* hist, int G, bool iota_vals, int S,
                     size_t seg_stride, cudaStream_t st);
// Gaussians of nv views in depth order (order[v][n], Gaussian ids) -> instances with key
// (v << tbits) | tile id and value Gaussian id, view by view, each view in depth order;
// writes the instance count to *n_inst (and the totals in ctr).  cams: the nv views'
// cameras (device); tiles 2^lw pixels wide (the rectangles are in tile units).
// scan_tmp: >= nv * ceil(n / 256) + 64 words.
void emit_instances(const uint32_t* order, const uint2* rects, int n, int nv, const CamDev* cams, int tbits, int lw,
                    uint32_t* inst_keys, uint32_t* inst_vals, uint32_t cap, uint32_t* scan_tmp, DevCounters* ctr,
                    unsigned long long* n_inst, cudaStream_t st);
// The tiles of one view ordered by descending list length, in power-of-two classes
// (order within a class unspecified): order[0..T) is a permutation of the tile ids.
// work (may be null): a persistent compositing launch's queue counter, set to zero.
void tile_order(const uint2* ranges, int T, uint32_t* order, uint32_t* work, cudaStream_t st);
// ranges[v][tile] = [start, end) of each (view, tile) key in the sorted instance keys
// (rows of max_tiles ranges per view; tiles of 2^lw x 2^lh pixels).
void tile_ranges(const uint32_t* keys, const unsigned long long* d_n, uint32_t n_max, uint2* ranges, int nv,
                 const CamDev* cams, int tbits, int lw, int lh, int max_tiles, cudaStream_t st);
void set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st);

// ---- compositing (k_composite.cu)
struct CompositeArgs {
    const uint2* ranges;
    const uint32_t* order;  // tile of CTA b = order[b] (longest lists first), or null: tile b
    uint32_t* work;         // persistent launch: queue counter (zero at launch), or null
    const uint32_t* inst_gid;
    const Splat* splats;
    int n_gauss;
    CamDev cam;
    KOpts o;
    float* rgb;        // render: [H][W][3]
    float* T;          // render: [H][W] (optional)
    uint32_t* s_bits;  // pixel resolution: float bits of s, atomicMax
    float* s_sum;      // scene / image resolution: sum of terms, atomicAdd
    float* tile_sum;   // tile resolution: per tile-list entry, the Gaussian's sum over the tile
    uint8_t* mskbuf;   // pixel / channel resolution: pass 1's warp mask per tile-list entry
    const float* wsel; // transfer: coreset weight per Gaussian (0 = removed)
    float* aux;        // transfer: [H][W][11] per-pixel outputs
    int* last;         // render: [H][W] index + 1 of each pixel's last contributor (optional)
    const float* grad_rgb;  // backward: dL/dC [H][W][3]
    float* g2d;        // backward: per Gaussian dL/d(mean x, mean y, Q xx, Q xy, Q yy, alpha, r, g, b)
    DevCounters* ctr;
    int stats;
};
void launch_composite_render(const CompositeArgs& a, cudaStream_t st);
void launch_composite_score(const CompositeArgs& a, cudaStream_t st);
void launch_composite_transfer(const CompositeArgs& a, cudaStream_t st);
void launch_composite_backward(const CompositeArgs& a, cudaStream_t st);
// Resident CTAs per SM of the persistent per-pixel score kernel for tiles of 2^lw x 2^lh.
int composite_resident_ctas(int lw, int lh);

// ---- sampling (k_sample.cu)
struct SampleTemp {
    double* partial;      // >= 1024
    double* S;            // 1
    unsigned long long* C;  // n
    uint32_t* counts;     // n
    uint32_t* scan_tmp;   // >= 2 * ceil(n / 2048) + 64
    unsigned long long* C_tmp;  // >= 2 * ceil(n / 2048) + 64
    uint32_t* n_out;      // 1
};
void sum_scores(const float* s, int64_t n, double* partial, double* S, cudaStream_t st);
void scene_normalise(float* s, int64_t n, const double* sumA, cudaStream_t st);
// s = (float)((double)s * f)
void scale_scores(float* s, int64_t n, double f, cudaStream_t st);
// image resolution: s = max(s, vbuf / A_view); vbuf = 0
void image_fold(float* s, float* vbuf, int64_t n, const double* sumA_view, cudaStream_t st);
void log_target(const float* s, int64_t n, float eps, float* t, cudaStream_t st);
void adam_update(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                 int step, cudaStream_t st);
// out[0] = sum of log a - log b over the i with a > 0 and b > 0, out[1] = their count (FP64,
// fixed order); partial >= 1024 doubles
void log_ratio_mean(const float* a, const float* b, int64_t n, double* partial, double* out, cudaStream_t st);
void residual_target(const float* s, const float* p, int64_t n, float eps, float mu, float* t, cudaStream_t st);
void surrogate_combine_prior(const float* y, const float* p, const float* s_exact, int64_t n, float eps, float mu,
                             int fill_only, float* out, cudaStream_t st);
void surrogate_combine(const float* y, const float* s_exact, int64_t n, float eps, int fill_only, float* out,
                       cudaStream_t st);
// zero (may be null): a float set to 0 by the same launch (the training loss of the step)
void gather_batch(const void* X, const float* t, int64_t n, int B, uint64_t seed, uint32_t step, void* Xb, float* tb,
                  float* zero, cudaStream_t st);
void probabilities_from_scores(const float* s, int64_t n, const double* S, double* p, cudaStream_t st);
void sample_draws(const double* p, int64_t n, int64_t m, uint64_t seed, const SampleTemp& t, int32_t* draws,
                  int32_t* idx, float* w, cudaStream_t st);

// ---- tensor cores (k_mlp.cu)
// first_wait: clock cycles of the completion wait (< 0: the kernels' full budget, 0: one
// non-blocking test); *d_err |= 1 when it ran out (2 if even the drain wait did)
int gemm_check(const void* A, const void* B, float* C, int K, int N, int* d_err, long long first_wait, int mn_major,
               cudaStream_t st);
// out[2i] = GELU(z[i]), out[2i+1] = GELU'(z[i]) with the surrogate kernels' device functions
void debug_gelu(const float* z, int n, float* out, cudaStream_t st);

// surrogate MLP 64 -> 256 -> 256 -> 1 (parameter block: W1, b1, W2, b2, w3, b3)
constexpr int kMlpParams = 256 * 64 + 256 + 256 * 256 + 256 + 256 + 1;
struct MlpBufs {
    float* P;             // FP32 master parameters
    __nv_bfloat16* W1b;   // [256][64]
    __nv_bfloat16* W2b;   // [256][256]
    __nv_bfloat16* W2Tb;  // [256][256] transpose of W2
};
struct MlpTemp {
    float* gd1;           // [B][256] GELU'(z1)
    __nv_bfloat16* h1;    // [B][256]
    __nv_bfloat16* dz2;   // [B][256]
    __nv_bfloat16* dz1;   // [B][256]
    float* wpart;         // split-K partials: mlp_wgrad_splits(B) x (256 x 256 + 256 x 64)
};
int mlp_wgrad_splits(int64_t B);
MlpBufs mlp_layout(float* P, __nv_bfloat16* W1b, __nv_bfloat16* W2b, __nv_bfloat16* W2Tb);
void mlp_refresh(const MlpBufs& m, cudaStream_t st);
void mlp_forward(const MlpBufs& m, const void* X, int B, float* y, int* err, cudaStream_t st);
void mlp_gradient(const MlpBufs& m, const void* X, const float* t, int B, float* y, float* G, float* loss,
                  const MlpTemp& tmp, int* err, cudaStream_t st);
// One training step on a gathered batch: the gradient kernels, then the split-K sums and
// Adam in one kernel.  G's bias and output-weight entries must be zero on entry (they are
// zero again on return) and *loss zero (it holds the batch's loss on return).
void mlp_train_step(const MlpBufs& m, const void* X, const float* t, int B, float* y, float* G, float* loss,
                    const MlpTemp& tmp, float* mo, float* vo, float lr, int step, int* err, cudaStream_t st);

}  // namespace csgs

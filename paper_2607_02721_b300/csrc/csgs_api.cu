// Host side of the C ABI declared in include/csgs.h: contexts, scenes, work buffers
// and the stream-ordered orchestration of the scoring, sampling and rendering paths.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <memory>
#include <random>
#include <string>
#include <algorithm>
#include <cmath>
#include <vector>

#include "csgs_internal.cuh"

using namespace csgs;

namespace csgs {
static std::atomic<long long> g_launches{0};
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace csgs

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Buffers of one view batch's binning (depth sort, instances, tile sort, ranges).  Scoring
// alternates over kBinSlots slots so that the binning of the next view batch, on its
// slot's own high-priority stream, overlaps the compositing of the current one.
struct BinSlot {
    DevBuf dkeys_b, dvals_a, dvals_b, ikeys_a, ikeys_b, ivals_a, ivals_b, ranges, hist, scan_tmp;
    DevBuf torder;  // scoring: a persistent launch's queue counter, then the view's tiles, longest lists first
    cudaStream_t st = nullptr;
    cudaEvent_t ready = nullptr;  // binning done
    cudaEvent_t freed = nullptr;  // the compositing that read the slot is done
};

struct SceneRec {
    bool alive = false;
    int64_t n = 0;
    int deg = 0;
    float* means = nullptr;
    float* log_scales = nullptr;
    float* quats = nullptr;
    float* opac = nullptr;
    float* sh = nullptr;
    std::vector<CamDev> cams;
    CamDev* d_cams = nullptr;
    int cams_cap = 0;  // views d_cams holds
    float uploaded_clamp = -1.f;  // clamp_fov of the cameras on the device (-1: none)
    int tuned_vb = 0;             // view batch chosen by csgs_autotune (0: automatic)
    int tuned_sb = 0;             // radix-sort grid chosen by csgs_autotune (0: the context's)
    int tuned_shape = 0;          // tile shape chosen by csgs_autotune (CSGS_TILE_*, 0: 16x16)
    int tuned_persist = 0;        // persistent compositing CTAs chosen by csgs_autotune (0: one per tile)
    // asynchronous load: the upload (copies + finiteness check on the context's upload
    // stream) is settled by the first call that uses the scene
    bool pending = false;
    cudaEvent_t uploaded = nullptr;
    DevCounters* d_chk = nullptr;  // the upload's check word (one of the context's slots)
    int chk_slot = -1;
};

}  // namespace

struct csgs_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<SceneRec> scenes;
    std::string err;
    DevCounters* d_ctr = nullptr;
    DevCounters* h_ctr = nullptr;  // pinned
    double* h_S = nullptr;         // pinned
    uint32_t* h_u32 = nullptr;     // pinned
    unsigned long long* d_nconst = nullptr;
    DevBuf splats[2], keys[2], rects[2];  // projected view batches, double-buffered
    BinSlot slot[kBinSlots];
    cudaStream_t pst = nullptr;           // projection stream (scoring)
    cudaEvent_t ev_start = nullptr;       // enqueue start on the context's stream
    cudaEvent_t ev_proj[2] = {};          // projection of the batch in buffer set k done
    cudaEvent_t ev_setfree[2] = {};       // last compositing that read buffer set k done
    // compositing streams besides the context's (view v composites on stream v % kCompStreams)
    cudaStream_t cst[kCompStreams - 1] = {};
    cudaEvent_t ev_csetfree[kCompStreams - 1][2] = {};  // ... last compositing that read buffer set k done
    cudaEvent_t ev_cdone[kCompStreams - 1] = {};        // ... last compositing of a scene done
    uint32_t cap = 0;
    int sort_blocks = kSortBlocks;  // radix-sort grid (autotuned)
    DevBuf partial, Sdev, C, counts, ctmp, stmp, nout, p, wfull;
    DevBuf tsum, vbuf;  // tile resolution: per instance; image resolution: per Gaussian
    DevBuf mskb;        // pixel / channel resolution: warp mask per instance (pass 1 -> pass 2)
    DevBuf mskbx[kCompStreams - 1], tsumx[kCompStreams - 1];  // ... and tile sums, for the other streams
    // surrogate model
    bool mlp_ready = false;
    DevBuf mP, mM, mV, mG, mW1b, mW2b, mW2Tb, mY, mXb, mTb, mLoss, mGd1, mH1, mDz2, mDz1, mPart;
    int64_t mlp_rows = 0;
    DevBuf bRgb, bT, bLast, g2d;  // render backward
    csgs_stats stats{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> evpool;  // phase timing
    cudaGraphExec_t graph_exec = nullptr;  // captured multi-scene scoring
    std::string graph_key;
    long long graph_nodes_launches = 0;
    unsigned long long buf_gen = 0;  // bumped whenever a work buffer is reallocated
    bool wide_keys = false;          // a view's depth range overflowed the narrow keys: 32-bit keys from then on
    int max_tiles = 0;               // ranges per view row in the binning slots
    // attribute buffers of freed scenes, kept for later loads of the same size (a scene
    // loaded and freed every step then allocates and frees nothing); released at destroy
    std::vector<std::pair<size_t, float*>> scene_pool;
    // camera buffers of freed scenes (views held, pointer), reused the same way
    std::vector<std::pair<int, CamDev*>> cams_pool;
    cudaStream_t ust = nullptr;  // upload stream of csgs_load_scene_async
    std::string scene_err;       // why the last settled asynchronous load was rejected
    // check words of pending asynchronous loads, allocated once (a cudaFree per load would
    // synchronise the device and wait for the next scene's upload)
    DevCounters* d_chk_slots = nullptr;
    uint32_t* h_chk_slots = nullptr;  // pinned: each slot's check word, copied by the upload stream
    uint32_t chk_used = 0;       // bit k: slot k belongs to a pending load
};

namespace {

csgs_status fail(csgs_ctx* ctx, csgs_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                          \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? CSGS_E_NOMEM : CSGS_E_CUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                              \
    } while (0)

csgs_status ensure(csgs_ctx* ctx, DevBuf& b, size_t bytes) {
    if (bytes <= b.bytes) return CSGS_OK;
    if (b.p) {
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
        CUDA_TRY(ctx, cudaFree(b.p));
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes + bytes / 8 + 256;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(ctx, CSGS_E_NOMEM, "device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    }
    b.bytes = want;
    ++ctx->buf_gen;
    return CSGS_OK;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

template <class T>
T* P(DevBuf& b) {
    return reinterpret_cast<T*>(b.p);
}

csgs_status launch_check(csgs_ctx* ctx, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, CSGS_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return CSGS_OK;
}

int ceil_log2(uint32_t v) {
    int b = 0;
    while ((1u << b) < v) ++b;
    return b;
}

bool finite3(const float* v, int k) {
    for (int i = 0; i < k; ++i)
        if (!isfinite(v[i])) return false;
    return true;
}

// Tile shape of a call: the per-tile resolution's query is a 16x16 tile, so it always bins
// 16x16 tiles; CSGS_TILE_AUTO is 16x16 until a scene-level choice replaces it
// (scene_tile_shape).
void set_tile_shape(KOpts* k, int shape) {
    k->tile_lw = kTileLw16;
    k->tile_lh = kTileLh16;
    if (k->resolution == CSGS_RES_TILE) return;
    if (shape == CSGS_TILE_32X8) {
        k->tile_lw = 5;
        k->tile_lh = 3;
    } else if (shape == CSGS_TILE_16X8) {
        k->tile_lw = 4;
        k->tile_lh = 3;
    } else if (shape == CSGS_TILE_8X8) {
        k->tile_lw = 3;
        k->tile_lh = 3;
    }
}

csgs_status make_kopts(csgs_ctx* ctx, const csgs_score_opts* o, KOpts* k) {
    if (!o) return fail(ctx, CSGS_E_INVAL, "opts is NULL");
    if (o->resolution < CSGS_RES_PIXEL || o->resolution > CSGS_RES_IMAGE)
        return fail(ctx, CSGS_E_INVAL, "resolution %d is not supported", o->resolution);
    if (o->variant < CSGS_VAR_L1 || o->variant > CSGS_VAR_NC)
        return fail(ctx, CSGS_E_INVAL, "variant %d is not supported", o->variant);
    if (!(o->alpha_min >= 0.f) || !(o->rho_max > 0.f && o->rho_max <= 1.f) || !(o->t_min >= 0.f) ||
        !(o->cut2 > 0.f) || !(o->dilation >= 0.f) || !(o->clamp_fov > 0.f) || !finite3(o->obj_w, 3) ||
        o->obj_w[0] < 0.f || o->obj_w[1] < 0.f || o->obj_w[2] < 0.f || o->view_batch < 0)
        return fail(ctx, CSGS_E_INVAL, "invalid scoring options");
    if (o->tile_shape < CSGS_TILE_AUTO || o->tile_shape > CSGS_TILE_8X8)
        return fail(ctx, CSGS_E_INVAL, "tile_shape %d is not supported", o->tile_shape);
    if (o->persist_ctas < -1 || o->persist_ctas > (1 << 20))
        return fail(ctx, CSGS_E_INVAL, "persist_ctas %d is out of range", o->persist_ctas);
    if (o->accumulate != 0 && o->accumulate != 1) return fail(ctx, CSGS_E_INVAL, "accumulate must be 0 or 1");
    if (o->accumulate && o->resolution == CSGS_RES_SCENE)
        return fail(ctx, CSGS_E_INVAL, "the per-scene resolution cannot accumulate over query sets");
    k->alpha_min = o->alpha_min;
    k->rho_max = o->rho_max;
    k->t_min = o->t_min;
    k->cut2 = o->cut2;
    k->qcut = (float)(0.5 * 1.4426950408889634 * (double)o->cut2);
    k->l2amin = o->alpha_min > 0.f ? (float)log2((double)o->alpha_min) : -1e30f;
    k->dilation = o->dilation;
    k->clamp_fov = o->clamp_fov;
    k->ow0 = o->obj_w[0];
    k->ow1 = o->obj_w[1];
    k->ow2 = o->obj_w[2];
    k->resolution = o->resolution;
    k->variant = o->variant;
    k->narrow_keys = ctx->wide_keys ? 0 : 1;
    set_tile_shape(k, o->tile_shape);
    k->persist_ctas = o->persist_ctas > 0 ? o->persist_ctas : 0;
    k->accumulate = o->accumulate;
    return CSGS_OK;
}

SceneRec* find_scene(csgs_ctx* ctx, int32_t id) {
    if (!ctx || id < 0 || id >= (int32_t)ctx->scenes.size() || !ctx->scenes[id].alive) return nullptr;
    return &ctx->scenes[id];
}


constexpr size_t kScenePoolMax = 32;
constexpr int kMaxPendingLoads = 16;

float* pool_take(csgs_ctx* ctx, size_t bytes) {
    for (size_t k = 0; k < ctx->scene_pool.size(); ++k)
        if (ctx->scene_pool[k].first == bytes) {
            float* p = ctx->scene_pool[k].second;
            ctx->scene_pool.erase(ctx->scene_pool.begin() + (long)k);
            return p;
        }
    return nullptr;
}

void pool_put(csgs_ctx* ctx, size_t bytes, float* p) {
    if (!p) return;
    ctx->scene_pool.push_back({bytes, p});
    if (ctx->scene_pool.size() > kScenePoolMax) {
        cudaFree(ctx->scene_pool.front().second);
        ctx->scene_pool.erase(ctx->scene_pool.begin());
    }
}

// Byte sizes of a scene's five attribute buffers (means, log-scales, quaternions,
// opacity logits, SH coefficients).
void scene_bytes(int64_t n, int deg, size_t out[5]) {
    const size_t nk = (size_t)(deg + 1) * (deg + 1);
    const size_t counts[5] = {3 * (size_t)n, 3 * (size_t)n, 4 * (size_t)n, (size_t)n, 3 * nk * (size_t)n};
    for (int k = 0; k < 5; ++k) out[k] = counts[k] * sizeof(float);
}


// Return a scene's attribute buffers to the context's pool and forget it.
void drop_scene(csgs_ctx* ctx, SceneRec* s) {
    size_t bytes[5];
    scene_bytes(s->n, s->deg, bytes);
    float* bufs[5] = {s->means, s->log_scales, s->quats, s->opac, s->sh};
    for (int k = 0; k < 5; ++k) pool_put(ctx, bytes[k], bufs[k]);
    if (s->d_cams) {
        if (ctx->cams_pool.size() >= (size_t)kScenePoolMax) {  // keep the pool small: drop the oldest
            cudaFree(ctx->cams_pool.front().second);
            ctx->cams_pool.erase(ctx->cams_pool.begin());
        }
        ctx->cams_pool.emplace_back(s->cams_cap, s->d_cams);
    }
    if (s->uploaded) cudaEventDestroy(s->uploaded);
    if (s->chk_slot >= 0) ctx->chk_used &= ~(1u << s->chk_slot);
    *s = SceneRec();
}

// Wait for an asynchronous load's upload and read its finiteness check; a scene with a
// non-finite attribute is released (its id becomes invalid) and false is returned.
bool settle_scene(csgs_ctx* ctx, SceneRec* s) {
    if (!s->pending) return true;
    s->pending = false;
    // the upload stream copied the check word to pinned memory before recording the event,
    // so waiting for this scene's event is enough (no copy here that could queue behind the
    // next scene's upload)
    uint32_t err = ~0u;
    if (cudaEventSynchronize(s->uploaded) == cudaSuccess)
        err = *static_cast<volatile uint32_t*>(ctx->h_chk_slots + s->chk_slot);
    else {
        cudaGetLastError();
        ctx->scene_err = "the scene's upload failed";
        drop_scene(ctx, s);
        return false;
    }
    if (err & kErrNonFinite) {
        ctx->scene_err = "scene attributes contain non-finite values (the scene is released)";
        drop_scene(ctx, s);
        return false;
    }
    ctx->chk_used &= ~(1u << s->chk_slot);
    s->chk_slot = -1;
    s->d_chk = nullptr;
    return true;
}

// The scene with this id, its asynchronous upload (if any) settled; nullptr if the id is
// invalid or the upload was rejected (ctx->scene_err says why).
SceneRec* get_scene(csgs_ctx* ctx, int32_t id) {
    SceneRec* s = find_scene(ctx, id);
    if (!s) return nullptr;
    if (!settle_scene(ctx, s)) return nullptr;
    return s;
}

// The error of a call given a scene id that get_scene rejected.
csgs_status scene_fail(csgs_ctx* ctx, int32_t id) {
    if (!ctx->scene_err.empty()) {
        std::string e = ctx->scene_err;
        ctx->scene_err.clear();
        return fail(ctx, CSGS_E_INVAL, "scene %d: %s", id, e.c_str());
    }
    return fail(ctx, CSGS_E_INVAL, "bad scene id %d", id);
}

SceneDev scene_dev(const SceneRec& s) {
    SceneDev d;
    d.n = (int)s.n;
    d.deg = s.deg;
    d.means = s.means;
    d.log_scales = s.log_scales;
    d.quats = s.quats;
    d.opac = s.opac;
    d.sh = s.sh;
    return d;
}

// Per-view buffers for a batch of `vb` views and the binning slots' buffers (one view
// each: scoring bins every view in its own chain).
csgs_status ensure_view_buffers(csgs_ctx* ctx, int64_t n, int vb, int max_tiles) {
    csgs_status r;
    for (int k = 0; k < 2; ++k) {
        if ((r = ensure(ctx, ctx->splats[k], sizeof(Splat) * (size_t)n * vb))) return r;
        if ((r = ensure(ctx, ctx->keys[k], sizeof(uint32_t) * (size_t)n * vb))) return r;
        if ((r = ensure(ctx, ctx->rects[k], sizeof(uint2) * (size_t)n * vb))) return r;
    }
    if (ctx->cap == 0) {
        uint64_t c = (uint64_t)n * 8;
        if (c < (1u << 20)) c = 1u << 20;
        if (c > 0xF0000000ull) c = 0xF0000000ull;
        ctx->cap = (uint32_t)c;
    }
    const size_t ib = sizeof(uint32_t) * (size_t)ctx->cap;
    const size_t nv = (size_t)n;
    // the row stride of the ranges only grows (a captured graph keeps the stride it saw)
    if (max_tiles > ctx->max_tiles) ctx->max_tiles = max_tiles;
    for (BinSlot& b : ctx->slot) {
        if ((r = ensure(ctx, b.dkeys_b, sizeof(uint32_t) * nv))) return r;
        if ((r = ensure(ctx, b.dvals_a, sizeof(uint32_t) * nv))) return r;
        if ((r = ensure(ctx, b.dvals_b, sizeof(uint32_t) * nv))) return r;
        if ((r = ensure(ctx, b.ranges, sizeof(uint2) * (size_t)ctx->max_tiles))) return r;
        if ((r = ensure(ctx, b.torder, sizeof(uint32_t) * ((size_t)ctx->max_tiles + 1)))) return r;
        if ((r = ensure(ctx, b.hist, sizeof(uint32_t) * sort_hist_stride(kSortMaxBlocks)))) return r;
        if ((r = ensure(ctx, b.scan_tmp, sizeof(uint32_t) * ((size_t)(n + 255) / 256 + 64)))) return r;
        if ((r = ensure(ctx, b.ikeys_a, ib))) return r;
        if ((r = ensure(ctx, b.ikeys_b, ib))) return r;
        if ((r = ensure(ctx, b.ivals_a, ib))) return r;
        if ((r = ensure(ctx, b.ivals_b, ib))) return r;
    }
    return CSGS_OK;
}

// Depth sort -> instances -> (view, tile) sort -> ranges for nv projected views (keys and
// rectangles [nv][n], cameras cams[0..nv) on host and device) in binning slot `k` on
// stream `st`.  Returns the instance value buffer (Gaussian ids in view, tile, depth
// order); view v's ranges are row v (ctx->max_tiles ranges per row) of slot k's `ranges`.
// Scoring bins one view per chain (nv = 1): one sort over a whole view batch (segments
// per view, (view, tile) keys) measured slower, because each radix pass is bound by the
// latency of its 2048-key sub-tiles, not by the array's size.  The slot buffers are sized
// for nv = 1.
const uint32_t* bin_batch(csgs_ctx* ctx, int k, int64_t n, int nv, uint32_t* keys, const uint2* rects,
                          const CamDev* h_cams, const CamDev* d_cams, const KOpts& ko, int grid, cudaStream_t st) {
    const bool narrow = ko.narrow_keys != 0;
    BinSlot& b = ctx->slot[k];
    unsigned long long* n_inst = &ctx->d_ctr->n_inst[k];
    // one segment per view; the grid is split over the segments
    int gseg = grid / nv;
    if (gseg < 8) gseg = 8;
    // narrow depth keys: three 9-bit passes; the float bits: four 8-bit passes
    int cur = radix_sort_pairs(keys, P<uint32_t>(b.dvals_a), P<uint32_t>(b.dkeys_b), P<uint32_t>(b.dvals_b),
                               ctx->d_nconst, (uint32_t)n, narrow ? kNarrowKeyBits : 32, narrow ? 9 : 8,
                               P<uint32_t>(b.hist), gseg, true, nv, (size_t)n, st);
    const uint32_t* order = cur ? P<uint32_t>(b.dvals_b) : P<uint32_t>(b.dvals_a);
    int tbits = 1;
    for (int v = 0; v < nv; ++v) {
        const int tb = ceil_log2((uint32_t)tiles_of(h_cams[v], ko.tile_lw, ko.tile_lh));
        if (tb > tbits) tbits = tb;
    }
    emit_instances(order, rects, (int)n, nv, d_cams, tbits, ko.tile_lw, P<uint32_t>(b.ikeys_a), P<uint32_t>(b.ivals_a), ctx->cap,
                   P<uint32_t>(b.scan_tmp), ctx->d_ctr, n_inst, st);
    const int kbits = tbits + ceil_log2((uint32_t)nv);
    // 9-bit digits once the key needs more than two 8-bit passes
    const int db = kbits > 16 ? 9 : 8;
    int cur2 = radix_sort_pairs(P<uint32_t>(b.ikeys_a), P<uint32_t>(b.ivals_a), P<uint32_t>(b.ikeys_b),
                                P<uint32_t>(b.ivals_b), n_inst, ctx->cap, kbits, db, P<uint32_t>(b.hist),
                                grid, false, 1, 0, st);
    const uint32_t* ik = cur2 ? P<uint32_t>(b.ikeys_b) : P<uint32_t>(b.ikeys_a);
    const uint32_t* iv = cur2 ? P<uint32_t>(b.ivals_b) : P<uint32_t>(b.ivals_a);
    tile_ranges(ik, n_inst, ctx->cap, P<uint2>(b.ranges), nv, d_cams, tbits, ko.tile_lw, ko.tile_lh, ctx->max_tiles,
                st);
    return iv;
}

csgs_status read_counters(csgs_ctx* ctx) {
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, ctx->st));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    return CSGS_OK;
}

csgs_status grow_capacity(csgs_ctx* ctx);

// After a run that flagged an overflow: 32-bit depth keys from now on if a depth left the
// narrow keys' range, a larger instance buffer if the instances did not fit.
csgs_status widen_or_grow(csgs_ctx* ctx, KOpts& ko) {
    const uint32_t e = ctx->h_ctr->err;
    if (e & kErrDepthRange) {
        if (!ko.narrow_keys) return fail(ctx, CSGS_E_DEVICE_CHECK, "depth key range flagged with 32-bit keys");
        ctx->wide_keys = true;
        ko.narrow_keys = 0;
    }
    if (e & kErrCapacity) return grow_capacity(ctx);
    return CSGS_OK;
}

csgs_status grow_capacity(csgs_ctx* ctx) {
    unsigned long long need = ctx->h_ctr->max_inst;
    unsigned long long c = need + need / 4 + 4096;
    if (c > 0xF0000000ull) return fail(ctx, CSGS_E_DEVICE_CHECK, "instance count %llu exceeds the 32-bit index range", need);
    ctx->cap = (uint32_t)c;
    csgs_status r;
    const size_t ib = sizeof(uint32_t) * (size_t)ctx->cap;
    for (BinSlot& b : ctx->slot) {
        if ((r = ensure(ctx, b.ikeys_a, ib))) return r;
        if ((r = ensure(ctx, b.ikeys_b, ib))) return r;
        if ((r = ensure(ctx, b.ivals_a, ib))) return r;
        if ((r = ensure(ctx, b.ivals_b, ib))) return r;
    }
    return CSGS_OK;
}

}  // namespace

extern "C" {

void csgs_default_opts(csgs_score_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->resolution = CSGS_RES_PIXEL;
    o->variant = CSGS_VAR_L1;
    o->obj_w[0] = o->obj_w[1] = o->obj_w[2] = 1.f;
    o->alpha_min = 1.f / 255.f;
    o->rho_max = 0.99f;
    o->t_min = 1e-4f;
    o->cut2 = 9.f;
    o->dilation = 0.3f;
    o->clamp_fov = 1.3f;
    o->view_batch = 0;
    o->collect_stats = 0;
    o->tile_shape = CSGS_TILE_AUTO;
    o->persist_ctas = 0;
    o->accumulate = 0;
}

csgs_status csgs_create(csgs_ctx** out, int32_t device, void* cuda_stream) {
    if (!out) return CSGS_E_INVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CSGS_E_INVAL;
    }
    if (cudaSetDevice(device) != cudaSuccess) return CSGS_E_CUDA;
    csgs_ctx* ctx = new csgs_ctx();
    ctx->device = device;
    if (cuda_stream) {
        ctx->st = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return CSGS_E_CUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaMalloc(&ctx->d_ctr, sizeof(DevCounters)) != cudaSuccess ||
        cudaMalloc(&ctx->d_nconst, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_ctr, sizeof(DevCounters)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_S, sizeof(double) * 2) != cudaSuccess ||
        cudaMallocHost(&ctx->h_u32, sizeof(uint32_t) * 2) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        csgs_destroy(ctx);
        return CSGS_E_NOMEM;
    }
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (BinSlot& b : ctx->slot) {
        if (cudaStreamCreateWithPriority(&b.st, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.freed, cudaEventDisableTiming) != cudaSuccess) {
            csgs_destroy(ctx);
            return CSGS_E_CUDA;
        }
    }
    bool ev_ok = cudaStreamCreateWithFlags(&ctx->pst, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaStreamCreateWithFlags(&ctx->ust, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < 2 && ev_ok; ++k)
        ev_ok = cudaEventCreateWithFlags(&ctx->ev_proj[k], cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&ctx->ev_setfree[k], cudaEventDisableTiming) == cudaSuccess;
    for (int c = 0; c < kCompStreams - 1 && ev_ok; ++c)
        ev_ok = cudaStreamCreateWithFlags(&ctx->cst[c], cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&ctx->ev_cdone[c], cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&ctx->ev_csetfree[c][0], cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&ctx->ev_csetfree[c][1], cudaEventDisableTiming) == cudaSuccess;
    if (!ev_ok) {
        csgs_destroy(ctx);
        return CSGS_E_CUDA;
    }
    cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), ctx->st);
    *out = ctx;
    return CSGS_OK;
}

void csgs_destroy(csgs_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    if (ctx->ust) cudaStreamSynchronize(ctx->ust);
    for (auto& s : ctx->scenes) {
        if (!s.alive) continue;
        if (s.uploaded) cudaEventDestroy(s.uploaded);
        cudaFree(s.means);
        cudaFree(s.log_scales);
        cudaFree(s.quats);
        cudaFree(s.opac);
        cudaFree(s.sh);
        cudaFree(s.d_cams);
    }
    for (auto& e : ctx->cams_pool) cudaFree(e.second);
    ctx->cams_pool.clear();
    for (auto& e : ctx->scene_pool) cudaFree(e.second);
    ctx->scene_pool.clear();
    if (ctx->d_chk_slots) cudaFree(ctx->d_chk_slots);
    if (ctx->h_chk_slots) cudaFreeHost(ctx->h_chk_slots);
    for (BinSlot& b : ctx->slot) {
        DevBuf* sb[] = {&b.dkeys_b, &b.dvals_a, &b.dvals_b, &b.ikeys_a, &b.ikeys_b,
                        &b.ivals_a, &b.ivals_b, &b.ranges,  &b.hist,    &b.scan_tmp};
        for (DevBuf* x : sb) release(*x);
        if (b.st) cudaStreamDestroy(b.st);
        if (b.ready) cudaEventDestroy(b.ready);
        if (b.freed) cudaEventDestroy(b.freed);
    }
    for (int k = 0; k < 2; ++k) {
        if (ctx->ev_proj[k]) cudaEventDestroy(ctx->ev_proj[k]);
        if (ctx->ev_setfree[k]) cudaEventDestroy(ctx->ev_setfree[k]);
        release(ctx->splats[k]);
        release(ctx->keys[k]);
        release(ctx->rects[k]);
    }
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    if (ctx->pst) cudaStreamDestroy(ctx->pst);
    if (ctx->ust) cudaStreamDestroy(ctx->ust);
    for (int c = 0; c < kCompStreams - 1; ++c) {
        if (ctx->ev_cdone[c]) cudaEventDestroy(ctx->ev_cdone[c]);
        for (int k = 0; k < 2; ++k)
            if (ctx->ev_csetfree[c][k]) cudaEventDestroy(ctx->ev_csetfree[c][k]);
        if (ctx->cst[c]) cudaStreamDestroy(ctx->cst[c]);
        release(ctx->mskbx[c]);
        release(ctx->tsumx[c]);
    }
    DevBuf* bufs[] = {
                      &ctx->partial, &ctx->Sdev,   &ctx->C,       &ctx->counts,  &ctx->ctmp,
                      &ctx->stmp,   &ctx->nout,    &ctx->p,       &ctx->wfull,   &ctx->tsum,    &ctx->vbuf,
                      &ctx->mskb,
                      &ctx->mP,     &ctx->mM,      &ctx->mV,      &ctx->mG,      &ctx->mW1b,    &ctx->mW2b,
                      &ctx->mW2Tb,  &ctx->mY,      &ctx->mXb,     &ctx->mTb,     &ctx->mLoss,   &ctx->mGd1,
                      &ctx->mH1,    &ctx->mDz2,    &ctx->mDz1,    &ctx->mPart,   &ctx->bRgb,    &ctx->bT,      &ctx->bLast,
                      &ctx->g2d};
    for (DevBuf* b : bufs) release(*b);
    if (ctx->d_ctr) cudaFree(ctx->d_ctr);
    if (ctx->d_nconst) cudaFree(ctx->d_nconst);
    if (ctx->h_ctr) cudaFreeHost(ctx->h_ctr);
    if (ctx->h_S) cudaFreeHost(ctx->h_S);
    if (ctx->h_u32) cudaFreeHost(ctx->h_u32);
    for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_stream && ctx->st) cudaStreamDestroy(ctx->st);
    delete ctx;
}

const char* csgs_last_error(const csgs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }


// Allocate (or reuse) a scene's buffers and enqueue the copies and the finiteness checks
// on stream `st`, the check writing to chk->err.  On success *s holds the buffers.
static csgs_status enqueue_scene_load(csgs_ctx* ctx, const csgs_scene_desc* d, SceneRec* s, DevCounters* chk,
                                      cudaStream_t st) {
    if (!d) return fail(ctx, CSGS_E_INVAL, "null argument");
    if (d->n <= 0 || d->n >= (1ll << 31)) return fail(ctx, CSGS_E_INVAL, "scene size %lld out of range", (long long)d->n);
    if (d->sh_degree < 0 || d->sh_degree > 3) return fail(ctx, CSGS_E_INVAL, "sh_degree %d not in 0..3", d->sh_degree);
    if (!d->means || !d->log_scales || !d->quats || !d->opacity_logits || !d->sh)
        return fail(ctx, CSGS_E_INVAL, "null attribute pointer");
    s->n = d->n;
    s->deg = d->sh_degree;
    const size_t n = (size_t)d->n;
    const size_t nk = (size_t)(d->sh_degree + 1) * (d->sh_degree + 1);
    struct {
        float** dst;
        const float* src;
        size_t count;
    } parts[] = {{&s->means, d->means, 3 * n},
                 {&s->log_scales, d->log_scales, 3 * n},
                 {&s->quats, d->quats, 4 * n},
                 {&s->opac, d->opacity_logits, n},
                 {&s->sh, d->sh, 3 * nk * n}};
    const cudaMemcpyKind kind = d->is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUDA_TRY(ctx, cudaMemsetAsync(&chk->err, 0, sizeof(uint32_t), st));
    for (auto& p : parts) {
        *p.dst = pool_take(ctx, p.count * sizeof(float));
        if (!*p.dst && cudaMalloc(p.dst, p.count * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            *p.dst = nullptr;
            cudaStreamSynchronize(st);  // copies already enqueued into the other buffers
            for (auto& q : parts) pool_put(ctx, q.count * sizeof(float), *q.dst);
            return fail(ctx, CSGS_E_NOMEM, "scene allocation failed");
        }
        CUDA_TRY(ctx, cudaMemcpyAsync(*p.dst, p.src, p.count * sizeof(float), kind, st));
        launch_check_finite(*p.dst, (int64_t)p.count, chk, st);
    }
    return CSGS_OK;
}

csgs_status csgs_load_scene(csgs_ctx* ctx, const csgs_scene_desc* d, int32_t* scene_id) {
    if (!ctx) return CSGS_E_INVAL;
    if (!scene_id) return fail(ctx, CSGS_E_INVAL, "null argument");
    cudaSetDevice(ctx->device);
    SceneRec s;
    csgs_status r = enqueue_scene_load(ctx, d, &s, ctx->d_ctr, ctx->st);
    if (r) return r;
    if ((r = read_counters(ctx))) return r;
    if (ctx->h_ctr->err & kErrNonFinite) {
        drop_scene(ctx, &s);
        return fail(ctx, CSGS_E_INVAL, "scene attributes contain non-finite values");
    }
    s.alive = true;
    ctx->scenes.push_back(s);
    *scene_id = (int32_t)ctx->scenes.size() - 1;
    return CSGS_OK;
}

csgs_status csgs_load_scene_async(csgs_ctx* ctx, const csgs_scene_desc* d, int32_t* scene_id) {
    if (!ctx) return CSGS_E_INVAL;
    if (!scene_id) return fail(ctx, CSGS_E_INVAL, "null argument");
    cudaSetDevice(ctx->device);
    SceneRec s;
    if (!ctx->d_chk_slots) {
        if (cudaMalloc(&ctx->d_chk_slots, sizeof(DevCounters) * kMaxPendingLoads) != cudaSuccess ||
            cudaHostAlloc(&ctx->h_chk_slots, sizeof(uint32_t) * kMaxPendingLoads, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            if (ctx->d_chk_slots) cudaFree(ctx->d_chk_slots);
            ctx->d_chk_slots = nullptr;
            ctx->h_chk_slots = nullptr;
            return fail(ctx, CSGS_E_NOMEM, "upload bookkeeping allocation failed");
        }
    }
    for (int k = 0; k < kMaxPendingLoads; ++k)
        if (!(ctx->chk_used & (1u << k))) {
            s.chk_slot = k;
            break;
        }
    if (s.chk_slot < 0)
        return fail(ctx, CSGS_E_INVAL, "more than %d asynchronous loads pending: use the scenes first",
                    kMaxPendingLoads);
    s.d_chk = ctx->d_chk_slots + s.chk_slot;
    if (cudaEventCreateWithFlags(&s.uploaded, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, CSGS_E_CUDA, "event creation failed");
    }
    csgs_status r = enqueue_scene_load(ctx, d, &s, s.d_chk, ctx->ust);
    if (r) {
        cudaStreamSynchronize(ctx->ust);
        cudaEventDestroy(s.uploaded);
        return r;
    }
    ctx->chk_used |= 1u << s.chk_slot;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_chk_slots + s.chk_slot, &s.d_chk->err, sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, ctx->ust));
    CUDA_TRY(ctx, cudaEventRecord(s.uploaded, ctx->ust));
    s.pending = true;
    s.alive = true;
    ctx->scenes.push_back(s);
    *scene_id = (int32_t)ctx->scenes.size() - 1;
    return CSGS_OK;
}

csgs_status csgs_free_scene(csgs_ctx* ctx, int32_t scene_id) {
    SceneRec* s = find_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (s->pending) cudaEventSynchronize(s->uploaded);  // its copies may still be landing
    cudaStreamSynchronize(ctx->st);
    drop_scene(ctx, s);
    return CSGS_OK;
}

csgs_status csgs_set_queries(csgs_ctx* ctx, int32_t scene_id, const csgs_camera* cams, int32_t n_views) {
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (!cams || n_views <= 0) return fail(ctx, CSGS_E_INVAL, "no cameras");
    std::vector<CamDev> v(n_views);
    for (int i = 0; i < n_views; ++i) {
        const csgs_camera& c = cams[i];
        if (!finite3(c.R, 9) || !finite3(c.t, 3) || !(c.fx > 0.f) || !(c.fy > 0.f) || !isfinite(c.cx) ||
            !isfinite(c.cy) || c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384 ||
            !(c.near_z > 0.f) || !isfinite(c.fx) || !isfinite(c.fy))
            return fail(ctx, CSGS_E_INVAL, "camera %d is invalid", i);
        CamDev& d = v[i];
        memcpy(d.R, c.R, sizeof(d.R));
        memcpy(d.t, c.t, sizeof(d.t));
        d.fx = c.fx;
        d.fy = c.fy;
        d.cx = c.cx;
        d.cy = c.cy;
        d.W = c.width;
        d.H = c.height;
        d.near_z = c.near_z;
        for (int k = 0; k < 3; ++k)
            d.campos[k] = (float)(-((double)c.R[k] * c.t[0] + (double)c.R[3 + k] * c.t[1] + (double)c.R[6 + k] * c.t[2]));
        d.limx = 0.f;  // set per call from clamp_fov
        d.limy = 0.f;
    }
    // The device copy is written by the next call's upload, in order on the context's stream
    // after every earlier call's work.  A buffer that is too small goes back to the pool; a
    // pooled buffer of a freed scene is taken before allocating (a scene loaded and freed every
    // step then allocates nothing, and no call waits for an upload in flight).
    if (s->d_cams && s->cams_cap < n_views) {
        ctx->cams_pool.emplace_back(s->cams_cap, s->d_cams);
        s->d_cams = nullptr;
        s->cams_cap = 0;
    }
    if (!s->d_cams) {
        for (size_t k = 0; k < ctx->cams_pool.size(); ++k)
            if (ctx->cams_pool[k].first >= n_views) {
                s->cams_cap = ctx->cams_pool[k].first;
                s->d_cams = ctx->cams_pool[k].second;
                ctx->cams_pool.erase(ctx->cams_pool.begin() + (long)k);
                break;
            }
    }
    if (!s->d_cams) {
        CUDA_TRY(ctx, cudaMalloc(&s->d_cams, sizeof(CamDev) * n_views));
        s->cams_cap = n_views;
    }
    s->cams = v;
    s->uploaded_clamp = -1.f;
    return CSGS_OK;
}

}  // extern "C"

namespace {

// Upload the cameras with the clamp limits of this call's options.
csgs_status upload_cams(csgs_ctx* ctx, SceneRec* s, const KOpts& k) {
    if (s->uploaded_clamp == k.clamp_fov) return CSGS_OK;
    s->uploaded_clamp = k.clamp_fov;
    for (auto& c : s->cams) {
        c.limx = (float)((double)k.clamp_fov * 0.5 * c.W / c.fx);
        c.limy = (float)((double)k.clamp_fov * 0.5 * c.H / c.fy);
    }
    CUDA_TRY(ctx, cudaMemcpyAsync(s->d_cams, s->cams.data(), sizeof(CamDev) * s->cams.size(), cudaMemcpyHostToDevice,
                                  ctx->st));
    // the host vector must outlive the copy
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    return CSGS_OK;
}

// Phase timer: events recorded on the stream around each phase; summed after the
// stream has been synchronised.
struct PhaseTimer {
    csgs_ctx* ctx;
    bool on;
    size_t used = 0;
    std::vector<std::pair<int, std::pair<size_t, size_t>>> spans;  // phase, (start, end) event index
    cudaEvent_t mark(cudaStream_t st) {
        if (used == ctx->evpool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ctx->evpool.push_back(e);
        }
        cudaEvent_t e = ctx->evpool[used++];
        cudaEventRecord(e, st);
        return e;
    }
    size_t begin(cudaStream_t st) {
        if (!on) return 0;
        mark(st);
        return used - 1;
    }
    void end(int phase, size_t b, cudaStream_t st) {
        if (!on) return;
        mark(st);
        spans.push_back({phase, {b, used - 1}});
    }
    void sum(double* ms3) {
        for (auto& sp : spans) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ctx->evpool[sp.second.first], ctx->evpool[sp.second.second]);
            ms3[sp.first] += t;
        }
    }
    // Length of the union of one phase's spans (spans on several streams overlap).
    double busy(int phase) {
        std::vector<std::pair<double, double>> iv;
        for (auto& sp : spans) {
            if (sp.first != phase) continue;
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ctx->evpool[0], ctx->evpool[sp.second.first]);
            cudaEventElapsedTime(&b, ctx->evpool[0], ctx->evpool[sp.second.second]);
            iv.push_back({a, b});
        }
        std::sort(iv.begin(), iv.end());
        double tot = 0.0, lo = 0.0, hi = -1e300;
        for (auto& x : iv) {
            if (x.first > hi) {
                if (hi > lo) tot += hi - lo;
                lo = x.first;
                hi = x.second;
            } else if (x.second > hi) {
                hi = x.second;
            }
        }
        if (hi > lo) tot += hi - lo;
        return tot;
    }
};

int auto_view_batch(int64_t n, int nv, int req) {
    if (req > 0) return req < nv ? req : nv;
    int64_t per = n * (int64_t)(sizeof(Splat) + 12);
    int64_t vb = ((int64_t)2 << 30) / (per > 0 ? per : 1);
    if (vb < 1) vb = 1;
    if (vb > 16) vb = 16;
    if (vb > nv) vb = nv;
    return (int)vb;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Enqueue the scoring of views [v0, v1) of one scene: no host synchronisation and no
// allocation (buffers must be sized), so it can be captured.  Three kinds of streams:
//   - projection (ctx->pst): view batch b into buffer set b % 2, once the compositing
//     that last read that set (batch b - 2) is done, so it runs ahead of the compositing;
//   - binning: view k in slot k % kBinSlots on the slot's high-priority stream, after the
//     projection of its batch and the compositing that last read the slot;
//   - compositing of view v on stream v % kCompStreams (0: the context's stream, others
//     ctx->cst), each view after its binning, so that the last tiles of one view overlap
//     the first of the next (the score reductions are max or sum atomics; the
//     per-instance pass-1 buffers exist once per stream); the image resolution, whose
//     per-view fold needs the views in turn, composites on the context's stream only;
//   - the reductions on the context's stream, after every compositing stream.
// Every side stream's last operation is waited on by the context's stream (the capture
// joins them).
csgs_status enqueue_scene_score(csgs_ctx* ctx, SceneRec* s, const KOpts& ko, int vb, int v0_all, int v1_all,
                                int stats, float* s_dev, double* S_dev, PhaseTimer& pt, long long& comp_launches) {
    const int64_t n = s->n;
    cudaStream_t st = ctx->st, ps = ctx->pst;
    csgs_status r;
    const SceneDev sd = scene_dev(*s);
    const int grid = s->tuned_sb > 0 ? s->tuned_sb : ctx->sort_blocks;
    set_u64(ctx->d_nconst, (unsigned long long)n, st);
    // the maxima of earlier query sets stay when accumulating
    if (!ko.accumulate) CUDA_TRY(ctx, cudaMemsetAsync(s_dev, 0, sizeof(float) * (size_t)n, st));
    if (ko.resolution == CSGS_RES_SCENE) CUDA_TRY(ctx, cudaMemsetAsync(&ctx->d_ctr->sumA, 0, sizeof(double), st));
    if (ko.resolution == CSGS_RES_IMAGE) CUDA_TRY(ctx, cudaMemsetAsync(ctx->vbuf.p, 0, sizeof(float) * (size_t)n, st));
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev_start, st));
    CUDA_TRY(ctx, cudaStreamWaitEvent(ps, ctx->ev_start, 0));
    const int ncs = ko.resolution == CSGS_RES_IMAGE ? 1 : kCompStreams;
    for (int c = 0; c + 1 < ncs; ++c) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->cst[c], ctx->ev_start, 0));
    bool freed_recorded[kBinSlots] = {};
    bool set_used[2] = {false, false};
    int view = 0, batch = 0;
    for (int v0 = v0_all; v0 < v1_all; v0 += vb, ++batch) {
        const int nb = (v1_all - v0) < vb ? (v1_all - v0) : vb;
        const int set = batch & 1;
        if (set_used[set]) {
            CUDA_TRY(ctx, cudaStreamWaitEvent(ps, ctx->ev_setfree[set], 0));
            for (int c = 0; c + 1 < ncs; ++c) CUDA_TRY(ctx, cudaStreamWaitEvent(ps, ctx->ev_csetfree[c][set], 0));
        }
        size_t e0 = pt.begin(ps);
        launch_project(sd, s->d_cams + v0, nb, nullptr, ko, P<Splat>(ctx->splats[set]), P<uint32_t>(ctx->keys[set]),
                       P<uint2>(ctx->rects[set]), ctx->d_ctr, ps);
        pt.end(0, e0, ps);
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev_proj[set], ps));
        for (int k = 0; k < nb; ++k, ++view) {
            const CamDev& cam = s->cams[v0 + k];
            const int sl = view % kBinSlots;
            BinSlot& slot = ctx->slot[sl];
            uint32_t* keys_v = P<uint32_t>(ctx->keys[set]) + (size_t)k * n;
            const uint2* rects_v = P<uint2>(ctx->rects[set]) + (size_t)k * n;
            CUDA_TRY(ctx, cudaStreamWaitEvent(slot.st, ctx->ev_proj[set], 0));
            if (freed_recorded[sl]) CUDA_TRY(ctx, cudaStreamWaitEvent(slot.st, slot.freed, 0));
            size_t e1 = pt.begin(slot.st);
            const uint32_t* iv = bin_batch(ctx, sl, n, 1, keys_v, rects_v, &cam, s->d_cams + v0 + k, ko, grid, slot.st);
            pt.end(1, e1, slot.st);
            // the view's tiles, longest lists first, at the end of its binning chain (the
            // compositing stream then only composites)
            tile_order(P<uint2>(slot.ranges), tiles_of(cam, ko.tile_lw, ko.tile_lh), P<uint32_t>(slot.torder) + 1,
                       P<uint32_t>(slot.torder), slot.st);
            CUDA_TRY(ctx, cudaEventRecord(slot.ready, slot.st));
            const int ci = view % ncs;  // compositing stream of this view
            cudaStream_t cs = ci ? ctx->cst[ci - 1] : st;
            CUDA_TRY(ctx, cudaStreamWaitEvent(cs, slot.ready, 0));
            CompositeArgs a{};
            a.ranges = P<uint2>(slot.ranges);
            a.work = P<uint32_t>(slot.torder);
            a.order = P<uint32_t>(slot.torder) + 1;
            a.inst_gid = iv;
            a.splats = P<Splat>(ctx->splats[set]) + (size_t)k * n;
            a.n_gauss = (int)n;
            a.cam = cam;
            a.o = ko;
            a.s_bits = reinterpret_cast<uint32_t*>(s_dev);
            a.s_sum = ko.resolution == CSGS_RES_IMAGE ? P<float>(ctx->vbuf) : s_dev;
            a.tile_sum = P<float>(ci ? ctx->tsumx[ci - 1] : ctx->tsum);
            a.mskbuf = P<uint8_t>(ci ? ctx->mskbx[ci - 1] : ctx->mskb);
            a.ctr = ctx->d_ctr;
            a.stats = stats & 1;
            if (ko.resolution == CSGS_RES_IMAGE)
                CUDA_TRY(ctx, cudaMemsetAsync(&ctx->d_ctr->sumA_view, 0, sizeof(double), st));

            size_t e2 = pt.begin(cs);
            launch_composite_score(a, cs);
            if (ko.resolution == CSGS_RES_IMAGE) image_fold(s_dev, P<float>(ctx->vbuf), n, &ctx->d_ctr->sumA_view, st);
            pt.end(2, e2, cs);
            CUDA_TRY(ctx, cudaEventRecord(slot.freed, cs));
            freed_recorded[sl] = true;
            ++comp_launches;
        }
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev_setfree[set], st));
        for (int c = 0; c + 1 < ncs; ++c) CUDA_TRY(ctx, cudaEventRecord(ctx->ev_csetfree[c][set], ctx->cst[c]));
        set_used[set] = true;
        if ((r = launch_check(ctx, "score kernels"))) return r;
    }
    for (int c = 0; c + 1 < ncs; ++c) {
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev_cdone[c], ctx->cst[c]));
        CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_cdone[c], 0));
    }
    if (ko.resolution == CSGS_RES_SCENE) scene_normalise(s_dev, n, &ctx->d_ctr->sumA, st);
    sum_scores(s_dev, n, P<double>(ctx->partial), S_dev, st);
    return launch_check(ctx, "score reduction");
}

// Size every buffer the scoring of these scenes needs.
csgs_status prepare_scoring(csgs_ctx* ctx, SceneRec** sc, const int* vb, int ns, const KOpts& ko) {
    csgs_status r;
    int64_t nmax = 0;
    int vbmax = 1, tiles = 0;
    for (int k = 0; k < ns; ++k) {
        if ((r = upload_cams(ctx, sc[k], ko))) return r;
        if (sc[k]->n > nmax) nmax = sc[k]->n;
        if (vb[k] > vbmax) vbmax = vb[k];
        // ranges for the shape with the most tiles (8x8), so that any scene's shape fits
        for (auto& c : sc[k]->cams)
            if (tiles_of(c, 3, 3) > tiles) tiles = tiles_of(c, 3, 3);
    }
    if ((r = ensure_view_buffers(ctx, nmax, vbmax, tiles))) return r;
    if ((r = ensure(ctx, ctx->partial, sizeof(double) * 1024))) return r;
    if ((r = ensure(ctx, ctx->Sdev, sizeof(double) * (ns + 1)))) return r;
    if (ko.resolution == CSGS_RES_IMAGE && (r = ensure(ctx, ctx->vbuf, sizeof(float) * (size_t)nmax))) return r;
    for (int c = 0; c < kCompStreams; ++c) {
        DevBuf& ts = c ? ctx->tsumx[c - 1] : ctx->tsum;
        DevBuf& mb = c ? ctx->mskbx[c - 1] : ctx->mskb;
        if (ko.resolution == CSGS_RES_TILE && (r = ensure(ctx, ts, sizeof(float) * (size_t)ctx->cap))) return r;
        if ((ko.resolution == CSGS_RES_PIXEL || ko.resolution == CSGS_RES_CHANNEL) &&
            (r = ensure(ctx, mb, (size_t)ctx->cap)))
            return r;
    }
    return CSGS_OK;
}

// The call's conventions with the scene's tuned tile shape and persistent grid where the
// caller left them to the library (CSGS_TILE_AUTO, persist_ctas 0).
KOpts scene_kopts(const KOpts& ko, const SceneRec* s, const csgs_score_opts* opts) {
    KOpts k = ko;
    if (opts->tile_shape == CSGS_TILE_AUTO && s->tuned_shape) set_tile_shape(&k, s->tuned_shape);
    if (opts->persist_ctas == 0) k.persist_ctas = s->tuned_persist;
    return k;
}

int scene_view_batch(const SceneRec* s, const csgs_score_opts* opts) {
    if (opts->view_batch > 0) return opts->view_batch < (int)s->cams.size() ? opts->view_batch : (int)s->cams.size();
    if (s->tuned_vb > 0) return s->tuned_vb < (int)s->cams.size() ? s->tuned_vb : (int)s->cams.size();
    return auto_view_batch(s->n, (int)s->cams.size(), 0);
}

}  // namespace

extern "C" {

csgs_status csgs_score(csgs_ctx* ctx, int32_t scene_id, const csgs_score_opts* opts, float* s_dev, double* S_out) {
    if (!ctx) return CSGS_E_INVAL;
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (!s_dev) return fail(ctx, CSGS_E_INVAL, "s_dev is NULL");
    if (s->cams.empty()) return fail(ctx, CSGS_E_INVAL, "no query views set");
    KOpts ko;
    csgs_status r;
    if ((r = make_kopts(ctx, opts, &ko))) return r;
    ko = scene_kopts(ko, s, opts);
    cudaSetDevice(ctx->device);
    const int nv = (int)s->cams.size();
    const int vb = scene_view_batch(s, opts);
    if ((r = prepare_scoring(ctx, &s, &vb, 1, ko))) return r;
    int64_t rays = 0;
    for (auto& c : s->cams) rays += (int64_t)c.W * c.H;
    cudaStream_t st = ctx->st;
    int retries = 0;
    const long long l0 = launches();
    PhaseTimer pt{ctx, (opts->collect_stats & 2) != 0};
    long long comp_launches = 0;
    for (;;) {
        pt.used = 0;
        pt.spans.clear();
        comp_launches = 0;
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st));
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, st));
        if ((r = enqueue_scene_score(ctx, s, ko, vb, 0, nv, opts->collect_stats, s_dev, P<double>(ctx->Sdev), pt,
                                     comp_launches)))
            return r;
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, st));
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_S, ctx->Sdev.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        if ((r = read_counters(ctx))) return r;
        if (ctx->h_ctr->err & (kErrCapacity | kErrDepthRange)) {
            if (++retries > 3) return fail(ctx, CSGS_E_DEVICE_CHECK, "instance capacity overflow persists");
            if ((r = widen_or_grow(ctx, ko))) return r;
            if ((r = prepare_scoring(ctx, &s, &vb, 1, ko))) return r;
            continue;
        }
        break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.views = nv;
    ctx->stats.rays = rays;
    ctx->stats.instances = (int64_t)ctx->h_ctr->inst_total;
    ctx->stats.pairs_evaluated = (int64_t)ctx->h_ctr->pairs_eval;
    ctx->stats.pairs_hit = (int64_t)ctx->h_ctr->pairs_hit;
    ctx->stats.pairs_evaluated2 = (int64_t)ctx->h_ctr->pairs_eval2;
    ctx->stats.pairs_hit2 = (int64_t)ctx->h_ctr->pairs_hit2;
    ctx->stats.capacity_retries = retries;
    ctx->stats.score_ms = ms;
    ctx->stats.kernel_launches = launches() - l0;
    ctx->stats.composite_launches = comp_launches;
    ctx->stats.queries = (int64_t)ctx->h_ctr->queries;
    ctx->stats.entries_staged = (int64_t)ctx->h_ctr->staged1;
    ctx->stats.entries_staged2 = (int64_t)ctx->h_ctr->staged2;
    ctx->stats.view_batches = (nv + vb - 1) / vb;
    ctx->stats.warp_entries = (int64_t)ctx->h_ctr->wentries1;
    ctx->stats.warp_entries2 = (int64_t)ctx->h_ctr->wentries2;
    ctx->stats.objective_sum = ctx->h_ctr->sumA;
    {
        double ph[3] = {0.0, 0.0, 0.0};
        pt.sum(ph);
        ctx->stats.project_ms = ph[0];
        ctx->stats.sort_ms = ph[1];
        ctx->stats.composite_ms = ph[2];
        ctx->stats.composite_busy_ms = pt.busy(2);
    }
    const double S = ctx->h_S[0];
    if (S_out) *S_out = S;
    if (!(S > 0.0)) return fail(ctx, CSGS_E_EMPTY, "every query has A = 0: total sensitivity is zero");
    return CSGS_OK;
}

csgs_status csgs_score_batch(csgs_ctx* ctx, int32_t n_scenes, const int32_t* scene_ids, const csgs_score_opts* opts,
                             float* const* s_devs, double* S_out, int32_t use_graph) {
    if (!ctx) return CSGS_E_INVAL;
    if (n_scenes <= 0 || n_scenes > 64 || !scene_ids || !s_devs || !S_out)
        return fail(ctx, CSGS_E_INVAL, "bad batch arguments");
    KOpts ko;
    csgs_status r;
    if ((r = make_kopts(ctx, opts, &ko))) return r;
    cudaSetDevice(ctx->device);
    std::vector<SceneRec*> sc(n_scenes);
    std::vector<int> vb(n_scenes);
    std::vector<KOpts> kos(n_scenes);  // per scene: its tile shape
    int64_t rays = 0;
    for (int k = 0; k < n_scenes; ++k) {
        sc[k] = get_scene(ctx, scene_ids[k]);
        if (!sc[k]) return scene_fail(ctx, scene_ids[k]);
        if (sc[k]->cams.empty() || !s_devs[k]) return fail(ctx, CSGS_E_INVAL, "bad scene %d in batch", k);
        vb[k] = scene_view_batch(sc[k], opts);
        kos[k] = scene_kopts(ko, sc[k], opts);
        for (auto& c : sc[k]->cams) rays += (int64_t)c.W * c.H;
    }
    if ((r = prepare_scoring(ctx, sc.data(), vb.data(), n_scenes, ko))) return r;
    cudaStream_t st = ctx->st;
    // identity of the captured work: scenes, their sizes and views, outputs, options, buffers
    std::string key((const char*)opts, sizeof(*opts));
    key.append((const char*)scene_ids, sizeof(int32_t) * n_scenes);
    key.append((const char*)s_devs, sizeof(float*) * n_scenes);
    // (the launches bake in the scene pointers, the host copies of the cameras and every
    // work-buffer address, so all of them are part of the key)
    for (int k = 0; k < n_scenes; ++k) {
        const int64_t meta[7] = {(int64_t)sc[k]->cams.size(), vb[k], (int64_t)(uintptr_t)sc[k]->d_cams,
                                 sc[k]->tuned_sb, kos[k].tile_lw, kos[k].tile_lh, kos[k].persist_ctas};
        key.append((const char*)meta, sizeof(meta));
        const SceneDev sd = scene_dev(*sc[k]);
        key.append((const char*)&sd, sizeof(sd));
        key.append((const char*)sc[k]->cams.data(), sizeof(CamDev) * sc[k]->cams.size());
    }
    PhaseTimer off{ctx, false};
    long long cl = 0;
    const long long l0 = launches();
    float ms = 0.f;
    long long replayed = 0;
    for (int attempt = 0;; ++attempt) {
        for (int k = 0; k < n_scenes; ++k) kos[k].narrow_keys = ko.narrow_keys;
        const int64_t bmeta[4] = {(int64_t)ctx->cap, ctx->sort_blocks, (int64_t)ctx->buf_gen, (int64_t)ko.narrow_keys};
        const std::string full_key = key + std::string((const char*)bmeta, sizeof(bmeta));
        const bool replay = use_graph && ctx->graph_exec && ctx->graph_key == full_key;
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, st));
        if (replay) {
            CUDA_TRY(ctx, cudaGraphLaunch(ctx->graph_exec, st));
            replayed += ctx->graph_nodes_launches;
        } else if (use_graph && attempt > 0) {
            // capture the whole batch (every launch and memset of every scene) once
            if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
            cudaGraph_t g = nullptr;
            const long long lc0 = launches();
            CUDA_TRY(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            csgs_status er = CSGS_OK;
            cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st);
            for (int k = 0; k < n_scenes && !er; ++k)
                er = enqueue_scene_score(ctx, sc[k], kos[k], vb[k], 0, (int)sc[k]->cams.size(), 0, s_devs[k],
                                         P<double>(ctx->Sdev) + k, off, cl);
            cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (er) {
                if (g) cudaGraphDestroy(g);
                return er;
            }
            if (ce != cudaSuccess) return fail(ctx, CSGS_E_CUDA, "stream capture: %s", cudaGetErrorString(ce));
            // keep the capturing streams' priorities (binning ahead of compositing) in the replay
            ce = cudaGraphInstantiate(&ctx->graph_exec, g, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return fail(ctx, CSGS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            ctx->graph_key = full_key;
            ctx->graph_nodes_launches = launches() - lc0;
            CUDA_TRY(ctx, cudaGraphLaunch(ctx->graph_exec, st));
        } else {
            // eager pass: settles the instance capacity before a capture
            CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st));
            for (int k = 0; k < n_scenes; ++k)
                if ((r = enqueue_scene_score(ctx, sc[k], kos[k], vb[k], 0, (int)sc[k]->cams.size(), 0, s_devs[k],
                                             P<double>(ctx->Sdev) + k, off, cl)))
                    return r;
        }
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, st));
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_S, ctx->Sdev.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        if ((r = read_counters(ctx))) return r;
        if (ctx->h_ctr->err & (kErrCapacity | kErrDepthRange)) {
            if (attempt > 4) return fail(ctx, CSGS_E_DEVICE_CHECK, "instance capacity overflow persists");
            if ((r = widen_or_grow(ctx, ko))) return r;
            if ((r = prepare_scoring(ctx, sc.data(), vb.data(), n_scenes, ko))) return r;
            ctx->graph_key.clear();
            continue;
        }
        if (use_graph && !replay && attempt == 0) continue;  // now capture
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        break;
    }
    CUDA_TRY(ctx, cudaMemcpy(S_out, ctx->Sdev.p, sizeof(double) * n_scenes, cudaMemcpyDeviceToHost));
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    int64_t views = 0;
    for (int k = 0; k < n_scenes; ++k) views += (int64_t)sc[k]->cams.size();
    ctx->stats.views = views;
    ctx->stats.rays = rays;
    ctx->stats.instances = (int64_t)ctx->h_ctr->inst_total;
    ctx->stats.score_ms = ms;
    ctx->stats.kernel_launches = launches() - l0 + replayed;
    ctx->stats.queries = (int64_t)ctx->h_ctr->queries;
    return CSGS_OK;
}

csgs_status csgs_autotune(csgs_ctx* ctx, int32_t scene_id, const csgs_score_opts* opts, int32_t probe_views,
                          csgs_tuning* out) {
    if (!ctx) return CSGS_E_INVAL;
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (s->cams.empty()) return fail(ctx, CSGS_E_INVAL, "scene %d has no query views", scene_id);
    KOpts ko;
    csgs_status r;
    if ((r = make_kopts(ctx, opts, &ko))) return r;
    cudaSetDevice(ctx->device);
    const int nv = (int)s->cams.size();
    const int pv = probe_views > 0 && probe_views < nv ? probe_views : (nv < 16 ? nv : 16);
    const int vbs[5] = {1, 2, 4, 8, 16};
    // radix-sort grids: from one CTA per two SMs (binning holds few SM slots beside the
    // compositing) to twelve per SM (binning alone as fast as it goes)
    const int gs[6] = {74, 148, 148 * 2, 148 * 4, 148 * 8, 148 * 12};
    float* s_tmp = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&s_tmp, sizeof(float) * (size_t)s->n));
    std::unique_ptr<float, cudaError_t (*)(void*)> s_tmp_owner(s_tmp, cudaFree);
    PhaseTimer off{ctx, false};
    long long cl = 0;
    int grows = 0;
    const int saved_sb = s->tuned_sb;
    // time the scoring of the first pv views with view batch vb, sort grid g and the tile
    // shape of kk (best of two runs after a warm-up that also settles the capacity)
    auto trial = [&](int vb, int g, KOpts& kk, float* t_out) -> csgs_status {
        csgs_status e;
        s->tuned_sb = g;
        if ((e = prepare_scoring(ctx, &s, &vb, 1, kk))) return e;
        float t = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), ctx->st));
            CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->st));
            if ((e = enqueue_scene_score(ctx, s, kk, vb, 0, pv, 0, s_tmp, P<double>(ctx->Sdev), off, cl))) return e;
            CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->st));
            if ((e = read_counters(ctx))) return e;
            if (ctx->h_ctr->err & (kErrCapacity | kErrDepthRange)) {
                if (++grows > 4) return fail(ctx, CSGS_E_DEVICE_CHECK, "instance capacity overflow persists");
                if ((e = widen_or_grow(ctx, kk)) || (e = prepare_scoring(ctx, &s, &vb, 1, kk))) return e;
                ko.narrow_keys = kk.narrow_keys;
                --rep;
                continue;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            if (rep > 0 && ms < t) t = ms;
        }
        *t_out = t;
        return CSGS_OK;
    };
    // view batch x sort grid at the requested shape (16x16 when left to the library), then
    // the tile shapes at the best pair
    float best = 1e30f;
    int best_vb = auto_view_batch(s->n, nv, 0), best_g = saved_sb > 0 ? saved_sb : ctx->sort_blocks;
    int best_shape = opts->tile_shape == CSGS_TILE_AUTO ? CSGS_TILE_16X16 : opts->tile_shape;
    KOpts k0 = ko;
    set_tile_shape(&k0, best_shape);
    r = CSGS_OK;
    for (int vb : vbs) {
        if (vb > pv) continue;
        if ((int64_t)vb * s->n * (int64_t)(sizeof(Splat) + 12) > ((int64_t)4 << 30)) continue;
        for (int g : gs) {
            float t = 1e30f;
            k0.narrow_keys = ko.narrow_keys;
            if ((r = trial(vb, g, k0, &t))) break;
            if (t < best) {
                best = t;
                best_vb = vb;
                best_g = g;
            }
        }
        if (r) break;
    }
    if (!r && opts->tile_shape == CSGS_TILE_AUTO && ko.resolution != CSGS_RES_TILE) {
        for (int shape : {CSGS_TILE_32X8, CSGS_TILE_16X8, CSGS_TILE_8X8}) {
            KOpts kk = ko;
            set_tile_shape(&kk, shape);
            float t = 1e30f;
            if ((r = trial(best_vb, best_g, kk, &t))) break;
            if (t < best) {
                best = t;
                best_shape = shape;
            }
        }
    }
    // persistent compositing launches (per-pixel score) of r, r - 1 and r - 2 CTAs per SM,
    // r the kernel's resident limit (fewer leave SM slots to the binning that runs beside it)
    int best_persist = ko.persist_ctas;
    if (!r && opts->persist_ctas == 0 && ko.resolution == CSGS_RES_PIXEL) {
        KOpts kk = ko;
        set_tile_shape(&kk, best_shape);
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        const int res = composite_resident_ctas(kk.tile_lw, kk.tile_lh);
        for (int m = res; m >= res - 2 && m >= 1 && sms > 0; --m) {
            kk.persist_ctas = m * sms;
            kk.narrow_keys = ko.narrow_keys;
            float t = 1e30f;
            if ((r = trial(best_vb, best_g, kk, &t))) break;
            if (t < best) {
                best = t;
                best_persist = kk.persist_ctas;
            }
        }
    }
    if (r) {
        s->tuned_sb = saved_sb;
        return r;
    }
    s->tuned_sb = best_g;
    s->tuned_vb = best_vb;
    ctx->sort_blocks = best_g;  // also the grid of scenes not tuned themselves
    if (opts->tile_shape == CSGS_TILE_AUTO && ko.resolution != CSGS_RES_TILE) s->tuned_shape = best_shape;
    if (opts->persist_ctas == 0 && ko.resolution == CSGS_RES_PIXEL) s->tuned_persist = best_persist;
    ctx->graph_key.clear();
    if (out) {
        out->view_batch = best_vb;
        out->sort_blocks = best_g;
        out->tile_shape = best_shape;
        out->persist_ctas = best_persist;
        out->probe_ms = best;
    }
    return CSGS_OK;
}

static csgs_status sample_common(csgs_ctx* ctx, const double* p, int64_t n, int64_t m, uint64_t seed, int32_t* idx,
                                 float* w, int64_t* n_distinct, int32_t* draws) {
    csgs_status r;
    const size_t nb = (size_t)(n + 2047) / 2048 + 64;
    if ((r = ensure(ctx, ctx->C, sizeof(unsigned long long) * (size_t)n))) return r;
    if ((r = ensure(ctx, ctx->counts, sizeof(uint32_t) * (size_t)n))) return r;
    if ((r = ensure(ctx, ctx->ctmp, sizeof(unsigned long long) * nb))) return r;
    if ((r = ensure(ctx, ctx->stmp, sizeof(uint32_t) * nb))) return r;
    if ((r = ensure(ctx, ctx->nout, sizeof(uint32_t) * 2))) return r;
    SampleTemp t;
    t.partial = nullptr;
    t.S = nullptr;
    t.C = P<unsigned long long>(ctx->C);
    t.counts = P<uint32_t>(ctx->counts);
    t.scan_tmp = P<uint32_t>(ctx->stmp);
    t.C_tmp = P<unsigned long long>(ctx->ctmp);
    t.n_out = P<uint32_t>(ctx->nout);
    sample_draws(p, n, m, seed, t, draws, idx, w, ctx->st);
    if ((r = launch_check(ctx, "sampling kernels"))) return r;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_u32, t.n_out, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->st));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    if (n_distinct) *n_distinct = (int64_t)ctx->h_u32[0];
    return CSGS_OK;
}

csgs_status csgs_sample_coreset(csgs_ctx* ctx, const float* s_dev, int64_t n, int64_t m, uint64_t seed,
                                int32_t* idx_dev, float* w_dev, int64_t* n_distinct) {
    if (!ctx) return CSGS_E_INVAL;
    if (!s_dev || !idx_dev || !w_dev) return fail(ctx, CSGS_E_INVAL, "null argument");
    if (n <= 0 || n >= (1ll << 31)) return fail(ctx, CSGS_E_INVAL, "n = %lld out of range", (long long)n);
    if (m <= 0 || m >= (1ll << 31)) return fail(ctx, CSGS_E_INVAL, "m = %lld out of range", (long long)m);
    cudaSetDevice(ctx->device);
    csgs_status r;
    if ((r = ensure(ctx, ctx->partial, sizeof(double) * 1024))) return r;
    if ((r = ensure(ctx, ctx->Sdev, sizeof(double) * 2))) return r;
    if ((r = ensure(ctx, ctx->p, sizeof(double) * (size_t)n))) return r;
    sum_scores(s_dev, n, P<double>(ctx->partial), P<double>(ctx->Sdev), ctx->st);
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_S, ctx->Sdev.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    const double S = ctx->h_S[0];
    if (!isfinite(S) || S < 0.0) return fail(ctx, CSGS_E_INVAL, "scores are negative or not finite");
    if (!(S > 0.0)) return fail(ctx, CSGS_E_EMPTY, "total sensitivity is zero");
    probabilities_from_scores(s_dev, n, P<double>(ctx->Sdev), P<double>(ctx->p), ctx->st);
    return sample_common(ctx, P<double>(ctx->p), n, m, seed, idx_dev, w_dev, n_distinct, nullptr);
}

csgs_status csgs_sample_coreset_p(csgs_ctx* ctx, const double* p_dev, int64_t n, int64_t m, uint64_t seed,
                                  int32_t* idx_dev, float* w_dev, int64_t* n_distinct, int32_t* draws_dev) {
    if (!ctx) return CSGS_E_INVAL;
    if (!p_dev || !idx_dev || !w_dev) return fail(ctx, CSGS_E_INVAL, "null argument");
    if (n <= 0 || n >= (1ll << 31)) return fail(ctx, CSGS_E_INVAL, "n = %lld out of range", (long long)n);
    if (m <= 0 || m >= (1ll << 31)) return fail(ctx, CSGS_E_INVAL, "m = %lld out of range", (long long)m);
    cudaSetDevice(ctx->device);
    return sample_common(ctx, p_dev, n, m, seed, idx_dev, w_dev, n_distinct, draws_dev);
}

csgs_status csgs_render(csgs_ctx* ctx, int32_t scene_id, int32_t view, const int32_t* idx_dev, const float* w_dev,
                        int64_t n_sel, const csgs_score_opts* opts, float* rgb_dev, float* T_dev) {
    if (!ctx) return CSGS_E_INVAL;
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (view < 0 || view >= (int32_t)s->cams.size()) return fail(ctx, CSGS_E_INVAL, "bad view %d", view);
    if (!rgb_dev) return fail(ctx, CSGS_E_INVAL, "rgb_dev is NULL");
    if ((idx_dev == nullptr) != (w_dev == nullptr)) return fail(ctx, CSGS_E_INVAL, "idx and w must both be given");
    if (idx_dev && (n_sel < 0 || n_sel > s->n)) return fail(ctx, CSGS_E_INVAL, "n_sel out of range");
    KOpts ko;
    csgs_status r;
    if ((r = make_kopts(ctx, opts, &ko))) return r;
    ko = scene_kopts(ko, s, opts);
    cudaSetDevice(ctx->device);
    if ((r = upload_cams(ctx, s, ko))) return r;
    const int64_t n = s->n;
    const CamDev& cam = s->cams[view];
    if ((r = ensure_view_buffers(ctx, n, 1, tiles_of(cam, ko.tile_lw, ko.tile_lh)))) return r;
    cudaStream_t st = ctx->st;
    const float* wts = nullptr;
    if (idx_dev) {
        if ((r = ensure(ctx, ctx->wfull, sizeof(float) * (size_t)n))) return r;
        wts = P<float>(ctx->wfull);
    }
    set_u64(ctx->d_nconst, (unsigned long long)n, st);
    const SceneDev sd = scene_dev(*s);
    int retries = 0;
    const long long l0 = launches();
    for (;;) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st));
        if (idx_dev) {
            CUDA_TRY(ctx, cudaMemsetAsync(ctx->wfull.p, 0, sizeof(float) * (size_t)n, st));
            scatter_weights(idx_dev, w_dev, n_sel, P<float>(ctx->wfull), n, ctx->d_ctr, st);
        }
        launch_project(sd, s->d_cams + view, 1, wts, ko, P<Splat>(ctx->splats[0]), P<uint32_t>(ctx->keys[0]),
                       P<uint2>(ctx->rects[0]), ctx->d_ctr, st);
        const uint32_t* iv = bin_batch(ctx, 0, n, 1, P<uint32_t>(ctx->keys[0]), P<uint2>(ctx->rects[0]), &cam,
                                       s->d_cams + view, ko, ctx->sort_blocks, st);
        CompositeArgs a{};
        a.ranges = P<uint2>(ctx->slot[0].ranges);
        a.inst_gid = iv;
        a.splats = P<Splat>(ctx->splats[0]);
        a.n_gauss = (int)n;
        a.cam = cam;
        a.o = ko;
        a.rgb = rgb_dev;
        a.T = T_dev;
        a.ctr = ctx->d_ctr;
        a.stats = opts->collect_stats & 1;
        launch_composite_render(a, st);
        if ((r = launch_check(ctx, "render kernels"))) return r;
        if ((r = read_counters(ctx))) return r;
        if (ctx->h_ctr->err & (kErrCapacity | kErrDepthRange)) {
            if (++retries > 3) return fail(ctx, CSGS_E_DEVICE_CHECK, "instance capacity overflow persists");
            if ((r = widen_or_grow(ctx, ko))) return r;
            continue;
        }
        break;
    }
    if (ctx->h_ctr->err & kErrIndex) return fail(ctx, CSGS_E_INVAL, "coreset index out of range");
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.views = 1;
    ctx->stats.rays = (int64_t)cam.W * cam.H;
    ctx->stats.instances = (int64_t)ctx->h_ctr->inst_total;
    ctx->stats.pairs_evaluated = (int64_t)ctx->h_ctr->pairs_eval;
    ctx->stats.pairs_hit = (int64_t)ctx->h_ctr->pairs_hit;
    ctx->stats.violations = (int64_t)ctx->h_ctr->violations;
    ctx->stats.capacity_retries = retries;
    ctx->stats.kernel_launches = launches() - l0;
    ctx->stats.composite_launches = 1 + retries;
    return CSGS_OK;
}

int64_t csgs_kernel_launch_count(void) { return (int64_t)launches(); }

static csgs_status tc_gemm_common(csgs_ctx* ctx, const void* A_dev, const void* B_dev, float* C_dev, int32_t K,
                                  int32_t N, long long first_wait, int mn_major = 0) {
    if (!ctx) return CSGS_E_INVAL;
    if (!A_dev || !B_dev || !C_dev) return fail(ctx, CSGS_E_INVAL, "null argument");
    if (K < 16 || K > 128 || K % 16 || N < 16 || N > 256 || N % 16)
        return fail(ctx, CSGS_E_INVAL, "unsupported GEMM shape K=%d N=%d", K, N);
    cudaSetDevice(ctx->device);
    CUDA_TRY(ctx, cudaMemsetAsync(&ctx->d_ctr->err, 0, sizeof(uint32_t), ctx->st));
    gemm_check(A_dev, B_dev, C_dev, K, N, reinterpret_cast<int*>(&ctx->d_ctr->err), first_wait, mn_major, ctx->st);
    csgs_status r;
    if ((r = launch_check(ctx, "tensor-core GEMM"))) return r;
    if ((r = read_counters(ctx))) return r;
    if (ctx->h_ctr->err & 2) return fail(ctx, CSGS_E_TIMEOUT, "MMA chain did not drain within the full budget");
    if (ctx->h_ctr->err) return fail(ctx, CSGS_E_TIMEOUT, "MMA completion not observed");
    return CSGS_OK;
}

csgs_status csgs_debug_tc_gemm(csgs_ctx* ctx, const void* A_dev, const void* B_dev, float* C_dev, int32_t K,
                               int32_t N) {
    return tc_gemm_common(ctx, A_dev, B_dev, C_dev, K, N, -1);
}

csgs_status csgs_debug_tc_gemm_mn(csgs_ctx* ctx, const void* A_dev, const void* B_dev, float* C_dev, int32_t K,
                                  int32_t N) {
    return tc_gemm_common(ctx, A_dev, B_dev, C_dev, K, N, -1, 1);
}

csgs_status csgs_debug_tc_gemm_wait(csgs_ctx* ctx, const void* A_dev, const void* B_dev, float* C_dev, int32_t K,
                                    int32_t N, int64_t first_wait_cycles) {
    if (first_wait_cycles < 0) return fail(ctx, CSGS_E_INVAL, "negative wait budget");
    return tc_gemm_common(ctx, A_dev, B_dev, C_dev, K, N, (long long)first_wait_cycles);
}

csgs_status csgs_debug_gelu(csgs_ctx* ctx, const float* z_dev, int64_t n, float* out_dev) {
    if (!ctx) return CSGS_E_INVAL;
    if (!z_dev || !out_dev || n <= 0 || n > (1ll << 30)) return fail(ctx, CSGS_E_INVAL, "bad arguments");
    cudaSetDevice(ctx->device);
    debug_gelu(z_dev, (int)n, out_dev, ctx->st);
    return launch_check(ctx, "GELU check");
}

double csgs_theorem2_sample_size(double S, double eps_c, double delta, int64_t n_queries) {
    if (!(S > 0.0) || !(eps_c > 0.0) || !(delta > 0.0) || n_queries <= 0) return 0.0;
    return ceil(3.0 * S / (eps_c * eps_c) * log(2.0 * (double)n_queries / delta));
}

double csgs_theorem3_eps(double gamma, double eps_c) {
    const double a = 1.0 - exp(-gamma) * (1.0 - eps_c);
    const double b = exp(gamma) * (1.0 + eps_c) - 1.0;
    return a > b ? a : b;
}

csgs_status csgs_transfer(csgs_ctx* ctx, int32_t scene_id, int32_t view, const int32_t* idx_dev, const float* w_dev,
                          int64_t n_sel, const csgs_score_opts* opts, float* out_dev) {
    if (!ctx) return CSGS_E_INVAL;
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (view < 0 || view >= (int32_t)s->cams.size()) return fail(ctx, CSGS_E_INVAL, "bad view %d", view);
    if (!out_dev || !idx_dev || !w_dev) return fail(ctx, CSGS_E_INVAL, "null argument");
    if (n_sel < 0 || n_sel > s->n) return fail(ctx, CSGS_E_INVAL, "n_sel out of range");
    KOpts ko;
    csgs_status r;
    if ((r = make_kopts(ctx, opts, &ko))) return r;
    ko = scene_kopts(ko, s, opts);
    cudaSetDevice(ctx->device);
    if ((r = upload_cams(ctx, s, ko))) return r;
    const int64_t n = s->n;
    const CamDev& cam = s->cams[view];
    if ((r = ensure_view_buffers(ctx, n, 1, tiles_of(cam, ko.tile_lw, ko.tile_lh)))) return r;
    if ((r = ensure(ctx, ctx->wfull, sizeof(float) * (size_t)n))) return r;
    cudaStream_t st = ctx->st;
    set_u64(ctx->d_nconst, (unsigned long long)n, st);
    const SceneDev sd = scene_dev(*s);
    int retries = 0;
    for (;;) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st));
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->wfull.p, 0, sizeof(float) * (size_t)n, st));
        scatter_weights(idx_dev, w_dev, n_sel, P<float>(ctx->wfull), n, ctx->d_ctr, st);
        launch_project(sd, s->d_cams + view, 1, nullptr, ko, P<Splat>(ctx->splats[0]), P<uint32_t>(ctx->keys[0]),
                       P<uint2>(ctx->rects[0]), ctx->d_ctr, st);
        const uint32_t* iv = bin_batch(ctx, 0, n, 1, P<uint32_t>(ctx->keys[0]), P<uint2>(ctx->rects[0]), &cam,
                                       s->d_cams + view, ko, ctx->sort_blocks, st);
        CompositeArgs a{};
        a.ranges = P<uint2>(ctx->slot[0].ranges);
        a.inst_gid = iv;
        a.splats = P<Splat>(ctx->splats[0]);
        a.n_gauss = (int)n;
        a.cam = cam;
        a.o = ko;
        a.wsel = P<float>(ctx->wfull);
        a.aux = out_dev;
        a.ctr = ctx->d_ctr;
        launch_composite_transfer(a, st);
        if ((r = launch_check(ctx, "transfer kernels"))) return r;
        if ((r = read_counters(ctx))) return r;
        if (ctx->h_ctr->err & (kErrCapacity | kErrDepthRange)) {
            if (++retries > 3) return fail(ctx, CSGS_E_DEVICE_CHECK, "instance capacity overflow persists");
            if ((r = widen_or_grow(ctx, ko))) return r;
            continue;
        }
        break;
    }
    if (ctx->h_ctr->err & kErrIndex) return fail(ctx, CSGS_E_INVAL, "coreset index out of range");
    return CSGS_OK;
}

csgs_status csgs_scale_scores(csgs_ctx* ctx, float* s_dev, int64_t n, double factor) {
    if (!ctx) return CSGS_E_INVAL;
    if (!s_dev || n <= 0) return fail(ctx, CSGS_E_INVAL, "bad score array");
    if (!std::isfinite(factor) || factor < 0.0) return fail(ctx, CSGS_E_INVAL, "bad scale factor");
    cudaSetDevice(ctx->device);
    scale_scores(s_dev, n, factor, ctx->st);
    return launch_check(ctx, "score scaling");
}

csgs_status csgs_total_sensitivity(csgs_ctx* ctx, const float* s_dev, int64_t n, double* S_out) {
    if (!ctx) return CSGS_E_INVAL;
    if (!s_dev || n <= 0 || !S_out) return fail(ctx, CSGS_E_INVAL, "bad arguments");
    cudaSetDevice(ctx->device);
    csgs_status r;
    if ((r = ensure(ctx, ctx->partial, sizeof(double) * 1024))) return r;
    if ((r = ensure(ctx, ctx->Sdev, sizeof(double) * 2))) return r;
    sum_scores(s_dev, n, P<double>(ctx->partial), P<double>(ctx->Sdev), ctx->st);
    if ((r = launch_check(ctx, "total sensitivity"))) return r;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_S, ctx->Sdev.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    *S_out = ctx->h_S[0];
    return CSGS_OK;
}

csgs_status csgs_sync(csgs_ctx* ctx) {
    if (!ctx) return CSGS_E_INVAL;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    return CSGS_OK;
}

csgs_status csgs_get_stats(csgs_ctx* ctx, csgs_stats* out) {
    if (!ctx || !out) return CSGS_E_INVAL;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    *out = ctx->stats;
    return CSGS_OK;
}

csgs_status csgs_debug_project(csgs_ctx* ctx, int32_t scene_id, int32_t view, const csgs_score_opts* opts,
                               float* out_dev) {
    if (!ctx) return CSGS_E_INVAL;
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (view < 0 || view >= (int32_t)s->cams.size()) return fail(ctx, CSGS_E_INVAL, "bad view %d", view);
    if (!out_dev) return fail(ctx, CSGS_E_INVAL, "out_dev is NULL");
    KOpts ko;
    csgs_status r;
    if ((r = make_kopts(ctx, opts, &ko))) return r;
    cudaSetDevice(ctx->device);
    if ((r = upload_cams(ctx, s, ko))) return r;
    launch_debug_project(scene_dev(*s), s->d_cams + view, ko, out_dev, ctx->st);
    return launch_check(ctx, "debug projection");
}

}  // extern "C"

// ======================================================================= surrogate model

namespace {

csgs_status mlp_alloc(csgs_ctx* ctx) {
    csgs_status r;
    const size_t np = sizeof(float) * kMlpParams;
    if ((r = ensure(ctx, ctx->mP, np)) || (r = ensure(ctx, ctx->mM, np)) || (r = ensure(ctx, ctx->mV, np)) ||
        (r = ensure(ctx, ctx->mG, np)) || (r = ensure(ctx, ctx->mW1b, 2 * 256 * 64)) ||
        (r = ensure(ctx, ctx->mW2b, 2 * 256 * 256)) || (r = ensure(ctx, ctx->mW2Tb, 2 * 256 * 256)) ||
        (r = ensure(ctx, ctx->mLoss, sizeof(float) * 2)))
        return r;
    return CSGS_OK;
}

csgs_status mlp_rows_buffers(csgs_ctx* ctx, int64_t B) {
    csgs_status r;
    if ((r = ensure(ctx, ctx->mY, sizeof(float) * B)) || (r = ensure(ctx, ctx->mXb, 2 * 64 * (size_t)B)) ||
        (r = ensure(ctx, ctx->mTb, sizeof(float) * B)) || (r = ensure(ctx, ctx->mGd1, sizeof(float) * 256 * (size_t)B)) ||
        (r = ensure(ctx, ctx->mH1, 2 * 256 * (size_t)B)) || (r = ensure(ctx, ctx->mDz2, 2 * 256 * (size_t)B)) ||
        (r = ensure(ctx, ctx->mDz1, 2 * 256 * (size_t)B)) ||
        (r = ensure(ctx, ctx->mPart, sizeof(float) * (size_t)mlp_wgrad_splits(B) * (256 * 256 + 256 * 64))))
        return r;
    return CSGS_OK;
}

MlpBufs mlp_bufs(csgs_ctx* ctx) {
    return mlp_layout(P<float>(ctx->mP), P<__nv_bfloat16>(ctx->mW1b), P<__nv_bfloat16>(ctx->mW2b),
                      P<__nv_bfloat16>(ctx->mW2Tb));
}

MlpTemp mlp_temp(csgs_ctx* ctx) {
    MlpTemp t;
    t.gd1 = P<float>(ctx->mGd1);
    t.h1 = P<__nv_bfloat16>(ctx->mH1);
    t.dz2 = P<__nv_bfloat16>(ctx->mDz2);
    t.dz1 = P<__nv_bfloat16>(ctx->mDz1);
    t.wpart = P<float>(ctx->mPart);
    return t;
}

csgs_status check_err(csgs_ctx* ctx, const char* what) {
    csgs_status r;
    if ((r = launch_check(ctx, what))) return r;
    if ((r = read_counters(ctx))) return r;
    if (ctx->h_ctr->err) return fail(ctx, CSGS_E_TIMEOUT, "%s: tensor-core completion not observed", what);
    return CSGS_OK;
}

}  // namespace

extern "C" {

csgs_status csgs_mlp_init(csgs_ctx* ctx, uint64_t seed) {
    if (!ctx) return CSGS_E_INVAL;
    cudaSetDevice(ctx->device);
    csgs_status r;
    if ((r = mlp_alloc(ctx))) return r;
    std::vector<float> h(kMlpParams, 0.f);
    std::mt19937_64 gen(seed);
    std::uniform_real_distribution<float> u1(-0.125f, 0.125f);    // 1 / sqrt(64)
    std::uniform_real_distribution<float> u2(-0.0625f, 0.0625f);  // 1 / sqrt(256)
    float* p = h.data();
    for (int i = 0; i < 256 * 64; ++i) p[i] = u1(gen);
    p += 256 * 64 + 256;
    for (int i = 0; i < 256 * 256; ++i) p[i] = u2(gen);
    p += 256 * 256 + 256;
    for (int i = 0; i < 256; ++i) p[i] = u2(gen);
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->mP.p, h.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, ctx->st));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->mM.p, 0, sizeof(float) * kMlpParams, ctx->st));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->mV.p, 0, sizeof(float) * kMlpParams, ctx->st));
    mlp_refresh(mlp_bufs(ctx), ctx->st);
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    ctx->mlp_ready = true;
    return launch_check(ctx, "mlp init");
}

csgs_status csgs_mlp_set_params(csgs_ctx* ctx, const float* P_dev) {
    if (!ctx || !P_dev) return CSGS_E_INVAL;
    cudaSetDevice(ctx->device);
    csgs_status r;
    if ((r = mlp_alloc(ctx))) return r;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->mP.p, P_dev, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, ctx->st));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->mM.p, 0, sizeof(float) * kMlpParams, ctx->st));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->mV.p, 0, sizeof(float) * kMlpParams, ctx->st));
    mlp_refresh(mlp_bufs(ctx), ctx->st);
    ctx->mlp_ready = true;
    return launch_check(ctx, "mlp set params");
}

csgs_status csgs_mlp_get_params(csgs_ctx* ctx, float* P_dev) {
    if (!ctx || !P_dev) return CSGS_E_INVAL;
    if (!ctx->mlp_ready) return fail(ctx, CSGS_E_INVAL, "surrogate model not initialised");
    CUDA_TRY(ctx, cudaMemcpyAsync(P_dev, ctx->mP.p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, ctx->st));
    return CSGS_OK;
}

csgs_status csgs_mlp_forward(csgs_ctx* ctx, const void* X_dev, int64_t B, float* y_dev) {
    if (!ctx || !X_dev || !y_dev) return CSGS_E_INVAL;
    if (!ctx->mlp_ready) return fail(ctx, CSGS_E_INVAL, "surrogate model not initialised");
    if (B <= 0 || B >= (1ll << 31)) return fail(ctx, CSGS_E_INVAL, "B out of range");
    cudaSetDevice(ctx->device);
    CUDA_TRY(ctx, cudaMemsetAsync(&ctx->d_ctr->err, 0, sizeof(uint32_t), ctx->st));
    mlp_forward(mlp_bufs(ctx), X_dev, (int)B, y_dev, reinterpret_cast<int*>(&ctx->d_ctr->err), ctx->st);
    return check_err(ctx, "mlp forward");
}

csgs_status csgs_mlp_gradient(csgs_ctx* ctx, const void* X_dev, const float* t_dev, int64_t B, float* G_dev,
                              float* loss_out) {
    if (!ctx || !X_dev || !t_dev || !G_dev) return CSGS_E_INVAL;
    if (!ctx->mlp_ready) return fail(ctx, CSGS_E_INVAL, "surrogate model not initialised");
    if (B <= 0 || B >= (1ll << 26)) return fail(ctx, CSGS_E_INVAL, "B out of range");
    cudaSetDevice(ctx->device);
    csgs_status r;
    if ((r = mlp_rows_buffers(ctx, B))) return r;
    CUDA_TRY(ctx, cudaMemsetAsync(&ctx->d_ctr->err, 0, sizeof(uint32_t), ctx->st));
    mlp_gradient(mlp_bufs(ctx), X_dev, t_dev, (int)B, P<float>(ctx->mY), G_dev, P<float>(ctx->mLoss), mlp_temp(ctx),
                 reinterpret_cast<int*>(&ctx->d_ctr->err), ctx->st);
    if ((r = check_err(ctx, "mlp gradient"))) return r;
    if (loss_out) {
        CUDA_TRY(ctx, cudaMemcpy(loss_out, ctx->mLoss.p, sizeof(float), cudaMemcpyDeviceToHost));
    }
    return CSGS_OK;
}

csgs_status csgs_mlp_train(csgs_ctx* ctx, const void* X_dev, const float* t_dev, int64_t n_rows, int32_t batch,
                           int32_t steps, float lr, uint64_t seed, float* final_loss) {
    if (!ctx || !X_dev || !t_dev) return CSGS_E_INVAL;
    if (!ctx->mlp_ready) return fail(ctx, CSGS_E_INVAL, "surrogate model not initialised");
    if (n_rows <= 0 || batch <= 0 || batch >= (1 << 26) || steps < 0 || !(lr > 0.f))
        return fail(ctx, CSGS_E_INVAL, "bad training arguments");
    cudaSetDevice(ctx->device);
    csgs_status r;
    if ((r = mlp_rows_buffers(ctx, batch))) return r;
    CUDA_TRY(ctx, cudaMemsetAsync(&ctx->d_ctr->err, 0, sizeof(uint32_t), ctx->st));
    const MlpBufs mb = mlp_bufs(ctx);
    const MlpTemp mt = mlp_temp(ctx);
    // the gradient's accumulated entries start at zero; each step's last kernel clears them
    // again, and its batch gather clears the loss
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->mG.p, 0, sizeof(float) * kMlpParams, ctx->st));
    for (int step = 1; step <= steps; ++step) {
        gather_batch(X_dev, t_dev, n_rows, batch, seed, (uint32_t)step, ctx->mXb.p, P<float>(ctx->mTb),
                     P<float>(ctx->mLoss), ctx->st);
        mlp_train_step(mb, ctx->mXb.p, P<float>(ctx->mTb), batch, P<float>(ctx->mY), P<float>(ctx->mG),
                       P<float>(ctx->mLoss), mt, P<float>(ctx->mM), P<float>(ctx->mV), lr, step,
                       reinterpret_cast<int*>(&ctx->d_ctr->err), ctx->st);
        if ((step & 63) == 0 && (r = launch_check(ctx, "mlp train"))) return r;
    }
    if ((r = check_err(ctx, "mlp train"))) return r;
    if (final_loss) {
        CUDA_TRY(ctx, cudaMemcpy(final_loss, ctx->mLoss.p, sizeof(float), cudaMemcpyDeviceToHost));
    }
    return CSGS_OK;
}

csgs_status csgs_view_stats(csgs_ctx* ctx, int32_t scene_id, const csgs_score_opts* opts, float* stats_dev) {
    if (!ctx) return CSGS_E_INVAL;
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (!stats_dev) return fail(ctx, CSGS_E_INVAL, "stats_dev is NULL");
    if (s->cams.empty()) return fail(ctx, CSGS_E_INVAL, "no query views set");
    KOpts ko;
    csgs_status r;
    if ((r = make_kopts(ctx, opts, &ko))) return r;
    cudaSetDevice(ctx->device);
    if ((r = upload_cams(ctx, s, ko))) return r;
    const int nv = (int)s->cams.size();
    for (int v0 = 0; v0 < nv; v0 += 32)
        launch_view_stats(scene_dev(*s), s->d_cams + v0, (nv - v0) < 32 ? (nv - v0) : 32, ko, stats_dev, v0 > 0,
                          ctx->st);
    return launch_check(ctx, "view statistics");
}

csgs_status csgs_features(csgs_ctx* ctx, int32_t scene_id, const float* stats_dev, const float* extra_dev,
                          void* X_dev) {
    if (!ctx) return CSGS_E_INVAL;
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (!stats_dev || !X_dev) return fail(ctx, CSGS_E_INVAL, "null argument");
    cudaSetDevice(ctx->device);
    launch_features(scene_dev(*s), stats_dev, extra_dev, X_dev, ctx->st);
    return launch_check(ctx, "features");
}

csgs_status csgs_log_target(csgs_ctx* ctx, const float* s_dev, int64_t n, float eps, float* t_dev) {
    if (!ctx || !s_dev || !t_dev || n <= 0 || !(eps > 0.f)) return CSGS_E_INVAL;
    cudaSetDevice(ctx->device);
    log_target(s_dev, n, eps, t_dev, ctx->st);
    return launch_check(ctx, "log target");
}

csgs_status csgs_surrogate_combine(csgs_ctx* ctx, const float* y_dev, const float* s_exact_dev, int64_t n, float eps,
                                   int32_t fill_only, float* s_out) {
    if (!ctx || !y_dev || !s_out || n <= 0 || !(eps >= 0.f)) return CSGS_E_INVAL;
    cudaSetDevice(ctx->device);
    surrogate_combine(y_dev, s_exact_dev, n, eps, fill_only, s_out, ctx->st);
    return launch_check(ctx, "surrogate combine");
}

csgs_status csgs_log_ratio_mean(csgs_ctx* ctx, const float* a_dev, const float* b_dev, int64_t n, double* mean_out,
                                int64_t* count_out) {
    if (!ctx) return CSGS_E_INVAL;
    if (!a_dev || !b_dev || n <= 0 || !mean_out) return fail(ctx, CSGS_E_INVAL, "bad arguments");
    cudaSetDevice(ctx->device);
    csgs_status r;
    if ((r = ensure(ctx, ctx->partial, sizeof(double) * 1024))) return r;
    if ((r = ensure(ctx, ctx->Sdev, sizeof(double) * 2))) return r;
    log_ratio_mean(a_dev, b_dev, n, P<double>(ctx->partial), P<double>(ctx->Sdev), ctx->st);
    if ((r = launch_check(ctx, "log ratio mean"))) return r;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_S, ctx->Sdev.p, sizeof(double) * 2, cudaMemcpyDeviceToHost, ctx->st));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->st));
    const double sum = ctx->h_S[0], cnt = ctx->h_S[1];
    *mean_out = cnt > 0.0 ? sum / cnt : 0.0;
    if (count_out) *count_out = (int64_t)cnt;
    return CSGS_OK;
}

csgs_status csgs_log_residual_target(csgs_ctx* ctx, const float* s_dev, const float* p_dev, int64_t n, float eps,
                                     double mu, float* t_dev) {
    if (!ctx || !s_dev || !p_dev || !t_dev || n <= 0 || !(eps > 0.f) || !isfinite(mu)) return CSGS_E_INVAL;
    cudaSetDevice(ctx->device);
    residual_target(s_dev, p_dev, n, eps, (float)mu, t_dev, ctx->st);
    return launch_check(ctx, "residual target");
}

csgs_status csgs_surrogate_combine_prior(csgs_ctx* ctx, const float* y_dev, const float* p_dev,
                                         const float* s_exact_dev, int64_t n, float eps, double mu, int32_t fill_only,
                                         float* s_out) {
    if (!ctx || !y_dev || !p_dev || !s_out || n <= 0 || !(eps > 0.f) || !isfinite(mu)) return CSGS_E_INVAL;
    cudaSetDevice(ctx->device);
    surrogate_combine_prior(y_dev, p_dev, s_exact_dev, n, eps, (float)mu, fill_only, s_out, ctx->st);
    return launch_check(ctx, "surrogate combine (prior)");
}

}  // extern "C"

// ======================================================================= finetune support

extern "C" {

csgs_status csgs_update_scene(csgs_ctx* ctx, int32_t scene_id, const csgs_scene_desc* d) {
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (!d || d->n != s->n || d->sh_degree != s->deg) return fail(ctx, CSGS_E_INVAL, "scene shape mismatch");
    if (!d->means || !d->log_scales || !d->quats || !d->opacity_logits || !d->sh)
        return fail(ctx, CSGS_E_INVAL, "null attribute pointer");
    cudaSetDevice(ctx->device);
    const size_t n = (size_t)s->n, nk = (size_t)(s->deg + 1) * (s->deg + 1);
    const cudaMemcpyKind kind = d->is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUDA_TRY(ctx, cudaMemcpyAsync(s->means, d->means, 3 * n * sizeof(float), kind, ctx->st));
    CUDA_TRY(ctx, cudaMemcpyAsync(s->log_scales, d->log_scales, 3 * n * sizeof(float), kind, ctx->st));
    CUDA_TRY(ctx, cudaMemcpyAsync(s->quats, d->quats, 4 * n * sizeof(float), kind, ctx->st));
    CUDA_TRY(ctx, cudaMemcpyAsync(s->opac, d->opacity_logits, n * sizeof(float), kind, ctx->st));
    CUDA_TRY(ctx, cudaMemcpyAsync(s->sh, d->sh, 3 * nk * n * sizeof(float), kind, ctx->st));
    return CSGS_OK;
}

csgs_status csgs_render_backward(csgs_ctx* ctx, int32_t scene_id, int32_t view, const int32_t* idx_dev,
                                 const float* w_dev, int64_t n_sel, const csgs_score_opts* opts, const float* grad_rgb_dev,
                                 float* g_means_dev, float* g_sh_dev, float* g_logit_dev) {
    if (!ctx) return CSGS_E_INVAL;
    SceneRec* s = get_scene(ctx, scene_id);
    if (!s) return scene_fail(ctx, scene_id);
    if (view < 0 || view >= (int32_t)s->cams.size()) return fail(ctx, CSGS_E_INVAL, "bad view %d", view);
    if (!grad_rgb_dev || !g_means_dev || !g_sh_dev || !g_logit_dev) return fail(ctx, CSGS_E_INVAL, "null argument");
    if ((idx_dev == nullptr) != (w_dev == nullptr)) return fail(ctx, CSGS_E_INVAL, "idx and w must both be given");
    if (idx_dev && (n_sel < 0 || n_sel > s->n)) return fail(ctx, CSGS_E_INVAL, "n_sel out of range");
    KOpts ko;
    csgs_status r;
    if ((r = make_kopts(ctx, opts, &ko))) return r;
    ko.tile_lw = kTileLw16;  // the backward kernel composites 16x16 tiles
    ko.tile_lh = kTileLh16;
    cudaSetDevice(ctx->device);
    if ((r = upload_cams(ctx, s, ko))) return r;
    const int64_t n = s->n;
    const CamDev& cam = s->cams[view];
    const size_t npx = (size_t)cam.W * cam.H;
    if ((r = ensure_view_buffers(ctx, n, 1, tiles_of(cam, ko.tile_lw, ko.tile_lh)))) return r;
    if ((r = ensure(ctx, ctx->bRgb, sizeof(float) * 3 * npx)) || (r = ensure(ctx, ctx->bT, sizeof(float) * npx)) ||
        (r = ensure(ctx, ctx->bLast, sizeof(int) * npx)) || (r = ensure(ctx, ctx->g2d, sizeof(float) * 9 * (size_t)n)))
        return r;
    const float* wts = nullptr;
    if (idx_dev) {
        if ((r = ensure(ctx, ctx->wfull, sizeof(float) * (size_t)n))) return r;
        wts = P<float>(ctx->wfull);
    }
    cudaStream_t st = ctx->st;
    set_u64(ctx->d_nconst, (unsigned long long)n, st);
    const SceneDev sd = scene_dev(*s);
    int retries = 0;
    for (;;) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(DevCounters), st));
        if (idx_dev) {
            CUDA_TRY(ctx, cudaMemsetAsync(ctx->wfull.p, 0, sizeof(float) * (size_t)n, st));
            scatter_weights(idx_dev, w_dev, n_sel, P<float>(ctx->wfull), n, ctx->d_ctr, st);
        }
        launch_project(sd, s->d_cams + view, 1, wts, ko, P<Splat>(ctx->splats[0]), P<uint32_t>(ctx->keys[0]),
                       P<uint2>(ctx->rects[0]), ctx->d_ctr, st);
        const uint32_t* iv = bin_batch(ctx, 0, n, 1, P<uint32_t>(ctx->keys[0]), P<uint2>(ctx->rects[0]), &cam,
                                       s->d_cams + view, ko, ctx->sort_blocks, st);
        CompositeArgs a{};
        a.ranges = P<uint2>(ctx->slot[0].ranges);
        a.inst_gid = iv;
        a.splats = P<Splat>(ctx->splats[0]);
        a.n_gauss = (int)n;
        a.cam = cam;
        a.o = ko;
        a.rgb = P<float>(ctx->bRgb);
        a.T = P<float>(ctx->bT);
        a.last = P<int>(ctx->bLast);
        a.ctr = ctx->d_ctr;
        launch_composite_render(a, st);
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->g2d.p, 0, sizeof(float) * 9 * (size_t)n, st));
        a.grad_rgb = grad_rgb_dev;
        a.g2d = P<float>(ctx->g2d);
        launch_composite_backward(a, st);
        if ((r = launch_check(ctx, "render backward kernels"))) return r;
        if ((r = read_counters(ctx))) return r;
        if (ctx->h_ctr->err & (kErrCapacity | kErrDepthRange)) {
            if (++retries > 3) return fail(ctx, CSGS_E_DEVICE_CHECK, "instance capacity overflow persists");
            if ((r = widen_or_grow(ctx, ko))) return r;
            continue;
        }
        break;
    }
    if (ctx->h_ctr->err & kErrIndex) return fail(ctx, CSGS_E_INVAL, "coreset index out of range");
    launch_project_backward(sd, s->d_cams + view, wts, ko, P<float>(ctx->g2d), g_means_dev, g_sh_dev, g_logit_dev, st);
    return launch_check(ctx, "projection backward");
}

csgs_status csgs_adam_update(csgs_ctx* ctx, float* p_dev, const float* g_dev, float* m_dev, float* v_dev, int64_t n,
                             float lr, float beta1, float beta2, float eps, int32_t step) {
    if (!ctx || !p_dev || !g_dev || !m_dev || !v_dev || n <= 0 || step < 1) return CSGS_E_INVAL;
    cudaSetDevice(ctx->device);
    adam_update(p_dev, g_dev, m_dev, v_dev, n, lr, beta1, beta2, eps, step, ctx->st);
    return launch_check(ctx, "adam");
}

}  // extern "C"

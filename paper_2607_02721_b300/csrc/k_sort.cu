// Binning of projected Gaussians into screen tiles in front-to-back order (the order
// "induced by the view depths", Sec. 3 "Scalar rendering function"), for a batch of
// views at once:
//   1. stable LSD radix sort of all Gaussians of every view by depth (ties keep index
//      order); one segment per view, all segments in the same launches;
//   2. one fused scan + emit pass over the batch that writes (view, tile, gid) instances,
//      view by view, each view in depth order;
//   3. stable LSD radix sort of the batch's instances by the key (view, tile id);
//   4. per-(view, tile) [start, end) ranges.
// Every tile list is therefore sorted by (depth, Gaussian index).  Sorting a whole view
// batch per launch keeps each pass a bandwidth-bound sweep over tens of millions of keys
// instead of a latency-bound one over a single view's.  No CUB: the sort is a
// reduce-then-scan radix sort with 8- or 9-bit digits and warp-level stable ranking (one
// ballot per digit bit).
#include <type_traits>

#include "csgs_internal.cuh"

namespace csgs {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortGroups = 8;                               // 32-key groups per warp per sub-tile
constexpr int kSubTile = kSortThreads * kSortGroups;          // 2048 keys
constexpr int kScanThreads = 256;
constexpr int kEmitBlocks = 148 * 4;  // grid bound of the emit kernels (chunks of kScanThreads Gaussians)

// chunk of the key array handled by block b of a grid of G blocks (multiples of sub-tiles)
__device__ __forceinline__ void sort_chunk(uint32_t n, int b, uint32_t& begin, uint32_t& end) {
    const uint32_t G = gridDim.x;
    uint32_t per = (n + G - 1) / G;
    per = (per + kSubTile - 1) / kSubTile * kSubTile;
    if (per < kSubTile) per = kSubTile;
    uint64_t bg = (uint64_t)per * b;
    begin = bg < n ? (uint32_t)bg : n;
    uint64_t en = bg + per;
    end = en < n ? (uint32_t)en : n;
}

__device__ __forceinline__ uint32_t read_n(const unsigned long long* d_n, uint32_t n_max) {
    unsigned long long v = *d_n;
    return v < n_max ? (uint32_t)v : n_max;
}

// Per-block digit counts of one pass (RB-bit digits, D = 2^RB).  Each warp counts into
// its own shared histogram with plain atomics (match.any costs grow with the number of
// distinct digits in the warp; conflicting shared atomics only serialise on equal digits).
// Segment blockIdx.y: keys + seg * seg_stride, histogram block hist + seg * hstride.
template <int RB>
__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t* __restrict__ keys,
                                                          const unsigned long long* d_n, uint32_t n_max, int shift,
                                                          uint32_t* __restrict__ hist, size_t seg_stride,
                                                          size_t hstride) {
    constexpr uint32_t D = 1u << RB;
    keys += blockIdx.y * seg_stride;
    hist += blockIdx.y * hstride;
    constexpr int DPT = (int)D / kSortThreads;  // digits per thread
    __shared__ uint32_t wh[kSortWarps][D];
    for (int k = threadIdx.x; k < kSortWarps * (int)D; k += kSortThreads) (&wh[0][0])[k] = 0u;
    __syncthreads();
    const uint32_t n = read_n(d_n, n_max);
    uint32_t begin, end;
    sort_chunk(n, blockIdx.x, begin, end);
    uint32_t* h = wh[threadIdx.x >> 5];
    // a chunk is a whole number of 2048-key sub-tiles: 8 coalesced loads in flight per thread
    for (uint32_t base = begin; base < end; base += kSubTile) {
        uint32_t d[kSortGroups];
        if (base + kSubTile <= end) {  // a full sub-tile: no bounds tests
#pragma unroll
            for (int g = 0; g < kSortGroups; ++g)
                d[g] = (__ldg(keys + base + g * kSortThreads + threadIdx.x) >> shift) & (D - 1u);
#pragma unroll
            for (int g = 0; g < kSortGroups; ++g) atomicAdd(h + d[g], 1u);
        } else {
#pragma unroll
            for (int g = 0; g < kSortGroups; ++g) {
                const uint32_t i = base + g * kSortThreads + threadIdx.x;
                d[g] = i < end ? (__ldg(keys + i) >> shift) & (D - 1u) : D;
            }
#pragma unroll
            for (int g = 0; g < kSortGroups; ++g)
                if (d[g] < D) atomicAdd(h + d[g], 1u);
        }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < DPT; ++e) {
        const int dg = threadIdx.x * DPT + e;
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) c += wh[w][dg];
        hist[dg * gridDim.x + blockIdx.x] = c;
    }
}

// Exclusive scan of each digit's row of the histogram (G per-block counts, G <=
// kSortMaxBlocks), one CTA per (digit, segment); the row totals of segment y go to
// hist + y * hstride + D * G.
__global__ void __launch_bounds__(256) k_rs_rowscan(uint32_t* __restrict__ hist, int G, int D, size_t hstride) {
    constexpr int kPer = (kSortMaxBlocks + 255) / 256;
    __shared__ uint32_t ws[8];
    hist += blockIdx.y * hstride;
    uint32_t* row_total = hist + (size_t)D * G;
    const int per = (G + 255) / 256;
    uint32_t* row = hist + (size_t)blockIdx.x * G;
    const int b0 = threadIdx.x * per;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = (k < per && b0 + k < G) ? row[b0 + k] : 0u;
        sum += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    uint32_t pre = x - sum;
    for (int w = 0; w < warp; ++w) pre += ws[w];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (k < per && b0 + k < G) row[b0 + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 255) row_total[blockIdx.x] = pre;
}

// Stable scatter of one radix pass (NBITS significant bits of an RB-bit digit, D = 2^RB
// digits, DPT = D / 256 consecutive digits per thread).  Each CTA walks its chunk in
// sub-tiles of 2048 keys: warps rank their keys per digit with one ballot per digit bit
// (stable: warp, group, lane order), the CTA turns the per-warp counts into positions,
// places the sub-tile in shared memory grouped by digit, and writes each digit's run to
// its global slot, so global stores are contiguous runs.
// Segment blockIdx.y: every key and value array + seg * seg_stride (positions are
// within the segment), histogram block hist + seg * hstride.  Four CTAs per SM (at most 64
// registers): at 74 registers and three CTAs the 9-bit passes took 45 us against 37 us.
template <int NBITS, int RB>
__global__ void __launch_bounds__(kSortThreads, 4) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                             const uint32_t* __restrict__ vin,
                                                             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                             const unsigned long long* d_n, uint32_t n_max, int shift,
                                                             const uint32_t* __restrict__ hist, size_t seg_stride,
                                                             size_t hstride) {
    constexpr uint32_t D = 1u << RB;
    constexpr int DPT = (int)D / kSortThreads;
    {
        const size_t so = blockIdx.y * seg_stride;
        kin += so;
        if (vin) vin += so;
        kout += so;
        vout += so;
        hist += blockIdx.y * hstride;
    }
    const uint32_t* __restrict__ row_total = hist + (size_t)D * gridDim.x;
    __shared__ __align__(16) uint32_t wcnt[kSortWarps][D + 1];  // (D + 1) kSortWarps is a multiple of 4
    __shared__ uint32_t gbase[D];
    __shared__ uint32_t lstart[D];
    __shared__ uint32_t skey[kSubTile];
    __shared__ uint32_t sval[kSubTile];
    __shared__ uint32_t ws[kSortWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    {
        // offset of digit d = sum of the totals of the smaller digits
        uint32_t t[DPT], sum = 0;
#pragma unroll
        for (int e = 0; e < DPT; ++e) {
            t[e] = row_total[tid * DPT + e];
            sum += t[e];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        uint32_t pre = x - sum;
        for (int w = 0; w < warp; ++w) pre += ws[w];
#pragma unroll
        for (int e = 0; e < DPT; ++e) {
            const int dg = tid * DPT + e;
            gbase[dg] = pre + hist[dg * gridDim.x + blockIdx.x];
            pre += t[e];
        }
    }
    for (int k = tid; k < kSortWarps * (int)(D + 1) / 4; k += kSortThreads)
        reinterpret_cast<uint4*>(&wcnt[0][0])[k] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const uint32_t n = read_n(d_n, n_max);
    uint32_t begin, end;
    sort_chunk(n, blockIdx.x, begin, end);
    for (uint32_t sub = begin; sub < end; sub += kSubTile) {
        const uint32_t nvalid = min((uint32_t)kSubTile, end - sub);
        uint32_t key[kSortGroups], val[kSortGroups], dig[kSortGroups], rank[kSortGroups];
        // loads and ranks of the sub-tile; FULL: every key of the sub-tile exists (all but a
        // chunk's last sub-tile), so no lane needs the bounds test or the invalid class
        auto load_rank = [&](auto full) {
            constexpr bool FULL = decltype(full)::value;
#pragma unroll
            for (int g = 0; g < kSortGroups; ++g) {
                const uint32_t i = sub + warp * (32 * kSortGroups) + g * 32 + lane;
                const bool ok = FULL || i < end;
                key[g] = ok ? __ldg(kin + i) : 0u;
                val[g] = ok ? (vin ? __ldg(vin + i) : i) : 0u;
                dig[g] = ok ? (key[g] >> shift) & (D - 1u) : D;
            }
            // lanes holding the same digit: one ballot per digit bit (NBITS, unrolled;
            // match.any is slower when the digits are spread out); invalid lanes (digit D)
            // form their own class.  The per-warp digit counters then give stable ranks in
            // (group, lane) order.
#pragma unroll
            for (int g = 0; g < kSortGroups; ++g) {
                const uint32_t d = dig[g];
                uint32_t pm = 0xffffffffu;
                if (!FULL) {
                    pm = __ballot_sync(0xffffffffu, d < D);
                    if (d >= D) pm = ~pm;
                }
#pragma unroll
                for (int bb = 0; bb < NBITS; ++bb) {
                    const uint32_t bal = __ballot_sync(0xffffffffu, (d >> bb) & 1u);
                    pm &= ((d >> bb) & 1u) ? bal : ~bal;
                }
                rank[g] = wcnt[warp][d] + __popc(pm & lt);
                __syncwarp();
                if (lane == __ffs(pm) - 1) wcnt[warp][d] += __popc(pm);
                __syncwarp();
            }
        };
        if (nvalid == (uint32_t)kSubTile)
            load_rank(std::true_type{});
        else
            load_rank(std::false_type{});
        __syncthreads();
        // this thread's digits: per-warp exclusive offsets within the digit, and its count
        uint32_t cnt_d[DPT], csum = 0;
#pragma unroll
        for (int e = 0; e < DPT; ++e) {
            const int dg = tid * DPT + e;
            cnt_d[e] = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = wcnt[w][dg];
                wcnt[w][dg] = cnt_d[e];
                cnt_d[e] += c;
            }
            csum += cnt_d[e];
        }
        // start of each digit's run inside the sub-tile
        {
            uint32_t x = csum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            __syncthreads();  // ws reuse
            if (lane == 31) ws[warp] = x;
            __syncthreads();
            uint32_t pre = x - csum;
            for (int w = 0; w < warp; ++w) pre += ws[w];
#pragma unroll
            for (int e = 0; e < DPT; ++e) {
                lstart[tid * DPT + e] = pre;
                pre += cnt_d[e];
            }
        }
        __syncthreads();
#pragma unroll
        for (int g = 0; g < kSortGroups; ++g) {
            if (dig[g] < D) {
                const uint32_t lp = lstart[dig[g]] + wcnt[warp][dig[g]] + rank[g];
                skey[lp] = key[g];
                sval[lp] = val[g];
            }
        }
        __syncthreads();
        for (uint32_t q = tid; q < nvalid; q += kSortThreads) {
            const uint32_t k = skey[q];
            const uint32_t d = (k >> shift) & (D - 1u);
            const uint32_t pos = gbase[d] + (q - lstart[d]);
            kout[pos] = k;
            vout[pos] = sval[q];
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < DPT; ++e) gbase[tid * DPT + e] += cnt_d[e];
        for (int k = tid; k < kSortWarps * (int)(D + 1) / 4; k += kSortThreads)
            reinterpret_cast<uint4*>(&wcnt[0][0])[k] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
    }
}

__device__ __forceinline__ uint32_t tile_count(uint2 r) {
    uint32_t x0 = r.x & 0xFFFFu, y0 = r.x >> 16, x1 = r.y & 0xFFFFu, y1 = r.y >> 16;
    return (x1 - x0) * (y1 - y0);
}

// block-wide exclusive scan of one value per thread; returns the prefix, *total the sum
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t pre = x - v + (warp > 0 ? warp_sums[warp - 1] : 0u);
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return pre;
}

// Emit, phase 1: instance count per chunk of 256 depth-ordered Gaussians of one view
// of the batch (chunk c: view c / nb, chunk c % nb of that view; nb chunks per view).
// The emit kernels loop over chunks on a grid of at most kEmitBlocks CTAs.
__global__ void __launch_bounds__(kScanThreads) k_emit_reduce(const uint32_t* __restrict__ order,
                                                              const uint2* __restrict__ rects, int n, int nv,
                                                              uint32_t* __restrict__ partial) {
    __shared__ uint32_t ws[32];
    const int nb = (n + kScanThreads - 1) / kScanThreads;
    for (int c = blockIdx.x; c < nb * nv; c += gridDim.x) {
        const int v = nv == 1 ? 0 : c / nb, cb = c - v * nb;
        const size_t vo = (size_t)v * n;
        const int j = cb * kScanThreads + threadIdx.x;
        const uint32_t c_ = j < n ? tile_count(__ldg(rects + vo + __ldg(order + vo + j))) : 0u;
        // the chunk's total: warp sums, then the CTA's
        const uint32_t wsum = __reduce_add_sync(0xffffffffu, c_);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = wsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0u;
#pragma unroll
            for (int w = 0; w < kScanThreads / 32; ++w) tot += ws[w];
            partial[c] = tot;
        }
        __syncthreads();  // ws is rewritten by the next chunk
    }
}

// Exclusive scan of the per-block totals in one CTA (any count), plus the grand total.
__global__ void __launch_bounds__(1024) k_scan_top_u32(uint32_t* __restrict__ partial, int nb, DevCounters* ctr,
                                                       unsigned long long* n_inst) {
    __shared__ uint32_t ws[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    // four consecutive entries per thread per round
    for (int b0 = 0; b0 < nb; b0 += 4096) {
        const int i0 = b0 + 4 * threadIdx.x;
        uint32_t v[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = i0 + k < nb ? partial[i0 + k] : 0u;
            sum += v[k];
        }
        uint32_t tot;
        uint32_t pre = block_exclusive_scan(sum, ws, &tot);
        const unsigned long long c = carry;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < nb) partial[i0 + k] = (uint32_t)(c + pre);
            pre += v[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && ctr) {
        // the other binning slot may update the totals concurrently
        unsigned long long t = carry;
        *n_inst = t;
        atomicAdd(&ctr->inst_total, t);
        atomicMax(&ctr->max_inst, t);
    }
}

// Emit, phase 3: every warp expands its 32 Gaussians' tile rectangles into a
// contiguous run of instances, lane l of each round of 32 writing instance f0 + l
// (coalesced), in depth order and row-major tile order within a Gaussian.  The owner of
// an instance is the last non-empty Gaussian run starting at or before it: from the bits
// of the run starts inside the round's window (one OR reduction) and the count of runs
// started before it (one ballot).  The key is
// (view << tbits) | tile id, the value the Gaussian id.
__global__ void __launch_bounds__(kScanThreads) k_emit_down(const uint32_t* __restrict__ order,
                                                            const uint2* __restrict__ rects, int n, int nv,
                                                            const CamDev* __restrict__ cams, int tbits, int lw,
                                                            const uint32_t* __restrict__ partial,
                                                            uint32_t* __restrict__ ikeys, uint32_t* __restrict__ ivals,
                                                            uint32_t cap, DevCounters* ctr) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t s_e[kScanThreads / 32][32];
    __shared__ uint32_t s_g[kScanThreads / 32][32];
    __shared__ uint2 s_r[kScanThreads / 32][32];
    __shared__ float s_iw[kScanThreads / 32][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = (n + kScanThreads - 1) / kScanThreads;
    for (int c = blockIdx.x; c < nb * nv; c += gridDim.x) {
        const int v = nv == 1 ? 0 : c / nb, cb = c - v * nb;
        const size_t vo = (size_t)v * n;
        const uint32_t tiles_x = (uint32_t)tiles_x_of(cams[v], lw);
        const uint32_t vkey = (uint32_t)v << tbits;
        const int j = cb * kScanThreads + threadIdx.x;
        const uint32_t gid = j < n ? __ldg(order + vo + j) : 0u;
        const uint2 rc = j < n ? __ldg(rects + vo + gid) : make_uint2(0u, 0u);
        const uint32_t cnt = tile_count(rc);
        uint32_t tot;
        const uint32_t off = block_exclusive_scan(cnt, ws, &tot) + partial[c];
        const uint32_t wbase = __shfl_sync(0xffffffffu, off, 0);
        const uint32_t wtot = __shfl_sync(0xffffffffu, off + cnt, 31) - wbase;
        const uint32_t e = off - wbase;  // this lane's run start within the warp's instances
        // the non-empty runs, compacted in lane order (their starts strictly increase)
        const uint32_t nz = __ballot_sync(0xffffffffu, cnt > 0u);
        if (cnt > 0u) {
            const int ci = __popc(nz & ((1u << lane) - 1u));
            s_e[warp][ci] = e;
            s_g[warp][ci] = gid;
            s_r[warp][ci] = rc;
            s_iw[warp][ci] = __frcp_rn((float)((rc.y & 0xFFFFu) - (rc.x & 0xFFFFu)));
        }
        __syncwarp();
        const bool fits = (unsigned long long)wbase + wtot <= cap;
        if (!fits && lane == 0 && wtot) atomicOr(&ctr->err, kErrCapacity);
        for (uint32_t f0 = 0; fits && f0 < wtot; f0 += 32) {
            // run starts inside the window [f0, f0 + 32) as bits, and the runs started before
            // it: position f0 + l belongs to the last run starting at or before it
            const uint32_t bit = (cnt > 0u && e >= f0 && e < f0 + 32u) ? 1u << (e - f0) : 0u;
            const uint32_t m = __reduce_or_sync(0xffffffffu, bit);
            const int before = __popc(__ballot_sync(0xffffffffu, cnt > 0u && e < f0));
            const uint32_t f = f0 + lane;
            if (f >= wtot) continue;  // only in the last window: the loop ends for every lane
            const int lo = before + __popc(m & ((2u << lane) - 1u)) - 1;
            const uint2 r = s_r[warp][lo];
            const uint32_t local = f - s_e[warp][lo];
            const uint32_t x0 = r.x & 0xFFFFu, y0 = r.x >> 16, x1 = r.y & 0xFFFFu;
            const uint32_t w = x1 - x0;
            // local / w in FP32: (local + 0.5) / w lies at least 0.5 / w from an integer and the
            // product with the rounded reciprocal is within (local + 0.5) 2^-23 / w of it, so
            // the floor is exact for local < 2^22 (integer division beyond)
            const uint32_t dy = local < (1u << 22) ? (uint32_t)(((float)local + 0.5f) * s_iw[warp][lo]) : local / w;
            const uint32_t tx = x0 + (local - dy * w), ty = y0 + dy;
            ikeys[wbase + f] = vkey | (ty * tiles_x + tx);
            ivals[wbase + f] = s_g[warp][lo];
        }
    }
}

// Tile ranges from the (view, tile)-sorted instance keys, one row of max_tiles ranges per
// view (blockIdx.y): thread t finds the first instance with key >= (view << tbits) + t by
// binary search and writes it as the start of tile t and the end of tile t - 1 (thread
// n_tiles of the view closes its last tile: no instance has that key), so every range of
// the view is written.
__global__ void k_ranges(const uint32_t* __restrict__ keys, const unsigned long long* d_n, uint32_t n_max,
                         uint2* __restrict__ ranges, const CamDev* __restrict__ cams, int tbits, int lw, int lh,
                         int max_tiles) {
    const int v = blockIdx.y;
    const uint32_t n_tiles = (uint32_t)tiles_of(cams[v], lw, lh);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > n_tiles) return;
    const uint32_t key = ((uint32_t)v << tbits) + t;
    const uint32_t n = read_n(d_n, n_max);
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(keys + mid) < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    uint2* rv = ranges + (size_t)v * max_tiles;
    if (t < n_tiles) rv[t].x = lo;
    if (t > 0) rv[t - 1].y = lo;
}

// Tiles by descending list length (classes floor(log2 n) + 1, the longest class first), so
// that the compositing launch starts its longest tiles in its first wave instead of its
// last.  One CTA: class counts, class offsets, then each tile at its class's next slot;
// the lanes of a warp with the same class share one shared-memory atomic.
__global__ void __launch_bounds__(1024) k_tile_order(const uint2* __restrict__ ranges, int T,
                                                     uint32_t* __restrict__ order, uint32_t* __restrict__ work) {
    __shared__ uint32_t cnt[34];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 34) cnt[tid] = 0u;
    if (tid == 0 && work) *work = 0u;
    __syncthreads();
    for (int t0 = 0; t0 < T; t0 += 1024) {
        const int t = t0 + tid;
        const int c = t < T ? 32 - __clz(ranges[t].y - ranges[t].x) : 33;
        const uint32_t peers = __match_any_sync(0xffffffffu, c);
        if (lane == __ffs(peers) - 1) atomicAdd(&cnt[c], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t s = 0;
        for (int c = 32; c >= 0; --c) {
            const uint32_t k = cnt[c];
            cnt[c] = s;
            s += k;
        }
    }
    __syncthreads();
    for (int t0 = 0; t0 < T; t0 += 1024) {
        const int t = t0 + tid;
        const int c = t < T ? 32 - __clz(ranges[t].y - ranges[t].x) : 33;
        const uint32_t peers = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && c < 33) base = atomicAdd(&cnt[c], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (c < 33) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
    }
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

// One pass with RB-bit digits (NBITS of them significant).
template <int RB>
void radix_pass(int nbits, const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                const unsigned long long* d_n, uint32_t n_max, int shift, uint32_t* hist, int G, int S,
                size_t seg_stride, cudaStream_t st) {
    constexpr int D = 1 << RB;
    const size_t hs = sort_hist_stride(G);
    k_rs_hist<RB><<<dim3(G, S), kSortThreads, 0, st>>>(kin, d_n, n_max, shift, hist, seg_stride, hs);
    count_launches(1);
    k_rs_rowscan<<<dim3(D, S), 256, 0, st>>>(hist, G, D, hs);
    count_launches(1);
#define CSGS_SCATTER(NB) \
    k_rs_scatter<NB, RB><<<dim3(G, S), kSortThreads, 0, st>>>(kin, vin, kout, vout, d_n, n_max, shift, hist, \
                                                              seg_stride, hs)
    switch (nbits) {
        case 1: CSGS_SCATTER(1); break;
        case 2: CSGS_SCATTER(2); break;
        case 3: CSGS_SCATTER(3); break;
        case 4: CSGS_SCATTER(4); break;
        case 5: CSGS_SCATTER(5); break;
        case 6: CSGS_SCATTER(6); break;
        case 7: CSGS_SCATTER(7); break;
        case 8: CSGS_SCATTER(8); break;
        default: CSGS_SCATTER(RB); break;
    }
#undef CSGS_SCATTER
    count_launches(1);
}

}  // namespace

int radix_sort_pairs(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, const unsigned long long* d_n,
                     uint32_t n_max, int bits, int digit_bits, uint32_t* hist, int G, bool iota_vals, int S,
                     size_t seg_stride, cudaStream_t st) {
    if (G < 1) G = 1;
    if (G > kSortMaxBlocks) G = kSortMaxBlocks;
    if (S < 1) S = 1;
    const int rb = digit_bits == 9 ? 9 : 8;
    int cur = 0;
    for (int shift = 0; shift < bits; shift += rb) {
        uint32_t* kin = cur ? kb : ka;
        uint32_t* vin = shift == 0 && iota_vals ? nullptr : (cur ? vb : va);
        uint32_t* kout = cur ? ka : kb;
        uint32_t* vout = cur ? va : vb;
        const int nbits = bits - shift < rb ? bits - shift : rb;
        if (rb == 9)
            radix_pass<9>(nbits, kin, vin, kout, vout, d_n, n_max, shift, hist, G, S, seg_stride, st);
        else
            radix_pass<8>(nbits, kin, vin, kout, vout, d_n, n_max, shift, hist, G, S, seg_stride, st);
        cur ^= 1;
    }
    return cur;
}

void emit_instances(const uint32_t* order, const uint2* rects, int n, int nv, const CamDev* cams, int tbits, int lw,
                    uint32_t* ikeys, uint32_t* ivals, uint32_t cap, uint32_t* scan_tmp, DevCounters* ctr,
                    unsigned long long* n_inst, cudaStream_t st) {
    const int nb = (n + kScanThreads - 1) / kScanThreads;
    const int nc = nb * nv;
    const int ng = nc < kEmitBlocks ? nc : kEmitBlocks;
    k_emit_reduce<<<ng, kScanThreads, 0, st>>>(order, rects, n, nv, scan_tmp);
    count_launches(1);
    k_scan_top_u32<<<1, 1024, 0, st>>>(scan_tmp, nc, ctr, n_inst);
    count_launches(1);
    k_emit_down<<<ng, kScanThreads, 0, st>>>(order, rects, n, nv, cams, tbits, lw, scan_tmp, ikeys, ivals, cap, ctr);
    count_launches(1);
}

void tile_ranges(const uint32_t* keys, const unsigned long long* d_n, uint32_t n_max, uint2* ranges, int nv,
                 const CamDev* cams, int tbits, int lw, int lh, int max_tiles, cudaStream_t st) {
    k_ranges<<<dim3((max_tiles + 1 + 255) / 256, nv), 256, 0, st>>>(keys, d_n, n_max, ranges, cams, tbits, lw, lh,
                                                                    max_tiles);
    count_launches(1);
}

void tile_order(const uint2* ranges, int T, uint32_t* order, uint32_t* work, cudaStream_t st) {
    k_tile_order<<<1, 1024, 0, st>>>(ranges, T, order, work);
    count_launches(1);
}

void set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st) {
    k_set_u64<<<1, 1, 0, st>>>(p, v);
    count_launches(1);
}

}  // namespace csgs

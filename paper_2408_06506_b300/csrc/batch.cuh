// Batched tactile step over uneven pads, SDF grids and images in one pair of launches
// (the paper's parallel environments, Sec. III and IV-A of arXiv 2408.06506, with every
// pad free to carry its own taxel layout, object and camera model).
//
// Force field: one warp per pad, as in the uniform kernel, but the pads come from a
// schedule in the workspace (grouped by object, largest first within an object) with their
// own taxel count, layout, object and output offset.  Pads are dealt either round-robin or from a counter that each warp
// bumps when it takes a pad (the next ticket is fetched while the current pad runs); the
// last warp out returns the counter to zero, so consecutive launches - and graph replays
// - need no reset in between.
//
// Image: the uniform kernel's producer / compute-warp pipeline with work items over
// (sensor model, block of M images of that model, tile), dealt from a counter.  Each
// model brings its own size, pixel pitch and coefficients; its images are listed
// contiguously in the workspace with their first pixel in the packed depth_map / rgb
// arrays, so an item's images need no filtering on the GPU.
#pragma once

#include "common.cuh"
#include "shade.cuh"
#include "taxel.cuh"

namespace tacsl {

constexpr int kMaxModels = 64;

// One pad as the force kernel schedules it (32 bytes; the workspace holds n_pad of them).
struct BatchPad {
    int32_t pad;      // row of pose / twist / wrench (and of the contact parameters)
    int32_t T;        // taxels of its layout
    int32_t obj;      // SDF of its object
    int32_t unused;
    int64_t first;    // first point of its layout in the taxel pool
    int64_t out;      // first taxel slot of the pad in depth / f_n / f_t
};
static_assert(sizeof(BatchPad) == 32, "BatchPad is 32 bytes");

struct BatchForceArgs {
    SdfTable tab;
    Params4 prm;
    const BatchPad* sched;
    int n_pad;
    const float* taxels;
    const float* pose;
    const float* twist;
    float* depth;
    float* f_n;
    float* f_t;
    float* wrench;
    unsigned int* ticket;   // [0]: next schedule slot, [1]: warps finished; both 0 between launches
};

template <int NP>
__device__ __forceinline__ void batch_pad(const BatchForceArgs& A, int slot) {
    const BatchPad* d = A.sched + slot;
    const int4 h = __ldg(reinterpret_cast<const int4*>(d));
    const longlong2 o = __ldg(reinterpret_cast<const longlong2*>(d) + 1);
    const int64_t b = h.x;
    pad_taxels_by_warp<NP>(A.tab, A.prm, A.prm.count == 1 ? 0 : h.x, h.z, h.y, A.taxels + o.x * 3, A.pose + b * 7,
                           A.twist + b * 6, A.depth + o.y, A.f_n + o.y * 3, A.f_t + o.y * 3,
                           A.wrench != nullptr ? A.wrench + b * 6 : nullptr);
}

template <int NP, bool DYNAMIC>
__global__ void __launch_bounds__(256) batch_force_kernel(const BatchForceArgs A) {
    const int lane = threadIdx.x & 31;
    const unsigned n_warps = gridDim.x * (blockDim.x >> 5);
    if (DYNAMIC) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        while (t < static_cast<unsigned>(A.n_pad)) {
            unsigned tn = 0;
            if (lane == 0) tn = atomicAdd(A.ticket, 1u);   // in flight while pad t runs
            batch_pad<NP>(A, static_cast<int>(t));
            t = __shfl_sync(0xffffffffu, tn, 0);
        }
        // every ticket of this warp has been drawn; the last warp out resets both counters
        if (lane == 0) {
            __threadfence();
            if (atomicAdd(A.ticket + 1, 1u) == n_warps - 1) {
                atomicExch(A.ticket, 0u);
                atomicExch(A.ticket + 1, 0u);
            }
        }
    } else {
        const unsigned w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        for (unsigned s = w; s < static_cast<unsigned>(A.n_pad); s += n_warps) batch_pad<NP>(A, static_cast<int>(s));
    }
}

// ---------------------------------------------------------------------------
// Image kernel over several sensor models
// ---------------------------------------------------------------------------

struct BatchModel {
    const float* coeffs;     // [6][3][HW], 16-byte aligned
    int H, W, HW, n_tiles;
    float cx_c, cx_e, cy_c, cy_e;   // 1/(2 pitch_x), 1/pitch_x, 1/(2 pitch_y), 1/pitch_y
    int img_begin, img_end;  // the model's images in the image list
    int item_begin;          // its first work item
    int unused;
};

struct BatchShadeArgs {
    BatchModel mdl[kMaxModels];
    const int64_t* img_px;   // image list: first pixel of each image in depth / rgb
    const float* depth;      // packed depth maps, 16-byte aligned
    uint8_t* rgb;            // packed RGB, 16-byte aligned
    unsigned int* ticket;    // [0]: next work item, [1]: CTAs finished; both 0 between launches
    int n_model, M, n_items, n_stages, stage_floats;
};

struct BatchItem {
    int m, blk, tile;
};

// Work item k -> (model, image block, tile); tile fastest within a model.
__device__ __forceinline__ BatchItem batch_item(const BatchShadeArgs& A, int k) {
    int m = 0;
    while (m + 1 < A.n_model && A.mdl[m + 1].item_begin <= k) ++m;
    BatchItem it;
    it.m = m;
    const int local = k - A.mdl[m].item_begin;
    it.blk = local / A.mdl[m].n_tiles;
    it.tile = local - it.blk * A.mdl[m].n_tiles;
    return it;
}

__device__ __forceinline__ void batch_load_coefficients(const BatchShadeArgs& A, int k, float* coef, uint64_t* cfull,
                                                        uint64_t pol) {
    const BatchItem it = batch_item(A, k);
    const int HW = A.mdl[it.m].HW;
    const int tile_start = it.tile * kShTile;
    const uint32_t row_bytes = static_cast<uint32_t>(min(kShTile, HW - tile_start)) * 4u;
    mbar_arrive_expect_tx(smem_u32(cfull), 18u * row_bytes);
    const float* src = A.mdl[it.m].coeffs + tile_start;
    for (int r = 0; r < 18; ++r)
        bulk_g2s(smem_u32(coef + r * kShTile), src + static_cast<int64_t>(r) * HW, row_bytes, smem_u32(cfull), pol);
}

// Producer warp: as in the uniform kernel (each image's tile plus halo rows into the
// stage ring; the next item's coefficients staged while the current item's images are
// still being issued), but items are dealt from a counter: a CTA draws its next item when
// its current one has about a ring's worth of images left to issue.  So consecutive items
// - neighbouring tiles of the same images - start within microseconds of each other on
// whichever CTAs are free, and the rows one tile reads as its halo are still in L2 when
// its neighbour reads them as its own (with a fixed round-robin, items of different
// models take different times and the CTAs drift apart).  The last producer out resets
// the counters.
__device__ __forceinline__ void batch_shade_producer(const BatchShadeArgs& A, unsigned char* smem) {
    const int lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOffFull);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + kOffEmpty);
    uint64_t* cfull = reinterpret_cast<uint64_t*>(smem + kOffCoefFull);
    uint64_t* cempty = reinterpret_cast<uint64_t*>(smem + kOffCoefEmpty);
    int2* meta = reinterpret_cast<int2*>(smem + kOffMeta);
    float* coef = reinterpret_cast<float*>(smem + kOffCoef);
    float* stages = reinterpret_cast<float*>(smem + kOffStage);
    const int NS = A.n_stages;
    const uint64_t pol_keep = policy_evict_last();
    int st = 0;
    uint32_t ph = 0, cph = 0;
    bool ok = true;
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(A.ticket, 1u);
    int k = static_cast<int>(__shfl_sync(0xffffffffu, t, 0));
    if (k < A.n_items && lane == 0) batch_load_coefficients(A, k, coef, cfull, pol_keep);   // buffer starts free
    while (k < A.n_items && ok) {
        const BatchItem it = batch_item(A, k);
        const int W = A.mdl[it.m].W, HW = A.mdl[it.m].HW;
        const int i0 = A.mdl[it.m].img_begin + it.blk * A.M;
        const int i1 = min(i0 + A.M, A.mdl[it.m].img_end);
        const int draw_at = max(i1 - NS, i0 + 1);   // draw the next item after issuing this image
        const int tile_start = it.tile * kShTile;
        const int tile_px = min(kShTile, HW - tile_start);
        const int lo_px = max(tile_start - W, 0);
        const uint32_t bytes = static_cast<uint32_t>(min(tile_start + tile_px + W, HW) - lo_px) * 4u;
        int kn = A.n_items;
        bool drawn = false, next_loaded = false;
        for (int base = i0; base < i1 && ok; base += 32) {
            const int64_t px = base + lane < i1 ? __ldg(A.img_px + base + lane) : 0;
            const int cnt = min(32, i1 - base);
            for (int j = 0; j < cnt && ok; ++j) {
                const int64_t pj = __shfl_sync(0xffffffffu, px, j);
                if (lane == 0) {
                    if (mbar_wait_bounded(smem_u32(&empty[st]), ph ^ 1u)) {
                        meta[st] = make_int2(base + j, k);
                        mbar_arrive_expect_tx(smem_u32(&full[st]), bytes);
                        // no L2 hint: the tile's first and last rows are read again, as
                        // halo, by the CTAs on the neighbouring tiles (an evict-first hint
                        // sent a share of them back to DRAM: 4.77 against 4.52 ms at 16384
                        // envs)
                        bulk_g2s_nohint(smem_u32(stages + static_cast<int64_t>(st) * A.stage_floats),
                                        A.depth + pj + lo_px, bytes, smem_u32(&full[st]));
                    } else {
                        raise_dev_error(TACSL_DEVERR_TIMEOUT);
                        ok = false;
                    }
                    if (ok && !drawn && base + j + 1 >= draw_at) {
                        kn = static_cast<int>(atomicAdd(A.ticket, 1u));
                        drawn = true;
                        next_loaded = kn >= A.n_items;
                    }
                    // stage the next item's coefficients once item k's have been taken
                    if (ok && drawn && !next_loaded && mbar_test(smem_u32(cempty), cph)) {
                        batch_load_coefficients(A, kn, coef, cfull, pol_keep);
                        next_loaded = true;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (++st == NS) { st = 0; ph ^= 1u; }
            }
        }
        if (lane == 0 && ok && !next_loaded) {
            // item k ended before its coefficients were taken: wait for that, then stage kn
            if (mbar_wait_bounded(smem_u32(cempty), cph))
                batch_load_coefficients(A, kn, coef, cfull, pol_keep);
            else {
                raise_dev_error(TACSL_DEVERR_TIMEOUT);
                ok = false;
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        kn = __shfl_sync(0xffffffffu, kn, 0);
        cph ^= 1u;
        k = kn;
    }
    if (lane == 0) {
        if (mbar_wait_bounded(smem_u32(&empty[st]), ph ^ 1u)) {
            meta[st] = make_int2(-1, -1);
            mbar_arrive(smem_u32(&full[st]));
        }
        // every ticket of this CTA has been drawn; the last producer out resets the counters
        __threadfence();
        if (atomicAdd(A.ticket + 1, 1u) == gridDim.x - 1) {
            atomicExch(A.ticket, 0u);
            atomicExch(A.ticket + 1, 0u);
        }
    }
}

__global__ void __launch_bounds__(kShThreads, 1) batch_shade_kernel(const BatchShadeArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOffFull);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + kOffEmpty);
    uint64_t* cfull = reinterpret_cast<uint64_t*>(smem + kOffCoefFull);
    uint64_t* cempty = reinterpret_cast<uint64_t*>(smem + kOffCoefEmpty);
    const int2* meta = reinterpret_cast<const int2*>(smem + kOffMeta);
    const float* coef = reinterpret_cast<const float*>(smem + kOffCoef);
    const float* stages = reinterpret_cast<const float*>(smem + kOffStage);
    const int NS = A.n_stages;

    shade_init_barriers(smem, NS);
    if (warp == kShConsumerWarps) {
        batch_shade_producer(A, smem);
        return;
    }

    TileGeom g;
    TileCoefs c;
    int cur_item = -1;
    int st = 0;
    uint32_t ph = 0, cph = 0;
    for (;;) {
        if (!mbar_wait_bounded(smem_u32(&full[st]), ph)) {
            if (lane == 0) raise_dev_error(TACSL_DEVERR_TIMEOUT);
            break;
        }
        const int2 m = meta[st];
        if (m.x < 0) break;
        if (m.y != cur_item) {
            cur_item = m.y;
            const BatchItem it = batch_item(A, m.y);
            const BatchModel& md = A.mdl[it.m];
            tile_geometry(md.H, md.W, md.HW, it.tile, md.cx_c, md.cx_e, md.cy_c, md.cy_e, A.stage_floats, tid, g);
            if (!mbar_wait_bounded(smem_u32(cfull), cph)) {
                if (lane == 0) raise_dev_error(TACSL_DEVERR_TIMEOUT);
                break;
            }
            cph ^= 1u;
            take_coefficients(coef, g, tid, c);
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(cempty));
        }
        const int64_t px0 = __ldg(A.img_px + m.x);
        uint32_t w0, w1, w2;
        shade_four(stages + static_cast<int64_t>(st) * A.stage_floats, g, c, &empty[st], lane, w0, w1, w2);
        if (g.px_valid) store_words(A.rgb + (px0 + g.tile_start + 4 * tid) * 3, w0, w1, w2);
        if (++st == NS) { st = 0; ph ^= 1u; }
    }
}

}  // namespace tacsl

// Tactile-image kernel: depth map -> normals -> per-pixel quadratic shading -> uint8
// RGB (Sec. III-B of arXiv 2408.06506, I_rgb = F(I_depth)).
//
// Design (B300):
// * Four horizontally adjacent pixels per compute thread; a tile is the compute warps'
//   pixels of the flattened H*W image (1408 for the uniform kernel's 11 compute warps,
//   1920 for the batched kernel's 15).  A work item is (block of M images, sensor s,
//   tile); one CTA per SM takes items and keeps the item's 18 shading coefficients per
//   pixel (72 floats per thread) in REGISTERS while it streams the block's images of
//   sensor s through them, so coefficients are read once per item, not once per image.
// * A producer warp streams each image's tile plus one halo row above and below (a
//   contiguous byte range) into a ring of shared-memory stages with the bulk copy
//   engine (cp.async.bulk), signalling full/empty mbarriers; the compute warps never
//   meet at a block-wide barrier.  In the uniform kernel a stage holds three images, so
//   a compute warp's fixed cost per stage is shared by three images and their shading
//   chains interleave.
// * Normals use only shared memory: the thread's 4 pixels, their up/down rows and
//   the two horizontal neighbours.  Borders use one-sided differences via
//   per-thread offsets and scale factors chosen once per item.
// * The producer also stages each item's coefficient rows into shared memory (a
//   coefficient full/empty barrier pair), so switching items costs a shared-memory
//   copy into registers, not an L2 round trip.
// * Arithmetic runs on FP32 pairs (f32x2), quantisation uses two FP instructions and a
//   saturating byte pack per value; horizontal neighbours are read from shared memory.
// * Sparsity of contact: a warp whose 128 pixels all have equal neighbours (the
//   undeformed gel) writes the item's background bytes, which are exactly what the
//   full evaluation gives for n = (0, 0, -1).
// * Each thread writes its four pixels' RGB as three 4-byte words straight to global
//   memory (L2 merges a warp's 384 contiguous bytes into whole sectors); the
//   coefficients carry an evict-last L2 policy.
// * Every barrier wait is bounded (2 s by default; the limit is a kernel argument in the
//   uniform kernel); a warp that gives up sets TACSL_DEVERR_TIMEOUT and leaves.
#pragma once

#include "common.cuh"
#include "taxel.cuh"

namespace tacsl {

constexpr int kShConsumerWarps = 15;                       // compute warps (+1 producer = 16)
constexpr int kShConsumers = kShConsumerWarps * 32;        // 480 compute threads
constexpr int kShThreads = kShConsumers + 32;              // + one producer warp
constexpr int kShTile = kShConsumers * 4;                  // pixels per tile, 4 per thread
constexpr int kShMaxStages = 16;
constexpr int kShCoefFloats = 18 * kShTile;                // one tile's shading coefficients

// Shared-memory layout (bytes).
constexpr int kOffFull = 0;                                        // kShMaxStages x u64
constexpr int kOffEmpty = kOffFull + kShMaxStages * 8;             // kShMaxStages x u64
constexpr int kOffCoefFull = kOffEmpty + kShMaxStages * 8;         // u64
constexpr int kOffCoefEmpty = kOffCoefFull + 8;                    // u64
constexpr int kOffMeta = kOffCoefEmpty + 8;                        // kShMaxStages x int2 (image, item)
constexpr int kOffCoef = ((kOffMeta + kShMaxStages * 8) + 127) / 128 * 128;
constexpr int kOffStage = kOffCoef + kShCoefFloats * 4;

__host__ __device__ constexpr int shade_smem_bytes(int n_stages, int stage_floats) {
    return kOffStage + n_stages * stage_floats * 4;
}

enum StoreMode { kStoreWord = 0, kStoreByte = 1 };

struct ShadeArgs {
    const float* coeffs;        // [S][6][3][HW], 16-byte aligned
    const int32_t* sensor_id;   // [B]
    const float* depth;         // [B][HW], 16-byte aligned
    uint8_t* rgb;               // [B][HW][3]
    int B;                      // images
    int H, W, S, HW, n_tiles;
    int M;                      // images per block (work-item granularity)
    int n_items;                // ceil(B / M) * S * n_tiles
    float cx_c, cx_e, cy_c, cy_e;   // 1/(2 pitch_x), 1/pitch_x, 1/(2 pitch_y), 1/pitch_y
    int n_stages, stage_floats;
    int store_mode;
    uint64_t wait_ns;           // limit of every barrier wait (TACSL default: 2 s)
};

// Work item k = (image block, sensor, tile), tile fastest: consecutive items - run at
// the same time by consecutive CTAs - are the neighbouring tiles of the same images, so
// the halo rows one CTA fetches are in L2 for its neighbours.
struct Item {
    int blk, s, tile;
};
__device__ __forceinline__ Item decode_item(const ShadeArgs& A, int k) {
    const int per_blk = A.S * A.n_tiles;
    Item it;
    it.blk = k / per_blk;
    const int r = k - it.blk * per_blk;
    it.s = r / A.n_tiles;
    it.tile = r - it.s * A.n_tiles;
    return it;
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (sm_100+ f32x2 instructions): lane-wise IEEE fp32, so results are
// bit-identical to the scalar forms.
// ---------------------------------------------------------------------------
typedef uint64_t f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lo(f2 r) { return __uint_as_float(static_cast<uint32_t>(r)); }
__device__ __forceinline__ float hi(f2 r) { return __uint_as_float(static_cast<uint32_t>(r >> 32)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Quantisation to floor(clamp(I, 0, 255) + 0.5).  The kernel evaluates the shading in
// units of 1/256 with the 1/2 folded into the bias term, so t = (I + 0.5)/256; the
// last FMA saturates t to [0, 1] (NaN -> 0).  Multiplying t by 2^-141 with round-down
// then lands on the subnormal k * 2^-149 with k = floor(256 t), whose bit pattern is
// the integer k in [0, 256]; the byte pack saturates 256 (I >= 255.5) to 255.
// (Denormals are kept: this file is built without ftz.)
__device__ __forceinline__ f2 floor256(float ta, float tb) {
    f2 d;
    asm("mul.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(ta, tb)), "l"(pk(__uint_as_float(0x100u), __uint_as_float(0x100u))));
    return d;
}

// 1/sqrt(x) for x >= 1 (the flush-to-zero form differs only on subnormal inputs).
__device__ __forceinline__ float rsqrt_ge1(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Bytes (b0, b1, b2, b3) in memory order from four integers, each saturated to [0, 255].
__device__ __forceinline__ uint32_t pack_u8x4(uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) {
    uint32_t h, w;
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, 0;" : "=r"(h) : "r"(b3), "r"(b2));
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(w) : "r"(b1), "r"(b0), "r"(h));
    return w;
}

// Does block `it` hold an image of sensor it.s?  (Warp-uniform; flags bad sensor ids once
// per block, on the item (sensor 0, tile 0).)
__device__ __forceinline__ bool item_has_images(const ShadeArgs& A, const Item& it) {
    const int lane = threadIdx.x & 31;
    const int b0 = it.blk * A.M, b1 = min(b0 + A.M, A.B);
    const bool check = it.s == 0 && it.tile == 0;
    bool any = false;
    for (int base = b0; base < b1; base += 32) {
        const int b = base + lane;
        const int sid = b < b1 ? __ldg(A.sensor_id + b) : -1;
        if (check && b < b1 && (sid < 0 || sid >= A.S)) raise_dev_error(TACSL_DEVERR_BAD_SENSOR_ID);
        if (__any_sync(0xffffffffu, sid == it.s)) {
            any = true;
            if (!check) break;
        }
    }
    return any;
}

// This CTA's next item (after k) with at least one image of its sensor, or n_items.
__device__ __forceinline__ int next_item(const ShadeArgs& A, int k) {
    for (k += gridDim.x; k < A.n_items; k += gridDim.x)
        if (item_has_images(A, decode_item(A, k))) return k;
    return A.n_items;
}

// ---------------------------------------------------------------------------
// Compute-warp building blocks of the batched image kernel (four pixels per thread)
// ---------------------------------------------------------------------------

// Where this thread's four pixels of one tile and their neighbours sit in a stage
// buffer (the tile plus one halo row above and below), and the derivative scales at
// those pixels: central differences inside, one-sided ones on the image border.
struct TileGeom {
    int tile_start;
    int oc, ou, od, oL, oR;
    f2 cxp0, cxp1, cyy;
    bool px_valid;
};

template <int TILE = kShTile>
__device__ __forceinline__ void tile_geometry(int H, int W, int HW, int tile, float cx_c, float cx_e, float cy_c,
                                              float cy_e, int stage_floats, int tid, TileGeom& g) {
    g.tile_start = tile * TILE;
    const int tile_px = min(TILE, HW - g.tile_start);
    const int lo_px = max(g.tile_start - W, 0);
    g.px_valid = 4 * tid < tile_px;
    const int p = g.tile_start + 4 * tid;
    if (g.px_valid) {
        const int y = p / W, x0 = p - y * W;
        const bool hasL = x0 > 0, hasR = x0 + 4 < W;
        g.oc = p - lo_px;
        g.ou = ((y > 0) ? p - W : p) - lo_px;
        g.od = ((y < H - 1) ? p + W : p) - lo_px;
        g.oL = (hasL ? p - 1 : p) - lo_px;
        g.oR = (hasR ? p + 4 : p + 3) - lo_px;
        const float cyv = (y > 0 && y < H - 1) ? cy_c : cy_e;
        g.cxp0 = pk(hasL ? cx_c : cx_e, cx_c);
        g.cxp1 = pk(cx_c, hasR ? cx_c : cx_e);
        g.cyy = pk(cyv, cyv);
    } else {
        // past the tile's end: read in-bounds stage words and store nothing
        g.oc = min(p - lo_px, stage_floats - 4);
        g.ou = g.od = g.oL = g.oR = g.oc;
        g.cxp0 = g.cxp1 = g.cyy = 0;
    }
}

// The tile's 18 shading coefficients of this thread's four pixels, in registers, and the
// RGB bytes of a flat neighbourhood.
struct TileCoefs {
    f2 cf[6][3][2];                   // term, channel, pixel pair
    uint32_t bg0, bg1, bg2;           // RGB of a flat neighbourhood (n = (0, 0, -1))
};

template <int TILE = kShTile>
__device__ __forceinline__ void take_coefficients(const float* coef, const TileGeom& g, int tid, TileCoefs& c) {
    // coefficients in units of 1/256 with the rounding half folded into the bias:
    // A0/256 + 1/512 and Ak/256 (exact power-of-two scaling)
    const int q = g.px_valid ? 4 * tid : 0;
    const f2 s256 = pk(0.00390625f, 0.00390625f), h512 = pk(0.001953125f, 0.001953125f);
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(coef + (k * 3 + ch) * TILE + q);
            c.cf[k][ch][0] = k == 0 ? fma2(v.x, s256, h512) : mul2(v.x, s256);
            c.cf[k][ch][1] = k == 0 ? fma2(v.y, s256, h512) : mul2(v.y, s256);
        }
    // a flat neighbourhood has m = (1, 0, 0, 0, 0, 0): the chain in shade_four then
    // returns its bias term exactly, so the bytes are those of the bias alone
    f2 qb[3][2];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
#pragma unroll
        for (int j = 0; j < 2; ++j)
            qb[ch][j] = floor256(__saturatef(lo(c.cf[0][ch][j])), __saturatef(hi(c.cf[0][ch][j])));
    c.bg0 = pack_u8x4(__float_as_uint(lo(qb[0][0])), __float_as_uint(lo(qb[1][0])), __float_as_uint(lo(qb[2][0])),
                      __float_as_uint(hi(qb[0][0])));
    c.bg1 = pack_u8x4(__float_as_uint(hi(qb[1][0])), __float_as_uint(hi(qb[2][0])), __float_as_uint(lo(qb[0][1])),
                      __float_as_uint(lo(qb[1][1])));
    c.bg2 = pack_u8x4(__float_as_uint(lo(qb[2][1])), __float_as_uint(hi(qb[0][1])), __float_as_uint(hi(qb[1][1])),
                      __float_as_uint(hi(qb[2][1])));
}

// RGB bytes of this thread's four pixels of the image in stage buffer sp, as three
// words in memory order.  The warp arrives on the stage's empty barrier as soon as its
// shared-memory reads are done.
__device__ __forceinline__ void shade_four(const float* sp, const TileGeom& g, const TileCoefs& c, uint64_t* empty_bar,
                                           int lane, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
    const f2 one2 = pk(1.f, 1.f);
    const float4 cv = *reinterpret_cast<const float4*>(sp + g.oc);
    const ulonglong2 up = *reinterpret_cast<const ulonglong2*>(sp + g.ou);
    const ulonglong2 dn = *reinterpret_cast<const ulonglong2*>(sp + g.od);
    // horizontal neighbours: oL / oR already point at the edge pixel itself on the border
    const float L = sp[g.oL];
    const float R = sp[g.oR];
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(empty_bar));   // this warp is done with the stage

    // depth differences of the pixel pairs (0,1) and (2,3)
    const float ex0 = cv.y - L, ex1 = cv.z - cv.x, ex2 = cv.w - cv.y, ex3 = R - cv.z;
    const f2 ey0 = sub2(dn.x, up.x), ey1 = sub2(dn.y, up.y);
    // Exactness shortcut: where all four pixels see equal neighbours, D_x = D_y = 0,
    // n = (0, 0, -1) and the shading is the bias term; the warp takes it when all of
    // its lanes can (bitwise the bytes of the full evaluation).
    const bool flat = ((__float_as_uint(ex0) | __float_as_uint(ex1) | __float_as_uint(ex2) | __float_as_uint(ex3) |
                        static_cast<uint32_t>(ey0) | static_cast<uint32_t>(ey0 >> 32) | static_cast<uint32_t>(ey1) |
                        static_cast<uint32_t>(ey1 >> 32)) &
                       0x7fffffffu) == 0u;
    w0 = c.bg0;
    w1 = c.bg1;
    w2 = c.bg2;
    if (__all_sync(0xffffffffu, flat || !g.px_valid)) return;
    const f2 gx0 = mul2(pk(ex0, ex1), g.cxp0);
    const f2 gx1 = mul2(pk(ex2, ex3), g.cxp1);
    const f2 gy0 = mul2(ey0, g.cyy);
    const f2 gy1 = mul2(ey1, g.cyy);
    f2 q[2][3];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const f2 gx = j ? gx1 : gx0, gy = j ? gy1 : gy0;
        const f2 s2 = fma2(gx, gx, fma2(gy, gy, one2));
        const f2 r = pk(rsqrt_ge1(lo(s2)), rsqrt_ge1(hi(s2)));
        const f2 nx = mul2(gx, r), ny = mul2(gy, r);
        const f2 m3 = mul2(nx, nx), m4 = mul2(ny, ny), m5 = mul2(nx, ny);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            // t = (I + 0.5)/256: four packed FMAs, the last term per lane with saturation
            const f2 part = fma2(c.cf[4][ch][j], m4,
                                 fma2(c.cf[3][ch][j], m3, fma2(c.cf[2][ch][j], ny, fma2(c.cf[1][ch][j], nx, c.cf[0][ch][j]))));
            const float ta = __saturatef(fmaf(lo(c.cf[5][ch][j]), lo(m5), lo(part)));
            const float tb = __saturatef(fmaf(hi(c.cf[5][ch][j]), hi(m5), hi(part)));
            q[j][ch] = floor256(ta, tb);
        }
    }
    // q[j][ch] holds pixels (2j, 2j+1); memory order is px0 rgb, px1 rgb, px2 rgb, px3 rgb
    w0 = pack_u8x4(__float_as_uint(lo(q[0][0])), __float_as_uint(lo(q[0][1])), __float_as_uint(lo(q[0][2])),
                   __float_as_uint(hi(q[0][0])));
    w1 = pack_u8x4(__float_as_uint(hi(q[0][1])), __float_as_uint(hi(q[0][2])), __float_as_uint(lo(q[1][0])),
                   __float_as_uint(lo(q[1][1])));
    w2 = pack_u8x4(__float_as_uint(lo(q[1][2])), __float_as_uint(hi(q[1][0])), __float_as_uint(hi(q[1][1])),
                   __float_as_uint(hi(q[1][2])));
}

// This thread's four pixels' RGB (12 bytes at dst, 4-byte aligned) as three plain word
// stores.  A warp's stores cover 384 contiguous bytes, which L2 merges into whole
// sectors.  Measured on 8192 images of 320x240: 0.78 ms, against 0.80 ms with an
// evict-first hint on each store, 0.87 ms with an 8-byte plus a 4-byte store, and
// 0.88 ms through a shared-memory transpose to 16-byte stores.
__device__ __forceinline__ void store_words(uint8_t* dst, uint32_t w0, uint32_t w1, uint32_t w2) {
    uint32_t* d32 = reinterpret_cast<uint32_t*>(dst);
    d32[0] = w0;
    d32[1] = w1;
    d32[2] = w2;
}

// Barrier set-up shared by both image kernels (thread 0, then a block barrier).
__device__ __forceinline__ void shade_init_barriers(unsigned char* smem, int NS) {
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOffFull);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + kOffEmpty);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), kShConsumerWarps);
        }
        mbar_init(smem_u32(smem + kOffCoefFull), 1);
        mbar_init(smem_u32(smem + kOffCoefEmpty), kShConsumerWarps);
        mbar_fence_init();
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Uniform image kernel (tacsl_shade_image, tacsl_tactile_step)
// ---------------------------------------------------------------------------
//
// The producer / compute-warp pipeline above, with IPS images per ring stage: the
// producer fills a stage with the tiles of IPS consecutive images of the item (one
// barrier phase for all their copies), and a compute warp takes them in one iteration.
// A warp's fixed cost per iteration (barrier wait, stage lookup, release, store
// addressing, loop) is then shared by IPS images, and their shading chains are
// independent, so the scheduler can interleave them.  NW compute warps of four pixels
// per thread make a tile of NW * 128 pixels.  The per-pixel arithmetic and its order are
// those of shade_four, so the bytes are the same for every NW and IPS.

template <int NW, int IPS>
struct ShadeCfg {
    static constexpr int kWarps = NW;                      // compute warps
    static constexpr int kImages = IPS;                    // images per ring stage
    static_assert(IPS >= 1 && IPS <= 3, "a stage's meta holds up to three images");
    static constexpr int kThreads = NW * 32 + 32;          // + one producer warp
    static constexpr int kTile = NW * 32 * 4;              // pixels per tile
    // shared memory: barriers, per-stage meta (int4), coefficient tile, ring
    static constexpr int kOffFull = 0;
    static constexpr int kOffEmpty = kOffFull + kShMaxStages * 8;
    static constexpr int kOffCoefFull = kOffEmpty + kShMaxStages * 8;
    static constexpr int kOffCoefEmpty = kOffCoefFull + 8;
    static constexpr int kOffMeta = kOffCoefEmpty + 8;
    static constexpr int kOffCoef = (kOffMeta + kShMaxStages * 16 + 127) / 128 * 128;
    static constexpr int kOffStage = kOffCoef + 18 * kTile * 4;
    // slot_floats: one image's tile plus its two halo rows
    static constexpr int smem_bytes(int n_stages, int slot_floats) {
        return kOffStage + n_stages * IPS * slot_floats * 4;
    }
};

// Stage item k's 18 coefficient rows into shared memory (lane 0 issues the copies).
template <int TILE>
__device__ __forceinline__ void load_item_coefficients(const ShadeArgs& A, int k, float* coef, uint64_t* cfull,
                                                       uint64_t pol) {
    const Item it = decode_item(A, k);
    const int tile_start = it.tile * TILE;
    const uint32_t row_bytes = static_cast<uint32_t>(min(TILE, A.HW - tile_start)) * 4u;
    mbar_arrive_expect_tx(smem_u32(cfull), 18u * row_bytes);
    const float* src = A.coeffs + static_cast<int64_t>(it.s) * 18 * A.HW + tile_start;
    for (int r = 0; r < 18; ++r)
        bulk_g2s(smem_u32(coef + r * TILE), src + static_cast<int64_t>(r) * A.HW, row_bytes, smem_u32(cfull), pol);
}

// Producer warp: walks this CTA's items that hold images of their sensor.  Each item's
// coefficient rows are staged into shared memory one item ahead: as soon as the compute
// warps have copied item k's coefficients into registers (coefficient-empty barrier),
// the producer copies item k+1's, while it keeps streaming item k's images - each
// image's tile plus one halo row above and below, a contiguous byte range - into the
// stage ring, IPS images per stage, announcing (images, item) in meta[] (missing
// images are -1).  Every wait is bounded by A.wait_ns; after a timeout the warp
// stops issuing, and before it returns it waits (bounded by the default limit) until
// every copy it issued has landed, so that the CTA never ends with a copy into its
// shared memory still in flight.
template <class CFG>
__device__ __forceinline__ void uniform_producer(const ShadeArgs& A, unsigned char* smem) {
    constexpr int TILE = CFG::kTile, IPS = CFG::kImages;
    const int lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + CFG::kOffFull);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + CFG::kOffEmpty);
    uint64_t* cfull = reinterpret_cast<uint64_t*>(smem + CFG::kOffCoefFull);
    uint64_t* cempty = reinterpret_cast<uint64_t*>(smem + CFG::kOffCoefEmpty);
    int4* meta = reinterpret_cast<int4*>(smem + CFG::kOffMeta);
    float* coef = reinterpret_cast<float*>(smem + CFG::kOffCoef);
    float* stages = reinterpret_cast<float*>(smem + CFG::kOffStage);
    const int NS = A.n_stages;
    const int64_t stage_stride = static_cast<int64_t>(IPS) * A.stage_floats;
    const uint64_t pol_keep = policy_evict_last();
    int st = 0;
    uint32_t ph = 0, cph = 0;   // cph: phase of the coefficient-empty barrier to wait for next
    uint32_t n_fill = 0, n_coef = 0;   // stage phases and coefficient phases started (lane 0)
    bool ok = true;
    int k = (static_cast<int>(blockIdx.x) < A.n_items && item_has_images(A, decode_item(A, blockIdx.x)))
                ? static_cast<int>(blockIdx.x)
                : next_item(A, blockIdx.x);
    if (k < A.n_items && lane == 0) {   // the coefficient buffer starts free
        load_item_coefficients<TILE>(A, k, coef, cfull, pol_keep);
        ++n_coef;
    }
    while (k < A.n_items && ok) {
        const int kn = next_item(A, k);
        bool next_loaded = kn >= A.n_items;
        const Item it = decode_item(A, k);
        const int b0 = it.blk * A.M, b1 = min(b0 + A.M, A.B);
        const int tile_start = it.tile * TILE;
        const int tile_px = min(TILE, A.HW - tile_start);
        const int lo_px = max(tile_start - A.W, 0);
        const uint32_t bytes = static_cast<uint32_t>(min(tile_start + tile_px + A.W, A.HW) - lo_px) * 4u;
        // fill one stage with the images g0, g1, g2 (the first n_grp of them; n_grp <= IPS)
        int g0 = -1, g1 = -1, g2 = -1;
        int n_grp = 0;
        auto fill = [&]() {
            if (lane == 0) {
                if (mbar_wait_bounded(smem_u32(&empty[st]), ph ^ 1u, A.wait_ns)) {
                    meta[st] = make_int4(g0, n_grp > 1 ? g1 : -1, n_grp > 2 ? g2 : -1, k);
                    mbar_arrive_expect_tx(smem_u32(&full[st]), static_cast<uint32_t>(n_grp) * bytes);
                    // the depth tiles carry no L2 hint: their first and last rows are read
                    // again, as halo, by the CTAs working on the neighbouring tiles
                    float* dst = stages + st * stage_stride;
                    const float* src = A.depth + lo_px;
                    bulk_g2s_nohint(smem_u32(dst), src + static_cast<int64_t>(g0) * A.HW, bytes, smem_u32(&full[st]));
                    if (IPS > 1 && n_grp > 1)
                        bulk_g2s_nohint(smem_u32(dst + A.stage_floats), src + static_cast<int64_t>(g1) * A.HW, bytes,
                                        smem_u32(&full[st]));
                    if (IPS > 2 && n_grp > 2)
                        bulk_g2s_nohint(smem_u32(dst + 2 * A.stage_floats), src + static_cast<int64_t>(g2) * A.HW,
                                        bytes, smem_u32(&full[st]));
                    ++n_fill;
                } else {
                    raise_dev_error(TACSL_DEVERR_TIMEOUT);
                    ok = false;
                }
                // stage the next item's coefficients once item k's have been taken
                if (ok && !next_loaded && mbar_test(smem_u32(cempty), cph)) {
                    load_item_coefficients<TILE>(A, kn, coef, cfull, pol_keep);
                    ++n_coef;
                    next_loaded = true;
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            next_loaded = __shfl_sync(0xffffffffu, next_loaded, 0);
            n_grp = 0;
            if (++st == NS) { st = 0; ph ^= 1u; }
        };
        for (int base = b0; base < b1 && ok; base += 32) {
            const int b = base + lane;
            const int sid = b < b1 ? __ldg(A.sensor_id + b) : -1;
            unsigned bal = __ballot_sync(0xffffffffu, sid == it.s);
            while (bal != 0u && ok) {
                const int img = base + __ffs(bal) - 1;
                bal &= bal - 1u;
                if (n_grp == 0) g0 = img;
                else if (n_grp == 1) g1 = img;
                else g2 = img;
                if (++n_grp == IPS) fill();
            }
        }
        if (ok && n_grp > 0) fill();
        if (ok && !next_loaded) {
            // item k ended before its coefficients were taken: wait for that, then stage kn
            if (lane == 0) {
                if (mbar_wait_bounded(smem_u32(cempty), cph, A.wait_ns)) {
                    load_item_coefficients<TILE>(A, kn, coef, cfull, pol_keep);
                    ++n_coef;
                } else {
                    raise_dev_error(TACSL_DEVERR_TIMEOUT);
                    ok = false;
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        cph ^= 1u;
        k = kn;
    }
    if (lane != 0) return;
    // end-of-stream marker: an arrival without bytes completes the stage's phase
    if (mbar_wait_bounded(smem_u32(&empty[st]), ph ^ 1u, A.wait_ns)) {
        meta[st] = make_int4(-1, -1, -1, -1);
        mbar_arrive(smem_u32(&full[st]));
        ++n_fill;
    } else {
        raise_dev_error(TACSL_DEVERR_TIMEOUT);
    }
    // Drain: stage phase i (i = 0, 1, ...) is stage i % NS with parity (i / NS) & 1, and
    // only this lane arrives on the full barriers, so a phase still pending is one whose
    // copies have not landed.  In a normal run the compute warps wait for every copy
    // anyway and these waits return at once; after a timeout they may have left already.
    const uint32_t uNS = static_cast<uint32_t>(NS);
    for (uint32_t i = n_fill > uNS ? n_fill - uNS : 0u; i < n_fill; ++i)
        if (!mbar_wait_bounded(smem_u32(&full[i % uNS]), (i / uNS) & 1u)) raise_dev_error(TACSL_DEVERR_TIMEOUT);
    if (n_coef > 0u && !mbar_wait_bounded(smem_u32(cfull), (n_coef - 1u) & 1u))
        raise_dev_error(TACSL_DEVERR_TIMEOUT);
}

// One elected lane arrives on the barrier after the warp's shared-memory reads (no branch).
__device__ __forceinline__ void warp_arrive(uint32_t bar) {
    __syncwarp();
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(bar)
        : "memory");
}

// Bounded wait on a barrier phase that every lane of the warp polls; the result is made
// warp-uniform, so that the warp either goes on or leaves as one.
__device__ __forceinline__ bool warp_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    const bool ok = mbar_wait_bounded(bar, parity, limit_ns);
    return __all_sync(0xffffffffu, ok);
}

// The full evaluation of the four pixels' RGB words (the arithmetic of shade_four).
__device__ __forceinline__ void quad_eval(const float (&ex)[4], const f2 (&ey)[2], const TileGeom& g,
                                          const TileCoefs& c, uint32_t (&w)[3]) {
    const f2 one2 = pk(1.f, 1.f);
    const f2 gx0 = mul2(pk(ex[0], ex[1]), g.cxp0);
    const f2 gx1 = mul2(pk(ex[2], ex[3]), g.cxp1);
    const f2 gy0 = mul2(ey[0], g.cyy);
    const f2 gy1 = mul2(ey[1], g.cyy);
    f2 q[2][3];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const f2 gx = j ? gx1 : gx0, gy = j ? gy1 : gy0;
        const f2 s2 = fma2(gx, gx, fma2(gy, gy, one2));
        const f2 r = pk(rsqrt_ge1(lo(s2)), rsqrt_ge1(hi(s2)));
        const f2 nx = mul2(gx, r), ny = mul2(gy, r);
        const f2 m3 = mul2(nx, nx), m4 = mul2(ny, ny), m5 = mul2(nx, ny);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            // t = (I + 0.5)/256: four packed FMAs, the last term per lane with saturation
            const f2 part = fma2(c.cf[4][ch][j], m4,
                                 fma2(c.cf[3][ch][j], m3, fma2(c.cf[2][ch][j], ny, fma2(c.cf[1][ch][j], nx, c.cf[0][ch][j]))));
            const float ta = __saturatef(fmaf(lo(c.cf[5][ch][j]), lo(m5), lo(part)));
            const float tb = __saturatef(fmaf(hi(c.cf[5][ch][j]), hi(m5), hi(part)));
            q[j][ch] = floor256(ta, tb);
        }
    }
    // q[j][ch] holds pixels (2j, 2j+1); memory order is px0 rgb, px1 rgb, px2 rgb, px3 rgb
    w[0] = pack_u8x4(__float_as_uint(lo(q[0][0])), __float_as_uint(lo(q[0][1])), __float_as_uint(lo(q[0][2])),
                     __float_as_uint(hi(q[0][0])));
    w[1] = pack_u8x4(__float_as_uint(hi(q[0][1])), __float_as_uint(hi(q[0][2])), __float_as_uint(lo(q[1][0])),
                     __float_as_uint(lo(q[1][1])));
    w[2] = pack_u8x4(__float_as_uint(lo(q[1][2])), __float_as_uint(hi(q[1][0])), __float_as_uint(hi(q[1][1])),
                     __float_as_uint(hi(q[1][2])));
}

template <int STORE>
__device__ __forceinline__ void quad_store(uint8_t* dst, const uint32_t (&w)[3]) {
    if constexpr (STORE == kStoreWord) {
        store_words(dst, w[0], w[1], w[2]);
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = static_cast<uint8_t>(w[k >> 2] >> (8 * (k & 3)));
    }
}

// The RGB words of this thread's four pixels in each of the stage's IPS images (slot i
// at sp + i * slot_floats; image i is missing when img[i] < 0).  The warp arrives on the
// stage's empty barrier as soon as its shared-memory reads are done.  A warp whose 128
// pixels of an image all see equal neighbours (the undeformed gel: D_x = D_y = 0,
// n = (0, 0, -1)) takes the item's background words for it, which are bitwise what the
// full evaluation gives; the other images get the full evaluation, in one block when all
// of them need it, so that their independent chains can interleave.
template <int IPS>
__device__ __forceinline__ void shade_stage(const float* sp, int slot_floats, const int (&img)[3], const TileGeom& g,
                                            const TileCoefs& c, uint32_t empty_bar, uint32_t (&w)[IPS][3]) {
    float4 cv[IPS];
    ulonglong2 up[IPS], dn[IPS];
    float L[IPS], R[IPS];
#pragma unroll
    for (int i = 0; i < IPS; ++i) {
        const float* s = sp + i * slot_floats;   // a missing image reads stale words of its slot
        cv[i] = *reinterpret_cast<const float4*>(s + g.oc);
        up[i] = *reinterpret_cast<const ulonglong2*>(s + g.ou);
        dn[i] = *reinterpret_cast<const ulonglong2*>(s + g.od);
        // horizontal neighbours: oL / oR already point at the edge pixel itself on the border
        L[i] = s[g.oL];
        R[i] = s[g.oR];
    }
    warp_arrive(empty_bar);   // this warp is done with the stage
    float ex[IPS][4];
    f2 ey[IPS][2];
    bool dense[IPS];
    bool any = false, all = true;
#pragma unroll
    for (int i = 0; i < IPS; ++i) {
        ex[i][0] = cv[i].y - L[i];
        ex[i][1] = cv[i].z - cv[i].x;
        ex[i][2] = cv[i].w - cv[i].y;
        ex[i][3] = R[i] - cv[i].z;
        ey[i][0] = sub2(dn[i].x, up[i].x);
        ey[i][1] = sub2(dn[i].y, up[i].y);
        const bool flat = ((__float_as_uint(ex[i][0]) | __float_as_uint(ex[i][1]) | __float_as_uint(ex[i][2]) |
                            __float_as_uint(ex[i][3]) | static_cast<uint32_t>(ey[i][0]) |
                            static_cast<uint32_t>(ey[i][0] >> 32) | static_cast<uint32_t>(ey[i][1]) |
                            static_cast<uint32_t>(ey[i][1] >> 32)) &
                           0x7fffffffu) == 0u;
        dense[i] = !__all_sync(0xffffffffu, flat || !g.px_valid || (i > 0 && img[i] < 0));
        any = any || dense[i];
        all = all && dense[i];
        w[i][0] = c.bg0;
        w[i][1] = c.bg1;
        w[i][2] = c.bg2;
    }
    if (!any) return;
    if (IPS == 1 || all) {
#pragma unroll
        for (int i = 0; i < IPS; ++i) quad_eval(ex[i], ey[i], g, c, w[i]);
    } else {
#pragma unroll
        for (int i = 0; i < IPS; ++i)
            if (dense[i]) quad_eval(ex[i], ey[i], g, c, w[i]);
    }
}

template <class CFG, int STORE>
__global__ void __launch_bounds__(CFG::kThreads, 1) shade_kernel(const ShadeArgs A) {
    constexpr int IPS = CFG::kImages, TILE = CFG::kTile;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + CFG::kOffFull);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + CFG::kOffEmpty);
    uint64_t* cfull = reinterpret_cast<uint64_t*>(smem + CFG::kOffCoefFull);
    uint64_t* cempty = reinterpret_cast<uint64_t*>(smem + CFG::kOffCoefEmpty);
    const int4* meta = reinterpret_cast<const int4*>(smem + CFG::kOffMeta);
    const float* coef = reinterpret_cast<const float*>(smem + CFG::kOffCoef);
    const float* stages = reinterpret_cast<const float*>(smem + CFG::kOffStage);
    const int NS = A.n_stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), CFG::kWarps);
        }
        mbar_init(smem_u32(cfull), 1);
        mbar_init(smem_u32(cempty), CFG::kWarps);
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == CFG::kWarps) {
        uniform_producer<CFG>(A, smem);
        return;
    }

    // ---- compute warps ----
    TileGeom g;
    TileCoefs c;
    int cur_item = -1;
    int st = 0;
    uint32_t ph = 0, cph = 0;
    for (;;) {
        if (!warp_wait_bounded(smem_u32(&full[st]), ph, A.wait_ns)) {
            if (lane == 0) raise_dev_error(TACSL_DEVERR_TIMEOUT);
            break;
        }
        const int4 m = meta[st];   // (image 0, image 1, image 2, item); -1: no image
        if (m.x < 0) break;
        if (m.w != cur_item) {
            // new item: geometry, then the tile's coefficients from shared memory
            cur_item = m.w;
            tile_geometry<TILE>(A.H, A.W, A.HW, decode_item(A, m.w).tile, A.cx_c, A.cx_e, A.cy_c, A.cy_e,
                                A.stage_floats, tid, g);
            if (!warp_wait_bounded(smem_u32(cfull), cph, A.wait_ns)) {
                if (lane == 0) raise_dev_error(TACSL_DEVERR_TIMEOUT);
                break;
            }
            cph ^= 1u;
            take_coefficients<TILE>(coef, g, tid, c);
            warp_arrive(smem_u32(cempty));
        }
        const int img[3] = {m.x, m.y, m.z};
        uint32_t w[IPS][3];
        shade_stage<IPS>(stages + static_cast<int64_t>(st) * IPS * A.stage_floats, A.stage_floats, img, g, c,
                         smem_u32(&empty[st]), w);
        if (g.px_valid) {
            const int64_t px = static_cast<int64_t>(g.tile_start) + 4 * tid;
#pragma unroll
            for (int i = 0; i < IPS; ++i)
                if (i == 0 || img[i] >= 0) quad_store<STORE>(A.rgb + (static_cast<int64_t>(img[i]) * A.HW + px) * 3, w[i]);
        }
        if (++st == NS) { st = 0; ph ^= 1u; }
    }
}

}  // namespace tacsl

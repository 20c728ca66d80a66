// Tactile-image kernel: depth map -> normals -> per-pixel quadratic shading -> uint8
// RGB (Sec. III-B of arXiv 2408.06506, I_rgb = F(I_depth)).
//
// Design (B300):
// * A tile is 1920 consecutive pixels of the flattened H*W image, 4 per compute
//   thread.  A work item is (block of M images, sensor s, tile); one CTA per SM takes
//   items round-robin and keeps the item's 18 shading coefficients per pixel (72
//   floats per thread) in REGISTERS while it streams the block's images of sensor s
//   through them, so coefficients are read once per item, not once per image.
// * A producer warp streams each image's tile plus one halo row above and below (a
//   contiguous byte range) into a ring of shared-memory stages with the bulk copy
//   engine (cp.async.bulk), signalling full/empty mbarriers; the 15 compute warps
//   never meet at a block-wide barrier.
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
//   memory (L2 merges a warp's 384 contiguous bytes into whole sectors); L2 policies
//   mark the depth stream evict-first and the coefficients evict-last.
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

// Stage item k's 18 coefficient rows into shared memory (lane 0 issues the copies).
__device__ __forceinline__ void load_coefficients(const ShadeArgs& A, int k, float* coef, uint64_t* cfull,
                                                  uint64_t pol) {
    const Item it = decode_item(A, k);
    const int tile_start = it.tile * kShTile;
    const uint32_t row_bytes = static_cast<uint32_t>(min(kShTile, A.HW - tile_start)) * 4u;
    mbar_arrive_expect_tx(smem_u32(cfull), 18u * row_bytes);
    const float* src = A.coeffs + static_cast<int64_t>(it.s) * 18 * A.HW + tile_start;
    for (int r = 0; r < 18; ++r)
        bulk_g2s(smem_u32(coef + r * kShTile), src + static_cast<int64_t>(r) * A.HW, row_bytes, smem_u32(cfull), pol);
}

// Producer warp: walks this CTA's items that hold images of their sensor.  Each item's
// coefficient rows are staged into shared memory one item ahead: as soon as the compute
// warps have copied item k's coefficients into registers (coefficient-empty barrier),
// the producer copies item k+1's, while it keeps streaming item k's images - each
// image's tile plus one halo row above and below, a contiguous byte range - into the
// stage ring, announcing (image, item) in meta[].
__device__ __forceinline__ void shade_producer(const ShadeArgs& A, unsigned char* smem) {
    const int lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOffFull);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + kOffEmpty);
    uint64_t* cfull = reinterpret_cast<uint64_t*>(smem + kOffCoefFull);
    uint64_t* cempty = reinterpret_cast<uint64_t*>(smem + kOffCoefEmpty);
    int2* meta = reinterpret_cast<int2*>(smem + kOffMeta);
    float* coef = reinterpret_cast<float*>(smem + kOffCoef);
    float* stages = reinterpret_cast<float*>(smem + kOffStage);
    const int NS = A.n_stages;
    const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
    int st = 0;
    uint32_t ph = 0, cph = 0;   // cph: phase of the coefficient-empty barrier to wait for next
    bool ok = true;
    int k = (static_cast<int>(blockIdx.x) < A.n_items && item_has_images(A, decode_item(A, blockIdx.x)))
                ? static_cast<int>(blockIdx.x)
                : next_item(A, blockIdx.x);
    if (k < A.n_items && lane == 0) load_coefficients(A, k, coef, cfull, pol_keep);   // buffer starts free
    while (k < A.n_items && ok) {
        const int kn = next_item(A, k);
        bool next_loaded = kn >= A.n_items;
        const Item it = decode_item(A, k);
        const int b0 = it.blk * A.M, b1 = min(b0 + A.M, A.B);
        const int tile_start = it.tile * kShTile;
        const int tile_px = min(kShTile, A.HW - tile_start);
        const int lo_px = max(tile_start - A.W, 0);
        const uint32_t bytes = static_cast<uint32_t>(min(tile_start + tile_px + A.W, A.HW) - lo_px) * 4u;
        for (int base = b0; base < b1 && ok; base += 32) {
            const int b = base + lane;
            const int sid = b < b1 ? __ldg(A.sensor_id + b) : -1;
            unsigned bal = __ballot_sync(0xffffffffu, sid == it.s);
            while (bal != 0u && ok) {
                const int j = __ffs(bal) - 1;
                bal &= bal - 1u;
                if (lane == 0) {
                    if (mbar_wait_bounded(smem_u32(&empty[st]), ph ^ 1u)) {
                        meta[st] = make_int2(base + j, k);
                        mbar_arrive_expect_tx(smem_u32(&full[st]), bytes);
                        bulk_g2s(smem_u32(stages + static_cast<int64_t>(st) * A.stage_floats),
                                 A.depth + static_cast<int64_t>(base + j) * A.HW + lo_px, bytes, smem_u32(&full[st]),
                                 pol_stream);
                    } else {
                        raise_dev_error(TACSL_DEVERR_TIMEOUT);
                        ok = false;
                    }
                    // stage the next item's coefficients once item k's have been taken
                    if (ok && !next_loaded && mbar_test(smem_u32(cempty), cph)) {
                        load_coefficients(A, kn, coef, cfull, pol_keep);
                        next_loaded = true;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                next_loaded = __shfl_sync(0xffffffffu, next_loaded, 0);
                if (++st == NS) { st = 0; ph ^= 1u; }
            }
        }
        if (ok && !next_loaded) {
            // item k ended before its coefficients were taken: wait for that, then stage kn
            if (lane == 0) {
                if (mbar_wait_bounded(smem_u32(cempty), cph))
                    load_coefficients(A, kn, coef, cfull, pol_keep);
                else {
                    raise_dev_error(TACSL_DEVERR_TIMEOUT);
                    ok = false;
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        cph ^= 1u;
        k = kn;
    }
    // end-of-stream marker: an arrival without bytes completes the stage's phase
    if (lane == 0 && mbar_wait_bounded(smem_u32(&empty[st]), ph ^ 1u)) {
        meta[st] = make_int2(-1, -1);
        mbar_arrive(smem_u32(&full[st]));
    }
}

// ---------------------------------------------------------------------------
// Compute-warp building blocks (shared by the uniform and the batched kernel)
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

__device__ __forceinline__ void tile_geometry(int H, int W, int HW, int tile, float cx_c, float cx_e, float cy_c,
                                              float cy_e, int stage_floats, int tid, TileGeom& g) {
    g.tile_start = tile * kShTile;
    const int tile_px = min(kShTile, HW - g.tile_start);
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

__device__ __forceinline__ void take_coefficients(const float* coef, const TileGeom& g, int tid, TileCoefs& c) {
    // coefficients in units of 1/256 with the rounding half folded into the bias:
    // A0/256 + 1/512 and Ak/256 (exact power-of-two scaling)
    const int q = g.px_valid ? 4 * tid : 0;
    const f2 s256 = pk(0.00390625f, 0.00390625f), h512 = pk(0.001953125f, 0.001953125f);
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(coef + (k * 3 + ch) * kShTile + q);
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

__global__ void __launch_bounds__(kShThreads, 1) shade_kernel(const ShadeArgs A) {
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
        shade_producer(A, smem);
        return;
    }

    // ---- compute warps ----
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
            // new item: geometry, then the tile's coefficients from shared memory
            cur_item = m.y;
            const Item it = decode_item(A, m.y);
            tile_geometry(A.H, A.W, A.HW, it.tile, A.cx_c, A.cx_e, A.cy_c, A.cy_e, A.stage_floats, tid, g);
            if (!mbar_wait_bounded(smem_u32(cfull), cph)) {
                if (lane == 0) raise_dev_error(TACSL_DEVERR_TIMEOUT);
                break;
            }
            cph ^= 1u;
            take_coefficients(coef, g, tid, c);
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(cempty));
        }
        uint32_t w0, w1, w2;
        shade_four(stages + static_cast<int64_t>(st) * A.stage_floats, g, c, &empty[st], lane, w0, w1, w2);
        const int64_t img = m.x;
        if (g.px_valid) {
            uint8_t* dst = A.rgb + (img * A.HW + g.tile_start + 4 * tid) * 3;
            if (A.store_mode == kStoreWord) {
                store_words(dst, w0, w1, w2);
            } else {
                const uint32_t ws[3] = {w0, w1, w2};
#pragma unroll
                for (int k = 0; k < 12; ++k) dst[k] = static_cast<uint8_t>(ws[k >> 2] >> (8 * (k & 3)));
            }
        }
        if (++st == NS) { st = 0; ph ^= 1u; }
    }
}

}  // namespace tacsl

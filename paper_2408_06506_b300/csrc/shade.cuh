// Tactile-image kernel: depth map -> normals -> per-pixel quadratic shading -> uint8
// RGB (Sec. III-B of arXiv 2408.06506, I_rgb = F(I_depth)), and the fused tactile
// step that runs the force field (taxel.cuh) in the same persistent launch.
//
// Design (B300):
// * The work is (sensor s, pixel tile, image) units.  A tile is 2048 consecutive
//   pixels of the flattened H*W image, 4 per thread of a 512-thread CTA.  One CTA per
//   SM runs persistently over a contiguous range of units ordered sensor-major,
//   tile-next, image-last, so a CTA keeps one tile's 18 shading coefficients per pixel
//   (72 floats per thread) in REGISTERS and streams many images through them.  The
//   coefficients are read once per CTA per tile instead of once per image.
// * Each unit's depth tile plus one row of halo above and below is a contiguous byte
//   range; the 1-D bulk copy engine (cp.async.bulk) moves it into a ring of
//   shared-memory stages, completion tracked by mbarriers, several images ahead.
// * Normals use only shared memory: the thread's 4 pixels, their up/down rows and
//   the two horizontal neighbours.  Borders use one-sided differences via
//   per-thread offsets and scale factors chosen once per tile.
// * Quantised RGB goes to a shared staging buffer (3 rotating) and leaves with one
//   bulk store per tile (when the output allows 16-byte bulk copies).
// * Images whose sensor differs from the unit's sensor are skipped by building, per
//   run, the list of the sensor's images from sensor_id with block-wide ballots.
#pragma once

#include "common.cuh"
#include "taxel.cuh"

namespace tacsl {

constexpr int kShThreads = 512;
constexpr int kShWarps = kShThreads / 32;
constexpr int kShTile = kShThreads * 4;   // pixels per tile
constexpr int kShList = 1024;             // images per run
constexpr int kShStaging = 3;             // RGB staging buffers
constexpr int kShMaxStages = 16;

// Shared-memory layout (bytes).
constexpr int kOffBar = 0;                                             // kShMaxStages x u64
constexpr int kOffList = kOffBar + kShMaxStages * 8;                   // kShList x i32
constexpr int kOffCnt = kOffList + kShList * 4;                        // kShWarps x TACSL_MAX_SENSOR x i32
constexpr int kOffWtot = kOffCnt + kShWarps * TACSL_MAX_SENSOR * 4;   // kShWarps x i32
constexpr int kOffNs = kOffWtot + kShWarps * 4;                        // TACSL_MAX_SENSOR x i32
constexpr int kOffFlag = kOffNs + TACSL_MAX_SENSOR * 4;                // i32
constexpr int kOffRed = kOffFlag + 16;                                 // kShWarps x 6 f32
constexpr int kOffStage = ((kOffRed + kShWarps * 6 * 4) + 127) / 128 * 128;
constexpr int kStagingBytes = kShTile * 3;

__host__ __device__ constexpr int shade_smem_bytes(int n_stages, int stage_floats) {
    return kOffStage + n_stages * stage_floats * 4 + kShStaging * kStagingBytes;
}

enum StoreMode { kStoreBulk = 0, kStoreWord = 1, kStoreByte = 2 };

struct ShadeArgs {
    const float* coeffs;        // [S][6][3][HW]
    const int32_t* sensor_id;   // [B]
    const float* depth;         // [B][HW], 16-byte aligned
    uint8_t* rgb;               // [B][HW][3]
    int B;                      // images
    int H, W, S, HW, n_tiles;
    float cx_c, cx_e, cy_c, cy_e;   // 1/(2 pitch_x), 1/pitch_x, 1/(2 pitch_y), 1/pitch_y
    int n_stages, stage_floats;
    int store_mode;
};

struct TaxelArgs {                  // force-field half of the fused step
    Params4 prm;
    int B, P, T;
    const float* taxels;
    const int32_t* obj_id;
    const float* pad_pose;
    const float* pad_twist;
    float* depth;
    float* f_n;
    float* f_t;
    float* wrench;
};

__device__ __forceinline__ uint32_t quantize_u8(float I) {
    // floor(clamp(I, 0, 255) + 0.5); fmaxf drops NaN to 0
    return __float2uint_rz(fminf(fmaxf(I, 0.f), 255.f) + 0.5f);
}

template <bool kTaxels>
__device__ __forceinline__ void shade_body(const ShadeArgs& A, const TaxelArgs& X, const SdfTable* tab,
                                           unsigned char* smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, cta = blockIdx.x;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
    int* list = reinterpret_cast<int*>(smem + kOffList);
    int* cnt = reinterpret_cast<int*>(smem + kOffCnt);
    int* wtot = reinterpret_cast<int*>(smem + kOffWtot);
    int* ns = reinterpret_cast<int*>(smem + kOffNs);
    volatile int* flag = reinterpret_cast<volatile int*>(smem + kOffFlag);
    float* red = reinterpret_cast<float*>(smem + kOffRed);
    float* stages = reinterpret_cast<float*>(smem + kOffStage);
    uint8_t* staging = smem + kOffStage + A.n_stages * A.stage_floats * 4;
    const int NS = A.n_stages;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
        mbar_fence_init();
        *flag = 0;
    }
    for (int i = tid; i < kShWarps * TACSL_MAX_SENSOR; i += kShThreads) cnt[i] = 0;
    __syncthreads();

    // ---- images per sensor (every CTA counts them; B int32 reads from L2) ----
    for (int base = 0; base < A.B; base += kShThreads) {
        const int b = base + tid;
        const int sid = b < A.B ? __ldg(A.sensor_id + b) : 0;
        const bool bad = b < A.B && (sid < 0 || sid >= A.S);
        if (__any_sync(0xffffffffu, bad) && lane == 0 && cta == 0) raise_dev_error(TACSL_DEVERR_BAD_SENSOR_ID);
        for (int s = 0; s < A.S; ++s) {
            const unsigned m = __ballot_sync(0xffffffffu, b < A.B && sid == s);
            if (lane == 0) cnt[warp * TACSL_MAX_SENSOR + s] += __popc(m);
        }
    }
    __syncthreads();
    if (tid < A.S) {
        int t = 0;
        for (int w = 0; w < kShWarps; ++w) t += cnt[w * TACSL_MAX_SENSOR + tid];
        ns[tid] = t;
    }
    __syncthreads();
    int64_t n_valid = 0;
    for (int s = 0; s < A.S; ++s) n_valid += ns[s];
    const int64_t U = n_valid * A.n_tiles;
    int64_t u = U * cta / G;
    const int64_t u1 = U * (cta + 1) / G;

    auto taxel_phase = [&]() {
        if constexpr (kTaxels) {
            const int64_t p0 = static_cast<int64_t>(X.B) * cta / G, p1 = static_cast<int64_t>(X.B) * (cta + 1) / G;
            for (int64_t b = p0; b < p1; ++b)
                process_pad<kShWarps>(*tab, X.prm, X.P, X.T, X.taxels, X.obj_id, X.pad_pose, X.pad_twist, X.depth,
                                      X.f_n, X.f_t, X.wrench, b, red);
        }
    };

    int64_t g = 0;   // items consumed by this CTA (drives stage index and barrier parity)
    // current run: sensor, tile, length; tile geometry
    int s = 0, tile = 0, run = 0;
    int tile_start = 0, tile_px = 0, lo = 0, load_floats = 0;

    // Decode unit u into (sensor, tile, rank), build the list of the run's images and
    // issue the first loads of the run.
    auto begin_run = [&]() {
        s = 0;
        int64_t cum = 0;
        while (cum + static_cast<int64_t>(ns[s]) * A.n_tiles <= u) { cum += static_cast<int64_t>(ns[s]) * A.n_tiles; ++s; }
        const int64_t local = u - cum;
        tile = static_cast<int>(local / ns[s]);
        const int j0 = static_cast<int>(local % ns[s]);
        run = static_cast<int>(min(min(u1 - u, static_cast<int64_t>(ns[s] - j0)), static_cast<int64_t>(kShList)));
        __syncthreads();   // previous run's readers of `list` are done
        int rank_base = 0;
        for (int base = 0; base < A.B && rank_base < j0 + run; base += kShThreads) {
            const int b = base + tid;
            const bool m = b < A.B && __ldg(A.sensor_id + b) == s;
            const unsigned bal = __ballot_sync(0xffffffffu, m);
            if (lane == 0) wtot[warp] = __popc(bal);
            __syncthreads();
            int woff = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kShWarps; ++w) {
                const int c = wtot[w];
                woff += (w < warp) ? c : 0;
                total += c;
            }
            const int r = rank_base + woff + __popc(bal & ((1u << lane) - 1u));
            if (m && r >= j0 && r < j0 + run) list[r - j0] = b;
            rank_base += total;
            __syncthreads();
        }
        tile_start = tile * kShTile;
        tile_px = min(kShTile, A.HW - tile_start);
        lo = max(tile_start - A.W, 0);
        load_floats = min(tile_start + tile_px + A.W, A.HW) - lo;
        if (tid == 0) {
            fence_proxy_async_smem();
            const int npro = min(run, NS);
            for (int i = 0; i < npro; ++i) {
                const int64_t gi = g + i;
                const int st = static_cast<int>(gi % NS);
                const uint32_t bar = smem_u32(&bars[st]);
                mbar_arrive_expect_tx(bar, load_floats * 4);
                bulk_g2s(smem_u32(stages + static_cast<int64_t>(st) * A.stage_floats),
                         A.depth + static_cast<int64_t>(list[i]) * A.HW + lo, load_floats * 4, bar);
            }
        }
    };

    // The first run's loads are in flight while the CTA computes its share of the
    // force field; the coefficient registers are not live yet.
    if (u < u1) begin_run();
    taxel_phase();

    float4 cf[6][3];
    int cur_s = -1, cur_tile = -1;
    int oc = 0, ou = 0, od = 0, oL = 0, oR = 0;
    float cxL = 0.f, cxR = 0.f, cyv = 0.f;
    bool px_valid = false;
    bool abort = false;

    while (u < u1) {
        if (s != cur_s || tile != cur_tile) {
            cur_s = s;
            cur_tile = tile;
            const int p = tile_start + 4 * tid;
            px_valid = (4 * tid) < tile_px;
            const int pp = px_valid ? p : tile_start;
            const int y = pp / A.W, x0 = pp - y * A.W;
            oc = pp - lo;
            ou = ((y > 0) ? pp - A.W : pp) - lo;
            od = ((y < A.H - 1) ? pp + A.W : pp) - lo;
            oL = ((x0 > 0) ? pp - 1 : pp) - lo;
            oR = ((x0 + 4 < A.W) ? pp + 4 : pp + 3) - lo;
            cxL = (x0 > 0) ? A.cx_c : A.cx_e;
            cxR = (x0 + 4 < A.W) ? A.cx_c : A.cx_e;
            cyv = (y > 0 && y < A.H - 1) ? A.cy_c : A.cy_e;
            const float4* cp = reinterpret_cast<const float4*>(A.coeffs + static_cast<int64_t>(s) * 18 * A.HW + pp);
#pragma unroll
            for (int k = 0; k < 6; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) cf[k][c] = __ldg(cp + static_cast<int64_t>(k * 3 + c) * (A.HW / 4));
        }

        // ---- pipeline over the run's images ----
        int i_abort = -1;
        for (int i = 0; i < run; ++i) {
            const int64_t gi = g + i;
            const int st = static_cast<int>(gi % NS);
            const uint32_t parity = static_cast<uint32_t>((gi / NS) & 1);
            if (!mbar_wait_bounded(smem_u32(&bars[st]), parity)) *flag = 1;
            const float* sp = stages + static_cast<int64_t>(st) * A.stage_floats;
            uint32_t w0 = 0, w1 = 0, w2 = 0;
            if (px_valid) {
                const float4 c = *reinterpret_cast<const float4*>(sp + oc);
                const float4 up = *reinterpret_cast<const float4*>(sp + ou);
                const float4 dn = *reinterpret_cast<const float4*>(sp + od);
                const float L = sp[oL], R = sp[oR];
                const float gx[4] = {(c.y - L) * cxL, (c.z - c.x) * A.cx_c, (c.w - c.y) * A.cx_c, (R - c.z) * cxR};
                const float gy[4] = {(dn.x - up.x) * cyv, (dn.y - up.y) * cyv, (dn.z - up.z) * cyv, (dn.w - up.w) * cyv};
                uint32_t q[12];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float r = rsqrtf(fmaf(gx[k], gx[k], fmaf(gy[k], gy[k], 1.f)));
                    const float nx = gx[k] * r, ny = gy[k] * r;
                    const float m3 = nx * nx, m4 = ny * ny, m5 = nx * ny;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const float a0 = (&cf[0][ch].x)[k], a1 = (&cf[1][ch].x)[k], a2 = (&cf[2][ch].x)[k];
                        const float a3 = (&cf[3][ch].x)[k], a4 = (&cf[4][ch].x)[k], a5 = (&cf[5][ch].x)[k];
                        const float I = fmaf(a5, m5, fmaf(a4, m4, fmaf(a3, m3, fmaf(a2, ny, fmaf(a1, nx, a0)))));
                        q[3 * k + ch] = quantize_u8(I);
                    }
                }
                w0 = q[0] | (q[1] << 8) | (q[2] << 16) | (q[3] << 24);
                w1 = q[4] | (q[5] << 8) | (q[6] << 16) | (q[7] << 24);
                w2 = q[8] | (q[9] << 8) | (q[10] << 16) | (q[11] << 24);
            }
            const int64_t img = list[i];
            if (A.store_mode == kStoreBulk) {
                uint32_t* sg = reinterpret_cast<uint32_t*>(staging + static_cast<int>(gi % kShStaging) * kStagingBytes);
                if (px_valid) { sg[3 * tid] = w0; sg[3 * tid + 1] = w1; sg[3 * tid + 2] = w2; }
                fence_proxy_async_smem();
            } else if (px_valid) {
                uint8_t* dst = A.rgb + (img * A.HW + tile_start + 4 * tid) * 3;
                if (A.store_mode == kStoreWord) {
                    uint32_t* d32 = reinterpret_cast<uint32_t*>(dst);
                    d32[0] = w0; d32[1] = w1; d32[2] = w2;
                } else {
                    const uint32_t ws[3] = {w0, w1, w2};
#pragma unroll
                    for (int k = 0; k < 12; ++k) dst[k] = static_cast<uint8_t>(ws[k >> 2] >> (8 * (k & 3)));
                }
            }
            __syncthreads();   // stage consumed, staging written
            if (*flag) { i_abort = i; break; }
            if (tid == 0) {
                if (A.store_mode == kStoreBulk) {
                    bulk_s2g(A.rgb + (img * A.HW + tile_start) * 3,
                             smem_u32(staging + static_cast<int>(gi % kShStaging) * kStagingBytes), tile_px * 3);
                    bulk_commit();
                }
                if (i + NS < run) {
                    fence_proxy_async_smem();
                    const uint32_t bar = smem_u32(&bars[st]);
                    mbar_arrive_expect_tx(bar, load_floats * 4);
                    bulk_g2s(smem_u32(stages + static_cast<int64_t>(st) * A.stage_floats),
                             A.depth + static_cast<int64_t>(list[i + NS]) * A.HW + lo, load_floats * 4, bar);
                }
                if (A.store_mode == kStoreBulk) bulk_wait_read<1>();
            }
        }
        if (i_abort >= 0) {
            // Loads of items [i_abort, i_abort + NS) may still be landing: wait for them
            // (bounded) before the CTA's shared memory goes away.
            if (tid == 0) {
                for (int i = i_abort; i < min(run, i_abort + NS); ++i) {
                    const int64_t gi = g + i;
                    mbar_wait_bounded(smem_u32(&bars[gi % NS]), static_cast<uint32_t>((gi / NS) & 1), 100000000ull);
                }
                raise_dev_error(TACSL_DEVERR_TIMEOUT);
            }
            abort = true;
            break;
        }
        g += run;
        u += run;
        if (u < u1) begin_run();
    }
    (void)abort;
    if (tid == 0 && A.store_mode == kStoreBulk) bulk_wait_all();
}

__global__ void __launch_bounds__(kShThreads, 1) shade_kernel(const ShadeArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const TaxelArgs X{};
    shade_body<false>(A, X, nullptr, smem);
}

__global__ void __launch_bounds__(kShThreads, 1) step_kernel(const ShadeArgs A, const TaxelArgs X, const SdfTable tab) {
    extern __shared__ __align__(128) unsigned char smem[];
    shade_body<true>(A, X, &tab, smem);
}

}  // namespace tacsl

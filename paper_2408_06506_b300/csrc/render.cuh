// Depth-map rendering for the tactile image (Sec. III-B of arXiv 2408.06506: a camera
// at the optical location inside the sensor renders the depth of the indenting object).
//
// Camera reading: orthographic, looking along the pad normal.  Pixel (i, j) sees the
// pad-frame column (x0 + i*pitch_x, y0 + j*pitch_y, z); the undeformed gel at z = 0 reads
// d0; where the object reaches below the gel, the camera sees the object's first point
// on the column: D = d0 - max(0, -z_hit), z_hit searched over [-z_max, 0] from below.
//
// March: conservative sphere tracing up the column - step kappa*phi inside the grid
// domain, kappa = 1/|d|_1 for the column's direction d = R e_z (each partial derivative
// of the trilinear interpolant of a 1-Lipschitz field is at most 1 in magnitude, so along
// d phi changes by at most |d|_1 per unit height, between 1 and sqrt 3: a step cannot
// pass the surface; the isotropic bound 1/sqrt 3 took 6.09 against 5.53 ms for 8192
// maps of 320x240), never less than voxel/8 - then
// bisection of the first bracket down to voxel * 2^-16; z_hit is the bracket's upper
// end.  phi is the trilinear interpolant of the force field (same cell rule and FMA
// order as phi_cell8), so image and force field see the same SDF; outside the grid's
// domain the SDF is undefined and no point there counts as inside the object.
//
// Two shortcuts leave the result unchanged.  The march runs over the part of the column
// inside the domain alone, found by a slab test: outside it the reference march's
// box-distance steps can only end in a miss or reach that part.  And when the distance
// bound already covers the rest of that part (with a 1e-4 relative margin) the column
// misses without further samples: by the same Lipschitz bound none of them could be
// inside the object.  Samples are taken in grid-index space (u = (x - origin) / voxel,
// affine in the column's height), not by posing each point; the current trilinear cell
// and its 8 nodes stay in registers while samples remain in it.  The step itself is
// longer than the reference march's isotropic kappa = 1/sqrt 3: both are conservative and
// share the voxel/8 minimum step, so they can differ only on a column where the object
// dips below it for less than that minimum step (92 of the 629M columns of the 4096-env
// workload: a hit on one side, a miss on the other, the hit on the surface).
//
// One thread per column: a warp takes 32 neighbouring columns of a row, whose marches
// take similar paths and whose SDF reads fall on neighbouring nodes.
#pragma once

#include "common.cuh"
#include "taxel.cuh"

namespace tacsl {

constexpr int kMarchMax = 1024;   // safety cap on march steps (never reached in practice)
constexpr int kBisectMax = 40;    // bisection stops at a bracket <= voxel * 2^-16 (~13 halvings)

struct CameraArgs {
    int H, W;
    float pitch_x, pitch_y, x0, y0, d0, z_max;
};

// The trilinear cell of the last sample (as float indices) and its 8 node values.
struct CellCacheF {
    float cx = -1.f, cy = -1.f, cz = -1.f;
    float v[2][2][2];
};

// phi at a continuous grid index u inside the domain: trilinear in the cell
// min(floor(u), n - 2), nodes re-read only when the cell changes.  The caller samples
// only the slab where every u_a lies in [0.5, n_a - 1.5] (up to ~1e-5 of rounding), so
// floor(u) is already in [0, n - 2]; fmaxf maps a NaN index (a degenerate pose) to cell
// 0, which keeps the loads in bounds.
__device__ __forceinline__ float column_phi_in(const DevSdf& S, float ux, float uy, float uz, uint64_t pol,
                                               CellCacheF& cc) {
    const float cx = fmaxf(floorf(ux), 0.f);
    const float cy = fmaxf(floorf(uy), 0.f);
    const float cz = fmaxf(floorf(uz), 0.f);
    if (cx != cc.cx || cy != cc.cy || cz != cc.cz) {
        const int n0 = S.n0, n01 = S.n0 * S.n1;
        const float* b = S.data + (static_cast<int64_t>(static_cast<int>(cz)) * n01 +
                                   static_cast<int64_t>(static_cast<int>(cy)) * n0 + static_cast<int>(cx));
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 2; ++i) cc.v[k][j][i] = ldg_f_hint(b + k * n01 + j * n0 + i, pol);
        cc.cx = cx;
        cc.cy = cy;
        cc.cz = cz;
    }
    const float fx = ux - cx, fy = uy - cy, fz = uz - cz;
    float c[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float r0 = fmaf(fx, cc.v[k][0][1], (1.f - fx) * cc.v[k][0][0]);
        const float r1 = fmaf(fx, cc.v[k][1][1], (1.f - fx) * cc.v[k][1][0]);
        c[k] = fmaf(fy, r1, (1.f - fy) * r0);
    }
    return fmaf(fz, c[1], (1.f - fz) * c[0]);
}

// One image's column frame in grid-index space: the continuous grid index of pixel
// (i, j) at height z is u = u00 + i ui + j uj + z du, i.e. (R (x_i, y_j, z) + t - origin)
// / voxel with x_i = x0 + i pitch_x, y_j = y0 + j pitch_y; inv_du = 1 / du (+-inf for a
// zero component) gives the heights where the column crosses the domain's faces.
struct __align__(16) RenderFrame {
    float u00[3];
    int id;          // object id, -1 when out of range
    float ui[3], kappa;   // kappa: march step per unit of phi, 1 / |R e_z|_1
    float uj[3];
    int tile_out;         // every column of the block's tile misses the grid's domain
    float du[3], pad2;
    float inv_du[3], pad3;
};
constexpr int kRenderFrames = 256;   // frames a block keeps in shared memory at a time

// Frame of the image of pad b (pose row b) against object id, for the tile of pixel
// columns i in [i0, i1], j in [j0, j1].
__device__ __forceinline__ void render_frame(const SdfTable& tab, int id, const float* pad_pose, int64_t b,
                                             const CameraArgs& cam, int i0, int i1, int j0, int j1,
                                             RenderFrame& f) {
    if (id < 0 || id >= tab.count) {
        f.id = -1;
        return;
    }
    const DevSdf& S = tab.s[id];
    const float* pose = pad_pose + b * 7;
    float r[9];
    quat_to_rot(__ldg(pose + 3), __ldg(pose + 4), __ldg(pose + 5), __ldg(pose + 6), r);
    const float t[3] = {__ldg(pose), __ldg(pose + 1), __ldg(pose + 2)};
    const float o[3] = {S.ox, S.oy, S.oz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f.u00[a] = (fmaf(r[3 * a], cam.x0, fmaf(r[3 * a + 1], cam.y0, t[a])) - o[a]) * S.inv_h;
        f.ui[a] = r[3 * a] * cam.pitch_x * S.inv_h;
        f.uj[a] = r[3 * a + 1] * cam.pitch_y * S.inv_h;
        f.du[a] = r[3 * a + 2] * S.inv_h;
        f.inv_du[a] = 1.f / f.du[a];
    }
    f.kappa = 1.f / (fabsf(r[2]) + fabsf(r[5]) + fabsf(r[8]));
    f.id = id;
    // The tile's columns fill the box i in [i0, i1], j in [j0, j1], z in [-z_max, 0], whose
    // image under the affine u has, per axis, the range [lo, hi] below; when some axis's
    // range lies outside [0.5, n_a - 1.5] (by a margin of 1/64 voxel, far above the
    // rounding of the per-column slab test), no column of the tile meets the domain, so
    // each reads d0, as its own slab test would find.
    const float n[3] = {static_cast<float>(S.n0), static_cast<float>(S.n1), static_cast<float>(S.n2)};
    bool out = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = f.u00[a] + fminf(i0 * f.ui[a], i1 * f.ui[a]) + fminf(j0 * f.uj[a], j1 * f.uj[a]) +
                         fminf(-cam.z_max * f.du[a], 0.f);
        const float hi = f.u00[a] + fmaxf(i0 * f.ui[a], i1 * f.ui[a]) + fmaxf(j0 * f.uj[a], j1 * f.uj[a]) +
                         fmaxf(-cam.z_max * f.du[a], 0.f);
        out = out || hi < 0.5f - 1.f / 64.f || lo > n[a] - 1.5f + 1.f / 64.f;
    }
    f.tile_out = out ? 1 : 0;
}

// Grid: (32 x 8 pixel tiles of the image, up to 64 image slots); block y takes images
// y, y + gridDim.y, ...  Each thread keeps its column across those images.  The images'
// frames are computed up front, kRenderFrames at a time, into shared memory.  Per
// column: the part of [-z_max, 0] inside the grid's domain (slab test on the affine
// u(z)); outside it the SDF is undefined and no point counts as inside the object, so
// the march runs over that part alone, 3 FMAs per sample.
// Image b is pad b of E x P pads (object obj_id[b / P], pixels at b * H * W) when img_po
// is NULL; otherwise the entry img_po[b] = (pad, object) of an image list, with its first
// pixel at img_px[b] (the batched render over one camera model).
__global__ void __launch_bounds__(256) render_kernel(const SdfTable tab, int64_t B, int P,
                                                     const int32_t* __restrict__ obj_id,
                                                     const float* __restrict__ pad_pose, const CameraArgs cam,
                                                     float* __restrict__ depth, const int2* __restrict__ img_po,
                                                     const int64_t* __restrict__ img_px) {
    __shared__ RenderFrame frames[kRenderFrames];
    const int tiles_x = (cam.W + 31) / 32;
    const int tile_y = static_cast<int>(blockIdx.x) / tiles_x, tile_x = static_cast<int>(blockIdx.x) - tile_y * tiles_x;
    const int i = tile_x * 32 + static_cast<int>(threadIdx.x & 31), j = tile_y * 8 + static_cast<int>(threadIdx.x >> 5);
    const bool live = i < cam.W && j < cam.H;
    const int64_t HW = static_cast<int64_t>(cam.H) * cam.W;
    const int pix = j * cam.W + i;
    const uint64_t pol = policy_evict_last();
    const float fi = static_cast<float>(i), fj = static_cast<float>(j);
    const int64_t n_img = (B - static_cast<int64_t>(blockIdx.y) + gridDim.y - 1) / gridDim.y;
    for (int64_t base = 0; base < n_img; base += kRenderFrames) {
        const int n_here = static_cast<int>(n_img - base < kRenderFrames ? n_img - base : kRenderFrames);
        __syncthreads();       // the previous frames are no longer read
        if (static_cast<int>(threadIdx.x) < n_here) {
            const int64_t b = static_cast<int64_t>(blockIdx.y) + (base + threadIdx.x) * gridDim.y;
            const int ti0 = tile_x * 32, tj0 = tile_y * 8;
            const int ti1 = min(ti0 + 31, cam.W - 1), tj1 = min(tj0 + 7, cam.H - 1);
            if (img_po == nullptr) {
                render_frame(tab, __ldg(obj_id + static_cast<int>(b / P)), pad_pose, b, cam, ti0, ti1, tj0, tj1,
                             frames[threadIdx.x]);
            } else {
                const int2 po = __ldg(img_po + b);
                render_frame(tab, po.y, pad_pose, po.x, cam, ti0, ti1, tj0, tj1, frames[threadIdx.x]);
            }
        }
        __syncthreads();
        if (!live) continue;
        for (int m = 0; m < n_here; ++m) {
            const int64_t b = static_cast<int64_t>(blockIdx.y) + (base + m) * gridDim.y;
            const int64_t k = (img_px == nullptr ? b * HW : __ldg(img_px + b)) + pix;
            const RenderFrame& F = frames[m];
            if (F.id < 0) {
                depth[k] = __int_as_float(0x7fc00000);
                raise_dev_error(TACSL_DEVERR_BAD_OBJ_ID);
                continue;
            }
            if (F.tile_out) {              // the whole tile misses the domain (block-uniform)
                depth[k] = cam.d0;
                continue;
            }
            const DevSdf& S = tab.s[F.id];
            const float du0 = F.du[0], du1 = F.du[1], du2 = F.du[2];
            const float u0 = fmaf(fj, F.uj[0], fmaf(fi, F.ui[0], F.u00[0]));
            const float u1 = fmaf(fj, F.uj[1], fmaf(fi, F.ui[1], F.u00[1]));
            const float u2 = fmaf(fj, F.uj[2], fmaf(fi, F.ui[2], F.u00[2]));
            // heights where the column is inside the domain: u_a(z) in [0.5, n_a - 1.5]
            float zlo = -cam.z_max, zhi = 0.f;
            {
                const float ua[3] = {u0, u1, u2}, hi[3] = {static_cast<float>(S.n0) - 1.5f,
                                                           static_cast<float>(S.n1) - 1.5f,
                                                           static_cast<float>(S.n2) - 1.5f};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float ta = (0.5f - ua[a]) * F.inv_du[a], tb = (hi[a] - ua[a]) * F.inv_du[a];
                    zlo = fmaxf(zlo, fminf(ta, tb));
                    zhi = fminf(zhi, fmaxf(ta, tb));
                }
            }
            float zhit = 1.f;   // > 0: no hit
            if (zlo <= zhi) {
                const float dmin = S.h * 0.125f, kappa = F.kappa;
                CellCacheF cc;
                float z = zlo;
                float phi = column_phi_in(S, fmaf(z, du0, u0), fmaf(z, du1, u1), fmaf(z, du2, u2), pol, cc);
                if (phi <= 0.f) {
                    zhit = z;
                } else {
                    for (int it = 0; it < kMarchMax; ++it) {
                        // no point of the object within the distance bound of the sample:
                        // when that covers the rest of the column's in-domain part, it misses
                        const float bound = kappa * phi;
                        if (bound > (zhi - z) * 1.0001f) break;
                        const float zn = fminf(z + fmaxf(bound, dmin), zhi);
                        const float phin =
                            column_phi_in(S, fmaf(zn, du0, u0), fmaf(zn, du1, u1), fmaf(zn, du2, u2), pol, cc);
                        if (phin <= 0.f) {
                            float lo = z, hi = zn;
                            const float eps = S.h * (1.f / 65536.f);
                            for (int q = 0; q < kBisectMax && hi - lo > eps; ++q) {
                                const float mid = 0.5f * (lo + hi);
                                const float pm = column_phi_in(S, fmaf(mid, du0, u0), fmaf(mid, du1, u1),
                                                               fmaf(mid, du2, u2), pol, cc);
                                if (pm <= 0.f) hi = mid; else lo = mid;
                            }
                            zhit = hi;
                            break;
                        }
                        if (zn >= zhi) break;
                        z = zn;
                        phi = phin;
                    }
                }
            }
            depth[k] = cam.d0 - ((zhit < 0.f) ? -zhit : 0.f);
        }
    }
}

}  // namespace tacsl

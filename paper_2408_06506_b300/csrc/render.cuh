// Depth-map rendering for the tactile image (Sec. III-B of arXiv 2408.06506: a camera
// at the optical location inside the sensor renders the depth of the indenting object).
//
// Camera reading: orthographic, looking along the pad normal.  Pixel (i, j) sees the
// pad-frame column (x0 + i*pitch_x, y0 + j*pitch_y, z); the undeformed gel at z = 0 reads
// d0; where the object reaches below the gel, the camera sees the object's first point
// on the column: D = d0 - max(0, -z_hit), z_hit searched over [-z_max, 0] from below.
//
// March: conservative sphere tracing up the column - step kappa*phi inside the grid
// domain (kappa = 1/sqrt 3: the trilinear interpolant of a 1-Lipschitz field is at most
// sqrt 3-Lipschitz, so a step cannot pass the surface), the exact distance to the
// domain box outside it, never less than voxel/8 - then bisection of the first bracket
// down to voxel * 2^-16; z_hit is the bracket's upper end.  The current trilinear cell
// and its 8 nodes stay in registers while samples remain in it.  phi is the 8-node cell value of the
// force-field path (phi_cell8), so image and force field see the same SDF.  Outside the
// grid's domain the SDF is undefined (as for the force field), so a point there is never
// inside the object; the distance to the domain box only sizes the step.
//
// One thread per column: a warp takes 32 neighbouring columns of a row, whose marches
// take similar paths and whose SDF reads fall on neighbouring nodes.
#pragma once

#include "common.cuh"
#include "taxel.cuh"

namespace tacsl {

constexpr int kMarchMax = 1024;   // safety cap on march steps (never reached in practice)
constexpr int kBisectMax = 40;    // bisection stops at a bracket <= voxel * 2^-16 (~13 halvings)

// The trilinear cell of the last sample and its 8 node values: successive samples of a
// column (small steps, bisection) mostly stay in one cell, so its nodes are read once.
// The value is computed exactly as phi_cell8 computes it (same nodes, same FMA order).
struct CellCache {
    int ix = -1, iy = -1, iz = -1;
    float v[2][2][2];
};

__device__ __forceinline__ float phi_cell8_cached(const DevSdf& S, const GridPos& g, uint64_t pol, CellCache& cc) {
    const int ix = min(static_cast<int>(floorf(g.ux)), S.n0 - 2);
    const int iy = min(static_cast<int>(floorf(g.uy)), S.n1 - 2);
    const int iz = min(static_cast<int>(floorf(g.uz)), S.n2 - 2);
    if (ix != cc.ix || iy != cc.iy || iz != cc.iz) {
        const int n0 = S.n0, n01 = S.n0 * S.n1;
        const float* b = S.data + (static_cast<int64_t>(iz) * n01 + static_cast<int64_t>(iy) * n0 + ix);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 2; ++i) cc.v[k][j][i] = ldg_f_hint(b + k * n01 + j * n0 + i, pol);
        cc.ix = ix;
        cc.iy = iy;
        cc.iz = iz;
    }
    const float fx = g.ux - static_cast<float>(ix), fy = g.uy - static_cast<float>(iy),
                fz = g.uz - static_cast<float>(iz);
    float c[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float r0 = fmaf(fx, cc.v[k][0][1], (1.f - fx) * cc.v[k][0][0]);
        const float r1 = fmaf(fx, cc.v[k][1][1], (1.f - fx) * cc.v[k][1][0]);
        c[k] = fmaf(fy, r1, (1.f - fy) * r0);
    }
    return fmaf(fz, c[1], (1.f - fz) * c[0]);
}

struct CameraArgs {
    int H, W;
    float pitch_x, pitch_y, x0, y0, d0, z_max;
};

// phi the march sees at object-frame point (x, y, z): trilinear in the domain, else the
// distance to the domain box (inside_out reports which).  Outside the domain the SDF is
// undefined, so such a point is never inside the object: callers test inside && phi <= 0.
__device__ __forceinline__ float column_phi(const DevSdf& S, float x, float y, float z, uint64_t pol,
                                            bool& inside_out, CellCache& cc) {
    const GridPos g = grid_pos(S, x, y, z);
    inside_out = g.inside;
    if (g.inside) return phi_cell8_cached(S, g, pol, cc);
    const float lox = S.ox + 0.5f * S.h, hix = S.ox + (static_cast<float>(S.n0) - 1.5f) * S.h;
    const float loy = S.oy + 0.5f * S.h, hiy = S.oy + (static_cast<float>(S.n1) - 1.5f) * S.h;
    const float loz = S.oz + 0.5f * S.h, hiz = S.oz + (static_cast<float>(S.n2) - 1.5f) * S.h;
    const float ex = fmaxf(fmaxf(lox - x, x - hix), 0.f);
    const float ey = fmaxf(fmaxf(loy - y, y - hiy), 0.f);
    const float ez = fmaxf(fmaxf(loz - z, z - hiz), 0.f);
    return sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
}

// Grid: (32 x 8 pixel tiles of the image, images); each warp marches 32 neighbouring
// columns of one row, and every thread keeps its column across the images it takes.
__global__ void __launch_bounds__(256) render_kernel(const SdfTable tab, int64_t B, int P,
                                                     const int32_t* __restrict__ obj_id,
                                                     const float* __restrict__ pad_pose, const CameraArgs cam,
                                                     float* __restrict__ depth) {
    const int tiles_x = (cam.W + 31) / 32;
    const int tile_y = static_cast<int>(blockIdx.x) / tiles_x, tile_x = static_cast<int>(blockIdx.x) - tile_y * tiles_x;
    const int i = tile_x * 32 + static_cast<int>(threadIdx.x & 31), j = tile_y * 8 + static_cast<int>(threadIdx.x >> 5);
    if (i >= cam.W || j >= cam.H) return;
    const int64_t HW = static_cast<int64_t>(cam.H) * cam.W;
    const int pix = j * cam.W + i;
    const uint64_t pol = policy_evict_last();
    for (int64_t b = blockIdx.y; b < B; b += gridDim.y) {
        const int64_t k = b * HW + pix;
        const int id = __ldg(obj_id + static_cast<int>(b) / P);
        if (id < 0 || id >= tab.count) {
            depth[k] = __int_as_float(0x7fc00000);
            raise_dev_error(TACSL_DEVERR_BAD_OBJ_ID);
            continue;
        }
        const DevSdf& S = tab.s[id];
        const float* pose = pad_pose + b * 7;
        float r[9];
        quat_to_rot(__ldg(pose + 3), __ldg(pose + 4), __ldg(pose + 5), __ldg(pose + 6), r);
        const float tx = __ldg(pose), ty = __ldg(pose + 1), tz = __ldg(pose + 2);
        const float px = fmaf(static_cast<float>(i), cam.pitch_x, cam.x0);
        const float py = fmaf(static_cast<float>(j), cam.pitch_y, cam.y0);
        // column point R (px, py, z) + t
        auto point = [&](float z, float& x, float& y, float& w) {
            x = fmaf(r[0], px, fmaf(r[1], py, fmaf(r[2], z, tx)));
            y = fmaf(r[3], px, fmaf(r[4], py, fmaf(r[5], z, ty)));
            w = fmaf(r[6], px, fmaf(r[7], py, fmaf(r[8], z, tz)));
        };
        const float dmin = S.h * 0.125f, kappa = 0.57735026918962576f;
        float x, y, w;
        bool in;
        float z = -cam.z_max;
        point(z, x, y, w);
        CellCache cc;
        float phi = column_phi(S, x, y, w, pol, in, cc);
        float zhit = 1.f;   // > 0: no hit
        if (in && phi <= 0.f) {
            zhit = z;
        } else {
            for (int it = 0; it < kMarchMax; ++it) {
                const float step = fmaxf(in ? kappa * phi : phi, dmin);
                const float zn = fminf(z + step, 0.f);
                point(zn, x, y, w);
                bool in_n;
                const float phin = column_phi(S, x, y, w, pol, in_n, cc);
                if (in_n && phin <= 0.f) {
                    float lo = z, hi = zn;
                    const float eps = S.h * (1.f / 65536.f);
                    for (int q = 0; q < kBisectMax && hi - lo > eps; ++q) {
                        const float mid = 0.5f * (lo + hi);
                        point(mid, x, y, w);
                        bool im;
                        const float pm = column_phi(S, x, y, w, pol, im, cc);
                        if (im && pm <= 0.f) hi = mid; else lo = mid;
                    }
                    zhit = hi;
                    break;
                }
                if (zn >= 0.f) break;
                z = zn;
                phi = phin;
                in = in_n;
            }
        }
        depth[k] = cam.d0 - ((zhit < 0.f) ? -zhit : 0.f);
    }
}

}  // namespace tacsl

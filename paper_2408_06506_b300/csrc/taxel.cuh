// Taxel-side kernels: SDF query with finite-difference gradient, penalty normal and
// friction-capped shear forces, per-pad wrench (Sec. III-C of arXiv 2408.06506).
//
// Interpolation reading: the grid's nodes are samples; between them the field is
// trilinear; the gradient is the central difference of that interpolant with step
// voxel/2 per axis.  All seven trilinear evaluations (centre and +-x, +-y, +-z) fall on
// a 3x3x3 node window, so one query gathers 27 nodes (nine rows of three along x)
// and folds them axis by axis with per-axis weight vectors: centre weights c[3] and
// difference weights d[3] = w(u + 1/2) - w(u - 1/2).
#pragma once

#include "common.cuh"

namespace tacsl {

// Per-axis weights over the node window {b, b+1, b+2}.  u is the continuous index,
// already known to lie in [0.5, n - 1.5].  Cells are min(floor(s), n - 2), as in the
// interpolation reading, so s = n - 1 uses the last cell with fraction 1.
__device__ __forceinline__ void axis_weights(float u, int n, int& b, float c[3], float d[3]) {
    const float sm = u - 0.5f, sp = u + 0.5f;   // exact for u < 2^22
    b = min(static_cast<int>(floorf(sm)), n - 3);
    float wm[3], wp[3];
    auto sample = [&](float s, float* w) {
        const int cell = min(static_cast<int>(floorf(s)), n - 2);
        const float f = s - static_cast<float>(cell);
        const bool r0 = (cell == b);
        w[0] = r0 ? 1.f - f : 0.f;
        w[1] = r0 ? f : 1.f - f;
        w[2] = r0 ? 0.f : f;
    };
    sample(sm, wm);
    sample(u, c);
    sample(sp, wp);
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = wp[k] - wm[k];
}

// SDF value and gradient at object-frame point (x, y, z).  Returns false outside the
// grid's domain (then phi = +inf, g = 0).
__device__ __forceinline__ bool sdf_stencil(const DevSdf& S, float x, float y, float z, float& phi,
                                            float g[3]) {
    const float ux = (x - S.ox) * S.inv_h, uy = (y - S.oy) * S.inv_h, uz = (z - S.oz) * S.inv_h;
    const bool inside = ux >= 0.5f && ux <= static_cast<float>(S.n0) - 1.5f && uy >= 0.5f &&
                        uy <= static_cast<float>(S.n1) - 1.5f && uz >= 0.5f &&
                        uz <= static_cast<float>(S.n2) - 1.5f;
    if (!inside) {
        phi = __int_as_float(0x7f800000);
        g[0] = g[1] = g[2] = 0.f;
        return false;
    }
    int bx, by, bz;
    float cx[3], dx[3], cy[3], dy[3], cz[3], dz[3];
    axis_weights(ux, S.n0, bx, cx, dx);
    axis_weights(uy, S.n1, by, cy, dy);
    axis_weights(uz, S.n2, bz, cz, dz);
    const int n0 = S.n0, n01 = S.n0 * S.n1;
    const float* __restrict__ base = S.data + (static_cast<int64_t>(bz) * n01 + static_cast<int64_t>(by) * n0 + bx);
    float v[3][3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) v[k][j][i] = __ldg(base + k * n01 + j * n0 + i);
    // fold x: rows -> centre value and x-difference per (k, j)
    float rc[3][3], rd[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rc[k][j] = fmaf(cx[2], v[k][j][2], fmaf(cx[1], v[k][j][1], cx[0] * v[k][j][0]));
            rd[k][j] = fmaf(dx[2], v[k][j][2], fmaf(dx[1], v[k][j][1], dx[0] * v[k][j][0]));
        }
    // fold y
    float cc[3], cd[3], xd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cc[k] = fmaf(cy[2], rc[k][2], fmaf(cy[1], rc[k][1], cy[0] * rc[k][0]));
        cd[k] = fmaf(dy[2], rc[k][2], fmaf(dy[1], rc[k][1], dy[0] * rc[k][0]));
        xd[k] = fmaf(cy[2], rd[k][2], fmaf(cy[1], rd[k][1], cy[0] * rd[k][0]));
    }
    // fold z
    phi = fmaf(cz[2], cc[2], fmaf(cz[1], cc[1], cz[0] * cc[0]));
    g[0] = fmaf(cz[2], xd[2], fmaf(cz[1], xd[1], cz[0] * xd[0])) * S.inv_h;
    g[1] = fmaf(cz[2], cd[2], fmaf(cz[1], cd[1], cz[0] * cd[0])) * S.inv_h;
    g[2] = fmaf(dz[2], cc[2], fmaf(dz[1], cc[1], dz[0] * cc[0])) * S.inv_h;
    return true;
}

// One taxel: pose, query, penalty normal force, friction-capped shear (object frame),
// then both forces rotated into the pad frame.
__device__ __forceinline__ void taxel_force(const DevSdf& S, const Pose& P, float px, float py, float pz,
                                            float kn, float kd, float kt, float mu, float& depth,
                                            float fn_pad[3], float ft_pad[3]) {
    const float* r = P.r;
    const float xo = fmaf(r[0], px, fmaf(r[1], py, fmaf(r[2], pz, P.t[0])));
    const float yo = fmaf(r[3], px, fmaf(r[4], py, fmaf(r[5], pz, P.t[1])));
    const float zo = fmaf(r[6], px, fmaf(r[7], py, fmaf(r[8], pz, P.t[2])));
    // relative velocity of the point: v + w x x
    const float vx = P.v[0] + (P.w[1] * zo - P.w[2] * yo);
    const float vy = P.v[1] + (P.w[2] * xo - P.w[0] * zo);
    const float vz = P.v[2] + (P.w[0] * yo - P.w[1] * xo);

    float phi, g[3];
    sdf_stencil(S, xo, yo, zo, phi, g);
    float fn[3] = {0.f, 0.f, 0.f}, ft[3] = {0.f, 0.f, 0.f};
    depth = 0.f;
    if (phi < 0.f) {
        depth = -phi;
        const float gn2 = fmaf(g[0], g[0], fmaf(g[1], g[1], g[2] * g[2]));
        if (gn2 >= 1e-24f) {
            const float inv = rsqrtf(gn2);
            const float nx = g[0] * inv, ny = g[1] * inv, nz = g[2] * inv;
            const float ddot = fmaf(nx, vx, fmaf(ny, vy, nz * vz));       // d' = n . x'
            const float mag = fmaxf(fmaf(kd, ddot, -kn) * phi, 0.f);      // (-k_n + k_d d') d, clamped
            fn[0] = mag * nx; fn[1] = mag * ny; fn[2] = mag * nz;
            const float tx = fmaf(-ddot, nx, vx), ty = fmaf(-ddot, ny, vy), tz = fmaf(-ddot, nz, vz);
            const float vt2 = fmaf(tx, tx, fmaf(ty, ty, tz * tz));
            if (vt2 > 0.f) {
                const float vtn = sqrtf(vt2);
                const float ftm = fminf(kt * vtn, mu * mag);
                const float sc = -ftm / vtn;
                ft[0] = sc * tx; ft[1] = sc * ty; ft[2] = sc * tz;
            }
        }
    }
    // pad frame: R^T f
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        fn_pad[a] = fmaf(r[a], fn[0], fmaf(r[3 + a], fn[1], r[6 + a] * fn[2]));
        ft_pad[a] = fmaf(r[a], ft[0], fmaf(r[3 + a], ft[1], r[6 + a] * ft[2]));
    }
}

// All taxels of pad b by the whole block (NWARPS warps), plus its wrench.
template <int NWARPS>
__device__ __forceinline__ void process_pad(const SdfTable& tab, const Params4& prm, int P, int T,
                                            const float* __restrict__ taxels, const int32_t* __restrict__ obj_id,
                                            const float* __restrict__ pad_pose, const float* __restrict__ pad_twist,
                                            float* __restrict__ depth, float* __restrict__ f_n,
                                            float* __restrict__ f_t, float* __restrict__ wrench, int64_t b,
                                            float* red_scratch) {
    constexpr int NT = NWARPS * 32;
    const int64_t e = b / P;
    const int id = __ldg(obj_id + e);
    const int64_t o = b * T;
    if (id < 0 || id >= tab.count) {
        const float qnan = __int_as_float(0x7fc00000);
        for (int t = threadIdx.x; t < T; t += NT) {
            depth[o + t] = qnan;
#pragma unroll
            for (int a = 0; a < 3; ++a) { f_n[(o + t) * 3 + a] = qnan; f_t[(o + t) * 3 + a] = qnan; }
        }
        if (wrench != nullptr && threadIdx.x < 6) wrench[b * 6 + threadIdx.x] = qnan;
        if (threadIdx.x == 0) raise_dev_error(TACSL_DEVERR_BAD_OBJ_ID);
        return;   // uniform across the block
    }
    const DevSdf& S = tab.s[id];
    Pose Pz;
    load_pose(pad_pose + b * 7, pad_twist + b * 6, Pz);
    const int pi = prm.count == 1 ? 0 : static_cast<int>(e);
    const float kn = __ldg(prm.k_n + pi), kd = __ldg(prm.k_d + pi), kt = __ldg(prm.k_t + pi),
                mu = __ldg(prm.mu + pi);
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int t = threadIdx.x; t < T; t += NT) {
        const float px = __ldg(taxels + 3 * t), py = __ldg(taxels + 3 * t + 1), pz = __ldg(taxels + 3 * t + 2);
        float dep, fn[3], ft[3];
        taxel_force(S, Pz, px, py, pz, kn, kd, kt, mu, dep, fn, ft);
        depth[o + t] = dep;
#pragma unroll
        for (int a = 0; a < 3; ++a) { f_n[(o + t) * 3 + a] = fn[a]; f_t[(o + t) * 3 + a] = ft[a]; }
        const float fx = fn[0] + ft[0], fy = fn[1] + ft[1], fz = fn[2] + ft[2];
        acc[0] += fx; acc[1] += fy; acc[2] += fz;
        acc[3] += py * fz - pz * fy;
        acc[4] += pz * fx - px * fz;
        acc[5] += px * fy - py * fx;
    }
    if (wrench != nullptr) {
        block_sum6<NWARPS>(acc, red_scratch);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) wrench[b * 6 + k] = acc[k];
        }
        __syncthreads();   // scratch reuse by the next pad
    }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) sdf_query_kernel(const SdfTable tab, int64_t n, const float* __restrict__ pts,
                                                        const int32_t* __restrict__ obj_id, float* __restrict__ phi,
                                                        float* __restrict__ grad) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int id = __ldg(obj_id + i);
        float p, g[3];
        if (id < 0 || id >= tab.count) {
            p = g[0] = g[1] = g[2] = __int_as_float(0x7fc00000);
            raise_dev_error(TACSL_DEVERR_BAD_OBJ_ID);
        } else {
            sdf_stencil(tab.s[id], __ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2), p, g);
        }
        phi[i] = p;
        grad[3 * i] = g[0];
        grad[3 * i + 1] = g[1];
        grad[3 * i + 2] = g[2];
    }
}

template <int NWARPS>
__global__ void __launch_bounds__(NWARPS * 32) penalty_kernel(const SdfTable tab, const Params4 prm, int64_t B, int P,
                                                              int T, const float* __restrict__ taxels,
                                                              const int32_t* __restrict__ obj_id,
                                                              const float* __restrict__ pad_pose,
                                                              const float* __restrict__ pad_twist,
                                                              float* __restrict__ depth, float* __restrict__ f_n,
                                                              float* __restrict__ f_t, float* __restrict__ wrench) {
    __shared__ float red[NWARPS * 6];
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x)
        process_pad<NWARPS>(tab, prm, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t, wrench, b, red);
}

template <int NWARPS>
__global__ void __launch_bounds__(NWARPS * 32) wrench_kernel(int64_t B, int T, const float* __restrict__ taxels,
                                                             const float* __restrict__ f_n,
                                                             const float* __restrict__ f_t,
                                                             float* __restrict__ wrench) {
    constexpr int NT = NWARPS * 32;
    __shared__ float red[NWARPS * 6];
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        const int64_t o = b * T;
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int t = threadIdx.x; t < T; t += NT) {
            const float px = __ldg(taxels + 3 * t), py = __ldg(taxels + 3 * t + 1), pz = __ldg(taxels + 3 * t + 2);
            const float fx = __ldg(f_n + (o + t) * 3) + __ldg(f_t + (o + t) * 3);
            const float fy = __ldg(f_n + (o + t) * 3 + 1) + __ldg(f_t + (o + t) * 3 + 1);
            const float fz = __ldg(f_n + (o + t) * 3 + 2) + __ldg(f_t + (o + t) * 3 + 2);
            acc[0] += fx; acc[1] += fy; acc[2] += fz;
            acc[3] += py * fz - pz * fy;
            acc[4] += pz * fx - px * fz;
            acc[5] += px * fy - py * fx;
        }
        block_sum6<NWARPS>(acc, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) wrench[b * 6 + k] = acc[k];
        }
        __syncthreads();
    }
}

}  // namespace tacsl

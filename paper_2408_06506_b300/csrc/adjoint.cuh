// Hand-written adjoints of the tactile step, for calibrating the sensor and contact
// models from observed force fields and images (the use the paper makes of measured
// contact stiffness, App. B, and of a calibrated image model, Sec. III-B).
//
// Force field (Sec. III-C).  For an upstream gradient of the depth, normal and shear
// force fields and of the per-pad wrench, the kernel returns the gradient w.r.t. each
// pad's pose (t, q), twist (v, w) and the contact parameters (k_n, k_d, k_t, mu).  It
// recomputes the forward values in the same float32 operations as the force kernel
// (so contact, clamp and stick/slip decisions match it) and runs the chain rule back:
//   f_pad = R^T f            -> dR, df
//   f_t = -(v_t/|v_t|) min(k_t |v_t|, mu |f_n|),  f_n = max((-k_n + k_d d') phi, 0) n,
//   v_t = x' - d' n,  d' = n . x',  n = g/|g|      -> dx', dphi, dg, parameters
//   phi(x), g(x): trilinear interpolant and its h/2 central difference; their
//     derivatives come from the same 27-node window folded with the derivative weights
//     of each axis (a sample's weights are (1-f, f) on its cell, so d/du is (-1, 1))
//   x' = v + w x x,  x = R p + t                   -> dt, dR, dv, dw
//   R = R(q/|q|)                                     -> dq (tangent to the unit sphere, / |q|)
// A taxel contributes only where it penetrates (phi < 0); elsewhere its outputs are
// constant zero.  One warp per env walks its P pads; lanes take taxels; pose / twist
// gradients are reduced per pad with shuffles, parameter gradients per env.
//
// Image (Sec. III-B).  The differentiable image is the clamped intensity
// clamp(sum_k A_k m_k(n), 0, 255) (the quantity the uint8 image rounds).  Its forward
// kernel writes float intensities; the adjoint returns the gradient w.r.t. the per-pixel
// coefficients (summed over the images of each sensor) and w.r.t. the depth maps (the
// transpose of the central / one-sided difference stencil of the normals).
#pragma once

#include "common.cuh"
#include "taxel.cuh"
#include "shade.cuh"

namespace tacsl {

// Derivative weights of one axis: for the centre sample (dc) and for the difference
// d = w(u + 1/2) - w(u - 1/2) (dd); a sample on the window's first cell has weights
// (1-f, f, 0), on the second (0, 1-f, f), so d/du of them is (-1, 1, 0) or (0, -1, 1).
__device__ __forceinline__ void axis_dweights(float u, int n, int b, float dc[3], float dd[3]) {
    auto dsample = [&](float s, float* w) {
        const int cell = min(static_cast<int>(floorf(s)), n - 2);
        const bool r0 = (cell == b);
        w[0] = r0 ? -1.f : 0.f;
        w[1] = r0 ? 1.f : -1.f;
        w[2] = r0 ? 0.f : 1.f;
    };
    float wm[3], wp[3];
    dsample(u - 0.5f, wm);
    dsample(u, dc);
    dsample(u + 0.5f, wp);
#pragma unroll
    for (int k = 0; k < 3; ++k) dd[k] = wp[k] - wm[k];
}

__device__ __forceinline__ float dot3w(const float* w, float a, float b, float c) {
    return fmaf(w[2], c, fmaf(w[1], b, w[0] * a));
}

// SDF sample of a penetrating taxel with derivatives, in continuous-index units:
// phi, g (per metre, as the force kernel), dphi[b] = d phi / d u_b and
// J[a][b] = d g_a / d u_b.
struct SdfJet {
    float phi, g[3], dphi[3], J[3][3];
};

__device__ __forceinline__ void sdf_jet(const DevSdf& S, const GridPos& gp, uint64_t pol, SdfJet& o) {
    Stencil q;
    q.inside = true;
    int bx, by, bz;
    axis_weights(gp.ux, S.n0, bx, q.cx, q.dx);
    axis_weights(gp.uy, S.n1, by, q.cy, q.dy);
    axis_weights(gp.uz, S.n2, bz, q.cz, q.dz);
    const int n0 = S.n0, n01 = S.n0 * S.n1;
    q.base = S.data + (static_cast<int64_t>(bz) * n01 + static_cast<int64_t>(by) * n0 + bx);
    float v[3][3][3];
    stencil_load(q, n0, n01, pol, v);
    stencil_fold(q, v, S.inv_h, o.phi, o.g);     // bitwise the force kernel's phi and g
    float ecx[3], edx[3], ecy[3], edy[3], ecz[3], edz[3];
    axis_dweights(gp.ux, S.n0, bx, ecx, edx);
    axis_dweights(gp.uy, S.n1, by, ecy, edy);
    axis_dweights(gp.uz, S.n2, bz, ecz, edz);
    // x stage: rows of the window folded along x with c, c', d, d'
    float rc[3][3], rdc[3][3], rd[3][3], rdd[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rc[k][j] = dot3w(q.cx, v[k][j][0], v[k][j][1], v[k][j][2]);
            rdc[k][j] = dot3w(ecx, v[k][j][0], v[k][j][1], v[k][j][2]);
            rd[k][j] = dot3w(q.dx, v[k][j][0], v[k][j][1], v[k][j][2]);
            rdd[k][j] = dot3w(edx, v[k][j][0], v[k][j][1], v[k][j][2]);
        }
    // y stage: the (x, y) weight pairs the sixteen (x, y, z) triples need
    float cc[3], cdc[3], cd[3], cdd[3], dcc[3], dcd[3], dc_[3], ddc[3], ddd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cc[k] = dot3w(q.cy, rc[k][0], rc[k][1], rc[k][2]);      // (c, c)
        cdc[k] = dot3w(ecy, rc[k][0], rc[k][1], rc[k][2]);      // (c, c')
        cd[k] = dot3w(q.dy, rc[k][0], rc[k][1], rc[k][2]);      // (c, d)
        cdd[k] = dot3w(edy, rc[k][0], rc[k][1], rc[k][2]);      // (c, d')
        dcc[k] = dot3w(q.cy, rdc[k][0], rdc[k][1], rdc[k][2]);  // (c', c)
        dcd[k] = dot3w(q.dy, rdc[k][0], rdc[k][1], rdc[k][2]);  // (c', d)
        dc_[k] = dot3w(q.cy, rd[k][0], rd[k][1], rd[k][2]);     // (d, c)
        ddc[k] = dot3w(ecy, rd[k][0], rd[k][1], rd[k][2]);      // (d, c')
        ddd[k] = dot3w(q.cy, rdd[k][0], rdd[k][1], rdd[k][2]);  // (d', c)
    }
    // z stage
    o.dphi[0] = dot3w(q.cz, dcc[0], dcc[1], dcc[2]);
    o.dphi[1] = dot3w(q.cz, cdc[0], cdc[1], cdc[2]);
    o.dphi[2] = dot3w(ecz, cc[0], cc[1], cc[2]);
    const float ih = S.inv_h;
    o.J[0][0] = dot3w(q.cz, ddd[0], ddd[1], ddd[2]) * ih;
    o.J[0][1] = dot3w(q.cz, ddc[0], ddc[1], ddc[2]) * ih;
    o.J[0][2] = dot3w(ecz, dc_[0], dc_[1], dc_[2]) * ih;
    o.J[1][0] = dot3w(q.cz, dcd[0], dcd[1], dcd[2]) * ih;
    o.J[1][1] = dot3w(q.cz, cdd[0], cdd[1], cdd[2]) * ih;
    o.J[1][2] = dot3w(ecz, cd[0], cd[1], cd[2]) * ih;
    o.J[2][0] = dot3w(q.dz, dcc[0], dcc[1], dcc[2]) * ih;
    o.J[2][1] = dot3w(q.dz, cdc[0], cdc[1], cdc[2]) * ih;
    o.J[2][2] = dot3w(edz, cc[0], cc[1], cc[2]) * ih;
}

struct ForceAdjointArgs {
    SdfTable tab;
    Params4 prm;
    int64_t E;
    int P, T;
    const float* taxels;
    const int32_t* obj_id;
    const float* pose;
    const float* twist;
    const float* g_depth;   // [B][T] or NULL
    const float* g_fn;      // [B][T][3] or NULL
    const float* g_ft;      // [B][T][3] or NULL
    const float* g_wrench;  // [B][6] or NULL
    float* grad_pose;       // [B][7] or NULL
    float* grad_twist;      // [B][6] or NULL
    float* grad_params;     // [count][4] or NULL
};

__device__ __forceinline__ float ld_or0(const float* p, int64_t i) { return p != nullptr ? __ldg(p + i) : 0.f; }

// Gradient of R(q/|q|) (row-major r) w.r.t. q, given dL/dR in gR.
__device__ __forceinline__ void quat_backward(const float* q4, const float* gR, float gq[4]) {
    const float s = rsqrtf(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
    const float w = q4[0] * s, x = q4[1] * s, y = q4[2] * s, z = q4[3] * s;
    // dL/dq_hat from the partial derivatives of each entry of R
    float gw = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    float gx = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] -
                      2.f * x * gR[8]);
    float gy = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] -
                      2.f * y * gR[8]);
    float gz = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] +
                      x * gR[6] + y * gR[7]);
    // through the normalisation: (I - q_hat q_hat^T) / |q|
    const float proj = w * gw + x * gx + y * gy + z * gz;
    gq[0] = (gw - w * proj) * s;
    gq[1] = (gx - x * proj) * s;
    gq[2] = (gy - y * proj) * s;
    gq[3] = (gz - z * proj) * s;
}

// acc layout: 0-2 t, 3-11 R (row-major), 12-14 v, 15-17 w, 18-21 k_n, k_d, k_t, mu
constexpr int kAdjAcc = 22;

__device__ __forceinline__ void taxel_adjoint(const DevSdf& S, const Pose& Pz, float kn, float kd, float kt, float mu,
                                              const float p[3], const float gfp[3], const float gtp[3], float gdep,
                                              uint64_t pol, float (&acc)[kAdjAcc]) {
    const float* r = Pz.r;
    const float x0 = fmaf(r[0], p[0], fmaf(r[1], p[1], fmaf(r[2], p[2], Pz.t[0])));
    const float x1 = fmaf(r[3], p[0], fmaf(r[4], p[1], fmaf(r[5], p[2], Pz.t[1])));
    const float x2 = fmaf(r[6], p[0], fmaf(r[7], p[1], fmaf(r[8], p[2], Pz.t[2])));
    const float xd[3] = {Pz.v[0] + (Pz.w[1] * x2 - Pz.w[2] * x1), Pz.v[1] + (Pz.w[2] * x0 - Pz.w[0] * x2),
                         Pz.v[2] + (Pz.w[0] * x1 - Pz.w[1] * x0)};
    const GridPos gp = grid_pos(S, x0, x1, x2);
    if (!gp.inside) return;
    if (!(phi_cell8(S, gp, pol) < 0.f)) return;         // no contact: constant zero outputs
    SdfJet jt;
    sdf_jet(S, gp, pol, jt);
    const float phi = jt.phi;
    float g_phi = -gdep;                                 // depth = -phi
    float g_g[3] = {0.f, 0.f, 0.f}, g_xd[3] = {0.f, 0.f, 0.f};
    const float gn2 = fmaf(jt.g[0], jt.g[0], fmaf(jt.g[1], jt.g[1], jt.g[2] * jt.g[2]));
    if (gn2 >= 1e-24f) {
        // forward, as contact_force
        const float inv = rsqrtf(gn2);
        const float n[3] = {jt.g[0] * inv, jt.g[1] * inv, jt.g[2] * inv};
        const float ddot = fmaf(n[0], xd[0], fmaf(n[1], xd[1], n[2] * xd[2]));
        const float craw = fmaf(kd, ddot, -kn);
        const float mraw = craw * phi;
        const float mag = fmaxf(mraw, 0.f);
        const float tv[3] = {fmaf(-ddot, n[0], xd[0]), fmaf(-ddot, n[1], xd[1]), fmaf(-ddot, n[2], xd[2])};
        const float vt2 = fmaf(tv[0], tv[0], fmaf(tv[1], tv[1], tv[2] * tv[2]));
        float fn[3], ft[3] = {0.f, 0.f, 0.f};
        fn[0] = mag * n[0]; fn[1] = mag * n[1]; fn[2] = mag * n[2];
        float s = 0.f, cap = 0.f, lim = 0.f, ftm = 0.f, sc = 0.f;
        if (vt2 > 0.f) {
            s = sqrtf(vt2);
            cap = kt * s;
            lim = mu * mag;
            ftm = fminf(cap, lim);
            sc = -ftm / s;
            ft[0] = sc * tv[0]; ft[1] = sc * tv[1]; ft[2] = sc * tv[2];
        }
        // upstream in the object frame (f_pad = R^T f  =>  df = R df_pad) and dR from it
        float gfn[3], gft[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gfn[a] = fmaf(r[3 * a], gfp[0], fmaf(r[3 * a + 1], gfp[1], r[3 * a + 2] * gfp[2]));
            gft[a] = fmaf(r[3 * a], gtp[0], fmaf(r[3 * a + 1], gtp[1], r[3 * a + 2] * gtp[2]));
        }
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[3 + 3 * j + a] += fmaf(fn[j], gfp[a], ft[j] * gtp[a]);
        float g_n[3] = {0.f, 0.f, 0.f}, g_tv[3] = {0.f, 0.f, 0.f}, g_mag = 0.f, g_ddot = 0.f;
        if (vt2 > 0.f) {
            // f_t = sc tv, sc = -ftm / s, ftm = min(k_t s, mu mag)
            const float g_sc = fmaf(tv[0], gft[0], fmaf(tv[1], gft[1], tv[2] * gft[2]));
#pragma unroll
            for (int a = 0; a < 3; ++a) g_tv[a] = sc * gft[a];
            const float g_ftm = -g_sc / s;
            float g_s = ftm * g_sc / (s * s);
            if (cap <= lim) {                  // stick (fminf takes cap)
                acc[20] += s * g_ftm;
                g_s += kt * g_ftm;
            } else {                           // slip
                acc[21] += mag * g_ftm;
                g_mag += mu * g_ftm;
            }
            const float k = g_s / s;
#pragma unroll
            for (int a = 0; a < 3; ++a) g_tv[a] = fmaf(k, tv[a], g_tv[a]);
            // tv = x' - ddot n
#pragma unroll
            for (int a = 0; a < 3; ++a) g_xd[a] += g_tv[a];
            g_ddot -= fmaf(n[0], g_tv[0], fmaf(n[1], g_tv[1], n[2] * g_tv[2]));
#pragma unroll
            for (int a = 0; a < 3; ++a) g_n[a] -= ddot * g_tv[a];
        }
        // f_n = mag n
        g_mag += fmaf(n[0], gfn[0], fmaf(n[1], gfn[1], n[2] * gfn[2]));
#pragma unroll
        for (int a = 0; a < 3; ++a) g_n[a] = fmaf(mag, gfn[a], g_n[a]);
        // mag = max(craw phi, 0), craw = k_d ddot - k_n
        if (mraw > 0.f) {
            const float g_c = phi * g_mag;
            g_phi = fmaf(craw, g_mag, g_phi);
            acc[18] -= g_c;
            acc[19] += ddot * g_c;
            g_ddot = fmaf(kd, g_c, g_ddot);
        }
        // ddot = n . x'
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g_n[a] = fmaf(xd[a], g_ddot, g_n[a]);
            g_xd[a] = fmaf(n[a], g_ddot, g_xd[a]);
        }
        // n = g / |g|
        const float pn = fmaf(n[0], g_n[0], fmaf(n[1], g_n[1], n[2] * g_n[2]));
#pragma unroll
        for (int a = 0; a < 3; ++a) g_g[a] = (g_n[a] - n[a] * pn) * inv;
    }
    // phi(x), g(x): d/dx = (1/h) d/du
    float g_x[3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
        g_x[b] = fmaf(jt.dphi[b], g_phi, fmaf(jt.J[0][b], g_g[0], fmaf(jt.J[1][b], g_g[1], jt.J[2][b] * g_g[2]))) *
                 S.inv_h;
    // x' = v + w x x
    const float xs[3] = {x0, x1, x2};
    acc[12] += g_xd[0]; acc[13] += g_xd[1]; acc[14] += g_xd[2];
    acc[15] += xs[1] * g_xd[2] - xs[2] * g_xd[1];
    acc[16] += xs[2] * g_xd[0] - xs[0] * g_xd[2];
    acc[17] += xs[0] * g_xd[1] - xs[1] * g_xd[0];
    g_x[0] += g_xd[1] * Pz.w[2] - g_xd[2] * Pz.w[1];
    g_x[1] += g_xd[2] * Pz.w[0] - g_xd[0] * Pz.w[2];
    g_x[2] += g_xd[0] * Pz.w[1] - g_xd[1] * Pz.w[0];
    // x = R p + t
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] += g_x[a];
#pragma unroll
        for (int j = 0; j < 3; ++j) acc[3 + 3 * a + j] = fmaf(g_x[a], p[j], acc[3 + 3 * a + j]);
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// One warp per env; 8 envs per 256-thread CTA; grid-stride over envs.
__global__ void __launch_bounds__(256) force_adjoint_kernel(const ForceAdjointArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * 8;
    const uint64_t pol = policy_evict_last();
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); e < A.E; e += nwarps) {
        const int id = __ldg(A.obj_id + e);
        const int pi = A.prm.count == 1 ? 0 : static_cast<int>(e);
        if (id < 0 || id >= A.tab.count) {
            const float qnan = __int_as_float(0x7fc00000);
            for (int p = 0; p < A.P; ++p) {
                const int64_t b = e * A.P + p;
                if (A.grad_pose != nullptr && lane < 7) A.grad_pose[b * 7 + lane] = qnan;
                if (A.grad_twist != nullptr && lane < 6) A.grad_twist[b * 6 + lane] = qnan;
            }
            if (A.grad_params != nullptr && lane < 4) {
                if (A.prm.count == 1) atomicAdd(A.grad_params + lane, qnan);
                else A.grad_params[static_cast<int64_t>(pi) * 4 + lane] = qnan;
            }
            if (lane == 0) raise_dev_error(TACSL_DEVERR_BAD_OBJ_ID);
            continue;
        }
        const DevSdf& S = A.tab.s[id];
        const float kn = __ldg(A.prm.k_n + pi), kd = __ldg(A.prm.k_d + pi), kt = __ldg(A.prm.k_t + pi),
                    mu = __ldg(A.prm.mu + pi);
        float kacc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int p = 0; p < A.P; ++p) {
            const int64_t b = e * A.P + p;
            Pose Pz;
            load_pose(A.pose + b * 7, A.twist + b * 6, Pz);
            float gW[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) gW[k] = ld_or0(A.g_wrench, b * 6 + k);
            float acc[kAdjAcc];
#pragma unroll
            for (int k = 0; k < kAdjAcc; ++k) acc[k] = 0.f;
            const int64_t o = b * A.T;
            for (int t = lane; t < A.T; t += 32) {
                const float pt[3] = {__ldg(A.taxels + 3 * t), __ldg(A.taxels + 3 * t + 1), __ldg(A.taxels + 3 * t + 2)};
                // wrench = (sum f, sum p x f): dL/df_i += g_F + g_tau x p_i, for f_n and f_t alike
                const float gwx = gW[0] + (gW[4] * pt[2] - gW[5] * pt[1]);
                const float gwy = gW[1] + (gW[5] * pt[0] - gW[3] * pt[2]);
                const float gwz = gW[2] + (gW[3] * pt[1] - gW[4] * pt[0]);
                const float gfp[3] = {ld_or0(A.g_fn, (o + t) * 3) + gwx, ld_or0(A.g_fn, (o + t) * 3 + 1) + gwy,
                                      ld_or0(A.g_fn, (o + t) * 3 + 2) + gwz};
                const float gtp[3] = {ld_or0(A.g_ft, (o + t) * 3) + gwx, ld_or0(A.g_ft, (o + t) * 3 + 1) + gwy,
                                      ld_or0(A.g_ft, (o + t) * 3 + 2) + gwz};
                taxel_adjoint(S, Pz, kn, kd, kt, mu, pt, gfp, gtp, ld_or0(A.g_depth, o + t), pol, acc);
            }
#pragma unroll
            for (int k = 0; k < kAdjAcc; ++k) acc[k] = warp_sum(acc[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) kacc[k] += acc[18 + k];
            if (lane == 0) {
                if (A.grad_pose != nullptr) {
                    const float q4[4] = {__ldg(A.pose + b * 7 + 3), __ldg(A.pose + b * 7 + 4), __ldg(A.pose + b * 7 + 5),
                                         __ldg(A.pose + b * 7 + 6)};
                    float gq[4];
                    quat_backward(q4, acc + 3, gq);
                    float* gp = A.grad_pose + b * 7;
                    gp[0] = acc[0]; gp[1] = acc[1]; gp[2] = acc[2];
                    gp[3] = gq[0]; gp[4] = gq[1]; gp[5] = gq[2]; gp[6] = gq[3];
                }
                if (A.grad_twist != nullptr) {
                    float* gt = A.grad_twist + b * 6;
#pragma unroll
                    for (int k = 0; k < 6; ++k) gt[k] = acc[12 + k];
                }
            }
        }
        if (A.grad_params != nullptr && lane == 0) {
            if (A.prm.count == 1) {
#pragma unroll
                for (int k = 0; k < 4; ++k) atomicAdd(A.grad_params + k, kacc[k]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) A.grad_params[static_cast<int64_t>(pi) * 4 + k] = kacc[k];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Image: clamped intensity and its adjoint
// ---------------------------------------------------------------------------

struct ShadeGeom {
    int H, W, S;
    int64_t HW;
    float px, py;   // pixel pitch
};

// Depth derivative of image D along x at (x, y) and its stencil: D_x = cx_lo D[.. lo] +
// cx_hi D[.. hi] (central inside, one-sided on the border, zero on a 1-wide axis).
__device__ __forceinline__ void axis_stencil(int i, int len, float pitch, int& lo, int& hi, float& c) {
    if (len < 2) { lo = hi = i; c = 0.f; return; }
    if (i == 0) { lo = 0; hi = 1; c = 1.f / pitch; return; }
    if (i == len - 1) { lo = len - 2; hi = len - 1; c = 1.f / pitch; return; }
    lo = i - 1; hi = i + 1; c = 1.f / (2.f * pitch);
}

struct PixelState {
    float dx, dy, r, nx, ny;
};

__device__ __forceinline__ PixelState pixel_state(const float* D, const ShadeGeom& G, int x, int y) {
    int lo, hi;
    float cx, cy;
    axis_stencil(x, G.W, G.px, lo, hi, cx);
    PixelState s;
    s.dx = (__ldg(D + static_cast<int64_t>(y) * G.W + hi) - __ldg(D + static_cast<int64_t>(y) * G.W + lo)) * cx;
    axis_stencil(y, G.H, G.py, lo, hi, cy);
    s.dy = (__ldg(D + static_cast<int64_t>(hi) * G.W + x) - __ldg(D + static_cast<int64_t>(lo) * G.W + x)) * cy;
    s.r = rsqrtf(fmaf(s.dx, s.dx, fmaf(s.dy, s.dy, 1.f)));
    s.nx = s.dx * s.r;
    s.ny = s.dy * s.r;
    return s;
}

// Work split of the per-pixel image kernels (intensity and coefficient gradient): a CTA of
// 8 warps owns 64 consecutive pixels of one sensor's image plane (two per lane, so the
// per-pixel coefficients stay in registers) and a range of images; its warps take equal
// slices of that range.
constexpr int kImgWarps = 8;

// Per-lane asynchronous 4-byte copy global -> shared (completion per thread, by group).
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kCgStages = 6;     // images in flight per warp
constexpr int kCgSeg = 128;      // images of a warp's slice listed at a time

// Bad sensor ids of the intensity forward: flagged once per image.
__global__ void __launch_bounds__(256) flag_bad_sensors_kernel(int64_t B, int S, const int32_t* __restrict__ sensor_id) {
    for (int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; b < B;
         b += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int s = __ldg(sensor_id + b);
        if (s < 0 || s >= S) raise_dev_error(TACSL_DEVERR_BAD_SENSOR_ID);
    }
}

constexpr int kCgPx = 64;        // pixels per tile: two per lane
constexpr int kCgSlots = 7;      // 8-byte slots per lane and image
constexpr size_t kCgRingBytes = size_t(kImgWarps) * kCgStages * kCgSlots * 32 * sizeof(float2);
constexpr size_t kCgSmemBytes = kCgRingBytes + size_t(kImgWarps) * kCgSeg * sizeof(int);

__device__ __forceinline__ void cp_async8(float2* smem, const float* gmem) {
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}

// dL/dA[s][k][c][px] = sum over images b of sensor s of g[b][px][c] m_k(b, px) (where the
// clamp passes).  Grid (64-pixel tiles, sensors); a CTA of 8 warps owns the tile, two
// horizontally adjacent pixels per lane, so the per-pixel coefficients and sums stay in
// registers; each warp sums its slice of the images in order and the eight partial sums
// are added in warp order (deterministic).  kMse = false: g is read from u = dL/dI.
// kMse = true: u is the target intensity, g = w2 (I - u), and loss_map[s][px] (if not
// NULL) receives sum_b sum_c (clamp(I) - u)^2 in the same order; grad_coeffs may then be
// NULL.  The arithmetic runs on FP32 pairs (f32x2, lane-wise IEEE).
// Each lane's inputs per image are fetched kCgStages images ahead by per-lane cp.async
// copies into a shared-memory ring (the warp first lists its slice's images of sensor s,
// kCgSeg at a time): the centre depth pair, the pairs above and below, the six upstream
// values (three 8-byte copies when that array is 8-byte aligned, kU8, else six 4-byte
// ones) and, for lanes 0 and 31, the pixel beyond the warp's row segment; the other
// lanes' horizontal neighbours come by shuffle.  Against one pixel per lane (7 four-byte
// copies and scalar arithmetic per pixel and image, issue-bound): the same bits, 0.78 ->
// 0.68 ms for the adjoint and 0.80 -> 0.78 ms for the loss form on 2048 maps of 320x240;
// the registers (126-128) leave two CTAs per SM.
// kSlopes: the kernel also writes, for every image it visits, the pixel slopes
// slopes[b][px] = (dL/dD_x, dL/dD_y) of the pixel's own term of L with respect to the
// two depth differences its normal reads (the chain of the Sec. III-B shading model
// through the normal n = (D_x, D_y, 1)/|.|), as one 16-byte store per lane; the depth
// gradient is then the transposed difference stencil of these slopes
// (slopes_to_depth_kernel), so the backward pass no longer evaluates the shading.
template <bool kMse, bool kU8, bool kSlopes>
__global__ void __launch_bounds__(256, 2) shade_coeff_grad_kernel(ShadeGeom G, int64_t B,
                                                                   const float* __restrict__ coeffs,
                                                                   const int32_t* __restrict__ sensor_id,
                                                                   const float* __restrict__ depth,
                                                                   const float* __restrict__ u_inten,
                                                                   const float* __restrict__ scale,
                                                                   float* __restrict__ grad_coeffs,
                                                                   float* __restrict__ loss_map,
                                                                   float* __restrict__ slopes) {
    constexpr int kTerms = kMse ? 19 : 18;
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* ring = reinterpret_cast<float2*>(dsm) + warp * (kCgStages * kCgSlots * 32);
    int* list = reinterpret_cast<int*>(dsm + kCgRingBytes) + warp * kCgSeg;
    const int s = blockIdx.y;
    const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kCgPx + 2 * lane;   // HW is even: p0 + 1 < HW too
    const bool valid = p0 < G.HW;
    const int y = valid ? static_cast<int>(p0 / G.W) : 0, x = valid ? static_cast<int>(p0 - static_cast<int64_t>(y) * G.W) : 0;
    // the two pixels' x stencils (W >= 4 and x even): pixel x reads (x - 1 or x, x + 1),
    // pixel x + 1 reads (x, x + 2 or x + 1), with the scales axis_stencil gives
    const bool hasL = x > 0, hasR = x + 2 < G.W;
    const float c_in = 1.f / (2.f * G.px), c_edge = 1.f / G.px;
    const float cx0 = hasL ? c_in : c_edge, cx1 = hasR ? c_in : c_edge;
    int ylo, yhi;
    float cy;
    axis_stencil(y, G.H, G.py, ylo, yhi, cy);
    const int o_c = y * G.W + x, o_u = ylo * G.W + x, o_d = yhi * G.W + x;
    const int o_e = lane == 0 ? (hasL ? o_c - 1 : -1) : lane == 31 ? (hasR ? o_c + 2 : -1) : -1;
    const f2 one2 = pk(1.f, 1.f), cyy = pk(cy, cy);
    const float w2s = kMse ? 2.f * (scale != nullptr ? __ldg(scale) : 1.f) : 1.f;
    f2 a[6][3], acc[6][3];
    f2 lacc = pk(0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < 6; ++kk)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 v = make_float2(0.f, 0.f);
            if (valid) v = __ldg(reinterpret_cast<const float2*>(coeffs + (static_cast<int64_t>(s) * 18 + kk * 3 + c) * G.HW + p0));
            a[kk][c] = pk(v.x, v.y);
            acc[kk][c] = pk(0.f, 0.f);
        }
    const int64_t per = (B + kImgWarps - 1) / kImgWarps;
    const int64_t w0 = min(warp * per, B), w1 = min(w0 + per, B);
    const unsigned below = (1u << lane) - 1u;
    for (int64_t seg = w0; seg < w1; seg += kCgSeg) {
        // this slice's images of sensor s, kCgSeg at a time, in order
        const int64_t seg_end = min(seg + kCgSeg, w1);
        int n = 0;
        for (int64_t base = seg; base < seg_end; base += 32) {
            const int sid = base + lane < seg_end ? __ldg(sensor_id + base + lane) : -1;
            const unsigned mask = __ballot_sync(0xffffffffu, sid == s);
            if (sid == s) list[n + __popc(mask & below)] = static_cast<int>(base + lane);
            n += __popc(mask);
        }
        __syncwarp();
        auto start = [&](int i) {
            if (i < n && valid) {
                float2* sl = ring + (i % kCgStages) * (kCgSlots * 32) + lane;
                const int64_t b = list[i];
                const float* D = depth + b * G.HW;
                cp_async8(sl, D + o_c);
                cp_async8(sl + 32, D + o_u);
                cp_async8(sl + 64, D + o_d);
                if (o_e >= 0) cp_async4(&sl[96].x, D + o_e);
                const float* U = u_inten + (b * G.HW + p0) * 3;
                if (kU8) {
                    cp_async8(sl + 128, U);
                    cp_async8(sl + 160, U + 2);
                    cp_async8(sl + 192, U + 4);
                } else {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        cp_async4(&sl[128 + 32 * q].x, U + 2 * q);
                        cp_async4(&sl[128 + 32 * q].y, U + 2 * q + 1);
                    }
                }
            }
            cp_async_commit();      // one group per image slot, empty or not
        };
#pragma unroll
        for (int i = 0; i < kCgStages - 1; ++i) start(i);
        for (int i = 0; i < n; ++i) {
            start(i + kCgStages - 1);
            cp_async_wait<kCgStages - 1>();      // this lane's copies of image i have landed
            const float2* sl = ring + (i % kCgStages) * (kCgSlots * 32) + lane;
            const float2 ce = sl[0], up = sl[32], dn = sl[64];
            // every lane takes part in the shuffles; lanes 0 and 31 read the pixel beyond
            // the warp's segment from their edge slot
            float L = __shfl_up_sync(0xffffffffu, ce.y, 1);
            float R = __shfl_down_sync(0xffffffffu, ce.x, 1);
            if (lane == 0) L = sl[96].x;
            if (lane == 31) R = sl[96].x;
            const f2 dxp = pk((ce.y - (hasL ? L : ce.x)) * cx0, ((hasR ? R : ce.y) - ce.x) * cx1);
            const f2 dyp = mul2(sub2(pk(dn.x, dn.y), pk(up.x, up.y)), cyy);
            // a warp whose pixels all see a flat gel (both depth differences exactly zero):
            // n = (0, 0), so m = (1, +-0, +-0, 0, 0, +-0) and every term but m_0's adds a
            // signed zero to a sum that is never -0; the flat path leaves those terms out,
            // with the same bits (coefficients finite)
            const bool flat = __all_sync(0xffffffffu, !valid || ((dxp | dyp) & 0x7fffffff7fffffffull) == 0ull);
            if (!valid) continue;
            const float2 u01 = sl[128], u23 = sl[160], u45 = sl[192];
            // |(D_x, D_y, 1)|^-1 (the flat form needs it only for the slopes)
            auto inv_norm = [&]() {
                const f2 s2 = fma2(dxp, dxp, fma2(dyp, dyp, one2));
                return pk(rsqrtf(lo(s2)), rsqrtf(hi(s2)));
            };
            const float ua[3] = {u01.x, u01.y, u23.x}, ub[3] = {u23.y, u45.x, u45.y};
            if (flat) {
                f2 gm1 = pk(0.f, 0.f), gm2 = pk(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 I = fma2(a[0][c], one2, pk(0.f, 0.f));
                    const float Ia = lo(I), Ib = hi(I);
                    if (kMse) {
                        const float ea = fminf(fmaxf(Ia, 0.f), 255.f) - ua[c];
                        const float eb = fminf(fmaxf(Ib, 0.f), 255.f) - ub[c];
                        lacc = pk(fmaf(ea, ea, lo(lacc)), fmaf(eb, eb, hi(lacc)));
                    }
                    const float ga = (Ia > 0.f && Ia < 255.f) ? (kMse ? w2s * (Ia - ua[c]) : ua[c]) : 0.f;
                    const float gb = (Ib > 0.f && Ib < 255.f) ? (kMse ? w2s * (Ib - ub[c]) : ub[c]) : 0.f;
                    const f2 gc = pk(ga, gb);
                    acc[0][c] = fma2(gc, one2, acc[0][c]);
                    if (kSlopes) {
                        gm1 = fma2(gc, a[1][c], gm1);
                        gm2 = fma2(gc, a[2][c], gm2);
                    }
                }
                if (kSlopes) {
                    // (dL/dD_x, dL/dD_y) = (gm_1, gm_2) r at n = 0
                    const f2 r = inv_norm();
                    const f2 sx = mul2(gm1, r), sy = mul2(gm2, r);
                    *reinterpret_cast<float4*>(slopes + (static_cast<int64_t>(list[i]) * G.HW + p0) * 2) =
                        make_float4(lo(sx), lo(sy), hi(sx), hi(sy));
                }
                continue;
            }
            const f2 r = inv_norm();
            const f2 nx = mul2(dxp, r), ny = mul2(dyp, r);
            const f2 m[6] = {one2, nx, ny, mul2(nx, nx), mul2(ny, ny), mul2(nx, ny)};
            // the accumulation reads the monomials with a non-finite depth difference set to
            // zero, so that such a pixel (whose intensity is NaN and never passes the clamp
            // test) adds nothing, as in the single-pixel kernel
            const bool fa = lo(nx) == lo(nx) && lo(ny) == lo(ny), fb = hi(nx) == hi(nx) && hi(ny) == hi(ny);
            f2 ma[6];
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) ma[kk] = pk(fa ? lo(m[kk]) : 0.f, fb ? hi(m[kk]) : 0.f);
            f2 gm[6];       // kSlopes: dL/dm_k, from the raw coefficients
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) gm[kk] = pk(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                f2 I = pk(0.f, 0.f);
#pragma unroll
                for (int kk = 0; kk < 6; ++kk) I = fma2(a[kk][c], m[kk], I);
                const float Ia = lo(I), Ib = hi(I);
                if (kMse) {
                    const float ea = fminf(fmaxf(Ia, 0.f), 255.f) - ua[c];
                    const float eb = fminf(fmaxf(Ib, 0.f), 255.f) - ub[c];
                    lacc = pk(fmaf(ea, ea, lo(lacc)), fmaf(eb, eb, hi(lacc)));
                }
                const float ga = (Ia > 0.f && Ia < 255.f) ? (kMse ? w2s * (Ia - ua[c]) : ua[c]) : 0.f;
                const float gb = (Ib > 0.f && Ib < 255.f) ? (kMse ? w2s * (Ib - ub[c]) : ub[c]) : 0.f;
                const f2 gc = pk(ga, gb);
#pragma unroll
                for (int kk = 0; kk < 6; ++kk) acc[kk][c] = fma2(gc, ma[kk], acc[kk][c]);
                if (kSlopes) {
#pragma unroll
                    for (int kk = 0; kk < 6; ++kk) gm[kk] = fma2(gc, a[kk][c], gm[kk]);
                }
            }
            if (kSlopes) {
                // n = (D_x, D_y, 1) r with r = |(D_x, D_y, 1)|^-1: dn_x/dD_x = r - D_x^2 r^3,
                // dn_x/dD_y = dn_y/dD_x = -D_x D_y r^3, dn_y/dD_y = r - D_y^2 r^3; and
                // m = (1, n_x, n_y, n_x^2, n_y^2, n_x n_y)
                const f2 two = pk(2.f, 2.f);
                const f2 gnx = fma2(mul2(two, nx), gm[3], fma2(ny, gm[5], gm[1]));
                const f2 gny = fma2(mul2(two, ny), gm[4], fma2(nx, gm[5], gm[2]));
                const f2 r3 = mul2(mul2(r, r), r);
                const f2 cxy = mul2(mul2(dxp, dyp), r3);
                const f2 kx = sub2(r, mul2(mul2(dxp, dxp), r3));
                const f2 ky = sub2(r, mul2(mul2(dyp, dyp), r3));
                const f2 sx = sub2(mul2(gnx, kx), mul2(gny, cxy));
                const f2 sy = sub2(mul2(gny, ky), mul2(gnx, cxy));
                *reinterpret_cast<float4*>(slopes + (static_cast<int64_t>(list[i]) * G.HW + p0) * 2) =
                    make_float4(lo(sx), lo(sy), hi(sx), hi(sy));
            }
        }
        cp_async_wait<0>();
        __syncwarp();               // the list and the ring are reused by the next segment
    }
    __syncthreads();                // every warp is done with the ring: it becomes the partial sums
    float* part = reinterpret_cast<float*>(dsm);    // [warp][term][kCgPx]
#pragma unroll
    for (int kk = 0; kk < 6; ++kk)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            *reinterpret_cast<float2*>(part + (warp * kTerms + kk * 3 + c) * kCgPx + 2 * lane) =
                make_float2(lo(acc[kk][c]), hi(acc[kk][c]));
    if (kMse) *reinterpret_cast<float2*>(part + (warp * kTerms + kTerms - 1) * kCgPx + 2 * lane) =
        make_float2(lo(lacc), hi(lacc));
    __syncthreads();
    // kTerms x 64 sums over the 8 warps, in warp order
    for (int i = threadIdx.x; i < kTerms * kCgPx; i += blockDim.x) {
        const int term = i / kCgPx, l = i - term * kCgPx;
        const int64_t p = static_cast<int64_t>(blockIdx.x) * kCgPx + l;
        if (p >= G.HW) continue;
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < kImgWarps; ++w) sum += part[(w * kTerms + term) * kCgPx + l];
        if (term < 18) {
            if (grad_coeffs != nullptr) grad_coeffs[(static_cast<int64_t>(s) * 18 + term) * G.HW + p] = sum;
        } else if (loss_map != nullptr) {
            loss_map[static_cast<int64_t>(s) * G.HW + p] = sum;
        }
    }
}

// Clamped intensity with two horizontally adjacent pixels per lane: grid (64-pixel tiles,
// sensors, image chunks), a CTA of 8 warps taking equal slices of its chunk.  Per lane and
// image the centre depth pair and the pairs above and below arrive as 8-byte cp.async
// copies kCgStages images ahead (lanes 0 and 31 also fetch the pixel beyond the warp's
// row segment; the other lanes' horizontal neighbours come by shuffle); the arithmetic
// runs on FP32 pairs in the operations and order of the single-pixel definition, and the
// six output floats leave as three 8-byte stores when the output is 8-byte aligned (kO8),
// else as six 4-byte ones.
constexpr int kInSlots = 4;       // 8-byte slots per lane and image
constexpr size_t kInSmemBytes =
    size_t(kImgWarps) * kCgStages * kInSlots * 32 * sizeof(float2) + size_t(kImgWarps) * kCgSeg * sizeof(int);

template <bool kO8>
__global__ void __launch_bounds__(256) shade_intensity_kernel(ShadeGeom G, int64_t B, int64_t chunk,
                                                               const float* __restrict__ coeffs,
                                                               const int32_t* __restrict__ sensor_id,
                                                               const float* __restrict__ depth,
                                                               float* __restrict__ inten) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* ring = reinterpret_cast<float2*>(dsm) + warp * (kCgStages * kInSlots * 32);
    int* list = reinterpret_cast<int*>(dsm + size_t(kImgWarps) * kCgStages * kInSlots * 32 * sizeof(float2)) +
                warp * kCgSeg;
    const int s = blockIdx.y;
    const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kCgPx + 2 * lane;   // HW is even: p0 + 1 < HW too
    const bool valid = p0 < G.HW;
    const int y = valid ? static_cast<int>(p0 / G.W) : 0, x = valid ? static_cast<int>(p0 - static_cast<int64_t>(y) * G.W) : 0;
    const bool hasL = x > 0, hasR = x + 2 < G.W;
    const float c_in = 1.f / (2.f * G.px), c_edge = 1.f / G.px;
    const float cx0 = hasL ? c_in : c_edge, cx1 = hasR ? c_in : c_edge;
    int ylo, yhi;
    float cy;
    axis_stencil(y, G.H, G.py, ylo, yhi, cy);
    const int o_c = y * G.W + x, o_u = ylo * G.W + x, o_d = yhi * G.W + x;
    const int o_e = lane == 0 ? (hasL ? o_c - 1 : -1) : lane == 31 ? (hasR ? o_c + 2 : -1) : -1;
    const f2 one2 = pk(1.f, 1.f), cyy = pk(cy, cy);
    f2 a[6][3];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 v = make_float2(0.f, 0.f);
            if (valid) v = __ldg(reinterpret_cast<const float2*>(coeffs + (static_cast<int64_t>(s) * 18 + kk * 3 + c) * G.HW + p0));
            a[kk][c] = pk(v.x, v.y);
        }
    const int64_t c0 = static_cast<int64_t>(blockIdx.z) * chunk, c1 = min(c0 + chunk, B);
    const int64_t per = (c1 - c0 + kImgWarps - 1) / kImgWarps;
    const int64_t w0 = min(c0 + warp * per, c1), w1 = min(w0 + per, c1);
    const unsigned below = (1u << lane) - 1u;
    for (int64_t seg = w0; seg < w1; seg += kCgSeg) {
        const int64_t seg_end = min(seg + kCgSeg, w1);
        int n = 0;
        for (int64_t base = seg; base < seg_end; base += 32) {
            const int sid = base + lane < seg_end ? __ldg(sensor_id + base + lane) : -1;
            const unsigned mask = __ballot_sync(0xffffffffu, sid == s);
            if (sid == s) list[n + __popc(mask & below)] = static_cast<int>(base + lane);
            n += __popc(mask);
        }
        __syncwarp();
        auto start = [&](int i) {
            if (i < n && valid) {
                float2* sl = ring + (i % kCgStages) * (kInSlots * 32) + lane;
                const float* D = depth + static_cast<int64_t>(list[i]) * G.HW;
                cp_async8(sl, D + o_c);
                cp_async8(sl + 32, D + o_u);
                cp_async8(sl + 64, D + o_d);
                if (o_e >= 0) cp_async4(&sl[96].x, D + o_e);
            }
            cp_async_commit();
        };
#pragma unroll
        for (int i = 0; i < kCgStages - 1; ++i) start(i);
        for (int i = 0; i < n; ++i) {
            start(i + kCgStages - 1);
            cp_async_wait<kCgStages - 1>();
            const float2* sl = ring + (i % kCgStages) * (kInSlots * 32) + lane;
            const float2 ce = sl[0], up = sl[32], dn = sl[64];
            float L = __shfl_up_sync(0xffffffffu, ce.y, 1);
            float R = __shfl_down_sync(0xffffffffu, ce.x, 1);
            if (lane == 0) L = sl[96].x;
            if (lane == 31) R = sl[96].x;
            const f2 dxp = pk((ce.y - (hasL ? L : ce.x)) * cx0, ((hasR ? R : ce.y) - ce.x) * cx1);
            const f2 dyp = mul2(sub2(pk(dn.x, dn.y), pk(up.x, up.y)), cyy);
            // a flat warp (both depth differences exactly zero at every pixel): I = A_0, with
            // the bits of the full sum (its other terms add signed zeros; coefficients finite)
            const bool flat = __all_sync(0xffffffffu, !valid || ((dxp | dyp) & 0x7fffffff7fffffffull) == 0ull);
            if (!valid) continue;
            float o[6];
            if (flat) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 I = fma2(a[0][c], one2, pk(0.f, 0.f));
                    o[c] = fminf(fmaxf(lo(I), 0.f), 255.f);
                    o[3 + c] = fminf(fmaxf(hi(I), 0.f), 255.f);
                }
            } else {
                const f2 s2 = fma2(dxp, dxp, fma2(dyp, dyp, one2));
                const f2 r = pk(rsqrtf(lo(s2)), rsqrtf(hi(s2)));
                const f2 nx = mul2(dxp, r), ny = mul2(dyp, r);
                const f2 m[6] = {one2, nx, ny, mul2(nx, nx), mul2(ny, ny), mul2(nx, ny)};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    f2 I = pk(0.f, 0.f);
#pragma unroll
                    for (int kk = 0; kk < 6; ++kk) I = fma2(a[kk][c], m[kk], I);
                    o[c] = fminf(fmaxf(lo(I), 0.f), 255.f);
                    o[3 + c] = fminf(fmaxf(hi(I), 0.f), 255.f);
                }
            }
            float* out = inten + (static_cast<int64_t>(list[i]) * G.HW + p0) * 3;
            if (kO8) {
#pragma unroll
                for (int q = 0; q < 3; ++q) reinterpret_cast<float2*>(out)[q] = make_float2(o[2 * q], o[2 * q + 1]);
            } else {
#pragma unroll
                for (int q = 0; q < 6; ++q) out[q] = o[q];
            }
        }
        cp_async_wait<0>();
        __syncwarp();
    }
}

// dL/dD[b][p]: the transpose of the difference stencils, gathered from the pixels q whose
// D_x (q in p's row, |q - p| <= 1) or D_y (q in p's column) reads D[p].  Along each axis
// at most two such q carry a nonzero weight (central inside; one-sided on the border), so
// a pixel has at most four "slots" (q, axis, weight); their coefficients are kept in
// registers while the warps walk the sensor's images (grid and image split as in
// shade_coeff_grad_kernel).  Images with a bad sensor id are zeroed by
// zero_bad_sensor_images_kernel.
struct DepthSlot {
    int qx, qy;
    float w;       // weight of D[p] in D_x(q) (axis 0) or D_y(q) (axis 1); 0 = unused
};

// The weight of D[me] in the derivative at c along an axis of length len.
__device__ __forceinline__ float stencil_weight(int c, int me, int len, float pitch) {
    int lo, hi;
    float cc;
    axis_stencil(c, len, pitch, lo, hi, cc);
    return (hi == me ? cc : 0.f) - (lo == me ? cc : 0.f);
}

// Per axis the two pixels whose derivative can read D[p]: the left one (x - 1, or p
// itself on the left border) and the right one (x + 1, or p itself on the right border);
// every other pixel's stencil misses p.
__device__ __forceinline__ void depth_slots(const ShadeGeom& G, int x, int y, DepthSlot (&sl)[4]) {
    const int xl = x >= 1 ? x - 1 : x, xr = x + 1 < G.W ? x + 1 : x;
    const int yl = y >= 1 ? y - 1 : y, yr = y + 1 < G.H ? y + 1 : y;
    sl[0] = DepthSlot{xl, y, stencil_weight(xl, x, G.W, G.px)};
    sl[1] = DepthSlot{xr, y, xr != xl ? stencil_weight(xr, x, G.W, G.px) : 0.f};
    sl[2] = DepthSlot{x, yl, stencil_weight(yl, y, G.H, G.py)};
    sl[3] = DepthSlot{x, yr, yr != yl ? stencil_weight(yr, y, G.H, G.py) : 0.f};
}

// (dL/dD_x, dL/dD_y) at one pixel from its coefficients a[k][c] (registers), its state
// and u (dL/dI, or the target when kMse).
template <bool kMse>
__device__ __forceinline__ void pixel_backward_reg(const float (&a)[6][3], const PixelState& st, const float u[3],
                                                   float w2, float& gDx, float& gDy) {
    const float m[6] = {1.f, st.nx, st.ny, st.nx * st.nx, st.ny * st.ny, st.nx * st.ny};
    float gm[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float I = 0.f;
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) I = fmaf(a[kk][c], m[kk], I);
        if (I > 0.f && I < 255.f) {
            const float gc = kMse ? w2 * (I - u[c]) : u[c];
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) gm[kk] = fmaf(gc, a[kk][c], gm[kk]);
        }
    }
    const float gnx = fmaf(2.f * st.nx, gm[3], fmaf(st.ny, gm[5], gm[1]));
    const float gny = fmaf(2.f * st.ny, gm[4], fmaf(st.nx, gm[5], gm[2]));
    const float r3 = st.r * st.r * st.r;
    gDx = gnx * (st.r - st.dx * st.dx * r3) - gny * st.dx * st.dy * r3;
    gDy = gny * (st.r - st.dy * st.dy * r3) - gnx * st.dx * st.dy * r3;
}

// Tile of the depth-gradient kernel: 32 x 8 pixels of one sensor's image plane, one per
// thread, plus a one-pixel halo whose (dL/dD_x, dL/dD_y) the stencils of the tile read.
constexpr int kDgTx = 32, kDgTy = 8, kDgHalo = 2 * kDgTx + 2 * kDgTy;

template <bool kMse>
__device__ __forceinline__ void load_coeffs18(const float* As, int64_t HW, int64_t q, bool ok, float (&a)[6][3]) {
#pragma unroll
    for (int kk = 0; kk < 6; ++kk)
#pragma unroll
        for (int c = 0; c < 3; ++c) a[kk][c] = ok ? __ldg(As + (kk * 3 + c) * HW + q) : 0.f;
}

// Grid (tiles, sensors, image chunks), 256 threads.  For each image of sensor s in the
// chunk (listed by warp 0, kCgSeg at a time, into shared memory): every thread evaluates
// (dL/dD_x, dL/dD_y) at its pixel and threads 0..79 at one halo pixel each, into shared
// memory; then each pixel sums its four stencil-transpose terms.  The coefficients of a
// thread's pixel and halo pixel stay in registers across the images, and its 14 inputs
// per image (4 depth samples and 3 upstream values, for each of the two pixels) are
// fetched kDgStages images ahead by per-thread cp.async copies into a shared ring.
constexpr int kDgStages = 3;
constexpr int kDgVals = 14;

template <bool kMse>
__global__ void __launch_bounds__(256, 3) shade_depth_grad_kernel(ShadeGeom G, int64_t B, const float* __restrict__ coeffs,
                                                                   const int32_t* __restrict__ sensor_id,
                                                                   const float* __restrict__ depth,
                                                                   const float* __restrict__ u_inten,
                                                                   const float* __restrict__ scale,
                                                                   float* __restrict__ grad_depth) {
    __shared__ float gx_s[kDgTy][kDgTx + 2];   // dL/dD_x at columns x0 - 1 .. x0 + 32
    __shared__ float gy_s[kDgTy + 2][kDgTx];   // dL/dD_y at rows y0 - 1 .. y0 + 8
    __shared__ float ring[kDgStages][kDgVals][256];
    __shared__ int list[kCgSeg];
    __shared__ int list_n;
    const int t = threadIdx.x, lane = t & 31;
    const int tiles_x = (G.W + kDgTx - 1) / kDgTx;
    const int x0 = (static_cast<int>(blockIdx.x) % tiles_x) * kDgTx, y0 = (static_cast<int>(blockIdx.x) / tiles_x) * kDgTy;
    const int tx = t & (kDgTx - 1), ty = t / kDgTx;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = x < G.W && y < G.H;
    const int s = blockIdx.y;
    const float w2 = kMse ? 2.f * (scale != nullptr ? __ldg(scale) : 1.f) : 1.f;
    const float* As = coeffs + static_cast<int64_t>(s) * 18 * G.HW;
    // own pixel and its four slots
    DepthSlot sl[4];
    depth_slots(G, valid ? x : 0, valid ? y : 0, sl);
    float a[6][3];
    load_coeffs18<kMse>(As, G.HW, static_cast<int64_t>(y) * G.W + x, valid, a);
    // halo pixel of threads 0..79: rows y0 - 1 and y0 + 8 (their D_y), columns x0 - 1 and
    // x0 + 32 (their D_x); absent outside the image
    int hx = 0, hy = 0, haxis = -1;
    if (t < kDgTx) { hx = x0 + t; hy = y0 - 1; haxis = 1; }
    else if (t < 2 * kDgTx) { hx = x0 + t - kDgTx; hy = y0 + kDgTy; haxis = 1; }
    else if (t < 2 * kDgTx + kDgTy) { hx = x0 - 1; hy = y0 + t - 2 * kDgTx; haxis = 0; }
    else if (t < kDgHalo) { hx = x0 + kDgTx; hy = y0 + t - 2 * kDgTx - kDgTy; haxis = 0; }
    const bool hvalid = haxis >= 0 && hx >= 0 && hx < G.W && hy >= 0 && hy < G.H;
    float ah[6][3];
    load_coeffs18<kMse>(As, G.HW, hvalid ? static_cast<int64_t>(hy) * G.W + hx : 0, hvalid, ah);
    // the difference stencils of both pixels (image-independent offsets and scales)
    int lo, hi;
    float cxo, cyo, cxh, cyh;
    axis_stencil(valid ? x : 0, G.W, G.px, lo, hi, cxo);
    // (offsets within one image: H * W < 2^28, so 32 bits hold them)
    const int oxh = y * G.W + hi, oxl = y * G.W + lo;
    axis_stencil(valid ? y : 0, G.H, G.py, lo, hi, cyo);
    const int oyh = hi * G.W + x, oyl = lo * G.W + x;
    axis_stencil(hvalid ? hx : 0, G.W, G.px, lo, hi, cxh);
    const int hxh = hy * G.W + hi, hxl = hy * G.W + lo;
    axis_stencil(hvalid ? hy : 0, G.H, G.py, lo, hi, cyh);
    const int hyh = hi * G.W + hx, hyl = lo * G.W + hx;
    const int qo = y * G.W + x, qh = hy * G.W + hx;
    auto state = [](float xh, float xl, float yh, float yl, float cx, float cy) {
        PixelState st;
        st.dx = (xh - xl) * cx;
        st.dy = (yh - yl) * cy;
        st.r = rsqrtf(fmaf(st.dx, st.dx, fmaf(st.dy, st.dy, 1.f)));
        st.nx = st.dx * st.r;
        st.ny = st.dy * st.r;
        return st;
    };
    const int64_t chunk = (B + gridDim.z - 1) / gridDim.z;
    const int64_t c0 = static_cast<int64_t>(blockIdx.z) * chunk, c1 = min(c0 + chunk, B);
    for (int64_t seg = c0; seg < c1; seg += kCgSeg) {
        const int64_t seg_end = min(seg + kCgSeg, c1);
        if (t < 32) {       // warp 0 lists the segment's images of sensor s
            int n = 0;
            for (int64_t base = seg; base < seg_end; base += 32) {
                const int sid = base + lane < seg_end ? __ldg(sensor_id + base + lane) : -1;
                const unsigned mask = __ballot_sync(0xffffffffu, sid == s);
                if (sid == s) list[n + __popc(mask & ((1u << lane) - 1u))] = static_cast<int>(base + lane);
                n += __popc(mask);
            }
            if (lane == 0) list_n = n;
        }
        __syncthreads();
        const int n = list_n;
        auto issue = [&](int i) {
            if (i < n) {
                const int64_t b = list[i];
                const float* D = depth + b * G.HW;
                const float* U = u_inten + b * G.HW * 3;
                float* st = &ring[i % kDgStages][0][t];
                if (valid) {
                    cp_async4(st + 0 * 256, D + oxh);
                    cp_async4(st + 1 * 256, D + oxl);
                    cp_async4(st + 2 * 256, D + oyh);
                    cp_async4(st + 3 * 256, D + oyl);
                    cp_async4(st + 4 * 256, U + 3 * qo);
                    cp_async4(st + 5 * 256, U + 3 * qo + 1);
                    cp_async4(st + 6 * 256, U + 3 * qo + 2);
                }
                if (hvalid) {
                    cp_async4(st + 7 * 256, D + hxh);
                    cp_async4(st + 8 * 256, D + hxl);
                    cp_async4(st + 9 * 256, D + hyh);
                    cp_async4(st + 10 * 256, D + hyl);
                    cp_async4(st + 11 * 256, U + 3 * qh);
                    cp_async4(st + 12 * 256, U + 3 * qh + 1);
                    cp_async4(st + 13 * 256, U + 3 * qh + 2);
                }
            }
            cp_async_commit();
        };
#pragma unroll
        for (int i = 0; i < kDgStages - 1; ++i) issue(i);
        for (int i = 0; i < n; ++i) {
            issue(i + kDgStages - 1);
            cp_async_wait<kDgStages - 1>();          // this thread's copies of image i have landed
            const float* st = &ring[i % kDgStages][0][t];
            if (valid) {
                const float u[3] = {st[4 * 256], st[5 * 256], st[6 * 256]};
                float gx, gy;
                pixel_backward_reg<kMse>(a, state(st[0], st[256], st[2 * 256], st[3 * 256], cxo, cyo), u, w2, gx, gy);
                gx_s[ty][tx + 1] = gx;
                gy_s[ty + 1][tx] = gy;
            }
            if (hvalid) {
                const float u[3] = {st[11 * 256], st[12 * 256], st[13 * 256]};
                float gx, gy;
                pixel_backward_reg<kMse>(ah, state(st[7 * 256], st[8 * 256], st[9 * 256], st[10 * 256], cxh, cyh), u,
                                         w2, gx, gy);
                if (haxis == 0) gx_s[hy - y0][hx - x0 + 1] = gx;
                else gy_s[hy - y0 + 1][hx - x0] = gy;
            }
            __syncthreads();
            if (valid) {
                float acc = sl[0].w * gx_s[ty][sl[0].qx - x0 + 1];
                acc = fmaf(sl[1].w, gx_s[ty][sl[1].qx - x0 + 1], acc);
                acc = fmaf(sl[2].w, gy_s[sl[2].qy - y0 + 1][tx], acc);
                acc = fmaf(sl[3].w, gy_s[sl[3].qy - y0 + 1][tx], acc);
                grad_depth[static_cast<int64_t>(list[i]) * G.HW + qo] = acc;
            }
            __syncthreads();
        }
        cp_async_wait<0>();
    }
}

// Zeroes the depth gradient of every image whose sensor id is out of range (the
// per-sensor kernels never visit such images).  One block per image slot.
__global__ void __launch_bounds__(256) zero_bad_sensor_images_kernel(int64_t B, int S, int64_t HW,
                                                                      const int32_t* __restrict__ sensor_id,
                                                                      float* __restrict__ grad_depth) {
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        const int s = __ldg(sensor_id + b);
        if (s >= 0 && s < S) continue;
        for (int64_t k = threadIdx.x; k < HW; k += blockDim.x) grad_depth[b * HW + k] = 0.f;
    }
}

// Depth gradient from pixel slopes: grad_depth[b][q] = scale * sum over the pixels p
// whose difference stencils read D[q] of w(p, q) * slope(p) (the transpose of the
// central / one-sided differences of the normal), with the four slots of depth_slots
// summed in slot order.  Grid (512-pixel strips of the image plane, image chunks), 256
// threads, two horizontally adjacent pixels per thread (W is a multiple of 4, so a pair
// never straddles a row): per image a thread reads its pair's slopes and the pairs in
// the rows above and below (16-byte loads; those rows are read again by the neighbouring
// strips at the same time, so they come from L2), takes the horizontal neighbours'
// D_x slopes by shuffle (lanes 0 and 31 load theirs), and writes its two gradients as
// one 8-byte store.  The stencil weights are fixed per pixel and computed once; images
// with a bad sensor id get zero.  Two images per iteration keep more loads in flight.
constexpr int kSdPx = 512;

struct SlopeRows {
    float4 own, up, dn;
    float left, right;
};

__global__ void __launch_bounds__(256, 4) slopes_to_depth_kernel(ShadeGeom G, int64_t B, int64_t chunk,
                                                              const int32_t* __restrict__ sensor_id,
                                                              const float* __restrict__ slopes,
                                                              const float* __restrict__ scale,
                                                              float* __restrict__ grad_depth) {
    const int lane = threadIdx.x & 31;
    const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kSdPx + 2 * threadIdx.x;
    const bool valid = p0 < G.HW;
    const int y = valid ? static_cast<int>(p0 / G.W) : 0, x = valid ? static_cast<int>(p0 - static_cast<int64_t>(y) * G.W) : 0;
    DepthSlot sa[4], sb[4];
    depth_slots(G, x, y, sa);
    depth_slots(G, x + 1, y, sb);
    // pixel x reads D_x at x - 1 (or x on the left border) and x + 1; pixel x + 1 at x and
    // x + 2 (or x + 1 on the right border); both read D_y in rows sa[2].qy and sa[3].qy
    const bool hasL = x > 0, hasR = x + 2 < G.W;
    const int o_up = sa[2].qy * G.W + x, o_dn = sa[3].qy * G.W + x, o_c = y * G.W + x;
    const float sc = scale != nullptr ? __ldg(scale) : 1.f;
    const int64_t c0 = static_cast<int64_t>(blockIdx.y) * chunk, c1 = min(c0 + chunk, B);
    auto load = [&](int64_t b, SlopeRows& v) {
        const float* Sb = slopes + b * G.HW * 2;
        if (valid) {
            v.own = __ldg(reinterpret_cast<const float4*>(Sb + 2 * static_cast<int64_t>(o_c)));
            v.up = __ldg(reinterpret_cast<const float4*>(Sb + 2 * static_cast<int64_t>(o_up)));
            v.dn = __ldg(reinterpret_cast<const float4*>(Sb + 2 * static_cast<int64_t>(o_dn)));
        } else {
            v.own = v.up = v.dn = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        v.left = (valid && lane == 0 && hasL) ? __ldg(Sb + 2 * static_cast<int64_t>(o_c - 1)) : 0.f;
        v.right = (valid && lane == 31 && hasR) ? __ldg(Sb + 2 * static_cast<int64_t>(o_c + 2)) : 0.f;
    };
    auto finish = [&](int64_t b, const SlopeRows& v) {
        // every lane takes part in the shuffles
        float L = __shfl_up_sync(0xffffffffu, v.own.z, 1);
        float R = __shfl_down_sync(0xffffffffu, v.own.x, 1);
        if (lane == 0) L = v.left;
        if (lane == 31) R = v.right;
        if (!valid) return;
        const int s = __ldg(sensor_id + b);
        float ga = 0.f, gb = 0.f;
        if (s >= 0 && s < G.S) {
            ga = sa[0].w * (hasL ? L : v.own.x);
            ga = fmaf(sa[1].w, v.own.z, ga);
            ga = fmaf(sa[2].w, v.up.y, ga);
            ga = fmaf(sa[3].w, v.dn.y, ga);
            gb = sb[0].w * v.own.x;
            gb = fmaf(sb[1].w, hasR ? R : v.own.z, gb);
            gb = fmaf(sb[2].w, v.up.w, gb);
            gb = fmaf(sb[3].w, v.dn.w, gb);
            ga *= sc;
            gb *= sc;
        }
        *reinterpret_cast<float2*>(grad_depth + b * G.HW + o_c) = make_float2(ga, gb);
    };
    int64_t b = c0;
    for (; b + 1 < c1; b += 2) {
        SlopeRows v0, v1;
        load(b, v0);
        load(b + 1, v1);
        finish(b, v0);
        finish(b + 1, v1);
    }
    if (b < c1) {
        SlopeRows v0;
        load(b, v0);
        finish(b, v0);
    }
}

}  // namespace tacsl

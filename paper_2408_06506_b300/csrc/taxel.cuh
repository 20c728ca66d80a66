// Taxel-side kernels: SDF query with finite-difference gradient, penalty normal and
// friction-capped shear forces, per-pad wrench (Sec. III-C of arXiv 2408.06506).
//
// Interpolation reading: the grid's nodes are samples; between them the field is
// trilinear; the gradient is the central difference of that interpolant with step
// voxel/2 per axis.  All seven trilinear evaluations (centre and +-x, +-y, +-z) fall on
// a 3x3x3 node window, so one query gathers 27 nodes (nine rows of three along x)
// and folds them axis by axis with per-axis weight vectors: centre weights c[3] and
// difference weights d[3] = w(u + 1/2) - w(u - 1/2).
//
// Sparsity: a taxel contributes only where it penetrates (phi < 0).  phi is first read
// from the 8 nodes of its cell (bitwise the value of the full fold); the other 19 nodes
// and the gradient are gathered only for penetrating taxels.
//
// Work split: ONE WARP PER PAD.  Lanes take taxels lane, lane+32, ..., NP at a time so
// that NP 8-node gathers are in flight per lane.  Taxels that do not penetrate get their
// outputs (depth 0, zero forces) at once; the penetrating ones of each round are then
// compacted over the warp's lanes, so the 27-node window and the force law run with as
// many lanes busy as there are such taxels instead of once per slot with a few lanes
// busy.  The warp folds the pad's wrench with shuffles - no block-wide barrier, so many
// pads progress at once and the gathers' latency overlaps.  SDF reads carry an L2
// evict-last policy (the grids are re-read every step).
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

// Node window of one query: base pointer and per-axis weights (centre c, difference d).
struct Stencil {
    const float* base;
    float cx[3], dx[3], cy[3], dy[3], cz[3], dz[3];
    bool inside;
};

__device__ __forceinline__ Stencil stencil_setup(const DevSdf& S, float x, float y, float z) {
    Stencil q;
    const float ux = (x - S.ox) * S.inv_h, uy = (y - S.oy) * S.inv_h, uz = (z - S.oz) * S.inv_h;
    q.inside = ux >= 0.5f && ux <= static_cast<float>(S.n0) - 1.5f && uy >= 0.5f &&
               uy <= static_cast<float>(S.n1) - 1.5f && uz >= 0.5f && uz <= static_cast<float>(S.n2) - 1.5f;
    int bx = 0, by = 0, bz = 0;
    if (q.inside) {
        axis_weights(ux, S.n0, bx, q.cx, q.dx);
        axis_weights(uy, S.n1, by, q.cy, q.dy);
        axis_weights(uz, S.n2, bz, q.cz, q.dz);
    }
    q.base = S.data + (static_cast<int64_t>(bz) * S.n0 * S.n1 + static_cast<int64_t>(by) * S.n0 + bx);
    return q;
}

__device__ __forceinline__ void stencil_load(const Stencil& q, int n0, int n01, uint64_t pol, float (&v)[3][3][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) v[k][j][i] = ldg_f_hint(q.base + k * n01 + j * n0 + i, pol);
}

// Fold the gathered window: phi and the h/2 central differences along x, y, z.
__device__ __forceinline__ void stencil_fold(const Stencil& q, const float (&v)[3][3][3], float inv_h, float& phi,
                                             float g[3]) {
    float rc[3][3], rd[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rc[k][j] = fmaf(q.cx[2], v[k][j][2], fmaf(q.cx[1], v[k][j][1], q.cx[0] * v[k][j][0]));
            rd[k][j] = fmaf(q.dx[2], v[k][j][2], fmaf(q.dx[1], v[k][j][1], q.dx[0] * v[k][j][0]));
        }
    float cc[3], cd[3], xd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cc[k] = fmaf(q.cy[2], rc[k][2], fmaf(q.cy[1], rc[k][1], q.cy[0] * rc[k][0]));
        cd[k] = fmaf(q.dy[2], rc[k][2], fmaf(q.dy[1], rc[k][1], q.dy[0] * rc[k][0]));
        xd[k] = fmaf(q.cy[2], rd[k][2], fmaf(q.cy[1], rd[k][1], q.cy[0] * rd[k][0]));
    }
    phi = fmaf(q.cz[2], cc[2], fmaf(q.cz[1], cc[1], q.cz[0] * cc[0]));
    g[0] = fmaf(q.cz[2], xd[2], fmaf(q.cz[1], xd[1], q.cz[0] * xd[0])) * inv_h;
    g[1] = fmaf(q.cz[2], cd[2], fmaf(q.cz[1], cd[1], q.cz[0] * cd[0])) * inv_h;
    g[2] = fmaf(q.dz[2], cc[2], fmaf(q.dz[1], cc[1], q.dz[0] * cc[0])) * inv_h;
}

// Position of the set bit of rank `rank` (0-based, from bit 0 up) of mask; rank must be
// below popc(mask).  Binary search on the position with population counts.
__device__ __forceinline__ int nth_set_bit(unsigned mask, int rank) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc((mask >> pos) & ((1u << w) - 1u));
        if (rank >= c) {
            rank -= c;
            pos += w;
        }
    }
    return pos;
}

// Continuous grid index of an object-frame point and its domain test.
struct GridPos {
    float ux, uy, uz;
    bool inside;
};
__device__ __forceinline__ GridPos grid_pos(const DevSdf& S, float x, float y, float z) {
    GridPos g;
    g.ux = (x - S.ox) * S.inv_h;
    g.uy = (y - S.oy) * S.inv_h;
    g.uz = (z - S.oz) * S.inv_h;
    g.inside = g.ux >= 0.5f && g.ux <= static_cast<float>(S.n0) - 1.5f && g.uy >= 0.5f &&
               g.uy <= static_cast<float>(S.n1) - 1.5f && g.uz >= 0.5f && g.uz <= static_cast<float>(S.n2) - 1.5f;
    return g;
}

// phi alone from the 8 nodes of the trilinear cell of u (cell min(floor(u), n-2) per
// axis, fraction f, weights 1-f and f), in the FMA order of stencil_fold, so the value
// is bitwise the phi of the full 27-node fold: there the zero-weight terms enter as
// fma(0, v, acc) = acc or as 0 * v + ..., which leaves every partial sum unchanged.
__device__ __forceinline__ float phi_cell8(const DevSdf& S, const GridPos& g, uint64_t pol) {
    const int ix = min(static_cast<int>(floorf(g.ux)), S.n0 - 2);
    const int iy = min(static_cast<int>(floorf(g.uy)), S.n1 - 2);
    const int iz = min(static_cast<int>(floorf(g.uz)), S.n2 - 2);
    const float fx = g.ux - static_cast<float>(ix), fy = g.uy - static_cast<float>(iy),
                fz = g.uz - static_cast<float>(iz);
    const int n0 = S.n0, n01 = S.n0 * S.n1;
    const float* b = S.data + (static_cast<int64_t>(iz) * n01 + static_cast<int64_t>(iy) * n0 + ix);
    float v[2][2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) v[k][j][i] = ldg_f_hint(b + k * n01 + j * n0 + i, pol);
    float c[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float r0 = fmaf(fx, v[k][0][1], (1.f - fx) * v[k][0][0]);
        const float r1 = fmaf(fx, v[k][1][1], (1.f - fx) * v[k][1][0]);
        c[k] = fmaf(fy, r1, (1.f - fy) * r0);
    }
    return fmaf(fz, c[1], (1.f - fz) * c[0]);
}

// SDF value and gradient at object-frame point (x, y, z).  Returns false outside the
// grid's domain (then phi = +inf, g = 0).
__device__ __forceinline__ bool sdf_stencil(const DevSdf& S, float x, float y, float z, float& phi, float g[3]) {
    const Stencil q = stencil_setup(S, x, y, z);
    if (!q.inside) {
        phi = __int_as_float(0x7f800000);
        g[0] = g[1] = g[2] = 0.f;
        return false;
    }
    float v[3][3][3];
    stencil_load(q, S.n0, S.n0 * S.n1, policy_evict_last(), v);
    stencil_fold(q, v, S.inv_h, phi, g);
    return true;
}

// Penalty normal force and friction-capped shear from the SDF sample (phi, g) at a
// point moving at (vx, vy, vz) relative to the object; both forces returned in the pad
// frame (R^T applied, r = row-major pad->object rotation).
__device__ __forceinline__ void contact_force(const float* r, float phi, const float g[3], float vx, float vy,
                                              float vz, float kn, float kd, float kt, float mu, float& depth,
                                              float fn_pad[3], float ft_pad[3]) {
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
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        fn_pad[a] = fmaf(r[a], fn[0], fmaf(r[3 + a], fn[1], r[6 + a] * fn[2]));
        ft_pad[a] = fmaf(r[a], ft[0], fmaf(r[3 + a], ft[1], r[6 + a] * ft[2]));
    }
}

// All T taxels of one pad by ONE warp (see the file comment); NP taxels per lane in
// flight.  The pad's pose / twist / outputs are addressed directly: depth[t],
// f_n[3t..3t+2], f_t[3t..3t+2], wrench[0..5] (wrench may be NULL); parameters come from
// entry pi of prm; id selects the object's SDF (out of range: NaN outputs and an error flag).
template <int NP>
__device__ __forceinline__ void pad_taxels_by_warp(const SdfTable& tab, const Params4& prm, int pi, int id, int T,
                                                   const float* __restrict__ taxels, const float* __restrict__ pose7,
                                                   const float* __restrict__ twist6, float* __restrict__ depth,
                                                   float* __restrict__ f_n, float* __restrict__ f_t,
                                                   float* __restrict__ wrench) {
    const int lane = threadIdx.x & 31;
    if (id < 0 || id >= tab.count) {
        const float qnan = __int_as_float(0x7fc00000);
        for (int t = lane; t < T; t += 32) {
            depth[t] = qnan;
#pragma unroll
            for (int a = 0; a < 3; ++a) { f_n[t * 3 + a] = qnan; f_t[t * 3 + a] = qnan; }
        }
        if (wrench != nullptr && lane < 6) wrench[lane] = qnan;
        if (lane == 0) raise_dev_error(TACSL_DEVERR_BAD_OBJ_ID);
        return;
    }
    const DevSdf& S = tab.s[id];
    Pose Pz;
    load_pose(pose7, twist6, Pz);
    const float kn = __ldg(prm.k_n + pi), kd = __ldg(prm.k_d + pi), kt = __ldg(prm.k_t + pi),
                mu = __ldg(prm.mu + pi);
    const uint64_t pol = policy_evict_last();
    const int n0 = S.n0, n01 = S.n0 * S.n1;
    const float* r = Pz.r;
    // A taxel that does not penetrate (phi >= 0, out of the domain, or NaN) has depth 0
    // and zero forces, whose pad-frame image R^T (0, 0, 0) carries the signs of R: the
    // same words contact_force writes for it.  It adds nothing to the wrench.
    float z[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) z[a] = fmaf(r[a], 0.f, fmaf(r[3 + a], 0.f, r[6 + a] * 0.f));
    // lane l < 24 writes floats 4l .. 4l+3 of a slot's 96 force floats: components (4l + i) % 3
    const int m0 = (4 * lane) % 3;   // component of this lane's first float; then m0+1, m0+2, m0 (mod 3)
    const float za = m0 == 0 ? z[0] : (m0 == 1 ? z[1] : z[2]);
    const float zb = m0 == 0 ? z[1] : (m0 == 1 ? z[2] : z[0]);
    const float zc = m0 == 0 ? z[2] : (m0 == 1 ? z[0] : z[1]);
    const float4 zq = make_float4(za, zb, zc, za);
    // whole-chunk stores where the pad's three output rows start 16-byte aligned (a slot
    // is 32 taxels, so the slots keep that alignment)
    const bool out16 = ((reinterpret_cast<uintptr_t>(depth) | reinterpret_cast<uintptr_t>(f_n) |
                         reinterpret_cast<uintptr_t>(f_t)) & 15u) == 0u;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // the round loop runs the same number of times on every lane (its body votes)
    for (int round = 0; round < T; round += 32 * NP) {
        const int t0 = round + lane;
        // pass 1, every lane: NP posed taxels and phi from their 8-node cells (all NP
        // gathers in flight together); the outputs of the taxels that do not penetrate
        float p[NP][3], phi8[NP];
        GridPos gp[NP];
        unsigned pen[NP];   // per slot u: the lanes whose taxel t0 - lane + 32u + (that lane) penetrates
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int t = t0 + 32 * u;
            const bool on = t < T;
            const int tt = on ? t : 0;
            p[u][0] = __ldg(taxels + 3 * tt);
            p[u][1] = __ldg(taxels + 3 * tt + 1);
            p[u][2] = __ldg(taxels + 3 * tt + 2);
            const float xo = fmaf(r[0], p[u][0], fmaf(r[1], p[u][1], fmaf(r[2], p[u][2], Pz.t[0])));
            const float yo = fmaf(r[3], p[u][0], fmaf(r[4], p[u][1], fmaf(r[5], p[u][2], Pz.t[1])));
            const float zo = fmaf(r[6], p[u][0], fmaf(r[7], p[u][1], fmaf(r[8], p[u][2], Pz.t[2])));
            gp[u] = grid_pos(S, xo, yo, zo);
            gp[u].inside = gp[u].inside && on;
        }
#pragma unroll
        for (int u = 0; u < NP; ++u)
            phi8[u] = gp[u].inside ? phi_cell8(S, gp[u], pol) : __int_as_float(0x7f800000);
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int t = t0 + 32 * u;
            const bool in_contact = gp[u].inside && phi8[u] < 0.f;
            const int slot = round + 32 * u;
            if (out16 && slot + 32 <= T) {
                // the slot's 32 taxels as whole 16-byte chunks, all with the no-contact
                // words; pass 2 then rewrites the penetrating ones (after a warp barrier)
                if (lane < 8) *reinterpret_cast<float4*>(depth + slot + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
                if (lane < 24) {
                    *reinterpret_cast<float4*>(f_n + 3 * slot + 4 * lane) = zq;
                    *reinterpret_cast<float4*>(f_t + 3 * slot + 4 * lane) = zq;
                }
            } else if (t < T && !in_contact) {
                depth[t] = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a) { f_n[t * 3 + a] = z[a]; f_t[t * 3 + a] = z[a]; }
            }
            pen[u] = __ballot_sync(0xffffffffu, in_contact);
        }
        __syncwarp();   // the chunk stores above come before pass 2's stores to the same words
        // pass 2: the penetrating taxels of this round, compacted over the lanes (slot-major,
        // lane-minor, so the work is deterministic): the 27-node window gives the gradient
        // and the same phi, then the force law
        int first[NP];   // index of slot u's first job
        int n_pen = 0;
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            first[u] = n_pen;
            n_pen += __popc(pen[u]);
        }
        for (int j0 = 0; j0 < n_pen; j0 += 32) {
            const int j = j0 + lane;
            float c6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // this lane's job: its wrench terms
            if (j < n_pen) {
                int u = 0, rank = j;
#pragma unroll
                for (int v = 0; v + 1 < NP; ++v)
                    if (u == v && rank >= __popc(pen[v])) { rank -= __popc(pen[v]); u = v + 1; }
                unsigned mk = pen[0];
#pragma unroll
                for (int v = 1; v < NP; ++v) mk = (u == v) ? pen[v] : mk;
                const int t = round + 32 * u + nth_set_bit(mk, rank);
                float q3[3];
                q3[0] = __ldg(taxels + 3 * t);
                q3[1] = __ldg(taxels + 3 * t + 1);
                q3[2] = __ldg(taxels + 3 * t + 2);
                // the posed point, with the same operations as pass 1, and its relative velocity
                const float xo = fmaf(r[0], q3[0], fmaf(r[1], q3[1], fmaf(r[2], q3[2], Pz.t[0])));
                const float yo = fmaf(r[3], q3[0], fmaf(r[4], q3[1], fmaf(r[5], q3[2], Pz.t[1])));
                const float zo = fmaf(r[6], q3[0], fmaf(r[7], q3[1], fmaf(r[8], q3[2], Pz.t[2])));
                const GridPos g3 = grid_pos(S, xo, yo, zo);
                const float vx = Pz.v[0] + (Pz.w[1] * zo - Pz.w[2] * yo);
                const float vy = Pz.v[1] + (Pz.w[2] * xo - Pz.w[0] * zo);
                const float vz = Pz.v[2] + (Pz.w[0] * yo - Pz.w[1] * xo);
                Stencil q;
                q.inside = true;
                int bx, by, bz;
                axis_weights(g3.ux, S.n0, bx, q.cx, q.dx);
                axis_weights(g3.uy, S.n1, by, q.cy, q.dy);
                axis_weights(g3.uz, S.n2, bz, q.cz, q.dz);
                q.base = S.data + (static_cast<int64_t>(bz) * n01 + static_cast<int64_t>(by) * n0 + bx);
                float v[3][3][3];
                stencil_load(q, n0, n01, pol, v);
                float phi, g[3];
                stencil_fold(q, v, S.inv_h, phi, g);
                float dep, fn[3], ft[3];
                contact_force(r, phi, g, vx, vy, vz, kn, kd, kt, mu, dep, fn, ft);
                depth[t] = dep;
#pragma unroll
                for (int a = 0; a < 3; ++a) { f_n[t * 3 + a] = fn[a]; f_t[t * 3 + a] = ft[a]; }
                const float fx = fn[0] + ft[0], fy = fn[1] + ft[1], fz = fn[2] + ft[2];
                c6[0] = fx; c6[1] = fy; c6[2] = fz;
                c6[3] = q3[1] * fz - q3[2] * fy;
                c6[4] = q3[2] * fx - q3[0] * fz;
                c6[5] = q3[0] * fy - q3[1] * fx;
            }
            // Each taxel's terms go back to the lane that owns it (taxel index mod 32), which
            // adds them in increasing taxel order: the wrench's summation order does not
            // depend on NP or on how the jobs were dealt.
#pragma unroll
            for (int u = 0; u < NP; ++u) {
                const int job = first[u] + __popc(pen[u] & ((1u << lane) - 1u));
                const bool here = ((pen[u] >> lane) & 1u) && job >= j0 && job < j0 + 32;
                const int from = here ? job - j0 : lane;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const float x = __shfl_sync(0xffffffffu, c6[k], from);
                    if (here) acc[k] += x;
                }
            }
        }
    }
    if (wrench != nullptr) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
        }
        if (lane < 6) {
            float w = acc[0];
#pragma unroll
            for (int k = 1; k < 6; ++k) w = (lane == k) ? acc[k] : w;
            wrench[lane] = w;
        }
    }
}

// Pad b = (env b / P, slot b % P) of a uniform batch: T taxels per pad, outputs at b*T.
template <int NP>
__device__ __forceinline__ void pad_by_warp(const SdfTable& tab, const Params4& prm, int P, int T,
                                            const float* __restrict__ taxels, const int32_t* __restrict__ obj_id,
                                            const float* __restrict__ pad_pose, const float* __restrict__ pad_twist,
                                            float* __restrict__ depth, float* __restrict__ f_n,
                                            float* __restrict__ f_t, float* __restrict__ wrench, int64_t b) {
    const int64_t e = b / P;
    const int64_t o = b * T;
    pad_taxels_by_warp<NP>(tab, prm, prm.count == 1 ? 0 : static_cast<int>(e), __ldg(obj_id + e), T, taxels,
                           pad_pose + b * 7, pad_twist + b * 6, depth + o, f_n + o * 3, f_t + o * 3,
                           wrench != nullptr ? wrench + b * 6 : nullptr);
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

// One warp per pad and per CTA, grid-stride over pads; registers capped for 20 CTAs/SM
// (96, no spills: 0.101 -> 0.098 ms at 4096 envs; 24 CTAs spill and run slower).
__global__ void __launch_bounds__(32, 20) penalty_kernel(const SdfTable tab, const Params4 prm, int64_t B, int P, int T,
                                                      const float* __restrict__ taxels,
                                                      const int32_t* __restrict__ obj_id,
                                                      const float* __restrict__ pad_pose,
                                                      const float* __restrict__ pad_twist, float* __restrict__ depth,
                                                      float* __restrict__ f_n, float* __restrict__ f_t,
                                                      float* __restrict__ wrench) {
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x)
        pad_by_warp<4>(tab, prm, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t, wrench, b);
}

// Wrench of given force fields: one block per pad, fixed-order block reduction.
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

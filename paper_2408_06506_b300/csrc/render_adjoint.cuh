// Adjoint of the depth render w.r.t. the pad poses (the pose -> depth -> image chain of
// sensor calibration, App. B of arXiv 2408.06506, through the column camera of
// Sec. III-B).
//
// A column that meets the object at z_hit in (-z_max, 0) reads D = d0 + z_hit, where
// phi(R p + t) = 0 at p = (x_i, y_j, z_hit).  Differentiating that identity (implicit
// function theorem): dD = -(grad phi . (dR p + dt)) / phi_z with phi_z = grad phi . R e_z,
// grad phi the analytic gradient of the trilinear interpolant in the hit's cell.  So a
// pixel with upstream gradient g adds s grad phi to dL/dt and s grad phi p^T to dL/dR,
// s = -g / phi_z.  No derivative: misses (D >= d0), columns clamped at the bottom of the
// camera's range (D <= d0 - z_max), grazing columns (|phi_z| < 0.05) and hits outside the
// grid's domain.  dL/dR is mapped to the raw quaternion through its normalisation.
//
// Launch: CTA clusters of C CTAs per pad, C chosen on the host so that the launch fills
// whole waves of resident CTAs (C = 1 when the batch alone does).  The C CTAs take
// contiguous pixel ranges of the pad's image; each warp of a CTA walks its share of the
// range in passes of 512 pixels (four coalesced float4 loads per lane), lists the pass's
// hit columns in its own slice of shared memory in a fixed order (a prefix sum of the
// lanes' counts by shuffles), and then its 32 lanes take the list entries e = lane,
// lane + 32, ...: the upstream gradient (read only at hit columns) and the SDF cell of
// each hit are gathered 32 at a time instead of one after another by the lane whose
// pixels hit (hits come in contact patches, so a few lanes held most of a warp's hits).
// The warps never wait for one another inside the walk.  Each CTA reduces its 12 sums
// (t, R) in a fixed order (shuffles, then warps in order); the cluster's rank 0 reads
// the other ranks' sums from their shared memory (DSMEM) in rank order after a cluster
// barrier, so the result does not depend on scheduling.
#pragma once

#include "adjoint.cuh"
#include "common.cuh"
#include "render.cuh"
#include "taxel.cuh"

namespace tacsl {

constexpr int kRenderAdjThreads = 256;
constexpr int kRenderAdjUnroll = 4;     // float4 loads in flight per lane
constexpr int kRenderAdjPass = 4 * kRenderAdjUnroll * 32;   // pixels per warp pass
constexpr int kRenderAdjMaxCluster = 8;
constexpr float kGrazing = 0.05f;   // |d phi / dz| below this: no derivative (grazing column)

struct RenderAdjointArgs {
    SdfTable tab;
    int64_t B;
    int P;
    int cluster;          // CTAs per pad (the launch's cluster size)
    const int32_t* obj_id;
    const float* pad_pose;
    CameraArgs cam;
    const float* depth;   // [B][H][W]
    const float* g_depth; // [B][H][W]
    float* grad_pose;     // [B][7]
};

__device__ __forceinline__ uint32_t cluster_cta_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Float at the same shared-memory offset in CTA `rank` of this cluster.
__device__ __forceinline__ float ld_cluster_f32(const float* smem_ptr, uint32_t rank) {
    const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(smem_ptr));
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
    return v;
}

// One hit pixel's contribution: acc[0..2] += s grad phi, acc[3 + 3a + b] += s grad_a p_b.
__device__ __forceinline__ void render_pixel_adjoint(const DevSdf& S, const float (&r)[9], const float (&t)[3],
                                                     float px, float py, float z, float g, uint64_t pol,
                                                     float (&acc)[12]) {
    const float x = fmaf(r[0], px, fmaf(r[1], py, fmaf(r[2], z, t[0])));
    const float y = fmaf(r[3], px, fmaf(r[4], py, fmaf(r[5], z, t[1])));
    const float w = fmaf(r[6], px, fmaf(r[7], py, fmaf(r[8], z, t[2])));
    const GridPos gp = grid_pos(S, x, y, w);
    if (!gp.inside) return;
    const int ix = min(static_cast<int>(floorf(gp.ux)), S.n0 - 2);
    const int iy = min(static_cast<int>(floorf(gp.uy)), S.n1 - 2);
    const int iz = min(static_cast<int>(floorf(gp.uz)), S.n2 - 2);
    const float fx = gp.ux - static_cast<float>(ix), fy = gp.uy - static_cast<float>(iy),
                fz = gp.uz - static_cast<float>(iz);
    const int n0 = S.n0, n01 = S.n0 * S.n1;
    const float* b = S.data + (static_cast<int64_t>(iz) * n01 + static_cast<int64_t>(iy) * n0 + ix);
    float v[2][2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) v[k][j][i] = ldg_f_hint(b + k * n01 + j * n0 + i, pol);
    // d phi / d f per axis: differences along the axis, interpolated across the other two
    const float wx[2] = {1.f - fx, fx}, wy[2] = {1.f - fy, fy}, wz[2] = {1.f - fz, fz};
    float dfx = 0.f, dfy = 0.f, dfz = 0.f;
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int j = 0; j < 2; ++j) dfx = fmaf(wz[k] * wy[j], v[k][j][1] - v[k][j][0], dfx);
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int i = 0; i < 2; ++i) dfy = fmaf(wz[k] * wx[i], v[k][1][i] - v[k][0][i], dfy);
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) dfz = fmaf(wy[j] * wx[i], v[1][j][i] - v[0][j][i], dfz);
    const float gx = dfx * S.inv_h, gy = dfy * S.inv_h, gz = dfz * S.inv_h;
    const float phi_z = fmaf(gx, r[2], fmaf(gy, r[5], gz * r[8]));
    if (!(fabsf(phi_z) >= kGrazing)) return;
    const float s = -g / phi_z;
    const float sg[3] = {s * gx, s * gy, s * gz};
    const float p[3] = {px, py, z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] += sg[a];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[3 + 3 * a + c] = fmaf(sg[a], p[c], acc[3 + 3 * a + c]);
    }
}

__global__ void __launch_bounds__(kRenderAdjThreads, 4) render_adjoint_kernel(const RenderAdjointArgs A) {
    __shared__ float warp_sum[kRenderAdjThreads / 32][12];
    __shared__ float cta_sum[12];
    __shared__ uint16_t hit_k[kRenderAdjThreads / 32][kRenderAdjPass];   // a pass's hits, per warp
    __shared__ float hit_d[kRenderAdjThreads / 32][kRenderAdjPass];
    const int C = A.cluster;
    const int64_t b = static_cast<int64_t>(blockIdx.x) / C;
    const uint32_t rank = C > 1 ? cluster_cta_rank() : 0u;
    const int id = __ldg(A.obj_id + static_cast<int>(b / A.P));
    const bool bad = id < 0 || id >= A.tab.count;
    const int warp = static_cast<int>(threadIdx.x >> 5), lane = static_cast<int>(threadIdx.x & 31);
    float acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.f;
    __shared__ float rt_s[12];              // the pad's R (row-major) and t, one copy per CTA
    if (!bad && threadIdx.x == 0) {
        const float* pose = A.pad_pose + b * 7;
        quat_to_rot(__ldg(pose + 3), __ldg(pose + 4), __ldg(pose + 5), __ldg(pose + 6), rt_s);
        rt_s[9] = __ldg(pose);
        rt_s[10] = __ldg(pose + 1);
        rt_s[11] = __ldg(pose + 2);
    }
    __syncthreads();
    if (!bad) {
        const DevSdf& S = A.tab.s[id];
        const CameraArgs& cam = A.cam;
        const int HW = cam.H * cam.W;            // a multiple of 4 (W is)
        const float bottom = cam.d0 - cam.z_max;
        const int n4 = HW >> 2;
        const int beg = static_cast<int>(static_cast<int64_t>(n4) * rank / C);
        const int end = static_cast<int>(static_cast<int64_t>(n4) * (rank + 1) / C);
        const float* G = A.g_depth + b * HW;
        const float4* D4 = reinterpret_cast<const float4*>(A.depth + b * HW);
        const uint64_t pol = policy_evict_last();
        float r[9], t[3];
#pragma unroll
        for (int q = 0; q < 9; ++q) r[q] = rt_s[q];
#pragma unroll
        for (int q = 0; q < 3; ++q) t[q] = rt_s[9 + q];
        uint16_t* wk = hit_k[warp];
        float* wd = hit_d[warp];
        constexpr int kQ = kRenderAdjPass / 4;   // float4 per pass
        // pass p of the CTA's range covers float4 beg + p * kQ ...; warp w takes p = w, w + 8, ...
        for (int q0 = beg + warp * kQ; q0 < end; q0 += (kRenderAdjThreads / 32) * kQ) {
            float4 dv[kRenderAdjUnroll];
#pragma unroll
            for (int u = 0; u < kRenderAdjUnroll; ++u) {
                const int q = q0 + u * 32 + lane;
                dv[u] = q < end ? __ldcs(D4 + q) : make_float4(cam.d0, cam.d0, cam.d0, cam.d0);
            }
            uint32_t hits = 0;
#pragma unroll
            for (int u = 0; u < kRenderAdjUnroll; ++u) {
                const float c4v[4] = {dv[u].x, dv[u].y, dv[u].z, dv[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (c4v[c] < cam.d0 && c4v[c] > bottom) hits |= 1u << (4 * u + c);
            }
            if (__ballot_sync(0xffffffffu, hits != 0u) == 0u) continue;
            // the pass's hits listed in (lane, u, c) order: prefix sum of the lanes' counts
            const int n = __popc(hits);
            int incl = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            int pos = incl - n;
#pragma unroll
            for (int u = 0; u < kRenderAdjUnroll; ++u) {
                const float c4v[4] = {dv[u].x, dv[u].y, dv[u].z, dv[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (hits & (1u << (4 * u + c))) {
                        wk[pos] = static_cast<uint16_t>(4 * (u * 32 + lane) + c);
                        wd[pos] = c4v[c];
                        ++pos;
                    }
            }
            __syncwarp();
            for (int e = lane; e < total; e += 32) {
                const int k = 4 * q0 + wk[e];            // pixel index in the image
                const float g = __ldcs(G + k);
                if (g == 0.f) continue;
                const int j = k / cam.W, i = k - j * cam.W;
                const float px = fmaf(static_cast<float>(i), cam.pitch_x, cam.x0);
                const float py = fmaf(static_cast<float>(j), cam.pitch_y, cam.y0);
                render_pixel_adjoint(S, r, t, px, py, wd[e] - cam.d0, g, pol, acc);
            }
            __syncwarp();          // the list is rewritten by the next pass
        }
    }
    // CTA reduction in a fixed order: lanes by xor shuffles, then warps in index order
#pragma unroll
    for (int k = 0; k < 12; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) warp_sum[warp][k] = acc[k];
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kRenderAdjThreads / 32; ++w) s += warp_sum[w][threadIdx.x];
        cta_sum[threadIdx.x] = s;
    }
    if (C > 1) cluster_sync_all();   // every rank's cta_sum is written (and stays until the second barrier)
    else __syncthreads();
    if (rank == 0 && threadIdx.x == 0) {
        float tot[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) tot[k] = cta_sum[k];
        for (int q = 1; q < C; ++q)
#pragma unroll
            for (int k = 0; k < 12; ++k) tot[k] += ld_cluster_f32(&cta_sum[k], static_cast<uint32_t>(q));
        float* out = A.grad_pose + b * 7;
        if (bad) {
            const float nan = __int_as_float(0x7fc00000);
#pragma unroll
            for (int k = 0; k < 7; ++k) out[k] = nan;
            raise_dev_error(TACSL_DEVERR_BAD_OBJ_ID);
        } else {
            const float* pose = A.pad_pose + b * 7;
            const float q4[4] = {__ldg(pose + 3), __ldg(pose + 4), __ldg(pose + 5), __ldg(pose + 6)};
            float gq[4];
            quat_backward(q4, tot + 3, gq);
            out[0] = tot[0];
            out[1] = tot[1];
            out[2] = tot[2];
#pragma unroll
            for (int k = 0; k < 4; ++k) out[3 + k] = gq[k];
        }
    }
    if (C > 1) cluster_sync_all();   // no CTA leaves while rank 0 may still read its shared memory
}

}  // namespace tacsl

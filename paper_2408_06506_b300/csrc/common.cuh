// Device-side building blocks shared by the tactile-step kernels (sm_103a).
//
// - inline-PTX wrappers for mbarriers and the bulk asynchronous copy engine
//   (cp.async.bulk, the 1-D form of TMA), used to stream depth maps through
//   shared memory and RGB tiles back out;
// - the device error word and bounded-wait helpers;
// - the SDF descriptor table passed by value as a kernel parameter;
// - the pose helpers and the fixed-order block reduction of pad wrenches.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tacsl.h"

namespace tacsl {

// ---------------------------------------------------------------------------
// Error word (one per device; read back by tacsl_check_errors)
// ---------------------------------------------------------------------------
__device__ unsigned int g_dev_err;

__device__ __forceinline__ void raise_dev_error(unsigned int bit) { atomicOr(&g_dev_err, bit); }

// ---------------------------------------------------------------------------
// SDF table: all grids of one call, by value in the kernel's parameter space
// ---------------------------------------------------------------------------
struct DevSdf {
    const float* data;
    int n0, n1, n2;
    float ox, oy, oz;   // origin
    float inv_h;        // 1 / voxel
    float h;            // voxel
};

struct SdfTable {
    DevSdf s[TACSL_MAX_SDF];
    int count;
};

struct Params4 {      // contact parameters (device arrays, count 1 or E)
    const float* k_n;
    const float* k_d;
    const float* k_t;
    const float* mu;
    int count;
};

// ---------------------------------------------------------------------------
// Shared-memory / async-copy PTX
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of a barrier phase.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the barrier's phase with the given parity has completed, for at most
// ~`limit_ns` nanoseconds.  Returns false on timeout (the caller then aborts).  A phase
// already complete costs one non-blocking test.  Otherwise the wait polls with try_wait
// (which may suspend the thread in hardware) and reads the clock every 64 polls; limits
// below 1 ms (tests of the timeout path) poll without suspending and read the clock every
// time, so that a wait longer than the limit reliably gives up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    if (limit_ns < 1000000ull) {
        for (;;) {
            if (mbar_test(bar, parity)) return true;
            if (global_timer_ns() - t0 > limit_ns) return false;
        }
    }
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// L2 eviction-priority policies for cache hints (streams leave L2 first; data re-read
// across the step - SDF grids, shading coefficients - stay).
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float4 ldg_f4_hint(const float4* p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ float ldg_f_hint(const float* p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

// Bulk copy global -> shared::cta, completion counted on an mbarrier (bytes % 16 == 0,
// both addresses 16-byte aligned), with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}

// The same without a cache hint.
__device__ __forceinline__ void bulk_g2s_nohint(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Bulk copy shared::cta -> global (bulk-group completion), with an L2 cache policy.
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes, uint64_t pol) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(src), "r"(bytes), "l"(pol)
                 : "memory");
}

// Named barrier over the first `nthreads` threads (id 1..15; id 0 is __syncthreads).
__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Make this thread's generic-proxy shared-memory writes visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Pose helpers (FP32)
// ---------------------------------------------------------------------------
struct Pose {
    float r[9];   // row-major rotation, pad -> object
    float t[3];
    float v[3], w[3];
};

// Rotation of the normalised quaternion (qw, qx, qy, qz).
__device__ __forceinline__ void quat_to_rot(float qw, float qx, float qy, float qz, float* r) {
    const float s = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= s; qx *= s; qy *= s; qz *= s;
    r[0] = 1.f - 2.f * (qy * qy + qz * qz); r[1] = 2.f * (qx * qy - qw * qz);       r[2] = 2.f * (qx * qz + qw * qy);
    r[3] = 2.f * (qx * qy + qw * qz);       r[4] = 1.f - 2.f * (qx * qx + qz * qz); r[5] = 2.f * (qy * qz - qw * qx);
    r[6] = 2.f * (qx * qz - qw * qy);       r[7] = 2.f * (qy * qz + qw * qx);       r[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

__device__ __forceinline__ void load_pose(const float* __restrict__ pose7, const float* __restrict__ twist6,
                                          Pose& P) {
    quat_to_rot(__ldg(pose7 + 3), __ldg(pose7 + 4), __ldg(pose7 + 5), __ldg(pose7 + 6), P.r);
    P.t[0] = __ldg(pose7 + 0); P.t[1] = __ldg(pose7 + 1); P.t[2] = __ldg(pose7 + 2);
    P.v[0] = __ldg(twist6 + 0); P.v[1] = __ldg(twist6 + 1); P.v[2] = __ldg(twist6 + 2);
    P.w[0] = __ldg(twist6 + 3); P.w[1] = __ldg(twist6 + 4); P.w[2] = __ldg(twist6 + 5);
}

// ---------------------------------------------------------------------------
// Fixed-order block reduction of 6 floats (warp xor-tree, then warps in order).
// `scratch` holds NWARPS*6 floats.  Result valid in thread 0.
// ---------------------------------------------------------------------------
// bar_id = 0 synchronises the whole block; otherwise a named barrier over the first
// NWARPS warps (lets the fused kernel reduce without its producer warp).
template <int NWARPS>
__device__ __forceinline__ void group_sync(int bar_id) {
    if (bar_id == 0)
        __syncthreads();
    else
        named_barrier(bar_id, NWARPS * 32);
}

template <int NWARPS>
__device__ __forceinline__ void block_sum6(float (&a)[6], float* scratch, int bar_id = 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) scratch[warp * 6 + k] = a[k];
    }
    group_sync<NWARPS>(bar_id);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float s = scratch[k];
            for (int w = 1; w < NWARPS; ++w) s += scratch[w * 6 + k];
            a[k] = s;
        }
    }
}

}  // namespace tacsl

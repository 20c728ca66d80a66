// libtacsl.so -- host side of the C ABI declared in include/tacsl.h and
// include/tacsl_batch.h.
//
// Every entry point validates its host-visible arguments, builds the kernel
// parameter structs (the SDF table travels by value in the launch), picks the launch
// shape for this device and enqueues its kernel(s) on the caller's stream.  Nothing
// here allocates device memory; tacsl_check_errors, tacsl_batch_autotune and the
// graph set-up synchronise.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "adjoint.cuh"
#include "batch.cuh"
#include "common.cuh"
#include "render.cuh"
#include "render_adjoint.cuh"
#include "shade.cuh"
#include "taxel.cuh"
#include "tacsl_batch.h"
#include "tacsl_grad.h"

namespace tacsl {
namespace {

thread_local char g_err_msg[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err_msg, sizeof(g_err_msg), fmt, ap);
    va_end(ap);
    return code;
}

int ok() {
    g_err_msg[0] = '\0';
    return TACSL_OK;
}

int check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
    return ok();
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Per-device facts, queried once per device.
struct DevInfo {
    int sms = 0;
    int max_smem_optin = 0;
    bool shade_attr_set = false;
    bool batch_shade_attr_set = false;
    bool cg_attr_set = false;                   // shade_coeff_grad_kernel: dynamic shared memory
    bool in_attr_set = false;                   // shade_intensity_kernel: dynamic shared memory
    int batch_force_ctas[4] = {0, 0, 0, 0};   // resident CTAs per SM: [np == 4][dynamic]
    int render_adj_slots[9] = {};               // render adjoint: co-resident CTAs in clusters of C (index C)
    // streams and events of tacsl_tactile_step_host, created on its first call here
    cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t pipe_start = nullptr, pipe_done[3] = {nullptr, nullptr, nullptr};
    std::mutex pipe_mu;
};
constexpr int kMaxDevices = 64;
DevInfo g_dev[kMaxDevices];
std::mutex g_dev_mu;

int device_info(DevInfo** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(TACSL_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevInfo& d = g_dev[dev];
    if (d.sms == 0) {
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) {
            d.sms = 0;
            return fail(TACSL_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
        }
    }
    *out = &d;
    return TACSL_OK;
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
int build_table(const tacsl_sdf_set* set, SdfTable& tab) {
    if (set == nullptr || set->sdfs == nullptr) return fail(TACSL_ERR_INVALID_ARG, "sdf set is NULL");
    if (set->n_sdf < 1 || set->n_sdf > TACSL_MAX_SDF)
        return fail(TACSL_ERR_INVALID_ARG, "n_sdf = %d outside [1, %d]", set->n_sdf, TACSL_MAX_SDF);
    memset(&tab, 0, sizeof(tab));
    tab.count = set->n_sdf;
    for (int i = 0; i < set->n_sdf; ++i) {
        const tacsl_sdf& s = set->sdfs[i];
        if (s.data == nullptr) return fail(TACSL_ERR_INVALID_ARG, "sdf %d: data is NULL", i);
        if (!aligned(s.data, 4)) return fail(TACSL_ERR_INVALID_ARG, "sdf %d: data not 4-byte aligned", i);
        for (int a = 0; a < 3; ++a) {
            if (s.n[a] < 3) return fail(TACSL_ERR_INVALID_ARG, "sdf %d: n[%d] = %d < 3", i, a, s.n[a]);
            if (!std::isfinite(s.origin[a])) return fail(TACSL_ERR_INVALID_ARG, "sdf %d: origin not finite", i);
        }
        if ((int64_t)s.n[0] * s.n[1] * s.n[2] >= (int64_t(1) << 31))
            return fail(TACSL_ERR_UNSUPPORTED, "sdf %d: %d x %d x %d nodes exceed 2^31", i, s.n[0], s.n[1], s.n[2]);
        if (!(s.voxel > 0.f) || !std::isfinite(s.voxel) || !std::isfinite(1.f / s.voxel))
            return fail(TACSL_ERR_INVALID_ARG, "sdf %d: voxel = %g is not a positive finite size", i, s.voxel);
        DevSdf& d = tab.s[i];
        d.data = s.data;
        d.n0 = s.n[0]; d.n1 = s.n[1]; d.n2 = s.n[2];
        d.ox = s.origin[0]; d.oy = s.origin[1]; d.oz = s.origin[2];
        d.h = s.voxel;
        d.inv_h = 1.f / s.voxel;
    }
    return TACSL_OK;
}

int build_params(const tacsl_contact_params* p, int32_t E, Params4& out) {
    if (p == nullptr) return fail(TACSL_ERR_INVALID_ARG, "contact params are NULL");
    if (p->k_n == nullptr || p->k_d == nullptr || p->k_t == nullptr || p->mu == nullptr)
        return fail(TACSL_ERR_INVALID_ARG, "a contact parameter array is NULL");
    if (!(p->count == 1 || p->count == E))
        return fail(TACSL_ERR_INVALID_ARG, "contact params count = %d must be 1 or E = %d", p->count, E);
    if (!aligned(p->k_n, 4) || !aligned(p->k_d, 4) || !aligned(p->k_t, 4) || !aligned(p->mu, 4))
        return fail(TACSL_ERR_INVALID_ARG, "contact parameter arrays must be 4-byte aligned");
    out = Params4{p->k_n, p->k_d, p->k_t, p->mu, p->count};
    return TACSL_OK;
}

int check_forces_args(int32_t E, int32_t P, int32_t T, const float* taxels, const int32_t* obj_id,
                      const float* pad_pose, const float* pad_twist, const float* depth, const float* f_n,
                      const float* f_t) {
    if (E < 0 || P < 0 || T < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size (E=%d P=%d T=%d)", E, P, T);
    if (T > TACSL_MAX_TAXELS) return fail(TACSL_ERR_UNSUPPORTED, "T = %d > %d taxels per pad", T, TACSL_MAX_TAXELS);
    if ((int64_t)E * P >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "E*P >= 2^31 pads");
    const void* ptrs[] = {taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t};
    const char* names[] = {"taxels", "obj_id", "pad_pose", "pad_twist", "depth", "f_n", "f_t"};
    for (int i = 0; i < 7; ++i) {
        if (ptrs[i] == nullptr) return fail(TACSL_ERR_INVALID_ARG, "%s is NULL", names[i]);
        if (!aligned(ptrs[i], 4)) return fail(TACSL_ERR_INVALID_ARG, "%s is not 4-byte aligned", names[i]);
    }
    return TACSL_OK;
}

// The uniform image kernel's configurations: 11 compute warps + 1 producer (12 warps, 3
// per SM sub-partition, so 168 registers a thread) over 1408-pixel tiles, three images per
// ring stage; images too wide for three such stages take one image per stage.  Measured
// on 8192 images of 320 x 240 against the earlier 15 warps x 1 image: realistic maps
// 0.789 against 0.780 ms, maps whose every pixel differs 1.090 against 1.232 ms.
using UniformCfg = ShadeCfg<11, 3>;
using UniformWideCfg = ShadeCfg<11, 1>;
static_assert(UniformCfg::kTile == UniformWideCfg::kTile, "one tile size for both configurations");

constexpr uint64_t kDefaultWaitNs = 2000000000ull;   // 2 s: the limit of every barrier wait

struct ShadePlan {
    ShadeArgs a;
    int smem;
    int grid;
    bool wide;   // one image per stage
};

// Host-visible checks of the image arguments (no CUDA calls).
int check_shade_args(const tacsl_shading* sh, int64_t B, const int32_t* sensor_id, const float* depth_map,
                     const uint8_t* rgb) {
    if (sh == nullptr) return fail(TACSL_ERR_INVALID_ARG, "shading is NULL");
    if (B < 0) return fail(TACSL_ERR_INVALID_ARG, "B = %lld < 0", (long long)B);
    if (B >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "B >= 2^31 images");
    if (sh->H < 1 || sh->W < 4 || sh->W % 4 != 0)
        return fail(TACSL_ERR_INVALID_ARG, "image %d x %d: need H >= 1 and W a positive multiple of 4", sh->H, sh->W);
    if ((int64_t)sh->H * sh->W >= (int64_t(1) << 28)) return fail(TACSL_ERR_UNSUPPORTED, "image too large");
    if (sh->n_sensor < 1 || sh->n_sensor > TACSL_MAX_SENSOR)
        return fail(TACSL_ERR_INVALID_ARG, "n_sensor = %d outside [1, %d]", sh->n_sensor, TACSL_MAX_SENSOR);
    if (!(sh->pitch_x > 0.f) || !(sh->pitch_y > 0.f) || !std::isfinite(sh->pitch_x) || !std::isfinite(sh->pitch_y))
        return fail(TACSL_ERR_INVALID_ARG, "pixel pitch must be positive and finite");
    if (sh->coeffs == nullptr || !aligned(sh->coeffs, 16))
        return fail(TACSL_ERR_INVALID_ARG, "shading coeffs must be non-NULL and 16-byte aligned");
    if (B == 0) return TACSL_OK;          // no images: the per-image arrays are not read
    if (sensor_id == nullptr || !aligned(sensor_id, 4))
        return fail(TACSL_ERR_INVALID_ARG, "sensor_id must be non-NULL and 4-byte aligned");
    if (depth_map == nullptr || !aligned(depth_map, 16))
        return fail(TACSL_ERR_INVALID_ARG, "depth_map must be non-NULL and 16-byte aligned");
    if (rgb == nullptr) return fail(TACSL_ERR_INVALID_ARG, "rgb is NULL");
    return TACSL_OK;
}

// Launch plan of the image kernel on this device (arguments already checked).
int plan_shade(const tacsl_shading* sh, int64_t B, const int32_t* sensor_id, const float* depth_map,
               uint8_t* rgb, const DevInfo& dev, ShadePlan& plan) {
    ShadeArgs& a = plan.a;
    a.coeffs = sh->coeffs;
    a.sensor_id = sensor_id;
    a.depth = depth_map;
    a.rgb = rgb;
    a.B = static_cast<int>(B);
    a.H = sh->H;
    a.W = sh->W;
    a.S = sh->n_sensor;
    a.HW = sh->H * sh->W;
    a.n_tiles = (a.HW + UniformCfg::kTile - 1) / UniformCfg::kTile;
    a.cx_c = 1.f / (2.f * sh->pitch_x);
    a.cx_e = 1.f / sh->pitch_x;
    a.cy_c = 1.f / (2.f * sh->pitch_y);
    a.cy_e = 1.f / sh->pitch_y;
    a.stage_floats = UniformCfg::kTile + 2 * a.W;
    a.wait_ns = kDefaultWaitNs;
    // ring stages that fit: three images per stage when at least three stages fit, else
    // one image per stage (at least two stages)
    const int free_bytes = dev.max_smem_optin - UniformCfg::smem_bytes(0, a.stage_floats);
    int ns = free_bytes / (UniformCfg::kImages * a.stage_floats * 4);
    plan.wide = ns < 3;
    if (plan.wide) ns = (dev.max_smem_optin - UniformWideCfg::smem_bytes(0, a.stage_floats)) / (a.stage_floats * 4);
    if (ns > 12) ns = 12;
    if (ns < 2)
        return fail(TACSL_ERR_UNSUPPORTED, "image width %d too large for the shared-memory pipeline", a.W);
    a.n_stages = ns;
    if (aligned(rgb, 4))
        a.store_mode = kStoreWord;
    else
        a.store_mode = kStoreByte;
    // Images per work item: the CTAs take items round-robin, so the launch lasts about
    // ceil(items / CTAs) items of M images each (plus about 8 images' worth of item
    // switching).  M in [16, 1024] minimising that makespan - whole rounds with few item
    // switches - among the choices that leave at least 16 items per CTA where the batch
    // allows it (item times vary with the depth maps' content; many items average that
    // out); ties go to the larger M.
    const int64_t per_blk = (int64_t)a.S * a.n_tiles;
    const bool deep = ((B + 15) / 16) * per_blk >= 16LL * dev.sms;
    int M = 16;
    double best = 0.0;
    for (int m = 1024; m >= 16; --m) {
        const int64_t items = ((B + m - 1) / m) * per_blk;
        const int64_t grid = std::min<int64_t>(items, dev.sms);
        if (deep && items < 16LL * grid) continue;
        const double cost = (double)((items + grid - 1) / grid) * (double)(std::min<int64_t>(m, B) + 8);
        if (best == 0.0 || cost < best) {
            best = cost;
            M = m;
        }
    }
    const int64_t n_items = ((B + M - 1) / M) * per_blk;
    if (n_items >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "too many work items");
    a.M = M;
    a.n_items = static_cast<int>(n_items);
    plan.smem = plan.wide ? UniformWideCfg::smem_bytes(ns, a.stage_floats) : UniformCfg::smem_bytes(ns, a.stage_floats);
    plan.grid = static_cast<int>(n_items < dev.sms ? (n_items > 0 ? n_items : 1) : dev.sms);
    return TACSL_OK;
}

}  // namespace
}  // namespace tacsl

namespace tacsl {
namespace {

template <class CFG>
int launch_shade_cfg(const ShadePlan& plan, tacsl_stream_t stream) {
    if (plan.a.store_mode == kStoreWord)
        shade_kernel<CFG, kStoreWord><<<plan.grid, CFG::kThreads, plan.smem, stream>>>(plan.a);
    else
        shade_kernel<CFG, kStoreByte><<<plan.grid, CFG::kThreads, plan.smem, stream>>>(plan.a);
    return check_launch("image kernel");
}

int launch_shade(const ShadePlan& plan, DevInfo& dev, tacsl_stream_t stream) {
    if (!dev.shade_attr_set) {
        const void* kernels[] = {reinterpret_cast<const void*>(shade_kernel<UniformCfg, kStoreWord>),
                                 reinterpret_cast<const void*>(shade_kernel<UniformCfg, kStoreByte>),
                                 reinterpret_cast<const void*>(shade_kernel<UniformWideCfg, kStoreWord>),
                                 reinterpret_cast<const void*>(shade_kernel<UniformWideCfg, kStoreByte>)};
        for (const void* k : kernels) {
            const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       dev.max_smem_optin);
            if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        }
        dev.shade_attr_set = true;
    }
    return plan.wide ? launch_shade_cfg<UniformWideCfg>(plan, stream) : launch_shade_cfg<UniformCfg>(plan, stream);
}

// One warp per pad, one warp per CTA: about half the pads are in contact and take longer,
// and a CTA's registers are freed only when its last warp ends, so single-warp CTAs keep
// the SMs evenly loaded (0.115 -> 0.103 ms at 4096 envs against 8-warp CTAs).
int launch_penalty(const SdfTable& tab, const Params4& prm, int64_t B, int P, int T, const float* taxels,
                   const int32_t* obj_id, const float* pad_pose, const float* pad_twist, float* depth, float* f_n,
                   float* f_t, float* wrench, const DevInfo& dev, tacsl_stream_t stream) {
    const int grid = static_cast<int>(B < (int64_t)dev.sms * 256 ? B : (int64_t)dev.sms * 256);
    penalty_kernel<<<grid, 32, 0, stream>>>(tab, prm, B, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t,
                                             wrench);
    return check_launch("force-field kernel");
}

}  // namespace
}  // namespace tacsl

namespace tacsl {
namespace {

int check_camera(const tacsl_camera* cam, CameraArgs& c) {
    if (cam == nullptr) return fail(TACSL_ERR_INVALID_ARG, "camera is NULL");
    if (cam->H < 1 || cam->W < 4 || cam->W % 4 != 0)
        return fail(TACSL_ERR_INVALID_ARG, "camera %d x %d: need H >= 1 and W a positive multiple of 4", cam->H, cam->W);
    if ((int64_t)cam->H * cam->W >= (int64_t(1) << 28)) return fail(TACSL_ERR_UNSUPPORTED, "camera image too large");
    const float v[] = {cam->pitch_x, cam->pitch_y, cam->x0, cam->y0, cam->d0, cam->z_max};
    for (float x : v)
        if (!std::isfinite(x)) return fail(TACSL_ERR_INVALID_ARG, "camera parameters must be finite");
    if (!(cam->pitch_x > 0.f) || !(cam->pitch_y > 0.f) || !(cam->z_max > 0.f))
        return fail(TACSL_ERR_INVALID_ARG, "camera pitches and z_max must be positive");
    c = CameraArgs{cam->H, cam->W, cam->pitch_x, cam->pitch_y, cam->x0, cam->y0, cam->d0, cam->z_max};
    return TACSL_OK;
}

int launch_render(const SdfTable& tab, int64_t B, int P, const int32_t* obj_id, const float* pad_pose,
                  const CameraArgs& c, float* depth_map, const DevInfo& /*dev*/, tacsl_stream_t stream) {
    const int64_t tiles = (int64_t)((c.W + 31) / 32) * ((c.H + 7) / 8);
    if (tiles > INT32_MAX) return fail(TACSL_ERR_UNSUPPORTED, "camera image too large");
    // each block loops over images: about (tiles x 64) blocks in all, whatever the batch
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(std::min<int64_t>(B, 64)));
    render_kernel<<<grid, 256, 0, stream>>>(tab, B, P, obj_id, pad_pose, c, depth_map, nullptr, nullptr);
    return check_launch("render kernel");
}

}  // namespace
}  // namespace tacsl

using namespace tacsl;

extern "C" {

const char* tacsl_last_error(void) { return g_err_msg; }

int32_t tacsl_abi_version(void) { return 1; }

int tacsl_check_errors(tacsl_stream_t stream, uint32_t* flags, int32_t clear) {
    if (flags == nullptr) return fail(TACSL_ERR_INVALID_ARG, "flags is NULL");
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(flags, g_dev_err, sizeof(uint32_t));
    if (e == cudaSuccess && clear) {
        const uint32_t zero = 0;
        e = cudaMemcpyToSymbol(g_dev_err, &zero, sizeof(uint32_t));
    }
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "tacsl_check_errors: %s", cudaGetErrorString(e));
    return ok();
}

int tacsl_sdf_query(const tacsl_sdf_set* set, int64_t n, const float* pts, const int32_t* obj_id, float* phi,
                    float* grad, tacsl_stream_t stream) {
    if (n < 0) return fail(TACSL_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    SdfTable tab;
    int rc = build_table(set, tab);
    if (rc) return rc;
    if (n == 0) return ok();
    const void* ptrs[] = {pts, obj_id, phi, grad};
    const char* names[] = {"pts", "obj_id", "phi", "grad"};
    for (int i = 0; i < 4; ++i) {
        if (ptrs[i] == nullptr) return fail(TACSL_ERR_INVALID_ARG, "%s is NULL", names[i]);
        if (!aligned(ptrs[i], 4)) return fail(TACSL_ERR_INVALID_ARG, "%s is not 4-byte aligned", names[i]);
    }
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    const int64_t blocks_needed = (n + 255) / 256;
    const int grid = static_cast<int>(blocks_needed < (int64_t)dev->sms * 16 ? blocks_needed : (int64_t)dev->sms * 16);
    sdf_query_kernel<<<grid, 256, 0, stream>>>(tab, n, pts, obj_id, phi, grad);
    return check_launch("tacsl_sdf_query");
}

int tacsl_penalty_forces(const tacsl_sdf_set* set, const tacsl_contact_params* params, int32_t E, int32_t P,
                         int32_t T, const float* taxels, const int32_t* obj_id, const float* pad_pose,
                         const float* pad_twist, float* depth, float* f_n, float* f_t, float* wrench,
                         tacsl_stream_t stream) {
    SdfTable tab;
    Params4 prm;
    int rc = build_table(set, tab);
    if (rc) return rc;
    if ((rc = build_params(params, E, prm))) return rc;
    if (E == 0 || P == 0 || T == 0) {
        if (E < 0 || P < 0 || T < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size");
        return ok();
    }
    if ((rc = check_forces_args(E, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t))) return rc;
    if (wrench != nullptr && !aligned(wrench, 4)) return fail(TACSL_ERR_INVALID_ARG, "wrench not 4-byte aligned");
    const int64_t B = (int64_t)E * P;
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    return launch_penalty(tab, prm, B, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t, wrench, *dev,
                          stream);
}

int tacsl_pad_wrench(int64_t B, int32_t T, const float* taxels, const float* f_n, const float* f_t, float* wrench,
                     tacsl_stream_t stream) {
    if (B < 0 || T < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size (B=%lld T=%d)", (long long)B, T);
    if (B == 0) return ok();
    if (T > TACSL_MAX_TAXELS) return fail(TACSL_ERR_UNSUPPORTED, "T = %d > %d", T, TACSL_MAX_TAXELS);
    if (B >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "B >= 2^31 pads");
    if (wrench == nullptr || !aligned(wrench, 4)) return fail(TACSL_ERR_INVALID_ARG, "wrench NULL or misaligned");
    if (T > 0) {
        const void* ptrs[] = {taxels, f_n, f_t};
        const char* names[] = {"taxels", "f_n", "f_t"};
        for (int i = 0; i < 3; ++i) {
            if (ptrs[i] == nullptr) return fail(TACSL_ERR_INVALID_ARG, "%s is NULL", names[i]);
            if (!aligned(ptrs[i], 4)) return fail(TACSL_ERR_INVALID_ARG, "%s is not 4-byte aligned", names[i]);
        }
    }
    if (T <= 128)
        wrench_kernel<4><<<static_cast<unsigned>(B), 128, 0, stream>>>(B, T, taxels, f_n, f_t, wrench);
    else
        wrench_kernel<8><<<static_cast<unsigned>(B), 256, 0, stream>>>(B, T, taxels, f_n, f_t, wrench);
    return check_launch("tacsl_pad_wrench");
}

int tacsl_shade_image(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id, const float* depth_map,
                      uint8_t* rgb, tacsl_stream_t stream) {
    return tacsl_shade_image_wait_limit(shading, B, sensor_id, depth_map, rgb, 0, stream);
}

int tacsl_shade_image_wait_limit(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                                 const float* depth_map, uint8_t* rgb, uint64_t wait_ns, tacsl_stream_t stream) {
    int rc = check_shade_args(shading, B, sensor_id, depth_map, rgb);
    if (B == 0 && shading != nullptr) return ok();
    if (rc) return rc;
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadePlan plan;
    if ((rc = plan_shade(shading, B, sensor_id, depth_map, rgb, *dev, plan))) return rc;
    if (wait_ns != 0) plan.a.wait_ns = wait_ns;
    return launch_shade(plan, *dev, stream);
}

int tacsl_tactile_step(const tacsl_sdf_set* set, const tacsl_contact_params* params, int32_t E, int32_t P, int32_t T,
                       const float* taxels, const int32_t* obj_id, const float* pad_pose, const float* pad_twist,
                       float* depth, float* f_n, float* f_t, float* wrench, const tacsl_shading* shading,
                       const int32_t* sensor_id, const float* depth_map, uint8_t* rgb, tacsl_stream_t stream) {
    if (shading == nullptr)
        return tacsl_penalty_forces(set, params, E, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t,
                                    wrench, stream);
    SdfTable tab;
    Params4 prm;
    int rc = build_table(set, tab);
    if (rc) return rc;
    if ((rc = build_params(params, E, prm))) return rc;
    if (E < 0 || P < 0 || T < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size (E=%d P=%d T=%d)", E, P, T);
    if ((int64_t)E * P == 0) return ok();
    if (T > 0 && (rc = check_forces_args(E, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t))) return rc;
    if (wrench != nullptr && !aligned(wrench, 4)) return fail(TACSL_ERR_INVALID_ARG, "wrench not 4-byte aligned");
    const int64_t B = (int64_t)E * P;
    if ((rc = check_shade_args(shading, B, sensor_id, depth_map, rgb))) return rc;
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadePlan plan;
    if ((rc = plan_shade(shading, B, sensor_id, depth_map, rgb, *dev, plan))) return rc;
    if ((rc = launch_shade(plan, *dev, stream))) return rc;
    if (T == 0) return ok();
    // The image kernel wants ~all of shared memory for its stage ring and coefficient
    // tile; the force field's scattered SDF gathers want a large L1.  Two launches, each
    // with its own carve-out, beat one persistent kernel doing both.
    return launch_penalty(tab, prm, B, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t, wrench, *dev,
                          stream);
}

int tacsl_render_depth(const tacsl_sdf_set* set, int32_t E, int32_t P, const int32_t* obj_id, const float* pad_pose,
                       const tacsl_camera* camera, float* depth_map, tacsl_stream_t stream) {
    SdfTable tab;
    int rc = build_table(set, tab);
    if (rc) return rc;
    CameraArgs c;
    if ((rc = check_camera(camera, c))) return rc;
    if (E < 0 || P < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size (E=%d P=%d)", E, P);
    if ((int64_t)E * P == 0) return ok();
    if ((int64_t)E * P >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "E*P >= 2^31 pads");
    if (obj_id == nullptr || !aligned(obj_id, 4) || pad_pose == nullptr || !aligned(pad_pose, 4))
        return fail(TACSL_ERR_INVALID_ARG, "obj_id and pad_pose must be non-NULL and 4-byte aligned");
    if (depth_map == nullptr || !aligned(depth_map, 16))
        return fail(TACSL_ERR_INVALID_ARG, "depth_map must be non-NULL and 16-byte aligned");
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    return launch_render(tab, (int64_t)E * P, P, obj_id, pad_pose, c, depth_map, *dev, stream);
}

int tacsl_render_step(const tacsl_sdf_set* set, const tacsl_contact_params* params, int32_t E, int32_t P, int32_t T,
                      const float* taxels, const int32_t* obj_id, const float* pad_pose, const float* pad_twist,
                      float* depth, float* f_n, float* f_t, float* wrench, const tacsl_shading* shading,
                      const tacsl_camera* camera, const int32_t* sensor_id, float* depth_map, uint8_t* rgb,
                      tacsl_stream_t stream) {
    SdfTable tab;
    Params4 prm;
    int rc = build_table(set, tab);
    if (rc) return rc;
    if ((rc = build_params(params, E, prm))) return rc;
    CameraArgs c;
    if ((rc = check_camera(camera, c))) return rc;
    if (E < 0 || P < 0 || T < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size (E=%d P=%d T=%d)", E, P, T);
    if ((int64_t)E * P == 0) return ok();
    if (T > 0 && (rc = check_forces_args(E, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t))) return rc;
    if (wrench != nullptr && !aligned(wrench, 4)) return fail(TACSL_ERR_INVALID_ARG, "wrench not 4-byte aligned");
    if (obj_id == nullptr || pad_pose == nullptr) return fail(TACSL_ERR_INVALID_ARG, "obj_id / pad_pose is NULL");
    const int64_t B = (int64_t)E * P;
    if ((rc = check_shade_args(shading, B, sensor_id, depth_map, rgb))) return rc;
    if (shading->H != c.H || shading->W != c.W)
        return fail(TACSL_ERR_INVALID_ARG, "camera %d x %d differs from the shading model %d x %d", c.H, c.W,
                    shading->H, shading->W);
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadePlan plan;
    if ((rc = plan_shade(shading, B, sensor_id, depth_map, rgb, *dev, plan))) return rc;
    if ((rc = launch_render(tab, B, P, obj_id, pad_pose, c, depth_map, *dev, stream))) return rc;
    if ((rc = launch_shade(plan, *dev, stream))) return rc;
    if (T == 0) return ok();
    return launch_penalty(tab, prm, B, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t, wrench, *dev,
                          stream);
}

}  // extern "C"

// ===========================================================================
// Batched step over uneven pads, objects and images (include/tacsl_batch.h)
// ===========================================================================
namespace tacsl {
namespace {

constexpr int64_t kBatchHeader = 256;        // workspace bytes before the pad schedule (the counters)
constexpr int kSmemOptinSm103 = 232448;      // opt-in shared memory per block on sm_103

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

uint64_t batch_fingerprint(const tacsl_batch_desc* d, const tacsl_batch_plan& plan) {
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, &d->n_pad, sizeof(d->n_pad));
    h = fnv1a(h, &d->n_layout, sizeof(d->n_layout));
    h = fnv1a(h, &d->n_points, sizeof(d->n_points));
    if (d->n_pad > 0) {
        h = fnv1a(h, d->obj_id, sizeof(int32_t) * d->n_pad);
        h = fnv1a(h, d->layout, sizeof(int32_t) * d->n_pad);
        h = fnv1a(h, d->sensor, sizeof(int32_t) * d->n_pad);
    }
    if (d->n_layout > 0) {
        h = fnv1a(h, d->layout_first, sizeof(int64_t) * d->n_layout);
        h = fnv1a(h, d->layout_count, sizeof(int32_t) * d->n_layout);
    }
    h = fnv1a(h, plan.model_h, sizeof(int32_t) * plan.n_model);
    h = fnv1a(h, plan.model_w, sizeof(int32_t) * plan.n_model);
    return h;
}

int shade_stage_floats(int max_w) { return kShTile + 2 * max_w; }

// Workspace offset of the per-image (pad, object) list, which follows the list of each
// image's first pixel (both grouped by model, pad order within a model).
int64_t image_po_offset(const tacsl_batch_plan& p) {
    return (p.off_images + (int64_t)sizeof(int64_t) * p.n_image + 255) / 256 * 256;
}

int batch_plan(const tacsl_batch_desc* d, const tacsl_sensor_set* sensors, tacsl_batch_plan* plan,
               int64_t* taxel_offset, int64_t* pixel_offset) {
    if (d == nullptr || plan == nullptr) return fail(TACSL_ERR_INVALID_ARG, "batch description or plan is NULL");
    if (d->n_pad < 0) return fail(TACSL_ERR_INVALID_ARG, "n_pad = %d < 0", d->n_pad);
    if (d->n_pad > 0 && (d->obj_id == nullptr || d->layout == nullptr || d->sensor == nullptr))
        return fail(TACSL_ERR_INVALID_ARG, "obj_id, layout and sensor must be non-NULL");
    if (d->n_pad > 0 && d->n_layout < 1) return fail(TACSL_ERR_INVALID_ARG, "n_layout = %d < 1", d->n_layout);
    if (d->n_layout > 0 && (d->layout_first == nullptr || d->layout_count == nullptr))
        return fail(TACSL_ERR_INVALID_ARG, "layout_first and layout_count must be non-NULL");
    tacsl_batch_plan p;
    memset(&p, 0, sizeof(p));
    p.n_pad = d->n_pad;
    p.force_np = 4;
    p.force_dynamic = 1;
    bool any_image = false;
    for (int b = 0; b < d->n_pad; ++b) any_image |= d->sensor[b] >= 0;
    if (any_image) {
        if (sensors == nullptr || sensors->models == nullptr)
            return fail(TACSL_ERR_INVALID_ARG, "a pad has an image but the sensor set is NULL");
        if (sensors->n_model < 1 || sensors->n_model > TACSL_MAX_MODEL)
            return fail(TACSL_ERR_INVALID_ARG, "n_model = %d outside [1, %d]", sensors->n_model, TACSL_MAX_MODEL);
        p.n_model = sensors->n_model;
        for (int m = 0; m < p.n_model; ++m) {
            const tacsl_sensor_model& sm = sensors->models[m];
            if (sm.H < 4 || sm.W < 4 || sm.H % 4 != 0 || sm.W % 4 != 0)
                return fail(TACSL_ERR_INVALID_ARG, "sensor model %d: %d x %d, H and W must be positive multiples of 4",
                            m, sm.H, sm.W);
            if ((int64_t)sm.H * sm.W >= (int64_t(1) << 28))
                return fail(TACSL_ERR_UNSUPPORTED, "sensor model %d: image too large", m);
            p.model_h[m] = sm.H;
            p.model_w[m] = sm.W;
            p.max_w = std::max(p.max_w, sm.W);
        }
        if (shade_smem_bytes(2, shade_stage_floats(p.max_w)) > kSmemOptinSm103)
            return fail(TACSL_ERR_UNSUPPORTED, "image width %d too large for the shared-memory pipeline", p.max_w);
    }
    for (int l = 0; l < d->n_layout; ++l) {
        if (d->layout_count[l] < 1 || d->layout_count[l] > TACSL_MAX_TAXELS)
            return fail(TACSL_ERR_INVALID_ARG, "layout %d: %d taxels outside [1, %d]", l, d->layout_count[l],
                        TACSL_MAX_TAXELS);
        if (d->layout_first[l] < 0 || d->layout_first[l] + d->layout_count[l] > d->n_points)
            return fail(TACSL_ERR_INVALID_ARG, "layout %d: points [%lld, %lld) outside the pool of %lld", l,
                        (long long)d->layout_first[l], (long long)(d->layout_first[l] + d->layout_count[l]),
                        (long long)d->n_points);
    }
    std::vector<int64_t> per_model(p.n_model + 1, 0);
    int64_t taxels = 0, pixels = 0;
    for (int b = 0; b < d->n_pad; ++b) {
        const int o = d->obj_id[b], l = d->layout[b], s = d->sensor[b];
        if (o < 0 || o >= TACSL_MAX_SDF) return fail(TACSL_ERR_INVALID_ARG, "pad %d: obj_id %d out of range", b, o);
        if (l < 0 || l >= d->n_layout) return fail(TACSL_ERR_INVALID_ARG, "pad %d: layout %d out of range", b, l);
        if (s < -1 || s >= p.n_model) return fail(TACSL_ERR_INVALID_ARG, "pad %d: sensor %d out of range", b, s);
        if (taxel_offset) taxel_offset[b] = taxels;
        taxels += d->layout_count[l];
        if (s >= 0) {
            if (pixel_offset) pixel_offset[b] = pixels;
            pixels += (int64_t)p.model_h[s] * p.model_w[s];
            ++per_model[s];
            ++p.n_image;
        } else if (pixel_offset) {
            pixel_offset[b] = -1;
        }
    }
    p.n_taxel_out = taxels;
    p.n_pixel_out = pixels;
    for (int m = 0; m < p.n_model; ++m) p.model_img_begin[m + 1] = p.model_img_begin[m] + (int32_t)per_model[m];
    p.off_sched = kBatchHeader;
    p.off_images = (p.off_sched + (int64_t)sizeof(BatchPad) * p.n_pad + 255) / 256 * 256;
    p.workspace_bytes = (image_po_offset(p) + (int64_t)sizeof(int2) * p.n_image + 255) / 256 * 256;
    p.fingerprint = batch_fingerprint(d, p);
    *plan = p;
    return ok();
}

int batch_pack(const tacsl_batch_plan* plan, const tacsl_batch_desc* d, void* host) {
    if (plan == nullptr || d == nullptr || host == nullptr)
        return fail(TACSL_ERR_INVALID_ARG, "plan, description or buffer is NULL");
    if (d->n_pad != plan->n_pad || batch_fingerprint(d, *plan) != plan->fingerprint)
        return fail(TACSL_ERR_INVALID_ARG, "batch description differs from the one the plan was made for");
    unsigned char* base = static_cast<unsigned char*>(host);
    memset(base, 0, (size_t)plan->workspace_bytes);
    // pad schedule: grouped by object (the pads in flight then share one grid's touched
    // sectors in L2), largest taxel count first within an object, ties in pad order
    std::vector<int32_t> order(d->n_pad);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (d->obj_id[a] != d->obj_id[b]) return d->obj_id[a] < d->obj_id[b];
        return d->layout_count[d->layout[a]] > d->layout_count[d->layout[b]];
    });
    std::vector<int64_t> out(d->n_pad), px(d->n_pad, -1);
    int64_t t = 0, q = 0;
    for (int b = 0; b < d->n_pad; ++b) {
        out[b] = t;
        t += d->layout_count[d->layout[b]];
        if (d->sensor[b] >= 0) {
            px[b] = q;
            q += (int64_t)plan->model_h[d->sensor[b]] * plan->model_w[d->sensor[b]];
        }
    }
    BatchPad* sched = reinterpret_cast<BatchPad*>(base + plan->off_sched);
    for (int i = 0; i < d->n_pad; ++i) {
        const int b = order[i];
        const int l = d->layout[b];
        sched[i] = BatchPad{b, d->layout_count[l], d->obj_id[b], 0, d->layout_first[l], out[b]};
    }
    // image list: grouped by model, pad order within a model; each image's first pixel,
    // then (in a second array) its pad and object
    int64_t* img = reinterpret_cast<int64_t*>(base + plan->off_images);
    int2* po = reinterpret_cast<int2*>(base + image_po_offset(*plan));
    std::vector<int32_t> fill(plan->model_img_begin, plan->model_img_begin + plan->n_model);
    for (int b = 0; b < d->n_pad; ++b)
        if (d->sensor[b] >= 0) {
            const int i = fill[d->sensor[b]]++;
            img[i] = px[b];
            po[i] = make_int2(b, d->obj_id[b]);
        }
    return ok();
}

int check_batch_io_forces(const tacsl_batch_plan* plan, const void* ws, const tacsl_batch_io* io) {
    if (plan == nullptr || io == nullptr) return fail(TACSL_ERR_INVALID_ARG, "plan or io is NULL");
    if (ws == nullptr || !aligned(ws, 256)) return fail(TACSL_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    if (plan->force_np != 0 && plan->force_np != 2 && plan->force_np != 4)
        return fail(TACSL_ERR_INVALID_ARG, "force_np = %d must be 0, 2 or 4", plan->force_np);
    if (plan->n_pad == 0) return TACSL_OK;
    const void* ptrs[] = {io->taxels, io->pad_pose, io->pad_twist, io->depth, io->f_n, io->f_t};
    const char* names[] = {"taxels", "pad_pose", "pad_twist", "depth", "f_n", "f_t"};
    for (int i = 0; i < 6; ++i) {
        if (ptrs[i] == nullptr) return fail(TACSL_ERR_INVALID_ARG, "io.%s is NULL", names[i]);
        if (!aligned(ptrs[i], 4)) return fail(TACSL_ERR_INVALID_ARG, "io.%s is not 4-byte aligned", names[i]);
    }
    if (io->wrench != nullptr && !aligned(io->wrench, 4))
        return fail(TACSL_ERR_INVALID_ARG, "io.wrench is not 4-byte aligned");
    return TACSL_OK;
}

int check_batch_io_shade(const tacsl_batch_plan* plan, const void* ws, const tacsl_sensor_set* sensors,
                         const tacsl_batch_io* io) {
    if (plan == nullptr || io == nullptr) return fail(TACSL_ERR_INVALID_ARG, "plan or io is NULL");
    if (ws == nullptr || !aligned(ws, 256)) return fail(TACSL_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    if (plan->img_block != 0 && (plan->img_block < 1 || plan->img_block > 1024 ||
                                 (plan->img_block & (plan->img_block - 1)) != 0))
        return fail(TACSL_ERR_INVALID_ARG, "img_block = %d must be 0 or a power of two <= 1024", plan->img_block);
    if (plan->n_stages != 0 && (plan->n_stages < 2 || plan->n_stages > 12))
        return fail(TACSL_ERR_INVALID_ARG, "n_stages = %d must be 0 or in [2, 12]", plan->n_stages);
    if (plan->n_image == 0) return TACSL_OK;
    if (sensors == nullptr || sensors->models == nullptr) return fail(TACSL_ERR_INVALID_ARG, "sensor set is NULL");
    if (sensors->n_model != plan->n_model)
        return fail(TACSL_ERR_INVALID_ARG, "n_model = %d, the plan has %d", sensors->n_model, plan->n_model);
    for (int m = 0; m < plan->n_model; ++m) {
        const tacsl_sensor_model& sm = sensors->models[m];
        if (sm.H != plan->model_h[m] || sm.W != plan->model_w[m])
            return fail(TACSL_ERR_INVALID_ARG, "sensor model %d is %d x %d, the plan has %d x %d", m, sm.H, sm.W,
                        plan->model_h[m], plan->model_w[m]);
        if (!(sm.pitch_x > 0.f) || !(sm.pitch_y > 0.f) || !std::isfinite(sm.pitch_x) || !std::isfinite(sm.pitch_y))
            return fail(TACSL_ERR_INVALID_ARG, "sensor model %d: pixel pitch must be positive and finite", m);
        if (sm.coeffs == nullptr || !aligned(sm.coeffs, 16))
            return fail(TACSL_ERR_INVALID_ARG, "sensor model %d: coeffs NULL or not 16-byte aligned", m);
    }
    if (io->depth_map == nullptr || !aligned(io->depth_map, 16))
        return fail(TACSL_ERR_INVALID_ARG, "io.depth_map NULL or not 16-byte aligned");
    if (io->rgb == nullptr || !aligned(io->rgb, 16)) return fail(TACSL_ERR_INVALID_ARG, "io.rgb NULL or not 16-byte aligned");
    return TACSL_OK;
}

// Resident CTAs per SM of each force-kernel variant (queried once per device).
int batch_force_ctas(DevInfo& dev, int np, bool dyn, int* out) {
    const int slot = (np == 4 ? 2 : 0) + (dyn ? 1 : 0);
    if (dev.batch_force_ctas[slot] == 0) {
        int n = 0;
        cudaError_t e;
        if (np == 4)
            e = dyn ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_force_kernel<4, true>, 256, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_force_kernel<4, false>, 256, 0);
        else
            e = dyn ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_force_kernel<2, true>, 256, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_force_kernel<2, false>, 256, 0);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(e));
        dev.batch_force_ctas[slot] = n > 0 ? n : 1;
    }
    *out = dev.batch_force_ctas[slot];
    return TACSL_OK;
}

int launch_batch_forces(const tacsl_batch_plan* plan, void* ws, const SdfTable& tab, const Params4& prm,
                        const tacsl_batch_io* io, DevInfo& dev, int np, bool dyn, tacsl_stream_t stream) {
    if (plan->n_pad == 0) return ok();
    BatchForceArgs a;
    a.tab = tab;
    a.prm = prm;
    a.sched = reinterpret_cast<const BatchPad*>(static_cast<const unsigned char*>(ws) + plan->off_sched);
    a.n_pad = plan->n_pad;
    a.taxels = io->taxels;
    a.pose = io->pad_pose;
    a.twist = io->pad_twist;
    a.depth = io->depth;
    a.f_n = io->f_n;
    a.f_t = io->f_t;
    a.wrench = io->wrench;
    a.ticket = static_cast<unsigned int*>(ws);
    int ctas = 0;
    int rc = batch_force_ctas(dev, np, dyn, &ctas);
    if (rc) return rc;
    const int64_t need = (plan->n_pad + 7) / 8;
    const int grid = static_cast<int>(std::min<int64_t>(need, (int64_t)dev.sms * ctas));
    if (np == 4) {
        if (dyn) batch_force_kernel<4, true><<<grid, 256, 0, stream>>>(a);
        else batch_force_kernel<4, false><<<grid, 256, 0, stream>>>(a);
    } else {
        if (dyn) batch_force_kernel<2, true><<<grid, 256, 0, stream>>>(a);
        else batch_force_kernel<2, false><<<grid, 256, 0, stream>>>(a);
    }
    return check_launch("batched force-field kernel");
}

// Work items of the image kernel with M images per item.
int64_t batch_items(const tacsl_batch_plan* plan, int M) {
    int64_t n = 0;
    for (int m = 0; m < plan->n_model; ++m) {
        const int64_t cnt = plan->model_img_begin[m + 1] - plan->model_img_begin[m];
        const int64_t tiles = ((int64_t)plan->model_h[m] * plan->model_w[m] + kShTile - 1) / kShTile;
        n += (cnt + M - 1) / M * tiles;
    }
    return n;
}

int batch_auto_block(const tacsl_batch_plan* plan, int sms) {
    int M = 1024;
    while (M > 32 && batch_items(plan, M) < 24LL * sms) M /= 2;
    return M;
}

int batch_max_stages(const tacsl_batch_plan* plan, const DevInfo& dev) {
    const int sf = shade_stage_floats(plan->max_w);
    return std::min(12, (dev.max_smem_optin - shade_smem_bytes(0, sf)) / (sf * 4));
}

int launch_batch_shade(const tacsl_batch_plan* plan, const void* ws, const tacsl_sensor_set* sensors,
                       const tacsl_batch_io* io, DevInfo& dev, int M, int ns, tacsl_stream_t stream) {
    if (plan->n_image == 0) return ok();
    BatchShadeArgs a;
    memset(&a, 0, sizeof(a));
    a.stage_floats = shade_stage_floats(plan->max_w);
    const int ns_max = batch_max_stages(plan, dev);
    if (ns_max < 2) return fail(TACSL_ERR_UNSUPPORTED, "image width %d too large for this device", plan->max_w);
    if (M == 0) M = batch_auto_block(plan, dev.sms);
    if (ns == 0 || ns > ns_max) ns = ns_max;
    int64_t items = 0;
    for (int m = 0; m < plan->n_model; ++m) {
        const tacsl_sensor_model& sm = sensors->models[m];
        BatchModel& md = a.mdl[m];
        md.coeffs = sm.coeffs;
        md.H = sm.H;
        md.W = sm.W;
        md.HW = sm.H * sm.W;
        md.n_tiles = (md.HW + kShTile - 1) / kShTile;
        md.cx_c = 1.f / (2.f * sm.pitch_x);
        md.cx_e = 1.f / sm.pitch_x;
        md.cy_c = 1.f / (2.f * sm.pitch_y);
        md.cy_e = 1.f / sm.pitch_y;
        md.img_begin = plan->model_img_begin[m];
        md.img_end = plan->model_img_begin[m + 1];
        md.item_begin = static_cast<int>(std::min<int64_t>(items, INT32_MAX));
        items += (int64_t)(md.img_end - md.img_begin + M - 1) / M * md.n_tiles;
    }
    if (items >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "too many work items");
    a.img_px = reinterpret_cast<const int64_t*>(static_cast<const unsigned char*>(ws) + plan->off_images);
    // the image kernel's item counter: words 2-3 of the workspace header (0-1: force kernel)
    a.ticket = static_cast<unsigned int*>(const_cast<void*>(ws)) + 2;
    a.depth = io->depth_map;
    a.rgb = io->rgb;
    a.n_model = plan->n_model;
    a.M = M;
    a.n_items = static_cast<int>(items);
    a.n_stages = ns;
    if (!dev.batch_shade_attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(batch_shade_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   dev.max_smem_optin);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        dev.batch_shade_attr_set = true;
    }
    const int grid = static_cast<int>(std::min<int64_t>(items, dev.sms));
    batch_shade_kernel<<<grid, kShThreads, shade_smem_bytes(ns, a.stage_floats), stream>>>(a);
    return check_launch("batched image kernel");
}

// Everything of a batch step that needs no launch: checks, tables, device facts.
struct BatchCall {
    SdfTable tab;
    Params4 prm;
    DevInfo* dev = nullptr;
};

int batch_prepare(const tacsl_batch_plan* plan, const void* ws, const tacsl_sdf_set* set,
                  const tacsl_contact_params* params, const tacsl_sensor_set* sensors, const tacsl_batch_io* io,
                  bool forces, bool images, BatchCall& c) {
    int rc;
    if (forces) {
        if ((rc = build_table(set, c.tab))) return rc;
        if ((rc = check_batch_io_forces(plan, ws, io))) return rc;
        if ((rc = build_params(params, plan->n_pad, c.prm))) return rc;
    }
    if (images && (rc = check_batch_io_shade(plan, ws, sensors, io))) return rc;
    if ((rc = device_info(&c.dev))) return rc;
    if (forces) {
        int ctas;
        const int np = plan->force_np == 2 ? 2 : 4;
        if ((rc = batch_force_ctas(*c.dev, np, plan->force_dynamic != 0, &ctas))) return rc;
    }
    return TACSL_OK;
}

int run_batch_forces(const tacsl_batch_plan* plan, void* ws, const BatchCall& c, const tacsl_batch_io* io,
                     tacsl_stream_t stream) {
    return launch_batch_forces(plan, ws, c.tab, c.prm, io, *c.dev, plan->force_np == 2 ? 2 : 4,
                               plan->force_dynamic != 0, stream);
}

int run_batch_shade(const tacsl_batch_plan* plan, const void* ws, const tacsl_sensor_set* sensors,
                    const BatchCall& c, const tacsl_batch_io* io, tacsl_stream_t stream) {
    return launch_batch_shade(plan, ws, sensors, io, *c.dev, plan->img_block, plan->n_stages, stream);
}

// Mean time of `reps` launches after one warm-up (ms), via events on the stream.
template <class F>
int time_launches(F&& launch, int reps, tacsl_stream_t stream, float* ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaEventCreate failed");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(TACSL_ERR_CUDA, "cudaEventCreate failed");
    }
    int rc = launch();
    if (!rc) {
        cudaEventRecord(e0, stream);
        for (int r = 0; r < reps && !rc; ++r) rc = launch();
        cudaEventRecord(e1, stream);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (!rc && e != cudaSuccess) rc = fail(TACSL_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
        if (!rc) {
            cudaEventElapsedTime(ms, e0, e1);
            *ms /= reps;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Depth maps of every image of a packed batch: one render launch per camera model, over
// that model's run of the image list (pad, object, first pixel).
int launch_batch_render(const tacsl_batch_plan* plan, const void* ws, const SdfTable& tab, const CameraArgs* cams,
                        const float* pad_pose, float* depth_map, tacsl_stream_t stream) {
    const unsigned char* w = static_cast<const unsigned char*>(ws);
    const int64_t* img = reinterpret_cast<const int64_t*>(w + plan->off_images);
    const int2* po = reinterpret_cast<const int2*>(w + image_po_offset(*plan));
    for (int m = 0; m < plan->n_model; ++m) {
        const int b0 = plan->model_img_begin[m], n = plan->model_img_begin[m + 1] - b0;
        if (n == 0) continue;
        const CameraArgs& c = cams[m];
        const int64_t tiles = (int64_t)((c.W + 31) / 32) * ((c.H + 7) / 8);
        const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(std::min(n, 64)));
        render_kernel<<<grid, 256, 0, stream>>>(tab, n, 1, nullptr, pad_pose, c, depth_map, po + b0, img + b0);
        const int rc = check_launch("batched render kernel");
        if (rc) return rc;
    }
    return TACSL_OK;
}

// Host checks of tacsl_batch_render's arguments; the cameras of the models with images
// are converted into cams (n_model entries).
int check_batch_render(const tacsl_batch_plan* plan, const void* ws, const tacsl_camera* cameras,
                       const float* pad_pose, const float* depth_map, CameraArgs* cams) {
    if (plan == nullptr) return fail(TACSL_ERR_INVALID_ARG, "plan is NULL");
    if (ws == nullptr || !aligned(ws, 256)) return fail(TACSL_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    if (plan->n_image == 0) return TACSL_OK;
    if (cameras == nullptr) return fail(TACSL_ERR_INVALID_ARG, "cameras is NULL");
    for (int m = 0; m < plan->n_model; ++m) {
        if (plan->model_img_begin[m + 1] == plan->model_img_begin[m]) continue;
        const int rc = check_camera(&cameras[m], cams[m]);
        if (rc) return rc;
        if (cams[m].H != plan->model_h[m] || cams[m].W != plan->model_w[m])
            return fail(TACSL_ERR_INVALID_ARG, "camera %d is %d x %d, sensor model %d is %d x %d", m, cams[m].H,
                        cams[m].W, m, plan->model_h[m], plan->model_w[m]);
    }
    if (pad_pose == nullptr || !aligned(pad_pose, 4)) return fail(TACSL_ERR_INVALID_ARG, "pad_pose NULL or misaligned");
    if (depth_map == nullptr || !aligned(depth_map, 16))
        return fail(TACSL_ERR_INVALID_ARG, "depth_map NULL or not 16-byte aligned");
    return TACSL_OK;
}

}  // namespace
}  // namespace tacsl

extern "C" {

int tacsl_batch_render(const tacsl_batch_plan* plan, const void* workspace, const tacsl_sdf_set* set,
                       const tacsl_camera* cameras, const float* pad_pose, float* depth_map, tacsl_stream_t stream) {
    using namespace tacsl;
    CameraArgs cams[TACSL_MAX_MODEL];
    int rc = check_batch_render(plan, workspace, cameras, pad_pose, depth_map, cams);
    if (rc) return rc;
    SdfTable tab;
    if ((rc = build_table(set, tab))) return rc;
    if (plan->n_image == 0) return ok();
    if ((rc = launch_batch_render(plan, workspace, tab, cams, pad_pose, depth_map, stream))) return rc;
    return ok();
}

int tacsl_batch_plan_create(const tacsl_batch_desc* desc, const tacsl_sensor_set* sensors, tacsl_batch_plan* plan,
                            int64_t* taxel_offset, int64_t* pixel_offset) {
    return batch_plan(desc, sensors, plan, taxel_offset, pixel_offset);
}

int tacsl_batch_pack(const tacsl_batch_plan* plan, const tacsl_batch_desc* desc, void* host_workspace) {
    return batch_pack(plan, desc, host_workspace);
}

int tacsl_batch_upload(const tacsl_batch_plan* plan, const tacsl_batch_desc* desc, void* workspace,
                       tacsl_stream_t stream) {
    if (workspace == nullptr || !aligned(workspace, 256))
        return fail(TACSL_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    if (plan == nullptr) return fail(TACSL_ERR_INVALID_ARG, "plan is NULL");
    std::vector<unsigned char> host((size_t)plan->workspace_bytes);
    int rc = batch_pack(plan, desc, host.data());
    if (rc) return rc;
    // from pageable memory: the copy is staged before the call returns, so the
    // temporary buffer may go
    const cudaError_t e = cudaMemcpyAsync(workspace, host.data(), host.size(), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "workspace upload: %s", cudaGetErrorString(e));
    return ok();
}

int tacsl_batch_forces(const tacsl_batch_plan* plan, void* workspace, const tacsl_sdf_set* set,
                       const tacsl_contact_params* params, const tacsl_batch_io* io, tacsl_stream_t stream) {
    BatchCall c;
    int rc = batch_prepare(plan, workspace, set, params, nullptr, io, true, false, c);
    if (rc) return rc;
    return run_batch_forces(plan, workspace, c, io, stream);
}

int tacsl_batch_shade(const tacsl_batch_plan* plan, const void* workspace, const tacsl_sensor_set* sensors,
                      const tacsl_batch_io* io, tacsl_stream_t stream) {
    BatchCall c;
    int rc = batch_prepare(plan, workspace, nullptr, nullptr, sensors, io, false, true, c);
    if (rc) return rc;
    return run_batch_shade(plan, workspace, sensors, c, io, stream);
}

int tacsl_batch_step(const tacsl_batch_plan* plan, void* workspace, const tacsl_sdf_set* set,
                     const tacsl_contact_params* params, const tacsl_sensor_set* sensors, const tacsl_batch_io* io,
                     tacsl_stream_t stream) {
    BatchCall c;
    int rc = batch_prepare(plan, workspace, set, params, sensors, io, true, true, c);
    if (rc) return rc;
    if ((rc = run_batch_shade(plan, workspace, sensors, c, io, stream))) return rc;
    return run_batch_forces(plan, workspace, c, io, stream);
}

int tacsl_batch_autotune(tacsl_batch_plan* plan, void* workspace, const tacsl_sdf_set* set,
                         const tacsl_contact_params* params, const tacsl_sensor_set* sensors, const tacsl_batch_io* io,
                         int32_t reps, double* best_ms, tacsl_stream_t stream) {
    if (reps < 1 || reps > 1000) return fail(TACSL_ERR_INVALID_ARG, "reps = %d outside [1, 1000]", reps);
    BatchCall c;
    int rc = batch_prepare(plan, workspace, set, params, sensors, io, true, true, c);
    if (rc) return rc;
    DevInfo& dev = *c.dev;
    double total = 0.0;
    // force kernel: taxels in flight per lane x pad dealing
    if (plan->n_pad > 0) {
        float best = 0.f;
        int best_np = 4, best_dyn = 1;
        for (int np : {4, 2})
            for (int dyn : {1, 0}) {
                float ms = 0.f;
                rc = time_launches([&] { return launch_batch_forces(plan, workspace, c.tab, c.prm, io, dev, np, dyn != 0,
                                                                    stream); },
                                   reps, stream, &ms);
                if (rc) return rc;
                if (best == 0.f || ms < best) { best = ms; best_np = np; best_dyn = dyn; }
            }
        plan->force_np = best_np;
        plan->force_dynamic = best_dyn;
        total += best;
    }
    // image kernel: images per item x stages in flight
    if (plan->n_image > 0) {
        const int ns_max = batch_max_stages(plan, dev);
        if (ns_max < 2) return fail(TACSL_ERR_UNSUPPORTED, "image width %d too large for this device", plan->max_w);
        std::vector<int> stage_set = {ns_max};
        for (int s : {4, 8})
            if (s < ns_max) stage_set.push_back(s);
        float best = 0.f;
        int best_m = 0, best_ns = 0;
        for (int M = 1024; M >= 16; M /= 2) {
            if (batch_items(plan, M) < dev.sms && M != 16) continue;   // fewer items than SMs: idle SMs
            for (int ns : stage_set) {
                float ms = 0.f;
                rc = time_launches([&] { return launch_batch_shade(plan, workspace, sensors, io, dev, M, ns, stream); },
                                   reps, stream, &ms);
                if (rc) return rc;
                if (best == 0.f || ms < best) { best = ms; best_m = M; best_ns = ns; }
            }
        }
        plan->img_block = best_m;
        plan->n_stages = best_ns;
        total += best;
    }
    if (best_ms) *best_ms = total;
    return ok();
}

int tacsl_batch_graph_create(const tacsl_batch_plan* plan, void* workspace, const tacsl_sdf_set* set,
                             const tacsl_contact_params* params, const tacsl_sensor_set* sensors,
                             const tacsl_batch_io* io, tacsl_graph_t* graph) {
    if (graph == nullptr) return fail(TACSL_ERR_INVALID_ARG, "graph is NULL");
    *graph = nullptr;
    BatchCall c;
    int rc = batch_prepare(plan, workspace, set, params, sensors, io, true, true, c);
    if (rc) return rc;
    // one-time device set-up (kernel attributes) happens outside the capture
    if (plan->n_image > 0 && !c.dev->batch_shade_attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(batch_shade_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   c.dev->max_smem_optin);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        c.dev->batch_shade_attr_set = true;
    }
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return fail(TACSL_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    rc = run_batch_shade(plan, workspace, sensors, c, io, s);
    if (!rc) rc = run_batch_forces(plan, workspace, c, io, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    if (!rc && e != cudaSuccess) rc = fail(TACSL_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    if (!rc) {
        e = cudaGraphInstantiate(&exec, g, 0);
        if (e != cudaSuccess) rc = fail(TACSL_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    *graph = reinterpret_cast<tacsl_graph_t>(exec);
    return ok();
}

int tacsl_graph_launch(tacsl_graph_t graph, tacsl_stream_t stream) {
    if (graph == nullptr) return fail(TACSL_ERR_INVALID_ARG, "graph is NULL");
    const cudaError_t e = cudaGraphLaunch(reinterpret_cast<cudaGraphExec_t>(graph), stream);
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    return ok();
}

int tacsl_graph_destroy(tacsl_graph_t graph) {
    if (graph == nullptr) return ok();
    const cudaError_t e = cudaGraphExecDestroy(reinterpret_cast<cudaGraphExec_t>(graph));
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaGraphExecDestroy: %s", cudaGetErrorString(e));
    return ok();
}

}  // extern "C"

// ===========================================================================
// Batched force field without a caller-provided workspace
// ===========================================================================
//
// Some callers cannot hand the library device memory for a workspace: a real-time
// control loop where cudaMalloc / cudaFree would synchronise the device and stall the
// step, or a plug-in running inside a host application that owns every device
// allocation and allows none from its callbacks.  tacsl_batch_forces_static serves
// them: the pad schedule and the two pad counters that tacsl_batch_forces keeps in the
// caller's workspace live instead in the fixed array below, which exists on every GPU
// that loads the library until the process exits.

namespace {
constexpr int64_t kStaticScratchBytes = int64_t(2) << 20;   // 2 MiB per GPU
constexpr int kStaticMaxPads = static_cast<int>((kStaticScratchBytes - tacsl::kBatchHeader) / sizeof(tacsl::BatchPad));
}  // namespace

// Counters (first 256 bytes) and pad schedule of tacsl_batch_forces_static.  In host
// code this name only stands for the array; its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char tacsl_static_scratch[kStaticScratchBytes];

namespace tacsl {
namespace {

unsigned char g_static_host[kStaticScratchBytes];   // host image of one call's scratch
std::mutex g_static_mu;
void* g_static_dev[kMaxDevices] = {};               // device address of the array, per device

// The array's address on the current device, looked up on the first call there.
int static_scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(TACSL_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (g_static_dev[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, tacsl_static_scratch);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_static_dev[dev] = p;
    }
    *out = g_static_dev[dev];
    return TACSL_OK;
}

}  // namespace
}  // namespace tacsl

extern "C" int tacsl_batch_forces_static(const tacsl_batch_desc* desc, const tacsl_sdf_set* set,
                                         const tacsl_contact_params* params, const tacsl_batch_io* io,
                                         tacsl_stream_t stream) {
    // host-visible checks first: nothing below them touches the GPU on failure
    if (desc == nullptr || io == nullptr) return fail(TACSL_ERR_INVALID_ARG, "batch description or io is NULL");
    const int n = desc->n_pad;
    if (n < 0) return fail(TACSL_ERR_INVALID_ARG, "n_pad = %d < 0", n);
    if (n > kStaticMaxPads)
        return fail(TACSL_ERR_UNSUPPORTED, "n_pad = %d exceeds the %d pads the static scratch (%lld bytes) holds", n,
                    kStaticMaxPads, (long long)kStaticScratchBytes);
    if (n > 0 && (desc->obj_id == nullptr || desc->layout == nullptr))
        return fail(TACSL_ERR_INVALID_ARG, "obj_id and layout must be non-NULL");
    if (n > 0 && (desc->n_layout < 1 || desc->layout_first == nullptr || desc->layout_count == nullptr))
        return fail(TACSL_ERR_INVALID_ARG, "the batch needs at least one taxel layout");
    for (int l = 0; l < desc->n_layout && n > 0; ++l) {
        if (desc->layout_count[l] < 1 || desc->layout_count[l] > TACSL_MAX_TAXELS)
            return fail(TACSL_ERR_INVALID_ARG, "layout %d: %d taxels outside [1, %d]", l, desc->layout_count[l],
                        TACSL_MAX_TAXELS);
        if (desc->layout_first[l] < 0 || desc->layout_first[l] + desc->layout_count[l] > desc->n_points)
            return fail(TACSL_ERR_INVALID_ARG, "layout %d lies outside the taxel pool", l);
    }
    for (int b = 0; b < n; ++b) {
        if (desc->obj_id[b] < 0 || desc->obj_id[b] >= TACSL_MAX_SDF)
            return fail(TACSL_ERR_INVALID_ARG, "pad %d: obj_id %d out of range", b, desc->obj_id[b]);
        if (desc->layout[b] < 0 || desc->layout[b] >= desc->n_layout)
            return fail(TACSL_ERR_INVALID_ARG, "pad %d: layout %d out of range", b, desc->layout[b]);
    }
    SdfTable tab;
    Params4 prm;
    int rc = build_table(set, tab);
    if (rc) return rc;
    if ((rc = build_params(params, n, prm))) return rc;
    if (n == 0) return ok();
    const void* ptrs[] = {io->taxels, io->pad_pose, io->pad_twist, io->depth, io->f_n, io->f_t};
    const char* names[] = {"taxels", "pad_pose", "pad_twist", "depth", "f_n", "f_t"};
    for (int i = 0; i < 6; ++i) {
        if (ptrs[i] == nullptr) return fail(TACSL_ERR_INVALID_ARG, "io.%s is NULL", names[i]);
        if (!aligned(ptrs[i], 4)) return fail(TACSL_ERR_INVALID_ARG, "io.%s is not 4-byte aligned", names[i]);
    }
    if (io->wrench != nullptr && !aligned(io->wrench, 4))
        return fail(TACSL_ERR_INVALID_ARG, "io.wrench is not 4-byte aligned");

    // A captured call would record a copy from the shared host image below, which the
    // next call rewrites: a replay would then upload another call's schedule.  So the
    // call refuses to be captured (tacsl_batch_graph_create is the capturable form).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(stream, &cap);
    if (ce != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(TACSL_ERR_UNSUPPORTED, "tacsl_batch_forces_static cannot be captured in a CUDA graph");

    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    void* scratch = nullptr;
    if ((rc = static_scratch_address(&scratch))) return rc;

    // the schedule as tacsl_batch_pack lays it out (by object, largest layout first,
    // outputs packed in pad order), behind 256 zero bytes: the pad counters start every
    // call at zero
    tacsl_batch_plan p;
    memset(&p, 0, sizeof(p));
    p.n_pad = n;
    p.off_sched = kBatchHeader;
    const size_t bytes = (size_t)kBatchHeader + sizeof(BatchPad) * (size_t)n;
    std::lock_guard<std::mutex> lk(g_static_mu);
    memset(g_static_host, 0, (size_t)kBatchHeader);
    BatchPad* sched = reinterpret_cast<BatchPad*>(g_static_host + kBatchHeader);
    int64_t out = 0;
    for (int b = 0; b < n; ++b) {   // pad order first: output offsets
        const int l = desc->layout[b];
        sched[b] = BatchPad{b, desc->layout_count[l], desc->obj_id[b], 0, desc->layout_first[l], out};
        out += desc->layout_count[l];
    }
    std::stable_sort(sched, sched + n, [](const BatchPad& a, const BatchPad& c) {
        return a.obj != c.obj ? a.obj < c.obj : a.T > c.T;
    });
    // A copy from pageable host memory may be synchronous with respect to the host: CUDA
    // may first wait for the work already on `stream`, then stages the bytes into pinned
    // memory of its own before the call returns.  The host image is therefore no longer
    // read once cudaMemcpyAsync has returned, and the next call may rewrite it as soon as
    // the lock is released.  (Pinned staging of our own would be an allocation.)
    const cudaError_t e = cudaMemcpyAsync(scratch, g_static_host, bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "scratch upload: %s", cudaGetErrorString(e));
    return launch_batch_forces(&p, scratch, tab, prm, io, *dev, 4, true, stream);
}

// ===========================================================================
// Gradients (include/tacsl_grad.h)
// ===========================================================================
namespace tacsl {
namespace {

int shade_geom(const tacsl_shading* sh, ShadeGeom& G) {
    G.H = sh->H;
    G.W = sh->W;
    G.S = sh->n_sensor;
    G.HW = (int64_t)sh->H * sh->W;
    G.px = sh->pitch_x;
    G.py = sh->pitch_y;
    return TACSL_OK;
}

// Coefficient gradient (and, for the image loss, the loss map; with slopes, the pixel
// slopes of the depth gradient): the two-pixels-per-lane kernel, with 8-byte copies of
// the upstream values where that array allows them.
template <bool kMse, bool kU8, bool kSlopes>
cudaError_t coeff_grad_attr(int bytes) {
    return cudaFuncSetAttribute(shade_coeff_grad_kernel<kMse, kU8, kSlopes>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <bool kMse>
int launch_coeff_grad(const ShadeGeom& G, int64_t B, const float* coeffs, const int32_t* sensor_id,
                      const float* depth, const float* u, const float* scale, float* grad_coeffs, float* loss_map,
                      float* slopes, DevInfo& dev, tacsl_stream_t stream) {
    const int64_t tiles = (G.HW + kCgPx - 1) / kCgPx;
    if (tiles > INT32_MAX || G.HW > INT32_MAX) return fail(TACSL_ERR_UNSUPPORTED, "image too large");
    if (!dev.cg_attr_set) {
        const int bytes = static_cast<int>(kCgSmemBytes);
        cudaError_t e = coeff_grad_attr<false, false, false>(bytes);
        if (e == cudaSuccess) e = coeff_grad_attr<false, true, false>(bytes);
        if (e == cudaSuccess) e = coeff_grad_attr<true, false, false>(bytes);
        if (e == cudaSuccess) e = coeff_grad_attr<true, true, false>(bytes);
        if (e == cudaSuccess) e = coeff_grad_attr<false, false, true>(bytes);
        if (e == cudaSuccess) e = coeff_grad_attr<false, true, true>(bytes);
        if (e == cudaSuccess) e = coeff_grad_attr<true, false, true>(bytes);
        if (e == cudaSuccess) e = coeff_grad_attr<true, true, true>(bytes);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        dev.cg_attr_set = true;
    }
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(G.S));
    const bool u8 = aligned(u, 8);
    if (slopes != nullptr) {
        if (u8)
            shade_coeff_grad_kernel<kMse, true, true><<<grid, 256, kCgSmemBytes, stream>>>(
                G, B, coeffs, sensor_id, depth, u, scale, grad_coeffs, loss_map, slopes);
        else
            shade_coeff_grad_kernel<kMse, false, true><<<grid, 256, kCgSmemBytes, stream>>>(
                G, B, coeffs, sensor_id, depth, u, scale, grad_coeffs, loss_map, slopes);
    } else if (u8) {
        shade_coeff_grad_kernel<kMse, true, false><<<grid, 256, kCgSmemBytes, stream>>>(
            G, B, coeffs, sensor_id, depth, u, scale, grad_coeffs, loss_map, nullptr);
    } else {
        shade_coeff_grad_kernel<kMse, false, false><<<grid, 256, kCgSmemBytes, stream>>>(
            G, B, coeffs, sensor_id, depth, u, scale, grad_coeffs, loss_map, nullptr);
    }
    return check_launch(kMse ? "tacsl_shade_mse (loss map / coefficients)" : "tacsl_shade_adjoint (coefficients)");
}

// The depth gradient from pixel slopes: CTAs over (512-pixel strips, image chunks), the
// number of chunks chosen (as for the depth-gradient kernel) so that the waves of four
// CTAs per SM (64 registers a thread) are nearly full, with at least 8 images per CTA.
int launch_slopes_to_depth(const ShadeGeom& G, int64_t B, const int32_t* sensor_id, const float* slopes,
                           const float* scale, float* grad_depth, const DevInfo& dev, tacsl_stream_t stream) {
    const int64_t strips = (G.HW + kSdPx - 1) / kSdPx;
    if (strips > INT32_MAX || G.HW > INT32_MAX) return fail(TACSL_ERR_UNSUPPORTED, "image too large");
    const int64_t slots = 4 * (int64_t)dev.sms;
    const int64_t c_max = std::max<int64_t>(1, std::min<int64_t>((B + 7) / 8, 65535));
    int64_t chunks = 1;
    double best = 1e30;
    for (int64_t c = 1; c <= std::min<int64_t>(c_max, 64); ++c) {
        const double t = (double)((strips * c + slots - 1) / slots) / (double)c;
        if (t < best - 1e-9) {
            best = t;
            chunks = c;
        }
    }
    const int64_t chunk = (B + chunks - 1) / chunks;
    const dim3 grid(static_cast<unsigned>(strips), static_cast<unsigned>((B + chunk - 1) / chunk));
    slopes_to_depth_kernel<<<grid, 256, 0, stream>>>(G, B, chunk, sensor_id, slopes, scale, grad_depth);
    return check_launch("depth gradient from slopes");
}

// Grid of the depth-gradient kernel: (32 x 8 tiles, sensors, image chunks), with enough
// image chunks that the launch gives every SM a few CTAs even for small images.
int launch_depth_grad(bool mse, const ShadeGeom& G, int64_t B, const float* coeffs, const int32_t* sensor_id,
                      const float* depth_map, const float* u, const float* scale, float* grad_depth,
                      const DevInfo& dev, tacsl_stream_t stream) {
    const int64_t tiles = (int64_t)((G.W + kDgTx - 1) / kDgTx) * ((G.H + kDgTy - 1) / kDgTy);
    if (tiles > INT32_MAX) return fail(TACSL_ERR_UNSUPPORTED, "image too large");
    // image chunks: at least 32 images per CTA (its coefficients are loaded once), and as
    // many chunks as keep the last wave of 3 CTAs per SM nearly full
    const int64_t base = tiles * G.S, slots = 3 * (int64_t)dev.sms;
    const int64_t c_max = std::max<int64_t>(1, std::min<int64_t>((B + 31) / 32, 65535));
    int64_t chunks = 1;
    double best = 1e30;
    for (int64_t c = 1; c <= std::min<int64_t>(c_max, 64); ++c) {
        const int64_t ctas = base * c;
        const double t = (double)((ctas + slots - 1) / slots) / (double)c;   // waves x work per CTA
        if (t < best - 1e-9) {
            best = t;
            chunks = c;
        }
    }
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(G.S), static_cast<unsigned>(chunks));
    if (mse)
        shade_depth_grad_kernel<true><<<grid, 256, 0, stream>>>(G, B, coeffs, sensor_id, depth_map, u, scale,
                                                                grad_depth);
    else
        shade_depth_grad_kernel<false><<<grid, 256, 0, stream>>>(G, B, coeffs, sensor_id, depth_map, u, scale,
                                                                 grad_depth);
    int rc = check_launch("depth gradient kernel");
    if (rc) return rc;
    zero_bad_sensor_images_kernel<<<static_cast<unsigned>(std::min<int64_t>(B, 4096)), 256, 0, stream>>>(
        B, G.S, G.HW, sensor_id, grad_depth);
    return check_launch("depth gradient kernel (bad sensor ids)");
}

int grid_for(int64_t n, int per_sm, const DevInfo& dev) {
    const int64_t blocks = (n + 255) / 256;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)dev.sms * per_sm)));
}

}  // namespace
}  // namespace tacsl

extern "C" {

int tacsl_penalty_forces_adjoint(const tacsl_sdf_set* set, const tacsl_contact_params* params, int32_t E, int32_t P,
                                 int32_t T, const float* taxels, const int32_t* obj_id, const float* pad_pose,
                                 const float* pad_twist, const float* g_depth, const float* g_f_n, const float* g_f_t,
                                 const float* g_wrench, float* grad_pose, float* grad_twist, float* grad_params,
                                 tacsl_stream_t stream) {
    SdfTable tab;
    Params4 prm;
    int rc = build_table(set, tab);
    if (rc) return rc;
    if ((rc = build_params(params, E, prm))) return rc;
    if (E < 0 || P < 0 || T < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size (E=%d P=%d T=%d)", E, P, T);
    if (T > TACSL_MAX_TAXELS) return fail(TACSL_ERR_UNSUPPORTED, "T = %d > %d taxels per pad", T, TACSL_MAX_TAXELS);
    if ((int64_t)E * P >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "E*P >= 2^31 pads");
    const void* req[] = {taxels, obj_id, pad_pose, pad_twist};
    const char* rn[] = {"taxels", "obj_id", "pad_pose", "pad_twist"};
    for (int i = 0; i < 4; ++i) {
        if (req[i] == nullptr && !(i == 0 && T == 0)) return fail(TACSL_ERR_INVALID_ARG, "%s is NULL", rn[i]);
        if (!aligned(req[i], 4)) return fail(TACSL_ERR_INVALID_ARG, "%s is not 4-byte aligned", rn[i]);
    }
    const void* opt[] = {g_depth, g_f_n, g_f_t, g_wrench, grad_pose, grad_twist, grad_params};
    for (const void* q : opt)
        if (!aligned(q, 4)) return fail(TACSL_ERR_INVALID_ARG, "a gradient array is not 4-byte aligned");
    if (E == 0) return ok();
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    if (grad_params != nullptr && prm.count == 1) {
        const cudaError_t e = cudaMemsetAsync(grad_params, 0, 4 * sizeof(float), stream);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    ForceAdjointArgs a{tab, prm, E, P, T, taxels, obj_id, pad_pose, pad_twist, g_depth, g_f_n, g_f_t, g_wrench,
                       grad_pose, grad_twist, grad_params};
    const int64_t blocks = ((int64_t)E + 7) / 8;
    const int grid = static_cast<int>(std::min<int64_t>(blocks, (int64_t)dev->sms * 16));
    force_adjoint_kernel<<<grid, 256, 0, stream>>>(a);
    return check_launch("tacsl_penalty_forces_adjoint");
}

int tacsl_shade_intensity(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id, const float* depth_map,
                          float* intensity, tacsl_stream_t stream) {
    if (shading != nullptr && B == 0) return ok();
    int rc = check_shade_args(shading, B, sensor_id, depth_map, reinterpret_cast<const uint8_t*>(intensity));
    if (rc) return rc;
    if (!aligned(intensity, 4)) return fail(TACSL_ERR_INVALID_ARG, "intensity is not 4-byte aligned");
    if (shading->H > 65535) return fail(TACSL_ERR_UNSUPPORTED, "image height %d > 65535", shading->H);
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadeGeom G;
    shade_geom(shading, G);
    if (G.HW > INT32_MAX) return fail(TACSL_ERR_UNSUPPORTED, "image too large");
    if (!dev->in_attr_set) {
        const int bytes = static_cast<int>(kInSmemBytes);
        cudaError_t e =
            cudaFuncSetAttribute(shade_intensity_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(shade_intensity_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        dev->in_attr_set = true;
    }
    // images per CTA: enough chunks to give every SM several CTAs
    const int64_t tiles = (G.HW + kCgPx - 1) / kCgPx;
    int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(65535, (int64_t)dev->sms * 8 / std::max<int64_t>(1, tiles * G.S) + 1));
    chunks = std::min<int64_t>(chunks, B);
    const int64_t chunk = (B + chunks - 1) / chunks;
    flag_bad_sensors_kernel<<<grid_for(B, 4, *dev), 256, 0, stream>>>(B, G.S, sensor_id);
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(G.S), static_cast<unsigned>((B + chunk - 1) / chunk));
    if (aligned(intensity, 8))
        shade_intensity_kernel<true><<<grid, 256, kInSmemBytes, stream>>>(G, B, chunk, shading->coeffs, sensor_id,
                                                                          depth_map, intensity);
    else
        shade_intensity_kernel<false><<<grid, 256, kInSmemBytes, stream>>>(G, B, chunk, shading->coeffs, sensor_id,
                                                                           depth_map, intensity);
    return check_launch("tacsl_shade_intensity");
}

int tacsl_shade_adjoint(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id, const float* depth_map,
                        const float* g_intensity, float* grad_coeffs, float* grad_depth, tacsl_stream_t stream) {
    if (shading != nullptr && B == 0 && grad_coeffs == nullptr) return ok();
    // the image checks of tacsl_shade_image, with g_intensity in the place of the output
    int rc = check_shade_args(shading, B, sensor_id, depth_map, reinterpret_cast<const uint8_t*>(g_intensity));
    if (rc) return rc;
    if (!aligned(g_intensity, 4) || !aligned(grad_coeffs, 4) || !aligned(grad_depth, 4))
        return fail(TACSL_ERR_INVALID_ARG, "gradient arrays must be 4-byte aligned");
    if (shading->H > 65535) return fail(TACSL_ERR_UNSUPPORTED, "image height %d > 65535", shading->H);
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadeGeom G;
    shade_geom(shading, G);
    if (grad_coeffs != nullptr) {
        if ((rc = launch_coeff_grad<false>(G, B, shading->coeffs, sensor_id, depth_map, g_intensity, nullptr,
                                           grad_coeffs, nullptr, nullptr, *dev, stream)))
            return rc;
    }
    if (grad_depth != nullptr && B > 0) {
        if ((rc = launch_depth_grad(false, G, B, shading->coeffs, sensor_id, depth_map, g_intensity, nullptr,
                                    grad_depth, *dev, stream)))
            return rc;
    }
    return ok();
}

int tacsl_shade_mse(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id, const float* depth_map,
                    const float* target, const float* scale, float* loss_map, float* grad_coeffs, float* grad_depth,
                    tacsl_stream_t stream) {
    const bool per_sensor = loss_map != nullptr || grad_coeffs != nullptr;
    if (shading != nullptr && B == 0 && !per_sensor) return ok();
    // the image checks of tacsl_shade_image, with the target in the place of the output
    int rc = check_shade_args(shading, B, sensor_id, depth_map, reinterpret_cast<const uint8_t*>(target));
    if (rc) return rc;
    if (!aligned(target, 4) || !aligned(scale, 4) || !aligned(loss_map, 4) || !aligned(grad_coeffs, 4) ||
        !aligned(grad_depth, 4))
        return fail(TACSL_ERR_INVALID_ARG, "target, scale, loss_map and gradient arrays must be 4-byte aligned");
    if (shading->H > 65535) return fail(TACSL_ERR_UNSUPPORTED, "image height %d > 65535", shading->H);
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadeGeom G;
    shade_geom(shading, G);
    if (per_sensor) {
        if ((rc = launch_coeff_grad<true>(G, B, shading->coeffs, sensor_id, depth_map, target, scale, grad_coeffs,
                                          loss_map, nullptr, *dev, stream)))
            return rc;
    }
    if (grad_depth != nullptr && B > 0) {
        if ((rc = launch_depth_grad(true, G, B, shading->coeffs, sensor_id, depth_map, target, scale, grad_depth,
                                    *dev, stream)))
            return rc;
    }
    return ok();
}

int tacsl_shade_mse_slopes(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id, const float* depth_map,
                           const float* target, float* loss_map, float* grad_coeffs, float* slopes,
                           tacsl_stream_t stream) {
    const bool per_sensor = loss_map != nullptr || grad_coeffs != nullptr;
    if (shading != nullptr && B == 0 && !per_sensor) return ok();
    int rc = check_shade_args(shading, B, sensor_id, depth_map, reinterpret_cast<const uint8_t*>(target));
    if (rc) return rc;
    if (!aligned(target, 4) || !aligned(loss_map, 4) || !aligned(grad_coeffs, 4))
        return fail(TACSL_ERR_INVALID_ARG, "target, loss_map and grad_coeffs must be 4-byte aligned");
    if (B > 0 && (slopes == nullptr || !aligned(slopes, 16)))
        return fail(TACSL_ERR_INVALID_ARG, "slopes must be non-NULL and 16-byte aligned");
    if (shading->H > 65535) return fail(TACSL_ERR_UNSUPPORTED, "image height %d > 65535", shading->H);
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadeGeom G;
    shade_geom(shading, G);
    return launch_coeff_grad<true>(G, B, shading->coeffs, sensor_id, depth_map, target, nullptr, grad_coeffs,
                                   loss_map, B > 0 ? slopes : nullptr, *dev, stream);
}

int tacsl_shade_adjoint_slopes(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                               const float* depth_map, const float* g_intensity, float* grad_coeffs, float* slopes,
                               tacsl_stream_t stream) {
    if (shading != nullptr && B == 0 && grad_coeffs == nullptr) return ok();
    int rc = check_shade_args(shading, B, sensor_id, depth_map, reinterpret_cast<const uint8_t*>(g_intensity));
    if (rc) return rc;
    if (!aligned(g_intensity, 4) || !aligned(grad_coeffs, 4))
        return fail(TACSL_ERR_INVALID_ARG, "g_intensity and grad_coeffs must be 4-byte aligned");
    if (B > 0 && (slopes == nullptr || !aligned(slopes, 16)))
        return fail(TACSL_ERR_INVALID_ARG, "slopes must be non-NULL and 16-byte aligned");
    if (shading->H > 65535) return fail(TACSL_ERR_UNSUPPORTED, "image height %d > 65535", shading->H);
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadeGeom G;
    shade_geom(shading, G);
    return launch_coeff_grad<false>(G, B, shading->coeffs, sensor_id, depth_map, g_intensity, nullptr, grad_coeffs,
                                    nullptr, B > 0 ? slopes : nullptr, *dev, stream);
}

int tacsl_shade_depth_from_slopes(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                                  const float* slopes, const float* scale, float* grad_depth, tacsl_stream_t stream) {
    if (shading != nullptr && B == 0) return ok();
    // the image checks of tacsl_shade_image, with the slopes in the places of the depth
    // maps and of the output
    int rc = check_shade_args(shading, B, sensor_id, slopes, reinterpret_cast<const uint8_t*>(grad_depth));
    if (rc) return rc;
    if (!aligned(grad_depth, 8) || !aligned(scale, 4))
        return fail(TACSL_ERR_INVALID_ARG, "grad_depth must be 8-byte and scale 4-byte aligned");
    if (shading->H > 65535) return fail(TACSL_ERR_UNSUPPORTED, "image height %d > 65535", shading->H);
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadeGeom G;
    shade_geom(shading, G);
    return launch_slopes_to_depth(G, B, sensor_id, slopes, scale, grad_depth, *dev, stream);
}

int tacsl_render_depth_adjoint(const tacsl_sdf_set* set, int32_t E, int32_t P, const int32_t* obj_id,
                               const float* pad_pose, const tacsl_camera* camera, const float* depth_map,
                               const float* g_depth, float* grad_pose, tacsl_stream_t stream) {
    SdfTable tab;
    int rc = build_table(set, tab);
    if (rc) return rc;
    CameraArgs c;
    if ((rc = check_camera(camera, c))) return rc;
    if (E < 0 || P < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size (E=%d P=%d)", E, P);
    const int64_t B = (int64_t)E * P;
    if (B == 0) return ok();
    if (obj_id == nullptr || !aligned(obj_id, 4) || pad_pose == nullptr || !aligned(pad_pose, 4))
        return fail(TACSL_ERR_INVALID_ARG, "obj_id and pad_pose must be non-NULL and 4-byte aligned");
    if (depth_map == nullptr || !aligned(depth_map, 16))
        return fail(TACSL_ERR_INVALID_ARG, "depth_map must be non-NULL and 16-byte aligned");
    if (g_depth == nullptr || !aligned(g_depth, 4) || grad_pose == nullptr || !aligned(grad_pose, 4))
        return fail(TACSL_ERR_INVALID_ARG, "g_depth and grad_pose must be non-NULL and 4-byte aligned");
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    const int64_t HW = (int64_t)c.H * c.W;
    if (dev->render_adj_slots[1] == 0) {
        // co-resident CTAs for each cluster size (the GPU places a cluster's CTAs together,
        // so clusters of 8 can leave SMs idle that single CTAs would fill)
        for (int cc = 1; cc <= kRenderAdjMaxCluster; ++cc) {
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3(static_cast<unsigned>(cc * 1024));
            q.blockDim = dim3(kRenderAdjThreads);
            cudaLaunchAttribute qa[1];
            qa[0].id = cudaLaunchAttributeClusterDimension;
            qa[0].val.clusterDim.x = static_cast<unsigned>(cc);
            qa[0].val.clusterDim.y = 1;
            qa[0].val.clusterDim.z = 1;
            q.attrs = qa;
            q.numAttrs = 1;
            int n = 0;
            const cudaError_t oe = cudaOccupancyMaxActiveClusters(&n, render_adjoint_kernel, &q);
            if (oe != cudaSuccess || n < 1) return fail(TACSL_ERR_CUDA, "render adjoint occupancy query failed");
            dev->render_adj_slots[cc] = n * cc;
        }
    }
    // CTAs per pad: the C in 1..8 (each CTA keeping at least 2048 pixels) whose launch
    // of B*C CTAs, each taking 1/C of an image, ends soonest on the co-resident CTAs of
    // clusters of C: minimise ceil(B*C / slots_C) / C, ties to the smaller C
    const int64_t c_max = std::min<int64_t>(kRenderAdjMaxCluster, std::max<int64_t>(1, HW / 2048));
    int C = 1;
    double best = (double)((B + dev->render_adj_slots[1] - 1) / dev->render_adj_slots[1]);
    for (int64_t cc = 2; cc <= c_max; ++cc) {
        const int64_t slots = dev->render_adj_slots[cc];
        const double t = (double)((B * cc + slots - 1) / slots) / (double)cc;
        if (t < best - 1e-9) {
            best = t;
            C = (int)cc;
        }
    }
    if (B * C > INT32_MAX) return fail(TACSL_ERR_UNSUPPORTED, "E*P = %lld pads in one call", (long long)B);
    RenderAdjointArgs A{tab, B, P, C, obj_id, pad_pose, c, depth_map, g_depth, grad_pose};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(B * C));
    cfg.blockDim = dim3(kRenderAdjThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, render_adjoint_kernel, A);
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "render adjoint launch: %s", cudaGetErrorString(e));
    return check_launch("render adjoint kernel");
}

}  // extern "C"

// ===========================================================================
// The tactile step from and to host memory, pipelined (tacsl_tactile_step_host)
// ===========================================================================
namespace tacsl {
namespace {

struct HostChunk {   // offsets of one chunk's device arrays in a workspace slot
    int64_t obj, pose, twist, sid, dmap, depth, fn, ft, wrench, rgb, bytes;
};

HostChunk host_chunk_layout(int64_t ec, int64_t P, int64_t T, int64_t HW) {
    HostChunk c;
    int64_t at = 0;
    auto take = [&](int64_t n) {
        const int64_t o = at;
        at += (std::max<int64_t>(n, 1) + 255) / 256 * 256;
        return o;
    };
    c.obj = take(4 * ec);
    c.pose = take(28 * ec * P);
    c.twist = take(24 * ec * P);
    c.sid = take(4 * ec * P);
    c.dmap = take(4 * ec * P * HW);
    c.depth = take(4 * ec * P * T);
    c.fn = take(12 * ec * P * T);
    c.ft = take(12 * ec * P * T);
    c.wrench = take(24 * ec * P);
    c.rgb = take(3 * ec * P * HW);
    c.bytes = at;
    return c;
}

int pipe_setup(DevInfo& dev) {
    if (dev.pipe[0] != nullptr) return TACSL_OK;
    cudaError_t e = cudaEventCreateWithFlags(&dev.pipe_start, cudaEventDisableTiming);
    for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
        e = cudaStreamCreateWithFlags(&dev.pipe[s], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&dev.pipe_done[s], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "pipeline streams: %s", cudaGetErrorString(e));
    return TACSL_OK;
}

}  // namespace
}  // namespace tacsl

extern "C" {

int64_t tacsl_tactile_step_host_workspace(int32_t chunk_envs, int32_t P, int32_t T, int32_t H, int32_t W) {
    if (chunk_envs < 1 || P < 0 || T < 0 || H < 0 || W < 0) return -1;
    return 3 * tacsl::host_chunk_layout(chunk_envs, P, T, (int64_t)H * W).bytes;
}

int tacsl_tactile_step_host(const tacsl_sdf_set* set, const tacsl_contact_params* params, int32_t E, int32_t P,
                            int32_t T, const float* taxels, const int32_t* obj_id, const float* pad_pose,
                            const float* pad_twist, float* depth, float* f_n, float* f_t, float* wrench,
                            const tacsl_shading* shading, const int32_t* sensor_id, const float* depth_map,
                            uint8_t* rgb, int32_t chunk_envs, void* workspace, int64_t workspace_bytes,
                            tacsl_stream_t stream) {
    SdfTable tab;
    Params4 prm;
    int rc = build_table(set, tab);
    if (rc) return rc;
    if ((rc = build_params(params, E, prm))) return rc;
    if (E < 0 || P < 0 || T < 0) return fail(TACSL_ERR_INVALID_ARG, "negative size (E=%d P=%d T=%d)", E, P, T);
    if (T > TACSL_MAX_TAXELS) return fail(TACSL_ERR_UNSUPPORTED, "T = %d > %d taxels per pad", T, TACSL_MAX_TAXELS);
    if ((int64_t)E * P >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "E*P >= 2^31 pads");
    if (chunk_envs < 1) return fail(TACSL_ERR_INVALID_ARG, "chunk_envs = %d < 1", chunk_envs);
    if ((int64_t)E * P == 0) return ok();
    const void* req[] = {taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t};
    const char* rn[] = {"taxels", "obj_id", "pad_pose", "pad_twist", "depth", "f_n", "f_t"};
    for (int i = 0; i < 7; ++i) {
        if (req[i] == nullptr && !(i == 0 && T == 0)) return fail(TACSL_ERR_INVALID_ARG, "%s is NULL", rn[i]);
        if (!aligned(req[i], 4)) return fail(TACSL_ERR_INVALID_ARG, "%s is not 4-byte aligned", rn[i]);
    }
    int64_t HW = 0;
    if (shading != nullptr) {
        // the image arguments as tacsl_shade_image checks them (host arrays here)
        if ((rc = check_shade_args(shading, (int64_t)E * P, sensor_id, depth_map, rgb))) return rc;
        HW = (int64_t)shading->H * shading->W;
    }
    const int32_t ch = std::min(chunk_envs, E);
    const HostChunk L = host_chunk_layout(ch, P, T, HW);
    if (workspace == nullptr || !aligned(workspace, 256) || workspace_bytes < 3 * L.bytes)
        return fail(TACSL_ERR_INVALID_ARG, "workspace NULL, not 256-byte aligned or below %lld bytes",
                    (long long)(3 * L.bytes));
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    std::lock_guard<std::mutex> lk(dev->pipe_mu);
    if ((rc = pipe_setup(*dev))) return rc;
    cudaError_t e = cudaEventRecord(dev->pipe_start, stream);
    const int n_chunks = (E + ch - 1) / ch;
    for (int s = 0; s < 3 && s < n_chunks && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(dev->pipe[s], dev->pipe_start, 0);
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "pipeline start: %s", cudaGetErrorString(e));
    auto h2d = [&](void* dst, const void* src, int64_t n, cudaStream_t st) {
        return n > 0 ? cudaMemcpyAsync(dst, src, (size_t)n, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    auto d2h = [&](void* dst, const void* src, int64_t n, cudaStream_t st) {
        return n > 0 ? cudaMemcpyAsync(dst, src, (size_t)n, cudaMemcpyDeviceToHost, st) : cudaSuccess;
    };
    for (int c = 0; c < n_chunks; ++c) {
        const int64_t e0 = (int64_t)c * ch, ec = std::min<int64_t>(ch, E - e0);
        const int64_t b0 = e0 * P, bc = ec * P;
        cudaStream_t st = dev->pipe[c % 3];
        char* base = static_cast<char*>(workspace) + (int64_t)(c % 3) * L.bytes;
        int32_t* d_obj = reinterpret_cast<int32_t*>(base + L.obj);
        float* d_pose = reinterpret_cast<float*>(base + L.pose);
        float* d_twist = reinterpret_cast<float*>(base + L.twist);
        int32_t* d_sid = reinterpret_cast<int32_t*>(base + L.sid);
        float* d_dmap = reinterpret_cast<float*>(base + L.dmap);
        float* d_depth = reinterpret_cast<float*>(base + L.depth);
        float* d_fn = reinterpret_cast<float*>(base + L.fn);
        float* d_ft = reinterpret_cast<float*>(base + L.ft);
        float* d_wr = reinterpret_cast<float*>(base + L.wrench);
        uint8_t* d_rgb = reinterpret_cast<uint8_t*>(base + L.rgb);
        // copies in (the slot's previous chunk is done with it: same stream)
        e = h2d(d_obj, obj_id + e0, 4 * ec, st);
        if (e == cudaSuccess) e = h2d(d_pose, pad_pose + 7 * b0, 28 * bc, st);
        if (e == cudaSuccess) e = h2d(d_twist, pad_twist + 6 * b0, 24 * bc, st);
        if (e == cudaSuccess && shading) e = h2d(d_sid, sensor_id + b0, 4 * bc, st);
        if (e == cudaSuccess && shading) e = h2d(d_dmap, depth_map + b0 * HW, 4 * bc * HW, st);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "pipeline copy-in: %s", cudaGetErrorString(e));
        // the step on this chunk
        if (shading) {
            ShadePlan plan;
            if ((rc = plan_shade(shading, bc, d_sid, d_dmap, d_rgb, *dev, plan))) return rc;
            if ((rc = launch_shade(plan, *dev, st))) return rc;
        }
        if (T > 0) {
            Params4 pc = prm;
            if (prm.count != 1) {
                pc.k_n += e0; pc.k_d += e0; pc.k_t += e0; pc.mu += e0;
                pc.count = static_cast<int>(ec);
            }
            if ((rc = launch_penalty(tab, pc, bc, P, T, taxels, d_obj, d_pose, d_twist, d_depth, d_fn, d_ft,
                                     wrench ? d_wr : nullptr, *dev, st)))
                return rc;
        }
        // copies out
        e = d2h(depth + b0 * T, d_depth, 4 * bc * T, st);
        if (e == cudaSuccess) e = d2h(f_n + 3 * b0 * T, d_fn, 12 * bc * T, st);
        if (e == cudaSuccess) e = d2h(f_t + 3 * b0 * T, d_ft, 12 * bc * T, st);
        if (e == cudaSuccess && wrench) e = d2h(wrench + 6 * b0, d_wr, 24 * bc, st);
        if (e == cudaSuccess && shading) e = d2h(rgb + 3 * b0 * HW, d_rgb, 3 * bc * HW, st);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "pipeline copy-out: %s", cudaGetErrorString(e));
    }
    // the caller's stream waits for every chunk
    for (int s = 0; s < 3 && s < n_chunks && e == cudaSuccess; ++s) {
        e = cudaEventRecord(dev->pipe_done[s], dev->pipe[s]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, dev->pipe_done[s], 0);
    }
    if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "pipeline end: %s", cudaGetErrorString(e));
    return ok();
}

}  // extern "C"

// ===========================================================================
// Serving (include/tacsl_serve.h)
// ===========================================================================
#include "serve.cuh"

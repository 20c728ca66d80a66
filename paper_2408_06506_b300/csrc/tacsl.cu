// libtacsl.so -- host side of the C ABI declared in include/tacsl.h.
//
// Every entry point validates its host-visible arguments, builds the kernel
// parameter structs (the SDF table travels by value in the launch), picks the launch
// shape for this device and enqueues its kernel(s) on the caller's stream.  Nothing
// here allocates device memory or synchronises, except tacsl_check_errors.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "render.cuh"
#include "shade.cuh"
#include "taxel.cuh"

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

struct ShadePlan {
    ShadeArgs a;
    int smem;
    int grid;
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
    a.n_tiles = (a.HW + kShTile - 1) / kShTile;
    a.cx_c = 1.f / (2.f * sh->pitch_x);
    a.cx_e = 1.f / sh->pitch_x;
    a.cy_c = 1.f / (2.f * sh->pitch_y);
    a.cy_e = 1.f / sh->pitch_y;
    a.stage_floats = kShTile + 2 * a.W;
    const int fixed = shade_smem_bytes(0, a.stage_floats);
    const int per_stage = a.stage_floats * 4;
    int ns = (dev.max_smem_optin - fixed) / per_stage;
    if (ns > 12) ns = 12;
    if (ns < 2)
        return fail(TACSL_ERR_UNSUPPORTED, "image width %d too large for the shared-memory pipeline", a.W);
    a.n_stages = ns;
    if (aligned(rgb, 16) && a.HW % 16 == 0)
        a.store_mode = kStoreVec;
    else if (aligned(rgb, 4))
        a.store_mode = kStoreWord;
    else
        a.store_mode = kStoreByte;
    // Images per work item: the largest power of two in [32, 1024] that still leaves
    // at least 24 items per CTA (a short tail), so coefficient reloads are amortised
    // over as many images as the load balance allows.
    const int64_t per_blk = (int64_t)a.S * a.n_tiles;
    int M = 1024;
    while (M > 32 && ((B + M - 1) / M) * per_blk < 24LL * dev.sms) M /= 2;
    const int64_t n_items = ((B + M - 1) / M) * per_blk;
    if (n_items >= (int64_t(1) << 31)) return fail(TACSL_ERR_UNSUPPORTED, "too many work items");
    a.M = M;
    a.n_items = static_cast<int>(n_items);
    plan.smem = shade_smem_bytes(ns, a.stage_floats);
    plan.grid = static_cast<int>(n_items < dev.sms ? (n_items > 0 ? n_items : 1) : dev.sms);
    return TACSL_OK;
}

}  // namespace
}  // namespace tacsl

namespace tacsl {
namespace {

int launch_shade(const ShadePlan& plan, DevInfo& dev, tacsl_stream_t stream) {
    if (!dev.shade_attr_set) {
        const cudaError_t e =
            cudaFuncSetAttribute(shade_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dev.max_smem_optin);
        if (e != cudaSuccess) return fail(TACSL_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        dev.shade_attr_set = true;
    }
    shade_kernel<<<plan.grid, kShThreads, plan.smem, stream>>>(plan.a);
    return check_launch("image kernel");
}

// One warp per pad, 8 pads per 256-thread CTA.
int launch_penalty(const SdfTable& tab, const Params4& prm, int64_t B, int P, int T, const float* taxels,
                   const int32_t* obj_id, const float* pad_pose, const float* pad_twist, float* depth, float* f_n,
                   float* f_t, float* wrench, const DevInfo& dev, tacsl_stream_t stream) {
    const int64_t blocks = (B + 7) / 8;
    const int grid = static_cast<int>(blocks < (int64_t)dev.sms * 32 ? blocks : (int64_t)dev.sms * 32);
    penalty_kernel<<<grid, 256, 0, stream>>>(tab, prm, B, P, T, taxels, obj_id, pad_pose, pad_twist, depth, f_n, f_t,
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
                  const CameraArgs& c, float* depth_map, const DevInfo& dev, tacsl_stream_t stream) {
    const int64_t n = B * c.H * c.W;
    const int64_t blocks = (n + 255) / 256;
    const int grid = static_cast<int>(blocks < (int64_t)dev.sms * 64 ? blocks : (int64_t)dev.sms * 64);
    render_kernel<<<grid, 256, 0, stream>>>(tab, B, P, obj_id, pad_pose, c, depth_map);
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
    int rc = check_shade_args(shading, B, sensor_id, depth_map, rgb);
    if (B == 0 && shading != nullptr) return ok();
    if (rc) return rc;
    DevInfo* dev;
    if ((rc = device_info(&dev))) return rc;
    ShadePlan plan;
    if ((rc = plan_shade(shading, B, sensor_id, depth_map, rgb, *dev, plan))) return rc;
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

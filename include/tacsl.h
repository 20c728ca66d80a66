/*
 * tacsl.h -- C ABI of the B300 (sm_103a) tactile-step library (libtacsl.so).
 *
 * The batched tactile step of TacSL (arXiv 2408.06506): SDF queries with
 * finite-difference gradients at every taxel of every sensor pad, penalty normal
 * and friction-capped shear forces, per-pad net wrenches (Sec. III-C), and the
 * depth map -> normals -> per-pixel shading -> uint8 RGB tactile image
 * (Sec. III-B), over thousands of environments on one GPU.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, contiguous, with
 *     natural alignment (4 bytes for float/int32); arguments that must be 16-byte
 *     aligned say so.  Descriptor structs (tacsl_sdf_set, tacsl_contact_params,
 *     tacsl_shading) are HOST memory read during the call; the device pointers
 *     inside them are read by the kernels later, on the stream.
 *   - Calls enqueue work on `stream` (NULL = the legacy default stream) and return
 *     without synchronising (tacsl_check_errors, tacsl_batch_autotune and
 *     tacsl_batch_graph_create do synchronise).  They never allocate or free device
 *     memory: buffers and workspaces are the caller's.  The exceptions are the server
 *     (tacsl_serve.h), which allocates one arena when it is created, and the CUDA streams
 *     and events that tacsl_tactile_step_host creates on its first call on a device.
 *   - Arguments are checked on the host before anything is launched; on failure the
 *     call returns a nonzero status, launches nothing and writes no output, and
 *     tacsl_last_error() describes the problem.
 *   - A zero-sized batch (n, E, P, T or B equal to 0) returns TACSL_OK and launches
 *     nothing, except that per-sensor sums over images (the coefficient gradient and
 *     loss map of tacsl_grad.h) are still written, as zeros.
 *   - Values that only exist on the device (object ids, sensor ids) are checked by the
 *     kernels: a bad one poisons the affected outputs as documented and sets a bit
 *     in the device error word, read with tacsl_check_errors().
 *
 * Frames (shared with the inputs' producers):
 *   object frame: the frame of the object's SDF grid;
 *   pad frame: taxels lie on its z = 0 plane, +z is the pad's outward normal
 *     pointing toward the object;
 *   pad_pose[7] = (tx, ty, tz, qw, qx, qy, qz): x_obj = R(q) x_pad + t; q need not
 *     be normalised (it is normalised in the kernel);
 *   pad_twist[6] = (vx, vy, vz, wx, wy, wz): the pad's velocity relative to the
 *     object, object frame, referenced at the object origin, so a pad point at
 *     x_obj moves at v + w x x_obj.
 */
#ifndef TACSL_H
#define TACSL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* tacsl_stream_t;

/* Status codes. */
#define TACSL_OK 0
#define TACSL_ERR_INVALID_ARG 1 /* a host-checkable argument is wrong; nothing launched */
#define TACSL_ERR_UNSUPPORTED 2 /* valid but beyond the library's limits; nothing launched */
#define TACSL_ERR_CUDA 3        /* the CUDA runtime reported an error (launch or query) */
#define TACSL_ERR_TIMEOUT 4     /* a bounded device wait gave up (see the error word) */

/* Bits of the device error word. */
#define TACSL_DEVERR_BAD_OBJ_ID 0x1u    /* an obj_id outside [0, n_sdf) was seen */
#define TACSL_DEVERR_BAD_SENSOR_ID 0x2u /* a sensor_id outside [0, n_sensor) was seen */
#define TACSL_DEVERR_TIMEOUT 0x4u       /* a kernel gave up on a bounded wait */

/* Build limits. */
#define TACSL_MAX_SDF 64      /* objects per call */
#define TACSL_MAX_SENSOR 16   /* sensor models per call */
#define TACSL_MAX_TAXELS 65536

/* One object's signed-distance grid (Sec. III-C: each contacting object carries an SDF).
 * Node (i, j, k) sits at origin + (i, j, k) * voxel; data is [n[2]][n[1]][n[0]],
 * x fastest, negative inside the object.  n[k] >= 3; n0*n1*n2 < 2^31. */
typedef struct {
    int32_t n[3];
    float origin[3];
    float voxel;
    const float* data; /* device */
} tacsl_sdf;

typedef struct {
    const tacsl_sdf* sdfs; /* host array of n_sdf descriptors */
    int32_t n_sdf;         /* 1 .. TACSL_MAX_SDF */
} tacsl_sdf_set;

/* Contact parameters of Sec. III-C: stiffness k_n, damping k_d, friction stiffness k_t
 * and friction coefficient mu.  Each is a device array of `count` floats, count = 1
 * (broadcast to every env) or count = E (one per env). */
typedef struct {
    const float* k_n;
    const float* k_d;
    const float* k_t;
    const float* mu;
    int32_t count;
} tacsl_contact_params;

/* Sensor shading model (Sec. III-B: I_rgb = F(I_depth) through a calibrated per-pixel
 * table).  F is the per-pixel quadratic
 *     I_c = sum_k A[s][k][c][y][x] m_k,   m = (1, n_x, n_y, n_x^2, n_y^2, n_x n_y),
 * of the depth-map normal n; A[s][0] is the sensor's background image.
 * coeffs: device, [n_sensor][6][3][H][W] float32, 16-byte aligned.
 * W must be a multiple of 4; pitch_x, pitch_y are the pixel spacings in metres. */
typedef struct {
    int32_t H, W;
    float pitch_x, pitch_y;
    const float* coeffs;
    int32_t n_sensor; /* 1 .. TACSL_MAX_SENSOR */
} tacsl_shading;

/* Orthographic tactile camera looking along the pad normal: the stand-in for the
 * in-sensor camera of Sec. III-B.  Pixel (i, j) sees the pad-frame column
 * (x0 + i*pitch_x, y0 + j*pitch_y, z); the undeformed gel (z = 0) reads d0; the column is
 * searched for the indenting object over z in [-z_max, 0].  H >= 1, W >= 4 and W % 4 = 0
 * (the image kernel's layout), pitches > 0, z_max > 0. */
typedef struct {
    int32_t H, W;
    float pitch_x, pitch_y;
    float x0, y0;
    float d0;
    float z_max;
} tacsl_camera;

/* Thread-local description of the last failing call on this thread ("" if none). */
const char* tacsl_last_error(void);

/* ABI version of this header (increments on any signature change). */
int32_t tacsl_abi_version(void);

/* Reads the calling device's error word into *flags (TACSL_DEVERR_* bits) and, if
 * `clear` is nonzero, resets it.  Synchronises `stream` first.  For tests/debugging. */
int tacsl_check_errors(tacsl_stream_t stream, uint32_t* flags, int32_t clear);

/*
 * SDF query with gradient (Sec. III-C: the penetration depth is read from the object's
 * SDF at each tactile point, and its gradient is taken by finite differences).
 *   pts    [n][3] object-frame points;  obj_id [n] grid per point.
 *   phi    [n]    trilinear interpolation of the grid at the point;
 *   grad   [n][3] central difference of that interpolant with step voxel/2 per axis.
 * A point is in the grid's domain iff every continuous index (x - origin)/voxel lies
 * in [0.5, n-1.5]; outside it phi = +INFINITY and grad = 0.  A bad obj_id gives NaN
 * phi and grad and sets TACSL_DEVERR_BAD_OBJ_ID.
 */
int tacsl_sdf_query(const tacsl_sdf_set* set, int64_t n, const float* pts,
                    const int32_t* obj_id, float* phi, float* grad, tacsl_stream_t stream);

/*
 * Penalty force field (Sec. III-C) of E envs x P pads x T taxels.
 *   taxels    [T][3]       rest taxel positions (pad frame), shared by all pads;
 *   obj_id    [E]          SDF touched by env e (all its pads);
 *   pad_pose  [E][P][7], pad_twist [E][P][6]   as in the frame conventions above.
 * Per taxel, with x = R p + t, x' = v + w x x, (phi, g) the SDF query at x and
 * n = g/|g|:
 *   depth = max(-phi, 0);
 *   if phi < 0 and |g| >= 1e-12:
 *     d'  = n . x'                                  (chain rule)
 *     f_n = max((-k_n + k_d d') phi, 0) n           (Sec. III-C law, clamped at 0, Eq. 3)
 *     v_t = x' - d' n
 *     f_t = -(v_t/|v_t|) min(k_t |v_t|, mu |f_n|)   (0 when |v_t| = 0)
 *   else f_n = f_t = 0.
 * Outputs (pad frame, R^T applied): depth [E][P][T], f_n [E][P][T][3],
 * f_t [E][P][T][3]; wrench [E][P][6] = (sum f, sum p x f) with f = f_n + f_t about
 * the pad origin, or NULL to skip it.  A bad obj_id fills that env's outputs with NaN
 * and sets TACSL_DEVERR_BAD_OBJ_ID.
 */
int tacsl_penalty_forces(const tacsl_sdf_set* set, const tacsl_contact_params* params,
                         int32_t E, int32_t P, int32_t T, const float* taxels,
                         const int32_t* obj_id, const float* pad_pose, const float* pad_twist,
                         float* depth, float* f_n, float* f_t, float* wrench,
                         tacsl_stream_t stream);

/*
 * Net wrench per pad from given force fields.  The paper has no such formula; it
 * feeds policies a per-finger net contact force (Sec. VI-B, privileged state) next to
 * the force field, and this is that reduction of the field plus its moment about the
 * pad origin.  f_n, f_t [B][T][3], taxels [T][3] ->
 * wrench [B][6] = (sum_i f_i, sum_i p_i x f_i), f_i = f_n,i + f_t,i.
 * Sums run in a fixed order: repeated calls give identical bits.
 */
int tacsl_pad_wrench(int64_t B, int32_t T, const float* taxels, const float* f_n,
                     const float* f_t, float* wrench, tacsl_stream_t stream);

/*
 * Tactile RGB images from depth maps (Sec. III-B, I_rgb = F(I_depth)).
 *   sensor_id [B]          shading model of image b;
 *   depth_map [B][H][W]    camera-to-gel distance [m], 16-byte aligned;
 *   rgb       [B][H][W][3] uint8, HWC.
 * Per pixel: D_x, D_y by central differences inside and one-sided differences on the
 * border (0 along an axis of length 1); n = (D_x, D_y, -1)/sqrt(1 + D_x^2 + D_y^2);
 * I_c as in tacsl_shading; rgb_c = floor(clamp(I_c, 0, 255) + 0.5), NaN -> 0.
 * An image whose sensor_id is outside [0, n_sensor) is left untouched and sets
 * TACSL_DEVERR_BAD_SENSOR_ID.
 */
int tacsl_shade_image(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                      const float* depth_map, uint8_t* rgb, tacsl_stream_t stream);

/*
 * tacsl_shade_image with the limit of its device-side barrier waits given explicitly, for
 * tests of those bounded waits (the paper has no counterpart).  The image kernel streams
 * depth tiles through a shared-memory ring guarded by barriers; every wait on them gives
 * up after wait_ns nanoseconds of %globaltimer (tacsl_shade_image uses 2 s), sets
 * TACSL_DEVERR_TIMEOUT in the device error word and ends its warp's loop, after the
 * producer warp has waited (with the 2 s limit) for the copies it already issued.  The
 * images are then incomplete.  wait_ns = 0 means the default.  A tiny limit makes the
 * waits run out on purpose; the next call with the default limit works normally.
 */
int tacsl_shade_image_wait_limit(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                                 const float* depth_map, uint8_t* rgb, uint64_t wait_ns,
                                 tacsl_stream_t stream);

/*
 * The whole tactile step in one call: tacsl_shade_image on the E*P depth maps (image
 * b = e*P + p belongs to pad (e, p)) and tacsl_penalty_forces on the E x P pads.
 * Arguments and results are exactly those of the two calls; shading may be NULL to skip
 * the images (then sensor_id, depth_map and rgb are ignored).  The call enqueues the
 * image kernel and then the force-field kernel on `stream`.
 */
int tacsl_tactile_step(const tacsl_sdf_set* set, const tacsl_contact_params* params,
                       int32_t E, int32_t P, int32_t T, const float* taxels,
                       const int32_t* obj_id, const float* pad_pose, const float* pad_twist,
                       float* depth, float* f_n, float* f_t, float* wrench,
                       const tacsl_shading* shading, const int32_t* sensor_id,
                       const float* depth_map, uint8_t* rgb, tacsl_stream_t stream);

/*
 * Depth maps of the E x P pads (Sec. III-B: a camera inside the sensor sees the depth of
 * the indenting object; the paper does this with a graphics render, here it is a CUDA
 * column march against the posed SDF).
 *   depth_map [E][P][H][W] float32 (16-byte aligned):
 *     D = d0 - max(0, -z_hit), z_hit = the first point of the object on the pixel's column
 *     over [-z_max, 0] (marching up from -z_max), D = d0 where the column misses it.
 * The march: where the column is inside the grid's domain (phi = the trilinear SDF) it
 * steps phi/|R e_z|_1, R e_z being the column's direction in the grid frame (each partial
 * derivative of the trilinear interpolant of a 1-Lipschitz grid is at most 1, so phi
 * changes by at most |R e_z|_1 per unit of column height; 1 for a pad aligned with the
 * grid, sqrt(3) at worst); the part of the column outside the domain is skipped by a slab
 * test; no step is below voxel/8.  The first step that lands inside the object (in the
 * domain with phi <= 0; outside the domain the SDF is undefined and never counts) closes
 * a bracket that is halved until it is at most voxel * 2^-16 wide; z_hit is its upper
 * end.  (The FP64 oracle's march keeps the isotropic step phi/sqrt(3); both are
 * conservative, so they can differ only on columns where the object dips below the
 * voxel/8 minimum step for less than one such step.)  A bad obj_id gives NaN maps and
 * sets TACSL_DEVERR_BAD_OBJ_ID.
 */
int tacsl_render_depth(const tacsl_sdf_set* set, int32_t E, int32_t P, const int32_t* obj_id,
                       const float* pad_pose, const tacsl_camera* camera, float* depth_map,
                       tacsl_stream_t stream);

/*
 * The tactile step from poses alone: tacsl_render_depth into depth_map (a caller buffer,
 * [E][P][H][W]), then tacsl_shade_image on it and tacsl_penalty_forces, in that order on
 * `stream`.  The camera's H and W must equal the shading model's.
 */
int tacsl_render_step(const tacsl_sdf_set* set, const tacsl_contact_params* params, int32_t E,
                      int32_t P, int32_t T, const float* taxels, const int32_t* obj_id,
                      const float* pad_pose, const float* pad_twist, float* depth, float* f_n,
                      float* f_t, float* wrench, const tacsl_shading* shading,
                      const tacsl_camera* camera, const int32_t* sensor_id, float* depth_map,
                      uint8_t* rgb, tacsl_stream_t stream);

/* Device workspace (bytes) tacsl_tactile_step_host needs for chunks of chunk_envs envs of
 * P pads x T taxels and H x W images (H = W = 0: no images).  Negative sizes give -1. */
int64_t tacsl_tactile_step_host_workspace(int32_t chunk_envs, int32_t P, int32_t T, int32_t H, int32_t W);

/* tacsl_tactile_step with the per-step arrays in HOST memory: obj_id [E], pad_pose
 * [E*P][7], pad_twist [E*P][6], sensor_id [E*P], depth_map [E*P][H][W] are read from
 * the host, and depth, f_n, f_t, wrench (may be NULL), rgb are written to the host, in
 * the layouts of tacsl_tactile_step; the SDFs, params, taxels and shading coefficients
 * stay on the device.  The envs go through in chunks of chunk_envs, pipelined on three
 * internal streams of this device (created, with their events, on the first call there): one chunk's inputs travel to the GPU while another
 * chunk computes and a third's outputs travel back.  workspace: device memory of at least
 * tacsl_tactile_step_host_workspace(chunk_envs, P, T, H, W) bytes, 256-byte aligned.  The
 * call enqueues everything after the work already on `stream` and makes `stream` wait for
 * it, so synchronising `stream` means the host outputs are complete.  Pinned (page-locked)
 * host memory is needed for the copies to overlap; depth_map must be 16-byte aligned.  Calls on one device are enqueued one
 * at a time (an internal lock). */
int tacsl_tactile_step_host(const tacsl_sdf_set* set, const tacsl_contact_params* params, int32_t E,
                            int32_t P, int32_t T, const float* taxels, const int32_t* obj_id,
                            const float* pad_pose, const float* pad_twist, float* depth, float* f_n,
                            float* f_t, float* wrench, const tacsl_shading* shading,
                            const int32_t* sensor_id, const float* depth_map, uint8_t* rgb,
                            int32_t chunk_envs, void* workspace, int64_t workspace_bytes,
                            tacsl_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TACSL_H */

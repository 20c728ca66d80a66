/*
 * tacsl_batch.h -- batched tactile step over uneven pads, objects and images
 * (libtacsl.so; see tacsl.h for the shared conventions, frames and status codes).
 *
 * The paper runs the tactile step over many parallel environments (Sec. IV-A: a
 * single GPU, thousands of environments); this interface lets every pad of such a
 * batch carry its own taxel layout (resolution), its own object SDF and its own
 * camera / shading model (image size, pixel pitch, coefficients), and runs the whole
 * batch as two kernel launches: the image kernel over all images of all models, then
 * the force-field kernel over all pads.  The per-pad arithmetic is exactly that of
 * tacsl_penalty_forces and tacsl_shade_image (Sec. III-B, III-C), so a batch gives
 * bit-for-bit the values those calls give for the same pad or image.
 *
 * Life cycle:
 *   1. tacsl_batch_plan_create (host only) sizes the batch: output offsets, the
 *      workspace size and a default launch configuration.
 *   2. The caller allocates the outputs and a device workspace of
 *      plan.workspace_bytes bytes (256-byte aligned); tacsl_batch_upload fills the
 *      workspace (pad schedule, image list) - or tacsl_batch_pack writes the same
 *      bytes to host memory for the caller to copy.
 *   3. tacsl_batch_step / _forces / _shade run a step; tacsl_batch_autotune may
 *      first pick the fastest launch configuration on the real inputs;
 *      tacsl_batch_graph_create captures one step as a CUDA graph for replay.
 *
 * Output layout (the same for every call of a plan):
 *   taxel outputs: pad b owns slots [taxel_offset[b], taxel_offset[b] + T_b) of
 *     depth[], f_n[][3], f_t[][3], with taxel_offset the exclusive prefix sum of T_b
 *     in pad order; wrench is [n_pad][6] in pad order;
 *   images: pad b with a sensor model owns pixels [pixel_offset[b],
 *     pixel_offset[b] + H_m W_m) of depth_map[] (input) and rgb[][3] (output),
 *     row-major within the image, with pixel_offset the exclusive prefix sum of H_m W_m
 *     over the pads that have an image, in pad order.
 */
#ifndef TACSL_BATCH_H
#define TACSL_BATCH_H

#include "tacsl.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TACSL_MAX_MODEL 64 /* sensor models per batch */

/* One camera / shading model (Sec. III-B): an H x W image with pixel pitch
 * (pitch_x, pitch_y) metres and per-pixel coefficients [6][3][H][W] (term, channel,
 * row, column) of the quadratic shading of tacsl_shade_image.  H and W are
 * multiples of 4, so every image of a packed batch starts 16-byte aligned. */
typedef struct {
    int32_t H, W;
    float pitch_x, pitch_y;
    const float* coeffs; /* device, 16-byte aligned */
} tacsl_sensor_model;

typedef struct {
    const tacsl_sensor_model* models; /* host array of n_model descriptors */
    int32_t n_model;                  /* 1 .. TACSL_MAX_MODEL */
} tacsl_sensor_set;

/* The batch: n_pad pads, each with an object, a taxel layout and an optional image.
 * All arrays are HOST memory, read during the call.  Layout l is the run of
 * layout_count[l] points (x, y, z pad frame) starting at point layout_first[l] of
 * the device taxel pool of n_points points passed at step time;
 * 1 <= layout_count[l] <= TACSL_MAX_TAXELS and layout_first[l] + layout_count[l] <= n_points. */
typedef struct {
    int32_t n_pad;
    const int32_t* obj_id;       /* [n_pad] SDF of each pad's object, in [0, TACSL_MAX_SDF) */
    const int32_t* layout;       /* [n_pad] taxel layout of each pad, in [0, n_layout) */
    const int32_t* sensor;       /* [n_pad] sensor model of each pad's image, or -1: no image */
    int32_t n_layout;
    const int64_t* layout_first; /* [n_layout] first point of each layout in the taxel pool */
    const int32_t* layout_count; /* [n_layout] points of each layout */
    int64_t n_points;            /* points in the taxel pool */
} tacsl_batch_desc;

/* Plan of one batch (plain host struct, owned by the caller).  The first block is for
 * the caller; the launch configuration may be set by hand (0 = automatic) or by
 * tacsl_batch_autotune; the rest is the library's and must not be modified. */
typedef struct {
    int32_t n_pad;
    int32_t n_image;          /* pads with an image */
    int64_t n_taxel_out;      /* taxel slots: sum of T_b */
    int64_t n_pixel_out;      /* pixels: sum of H_m W_m over images */
    int64_t workspace_bytes;  /* device workspace the step needs */
    /* launch configuration; results do not depend on it */
    int32_t img_block;        /* images per work item of the image kernel: a power of two <= 1024, 0 = auto */
    int32_t n_stages;         /* depth-map stages in flight per CTA: 2..12, 0 = as many as fit */
    int32_t force_np;         /* taxels in flight per lane in the force kernel: 2 or 4 (0 = 4) */
    int32_t force_dynamic;    /* 1: pads dealt from a counter in schedule order (by object, largest first); 0: round-robin */
    /* library-owned */
    int32_t n_model;
    int32_t max_w;
    int32_t model_h[TACSL_MAX_MODEL];
    int32_t model_w[TACSL_MAX_MODEL];
    int32_t model_img_begin[TACSL_MAX_MODEL + 1];
    int64_t off_sched;
    int64_t off_images;
    uint64_t fingerprint;     /* hash of the batch description and model sizes */
} tacsl_batch_plan;

/* Per-step buffers: DEVICE pointers, owned by the caller. */
typedef struct {
    const float* taxels;    /* taxel pool [n_points][3]; layouts index into it */
    const float* pad_pose;  /* [n_pad][7], as tacsl_penalty_forces */
    const float* pad_twist; /* [n_pad][6] */
    float* depth;           /* [n_taxel_out] penetration depth */
    float* f_n;             /* [n_taxel_out][3] normal force, pad frame */
    float* f_t;             /* [n_taxel_out][3] shear force, pad frame */
    float* wrench;          /* [n_pad][6] (F, tau) pad frame, or NULL */
    const float* depth_map; /* [n_pixel_out] packed depth maps, 16-byte aligned */
    uint8_t* rgb;           /* [n_pixel_out][3] packed RGB, 16-byte aligned */
} tacsl_batch_io;

/* Opaque CUDA graph of one batch step (a cudaGraphExec_t). */
typedef struct tacsl_graph_s* tacsl_graph_t;

/* Size a batch (host only; no CUDA call).  Fills *plan.  taxel_offset and
 * pixel_offset, when not NULL, are host arrays of n_pad receiving each pad's first
 * taxel slot and first pixel (-1 for a pad without image).  Errors: NULL or
 * inconsistent description, ids out of range, a sensor model with H or W not a
 * positive multiple of 4 (TACSL_ERR_INVALID_ARG); totals beyond 2^31 pads or images,
 * work items or a model wider than the shared-memory pipeline (TACSL_ERR_UNSUPPORTED). */
int tacsl_batch_plan_create(const tacsl_batch_desc* desc, const tacsl_sensor_set* sensors,
                            tacsl_batch_plan* plan, int64_t* taxel_offset, int64_t* pixel_offset);

/* Write the workspace contents for (plan, desc) into host memory of
 * plan->workspace_bytes bytes (host only).  desc must be the description the plan was
 * made from (checked by fingerprint). */
int tacsl_batch_pack(const tacsl_batch_plan* plan, const tacsl_batch_desc* desc, void* host_workspace);

/* tacsl_batch_pack into a temporary host buffer, then one copy to the device
 * workspace on stream (the host buffer is released before the call returns). */
int tacsl_batch_upload(const tacsl_batch_plan* plan, const tacsl_batch_desc* desc, void* workspace,
                       tacsl_stream_t stream);

/* The force field and wrenches of every pad (Sec. III-C; per pad exactly
 * tacsl_penalty_forces).  params: count 1 or n_pad (one entry per pad).  A pad whose
 * obj_id is >= set->n_sdf gets NaN outputs and TACSL_DEVERR_BAD_OBJ_ID.  The
 * workspace is read, and with force_dynamic its two counters are used and left at
 * zero: launches that share a workspace must not overlap on the GPU. */
int tacsl_batch_forces(const tacsl_batch_plan* plan, void* workspace, const tacsl_sdf_set* set,
                       const tacsl_contact_params* params, const tacsl_batch_io* io,
                       tacsl_stream_t stream);

/* tacsl_batch_forces for callers that cannot give the library device memory: a
 * real-time loop in which cudaMalloc / cudaFree would synchronise the device, or a
 * plug-in whose host application owns every device allocation.  The paper has no
 * counterpart; this is an interface convenience.  The call takes the batch description
 * itself (no plan, no workspace) and allocates nothing.  The pad schedule and the pad
 * counters live in one fixed 2 MiB array inside the library, present on every GPU that
 * loads it until the process exits; each call copies its schedule there (from host
 * memory, on stream) with the counters cleared to zero, then launches the force kernel.
 * Outputs are laid out as for a plan of the same description (taxel_offset = prefix sum
 * of T in pad order; wrench [n_pad][6]); desc->sensor is ignored.
 *   - At most 65528 pads per call; more returns TACSL_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the array's address there (set-up, once per
 *     device, with that device current).
 *   - The call cannot be captured in a CUDA graph: on a stream that is capturing it
 *     returns TACSL_ERR_UNSUPPORTED and enqueues nothing (tacsl_batch_graph_create is
 *     the capturable form).
 *   - The schedule is copied from pageable host memory, which CUDA may do synchronously:
 *     the call can block until the work already on stream has finished.
 *   - Every call shares the one array and it keeps the last call's contents: calls whose
 *     work overlaps on the GPU (different streams, or different host threads without
 *     ordering) race on it.  Calls on one stream are ordered and safe. */
int tacsl_batch_forces_static(const tacsl_batch_desc* desc, const tacsl_sdf_set* set,
                              const tacsl_contact_params* params, const tacsl_batch_io* io,
                              tacsl_stream_t stream);

/* The RGB image of every pad that has one (Sec. III-B; per image exactly
 * tacsl_shade_image with that model).  sensors must have the model sizes of the plan. */
int tacsl_batch_shade(const tacsl_batch_plan* plan, const void* workspace, const tacsl_sensor_set* sensors,
                      const tacsl_batch_io* io, tacsl_stream_t stream);

/* The depth map of every pad that has an image, rendered from its pose (Sec. III-B: the
 * camera inside the sensor sees the depth of the indenting object; per image exactly
 * tacsl_render_depth with that model's camera), into depth_map [n_pixel_out] (device,
 * 16-byte aligned; the packed layout the image kernel reads).  cameras: host array of
 * n_model cameras, camera m with the H and W of sensor model m (only models that have
 * images are read).  pad_pose [n_pad][7] device.  A pad whose obj_id is >= set->n_sdf
 * gets a NaN map and TACSL_DEVERR_BAD_OBJ_ID.  One launch per model with images. */
int tacsl_batch_render(const tacsl_batch_plan* plan, const void* workspace, const tacsl_sdf_set* set,
                       const tacsl_camera* cameras, const float* pad_pose, float* depth_map,
                       tacsl_stream_t stream);

/* Both: the image kernel, then the force-field kernel, on stream. */
int tacsl_batch_step(const tacsl_batch_plan* plan, void* workspace, const tacsl_sdf_set* set,
                     const tacsl_contact_params* params, const tacsl_sensor_set* sensors,
                     const tacsl_batch_io* io, tacsl_stream_t stream);

/* Time candidate launch configurations of both kernels on these buffers (outputs are
 * overwritten) and store the fastest in plan->img_block, n_stages, force_np and
 * force_dynamic.  reps timed launches per candidate after one warm-up; best_ms (may
 * be NULL) receives the best step time found.  Synchronises stream; must not be called
 * while stream is being captured. */
int tacsl_batch_autotune(tacsl_batch_plan* plan, void* workspace, const tacsl_sdf_set* set,
                         const tacsl_contact_params* params, const tacsl_sensor_set* sensors,
                         const tacsl_batch_io* io, int32_t reps, double* best_ms, tacsl_stream_t stream);

/* Capture one tacsl_batch_step with these arguments (pointers, plan configuration and
 * descriptor contents are baked in) into an instantiated CUDA graph.  Creates its own
 * capture stream; launches nothing.  *graph receives the handle. */
int tacsl_batch_graph_create(const tacsl_batch_plan* plan, void* workspace, const tacsl_sdf_set* set,
                             const tacsl_contact_params* params, const tacsl_sensor_set* sensors,
                             const tacsl_batch_io* io, tacsl_graph_t* graph);

/* Replay a captured step on stream (cudaGraphLaunch). */
int tacsl_graph_launch(tacsl_graph_t graph, tacsl_stream_t stream);

/* Release a graph (NULL is a no-op). */
int tacsl_graph_destroy(tacsl_graph_t graph);

#ifdef __cplusplus
}
#endif
#endif /* TACSL_BATCH_H */

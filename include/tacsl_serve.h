/*
 * tacsl_serve.h -- continuous-batching server of tactile steps (libtacsl.so; conventions,
 * frames and status codes as in tacsl.h, batches as in tacsl_batch.h).
 *
 * RL rollout workers (the paper trains its policies from thousands of parallel
 * environments, Sec. IV-A and VI) ask for tactile steps of different sizes at different
 * times.  The server keeps the object SDFs, sensor models and taxel layouts resident on
 * the GPU and serves such requests as they arrive:
 *   - a request is a list of pads (object, taxel layout, sensor model or none) with its
 *     host inputs (poses, twists, contact parameters, depth maps) and host outputs;
 *   - a worker thread admits pending requests while their device memory fits in the
 *     HBM budget (one arena allocated at creation) and whenever one of its streams is
 *     free puts every admitted request into one batch: inputs copied in, the batched
 *     image and force kernels, outputs copied back, all on that stream, so batches on
 *     different streams overlap on the device and requests that arrive meanwhile join
 *     the next batch (continuous batching);
 *   - a pad's result depends only on that pad, so every request gets bit-for-bit the
 *     values it would get alone.
 * Host buffers of a request must stay valid until it completes; pinned (page-locked)
 * host memory lets its copies overlap other work.
 */
#ifndef TACSL_SERVE_H
#define TACSL_SERVE_H

#include "tacsl_batch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tacsl_server_s* tacsl_server_t;

typedef struct {
    int64_t hbm_budget_bytes; /* device memory for requests in flight (one arena) */
    int32_t max_pads;         /* pads per batch (>= the largest request) */
    int32_t n_streams;        /* batches in flight at once, 1..8 */
    int32_t batch_timeout_ms; /* a batch not finished after this long fails its requests with TACSL_ERR_TIMEOUT */
} tacsl_server_config;

/* One request.  Host arrays; n_pad entries unless stated. */
typedef struct {
    int32_t n_pad;
    const int32_t* obj_id;   /* object of each pad (index into the server's SDF set) */
    const int32_t* layout;   /* taxel layout of each pad */
    const int32_t* sensor;   /* sensor model of each pad's image, or -1 */
    const float* pad_pose;   /* [n_pad][7] */
    const float* pad_twist;  /* [n_pad][6] */
    const float* k_n;        /* [n_pad] contact parameters per pad */
    const float* k_d;
    const float* k_t;
    const float* mu;
    const float* depth_map;  /* packed depth maps of the pads with an image, pad order */
    float* depth;            /* outputs, laid out as a batch of this request alone */
    float* f_n;
    float* f_t;
    float* wrench;           /* [n_pad][6] */
    uint8_t* rgb;
} tacsl_request;

/* A request that carries poses only (the RL loop's per-step inputs): the server renders
 * each image's depth map on the device from the pad's pose with the camera of its sensor
 * model (tacsl_batch_render; cameras set with tacsl_server_set_cameras), then shades it
 * and computes the force field.  Every output pointer may be NULL: only the outputs the
 * caller asks for travel back.  Host arrays; n_pad entries unless stated. */
typedef struct {
    int32_t n_pad;
    const int32_t* obj_id;   /* object of each pad (index into the server's SDF set) */
    const int32_t* layout;   /* taxel layout of each pad */
    const int32_t* sensor;   /* sensor model of each pad's image, or -1 */
    const float* pad_pose;   /* [n_pad][7] */
    const float* pad_twist;  /* [n_pad][6] */
    const float* k_n;        /* [n_pad] contact parameters per pad */
    const float* k_d;
    const float* k_t;
    const float* mu;
    float* wrench;           /* [n_pad][6], or NULL */
    float* depth;            /* taxel outputs laid out as a batch of this request alone, or NULL */
    float* f_n;
    float* f_t;
    uint8_t* rgb;            /* packed RGB of the pads with an image, pad order, or NULL */
    float* depth_map;        /* the rendered depth maps, same packing, or NULL */
} tacsl_pose_request;

typedef struct {
    int64_t submitted, completed, batches, pads_served;
    int64_t arena_bytes, arena_peak_bytes, arena_used_bytes;
    int32_t max_batch_requests; /* most requests put into one batch so far */
    int32_t pending;            /* requests waiting for admission */
} tacsl_server_stats;

/* Start a server.  sdfs, sensors (may be NULL if no request has images) and the taxel
 * pool (device, [n_points][3]) with its layouts (host arrays) are used for the server's
 * lifetime: their device memory must stay valid until tacsl_server_destroy.  Allocates the
 * arena (cudaMalloc), n_streams streams and events, and starts the worker thread on the
 * current device. */
int tacsl_server_create(const tacsl_server_config* config, const tacsl_sdf_set* sdfs,
                        const tacsl_sensor_set* sensors, const float* taxels, int64_t n_points,
                        int32_t n_layout, const int64_t* layout_first, const int32_t* layout_count,
                        tacsl_server_t* server);

/* Queue a request (its arrays are read during the call except the input / output data,
 * which are read / written later by the worker).  *request_id receives its id.  A request
 * that could never fit (more pads than max_pads, or more memory than the budget) is
 * refused with TACSL_ERR_UNSUPPORTED. */
int tacsl_server_submit(tacsl_server_t server, const tacsl_request* request, int64_t* request_id);

/* Wait up to timeout_ms (< 0: no limit) for a request.  Returns TACSL_OK once it has
 * finished, with its outcome in *status (TACSL_OK, TACSL_ERR_TIMEOUT if its batch overran
 * batch_timeout_ms, TACSL_ERR_CUDA) and, if latency_ms is not NULL, the time from its
 * submission until the worker saw its outputs arrive in host memory.  Returns
 * TACSL_ERR_TIMEOUT if it has not finished within timeout_ms (it keeps running; wait
 * again).  A finished request is forgotten after its first successful wait.  After a
 * TACSL_ERR_TIMEOUT outcome the GPU may still write the request's host outputs until its
 * batch ends: keep them valid until tacsl_server_destroy returns. */
int tacsl_server_wait(tacsl_server_t server, int64_t request_id, int32_t timeout_ms, int32_t* status,
                      double* latency_ms);

/* The tactile camera of each sensor model, for pose requests: n_camera must equal the
 * number of sensor models given at creation and camera m must have model m's H and W.
 * May be called again to change them; requests already submitted use the cameras set
 * when their batch is formed. */
int tacsl_server_set_cameras(tacsl_server_t server, const tacsl_camera* cameras, int32_t n_camera);

/* Queue a pose request (checks as tacsl_server_submit; a request with images needs the
 * cameras).  A batch holds requests of one kind: pose requests, or requests that bring
 * their depth maps; the worker takes the oldest pending requests of the kind of the
 * oldest one.  A pad's result depends only on that pad, as for tacsl_server_submit. */
int tacsl_server_submit_poses(tacsl_server_t server, const tacsl_pose_request* request, int64_t* request_id);

int tacsl_server_get_stats(tacsl_server_t server, tacsl_server_stats* stats);

/* Finish all queued and running requests, stop the worker, free the arena. */
int tacsl_server_destroy(tacsl_server_t server);

#ifdef __cplusplus
}
#endif
#endif /* TACSL_SERVE_H */

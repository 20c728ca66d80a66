/*
 * tacsl_grad.h -- gradients of the tactile step (libtacsl.so; conventions, frames and
 * status codes as in tacsl.h).
 *
 * Calibrating a tactile sensor model means fitting the contact parameters (the paper
 * measures the contact stiffness of its pads, App. B) and the image model (the
 * calibrated depth-to-RGB mapping of Sec. III-B) to observations.  These entry points
 * give the gradients such a fit needs, computed by hand-written adjoint kernels:
 *   - of the force field and wrenches (Sec. III-C) w.r.t. each pad's pose and twist and
 *     the contact parameters k_n, k_d, k_t, mu;
 *   - of the image w.r.t. the per-pixel shading coefficients and the depth maps;
 *   - of the rendered depth maps w.r.t. each pad's pose.
 * The differentiable image is the clamped intensity clamp(sum_k A_k m_k, 0, 255), the
 * continuous quantity the uint8 image rounds.  Gradients are those of the smooth piece
 * a point lies in: contact on/off, the unilateral clamp, stick/slip, the interpolation
 * cell and the intensity clamp carry no derivative.
 */
#ifndef TACSL_GRAD_H
#define TACSL_GRAD_H

#include "tacsl.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Adjoint of tacsl_penalty_forces (same set, params, E, P, T, taxels, obj_id, pad_pose,
 * pad_twist).  Upstream gradients (device, may be NULL = zero): g_depth [E*P][T],
 * g_f_n and g_f_t [E*P][T][3] (pad frame), g_wrench [E*P][6].  Outputs (device, may be
 * NULL = not wanted): grad_pose [E*P][7] (t and the raw quaternion q; the rotation uses
 * q/|q|, so the q part is tangent to the sphere through q, divided by |q|),
 * grad_twist [E*P][6], grad_params [params->count][4] = (k_n, k_d, k_t, mu).  With
 * count E each env's entry is its sum in a fixed order; with count 1 the call first
 * zeroes grad_params and every env adds into it with atomics (the summation order, and so
 * the last bits, vary between runs).  A bad obj_id gives NaN gradients for its env and sets
 * TACSL_DEVERR_BAD_OBJ_ID. */
int tacsl_penalty_forces_adjoint(const tacsl_sdf_set* set, const tacsl_contact_params* params, int32_t E,
                                 int32_t P, int32_t T, const float* taxels, const int32_t* obj_id,
                                 const float* pad_pose, const float* pad_twist, const float* g_depth,
                                 const float* g_f_n, const float* g_f_t, const float* g_wrench,
                                 float* grad_pose, float* grad_twist, float* grad_params,
                                 tacsl_stream_t stream);

/* Clamped intensities [B][H][W][3] (float, HWC) of the images tacsl_shade_image would
 * quantise: the forward of the differentiable image.  An image with a bad sensor_id is
 * left untouched and sets TACSL_DEVERR_BAD_SENSOR_ID.
 * The image entry points below take finite coefficients: where a group of pixels sees a
 * flat gel (n = 0) the kernels leave out the terms of the zero monomials, which is exact
 * for finite coefficients but drops a NaN or infinity such a term would have carried. */
int tacsl_shade_intensity(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                          const float* depth_map, float* intensity, tacsl_stream_t stream);

/* Adjoint of tacsl_shade_intensity for upstream g_intensity [B][H][W][3] (device).
 * grad_coeffs [S][6][3][H][W] (may be NULL): for each sensor, the sum over its images,
 * in image order.  grad_depth [B][H][W] (may be NULL): zero for an image with a bad
 * sensor_id. */
int tacsl_shade_adjoint(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                        const float* depth_map, const float* g_intensity, float* grad_coeffs,
                        float* grad_depth, tacsl_stream_t stream);

/* Squared error of the clamped intensities against target images, and its gradient,
 * without writing the intensities (the image loss of sensor calibration: fitting the
 * shading model and the depth maps to observed images):
 *   loss_map [S][H][W] (device, may be NULL): for each sensor s and pixel, the sum over
 *     the images b with sensor_id[b] = s, in image order, and the channels c of
 *     (clamp(I_c(b, y, x), 0, 255) - target[b][y][x][c])^2;
 *   with L = scale * sum(loss_map) (scale: device float[1], NULL = 1), grad_coeffs
 *     [S][6][3][H][W] and grad_depth [B][H][W] (device, may be NULL) receive dL/dA and
 *     dL/dD as tacsl_shade_adjoint gives them for dL/dI = 2 scale (clamp(I) - target).
 * target [B][H][W][3] (device) in the layout of tacsl_shade_intensity's output.  An image
 * with a bad sensor_id contributes nothing (its grad_depth is zero). */
int tacsl_shade_mse(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id, const float* depth_map,
                    const float* target, const float* scale, float* loss_map, float* grad_coeffs,
                    float* grad_depth, tacsl_stream_t stream);

/* The depth gradient in two passes (the form the torch.autograd bindings take): the pass
 * that evaluates the shading anyway (the loss forward, or the coefficient adjoint) also
 * writes per-pixel slopes, and the backward applies the transposed difference stencil
 * to them, so that the shading is evaluated once per pixel and image instead of again,
 * with a halo, in the backward.
 *
 * slopes [B][H][W][2] (device, 16-byte aligned, caller-owned; B*H*W*8 bytes): for each
 * image b with a valid sensor id and pixel (y, x), (dL/dD_x, dL/dD_y) of that pixel's
 * own term of L, D_x and D_y the depth differences its normal reads (central inside,
 * one-sided on the border, as in tacsl_shade_image).  Images with a bad sensor_id are
 * not written.
 *
 * tacsl_shade_mse_slopes: tacsl_shade_mse's loss_map and grad_coeffs for scale = 1 (both
 * may be NULL) and the slopes of L = sum(loss_map).  Same arguments and checks as
 * tacsl_shade_mse otherwise. */
int tacsl_shade_mse_slopes(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                           const float* depth_map, const float* target, float* loss_map,
                           float* grad_coeffs, float* slopes, tacsl_stream_t stream);

/* tacsl_shade_adjoint's grad_coeffs (may be NULL) and the slopes of L with dL/dI =
 * g_intensity.  Same arguments and checks as tacsl_shade_adjoint otherwise. */
int tacsl_shade_adjoint_slopes(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                               const float* depth_map, const float* g_intensity, float* grad_coeffs,
                               float* slopes, tacsl_stream_t stream);

/* grad_depth [B][H][W] (device, 8-byte aligned, overwritten) = scale * dL/dD from the
 * slopes one of the two calls above wrote for the same images and sensor ids:
 * grad_depth[b][q] = scale * sum over the pixels p whose difference stencils read
 * D[b][q] of (stencil weight of D[q] at p) * slope(p), the two axes' slots summed in the
 * order of tacsl_shade_mse's depth gradient.  scale: device float[1], NULL = 1.  Zero for
 * an image with a bad sensor_id.  Of the shading only H, W, n_sensor and the pitch are
 * used (its coeffs pointer is checked as for every shading call, not read). */
int tacsl_shade_depth_from_slopes(const tacsl_shading* shading, int64_t B, const int32_t* sensor_id,
                                  const float* slopes, const float* scale, float* grad_depth,
                                  tacsl_stream_t stream);

/* Adjoint of tacsl_render_depth w.r.t. the pad poses (the pose -> depth -> image chain;
 * same set, E, P, obj_id, pad_pose, camera).  depth_map [E*P][H][W] (device, 16-byte
 * aligned) is the render of these poses and g_depth [E*P][H][W] (device) the upstream
 * gradient, read only at the columns that carry a derivative; grad_pose
 * [E*P][7] (device, overwritten) receives dL/dt and dL/dq for the raw quaternion, as
 * tacsl_penalty_forces_adjoint gives them.  A column that hits the object at z_hit in
 * (-z_max, 0) has D = d0 + z_hit with phi(R p + t) = 0, p = (x_i, y_j, z_hit), so (implicit
 * function theorem) dD = -(grad phi . (dR p + dt)) / (grad phi . R e_z), grad phi the
 * analytic gradient of the trilinear interpolant at the hit.  Columns are classed on D:
 * D >= d0 (miss), D <= d0 - z_max (clamped at the bottom of the range), grazing columns
 * (|grad phi . R e_z| < 0.05) and hits outside the grid's domain carry no derivative.
 * Each pad's sums are reduced in a fixed order (bitwise reproducible).  A bad obj_id
 * gives NaN for its pads and sets TACSL_DEVERR_BAD_OBJ_ID. */
int tacsl_render_depth_adjoint(const tacsl_sdf_set* set, int32_t E, int32_t P, const int32_t* obj_id,
                               const float* pad_pose, const tacsl_camera* camera, const float* depth_map,
                               const float* g_depth, float* grad_pose, tacsl_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TACSL_GRAD_H */

/*
 * FP64 CPU oracle of the TacSL tactile step (arXiv 2408.06506).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library; it is
 * not part of the product path.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load it.  It shares no code, header,
 * constant or helper with the CUDA library.
 *
 * Every function reads the same float32 inputs the CUDA library reads, promotes
 * them to double, and computes in double.  Work is split over (env, pad) units or
 * images with OpenMP; each unit's sums run in ascending index order, so results
 * do not depend on the thread count.
 *
 * Readings of the paper where it is silent (each one also stated in the .c file):
 *   - the SDF is trilinear between nodes at origin + i*voxel (Sec. III-C says only
 *     that the SDF is queried);
 *   - the gradient is the central difference of that interpolant with step
 *     voxel/2 per axis (Sec. III-C names finite differences, no scheme or step);
 *   - a point is in the grid's domain iff every continuous index u lies in
 *     [0.5, n-1.5]; outside, phi = +inf, gradient 0, no force;
 *   - the normal force is clamped at zero (the unilateral law of Eq. 3);
 *   - forces are reported in the pad frame; the wrench is about the pad origin;
 *   - the depth-map gradient is central inside, one-sided at the borders;
 *   - the tactile-image map F is a per-pixel quadratic in (n_x, n_y).
 */
#ifndef TACSL_ORACLE_H
#define TACSL_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n[3];        /* nodes along x, y, z */
    float origin[3];     /* object-frame position of node (0,0,0) */
    float voxel;         /* node spacing [m] */
    const float* data;   /* [n2][n1][n0], x fastest */
} orc_sdf;

/* Trilinear interpolation at continuous index u (no domain test). */
double orc_trilinear(const orc_sdf* sdf, const double u[3]);

/* SDF value and finite-difference gradient at object-frame point x.
 * Returns 1 in domain, 0 outside (phi = +inf, grad = 0). */
int orc_sdf_eval(const orc_sdf* sdf, const double x[3], double* phi, double grad[3]);

/* Batched query: pts [n][3] (object frame), obj_id [n] -> phi [n], grad [n][3].
 * A bad obj_id gives NaN outputs. Returns the number of bad ids. */
int64_t orc_sdf_query(const orc_sdf* sdfs, int32_t n_sdf, int64_t n, const float* pts,
                      const int32_t* obj_id, double* phi, double* grad, int32_t nthreads);

/* Penalty normal/shear force field for E envs x P pads x T taxels.
 * taxels [T][3] (pad frame), obj_id [E], pad_pose [E][P][7], pad_twist [E][P][6],
 * k_n/k_d/k_t/mu each [n_params] with n_params = 1 (broadcast) or E.
 * Outputs: depth [E][P][T], f_n [E][P][T][3], f_t [E][P][T][3] (pad frame),
 * wrench [E][P][6] (may be NULL). Returns the number of pads whose obj id is bad. */
int64_t orc_penalty_forces(const orc_sdf* sdfs, int32_t n_sdf, int32_t E, int32_t P, int32_t T,
                           const float* taxels, const int32_t* obj_id, const float* pad_pose,
                           const float* pad_twist, const float* k_n, const float* k_d,
                           const float* k_t, const float* mu, int32_t n_params,
                           double* depth, double* f_n, double* f_t, double* wrench,
                           int32_t nthreads);

/* Per-pad wrench from given float32 force fields: wrench [B][6]. */
void orc_pad_wrench(int64_t B, int32_t T, const float* taxels, const float* f_n,
                    const float* f_t, double* wrench, int32_t nthreads);

/* Surface normals of one depth map: normals [H][W][3]. */
void orc_depth_normals(int32_t H, int32_t W, float pitch_x, float pitch_y, const float* depth,
                       double* normals);

/* Depth maps -> shaded intensities and uint8 RGB (HWC).
 * coeffs [S][6][3][H][W]; sensor_id [B]; depth [B][H][W];
 * intensity [B][H][W][3] (may be NULL); rgb [B][H][W][3].
 * A sensor id outside [0, S) leaves that image's outputs untouched.
 * Returns the number of bad sensor ids. */
int64_t orc_shade(const float* coeffs, int32_t S, int32_t H, int32_t W, float pitch_x,
                  float pitch_y, int64_t B, const int32_t* sensor_id, const float* depth,
                  double* intensity, uint8_t* rgb, int32_t nthreads);

/* Orthographic tactile camera along the pad normal (stand-in for the in-sensor camera
 * of Sec. III-B).  Pixel (i, j) looks along +z of the pad frame through the pad-frame
 * point (x0 + i*pitch_x, y0 + j*pitch_y, 0); the undeformed gel reads d0. */
typedef struct {
    int32_t H, W;
    float pitch_x, pitch_y;
    float x0, y0;
    float d0;
    float z_max;
} orc_camera;

/* Depth maps [E][P][H][W]: D = d0 - max(0, -z_hit), z_hit the first point of the object
 * met by the column z in [-z_max, 0] (marching up from -z_max), else no hit (D = d0).
 * Returns the number of pads whose obj id is bad (their maps are NaN). */
int64_t orc_render_depth(const orc_sdf* sdfs, int32_t n_sdf, int32_t E, int32_t P, const int32_t* obj_id,
                         const float* pad_pose, const orc_camera* cam, double* depth, int32_t nthreads);

/* The SDF value the column march sees at pad-frame point (x, y, z) of a pad posed by
 * pose7 (inside the grid domain: trilinear; outside: distance to the domain box). */
double orc_column_phi(const orc_sdf* sdf, const float* pose7, double x, double y, double z);

/* Quantisation of one intensity: clamp to [0, 255], round half up; NaN -> 0. */
uint8_t orc_quantize(double v);

#ifdef __cplusplus
}
#endif
#endif

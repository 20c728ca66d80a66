/*
 * FP64 CPU oracle of the TacSL tactile step (arXiv 2408.06506).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU baseline; never by the product path.  Plain, slow, written to
 * be read against the paper: one function per step, no blocking, no fusion.
 *
 * Passages followed:
 *   Sec. III-C (force field): f_n = (-k_n + k_d d') d n,
 *       f_t = -(v_t/|v_t|) min(k_t |v_t|, mu |f_n|);  d from an SDF query at the
 *       tactile points, d' = (grad d)^T x' by the chain rule, n = grad d by
 *       finite differences.
 *   Eq. 3 (Kelvin-Voigt): the contact force is unilateral -> clamp at zero.
 *   Sec. III-B and App. F (tactile image visualisation): I_rgb = F(I_depth) with
 *       F a calibrated per-pixel polynomial table; read here as a quadratic in
 *       the depth-map normal (n_x, n_y) with per-pixel coefficients.
 */
#include "tacsl_oracle.h"

#include <math.h>
#include <stddef.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* SDF query (Sec. III-C)                                                     */
/* ------------------------------------------------------------------------- */

static double sdf_node(const orc_sdf* s, int i, int j, int k) {
    return (double)s->data[((size_t)k * (size_t)s->n[1] + (size_t)j) * (size_t)s->n[0] + (size_t)i];
}

/* Reading: the grid holds node samples; between nodes the field is trilinear.
 * Cell index i0 = floor(u) kept inside [0, n-2] so that u = n-1 uses the last
 * cell with fraction 1. */
double orc_trilinear(const orc_sdf* s, const double u[3]) {
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(u[a]);
        int i = (int)fl;
        if (i > s->n[a] - 2) i = s->n[a] - 2;
        if (i < 0) i = 0;
        i0[a] = i;
        f[a] = u[a] - (double)i;
    }
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                           (dz ? f[2] : 1.0 - f[2]);
                acc += w * sdf_node(s, i0[0] + dx, i0[1] + dy, i0[2] + dz);
            }
    return acc;
}

/* Reading: gradient by central differences of the interpolant, step voxel/2
 * along each axis (u +- 0.5 in index units); domain = every u in [0.5, n-1.5],
 * which keeps both difference points inside the grid. */
int orc_sdf_eval(const orc_sdf* s, const double x[3], double* phi, double grad[3]) {
    const double h = (double)s->voxel;
    double u[3];
    int inside = 1;
    for (int a = 0; a < 3; ++a) {
        u[a] = (x[a] - (double)s->origin[a]) / h;
        if (!(u[a] >= 0.5 && u[a] <= (double)s->n[a] - 1.5)) inside = 0;
    }
    if (!inside) {
        *phi = INFINITY;
        grad[0] = grad[1] = grad[2] = 0.0;
        return 0;
    }
    *phi = orc_trilinear(s, u);
    for (int a = 0; a < 3; ++a) {
        double up[3] = {u[0], u[1], u[2]};
        double dn[3] = {u[0], u[1], u[2]};
        up[a] += 0.5;
        dn[a] -= 0.5;
        grad[a] = (orc_trilinear(s, up) - orc_trilinear(s, dn)) / h;
    }
    return 1;
}

int64_t orc_sdf_query(const orc_sdf* sdfs, int32_t n_sdf, int64_t n, const float* pts,
                      const int32_t* obj_id, double* phi, double* grad, int32_t nthreads) {
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t i = 0; i < n; ++i) {
        int32_t id = obj_id[i];
        if (id < 0 || id >= n_sdf) {
            phi[i] = NAN;
            grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = NAN;
            ++bad;
            continue;
        }
        double x[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
        orc_sdf_eval(&sdfs[id], x, &phi[i], &grad[3 * i]);
    }
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Rigid transforms                                                           */
/* ------------------------------------------------------------------------- */

/* Rotation matrix of the quaternion (w, x, y, z) after normalising it. */
static void quat_to_rot(const float* qf, double R[3][3]) {
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    double s = sqrt(w * w + x * x + y * y + z * z);
    w /= s; x /= s; y /= s; z /= s;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------- */
/* Penalty force field (Sec. III-C)                                           */
/* ------------------------------------------------------------------------- */

/* One tactile point.  p: rest position (pad frame).  Outputs in the pad frame. */
static void taxel_force(const orc_sdf* s, const double R[3][3], const double t[3],
                        const double v[3], const double w[3], const float* p,
                        double kn, double kd, double kt, double mu,
                        double* depth, double fn_pad[3], double ft_pad[3]) {
    /* pose the tactile point into the object frame: x_o = R p + t */
    double xo[3];
    for (int a = 0; a < 3; ++a)
        xo[a] = R[a][0] * (double)p[0] + R[a][1] * (double)p[1] + R[a][2] * (double)p[2] + t[a];
    /* relative velocity of the point w.r.t. the object: x' = v + w x x_o */
    double wx[3], xdot[3];
    cross3(w, xo, wx);
    for (int a = 0; a < 3; ++a) xdot[a] = v[a] + wx[a];

    double d, g[3];
    orc_sdf_eval(s, xo, &d, g);

    double fn[3] = {0, 0, 0}, ft[3] = {0, 0, 0};
    *depth = 0.0;
    if (d < 0.0) {                              /* interpenetration */
        *depth = -d;
        double gn = sqrt(dot3(g, g));
        if (gn >= 1e-12) {
            double n[3] = {g[0] / gn, g[1] / gn, g[2] / gn};   /* contact normal */
            double ddot = dot3(n, xdot);                       /* d' = n . x' */
            double mag = (-kn + kd * ddot) * d;                /* f_n = (-k_n + k_d d') d n */
            if (mag < 0.0) mag = 0.0;                          /* unilateral (Eq. 3) */
            for (int a = 0; a < 3; ++a) fn[a] = mag * n[a];
            double vt[3];                                      /* tangential velocity */
            for (int a = 0; a < 3; ++a) vt[a] = xdot[a] - ddot * n[a];
            double vtn = sqrt(dot3(vt, vt));
            if (vtn > 0.0) {
                double cap = kt * vtn;
                double lim = mu * mag;                         /* mu |f_n| */
                double ftm = cap < lim ? cap : lim;
                for (int a = 0; a < 3; ++a) ft[a] = -(vt[a] / vtn) * ftm;
            }
        }
    }
    /* report in the pad frame: R^T f */
    for (int a = 0; a < 3; ++a) {
        fn_pad[a] = R[0][a] * fn[0] + R[1][a] * fn[1] + R[2][a] * fn[2];
        ft_pad[a] = R[0][a] * ft[0] + R[1][a] * ft[1] + R[2][a] * ft[2];
    }
}

/* Net wrench of one pad: F = sum (f_n + f_t), tau = sum p x (f_n + f_t), pad frame,
 * about the pad origin, ascending taxel order. */
static void wrench_sum_d(int32_t T, const float* taxels, const double* fn, const double* ft,
                         double out[6]) {
    double F[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
    for (int32_t i = 0; i < T; ++i) {
        double f[3] = {fn[3 * i] + ft[3 * i], fn[3 * i + 1] + ft[3 * i + 1], fn[3 * i + 2] + ft[3 * i + 2]};
        double p[3] = {taxels[3 * i], taxels[3 * i + 1], taxels[3 * i + 2]};
        double m[3];
        cross3(p, f, m);
        for (int a = 0; a < 3; ++a) { F[a] += f[a]; tau[a] += m[a]; }
    }
    out[0] = F[0]; out[1] = F[1]; out[2] = F[2];
    out[3] = tau[0]; out[4] = tau[1]; out[5] = tau[2];
}

int64_t orc_penalty_forces(const orc_sdf* sdfs, int32_t n_sdf, int32_t E, int32_t P, int32_t T,
                           const float* taxels, const int32_t* obj_id, const float* pad_pose,
                           const float* pad_twist, const float* k_n, const float* k_d,
                           const float* k_t, const float* mu, int32_t n_params,
                           double* depth, double* f_n, double* f_t, double* wrench,
                           int32_t nthreads) {
    int64_t bad = 0;
    const int64_t B = (int64_t)E * P;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : bad) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t b = 0; b < B; ++b) {
        const int64_t e = b / P;
        const int32_t id = obj_id[e];
        double* dep = depth + b * T;
        double* fn = f_n + b * T * 3;
        double* ft = f_t + b * T * 3;
        if (id < 0 || id >= n_sdf) {
            for (int64_t i = 0; i < (int64_t)T; ++i) dep[i] = NAN;
            for (int64_t i = 0; i < (int64_t)T * 3; ++i) fn[i] = ft[i] = NAN;
            if (wrench)
                for (int a = 0; a < 6; ++a) wrench[b * 6 + a] = NAN;
            ++bad;
            continue;
        }
        const int64_t pi = n_params == 1 ? 0 : e;
        const float* pose = pad_pose + b * 7;
        const float* tw = pad_twist + b * 6;
        double R[3][3];
        quat_to_rot(pose + 3, R);
        double t[3] = {pose[0], pose[1], pose[2]};
        double v[3] = {tw[0], tw[1], tw[2]};
        double w[3] = {tw[3], tw[4], tw[5]};
        for (int32_t i = 0; i < T; ++i)
            taxel_force(&sdfs[id], R, t, v, w, taxels + 3 * i, k_n[pi], k_d[pi], k_t[pi], mu[pi],
                        &dep[i], &fn[3 * i], &ft[3 * i]);
        if (wrench) wrench_sum_d(T, taxels, fn, ft, wrench + b * 6);
    }
    return bad;
}

void orc_pad_wrench(int64_t B, int32_t T, const float* taxels, const float* f_n,
                    const float* f_t, double* wrench, int32_t nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t b = 0; b < B; ++b) {
        double F[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
        for (int32_t i = 0; i < T; ++i) {
            const float* a = f_n + (b * T + i) * 3;
            const float* c = f_t + (b * T + i) * 3;
            double f[3] = {(double)a[0] + (double)c[0], (double)a[1] + (double)c[1], (double)a[2] + (double)c[2]};
            double p[3] = {taxels[3 * i], taxels[3 * i + 1], taxels[3 * i + 2]};
            double m[3];
            cross3(p, f, m);
            for (int k = 0; k < 3; ++k) { F[k] += f[k]; tau[k] += m[k]; }
        }
        for (int k = 0; k < 3; ++k) { wrench[b * 6 + k] = F[k]; wrench[b * 6 + 3 + k] = tau[k]; }
    }
}

/* ------------------------------------------------------------------------- */
/* Tactile image (Sec. III-B): depth map -> normals -> per-pixel shading       */
/* ------------------------------------------------------------------------- */

/* Reading: derivative along one image axis, central inside and one-sided at
 * the two borders (spacing = pixel pitch); zero along an axis of length 1. */
static double axis_derivative(const float* D, int32_t len, int64_t stride, int32_t i, double pitch) {
    if (len < 2) return 0.0;
    if (i == 0) return ((double)D[stride] - (double)D[0]) / pitch;
    if (i == len - 1) return ((double)D[(int64_t)(len - 1) * stride] - (double)D[(int64_t)(len - 2) * stride]) / pitch;
    return ((double)D[(int64_t)(i + 1) * stride] - (double)D[(int64_t)(i - 1) * stride]) / (2.0 * pitch);
}

/* Unit normal of the surface z = D(x, y) seen from the camera: (D_x, D_y, -1)/norm. */
static void pixel_normal(int32_t H, int32_t W, double px, double py, const float* D, int32_t y,
                         int32_t x, double n[3]) {
    double dx = axis_derivative(D + (int64_t)y * W, W, 1, x, px);
    double dy = axis_derivative(D + x, H, W, y, py);
    double inv = 1.0 / sqrt(1.0 + dx * dx + dy * dy);
    n[0] = dx * inv;
    n[1] = dy * inv;
    n[2] = -inv;
}

void orc_depth_normals(int32_t H, int32_t W, float pitch_x, float pitch_y, const float* depth,
                       double* normals) {
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x)
            pixel_normal(H, W, pitch_x, pitch_y, depth, y, x, normals + ((int64_t)y * W + x) * 3);
}

uint8_t orc_quantize(double v) {
    if (!(v > 0.0)) return 0;      /* also NaN */
    if (v > 255.0) v = 255.0;
    return (uint8_t)floor(v + 0.5);
}

int64_t orc_shade(const float* coeffs, int32_t S, int32_t H, int32_t W, float pitch_x,
                  float pitch_y, int64_t B, const int32_t* sensor_id, const float* depth,
                  double* intensity, uint8_t* rgb, int32_t nthreads) {
    int64_t bad = 0;
    const int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t b = 0; b < B; ++b) {
        const int32_t s = sensor_id[b];
        if (s < 0 || s >= S) { ++bad; continue; }
        const float* D = depth + b * HW;
        const float* A = coeffs + (int64_t)s * 18 * HW;   /* [6][3][H][W] */
        for (int32_t y = 0; y < H; ++y)
            for (int32_t x = 0; x < W; ++x) {
                double n[3];
                pixel_normal(H, W, pitch_x, pitch_y, D, y, x, n);
                const double m[6] = {1.0, n[0], n[1], n[0] * n[0], n[1] * n[1], n[0] * n[1]};
                const int64_t px = (int64_t)y * W + x;
                for (int c = 0; c < 3; ++c) {
                    double I = 0.0;
                    for (int k = 0; k < 6; ++k) I += (double)A[(int64_t)(k * 3 + c) * HW + px] * m[k];
                    if (intensity) intensity[(b * HW + px) * 3 + c] = I;
                    rgb[(b * HW + px) * 3 + c] = orc_quantize(I);
                }
            }
    }
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Depth-map rendering (Sec. III-B: a camera behind the gel renders the depth  */
/* of the indenting object).                                                   */
/* ------------------------------------------------------------------------- */

/* Reading: an orthographic camera looks along the pad normal; pixel (i, j)'s ray is
 * the pad-frame column (x_i, y_j, z).  The gel surface is z = 0 at distance d0; where
 * the object reaches below it, the camera sees the object's first point on the column,
 * so D = d0 - max(0, -z_hit).  The column is searched over [-z_max, 0] from below. */

#define ORC_MARCH_MAX 1024
#define ORC_BISECT_MAX 40

/* Distance from object-frame point x to the grid's domain box (0 inside). */
static double domain_box_distance(const orc_sdf* s, const double x[3]) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double lo = (double)s->origin[a] + 0.5 * (double)s->voxel;
        const double hi = (double)s->origin[a] + ((double)s->n[a] - 1.5) * (double)s->voxel;
        double e = 0.0;
        if (x[a] < lo) e = lo - x[a];
        else if (x[a] > hi) e = x[a] - hi;
        d2 += e * e;
    }
    return sqrt(d2);
}

/* phi seen by the march: trilinear inside the domain; outside, the distance to the
 * domain box (the object lies inside the domain, so that bounds the distance to it).
 * Outside the domain the SDF is undefined (phi = +inf there, as for the force field), so
 * a point there is never inside the object; the box distance only sizes the step. */
static double column_phi_obj(const orc_sdf* s, const double x[3], int* inside) {
    double phi, g[3];
    *inside = orc_sdf_eval(s, x, &phi, g);
    return *inside ? phi : domain_box_distance(s, x);
}

double orc_column_phi(const orc_sdf* s, const float* pose7, double x, double y, double z) {
    double R[3][3];
    quat_to_rot(pose7 + 3, R);
    double xo[3];
    for (int a = 0; a < 3; ++a) xo[a] = R[a][0] * x + R[a][1] * y + R[a][2] * z + (double)pose7[a];
    int inside;
    return column_phi_obj(s, xo, &inside);
}

/* z_hit of one column (returns 1 on a hit).  March: from z = -z_max step up by
 * kappa*phi inside the domain (kappa = 1/sqrt(3): the trilinear interpolant of a
 * 1-Lipschitz field is at most sqrt(3)-Lipschitz, so the step cannot pass the surface)
 * or by the box distance outside it, never less than voxel/8; the first sample inside
 * the object closes a bracket that is halved until it is at most voxel * 2^-16 wide;
 * z_hit is its upper end. */
static int column_hit(const orc_sdf* s, const double R[3][3], const double t[3], double px, double py,
                      double z_max, double* z_hit) {
    const double dmin = (double)s->voxel / 8.0;
    const double kappa = 1.0 / sqrt(3.0);
    double x[3];
    int inside;
#define COLUMN_POINT(zz)                                                         \
    for (int a = 0; a < 3; ++a) x[a] = R[a][0] * px + R[a][1] * py + R[a][2] * (zz) + t[a];
    double z = -z_max;
    COLUMN_POINT(z);
    double phi = column_phi_obj(s, x, &inside);
    if (inside && phi <= 0.0) { *z_hit = z; return 1; }   /* the object reaches below -z_max */
    for (int it = 0; it < ORC_MARCH_MAX; ++it) {
        double step = inside ? kappa * phi : phi;
        if (step < dmin) step = dmin;
        double zn = z + step;
        if (zn > 0.0) zn = 0.0;
        COLUMN_POINT(zn);
        int inside_n;
        const double phin = column_phi_obj(s, x, &inside_n);
        if (inside_n && phin <= 0.0) {
            double lo = z, hi = zn;
            const double eps = (double)s->voxel / 65536.0;
            for (int k = 0; k < ORC_BISECT_MAX && hi - lo > eps; ++k) {
                const double mid = 0.5 * (lo + hi);
                COLUMN_POINT(mid);
                int im;
                const double pm = column_phi_obj(s, x, &im);
                if (im && pm <= 0.0) hi = mid; else lo = mid;
            }
            *z_hit = hi;
            return 1;
        }
        if (zn >= 0.0) return 0;
        z = zn; phi = phin; inside = inside_n;
    }
#undef COLUMN_POINT
    return 0;
}

int64_t orc_render_depth(const orc_sdf* sdfs, int32_t n_sdf, int32_t E, int32_t P, const int32_t* obj_id,
                         const float* pad_pose, const orc_camera* cam, double* depth, int32_t nthreads) {
    int64_t bad = 0;
    const int64_t B = (int64_t)E * P, HW = (int64_t)cam->H * cam->W;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t b = 0; b < B; ++b) {
        double* D = depth + b * HW;
        const int32_t id = obj_id[b / P];
        if (id < 0 || id >= n_sdf) {
            for (int64_t k = 0; k < HW; ++k) D[k] = NAN;
            ++bad;
            continue;
        }
        const float* pose = pad_pose + b * 7;
        double R[3][3];
        quat_to_rot(pose + 3, R);
        const double t[3] = {pose[0], pose[1], pose[2]};
        for (int32_t j = 0; j < cam->H; ++j)
            for (int32_t i = 0; i < cam->W; ++i) {
                const double px = (double)cam->x0 + (double)i * (double)cam->pitch_x;
                const double py = (double)cam->y0 + (double)j * (double)cam->pitch_y;
                double zh;
                const int hit = column_hit(&sdfs[id], R, t, px, py, (double)cam->z_max, &zh);
                D[(int64_t)j * cam->W + i] = (double)cam->d0 - (hit && zh < 0.0 ? -zh : 0.0);
            }
    }
    return bad;
}

"""The pins bite: plant plausible mistakes in a copy of the oracle and check that the
pin suite catches every one (CPU only; the shipped oracle is never modified).

Each mutation is a textual edit of the oracle's C source that a careless
implementation could make: a wrong finite-difference step, a flipped sign, a
transposed rotation, a swapped cross product, a missing clamp, a wrong
quantisation rounding, and so on.  For each, the pin tests are re-run against the
mutated build and at least one must fail.
"""
import os
import subprocess
import sys

import pytest

import oracle

MUTATIONS = {
    "fd_step": ("up[a] += 0.5;", "up[a] += 1.0;"),
    "fd_divisor": ("grad[a] = (orc_trilinear(s, up) - orc_trilinear(s, dn)) / h;",
                   "grad[a] = (orc_trilinear(s, up) - orc_trilinear(s, dn)) / (2.0 * h);"),
    "domain_upper": ("u[a] <= (double)s->n[a] - 1.5", "u[a] <= (double)s->n[a] - 1.0"),
    "trilinear_weight": ("(dy ? f[1] : 1.0 - f[1])", "(dy ? 1.0 - f[1] : f[1])"),
    "node_stride": ("((size_t)k * (size_t)s->n[1] + (size_t)j) * (size_t)s->n[0] + (size_t)i",
                    "((size_t)i * (size_t)s->n[1] + (size_t)j) * (size_t)s->n[0] + (size_t)k"),
    "quat_no_normalise": ("w /= s; x /= s; y /= s; z /= s;", ""),
    "rotation_transposed_pose": ("xo[a] = R[a][0] * (double)p[0] + R[a][1] * (double)p[1] + R[a][2] * (double)p[2] + t[a];",
                                 "xo[a] = R[0][a] * (double)p[0] + R[1][a] * (double)p[1] + R[2][a] * (double)p[2] + t[a];"),
    "output_not_transposed": ("fn_pad[a] = R[0][a] * fn[0] + R[1][a] * fn[1] + R[2][a] * fn[2];",
                              "fn_pad[a] = R[a][0] * fn[0] + R[a][1] * fn[1] + R[a][2] * fn[2];"),
    "omega_cross_order": ("cross3(w, xo, wx);", "cross3(xo, w, wx);"),
    "damping_sign": ("double mag = (-kn + kd * ddot) * d;", "double mag = (-kn - kd * ddot) * d;"),
    "no_unilateral_clamp": ("if (mag < 0.0) mag = 0.0;", ""),
    "shear_sign": ("ft[a] = -(vt[a] / vtn) * ftm;", "ft[a] = (vt[a] / vtn) * ftm;"),
    "friction_max": ("double ftm = cap < lim ? cap : lim;", "double ftm = cap > lim ? cap : lim;"),
    "vt_not_projected": ("vt[a] = xdot[a] - ddot * n[a];", "vt[a] = xdot[a];"),
    "torque_order": ("cross3(p, f, m);\n        for (int a = 0; a < 3; ++a) { F[a] += f[a]; tau[a] += m[a]; }",
                     "cross3(f, p, m);\n        for (int a = 0; a < 3; ++a) { F[a] += f[a]; tau[a] += m[a]; }"),
    "wrench_drops_shear": ("double f[3] = {fn[3 * i] + ft[3 * i], fn[3 * i + 1] + ft[3 * i + 1], fn[3 * i + 2] + ft[3 * i + 2]};",
                           "double f[3] = {fn[3 * i], fn[3 * i + 1], fn[3 * i + 2]};"),
    "normal_pitch_swapped": ("double dx = axis_derivative(D + (int64_t)y * W, W, 1, x, px);",
                             "double dx = axis_derivative(D + (int64_t)y * W, W, 1, x, py);"),
    "edge_not_one_sided": ("if (i == 0) return ((double)D[stride] - (double)D[0]) / pitch;",
                           "if (i == 0) return ((double)D[stride] - (double)D[0]) / (2.0 * pitch);"),
    "normal_z_sign": ("n[2] = -inv;", "n[2] = inv;"),
    "monomial_swap": ("const double m[6] = {1.0, n[0], n[1], n[0] * n[0], n[1] * n[1], n[0] * n[1]};",
                      "const double m[6] = {1.0, n[1], n[0], n[0] * n[0], n[1] * n[1], n[0] * n[1]};"),
    "coeff_channel_index": ("(double)A[(int64_t)(k * 3 + c) * HW + px]", "(double)A[(int64_t)(c * 6 + k) * HW + px]"),
    "quantise_truncates": ("return (uint8_t)floor(v + 0.5);", "return (uint8_t)floor(v);"),
    "render_pixel_axes_swapped": ("const double px = (double)cam->x0 + (double)i * (double)cam->pitch_x;",
                                  "const double px = (double)cam->x0 + (double)j * (double)cam->pitch_x;"),
    "render_depth_sign": ("D[(int64_t)j * cam->W + i] = (double)cam->d0 - (hit && zh < 0.0 ? -zh : 0.0);",
                          "D[(int64_t)j * cam->W + i] = (double)cam->d0 + (hit && zh < 0.0 ? -zh : 0.0);"),
    "render_bisection_reversed": ("if (im && pm <= 0.0) hi = mid; else lo = mid;",
                                  "if (im && pm > 0.0) hi = mid; else lo = mid;"),
}

PINS = os.path.join(os.path.dirname(__file__), "test_oracle_pins.py")


def test_every_mutation_site_exists():
    src = oracle.source()
    for name, (old, new) in MUTATIONS.items():
        assert src.count(old) >= 1, name


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source().replace(old, new)
    variant = tmp_path / "variant.c"
    variant.write_text(src)
    # run the pin suite in a child process against the mutated build
    code = (
        "import sys, pytest, oracle\n"
        f"sys.path.insert(0, {os.path.dirname(os.path.dirname(PINS))!r})\n"
        f"cm = oracle.use_source(open({str(variant)!r}).read(), {str(tmp_path)!r})\n"
        "cm.__enter__()\n"
        "oracle._load = lambda: oracle._lib\n"
        f"sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', {PINS!r}]))\n"
    )
    env = dict(os.environ)
    env["PYTHONPATH"] = os.path.dirname(os.path.dirname(PINS)) + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 1, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}\n{r.stderr[-2000:]}"

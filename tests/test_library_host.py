"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports every
function include/tacsl.h declares, and rejects bad host-visible arguments before
touching the GPU (no CUDA call is reached on these paths)."""
import ctypes as C
import os
import re

import pytest

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]

INVALID, UNSUPPORTED = 1, 2
FAKE = 0x7F0000001000          # 16-byte aligned, never dereferenced on these paths
FAKE_ODD = FAKE + 2


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tacsl.load()


def _declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(tacsl_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("tacsl_sdf_query", "tacsl_penalty_forces", "tacsl_pad_wrench", "tacsl_shade_image",
              "tacsl_tactile_step", "tacsl_last_error", "tacsl_check_errors"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared_functions():
        assert hasattr(lib, n), n


def test_abi_version(lib):
    assert lib.tacsl_abi_version() == 1


def _sdf(n=(8, 8, 8), voxel=1e-3, data=FAKE):
    s = tacsl._Sdf()
    s.n[0], s.n[1], s.n[2] = n
    for a in range(3):
        s.origin[a] = 0.0
    s.voxel = voxel
    s.data = data
    return s


def _set(*sdfs):
    arr = (tacsl._Sdf * len(sdfs))(*sdfs)
    st = tacsl._SdfSet(C.cast(arr, C.POINTER(tacsl._Sdf)), len(sdfs))
    st._keep = arr
    return st


def _params(count=1, k_n=FAKE):
    return tacsl._Params(k_n, FAKE, FAKE, FAKE, count)


def _forces(lib, st, prm, E=2, P=2, T=10, taxels=FAKE, ids=FAKE, pose=FAKE, twist=FAKE, depth=FAKE,
            fn=FAKE, ft=FAKE, wrench=FAKE):
    return lib.tacsl_penalty_forces(C.byref(st), C.byref(prm), E, P, T, taxels, ids, pose, twist, depth, fn, ft,
                                    wrench, None)


@pytest.mark.parametrize("case,code", [
    ("null_set", INVALID), ("n_sdf_zero", INVALID), ("too_many_sdf", INVALID), ("null_grid", INVALID),
    ("small_grid", INVALID), ("bad_voxel", INVALID), ("nan_voxel", INVALID), ("null_params", INVALID),
    ("bad_count", INVALID), ("negative_E", INVALID), ("null_pose", INVALID), ("odd_pose", INVALID),
    ("too_many_taxels", UNSUPPORTED), ("odd_wrench", INVALID), ("huge_grid", UNSUPPORTED),
])
def test_penalty_forces_rejects(lib, case, code):
    st, prm, kw = _set(_sdf()), _params(), {}
    if case == "null_set":
        rc = lib.tacsl_penalty_forces(None, C.byref(prm), 2, 2, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                                      None)
        assert rc == code and "sdf set" in lib.tacsl_last_error().decode()
        return
    if case == "n_sdf_zero":
        st.n_sdf = 0
    elif case == "too_many_sdf":
        st = _set(*[_sdf() for _ in range(tacsl.MAX_SDF + 1)])
    elif case == "null_grid":
        st = _set(_sdf(), _sdf(data=0))
    elif case == "small_grid":
        st = _set(_sdf(n=(8, 2, 8)))
    elif case == "bad_voxel":
        st = _set(_sdf(voxel=-1.0))
    elif case == "nan_voxel":
        st = _set(_sdf(voxel=float("nan")))
    elif case == "huge_grid":
        st = _set(_sdf(n=(2048, 2048, 1024)))
    elif case == "null_params":
        rc = lib.tacsl_penalty_forces(C.byref(st), None, 2, 2, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                                      None)
        assert rc == code
        return
    elif case == "bad_count":
        prm = _params(count=3)
    elif case == "negative_E":
        kw["E"] = -1
    elif case == "null_pose":
        kw["pose"] = 0
    elif case == "odd_pose":
        kw["pose"] = FAKE_ODD
    elif case == "too_many_taxels":
        kw["T"] = 70000
    elif case == "odd_wrench":
        kw["wrench"] = FAKE_ODD
    rc = _forces(lib, st, prm, **kw)
    assert rc == code, lib.tacsl_last_error().decode()
    assert lib.tacsl_last_error().decode() != ""


def test_zero_sized_batches_are_noops(lib):
    st, prm = _set(_sdf()), _params()
    assert _forces(lib, st, prm, E=0) == 0
    assert _forces(lib, st, prm, T=0, P=0) == 0
    assert lib.tacsl_sdf_query(C.byref(st), 0, None, None, None, None, None) == 0
    assert lib.tacsl_pad_wrench(0, 10, None, None, None, None, None) == 0
    sh = tacsl._Shading(4, 8, 1e-4, 1e-4, FAKE, 1)
    assert lib.tacsl_shade_image(C.byref(sh), 0, None, None, None, None) == 0


def _shading(H=12, W=16, px=1e-4, py=1e-4, coeffs=FAKE, S=2):
    return tacsl._Shading(H, W, px, py, coeffs, S)


@pytest.mark.parametrize("case,code", [
    ("w_not_mult4", INVALID), ("w_small", INVALID), ("h_zero", INVALID), ("pitch", INVALID),
    ("sensors", INVALID), ("too_many_sensors", INVALID), ("coeff_align", INVALID), ("depth_align", INVALID),
    ("null_rgb", INVALID), ("null_sid", INVALID), ("neg_B", INVALID), ("huge_image", UNSUPPORTED),
])
def test_shade_image_rejects(lib, case, code):
    sh, B, sid, dep, rgb = _shading(), 4, FAKE, FAKE, FAKE
    if case == "w_not_mult4":
        sh = _shading(W=18)
    elif case == "w_small":
        sh = _shading(W=0)
    elif case == "h_zero":
        sh = _shading(H=0)
    elif case == "pitch":
        sh = _shading(px=0.0)
    elif case == "sensors":
        sh = _shading(S=0)
    elif case == "too_many_sensors":
        sh = _shading(S=17)
    elif case == "coeff_align":
        sh = _shading(coeffs=FAKE + 4)
    elif case == "depth_align":
        dep = FAKE + 4
    elif case == "null_rgb":
        rgb = 0
    elif case == "null_sid":
        sid = 0
    elif case == "neg_B":
        B = -1
    elif case == "huge_image":
        sh = _shading(H=1 << 15, W=1 << 14)
    assert lib.tacsl_shade_image(C.byref(sh), B, sid, dep, rgb, None) == code
    # the fused step applies the same image checks before any launch
    st, prm = _set(_sdf()), _params()
    if case != "neg_B":
        rc = lib.tacsl_tactile_step(C.byref(st), C.byref(prm), 2, 2, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                                    FAKE, C.byref(sh), sid, dep, rgb, None)
        assert rc == code


def test_sdf_query_rejects(lib):
    st = _set(_sdf())
    assert lib.tacsl_sdf_query(C.byref(st), -1, FAKE, FAKE, FAKE, FAKE, None) == INVALID
    assert lib.tacsl_sdf_query(C.byref(st), 5, FAKE, 0, FAKE, FAKE, None) == INVALID
    assert lib.tacsl_sdf_query(C.byref(st), 5, FAKE_ODD, FAKE, FAKE, FAKE, None) == INVALID


def test_pad_wrench_rejects(lib):
    assert lib.tacsl_pad_wrench(-1, 3, FAKE, FAKE, FAKE, FAKE, None) == INVALID
    assert lib.tacsl_pad_wrench(4, 3, FAKE, FAKE, FAKE, 0, None) == INVALID
    assert lib.tacsl_pad_wrench(4, 3, 0, FAKE, FAKE, FAKE, None) == INVALID
    assert lib.tacsl_pad_wrench(4, 70000, FAKE, FAKE, FAKE, FAKE, None) == UNSUPPORTED


def test_check_errors_rejects_null(lib):
    assert lib.tacsl_check_errors(None, None, 1) == INVALID


def test_binding_refuses_cpu_tensors():
    import torch
    with pytest.raises(TypeError):
        tacsl.sdf_query(None, torch.zeros(3, 3), torch.zeros(3, dtype=torch.int32))


def _camera(H=8, W=16, px=1e-4, py=1e-4, z_max=3e-3, d0=0.02):
    return tacsl._Camera(H, W, px, py, -8e-4, -4e-4, d0, z_max)


@pytest.mark.parametrize("cam_kw,code", [
    (dict(W=18), INVALID), (dict(H=0), INVALID), (dict(px=0.0), INVALID), (dict(z_max=0.0), INVALID),
    (dict(d0=float("inf")), INVALID), (dict(H=1 << 15, W=1 << 14), UNSUPPORTED),
])
def test_render_depth_rejects(lib, cam_kw, code):
    st, cam = _set(_sdf()), _camera(**cam_kw)
    assert lib.tacsl_render_depth(C.byref(st), 2, 2, FAKE, FAKE, C.byref(cam), FAKE, None) == code


def test_render_depth_rejects_pointers(lib):
    st, cam = _set(_sdf()), _camera()
    assert lib.tacsl_render_depth(C.byref(st), 2, 2, FAKE, FAKE, C.byref(cam), FAKE + 4, None) == INVALID
    assert lib.tacsl_render_depth(C.byref(st), 2, 2, 0, FAKE, C.byref(cam), FAKE, None) == INVALID
    assert lib.tacsl_render_depth(C.byref(st), 2, 2, FAKE, FAKE, None, FAKE, None) == INVALID
    assert lib.tacsl_render_depth(C.byref(st), 0, 2, FAKE, FAKE, C.byref(cam), FAKE, None) == 0


def test_render_adjoint_rejects(lib):
    from paper_2408_06506_b300 import autograd as ta
    f = ta._lib().tacsl_render_depth_adjoint
    st, cam = _set(_sdf()), _camera()
    assert f(C.byref(st), 2, 2, FAKE, FAKE, C.byref(_camera(W=18)), FAKE, FAKE, FAKE, None) == INVALID
    assert f(C.byref(st), 2, 2, FAKE, FAKE, None, FAKE, FAKE, FAKE, None) == INVALID
    assert f(C.byref(st), -1, 2, FAKE, FAKE, C.byref(cam), FAKE, FAKE, FAKE, None) == INVALID
    for k in range(5):         # obj_id, pad_pose, depth_map, g_depth, grad_pose: NULL or misaligned
        for bad in (0, FAKE + 2):
            args = [FAKE] * 5
            args[k] = bad
            assert f(C.byref(st), 2, 2, args[0], args[1], C.byref(cam), *args[2:], None) == INVALID, (k, bad)
    assert f(C.byref(st), 0, 2, FAKE, FAKE, C.byref(cam), FAKE, FAKE, FAKE, None) == 0


def test_shade_mse_rejects(lib):
    from paper_2408_06506_b300 import autograd as ta
    f = ta._lib().tacsl_shade_mse
    sh = _shading()
    ok = dict(sid=FAKE, dm=FAKE, tgt=FAKE, scale=None, lm=FAKE, gc=FAKE, gd=FAKE)

    def call(shading=sh, B=4, **kw):
        a = dict(ok, **kw)
        return f(C.byref(shading) if shading is not None else None, B, a["sid"], a["dm"], a["tgt"], a["scale"],
                 a["lm"], a["gc"], a["gd"], None)

    assert call(shading=None) == INVALID
    assert call(shading=_shading(W=18)) == INVALID
    assert call(B=-1) == INVALID
    assert call(tgt=0) == INVALID                 # the target stands where the image output would
    assert call(sid=0) == INVALID and call(dm=FAKE + 4) == INVALID
    for k in ("tgt", "scale", "lm", "gc", "gd"):  # 4-byte alignment of the other arrays
        assert call(**{k: FAKE + 2}) == INVALID, k
    assert call(B=0, lm=None, gc=None, gd=None) == 0   # nothing to do


def test_shade_slopes_entry_points_reject(lib):
    """The two-pass depth gradient's entry points refuse bad arguments on the host, before
    any device call (so this runs without a GPU)."""
    from paper_2408_06506_b300 import autograd as ta
    L = ta._lib()
    sh = _shading()
    S = C.byref(sh)
    # tacsl_shade_mse_slopes(shading, B, sid, dm, target, loss_map, grad_coeffs, slopes, stream)
    f = L.tacsl_shade_mse_slopes
    assert f(None, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, None) == INVALID
    assert f(C.byref(_shading(W=18)), 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, None) == INVALID
    assert f(S, -1, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, None) == INVALID
    assert f(S, 4, FAKE, FAKE, FAKE, FAKE, FAKE, None, None) == INVALID          # slopes missing
    assert f(S, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE + 8, None) == INVALID      # not 16-byte aligned
    assert f(S, 4, FAKE, FAKE, FAKE + 2, FAKE, FAKE, FAKE, None) == INVALID      # target
    assert f(S, 4, FAKE, FAKE + 4, FAKE, FAKE, FAKE, FAKE, None) == INVALID      # depth maps
    assert f(S, 0, None, None, None, None, None, None, None) == 0               # nothing to do
    # tacsl_shade_adjoint_slopes(shading, B, sid, dm, g_intensity, grad_coeffs, slopes, stream)
    g = L.tacsl_shade_adjoint_slopes
    assert g(None, 4, FAKE, FAKE, FAKE, FAKE, FAKE, None) == INVALID
    assert g(S, 4, FAKE, FAKE, FAKE, FAKE, None, None) == INVALID
    assert g(S, 4, FAKE, FAKE, FAKE, FAKE + 2, FAKE, None) == INVALID            # grad_coeffs
    assert g(S, 4, 0, FAKE, FAKE, FAKE, FAKE, None) == INVALID                   # sensor ids
    assert g(S, 0, None, None, None, None, None, None) == 0
    # tacsl_shade_depth_from_slopes(shading, B, sid, slopes, scale, grad_depth, stream)
    h = L.tacsl_shade_depth_from_slopes
    assert h(None, 4, FAKE, FAKE, None, FAKE, None) == INVALID
    assert h(S, 4, FAKE, FAKE + 8, None, FAKE, None) == INVALID                 # slopes: 16-byte aligned
    assert h(S, 4, FAKE, FAKE, None, FAKE + 4, None) == INVALID                 # grad_depth: 8-byte aligned
    assert h(S, 4, FAKE, FAKE, FAKE + 2, FAKE, None) == INVALID                 # scale
    assert h(S, 4, FAKE, FAKE, None, None, None) == INVALID
    assert h(S, 0, None, None, None, None, None) == 0


def test_render_step_requires_matching_camera(lib):
    st, prm, cam = _set(_sdf()), _params(), _camera(H=8, W=16)
    sh = _shading(H=12, W=16)
    rc = lib.tacsl_render_step(C.byref(st), C.byref(prm), 2, 2, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                               C.byref(sh), C.byref(cam), FAKE, FAKE, FAKE, None)
    assert rc == INVALID and "camera" in lib.tacsl_last_error().decode()


def test_host_step_workspace_and_rejections(lib):
    ws = lib.tacsl_tactile_step_host_workspace
    ws.restype = C.c_int64
    ws.argtypes = [C.c_int32] * 5
    assert ws(0, 2, 10, 8, 16) == -1 and ws(4, -1, 10, 8, 16) == -1
    one, two = ws(1, 2, 10, 8, 16), ws(2, 2, 10, 8, 16)
    assert one > 0 and two > one and one % 256 == 0
    st, prm = _set(_sdf()), _params()
    sh = _shading(H=8, W=16)
    f = lib.tacsl_tactile_step_host

    def call(chunk=2, wsp=FAKE, wsb=1 << 30, pose=FAKE, dmap=FAKE):
        return f(C.byref(st), C.byref(prm), 4, 2, 10, FAKE, FAKE, pose, FAKE, FAKE, FAKE, FAKE, FAKE, C.byref(sh),
                 FAKE, dmap, FAKE, chunk, wsp, wsb, None)
    assert call(chunk=0) == INVALID
    assert call(wsb=ws(2, 2, 10, 8, 16) - 1) == INVALID
    assert call(wsp=FAKE + 16) == INVALID
    assert call(pose=0) == INVALID
    assert call(dmap=FAKE + 4) == INVALID

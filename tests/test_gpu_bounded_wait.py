"""Device-side bounded waits of the image kernel.

The image kernel streams depth tiles through a shared-memory ring guarded by mbarriers;
every wait on them gives up after a limit (2 s in normal calls), sets TACSL_DEVERR_TIMEOUT
in the device error word and ends the warp's loop, after the producer warp has waited for
the copies it already issued.  tacsl_shade_image_wait_limit takes that limit explicitly:
with 1 ns the waits run out at once (the first tiles have not even been requested when
the compute warps start waiting), the kernel returns, the host reads the timeout bit, and
the next call with the default limit works normally and matches the FP64 oracle."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import synth

from gpu_common import assert_rgb_close, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


def test_image_kernel_wait_runs_out_then_next_call_succeeds(orc):
    sc = synth.scene_objects(seed=13, E=96, P=2, ny=5, nx=6, n=32, H=60, W=80)
    coeffs, sid, dm = dev(sc.coeffs), dev(sc.sensor_id), dev(sc.depth_map)
    sh = tacsl.Shading(coeffs, sc.pitch_x, sc.pitch_y)
    B = sc.E * sc.P
    lib = tacsl.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert tacsl.check_errors(clear=True) == 0
    rgb = torch.zeros(B, sc.H, sc.W, 3, dtype=torch.uint8, device="cuda")
    rc = lib.tacsl_shade_image_wait_limit(C.byref(sh.c), B, C.c_void_p(sid.data_ptr()), C.c_void_p(dm.data_ptr()),
                                          C.c_void_p(rgb.data_ptr()), 1, stream)
    assert rc == 0, lib.tacsl_last_error().decode()
    flags = tacsl.check_errors(clear=True)
    assert flags == tacsl.DEVERR_TIMEOUT, flags
    # the context is intact: a normal call succeeds, reports nothing and shades correctly
    out = tacsl.shade_image(sh, sid, dm)
    assert tacsl.check_errors(clear=True) == 0
    ref_rgb, ref_I, bad = orc.shade(sc.coeffs, sc.pitch_x, sc.pitch_y, sc.sensor_id, sc.depth_map,
                                    with_intensity=True)
    assert bad == 0
    assert_rgb_close(out.cpu().numpy(), ref_rgb, ref_I)
    # wait_ns = 0 is the default limit: the same bytes as tacsl_shade_image
    rgb0 = torch.zeros_like(rgb)
    rc = lib.tacsl_shade_image_wait_limit(C.byref(sh.c), B, C.c_void_p(sid.data_ptr()), C.c_void_p(dm.data_ptr()),
                                          C.c_void_p(rgb0.data_ptr()), 0, stream)
    assert rc == 0
    assert tacsl.check_errors(clear=True) == 0
    assert torch.equal(rgb0, out.view_as(rgb0))


def test_wait_limit_argument_checks_match_shade_image():
    """The host-side argument checks are those of tacsl_shade_image."""
    lib = tacsl.load()
    coeffs = torch.zeros(1, 6, 3, 4, 6, device="cuda")
    sh = tacsl.Shading(coeffs, 1e-4, 1e-4)   # W = 6 is not a multiple of 4
    d = torch.zeros(1, 4, 6, device="cuda")
    sid = torch.zeros(1, dtype=torch.int32, device="cuda")
    rgb = torch.zeros(1, 4, 6, 3, dtype=torch.uint8, device="cuda")
    rc = lib.tacsl_shade_image_wait_limit(C.byref(sh.c), 1, C.c_void_p(sid.data_ptr()), C.c_void_p(d.data_ptr()),
                                          C.c_void_p(rgb.data_ptr()), 1000, None)
    assert rc == 1   # TACSL_ERR_INVALID_ARG: nothing launched
    assert not rgb.any()

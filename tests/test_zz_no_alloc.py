"""The allocation-free entry point (raygs_render_noalloc) against the plan-based path.

raygs_render_noalloc is for callers that may not allocate device memory (a plugin running
inside a host application that owns the device heap, or code under an outer allocator's
budget): it keeps all its intermediate buffers in one fixed device array inside the library.
Here it is called twice in a row through the C ABI on the same inputs and each output is
compared with the output of raygs_preprocess + raygs_bin_sort + raygs_render (the regular
entry points, which work in a caller-allocated workspace), within the parity tolerance the
other tests use.  A scene too large for the fixed array must be refused.
"""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture(scope="module")
def rg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18682_gb300 import build, raygs
    build.build()
    return raygs


def _outputs(torch, npx):
    return (torch.full((npx, 3), -1.0, device="cuda"), torch.full((npx,), -1.0, device="cuda"),
            torch.full((npx,), -1, dtype=torch.int32, device="cuda"))


def test_noalloc_matches_plan_render_twice(rg):
    import torch
    scene = scenes.uniform_scene(2000, seed=31)
    R1, t1 = scenes.look_at([0.3, -0.2, -0.6], [0.0, 0.0, 3.0])
    cams = [scenes.make_camera(64, 64, 64.0, 64.0, 32.0, 32.0),
            scenes.make_camera(70, 45, 50.0, 50.0, R=R1, t=t1, mip=True)]
    st = rg.scene_to_device(scene)
    ref = rg.Renderer(cams, 2000)
    rgb0, T0, nc0 = ref.forward(st)
    torch.cuda.synchronize()
    cfg = rg.make_config()
    sc = rg.make_scene(st)
    for call in range(2):
        rgb, T, nc = _outputs(torch, ref.num_pixels)
        status = rg.raygs_render_noalloc(cams, sc, cfg, rgb, T, nc, check=False)
        assert status == 0, rg.lib().raygs_status_string(status)
        torch.cuda.synchronize()
        assert float((rgb - rgb0).abs().max()) <= TOL, call
        assert float((T - T0).abs().max()) <= TOL, call
        assert torch.equal(nc, nc0), call


def test_noalloc_rejects_scene_beyond_scratch(rg):
    import torch
    n = 400_000   # ~140 bytes per (primitive, view) -> more than the 32 MiB array
    scene = scenes.uniform_scene(n, seed=32)
    st = rg.scene_to_device(scene)
    cams = [scenes.make_camera(32, 32, 32.0, 32.0)]
    rgb, T, nc = _outputs(torch, 32 * 32)
    status = rg.raygs_render_noalloc(cams, rg.make_scene(st), None, rgb, T, nc, check=False)
    assert status == 2  # RAYGS_ERR_CAPACITY, refused before any work
    torch.cuda.synchronize()
    assert float(rgb.min()) == -1.0 and float(rgb.max()) == -1.0   # outputs untouched


def test_noalloc_gs_divergence_and_exact_refusal(rg):
    """The GS divergence runs through the fixed array too (same image as the plan path);
    exact anti-aliasing views need the second record buffer and are refused."""
    import torch
    scene = scenes.uniform_scene(1500, seed=33)
    cams = [scenes.make_camera(64, 48, 60.0, 60.0)]
    st = rg.scene_to_device(scene)
    ref = rg.Renderer(cams, 1500, divergence=1)
    rgb0, T0, nc0 = ref.forward(st)
    torch.cuda.synchronize()
    rgb, T, nc = _outputs(torch, ref.num_pixels)
    status = rg.raygs_render_noalloc(cams, rg.make_scene(st), rg.make_config(divergence=1), rgb, T, nc, check=False)
    assert status == 0, rg.lib().raygs_status_string(status)
    torch.cuda.synchronize()
    assert float((rgb - rgb0).abs().max()) <= TOL and float((T - T0).abs().max()) <= TOL
    assert torch.equal(nc, nc0)
    rgb, T, nc = _outputs(torch, ref.num_pixels)
    status = rg.raygs_render_noalloc([dict(cams[0], mip="exact")], rg.make_scene(st), None, rgb, T, nc,
                                     check=False)
    assert status == 1  # RAYGS_ERR_INVALID_ARG


def test_noalloc_instance_overflow_then_normal_call(rg):
    """Few large primitives over a 1920x1080 view emit far more (primitive, tile) instances
    than the array's remaining space holds: the call renders what fits and reports
    RAYGS_ERR_CAPACITY.  The next call on a small scene is unaffected (same image as the
    plan path)."""
    import torch
    big = scenes.uniform_scene(5000, seed=34)
    big["log_scales"][:] = np.float32(np.log(0.5))
    cams = [scenes.make_camera(1920, 1080, 1000.0, 1000.0)]
    st = rg.scene_to_device(big)
    rgb, T, nc = _outputs(torch, 1920 * 1080)
    status = rg.raygs_render_noalloc(cams, rg.make_scene(st), None, rgb, T, nc, check=False)
    assert status == 2, rg.lib().raygs_status_string(status)  # RAYGS_ERR_CAPACITY after the render
    torch.cuda.synchronize()
    scene = scenes.uniform_scene(2000, seed=31)
    cams = [scenes.make_camera(64, 64, 64.0, 64.0, 32.0, 32.0)]
    st = rg.scene_to_device(scene)
    ref = rg.Renderer(cams, 2000)
    rgb0, T0, nc0 = ref.forward(st)
    torch.cuda.synchronize()
    rgb, T, nc = _outputs(torch, ref.num_pixels)
    status = rg.raygs_render_noalloc(cams, rg.make_scene(st), None, rgb, T, nc, check=False)
    assert status == 0, rg.lib().raygs_status_string(status)
    torch.cuda.synchronize()
    assert float((rgb - rgb0).abs().max()) <= TOL and float((T - T0).abs().max()) <= TOL
    assert torch.equal(nc, nc0)

"""Full-size parity in the benchmark's launch configuration.  The 3M-primitive stereo
batch (16 views of uneven size, 10% near-flat primitives) is rendered as the benchmark
renders it: the tile shape and batch size picked by the autotuner on this workload, the
plan sized from a first pass, the pipeline replayed as a captured CUDA graph.  Sampled
pixels of every view are compared with the oracle, which computes them one by one against
all 3M primitives (forward tolerance: 2e-4 max-abs; only oracle-flagged pixels may be
excluded, and no more than a 0.01% rate allows in the pooled sample)."""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import assert_parity_sampled, compare, sample_pixels, view_slice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stereo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18682_gb300 import build, raygs
    build.build()
    scene, cams = scenes.workload_stereo_batch()
    return scene, cams, raygs.scene_to_device(scene)


def graph_render(cams, st, n, **cfg):
    """Size a plan on a first pass, then render through a captured graph (twice)."""
    import torch
    from paper_2503_18682_gb300 import raygs
    r0 = raygs.Renderer(cams, n, **cfg)
    r0.forward(st)
    cap = int(r0.last_counters["n_instances"] * 1.10 + 65536)
    del r0
    torch.cuda.empty_cache()
    r = raygs.Renderer(cams, n, capacity=cap, **cfg)
    rgb, T, nc = r.alloc_outputs()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        r.forward(st, rgb, T, nc, stream=s)
        raygs.raygs_graph_capture(r.plan, raygs.make_scene(st), rgb, T, nc, s)
        rgb.zero_()
        for _ in range(2):
            raygs.raygs_graph_launch(r.plan, s)
    s.synchronize()
    ctr = raygs.raygs_read_counters(r.plan)
    assert ctr["overflow"] == 0
    return r, rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)


def check_sampled(oracle_lib, scene, cams, r, rgb, T, per_view, ocfg=None):
    stats = []
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        pix, idx = sample_pixels(cam, per_view, seed=100 + v)
        orc = oracle_lib.render(scene, cam, cfg=ocfg, pixels=pix)
        stats.append(compare(rgb[sl][idx], T[sl][idx], orc))
    assert_parity_sampled(stats)


def test_stereo_batch_autotuned_graph_sampled(oracle_lib, stereo):
    import torch
    from paper_2503_18682_gb300 import raygs
    scene, cams, st = stereo
    n = scene["means"].shape[0]
    r0 = raygs.Renderer(cams, n)
    r0.forward(st)
    cap = int(r0.last_counters["n_instances"] * 3.2 + 65536)
    del r0
    torch.cuda.empty_cache()
    kw, _ = raygs.autotune(cams, st, cap, iters=1)
    torch.cuda.empty_cache()
    shape = {k: kw[k] for k in ("tile_w", "tile_h", "batch_records")}
    r, rgb, T = graph_render(cams, st, n, **shape)
    check_sampled(oracle_lib, scene, cams, r, rgb, T, per_view=64)


def test_stereo_batch_gs_divergence_sampled(oracle_lib, stereo):
    scene, cams, st = stereo
    r, rgb, T = graph_render(cams, st, scene["means"].shape[0], divergence=1)
    check_sampled(oracle_lib, scene, cams, r, rgb, T, per_view=32, ocfg=dict(divergence=1))


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_precision_workload_full_size_sampled(oracle_lib, dt):
    """The 6M-primitive precision workload at full size (4 views at 3840x2160 and the same
    poses at 960x540 with the MIP filter), SH and log-scales stored in FP16 / BF16 and
    opacity in FP16: the reduced form is bit-equal to the FP32 form of the widened stored
    values, and 48 sampled pixels per view match the oracle on those values."""
    import torch
    from paper_2503_18682_gb300 import build, raygs
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    scene, cams = scenes.workload_precision()
    red = scenes.to_storage(scene, dt)
    wide = scenes.widen(red)
    del scene
    n = red["means"].shape[0]
    outs = []
    for sc in (red, wide):
        r = raygs.Renderer(cams, n)
        rgb, T, _ = r.forward(raygs.scene_to_device(sc))
        torch.cuda.synchronize()
        outs.append((r, rgb.cpu().numpy(), T.cpu().numpy()))
        del rgb, T
        torch.cuda.empty_cache()
    (r, rgb_red, T_red), (_, rgb_wide, T_wide) = outs
    assert np.array_equal(rgb_red, rgb_wide) and np.array_equal(T_red, T_wide)
    stats = []
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        pix, idx = sample_pixels(cam, 48, seed=200 + v)
        orc = oracle_lib.render(wide, cam, pixels=pix)
        stats.append(compare(rgb_red[sl][idx].astype(np.float64), T_red[sl][idx].astype(np.float64), orc))
    assert_parity_sampled(stats)

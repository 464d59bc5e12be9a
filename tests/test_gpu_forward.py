"""Forward parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element, on seeded scenes that span several tiles and ragged image edges; plus edge cases.
Tolerance: 2e-4 max-abs per channel (and on T), excluding at most 0.01% of pixels, each of
which the oracle flags as sitting at the opacity cut-off (or reached by a primitive whose skip
decision lies within FP64 rounding of its threshold)."""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import assert_parity, assert_parity_sampled, compare, gpu_render, sample_pixels, view_slice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18682_gb300 import build
    build.build()


def check_views(scene, cams, oracle_lib, **cfg):
    r, _, rgb, T, nc = gpu_render(scene, cams, **cfg)
    out = []
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        orc = oracle_lib.render(scene, cam)
        st = compare(rgb[sl], T[sl], orc)
        assert_parity(st)
        out.append(st)
    return r, out


def test_small_scene_matches_stored_oracle_values():
    """The CUDA image of the 64x64 scene against the oracle values stored under
    tests/golden (written from the oracle alone), at the stored pixels."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "small_uniform_64x64.txt")
    a = np.loadtxt(path, comments="#")
    pix = a[:, :2].astype(np.int64)
    orc = dict(rgb=a[:, 2:5], T=a[:, 5], flags=a[:, 6].astype(np.int32))
    scene, cams = scenes.workload_small()
    _, _, rgb, T, _ = gpu_render(scene, cams)
    idx = pix[:, 1] * 64 + pix[:, 0]
    assert_parity(compare(rgb[idx], T[idx], orc))


def test_small_uniform_scene(oracle_lib):
    """1 view 64x64, 1,000 primitives, SH degree 0: the small workload, full image."""
    scene, cams = scenes.workload_small()
    r, st = check_views(scene, cams, oracle_lib)
    assert r.last_counters["n_visible"] > 500


@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (32, 16), (8, 8)])
def test_ragged_multiview(oracle_lib, tile):
    """3 views of ragged sizes and poses in one batch, every tile shape."""
    scene = scenes.uniform_scene(2000, seed=7)
    R1, t1 = scenes.look_at([0.4, -0.3, -0.5], [0.0, 0.0, 3.0])
    R2, t2 = scenes.look_at([-1.5, 0.5, 3.0], [0.0, 0.0, 3.0])
    cams = [scenes.make_camera(70, 53, 60.0, 58.0, 33.3, 27.1),
            scenes.make_camera(33, 17, 20.0, 20.0, R=R1, t=t1),
            scenes.make_camera(100, 64, 80.0, 80.0, R=R2, t=t2)]
    check_views(scene, cams, oracle_lib, tile_w=tile[0], tile_h=tile[1])


def test_blob_scene_sh3_mip(oracle_lib):
    """Blob-mixture scene with degree-3 colour and the MIP filter (the 720p MIP workload
    shrunk to 20k primitives at 320x180, fx = fy = 250)."""
    scene = scenes.blob_scene(20000, seed=1)
    cams = [scenes.make_camera(320, 180, 250.0, 250.0, mip=True)]
    check_views(scene, cams, oracle_lib)


def test_blob_scene_plain_sh3(oracle_lib):
    scene = scenes.blob_scene(20000, seed=2)
    cams = [scenes.make_camera(320, 180, 250.0, 250.0)]
    check_views(scene, cams, oracle_lib)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_sh_degrees(oracle_lib, deg):
    """Every SH degree against the oracle, full image: the vertex stage stages FP32 rows of
    whole 16-byte slots (degrees 1 and 3) with asynchronous copies and the others (degrees
    0 and 2) synchronously."""
    scene = scenes.blob_scene(6000, seed=40 + deg, sh_degree=deg)
    R1, t1 = scenes.look_at([1.0, 0.5, 0.0], [0.0, 0.0, 6.0])
    cams = [scenes.make_camera(96, 64, 80.0, 80.0), scenes.make_camera(64, 80, 70.0, 70.0, R=R1, t=t1)]
    check_views(scene, cams, oracle_lib)


@pytest.mark.parametrize("fp64", [2, 1, 0])
def test_near_degenerate_primitives(oracle_lib, fp64):
    """10% near-flat primitives (axis ratio > 1e3) seen from the stereo-batch poses, shrunk
    to 20k primitives and small views; FP64 vertex stage in every view (2), only in views
    where the float32 solve is ill-conditioned (1, default), never (0)."""
    scene = scenes.blob_scene(20000, seed=3, degenerate_frac=0.10)
    poses = scenes.stereo_batch_cameras(seed=3, n_pairs=1, n_extra=2)
    sizes = [(160, 172), (160, 172), (200, 150), (123, 97)]
    cams = [scenes.make_camera(w, h, 0.53 * w, 0.53 * w, R=c["R"], t=c["t"])
            for (w, h), c in zip(sizes, poses)]
    check_views(scene, cams, oracle_lib, fp64_degenerate=fp64)


def test_empty_and_all_culled(oracle_lib):
    import torch
    from paper_2503_18682_gb300 import raygs
    cams = [scenes.make_camera(40, 24, 30.0, 30.0)]
    empty = scenes.uniform_scene(0, seed=0)
    r, _, rgb, T, nc = gpu_render(empty, cams)
    assert np.all(rgb == 0) and np.all(T == 1) and np.all(nc == 0)
    behind = scenes.uniform_scene(500, seed=1)
    behind["means"][:, 2] = -behind["means"][:, 2]
    r, _, rgb, T, nc = gpu_render(behind, cams)
    assert np.all(rgb == 0) and np.all(T == 1)
    assert r.last_counters["n_visible"] == 0


def test_camera_inside_and_full_view_quads(oracle_lib):
    """Primitives that contain the camera (c^2 <= kappa, skipped) and large primitives close
    to the camera whose quad reaches behind it (full-view rectangle)."""
    rng = np.random.default_rng(12)
    n = 300
    sc = scenes.uniform_scene(n, seed=12)
    sc["means"] = np.concatenate([
        rng.uniform([-0.3, -0.3, 0.05], [0.3, 0.3, 0.4], (n // 3, 3)),
        rng.uniform([-1, -1, 0.5], [1, 1, 1.5], (n // 3, 3)),
        rng.uniform([-1, -1, 2], [1, 1, 4], (n - 2 * (n // 3), 3))]).astype(np.float32)
    sc["log_scales"][: 2 * (n // 3)] = rng.uniform(np.log(0.05), np.log(0.6), (2 * (n // 3), 3)).astype(np.float32)
    cams = [scenes.make_camera(96, 80, 70.0, 70.0)]
    check_views(sc, cams, oracle_lib)


def test_nonfinite_attributes_are_culled(oracle_lib):
    scene, cams = scenes.workload_small()
    scene = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    scene["means"][3, 0] = np.nan
    scene["log_scales"][10, 2] = np.inf
    scene["quats"][20] = 0.0
    r, _, rgb, T, nc = gpu_render(scene, cams)
    assert r.last_counters["n_nonfinite"] == 3
    keep = np.ones(1000, bool)
    keep[[3, 10, 20]] = False
    ref = oracle_lib.render(scenes.subset(scene, keep), cams[0])
    assert_parity(compare(rgb, T, ref))


def test_capacity_overflow_is_reported_and_retried(oracle_lib):
    from paper_2503_18682_gb300 import raygs
    import torch
    scene, cams = scenes.workload_small()
    r = raygs.Renderer(cams, 1000, capacity=64)
    st = raygs.scene_to_device(scene)
    sc = raygs.make_scene(st)
    rgb, T, nc = r.alloc_outputs()
    raygs.raygs_preprocess(r.plan, sc)
    raygs.raygs_bin_sort(r.plan)
    raygs.raygs_render(r.plan, rgb, T, nc)
    ctr = raygs.raygs_read_counters(r.plan)
    assert ctr["overflow"] == 1 and ctr["n_instances"] > 64
    rgb, T, nc = r.forward(st)      # regrows the plan
    torch.cuda.synchronize()
    assert r.last_counters["overflow"] == 0
    assert_parity(compare(rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64),
                          oracle_lib.render(scene, cams[0])))


def test_graph_capture_matches_direct(oracle_lib):
    import torch
    from paper_2503_18682_gb300 import raygs
    scene = scenes.uniform_scene(2000, seed=9)
    cams = [scenes.make_camera(70, 53, 60.0, 58.0), scenes.make_camera(48, 40, 40.0, 40.0)]
    r = raygs.Renderer(cams, 2000)
    st = raygs.scene_to_device(scene)
    rgb0, T0, nc0 = r.forward(st)
    s = torch.cuda.Stream()
    rgb, T, nc = r.alloc_outputs()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        raygs.raygs_graph_capture(r.plan, raygs.make_scene(st), rgb, T, nc, s)
        for _ in range(3):
            raygs.raygs_graph_launch(r.plan, s)
    s.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(rgb, rgb0) and torch.equal(T, T0) and torch.equal(nc, nc0)


def test_full_size_mip_720p_sampled(oracle_lib):
    """The 720p MIP workload at full size (500k primitives, 1280x720): 1,536 sampled
    pixels against the oracle, computed one by one."""
    scene, cams = scenes.workload_mip_720p()
    r, _, rgb, T, nc = gpu_render(scene, cams)
    pix, idx = sample_pixels(cams[0], 1536, seed=5)
    orc = oracle_lib.render(scene, cams[0], pixels=pix)
    assert_parity_sampled([compare(rgb[idx], T[idx], orc)])


def test_autotuner_picks_a_compiled_shape(oracle_lib):
    """raygs_autotune times every tile shape on the caller's scene and views; the chosen
    shape renders the same image (oracle parity)."""
    from paper_2503_18682_gb300 import raygs
    scene = scenes.uniform_scene(3000, seed=13)
    R1, t1 = scenes.look_at([0.4, -0.3, -0.5], [0.0, 0.0, 3.0])
    cams = [scenes.make_camera(96, 72, 80.0, 80.0), scenes.make_camera(50, 41, 40.0, 40.0, R=R1, t=t1)]
    st = raygs.scene_to_device(scene)
    kw, times = raygs.autotune(cams, st, capacity=1 << 20)
    assert (kw["tile_w"], kw["tile_h"], kw["batch_records"]) in raygs.AUTOTUNE_CANDIDATES
    assert len(times) == 8 and all(v > 0 for v in times.values()), times
    assert times[f"{kw['tile_w']}x{kw['tile_h']}/b{kw['batch_records']}"] == min(times.values())
    check_views(scene, cams, oracle_lib, tile_w=kw["tile_w"], tile_h=kw["tile_h"], batch_records=kw["batch_records"])


@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (32, 16), (8, 8)])
def test_segment_filter_never_changes_a_pixel(tile):
    """The rasteriser skips a thread's row segment when a conservative bound says no pixel
    of it can pass the support test; the instrumented variant tests every pixel.  Both
    images (rgb, T, last index) must be bit-identical, on large, small, MIP-filtered and
    near-degenerate footprints."""
    import torch
    from paper_2503_18682_gb300 import raygs
    scene = scenes.blob_scene(60000, seed=21, degenerate_frac=0.1)
    R1, t1 = scenes.look_at([0.0, 0.0, 0.5], [0.0, 0.0, 6.0])
    R2, t2 = scenes.look_at([2.5, 1.0, 3.0], [0.0, 0.0, 6.0])
    cams = [scenes.make_camera(301, 197, 260.0, 260.0, R=R1, t=t1),
            scenes.make_camera(256, 160, 500.0, 500.0, R=R2, t=t2),
            scenes.make_camera(120, 90, 90.0, 90.0, R=R2, t=t2, mip=True)]
    r = raygs.Renderer(cams, scene["means"].shape[0], tile_w=tile[0], tile_h=tile[1])
    st = raygs.scene_to_device(scene)
    rgb, T, nc = r.forward(st)
    rgb2, T2, nc2 = r.alloc_outputs()
    evals, comps = r.counted_render(rgb2, T2, nc2)
    torch.cuda.synchronize()
    assert 0 < comps <= evals
    assert torch.equal(rgb, rgb2) and torch.equal(T, T2) and torch.equal(nc, nc2)

"""Exact, pixel-dependent anti-aliasing (Sec. 5, the form Eq. mip approximates) on the GPU
against the oracle's plain FP64 evaluation of it, element by element, with the forward
tolerance (2e-4 max-abs per channel and on T, at most 0.01% of pixels excluded, each
flagged by the oracle at a cut-off / stop boundary).  Full images on small scenes cover
the binning bound: a pixel the inflated support dropped would show up as a missing
contribution."""
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


def exact(cams):
    return [dict(c, mip="exact") for c in cams]


def check_views(scene, cams, oracle_lib, sig2=0.1, **cfg):
    r, _, rgb, T, nc = gpu_render(scene, cams, mip_sigma2=sig2, **cfg)
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        assert_parity(compare(rgb[sl], T[sl], oracle_lib.render(scene, cam, cfg=dict(mip_sigma2=sig2))))
    return r, rgb, T


@pytest.mark.parametrize("sig2", [0.1, 4.0])
def test_small_uniform_scene(oracle_lib, sig2):
    scene, cams = scenes.workload_small()
    r, _, _ = check_views(scene, exact(cams), oracle_lib, sig2=sig2)
    assert r.last_counters["n_visible"] > 500


@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (32, 16), (8, 8)])
def test_ragged_multiview(oracle_lib, tile):
    scene = scenes.uniform_scene(2000, seed=7)
    R1, t1 = scenes.look_at([0.4, -0.3, -0.5], [0.0, 0.0, 3.0])
    R2, t2 = scenes.look_at([-1.5, 0.5, 3.0], [0.0, 0.0, 3.0])
    cams = [scenes.make_camera(70, 53, 60.0, 58.0, 33.3, 27.1),
            scenes.make_camera(33, 17, 20.0, 20.0, R=R1, t=t1),
            scenes.make_camera(100, 64, 80.0, 80.0, R=R2, t=t2)]
    check_views(scene, exact(cams), oracle_lib, sig2=2.0, tile_w=tile[0], tile_h=tile[1])


def test_blob_scene_sh3(oracle_lib):
    """The 720p workload's generator shrunk to 20k primitives at 320x180 (fx = fy = 250)."""
    scene = scenes.blob_scene(20000, seed=1)
    cams = exact([scenes.make_camera(320, 180, 250.0, 250.0)])
    check_views(scene, cams, oracle_lib)


@pytest.mark.parametrize("fp64", [1, 0])
def test_near_degenerate_primitives(oracle_lib, fp64):
    """10% near-flat primitives: their axis ratio defeats the lambda bound, so those pairs
    cover their whole view (and the FP64 stage rebuilds them when fp64 = 1)."""
    scene = scenes.blob_scene(20000, seed=3, degenerate_frac=0.10)
    poses = scenes.stereo_batch_cameras(seed=3, n_pairs=1, n_extra=2)
    sizes = [(160, 172), (160, 172), (200, 150), (123, 97)]
    cams = exact([scenes.make_camera(w, h, 0.53 * w, 0.53 * w, R=c["R"], t=c["t"])
                  for (w, h), c in zip(sizes, poses)])
    check_views(scene, cams, oracle_lib, fp64_degenerate=fp64)


def test_primitives_near_the_camera(oracle_lib):
    """Primitives that contain the camera (skipped, Eq. c on the plain primitive) and large
    ones close to it, whose inflated support reaches the camera (whole-view pairs)."""
    rng = np.random.default_rng(12)
    n = 300
    sc = scenes.uniform_scene(n, seed=12)
    sc["means"] = np.concatenate([
        rng.uniform([-0.3, -0.3, 0.05], [0.3, 0.3, 0.4], (n // 3, 3)),
        rng.uniform([-1, -1, 0.5], [1, 1, 1.5], (n // 3, 3)),
        rng.uniform([-1, -1, 2], [1, 1, 4], (n - 2 * (n // 3), 3))]).astype(np.float32)
    sc["log_scales"][: 2 * (n // 3)] = rng.uniform(np.log(0.05), np.log(0.6), (2 * (n // 3), 3)).astype(np.float32)
    cams = exact([scenes.make_camera(96, 80, 70.0, 70.0)])
    check_views(sc, cams, oracle_lib, sig2=2.0)


def test_exact_differs_from_the_approximation(oracle_lib):
    """With a strong filter on a wide view the pixel-dependent form and Eq. mip give
    different images (each matching its own oracle), and agree on a narrow view of small,
    distant primitives, where the approximation's assumptions hold."""
    scene = scenes.blob_scene(20000, seed=5)
    wide = [scenes.make_camera(160, 120, 60.0, 60.0)]
    _, rgb_x, _ = check_views(scene, exact(wide), oracle_lib, sig2=4.0)
    r, _, rgb_a, T_a, _ = gpu_render(scene, [dict(wide[0], mip=True)], mip_sigma2=4.0)
    assert_parity(compare(rgb_a, T_a, oracle_lib.render(scene, dict(wide[0], mip=True), cfg=dict(mip_sigma2=4.0))))
    assert np.abs(rgb_x - rgb_a).max() > 0.01


def test_full_size_720p_sampled(oracle_lib):
    """The 720p workload (500k primitives, 1280x720) with the exact form: 1,024 sampled
    pixels against the oracle."""
    scene, cams = scenes.workload_mip_720p()
    cams = exact(cams)
    r, _, rgb, T, nc = gpu_render(scene, cams)
    pix, idx = sample_pixels(cams[0], 1024, seed=6)
    orc = oracle_lib.render(scene, cams[0], pixels=pix)
    assert_parity_sampled([compare(rgb[idx], T[idx], orc)])


def test_refusals():
    from paper_2503_18682_gb300 import raygs
    cams = [scenes.make_camera(32, 32, 30.0, 30.0, mip="exact"), scenes.make_camera(32, 32, 30.0, 30.0)]
    with pytest.raises(RuntimeError):      # exact and other views in one batch
        raygs.Renderer(cams, 10)
    with pytest.raises(RuntimeError):      # GS has no anti-aliasing term
        raygs.Renderer(cams[:1], 10, divergence=1)
    with pytest.raises(RuntimeError):      # mode out of range
        raygs.Renderer([dict(cams[1], mip=3)], 10)

"""Supersampled anti-aliasing (the box-filter counterpart of the paper's MSAA comparison,
Sec. 6): views rendered at factor-times the resolution and resolved by the library's
block-mean kernel, against the FP64 oracle rendered at the same sub-pixel rays and averaged
here.  Factor 1 is the identity; a view whose size is not a multiple of the factor is
refused."""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import TOL, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18682_gb300 import build
    build.build()


def _render_resolved(scene, cams, factor):
    import torch
    from paper_2503_18682_gb300 import raygs
    hi = raygs.supersampled_cameras(cams, factor)
    r = raygs.Renderer(hi, scene["means"].shape[0])
    st = raygs.scene_to_device(scene)
    rgb_hi, T_hi, _ = r.forward(st)
    n_lo = sum(c["width"] * c["height"] for c in cams)
    rgb = torch.empty((n_lo, 3), dtype=torch.float32, device="cuda")
    T = torch.empty(n_lo, dtype=torch.float32, device="cuda")
    raygs.raygs_resolve_supersampled(r.plan, factor, rgb_hi, T_hi, rgb, T)
    torch.cuda.synchronize()
    return hi, rgb_hi.cpu().numpy(), T_hi.cpu().numpy(), rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)


def test_supersampled_views_match_oracle_sub_pixel_mean(oracle_lib):
    scene = scenes.uniform_scene(1500, seed=51)
    R1, t1 = scenes.look_at([0.3, 0.1, -0.4], [0.0, 0.0, 3.0])
    cams = [scenes.make_camera(64, 48, 60.0, 60.0), scenes.make_camera(40, 30, 30.0, 30.0, R=R1, t=t1)]
    f = 2
    hi, _, _, rgb, T = _render_resolved(scene, cams, f)
    base = 0
    for cam, ch in zip(cams, hi):
        w, h = cam["width"], cam["height"]
        orc = oracle_lib.render(scene, ch)
        o_rgb = orc["rgb"].reshape(h, f, w, f, 3).mean(axis=(1, 3)).reshape(-1, 3)
        o_T = orc["T"].reshape(h, f, w, f).mean(axis=(1, 3)).reshape(-1)
        o_flag = np.bitwise_or.reduce(orc["flags"].reshape(h, f, w, f), axis=(1, 3)).reshape(-1)
        st = compare(rgb[base:base + w * h], T[base:base + w * h], dict(rgb=o_rgb, T=o_T, flags=o_flag))
        assert st["n_unexplained"] == 0 and st["max_err"] <= TOL and st["max_err_T"] <= TOL, st
        base += w * h


def test_factor_one_is_identity_and_bad_factor_is_refused():
    import torch
    from paper_2503_18682_gb300 import raygs
    scene = scenes.uniform_scene(500, seed=52)
    cams = [scenes.make_camera(30, 20, 30.0, 30.0)]
    _, rgb_hi, T_hi, rgb, T = _render_resolved(scene, cams, 1)
    assert np.array_equal(rgb.astype(np.float32), rgb_hi) and np.array_equal(T.astype(np.float32), T_hi)
    r = raygs.Renderer(cams, 500)
    out = torch.empty((30 * 20, 3), device="cuda")
    with pytest.raises(raygs.RayGSError):
        raygs.raygs_resolve_supersampled(r.plan, 4, out, None, out)   # 30 x 20 is not a multiple of 4

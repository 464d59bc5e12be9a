"""Reduced-precision storage (SH coefficients and log-scales in FP16 or BF16, opacity logits
in FP16, means and quaternions FP32; all arithmetic FP32): the precision workload shrunk
to 50k primitives, 4 poses at 384x216 plus the same poses at 96x54 with the MIP filter.

  * the reduced form equals the FP32 form rendered from the same stored values (widened
    exactly to float32) to <= 1e-3 max-abs (the kernels convert on load, so exactly);
  * both match the FP64 oracle on the stored values (parity tolerance, sampled pixels);
  * the storage rounding itself (reduced form vs the unrounded FP32 scene) is reported.
"""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import assert_parity, compare, gpu_render, sample_pixels, view_slice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18682_gb300 import build
    build.build()


def shrunk_cameras():
    full = scenes.precision_cameras(seed=4)
    out = []
    for c in full:
        s = 0.1 if c["width"] == 3840 else 0.1
        w, h = int(round(c["width"] * s)), int(round(c["height"] * s))
        out.append(scenes.make_camera(w, h, float(c["fx"]) * s, float(c["fy"]) * s, R=c["R"], t=c["t"],
                                      mip=c["mip"]))
    return out


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_reduced_precision_storage(oracle_lib, dt):
    scene = scenes.blob_scene(50000, seed=4)
    cams = shrunk_cameras()
    red = scenes.to_storage(scene, dt)
    wide = scenes.widen(red)
    r, _, rgb_red, T_red, _ = gpu_render(red, cams)
    _, _, rgb_wide, T_wide, _ = gpu_render(wide, cams)
    _, _, rgb_f32, _, _ = gpu_render(scene, cams)
    assert np.abs(rgb_red - rgb_wide).max() <= 1e-3
    assert np.abs(T_red - T_wide).max() <= 1e-3
    assert np.array_equal(rgb_red, rgb_wide)            # conversion on load is exact
    q_err = np.abs(rgb_red - rgb_f32).max()
    print(f"\n{dt}: storage rounding vs unrounded FP32 scene: max-abs {q_err:.3g}, "
          f"PSNR {psnr(rgb_red, rgb_f32):.1f} dB")
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        pix, idx = sample_pixels(cam, 400, seed=v)
        orc = oracle_lib.render(wide, cam, pixels=pix)
        assert_parity(compare(rgb_red[sl][idx], T_red[sl][idx], orc))

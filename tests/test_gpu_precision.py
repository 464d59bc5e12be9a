"""Reduced-precision storage (all arithmetic FP32 after the load): the precision workload
shrunk to 50k primitives, 4 poses at 384x216 plus the same poses at 96x54 with the MIP
filter.

  * The literal forms (SH and log-scales in FP16 or BF16, opacity logits in FP16): the
    reduced form equals, bit for bit, the FP32 form rendered from the same stored values
    widened to float32 (the kernels convert on load, exactly), and matches the FP64 oracle
    on those values.  Against the unrounded FP32 scene their error is the rounding of the
    stored log-scales and logits, reported here and not asserted: it exceeds 1e-3.
  * The SH-only form (SH coefficients in FP16, the rest FP32): against the FP32 form of
    the unrounded scene on the same GPU, max-abs <= 1e-3 (the reduced-precision target),
    asserted on every pixel.  The SH coefficients are half of the attribute bytes.
  * Every form against the FP64 oracle of the unrounded scene on sampled pixels: max-abs
    and PSNR reported; the FP32 and SH-only forms asserted within the parity tolerance plus
    the target (2e-4 + 1e-3).
"""
import json
import os

import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import TOL, assert_parity, assert_parity_sampled, compare, gpu_render, sample_pixels, view_slice

pytestmark = pytest.mark.gpu

TARGET = 1e-3  # reduced-precision form against the FP32 form, max-abs per channel


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
        s = 0.1
        w, h = int(round(c["width"] * s)), int(round(c["height"] * s))
        out.append(scenes.make_camera(w, h, float(c["fx"]) * s, float(c["fy"]) * s, R=c["R"], t=c["t"],
                                      mip=c["mip"]))
    return out


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


def _record(**kw):
    log = os.environ.get("RAYGS_PRECISION_LOG")
    if log:
        with open(log, "a") as f:
            f.write(json.dumps(kw) + "\n")


@pytest.fixture(scope="module")
def f32_case():
    scene = scenes.blob_scene(50000, seed=4)
    cams = shrunk_cameras()
    r, _, rgb, T, _ = gpu_render(scene, cams)
    return scene, cams, r, rgb, T


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_literal_reduced_forms_are_exact_on_their_stored_values(oracle_lib, f32_case, dt):
    scene, cams, _, rgb_f32, _ = f32_case
    red = scenes.to_storage(scene, dt)
    wide = scenes.widen(red)
    r, _, rgb_red, T_red, _ = gpu_render(red, cams)
    _, _, rgb_wide, T_wide, _ = gpu_render(wide, cams)
    assert np.array_equal(rgb_red, rgb_wide) and np.array_equal(T_red, T_wide)  # exact conversion on load
    q_err = float(np.abs(rgb_red - rgb_f32).max())
    _record(test="literal_vs_unrounded_f32", form=dt, max_abs=q_err, psnr_db=psnr(rgb_red, rgb_f32))
    print(f"\n{dt}: storage rounding vs unrounded FP32 scene: max-abs {q_err:.3g} "
          f"(target {TARGET:g} not met by this form), PSNR {psnr(rgb_red, rgb_f32):.1f} dB")
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        pix, idx = sample_pixels(cam, 400, seed=v)
        orc = oracle_lib.render(wide, cam, pixels=pix)
        assert_parity(compare(rgb_red[sl][idx], T_red[sl][idx], orc))


def test_sh_f16_form_meets_the_target(f32_case):
    """SH coefficients stored in FP16 (log-scales, opacity logits FP32): every pixel within
    1e-3 of the FP32 form of the unrounded scene."""
    scene, cams, _, rgb_f32, T_f32 = f32_case
    red = scenes.to_storage_form(scene, sh="f16")
    assert red["sh"].dtype == np.float16
    _, _, rgb_red, T_red, _ = gpu_render(red, cams)
    err = float(np.abs(rgb_red - rgb_f32).max())
    _record(test="sh_f16_vs_unrounded_f32", max_abs=err, psnr_db=psnr(rgb_red, rgb_f32))
    print(f"\nsh_f16: max-abs vs FP32 {err:.3g}, PSNR {psnr(rgb_red, rgb_f32):.1f} dB")
    assert err <= TARGET
    assert np.array_equal(T_red, T_f32)  # colour storage does not touch opacity or T


@pytest.mark.parametrize("form", ["f32", "sh_f16", "f16", "bf16"])
def test_forms_against_the_oracle_of_the_unrounded_scene(oracle_lib, f32_case, form):
    scene, cams, r, rgb_f32, _ = f32_case
    sh, sc, op = dict(f32=("f32", "f32", "f32"), sh_f16=("f16", "f32", "f32"), f16=("f16", "f16", "f16"),
                      bf16=("bf16", "bf16", "f16"))[form]
    red = scene if form == "f32" else scenes.to_storage_form(scene, sh=sh, scales=sc, opacity=op)
    _, _, rgb, T, _ = gpu_render(red, cams)
    worst, sq, npx, stats = 0.0, 0.0, 0, []
    tol = TOL + (TARGET if form == "sh_f16" else 0.0)
    for v in (0, 4):
        cam = cams[v]
        sl = view_slice(r, v)
        pix, idx = sample_pixels(cam, 600, seed=100 + v)
        orc = oracle_lib.render(scene, cam, pixels=pix)
        d = rgb[sl][idx] - orc["rgb"]
        worst = max(worst, float(np.abs(d).max()))
        sq += float(np.sum(d ** 2))
        npx += d.size
        stats.append(compare(rgb[sl][idx], T[sl][idx], orc, tol=tol))
    p = float("inf") if sq == 0 else 10 * np.log10(npx / sq)
    _record(test="form_vs_oracle_unrounded", form=form, max_abs=worst, psnr_db=p)
    print(f"\n{form}: vs FP64 oracle of the unrounded scene (1,200 sampled pixels): max-abs {worst:.3g}, "
          f"PSNR {p:.1f} dB")
    if form in ("f32", "sh_f16"):
        assert_parity_sampled(stats, tol=tol)

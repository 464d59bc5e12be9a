"""The oracle's exclusion flags (CPU): which pixels the parity rule may exclude.

FLAG_BORDER marks the pixels reached (opacity >= p_min / 2) by a primitive whose skip
decision of Eq. c (camera inside, c^2 <= kappa) lies within FP64 rounding of its
threshold, and no other pixel.  The case is built from a thin primitive seen from near its
own plane, where the rounding of the camera-frame mean, divided by the thin scale, widens
that band.  The reached pixels are recomputed from the plain definition (Eq. Q_ray through
oracle.D_ray with Sigma^-1 written out here), not from the renderer's loop.
"""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes

PMIN = 1.0 / 255.0
FLAG_CUTOFF, FLAG_STOP, FLAG_BORDER = 1, 2, 4


def _thin_plane(logit):
    # R = I: thin axis x (scale 1e-6) at x = 3e-6, so that m_x = 3; huge in-plane scales
    s = np.array([1e-6, 50.0, 50.0])
    sc = dict(means=np.array([[3e-6, 0.0, 3.0]], np.float32),
              log_scales=np.log(s).astype(np.float32)[None, :],
              quats=np.array([[1.0, 0.0, 0.0, 0.0]], np.float32),
              opacity_logits=np.array([logit], np.float32),
              sh=np.full((1, 1, 3), 0.5, np.float32), sh_degree=0)
    return sc


def _logit_at_threshold():
    """The float32 logit whose kappa = -2 ln(p_min / o) equals c^2 of the thin primitive."""
    sc = _thin_plane(0.0)
    mu = sc["means"][0].astype(np.float64)
    s = np.exp(sc["log_scales"][0].astype(np.float64))
    c2 = float(np.sum((mu / s) ** 2))
    o = PMIN * np.exp(c2 / 2.0)
    return np.float32(np.log(o / (1.0 - o))), c2


def test_border_flag_marks_only_the_reached_pixels(oracle_lib):
    logit, c2 = _logit_at_threshold()
    sc = _thin_plane(logit)
    cam = scenes.make_camera(40, 30, 30.0, 30.0)
    g = oracle_lib.prepare(sc, cam)[0]
    OG = oracle_lib.OG
    assert abs(g[OG["C2"]] - g[OG["KAPPA"]]) < 1e-5 * g[OG["KAPPA"]], (g[OG["C2"]], g[OG["KAPPA"]])
    assert g[OG["BORDER"]] == 1
    out = oracle_lib.render(sc, cam)
    flagged = (out["flags"] & FLAG_BORDER) != 0
    # reached: tau > 0 and o exp(-D/2) >= p_min / 2, from Eq. Q_ray
    o = 1.0 / (1.0 + np.exp(-np.float64(logit)))
    s = np.exp(sc["log_scales"][0].astype(np.float64))
    Si = np.diag(1.0 / s ** 2)
    mu = sc["means"][0].astype(np.float64)
    k_reach = 2.0 * np.log(2.0 * o / PMIN)
    reached = np.zeros(40 * 30, bool)
    margin = np.zeros(40 * 30, bool)
    for p in range(40 * 30):
        i, j = p % 40, p // 40
        x = np.array([(i + 0.5 - 20.0) / 30.0, (j + 0.5 - 15.0) / 30.0, 1.0])
        D, tau = oracle_lib.D_ray(mu, Si, x)
        reached[p] = tau > 0 and D <= k_reach
        margin[p] = abs(D - k_reach) <= 1e-9 * k_reach
    assert 0 < reached.sum() < reached.size
    assert np.array_equal(flagged[~margin], reached[~margin])


def test_no_border_flag_away_from_the_threshold(oracle_lib):
    logit, _ = _logit_at_threshold()
    cam = scenes.make_camera(40, 30, 30.0, 30.0)
    for shift in (-1e-3, 1e-3):
        sc = _thin_plane(np.float32(logit + shift))
        g = oracle_lib.prepare(sc, cam)[0]
        assert g[oracle_lib.OG["BORDER"]] == 0
        out = oracle_lib.render(sc, cam)
        assert not np.any(out["flags"] & FLAG_BORDER)


def test_uniform_scene_has_no_border_pixels(oracle_lib):
    """On the 64x64 workload no skip decision comes within FP64 rounding of its threshold."""
    scene, cams = scenes.workload_small()
    out = oracle_lib.render(scene, cams[0])
    assert not np.any(out["flags"] & FLAG_BORDER)

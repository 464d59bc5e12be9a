"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle).

Exclusion rule.  A pixel whose error exceeds the tolerance may be excluded only when the
oracle flags it as eligible, and at most 0.01 % of a view's pixels may be excluded:
  - FLAG_CUTOFF: some primitive's opacity at the pixel lies within 1e-6 of the cut-off
    p_min (the float32 renderer and the FP64 oracle may take the cut-off apart);
  - FLAG_BORDER: the pixel is reached (opacity >= p_min / 2) by a primitive whose skip
    decision (kappa <= 0, or the camera-inside test of Eq. c) lies within FP64 rounding of
    its threshold; both sides take those decisions in FP64, so only the order of FP64
    roundings can part them.
The transmittance-stop band (FLAG_STOP) is reported but does not make a pixel eligible.
"""
import json
import os

import numpy as np

TOL = 2e-4          # max-abs per channel, FP32 path vs FP64 oracle
EXCL_FRAC = 1e-4    # at most 0.01% of pixels may be excluded, and only eligible ones
FLAG_CUTOFF, FLAG_STOP, FLAG_BORDER = 1, 2, 4
ELIGIBLE = FLAG_CUTOFF | FLAG_BORDER


def gpu_render(scene, cams, capacity=None, **cfg):
    import torch
    from paper_2503_18682_gb300 import raygs
    r = raygs.Renderer(cams, scene["means"].shape[0], capacity=capacity, **cfg)
    st = raygs.scene_to_device(scene)
    rgb, T, nc = r.forward(st)
    torch.cuda.synchronize()
    return r, st, rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64), nc.cpu().numpy()


def view_slice(r, v):
    o = r.pixel_offsets[v]
    c = r.cams[v]
    return slice(o, o + c["width"] * c["height"])


def compare(gpu_rgb, gpu_T, orc, tol=TOL, excl_frac=EXCL_FRAC):
    """Element-wise comparison; returns stats and asserts nothing.  n_excluded counts the
    pixels off by more than tol that the rule above allows to exclude; n_unexplained the
    others.  n_bad_cutoff / n_bad_border / n_bad_stop break the off pixels down by flag."""
    err = np.abs(gpu_rgb - orc["rgb"]).max(axis=1)
    errT = np.abs(gpu_T - orc["T"])
    bad = (err > tol) | (errT > tol)
    flags = np.asarray(orc["flags"]).astype(np.int64)
    eligible = (flags & ELIGIBLE) != 0
    excluded = bad & eligible
    keep = ~excluded
    st = dict(max_err=float(err[keep].max()) if keep.any() else 0.0,
              max_err_T=float(errT[keep].max()) if keep.any() else 0.0,
              n_bad=int(bad.sum()), n_excluded=int(excluded.sum()),
              n_unexplained=int((bad & ~eligible).sum()), n_flagged=int(eligible.sum()),
              n_bad_cutoff=int((bad & ((flags & FLAG_CUTOFF) != 0)).sum()),
              n_bad_border=int((bad & ((flags & FLAG_BORDER) != 0)).sum()),
              n_bad_stop=int((bad & ((flags & FLAG_STOP) != 0)).sum()),
              allowed=int(excl_frac * len(err)), n=len(err),
              worst=int(np.argmax(np.where(keep, err, 0))))
    log = os.environ.get("RAYGS_PARITY_LOG")
    if log:
        test = os.environ.get("PYTEST_CURRENT_TEST", "")
        with open(log, "a") as f:
            f.write(json.dumps(dict(test=test, **{k: v for k, v in st.items() if k != "worst"})) + "\n")
    return st


def assert_parity(stats, tol=TOL):
    assert stats["n_unexplained"] == 0, stats
    assert stats["n_excluded"] <= stats["allowed"], stats
    assert stats["max_err"] <= tol and stats["max_err_T"] <= tol, stats


def allowed_in_sample(n_sampled, frac=EXCL_FRAC, p_fail=1e-3):
    """Excluded pixels a uniform sample of n_sampled pixels may hold when the image's rate is
    at most `frac`: the smallest k with P(Poisson(frac n_sampled) > k) < p_fail.  A sample of
    1,024 pixels allows 2 and catches only rates well above 0.01% (a true rate of 0.5% fails
    it with probability 0.88)."""
    import math
    lam = frac * n_sampled
    k, term, cdf = 0, math.exp(-lam), math.exp(-lam)
    while 1.0 - cdf >= p_fail:
        k += 1
        term *= lam / k
        cdf += term
    return k


def assert_parity_sampled(stats_list, tol=TOL):
    """Sampled pixels of several views, pooled: no unflagged pixel off by more than tol,
    and no more flagged exclusions than allowed_in_sample grants the pooled sample."""
    n = sum(s["n"] for s in stats_list)
    excl = sum(s["n_excluded"] for s in stats_list)
    for s in stats_list:
        assert s["n_unexplained"] == 0, s
        assert s["max_err"] <= tol and s["max_err_T"] <= tol, s
    assert excl <= allowed_in_sample(n), (excl, n, stats_list)


def sample_pixels(cam, n, seed):
    rng = np.random.default_rng(seed)
    W, H = cam["width"], cam["height"]
    idx = rng.choice(W * H, size=min(n, W * H), replace=False)
    idx.sort()
    return np.stack([idx % W, idx // W], axis=1).astype(np.int32), idx

"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
import numpy as np

TOL = 2e-4          # max-abs per channel, FP32 path vs FP64 oracle
EXCL_FRAC = 1e-4    # at most 0.01% of pixels may be excluded, and only flagged ones


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
    """Element-wise comparison; returns stats and asserts nothing."""
    err = np.abs(gpu_rgb - orc["rgb"]).max(axis=1)
    errT = np.abs(gpu_T - orc["T"])
    bad = (err > tol) | (errT > tol)
    flagged = orc["flags"] != 0
    excluded = bad & flagged
    keep = ~excluded
    return dict(max_err=float(err[keep].max()) if keep.any() else 0.0,
                max_err_T=float(errT[keep].max()) if keep.any() else 0.0,
                n_bad=int(bad.sum()), n_excluded=int(excluded.sum()),
                n_unexplained=int((bad & ~flagged).sum()), n_flagged=int(flagged.sum()),
                allowed=int(excl_frac * len(err)), n=len(err),
                worst=int(np.argmax(np.where(keep, err, 0))))


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

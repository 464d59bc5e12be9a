"""Host-side helpers that need no GPU: the pooled-sample exclusion rule of the sampled parity
tests, the camera anti-aliasing modes, the supersampled cameras and the benchmark's
algorithmic byte model of the binning stage."""
import math
import os
import sys

import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import allowed_in_sample

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def poisson_tail(lam, k):
    """P(X > k) for X ~ Poisson(lam), summed directly."""
    return 1.0 - sum(math.exp(-lam) * lam ** i / math.factorial(i) for i in range(k + 1))


def test_allowed_in_sample_is_the_poisson_quantile():
    for n in (1, 100, 1024, 6144, 100_000):
        k = allowed_in_sample(n)
        lam = 1e-4 * n
        assert poisson_tail(lam, k) < 1e-3
        assert k == 0 or poisson_tail(lam, k - 1) >= 1e-3
    assert allowed_in_sample(1024) == 2
    ks = [allowed_in_sample(n) for n in (10, 1000, 10_000, 100_000)]
    assert ks == sorted(ks)


def test_camera_mip_modes():
    import oracle
    assert scenes.make_camera(8, 8, 8.0, 8.0)["mip"] == 0
    assert scenes.make_camera(8, 8, 8.0, 8.0, mip=True)["mip"] == 1
    assert scenes.make_camera(8, 8, 8.0, 8.0, mip="exact")["mip"] == 2
    for m, code in ((False, 0), (True, 1), (1, 1), ("exact", 2), (2, 2)):
        assert oracle.cam_array(dict(scenes.make_camera(8, 8, 8.0, 8.0), mip=m))[19] == code
    with pytest.raises(ValueError):
        oracle.cam_array(dict(scenes.make_camera(8, 8, 8.0, 8.0), mip=3))


def test_supersampled_cameras_put_subpixel_rays_at_subpixel_centres():
    from paper_2503_18682_gb300 import raygs
    cam = scenes.make_camera(37, 21, 30.5, 28.0, 17.25, 9.5)
    for f in (2, 3, 4):
        hi = raygs.supersampled_cameras([cam], f)[0]
        assert (hi["width"], hi["height"]) == (37 * f, 21 * f)
        for i, j in ((0, 0), (36, 20), (11, 7)):
            for a in range(f):
                for b in range(f):
                    # ray of the high-resolution pixel (f i + a, f j + b) ...
                    xh = (f * i + a + 0.5 - float(hi["cx"])) / float(hi["fx"])
                    yh = (f * j + b + 0.5 - float(hi["cy"])) / float(hi["fy"])
                    # ... is the ray through the sub-pixel centre of pixel (i, j)
                    xs = (i + (a + 0.5) / f - float(cam["cx"])) / float(cam["fx"])
                    ys = (j + (b + 0.5) / f - float(cam["cy"])) / float(cam["fy"])
                    assert xh == pytest.approx(xs, rel=1e-6, abs=1e-9)
                    assert yh == pytest.approx(ys, rel=1e-6, abs=1e-9)


def test_binning_byte_model():
    sys.path.insert(0, ROOT)
    import bench
    ctr = dict(n_visible=10, n_rows=30, n_rows_kept=25, n_instances=100)
    b = bench.binning_bytes(ctr, 40)
    # depth sort, support rows, tile-row sort, chunk counts and expansion, term by term
    depth = 5 * 40 + 8 * 10 + 3 * 16 * 10 + 4 * 40 + 3 * 4 * 10
    expect = depth + (32 * 10 + 12 * 30) + (12 * 30 + 12 * 25 + 24 * 25 + 4 * 30 + 4 * 25) + 4 * 25 + (8 * 25 + 4 * 100)
    assert b == expect
    # linear in every count
    ctr2 = {k: 2 * v for k, v in ctr.items()}
    assert bench.binning_bytes(ctr2, 80) == 2 * b
    assert np.isfinite(b)

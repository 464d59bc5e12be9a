"""Seeded sweep over small random configurations, full images against the oracle with the
forward tolerance: 1-4 views of 5-140 px per side (many narrower than a tile or ragged),
off-centre principal points, unequal focal lengths, random poses around the scene, every
tile shape and rasteriser batch, both divergences and all three anti-aliasing modes (where
the combination is valid), uniform and blob scenes with near-flat primitives."""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import assert_parity, compare, gpu_render, view_slice

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (16, 8), (32, 16), (8, 8)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18682_gb300 import build
    build.build()


def random_case(seed):
    rng = np.random.default_rng(1000 + seed)
    if rng.random() < 0.5:
        scene = scenes.uniform_scene(int(rng.integers(200, 2500)), seed=seed)
        centre = np.array([0.0, 0.0, 3.0])
    else:
        scene = scenes.blob_scene(int(rng.integers(500, 4000)), seed=seed, sh_degree=int(rng.integers(0, 4)),
                                  degenerate_frac=float(rng.choice([0.0, 0.1])))
        centre = np.array([0.0, 0.0, 6.0])
    divergence = int(rng.random() < 0.25)
    mip = 0 if divergence else int(rng.choice([0, 1, 2]))
    n_views = int(rng.integers(1, 5))
    cams = []
    for v in range(n_views):
        w, h = int(rng.integers(5, 141)), int(rng.integers(5, 141))
        f = float(rng.uniform(0.4, 1.5)) * max(w, h)
        fx, fy = f, f * float(rng.uniform(0.8, 1.25))
        cx, cy = w * float(rng.uniform(0.3, 0.7)), h * float(rng.uniform(0.3, 0.7))
        if v == 0 and rng.random() < 0.5:
            R, t = None, None
        else:
            d = rng.standard_normal(3)
            eye = centre + float(rng.uniform(2.0, 5.0)) * d / np.linalg.norm(d)
            R, t = scenes.look_at(eye, centre + rng.uniform(-0.5, 0.5, 3))
        cams.append(scenes.make_camera(w, h, fx, fy, cx, cy, R=R, t=t, mip=(mip if mip < 2 else "exact")))
    if mip == 2:
        cams = [dict(c, mip="exact") for c in cams]   # exact views cannot be mixed with others
    tw, th = SHAPES[int(rng.integers(0, 4))]
    cfg = dict(tile_w=tw, tile_h=th, batch_records=int(rng.integers(1, 3)), divergence=divergence,
               mip_sigma2=float(rng.choice([0.1, 1.0])))
    return scene, cams, cfg


@pytest.mark.parametrize("seed", range(24))
def test_random_configuration(oracle_lib, seed):
    scene, cams, cfg = random_case(seed)
    r, _, rgb, T, nc = gpu_render(scene, cams, **cfg)
    ocfg = dict(divergence=cfg["divergence"], mip_sigma2=cfg["mip_sigma2"])
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        assert_parity(compare(rgb[sl], T[sl], oracle_lib.render(scene, cam, cfg=ocfg)))

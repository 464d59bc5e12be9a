"""Pins of the dense FP64 reference (oracle/ref_torch.py) used for reference gradients:
its image equals the C oracle's, and its autograd gradients of an L1 image loss equal
central finite differences of the C oracle (where the composited set does not change)."""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes

torch = pytest.importorskip("torch")


def small_scene(seed=41, n=60, deg=2):
    sc = scenes.uniform_scene(n, seed=seed)
    rng = np.random.default_rng(seed)
    k = (deg + 1) ** 2
    sh = np.zeros((n, k, 3), np.float32)
    sh[:, 0] = sc["sh"][:, 0]
    sh[:, 1:] = 0.1 * rng.standard_normal((n, k - 1, 3))
    sc["sh"] = sh
    sc["sh_degree"] = deg
    sc["log_scales"] = (sc["log_scales"] + np.float32(0.7)).astype(np.float32)  # larger, overlapping
    sc["opacity_logits"] = (sc["opacity_logits"] + np.float32(1.0)).astype(np.float32)
    return sc


def test_dense_reference_matches_oracle_image(oracle_lib):
    from oracle import ref_torch
    sc = small_scene()
    R, t = scenes.look_at([0.2, -0.1, -0.3], [0, 0, 3.0])
    cam = scenes.make_camera(24, 20, 22.0, 21.0, 11.7, 10.2, R=R, t=t)
    ref = oracle_lib.render(sc, cam)
    p = ref_torch.params_from_scene(sc, requires_grad=False)
    rgb, T = ref_torch.render_dense(p, sc, cam)
    np.testing.assert_allclose(rgb.numpy(), ref["rgb"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(T.numpy(), ref["T"], rtol=0, atol=1e-11)
    assert ref["ncontrib"].max() >= 5


def test_dense_reference_gradients_match_finite_differences(oracle_lib):
    from oracle import fd, ref_torch
    sc = small_scene()
    cam = scenes.make_camera(24, 20, 22.0, 21.0, 11.7, 10.2)
    rng = np.random.default_rng(3)
    target = rng.uniform(0, 1, (24 * 20, 3))
    p = ref_torch.params_from_scene(sc)
    rgb, _ = ref_torch.render_dense(p, sc, cam)
    loss = (rgb - torch.as_tensor(target)).abs().sum()
    loss.backward()
    info = oracle_lib.prepare(sc, cam)
    gids = [g for g in np.argsort(-info[:, 7]) if info[g, 0] == 0][:5]
    checked = 0
    for g in gids:
        for key, idxs, h in (("means", [(g, 0), (g, 1), (g, 2)], 1e-4),
                             ("log_scales", [(g, 0), (g, 1), (g, 2)], 1e-4),
                             ("quats", [(g, 0), (g, 1), (g, 2), (g, 3)], 1e-4),
                             ("opacity_logits", [(g,)], 1e-4),
                             ("sh", [(g, 0, 0), (g, 0, 2), (g, 3, 1), (g, 7, 0)], 1e-3)):
            for idx in idxs:
                num = fd.central_difference(sc, cam, target, key, idx, h)
                if num is None:
                    continue
                ana = float(p[key].grad[idx])
                assert ana == pytest.approx(num, rel=2e-4, abs=2e-5 * (1 + abs(num))), (key, idx, ana, num)
                checked += 1
    assert checked >= 60

"""Backward parity: gradients of an L1 image loss from the CUDA backward (through the C ABI)
against (a) autograd through the dense FP64 reference (oracle/ref_torch.py, itself pinned to
finite differences of the C oracle) on small scenes, and (b) central finite differences of
the FP64 oracle on a 2k-primitive 128x128 copy of the 1.5M-primitive workload, for 32
sampled primitives."""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes

pytestmark = pytest.mark.gpu

KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18682_gb300 import build
    build.build()


def gpu_grads(scene, cams, target, **cfg):
    import torch
    from paper_2503_18682_gb300 import raygs
    r = raygs.Renderer(cams, scene["means"].shape[0], enable_backward=1, **cfg)
    st = raygs.scene_to_device(scene)
    params = {k: st[k].clone().requires_grad_(True) for k in KEYS}
    params["sh_degree"] = scene["sh_degree"]
    rgb, T, nc = raygs.render(r, params)
    loss = (rgb.double() - torch.as_tensor(target, device="cuda")).abs().sum()
    loss.backward()
    torch.cuda.synchronize()
    return {k: params[k].grad.double().cpu().numpy() for k in KEYS}, rgb.detach().cpu().numpy()


def ref_grads(scene, cams, target):
    import torch
    from oracle import ref_torch
    p = ref_torch.params_from_scene(scene)
    loss = 0.0
    off = 0
    for cam in cams:
        rgb, _ = ref_torch.render_dense(p, scene, cam)
        npx = cam["width"] * cam["height"]
        loss = loss + (rgb - torch.as_tensor(target[off:off + npx])).abs().sum()
        off += npx
    loss.backward()
    return {k: p[k].grad.numpy() for k in KEYS}


def assert_close_grads(g, ref, rtol=3e-3, atol_frac=2e-3):
    for k in KEYS:
        a, b = g[k], ref[k]
        scale = np.abs(b).max() + 1e-12
        err = np.abs(a - b)
        bad = err > atol_frac * scale + rtol * np.abs(b)
        assert not bad.any(), (k, float(err.max()), float(scale), np.argwhere(bad)[:5].tolist())


def small_scene(seed, n, deg):
    sc = scenes.uniform_scene(n, seed=seed)
    rng = np.random.default_rng(seed)
    kk = (deg + 1) ** 2
    sh = np.zeros((n, kk, 3), np.float32)
    sh[:, 0] = sc["sh"][:, 0]
    if kk > 1:
        sh[:, 1:] = 0.1 * rng.standard_normal((n, kk - 1, 3))
    sc["sh"], sc["sh_degree"] = sh, deg
    sc["log_scales"] = (sc["log_scales"] + np.float32(0.5)).astype(np.float32)
    return sc


@pytest.mark.parametrize("deg", [0, 3])
def test_backward_matches_dense_autograd(deg):
    sc = small_scene(51 + deg, 300, deg)
    R1, t1 = scenes.look_at([0.3, -0.2, -0.5], [0, 0, 3.0])
    cams = [scenes.make_camera(48, 40, 45.0, 44.0, 23.1, 19.7),
            scenes.make_camera(37, 29, 30.0, 30.0, R=R1, t=t1)]
    P = sum(c["width"] * c["height"] for c in cams)
    target = np.random.default_rng(7).uniform(0, 1, (P, 3))
    g, _ = gpu_grads(sc, cams, target)
    ref = ref_grads(sc, cams, target)
    assert_close_grads(g, ref)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_backward_tile_shapes_agree(tile):
    sc = small_scene(61, 400, 1)
    cams = [scenes.make_camera(64, 48, 55.0, 55.0)]
    target = np.random.default_rng(8).uniform(0, 1, (64 * 48, 3))
    g, _ = gpu_grads(sc, cams, target, tile_w=tile[0], tile_h=tile[1])
    ref = ref_grads(sc, cams, target)
    assert_close_grads(g, ref)


def test_backward_matches_oracle_finite_differences(oracle_lib):
    """2k primitives of the blob generator (seed 2), 128x128 (fx = fy = 100), L1 loss
    against a uniform random target; 32 primitives sampled among those that reach pixels;
    every parameter group is compared where the central difference exists."""
    from oracle import fd
    scene = scenes.blob_scene(2000, seed=2)
    cam = scenes.make_camera(128, 128, 100.0, 100.0)
    target = np.random.default_rng(2).uniform(0, 1, (128 * 128, 3))
    g, _ = gpu_grads(scene, [cam], target)
    info = oracle_lib.prepare(scene, cam)
    cand = np.nonzero((info[:, 0] == 0) & (np.abs(g["opacity_logits"]) > 1e-3))[0]
    rng = np.random.default_rng(12)
    pick = rng.choice(cand, size=min(32, len(cand)), replace=False)
    checked = skipped = 0
    scale = {k: float(np.abs(g[k]).max()) for k in KEYS}
    for gi in pick:
        for key, idxs, h in (("means", [(gi, 0), (gi, 1), (gi, 2)], 2e-4),
                             ("log_scales", [(gi, 0), (gi, 1), (gi, 2)], 2e-4),
                             ("quats", [(gi, 0), (gi, 1), (gi, 2), (gi, 3)], 2e-4),
                             ("opacity_logits", [(gi,)], 2e-4),
                             ("sh", [(gi, 0, 0), (gi, 1, 1), (gi, 8, 2)], 2e-3)):
            for idx in idxs:
                num = fd.central_difference(scene, cam, target, key, idx, h)
                if num is None:
                    skipped += 1
                    continue
                ana = float(g[key][idx])
                tol = 5e-3 * abs(num) + 1e-3 * scale[key]
                assert abs(ana - num) <= tol, (key, idx, ana, num, scale[key])
                checked += 1
    assert checked >= 300, (checked, skipped)


def test_backward_refuses_mip_and_disabled():
    import torch
    from paper_2503_18682_gb300 import raygs
    sc = small_scene(71, 50, 0)
    st = raygs.scene_to_device(sc)
    r = raygs.Renderer([scenes.make_camera(16, 16, 16.0, 16.0, mip=True)], 50, enable_backward=1)
    rgb, T, nc = r.forward(st)
    with pytest.raises(raygs.RayGSError):
        r.backward(st, T, nc, torch.ones_like(rgb))
    r2 = raygs.Renderer([scenes.make_camera(16, 16, 16.0, 16.0)], 50)
    rgb, T, nc = r2.forward(st)
    with pytest.raises(raygs.RayGSError):
        r2.backward(st, T, nc, torch.ones_like(rgb))

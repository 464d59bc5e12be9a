"""Pose updates (raygs_plan_set_poses): new camera poses for the same views, as a VR loop
sends every frame.  The direct pipeline and a captured graph replayed after the update
render the new poses (against the oracle, forward tolerance); changing a view's size or
intrinsics through the update is refused."""
import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import assert_parity, compare, view_slice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18682_gb300 import build, raygs
    build.build()
    return raygs


def poses(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        d = rng.standard_normal(3)
        eye = np.array([0.0, 0.0, 3.0]) + 2.5 * d / np.linalg.norm(d)
        out.append(scenes.look_at(eye, [0.0, 0.0, 3.0]))
    return out


def cams_at(ps):
    sizes = [(80, 64, 70.0), (57, 43, 50.0)]
    return [scenes.make_camera(w, h, f, f, R=R, t=t) for (w, h, f), (R, t) in zip(sizes, ps)]


def check(oracle_lib, scene, r, cams, rgb, T):
    rgb = rgb.cpu().numpy().astype(np.float64)
    T = T.cpu().numpy().astype(np.float64)
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        assert_parity(compare(rgb[sl], T[sl], oracle_lib.render(scene, cam)))


def test_pose_update_direct_and_graph(oracle_lib, rg):
    import torch
    scene = scenes.uniform_scene(1500, seed=41)
    st = rg.scene_to_device(scene)
    sc = rg.make_scene(st)
    cams_a, cams_b = cams_at(poses(1, 2)), cams_at(poses(2, 2))
    r = rg.Renderer(cams_a, 1500, capacity=1 << 22)
    rgb, T, nc = r.forward(st)
    torch.cuda.synchronize()
    check(oracle_lib, scene, r, cams_a, rgb, T)
    # direct pipeline after the update
    rg.raygs_plan_set_poses(r.plan, cams_b)
    r.cams = cams_b
    rgb, T, nc = r.forward(st)
    torch.cuda.synchronize()
    check(oracle_lib, scene, r, cams_b, rgb, T)
    # a graph captured at poses a, replayed after updates to b and back to a
    rg.raygs_plan_set_poses(r.plan, cams_a)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    out = r.alloc_outputs()
    with torch.cuda.stream(s):
        rg.raygs_graph_capture(r.plan, sc, *out, s)
        rg.raygs_plan_set_poses(r.plan, cams_b, s)
        rg.raygs_graph_launch(r.plan, s)
    s.synchronize()
    assert rg.raygs_read_counters(r.plan)["overflow"] == 0
    check(oracle_lib, scene, r, cams_b, out[0], out[1])
    with torch.cuda.stream(s):
        rg.raygs_plan_set_poses(r.plan, cams_a, s)
        rg.raygs_graph_launch(r.plan, s)
    s.synchronize()
    check(oracle_lib, scene, r, cams_a, out[0], out[1])


def test_pose_update_refuses_other_intrinsics(rg):
    cams = cams_at(poses(3, 2))
    r = rg.Renderer(cams, 100)
    for change in (dict(width=81), dict(fx=71.0), dict(cy=10.0), dict(mip=True), dict(near=0.5)):
        bad = [dict(cams[0], **change), cams[1]]
        with pytest.raises(RuntimeError):
            rg.raygs_plan_set_poses(r.plan, bad)

"""Binning parity: depth keys against the oracle (bit-exact), the stable depth sort, the
instance emission order, the tile sort and the tile ranges against a CPU re-binning of the
GPU's own keys and rectangles (bit-exact); tile rectangles against the oracle's quad."""
import math

import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import gpu_render

pytestmark = pytest.mark.gpu

CULLED = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


class _DevView:
    """Zero-copy view of a raw device buffer (CUDA array interface)."""

    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = dict(shape=(count,), typestr=typestr, data=(ptr, False),
                                             version=3, strides=None)


def fetch(ptr, count, dtype):
    import torch
    assert ptr
    ts = {np.uint32: "<i4", np.float32: "<f4"}[dtype]
    t = torch.as_tensor(_DevView(ptr, count, ts), device="cuda")
    torch.cuda.synchronize()
    return t.cpu().numpy().view(dtype).copy()


def rebin(r, scene_n, n_views, keys, rects):
    VN = scene_n * n_views
    vis = np.nonzero(keys != CULLED)[0]
    order = vis[np.argsort(keys[vis], kind="stable")]
    inst_tile, inst_pos = [], []
    for p, pair in enumerate(order):
        v = pair // scene_n
        cam = r.cams[v]
        tw, th = r.cfg.tile_w, r.cfg.tile_h
        tiles_x = -(-cam["width"] // tw)
        base = sum((-(-c["width"] // tw)) * (-(-c["height"] // th)) for c in r.cams[:v])
        x0, y0 = rects[pair, 0] & 0xFFFF, rects[pair, 0] >> 16
        x1, y1 = rects[pair, 1] & 0xFFFF, rects[pair, 1] >> 16
        for ty in range(y0, y1 + 1):
            for tx in range(x0, x1 + 1):
                inst_tile.append(base + ty * tiles_x + tx)
                inst_pos.append(p)
    inst_tile = np.array(inst_tile, dtype=np.int64)
    inst_pos = np.array(inst_pos, dtype=np.int64)
    srt = np.argsort(inst_tile, kind="stable")
    return order, inst_tile[srt], inst_pos[srt]


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_sort_and_tile_lists_bit_exact(oracle_lib, tile):
    scene = scenes.uniform_scene(3000, seed=21)
    scene["means"][100:110] = scene["means"][50]          # exact depth ties
    R1, t1 = scenes.look_at([0.5, 0.2, -0.4], [0.0, 0.0, 3.0])
    cams = [scenes.make_camera(130, 77, 100.0, 100.0), scenes.make_camera(64, 96, 50.0, 50.0, R=R1, t=t1)]
    r, _, rgb, T, nc = gpu_render(scene, cams, tile_w=tile[0], tile_h=tile[1])
    n, V = 3000, 2
    keys = fetch(r.debug_buffer(0), n * V, np.uint32)
    rects = fetch(r.debug_buffer(1), 2 * n * V, np.uint32).reshape(-1, 2)
    ctr = r.last_counters
    order, tiles, pos = rebin(r, n, V, keys, rects)
    assert ctr["n_visible"] == len(order)
    assert ctr["n_instances"] == len(tiles)
    g_order = fetch(r.debug_buffer(3), len(order), np.uint32)
    np.testing.assert_array_equal(g_order, order)
    g_tiles = fetch(r.debug_buffer(4), len(tiles), np.uint32)
    g_pos = fetch(r.debug_buffer(5), len(tiles), np.uint32)
    np.testing.assert_array_equal(g_tiles, tiles)
    np.testing.assert_array_equal(g_pos, pos)
    ranges = fetch(r.debug_buffer(6), 2 * r.num_tiles, np.uint32).reshape(-1, 2)
    for t in range(r.num_tiles):
        idx = np.nonzero(tiles == t)[0]
        if len(idx):
            assert tuple(ranges[t]) == (idx[0], idx[-1] + 1)
        else:
            assert ranges[t, 0] == ranges[t, 1]
    # depth keys equal the oracle's (same float32 chain), for every primitive the GPU kept
    for v, cam in enumerate(cams):
        info = oracle_lib.prepare(scene, cam)
        kv = keys[v * n:(v + 1) * n]
        kept = kv != CULLED
        np.testing.assert_array_equal(kv[kept], info[kept, 1].astype(np.uint32))
        assert np.all(info[kept, 0] == 0)


def test_rects_match_oracle_quad(oracle_lib):
    """The GPU tile rectangle equals the tiles of the oracle's projected quad bounding box
    (Eq. V_ray), except where a box edge sits within 0.01 px of a tile boundary."""
    scene = scenes.blob_scene(4000, seed=22)
    cam = scenes.make_camera(256, 144, 200.0, 200.0, mip=True)
    r, _, rgb, T, nc = gpu_render(scene, [cam])
    n = 4000
    keys = fetch(r.debug_buffer(0), n, np.uint32)
    rects = fetch(r.debug_buffer(1), 2 * n, np.uint32).reshape(-1, 2)
    info = oracle_lib.prepare(scene, cam)
    W, H, fx, cx, cy = 256, 144, 200.0, 128.0, 72.0
    checked = 0
    for g in range(n):
        if info[g, 0] != 0:
            assert keys[g] == CULLED
            continue
        qd = oracle_lib.quad(info[g, 2:5], info[g, 14:23].reshape(3, 3), info[g, 11:14], info[g, 6])
        V = qd["V"]
        if np.any(V[2] <= 1e-9):
            if keys[g] != CULLED:
                assert tuple(rects[g]) == (0, (W - 1) // 16 | (((H - 1) // 16) << 16))
            continue
        u = fx * V[0] / V[2] + cx
        v = fx * V[1] / V[2] + cy
        i0, i1 = math.ceil(u.min() - 0.5), math.floor(u.max() - 0.5)
        j0, j1 = math.ceil(v.min() - 0.5), math.floor(v.max() - 0.5)
        i0, j0, i1, j1 = max(i0, 0), max(j0, 0), min(i1, W - 1), min(j1, H - 1)
        near_edge = min(abs((u.min() - 0.5) - round(u.min() - 0.5)), abs((u.max() - 0.5) - round(u.max() - 0.5)),
                        abs((v.min() - 0.5) - round(v.min() - 0.5)), abs((v.max() - 0.5) - round(v.max() - 0.5))) < 1e-2
        if i0 > i1 or j0 > j1:
            assert keys[g] == CULLED or near_edge
            continue
        if keys[g] == CULLED:
            # culled by the conservative frustum test although the (larger) quad reaches
            # the image: no pixel centre of the box may lie in the support.
            Si = info[g, 14:23].reshape(3, 3) @ np.diag(info[g, 11:14] ** -2.0) @ info[g, 14:23].reshape(3, 3).T
            for jj in range(j0, j1 + 1):
                for ii in range(i0, i1 + 1):
                    D, tau = oracle_lib.D_ray(info[g, 2:5], Si, [(ii + 0.5 - cx) / fx, (jj + 0.5 - cy) / fx, 1.0])
                    assert not (tau > 0 and D <= info[g, 6]), (g, ii, jj)
            continue
        want = (i0 // 16, j0 // 16, i1 // 16, j1 // 16)
        got = (rects[g, 0] & 0xFFFF, rects[g, 0] >> 16, rects[g, 1] & 0xFFFF, rects[g, 1] >> 16)
        assert got == want or near_edge, (g, got, want)
        checked += 1
    assert checked > 500

"""Binning parity: depth keys against the oracle (bit-exact), the stable depth sort, the
instance emission order, the tile sort and the tile ranges against a CPU re-binning of the
GPU's own keys and rectangles (bit-exact); tile rectangles against the oracle's quad."""
import math

import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes
from tests.gpu_util import assert_parity, compare, gpu_render, sample_pixels, view_slice

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


def instance_lists(r, ni):
    """(tile id, sorted pair position) of every instance.  The tile ranges must partition
    the instance array in tile order."""
    ranges = fetch(r.debug_buffer(6), 2 * r.num_tiles, np.uint32).reshape(-1, 2).astype(np.int64)
    assert ranges[0, 0] == 0 and ranges[-1, 1] == ni
    np.testing.assert_array_equal(ranges[1:, 0], ranges[:-1, 1])
    assert np.all(ranges[:, 1] >= ranges[:, 0])
    g_tiles = np.repeat(np.arange(r.num_tiles, dtype=np.int64), ranges[:, 1] - ranges[:, 0])
    g_pos = fetch(r.debug_buffer(5), ni, np.uint32).astype(np.int64)
    return g_tiles, g_pos


def tile_base_of(r, v):
    tw, th = r.cfg.tile_w, r.cfg.tile_h
    return sum((-(-c["width"] // tw)) * (-(-c["height"] // th)) for c in r.cams[:v])


def rect_of(rects, pair):
    x0, y0 = rects[pair, 0] & 0xFFFF, rects[pair, 0] >> 16
    x1, y1 = rects[pair, 1] & 0xFFFF, rects[pair, 1] >> 16
    return int(x0), int(y0), int(x1), int(y1)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_sort_and_tile_lists(oracle_lib, tile):
    """Depth keys equal the oracle's bit for bit; the visible pairs come out in (key, index)
    order (CPU stable sort of the GPU's own keys, bit-exact); every instance lies in its
    pair's tile rectangle, each tile's list is in increasing depth order and the ranges
    delimit the tile-sorted list; no tile dropped by the ellipse test holds a pixel centre
    of the pair's support (FP64 oracle, brute force)."""
    scene = scenes.uniform_scene(3000, seed=21)
    scene["means"][100:110] = scene["means"][50]          # exact depth ties
    R1, t1 = scenes.look_at([0.5, 0.2, -0.4], [0.0, 0.0, 3.0])
    cams = [scenes.make_camera(130, 77, 100.0, 100.0), scenes.make_camera(64, 96, 50.0, 50.0, R=R1, t=t1)]
    r, _, rgb, T, nc = gpu_render(scene, cams, tile_w=tile[0], tile_h=tile[1])
    n, V = 3000, 2
    tw, th = tile
    keys = fetch(r.debug_buffer(0), n * V, np.uint32)
    rects = fetch(r.debug_buffer(1), 2 * n * V, np.uint32).reshape(-1, 2)
    ctr = r.last_counters
    vis = np.nonzero(keys != CULLED)[0]
    order = vis[np.argsort(keys[vis], kind="stable")]
    assert ctr["n_visible"] == len(order)
    g_order = fetch(r.debug_buffer(3), len(order), np.uint32)
    np.testing.assert_array_equal(g_order, order)
    ni = ctr["n_instances"]
    g_tiles, g_pos = instance_lists(r, ni)
    same = np.diff(g_tiles) == 0
    assert np.all(np.diff(g_pos)[same] > 0)             # depth order inside a tile
    # instances inside the rectangles; dropped rectangle tiles miss the support
    dropped, _, _ = assert_dropped_tiles_miss_support(oracle_lib, scene, cams, r, n, tile, {int(p) for p in order})
    assert dropped > 0
    infos = [oracle_lib.prepare(scene, cam) for cam in cams]
    # depth keys equal the oracle's (same float32 chain), for every primitive the GPU kept
    for v, cam in enumerate(cams):
        info = infos[v]
        kv = keys[v * n:(v + 1) * n]
        k = kv != CULLED
        np.testing.assert_array_equal(kv[k], info[k, 1].astype(np.uint32))
        assert np.all(info[k, 0] == 0)


def assert_dropped_tiles_miss_support(oracle_lib, scene, cams, r, n, tile, pairs_to_check):
    """Every tile of a pair's rectangle that the binning dropped holds no pixel centre of the
    pair's support (FP64 oracle, brute force).  Returns (dropped tiles checked, rectangle
    tiles, kept instances) over the checked pairs."""
    tw, th = tile
    rects = fetch(r.debug_buffer(1), 2 * n * len(cams), np.uint32).reshape(-1, 2)
    ctr = r.last_counters
    order = fetch(r.debug_buffer(3), ctr["n_visible"], np.uint32)
    g_tiles, g_pos = instance_lists(r, ctr["n_instances"])
    kept = {}
    for t, p in zip(g_tiles, g_pos):
        kept.setdefault(int(p), set()).add(int(t))
    infos = [oracle_lib.prepare(scene, cam) for cam in cams]
    dropped = n_rect = n_kept = 0
    for p, pair in enumerate(order):
        if int(pair) not in pairs_to_check:
            continue
        v, g = divmod(int(pair), n)
        x0, y0, x1, y1 = rect_of(rects, pair)
        base = tile_base_of(r, v)
        tx_n = -(-cams[v]["width"] // tw)
        rect_tiles = {base + ty * tx_n + tx for ty in range(y0, y1 + 1) for tx in range(x0, x1 + 1)}
        mine = kept.get(p, set())
        assert mine <= rect_tiles, (p, pair)
        n_rect += len(rect_tiles)
        n_kept += len(mine)
        info = infos[v][g]
        Si = info[14:23].reshape(3, 3) @ np.diag(info[11:14] ** -2.0) @ info[14:23].reshape(3, 3).T
        cam = cams[v]
        for t in rect_tiles - mine:
            ty, tx = divmod(t - base, tx_n)
            w = min(tw, cam["width"] - tx * tw)
            h = min(th, cam["height"] - ty * th)
            m = oracle_lib.support_mask(info[2:5], Si, info[6], cam, tx * tw, ty * th, w, h)
            assert not m.any(), (pair, t)
            dropped += 1
    return dropped, n_rect, n_kept


@pytest.mark.parametrize("tile", [(16, 16), (32, 16)])
def test_unbounded_supports_keep_every_covered_tile(oracle_lib, tile):
    """Large primitives near the camera whose support is not a bounded ellipse in the image
    (their cone of rays reaches the camera plane): binning scans each tile row from both
    ends for the first and last tile whose pixel centres can meet the support.  Every
    dropped tile misses the support (oracle brute force), the scan drops tiles, and the
    image keeps oracle parity."""
    rng = np.random.default_rng(31)
    n = 400
    sc = scenes.uniform_scene(n, seed=31)
    sc["means"] = np.concatenate([
        rng.uniform([-0.4, -0.4, 0.03], [0.4, 0.4, 0.3], (n // 2, 3)),
        rng.uniform([-1, -1, 0.3], [1, 1, 2.0], (n - n // 2, 3))]).astype(np.float32)
    sc["log_scales"] = rng.uniform(np.log(0.03), np.log(0.5), (n, 3)).astype(np.float32)
    R1, t1 = scenes.look_at([0.2, -0.1, -0.2], [0.0, 0.0, 1.0])
    cams = [scenes.make_camera(96, 80, 70.0, 70.0), scenes.make_camera(120, 64, 60.0, 60.0, R=R1, t=t1),
            scenes.make_camera(1200, 48, 300.0, 300.0)]    # long tile rows
    r, _, rgb, T, nc = gpu_render(sc, cams, tile_w=tile[0], tile_h=tile[1])
    ell = fetch(r.debug_buffer(7), 8 * n * len(cams), np.float32).reshape(-1, 8)
    order = fetch(r.debug_buffer(3), r.last_counters["n_visible"], np.uint32)
    unbounded = {int(p) for p in order if not ell[p, 4] > 0}   # (r0, r1, cx, cy, a, b, d, det)
    assert len(unbounded) >= 10, len(unbounded)
    dropped, n_rect, n_kept = assert_dropped_tiles_miss_support(oracle_lib, sc, cams, r, n, tile, unbounded)
    assert dropped > 0 and n_kept < n_rect
    for v, cam in enumerate(cams):
        sl = view_slice(r, v)
        pix, idx = sample_pixels(cam, 1000, seed=v)
        orc = oracle_lib.render(sc, cam, pixels=pix)
        assert_parity(compare(rgb[sl][idx], T[sl][idx], orc))


def test_tall_view_row_counts(oracle_lib):
    """The depth sort carries each pair's tile-row count in a byte saturated at 255; a pair
    whose rectangle spans 255 tile rows or more takes its count from the rectangle instead.
    On a 64 x 2400 view with 8 x 8 tiles (300 tile rows) with large primitives, both kinds
    occur; the rows the binning counts equal the rectangles' rows, and the image keeps
    oracle parity."""
    rng = np.random.default_rng(41)
    n = 300
    sc = scenes.uniform_scene(n, seed=41)
    sc["means"] = np.stack([rng.uniform(-0.1, 0.1, n), rng.uniform(-2.0, 2.0, n),
                            rng.uniform(1.0, 2.5, n)], axis=1).astype(np.float32)
    sc["log_scales"] = rng.uniform(np.log(0.05), np.log(2.0), (n, 3)).astype(np.float32)
    cam = scenes.make_camera(64, 2400, 300.0, 300.0)
    r, _, rgb, T, nc = gpu_render(sc, [cam], tile_w=8, tile_h=8)
    ctr = r.last_counters
    rects = fetch(r.debug_buffer(1), 2 * n, np.uint32).reshape(-1, 2)
    order = fetch(r.debug_buffer(3), ctr["n_visible"], np.uint32)
    rows = np.array([rect_of(rects, int(p))[3] - rect_of(rects, int(p))[1] + 1 for p in order])
    assert np.sum(rows >= 255) >= 1 and np.sum(rows < 255) >= 1, np.bincount(np.minimum(rows, 255))
    assert ctr["n_rows"] == int(rows.sum())
    pix, idx = sample_pixels(cam, 1500, seed=3)
    orc = oracle_lib.render(sc, cam, pixels=pix)
    assert_parity(compare(rgb[idx], T[idx], orc))


def test_rects_match_oracle_quad(oracle_lib):
    """The GPU tile rectangle lies inside the tiles of the oracle's projected quad bounding
    box (Eq. V_ray; the GPU further intersects it with the support ellipse's box), except
    where a box edge sits within 0.01 px of a tile boundary; a primitive the GPU culls has
    no pixel centre in its support."""
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
        # the GPU intersects the quad's box with the support ellipse's box
        inside = got[0] >= want[0] and got[1] >= want[1] and got[2] <= want[2] and got[3] <= want[3]
        assert inside or near_edge, (g, got, want)
        checked += 1
    assert checked > 500


def test_many_tile_rows_keep_order_and_parity(oracle_lib):
    """More tile rows than the row sort keeps in shared memory (64 tall narrow views at 8x8
    tiles: 64 x 200 = 12,800 tile rows): the row counters then live in the histogram itself.
    Tile lists stay in depth order, the ranges partition the instances, and sampled pixels
    of several views keep oracle parity."""
    scene = scenes.uniform_scene(3000, seed=41)
    rng = np.random.default_rng(41)
    cams = []
    for _ in range(64):
        R1, t1 = scenes.look_at(rng.uniform(-0.5, 0.5, 3) * [1, 1, 0] + [0, 0, -0.5], [0.0, 0.0, 3.0])
        cams.append(scenes.make_camera(8, 1600, 400.0, 400.0, R=R1, t=t1))
    r, _, rgb, T, nc = gpu_render(scene, cams, tile_w=8, tile_h=8)
    assert sum(-(-c["height"] // 8) for c in cams) > 12288
    g_tiles, g_pos = instance_lists(r, r.last_counters["n_instances"])
    same = np.diff(g_tiles) == 0
    assert np.all(np.diff(g_pos)[same] > 0)
    for v in (0, 31, 63):
        sl = view_slice(r, v)
        pix, idx = sample_pixels(cams[v], 300, seed=v)
        orc = oracle_lib.render(scene, cams[v], pixels=pix)
        assert_parity(compare(rgb[sl][idx], T[sl][idx], orc))

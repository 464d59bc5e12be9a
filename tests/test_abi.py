"""The C-ABI library builds, loads and exports every entry point include/raygs.h declares;
host-side argument checks need no GPU (no kernel is launched here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rg():
    from paper_2503_18682_gb300 import build, raygs
    build.build()
    return raygs


def declared_functions():
    src = open(os.path.join(ROOT, "include", "raygs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(raygs_\w+)\s*\(", src)))


def test_header_symbols_exported(rg):
    L = rg.lib()
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(L, name), name
    bound = {s[0] for s in rg._SIGS}
    assert set(names) <= bound, set(names) - bound


def test_config_defaults(rg):
    cfg = rg.make_config()
    assert cfg.p_min == pytest.approx(1 / 255)
    assert cfg.t_stop == pytest.approx(1e-4)
    assert cfg.alpha_max == pytest.approx(0.99)
    assert cfg.mip_sigma2 == pytest.approx(0.1)
    assert (cfg.tile_w, cfg.tile_h) == (16, 16)
    assert cfg.fp64_degenerate == 1 and cfg.degenerate_ratio == pytest.approx(1e3)


def test_plan_validation_host_only(rg):
    from paper_2503_18682_gb300 import scenes
    cams = [scenes.make_camera(64, 48, 60.0, 60.0)]
    p = rg.raygs_plan_create(cams, 100, 1000)
    try:
        assert rg.lib().raygs_plan_num_pixels(p) == 64 * 48
        assert rg.lib().raygs_plan_num_tiles(p) == 4 * 3
        assert rg.raygs_plan_workspace_bytes(p) > 100 * (64 + 8 + 4)
        assert rg.lib().raygs_plan_pixel_offset(p, 0) == 0
        assert rg.lib().raygs_plan_pixel_offset(p, 1) == -1
        # binding a misaligned or too small workspace is refused before any CUDA call
        assert rg.lib().raygs_plan_bind(p, C.c_void_p(16), 1 << 40) == 1
        assert rg.lib().raygs_plan_bind(p, C.c_void_p(1 << 20), 16) == 2
        # calls out of order / unbound
        assert rg.lib().raygs_bin_sort(p, None) == 1
    finally:
        rg.raygs_plan_destroy(p)
    bad = [
        dict(n=-1), dict(n=1 << 31), dict(cap=-5),
        dict(cfg=dict(tile_w=12)), dict(cfg=dict(p_min=0.0)), dict(cfg=dict(alpha_max=1.0)),
        dict(cam=dict(width=0)), dict(cam=dict(fx=0.0)), dict(cam=dict(near=0.0)),
        # mode combinations the header refuses: GS with backward or with an anti-aliasing
        # term, an unknown divergence or anti-aliasing mode, a batch mixing exact views
        dict(cfg=dict(divergence=1, enable_backward=1)), dict(cfg=dict(divergence=1), cam=dict(mip=1)),
        dict(cfg=dict(divergence=1), cam=dict(mip=2)), dict(cfg=dict(divergence=2)),
        dict(cam=dict(mip=3)), dict(cfg=dict(batch_records=3)),
    ]
    for b in bad:
        cam = dict(cams[0], **b.get("cam", {}))
        cfg = rg.make_config(**b.get("cfg", {}))
        h = C.c_void_p()
        st = rg.lib().raygs_plan_create(rg.make_cameras([cam]), 1, b.get("n", 10), b.get("cap", 100),
                                        C.byref(cfg), C.byref(h))
        assert st == 1, b
        assert not h.value
    h = C.c_void_p()
    mixed = [dict(cams[0], mip="exact"), cams[0]]
    assert rg.lib().raygs_plan_create(rg.make_cameras(mixed), 2, 10, 10, None, C.byref(h)) == 1
    for ok in ([dict(cams[0], mip="exact")] * 2, [dict(cams[0], mip=1), cams[0]]):
        h = C.c_void_p()
        assert rg.lib().raygs_plan_create(rg.make_cameras(ok), 2, 10, 10, None, C.byref(h)) == 0
        rg.lib().raygs_plan_destroy(h)
    h = C.c_void_p()
    assert rg.lib().raygs_plan_create(rg.make_cameras(cams), 0, 10, 10, None, C.byref(h)) == 1
    assert rg.lib().raygs_plan_create(rg.make_cameras(cams * 65), 65, 10, 10, None, C.byref(h)) == 1


def test_status_strings(rg):
    for s in range(5):
        assert rg.lib().raygs_status_string(s)
    with pytest.raises(rg.RayGSError):
        rg._check(1, "x")
    # the failed-CUDA-call record is per thread and starts clear in a new thread
    import threading
    seen = []
    th = threading.Thread(target=lambda: seen.append(rg.lib().raygs_last_cuda_error()))
    th.start()
    th.join()
    assert seen == [0]

"""Thin Python binding of the RayGS C ABI (include/raygs.h).

Argument marshalling only: every step of the hot path runs in the CUDA library
(``libraygs.so``, built in-tree by ``build.py``).  PyTorch supplies device memory and the
current stream.  The functions named ``raygs_*`` mirror the C entry points one to one;
``Renderer`` strings them together (plan sizing, workspace allocation, capacity retry).
There is no fallback: if the library is missing every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libraygs.so")

F32, F16, BF16 = 0, 1, 2
MAX_VIEWS = 64


class RayGSError(RuntimeError):
    pass


class Camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("R", C.c_float * 9),
                ("t", C.c_float * 3), ("near_z", C.c_float), ("mip", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("p_min", C.c_float), ("t_stop", C.c_float), ("alpha_max", C.c_float),
                ("mip_sigma2", C.c_float), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("fp64_degenerate", C.c_int32), ("degenerate_ratio", C.c_float),
                ("enable_backward", C.c_int32), ("batch_records", C.c_int32),
                ("divergence", C.c_int32)]


class Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacity_logits", C.c_void_p), ("sh", C.c_void_p),
                ("sh_degree", C.c_int32), ("scale_dtype", C.c_int32),
                ("opacity_dtype", C.c_int32), ("sh_dtype", C.c_int32)]


class Counters(C.Structure):
    _fields_ = [("n_visible", C.c_int64), ("n_instances", C.c_int64), ("capacity", C.c_int64),
                ("n_nonfinite", C.c_int64), ("overflow", C.c_int32), ("pad", C.c_int32),
                ("n_rows", C.c_int64), ("n_rows_kept", C.c_int64)]


class Grads(C.Structure):
    _fields_ = [("d_means", C.c_void_p), ("d_log_scales", C.c_void_p), ("d_quats", C.c_void_p),
                ("d_opacity_logits", C.c_void_p), ("d_sh", C.c_void_p)]


_lib = None

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("raygs_config_default", None, [C.POINTER(Config)]),
    ("raygs_status_string", C.c_char_p, [C.c_int]),
    ("raygs_last_cuda_error", C.c_int, []),
    ("raygs_plan_create", C.c_int, [C.POINTER(Camera), C.c_int32, C.c_int64, C.c_int64,
                                    C.POINTER(Config), C.POINTER(C.c_void_p)]),
    ("raygs_plan_destroy", None, [C.c_void_p]),
    ("raygs_plan_workspace_bytes", C.c_size_t, [C.c_void_p]),
    ("raygs_plan_bind", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("raygs_plan_set_poses", C.c_int, [C.c_void_p, C.POINTER(Camera), C.c_void_p]),
    ("raygs_plan_num_pixels", C.c_int64, [C.c_void_p]),
    ("raygs_plan_pixel_offset", C.c_int64, [C.c_void_p, C.c_int32]),
    ("raygs_plan_num_tiles", C.c_int64, [C.c_void_p]),
    ("raygs_preprocess", C.c_int, [C.c_void_p, C.POINTER(Scene), C.c_void_p]),
    ("raygs_bin_sort", C.c_int, [C.c_void_p, C.c_void_p]),
    ("raygs_render", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("raygs_resolve_supersampled", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]),
    ("raygs_render_backward", C.c_int, [C.c_void_p, C.POINTER(Scene), C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.POINTER(Grads), C.c_void_p]),
    ("raygs_read_counters", C.c_int, [C.c_void_p, C.POINTER(Counters), C.c_void_p]),
    ("raygs_graph_capture", C.c_int, [C.c_void_p, C.POINTER(Scene), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    ("raygs_graph_launch", C.c_int, [C.c_void_p, C.c_void_p]),
    ("raygs_autotune", C.c_int, [C.POINTER(Camera), C.c_int32, C.POINTER(Scene), C.c_int64,
                                 C.POINTER(Config), C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_float)]),
    ("raygs_autotune_workspace_bytes", C.c_size_t, [C.POINTER(Camera), C.c_int32, C.c_int64, C.c_int64,
                                                    C.POINTER(Config)]),
    ("raygs_render_noalloc", C.c_int, [C.POINTER(Camera), C.c_int32, C.POINTER(Scene),
                                       C.POINTER(Config), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
]
_DEBUG_SIGS = [
    ("raygs_debug_render_counted", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.POINTER(C.c_ulonglong), C.c_void_p]),
    ("raygs_debug_buffer", C.c_void_p, [C.c_void_p, C.c_int]),
]


def lib():
    """Load libraygs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RayGSError(f"RayGS CUDA library not built ({LIB_PATH}); run "
                             "`python -m paper_2503_18682_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS + _DEBUG_SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        msg = lib().raygs_status_string(status).decode()
        extra = f" (cudaError {lib().raygs_last_cuda_error()})" if status == 3 else ""
        raise RayGSError(f"{what}: {msg}{extra}")


# ------------------------------------------------------------------ marshalling helpers

def _torch():
    import torch
    return torch


def stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_cameras(cams) -> C.Array:
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        a = arr[i]
        a.fx, a.fy, a.cx, a.cy = float(c["fx"]), float(c["fy"]), float(c["cx"]), float(c["cy"])
        a.width, a.height = int(c["width"]), int(c["height"])
        R = np.asarray(c["R"], dtype=np.float32).reshape(9)
        t = np.asarray(c["t"], dtype=np.float32).reshape(3)
        for k in range(9):
            a.R[k] = float(R[k])
        for k in range(3):
            a.t[k] = float(t[k])
        a.near_z = float(c.get("near", 0.01))
        m = c.get("mip", False)
        a.mip = 2 if m == "exact" else int(m)
    return arr


def make_config(**kw) -> Config:
    cfg = Config()
    lib().raygs_config_default(C.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


_DT = {"f32": F32, "f16": F16, "bf16": BF16}


def scene_to_device(scene: dict, device="cuda") -> dict:
    """numpy scene (scenes.py layout) -> dict of contiguous torch tensors on `device`."""
    torch = _torch()
    out = {"sh_degree": int(scene["sh_degree"])}
    for key, tag in (("means", None), ("log_scales", "scale_dtype"), ("quats", None),
                     ("opacity_logits", "opacity_dtype"), ("sh", "sh_dtype")):
        a = np.ascontiguousarray(scene[key])
        dt = scene.get(tag, "f32") if tag else "f32"
        if dt == "bf16":
            t = torch.from_numpy(a.view(np.int16)).view(torch.bfloat16)
        elif dt == "f16":
            t = torch.from_numpy(a.astype(np.float16))
        else:
            t = torch.from_numpy(a.astype(np.float32))
        out[key] = t.to(device).contiguous()
    return out


def _dtype_code(t) -> int:
    torch = _torch()
    return {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}[t.dtype]


def make_scene(st: dict) -> Scene:
    s = Scene()
    s.n = int(st["means"].shape[0])
    s.means = st["means"].data_ptr()
    s.log_scales = st["log_scales"].data_ptr()
    s.quats = st["quats"].data_ptr()
    s.opacity_logits = st["opacity_logits"].data_ptr()
    s.sh = st["sh"].data_ptr()
    s.sh_degree = int(st["sh_degree"])
    s.scale_dtype = _dtype_code(st["log_scales"])
    s.opacity_dtype = _dtype_code(st["opacity_logits"])
    s.sh_dtype = _dtype_code(st["sh"])
    return s


# ------------------------------------------------------------------ C entry points

def raygs_plan_create(cams, n_gaussians: int, max_instances: int, cfg: Config | None = None):
    arr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    h = C.c_void_p()
    _check(lib().raygs_plan_create(arr, len(arr), int(n_gaussians), int(max_instances),
                                   C.byref(cfg) if cfg is not None else None, C.byref(h)),
           "raygs_plan_create")
    return h


def raygs_plan_destroy(plan):
    lib().raygs_plan_destroy(plan)


def raygs_plan_workspace_bytes(plan) -> int:
    return int(lib().raygs_plan_workspace_bytes(plan))


def raygs_plan_bind(plan, ptr: int, nbytes: int):
    _check(lib().raygs_plan_bind(plan, C.c_void_p(ptr), nbytes), "raygs_plan_bind")


def raygs_plan_set_poses(plan, cams, stream=None):
    arr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    _check(lib().raygs_plan_set_poses(plan, arr, stream_ptr(stream)), "raygs_plan_set_poses")


def raygs_preprocess(plan, scene: Scene, stream=None):
    _check(lib().raygs_preprocess(plan, C.byref(scene), stream_ptr(stream)), "raygs_preprocess")


def raygs_bin_sort(plan, stream=None):
    _check(lib().raygs_bin_sort(plan, stream_ptr(stream)), "raygs_bin_sort")


def raygs_render(plan, rgb, T_final=None, n_contrib=None, stream=None):
    _check(lib().raygs_render(plan, rgb.data_ptr(), T_final.data_ptr() if T_final is not None else None,
                              n_contrib.data_ptr() if n_contrib is not None else None,
                              stream_ptr(stream)), "raygs_render")


def raygs_render_backward(plan, scene: Scene, T_final, n_contrib, dL_drgb, dL_dT, grads: Grads,
                          stream=None):
    _check(lib().raygs_render_backward(plan, C.byref(scene), T_final.data_ptr(), n_contrib.data_ptr(),
                                       dL_drgb.data_ptr(), dL_dT.data_ptr() if dL_dT is not None else None,
                                       C.byref(grads), stream_ptr(stream)), "raygs_render_backward")


def raygs_resolve_supersampled(plan, factor: int, rgb_hi, T_hi, rgb_lo, T_lo=None, stream=None):
    """Box-filter resolve of views rendered at `factor` times the resolution (see
    supersampled_cameras) into rgb_lo / T_lo."""
    _check(lib().raygs_resolve_supersampled(plan, int(factor), rgb_hi.data_ptr(),
                                            T_hi.data_ptr() if T_hi is not None else None, rgb_lo.data_ptr(),
                                            T_lo.data_ptr() if T_lo is not None else None, stream_ptr(stream)),
           "raygs_resolve_supersampled")


def supersampled_cameras(cams, factor: int):
    """The cameras at `factor` times the resolution whose factor x factor pixel blocks hold
    each original pixel's sub-pixel rays (width, height, fx, fy, cx, cy all scaled)."""
    out = []
    for c in cams:
        d = dict(c)
        for k in ("width", "height"):
            d[k] = int(c[k]) * factor
        for k in ("fx", "fy", "cx", "cy"):
            d[k] = np.float32(float(c[k]) * factor)
        out.append(d)
    return out


def raygs_read_counters(plan, stream=None) -> dict:
    c = Counters()
    _check(lib().raygs_read_counters(plan, C.byref(c), stream_ptr(stream)), "raygs_read_counters")
    return dict(n_visible=c.n_visible, n_instances=c.n_instances, capacity=c.capacity,
                n_nonfinite=c.n_nonfinite, overflow=c.overflow, n_rows=c.n_rows, n_rows_kept=c.n_rows_kept)


def raygs_graph_capture(plan, scene: Scene, rgb, T_final=None, n_contrib=None, stream=None):
    _check(lib().raygs_graph_capture(plan, C.byref(scene), rgb.data_ptr(),
                                     T_final.data_ptr() if T_final is not None else None,
                                     n_contrib.data_ptr() if n_contrib is not None else None,
                                     stream_ptr(stream)), "raygs_graph_capture")


def raygs_graph_launch(plan, stream=None):
    _check(lib().raygs_graph_launch(plan, stream_ptr(stream)), "raygs_graph_launch")


TILE_CANDIDATES = [(16, 16), (16, 8), (32, 16), (8, 8)]
# autotuner candidates in its order: (tile_w, tile_h, batch_records), shape-major
AUTOTUNE_CANDIDATES = [(w, h, b) for (w, h) in TILE_CANDIDATES for b in (1, 2)]


def raygs_autotune_workspace_bytes(cams, n_gaussians: int, max_instances: int, cfg: Config | None = None) -> int:
    arr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    return int(lib().raygs_autotune_workspace_bytes(arr, len(arr), int(n_gaussians), int(max_instances),
                                                    C.byref(cfg) if cfg is not None else None))


def raygs_autotune(cams, scene: Scene, max_instances: int, cfg: Config, workspace, rgb, T_final=None,
                   n_contrib=None, iters: int = 3, stream=None):
    """Pick the fastest tile shape and rasteriser batch (written into cfg); returns
    {"WxH/bN": ms per pass}."""
    arr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    ms = (C.c_float * len(AUTOTUNE_CANDIDATES))()
    _check(lib().raygs_autotune(arr, len(arr), C.byref(scene), int(max_instances), C.byref(cfg),
                                workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                rgb.data_ptr(), T_final.data_ptr() if T_final is not None else None,
                                n_contrib.data_ptr() if n_contrib is not None else None, int(iters),
                                stream_ptr(stream), ms), "raygs_autotune")
    return {f"{w}x{h}/b{b}": float(ms[i]) for i, (w, h, b) in enumerate(AUTOTUNE_CANDIDATES)}


def autotune(cams, scene_t: dict, capacity: int, device="cuda", iters: int = 3, **cfg_kw):
    """Convenience: allocate the autotuning workspace, run raygs_autotune, return
    (config kwargs of the fastest shape, timings)."""
    torch = _torch()
    cfg = make_config(**cfg_kw)
    nb = raygs_autotune_workspace_bytes(cams, scene_t["means"].shape[0], capacity, cfg)
    ws = torch.empty(nb, dtype=torch.uint8, device=device)
    npx = sum(int(c["width"]) * int(c["height"]) for c in cams)
    rgb = torch.empty((npx, 3), dtype=torch.float32, device=device)
    T = torch.empty(npx, dtype=torch.float32, device=device)
    nc = torch.empty(npx, dtype=torch.int32, device=device)
    times = raygs_autotune(cams, make_scene(scene_t), capacity, cfg, ws, rgb, T, nc, iters)
    del ws
    return dict(cfg_kw, tile_w=int(cfg.tile_w), tile_h=int(cfg.tile_h), batch_records=int(cfg.batch_records)), times


def raygs_render_noalloc(cams, scene: Scene, cfg: Config | None, rgb, T_final=None, n_contrib=None,
                         stream=None, check=True) -> int:
    """Allocation-free forward render (see include/raygs.h); returns the status code and
    raises on failure when check=True."""
    arr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    st = lib().raygs_render_noalloc(arr, len(arr), C.byref(scene), C.byref(cfg) if cfg is not None else None,
                                    rgb.data_ptr(), T_final.data_ptr() if T_final is not None else None,
                                    n_contrib.data_ptr() if n_contrib is not None else None,
                                    stream_ptr(stream))
    if check:
        _check(st, "raygs_render_noalloc")
    return st


# ------------------------------------------------------------------ convenience wrapper

class Renderer:
    """A plan + its device workspace for a fixed camera set and primitive count."""

    def __init__(self, cams, n_gaussians: int, capacity: int | None = None, device="cuda", **cfg):
        torch = _torch()
        self.cams = list(cams)
        self.n = int(n_gaussians)
        self.device = torch.device(device)
        self.cfg = make_config(**cfg)
        if capacity is None:
            capacity = max(1 << 16, 4 * self.n * len(self.cams))
        self.capacity = int(min(capacity, (1 << 32) - 4096))
        self.plan = None
        self._ws = None
        self._make_plan()

    def _make_plan(self):
        torch = _torch()
        if self.plan is not None:
            raygs_plan_destroy(self.plan)
            self.plan = None
        self._ws = None  # release the old workspace before sizing the new one
        self.plan = raygs_plan_create(self.cams, self.n, self.capacity, self.cfg)
        nb = raygs_plan_workspace_bytes(self.plan)
        self._ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        raygs_plan_bind(self.plan, self._ws.data_ptr(), nb)
        self.num_pixels = int(lib().raygs_plan_num_pixels(self.plan))
        self.num_tiles = int(lib().raygs_plan_num_tiles(self.plan))
        self.pixel_offsets = [int(lib().raygs_plan_pixel_offset(self.plan, v))
                              for v in range(len(self.cams))]

    def __del__(self):
        try:
            if self.plan is not None:
                raygs_plan_destroy(self.plan)
        except Exception:
            pass

    def alloc_outputs(self):
        torch = _torch()
        rgb = torch.empty((self.num_pixels, 3), dtype=torch.float32, device=self.device)
        T = torch.empty(self.num_pixels, dtype=torch.float32, device=self.device)
        nc = torch.empty(self.num_pixels, dtype=torch.int32, device=self.device)
        return rgb, T, nc

    def forward(self, scene_t: dict, rgb=None, T=None, nc=None, stream=None, check=True):
        """preprocess + bin_sort + render (see _forward)."""
        out = self._forward(scene_t, rgb, T, nc, stream, check)
        self.forward_id = getattr(self, "forward_id", 0) + 1
        return out

    def backward(self, scene_t: dict, T, nc, dL_drgb, dL_dT=None, stream=None, forward_id=None):
        """Gradients of the last forward's image (needs enable_backward=1).  Returns a dict
        of float32 tensors shaped like the scene attributes."""
        torch = _torch()
        if forward_id is not None and forward_id != getattr(self, "forward_id", None):
            raise RayGSError("backward must follow its own forward on this Renderer")
        dev = self.device
        n = self.n
        k = (int(scene_t["sh_degree"]) + 1) ** 2
        out = dict(means=torch.empty((n, 3), dtype=torch.float32, device=dev),
                   log_scales=torch.empty((n, 3), dtype=torch.float32, device=dev),
                   quats=torch.empty((n, 4), dtype=torch.float32, device=dev),
                   opacity_logits=torch.empty((n,), dtype=torch.float32, device=dev),
                   sh=torch.empty((n, k, 3), dtype=torch.float32, device=dev))
        g = Grads()
        g.d_means, g.d_log_scales, g.d_quats = (out["means"].data_ptr(), out["log_scales"].data_ptr(),
                                                out["quats"].data_ptr())
        g.d_opacity_logits, g.d_sh = out["opacity_logits"].data_ptr(), out["sh"].data_ptr()
        raygs_render_backward(self.plan, make_scene(scene_t), T, nc, dL_drgb.contiguous(),
                              dL_dT.contiguous() if dL_dT is not None else None, g, stream)
        return out

    def _forward(self, scene_t: dict, rgb=None, T=None, nc=None, stream=None, check=True):
        """preprocess + bin_sort + render.  With check=True the counters are read (one
        sync) and the plan is regrown and the call repeated if the instance capacity
        overflowed."""
        if rgb is None:
            rgb, T, nc = self.alloc_outputs()
        sc = make_scene(scene_t)
        for _attempt in range(3):
            raygs_preprocess(self.plan, sc, stream)
            raygs_bin_sort(self.plan, stream)
            raygs_render(self.plan, rgb, T, nc, stream)
            if not check:
                break
            ctr = raygs_read_counters(self.plan, stream)
            self.last_counters = ctr
            if not ctr["overflow"]:
                break
            self.capacity = int(min(ctr["n_instances"] * 1.15 + 4096, (1 << 32) - 4096))
            self._make_plan()
        return rgb, T, nc

    def view_image(self, rgb, v: int):
        c = self.cams[v]
        o = self.pixel_offsets[v]
        return rgb[o:o + c["width"] * c["height"]].view(c["height"], c["width"], -1)

    def counted_render(self, rgb, T=None, nc=None, stream=None):
        """Instrumented render: returns (evaluated pairs, composited pairs)."""
        st = self.counted_render_stats(rgb, T, nc, stream)
        return st["evaluated"], st["composited"]

    def counted_render_stats(self, rgb, T=None, nc=None, stream=None) -> dict:
        """Instrumented render: evaluated and composited (pixel, primitive) pairs, consumed
        list entries (records the tiles staged before they stopped) and the rasteriser's
        (thread, record) iterations."""
        out = (C.c_ulonglong * 4)()
        _check(lib().raygs_debug_render_counted(self.plan, rgb.data_ptr(),
                                                T.data_ptr() if T is not None else None,
                                                nc.data_ptr() if nc is not None else None,
                                                out, stream_ptr(stream)), "raygs_debug_render_counted")
        return dict(evaluated=int(out[0]), composited=int(out[1]), consumed=int(out[2]),
                    iterations=int(out[3]))

    def debug_buffer(self, which: int) -> int:
        return int(lib().raygs_debug_buffer(self.plan, which) or 0)


# ------------------------------------------------------------------ autograd

def _autograd_function():
    torch = _torch()

    class RenderFunction(torch.autograd.Function):
        """Differentiable RayGS render through the C ABI (forward: raygs_preprocess +
        raygs_bin_sort + raygs_render; backward: raygs_render_backward)."""

        @staticmethod
        def forward(ctx, renderer, sh_degree, means, log_scales, quats, opacity_logits, sh):
            st = dict(means=means.detach().contiguous(), log_scales=log_scales.detach().contiguous(),
                      quats=quats.detach().contiguous(), opacity_logits=opacity_logits.detach().contiguous(),
                      sh=sh.detach().contiguous(), sh_degree=int(sh_degree))
            rgb, T, nc = renderer.forward(st)
            ctx.renderer, ctx.st, ctx.fid = renderer, st, renderer.forward_id
            ctx.save_for_backward(T, nc)
            ctx.mark_non_differentiable(nc)
            return rgb, T, nc

        @staticmethod
        def backward(ctx, g_rgb, g_T, _g_nc):
            T, nc = ctx.saved_tensors
            g = ctx.renderer.backward(ctx.st, T, nc, g_rgb, g_T, forward_id=ctx.fid)
            return (None, None, g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"])

    return RenderFunction


_RENDER_FN = None


def render(renderer: "Renderer", params: dict):
    """Differentiable render of torch parameters (means, log_scales, quats,
    opacity_logits, sh, sh_degree) with a Renderer created with enable_backward=1.
    Returns (rgb [P,3], T [P], n_contrib [P])."""
    global _RENDER_FN
    if _RENDER_FN is None:
        _RENDER_FN = _autograd_function()
    return _RENDER_FN.apply(renderer, int(params["sh_degree"]), params["means"], params["log_scales"],
                            params["quats"], params["opacity_logits"], params["sh"])

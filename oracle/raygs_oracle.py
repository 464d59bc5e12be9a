"""ctypes wrapper of the FP64 CPU oracle (raygs_oracle.c).  Test infrastructure only."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raygs_oracle.c")
_LIB = os.path.join(_HERE, "libraygs_oracle.so")
_lock = threading.Lock()
_lib = None

# per-primitive record layout of oracle_prepare (see the enum in raygs_oracle.c)
OG = dict(STATUS=0, KEY=1, MU=slice(2, 5), C2=5, KAPPA=6, O=7, RGB=slice(8, 11),
          S=slice(11, 14), RC=slice(14, 23), BORDER=23, LEN=24)

# divergence: 0 the ray divergence (Eq. Q_ray), 1 the GS divergence of Sec. 3.1
DEFAULT_CFG = dict(p_min=1.0 / 255.0, t_stop=1e-4, alpha_max=0.99, mip_sigma2=0.1, divergence=0)

FLAG_CUTOFF, FLAG_STOP, FLAG_BORDER = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                                   "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.oracle_prepare.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, P, P, P]
        L.oracle_prepare.restype = C.c_int
        L.oracle_render.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, P, P, C.c_int64, P,
                                    P, P, P, P, P, C.c_int]
        L.oracle_render.restype = C.c_int
        L.oracle_quad.argtypes = [P, P, P, C.c_double, P]
        L.oracle_quad.restype = None
        L.oracle_rot_align.argtypes = [P, P]
        L.oracle_rot_align.restype = None
        L.oracle_D_ray.argtypes = [P, P, P, P]
        L.oracle_D_ray.restype = C.c_double
        L.oracle_support_mask.argtypes = [P, P, C.c_double, P, C.c_int, C.c_int, C.c_int, C.c_int, P]
        L.oracle_support_mask.restype = None
        L.oracle_sh_basis.argtypes = [C.c_int, P, P]
        L.oracle_sh_basis.restype = None
        L.oracle_quat_to_rot.argtypes = [P, P]
        L.oracle_quat_to_rot.restype = None
        L.oracle_depth_key.argtypes = [P, C.c_float, P, P]
        L.oracle_depth_key.restype = C.c_uint32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def mip_mode(m) -> int:
    """Camera anti-aliasing mode: 0 off, 1 (or True) the pixel-invariant Eq. mip, 2 (or
    "exact") the pixel-dependent form of Sec. 5."""
    if m == "exact":
        return 2
    m = int(m)
    if m not in (0, 1, 2):
        raise ValueError(f"mip mode {m}")
    return m


def cam_array(cam: dict) -> np.ndarray:
    """Camera dict (scenes.make_camera) -> 20 doubles holding its float32 values."""
    a = np.zeros(20, dtype=np.float64)
    a[0] = np.float32(cam["fx"]); a[1] = np.float32(cam["fy"])
    a[2] = np.float32(cam["cx"]); a[3] = np.float32(cam["cy"])
    a[4] = cam["width"]; a[5] = cam["height"]
    a[6:15] = np.asarray(cam["R"], dtype=np.float32).reshape(9)
    a[15:18] = np.asarray(cam["t"], dtype=np.float32).reshape(3)
    a[18] = np.float32(cam.get("near", 0.01))
    a[19] = float(mip_mode(cam.get("mip", False)))
    return a


def cfg_array(cfg: dict | None = None) -> np.ndarray:
    c = dict(DEFAULT_CFG)
    if cfg:
        c.update(cfg)
    return np.array([c["p_min"], c["t_stop"], c["alpha_max"], c["mip_sigma2"], c["divergence"]], dtype=np.float64)


def _scene_arrays(scene: dict):
    for tag in ("scale_dtype", "sh_dtype", "opacity_dtype"):
        if scene.get(tag, "f32") != "f32":
            raise ValueError("the oracle takes float32 attributes: widen the scene first")
    f = lambda k: np.ascontiguousarray(scene[k], dtype=np.float32)
    return (f("means"), f("log_scales"), f("quats"), f("opacity_logits"), f("sh"),
            int(scene["sh_degree"]))


def prepare(scene: dict, cam: dict, cfg: dict | None = None) -> np.ndarray:
    """Per-primitive FP64 quantities for one camera: array [N, OG['LEN']]."""
    m, ls, q, lo, sh, deg = _scene_arrays(scene)
    n = m.shape[0]
    out = np.zeros((n, OG["LEN"]), dtype=np.float64)
    ca, cf = cam_array(cam), cfg_array(cfg)
    rc = lib().oracle_prepare(n, _p(m), _p(ls), _p(q), _p(lo), _p(sh), deg, _p(ca), _p(cf), _p(out))
    if rc:
        raise RuntimeError(f"oracle_prepare failed ({rc})")
    return out


def render(scene: dict, cam: dict, cfg: dict | None = None, pixels=None, threads: int = 0) -> dict:
    """Brute-force FP64 render of one camera.

    ``pixels``: None for the full image (row-major), else an int array [P, 2] of (x, y).
    Returns rgb [P, 3], T [P], ncontrib [P], flags [P], sig [P] (uint64).
    """
    m, ls, q, lo, sh, deg = _scene_arrays(scene)
    n = m.shape[0]
    W, H = int(cam["width"]), int(cam["height"])
    if pixels is None:
        npx = W * H
        pix_ptr = None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        npx = pix.shape[0]
        pix_ptr = _p(pix)
    rgb = np.zeros((npx, 3), dtype=np.float64)
    T = np.zeros(npx, dtype=np.float64)
    nc = np.zeros(npx, dtype=np.int32)
    fl = np.zeros(npx, dtype=np.int32)
    sig = np.zeros(npx, dtype=np.uint64)
    ca, cf = cam_array(cam), cfg_array(cfg)
    rc = lib().oracle_render(n, _p(m), _p(ls), _p(q), _p(lo), _p(sh), deg, _p(ca), _p(cf),
                             npx, pix_ptr, _p(rgb), _p(T), _p(nc), _p(fl), _p(sig), int(threads))
    if rc:
        raise RuntimeError(f"oracle_render failed ({rc})")
    return dict(rgb=rgb, T=T, ncontrib=nc, flags=fl, sig=sig)


def quad(mu, Rc, s, kappa) -> dict:
    """The paper's vertex stage (Sec. 4.1) for one primitive in the camera frame."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    Rc = np.ascontiguousarray(Rc, dtype=np.float64).reshape(9)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros(48, dtype=np.float64)
    lib().oracle_quad(_p(mu), _p(Rc), _p(s), float(kappa), _p(out))
    return dict(V=out[0:12].reshape(4, 3).T.copy(), Z=out[12:20].reshape(4, 2).T.copy(),
                U=out[20:24].reshape(2, 2).T.copy(), c2=out[24], b=out[25], a=out[26],
                Q=out[27:36].reshape(3, 3).copy(), Ralign=out[36:45].reshape(3, 3).copy(),
                muhat=out[45:48].copy())


def rot_align(muhat) -> np.ndarray:
    mh = np.ascontiguousarray(muhat, dtype=np.float64)
    R = np.zeros(9, dtype=np.float64)
    lib().oracle_rot_align(_p(mh), _p(R))
    return R.reshape(3, 3)


def D_ray(mu, Sigma_inv, x):
    """Eq. Q_ray for one ray: returns (D, tau)."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    Si = np.ascontiguousarray(Sigma_inv, dtype=np.float64).reshape(9)
    x = np.ascontiguousarray(x, dtype=np.float64)
    tau = np.zeros(1, dtype=np.float64)
    D = lib().oracle_D_ray(_p(mu), _p(Si), _p(x), _p(tau))
    return float(D), float(tau[0])


def support_mask(mu, Sigma_inv, kappa, cam, x0, y0, w, h) -> np.ndarray:
    """Pixels of the rectangle [x0, x0+w) x [y0, y0+h) whose centre ray has tau > 0 and
    D <= kappa (Eq. Q_ray with the cut-off): bool array [h, w]."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    Si = np.ascontiguousarray(Sigma_inv, dtype=np.float64).reshape(9)
    c = np.array([float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])], dtype=np.float64)
    out = np.zeros(h * w, dtype=np.uint8)
    lib().oracle_support_mask(_p(mu), _p(Si), float(kappa), _p(c), int(x0), int(y0), int(w), int(h), _p(out))
    return out.reshape(h, w).astype(bool)


def sh_basis(degree: int, d) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.float64)
    Y = np.zeros(16, dtype=np.float64)
    lib().oracle_sh_basis(int(degree), _p(d), _p(Y))
    return Y[: (degree + 1) ** 2].copy()


def quat_to_rot(q) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros(9, dtype=np.float64)
    lib().oracle_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def depth_key(r2, t2, mu):
    r2 = np.ascontiguousarray(r2, dtype=np.float32)
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    z = np.zeros(1, dtype=np.float32)
    k = lib().oracle_depth_key(_p(r2), C.c_float(float(t2)), _p(mu), _p(z))
    return int(k), float(z[0])

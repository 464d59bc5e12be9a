"""Seeded synthetic scenes and cameras.

This module only draws random inputs; it holds none of the renderer's arithmetic, so both
the CUDA path (through the binding) and the FP64 CPU oracle consume its arrays as data.

The scenes stand in for the MipNeRF360 / Tanks&Temples reconstructions the paper renders
(Sec. 6, Table 1: 0.82M-5.35M primitives, real captures).  Those datasets and trained
models are not available, so every scene here is synthetic; none of their content is
reproduced.

Conventions
-----------
* Primitive parameters follow Sec. 3 ("Scene representation"): a mean, a covariance
  factored as rotation x diagonal scale, a prior opacity and a feature (colour) vector.
  They are stored as

  - ``means``          float32 [N, 3]   world-frame centres
  - ``log_scales``     float32 [N, 3]   log of the diagonal of S
  - ``quats``          float32 [N, 4]   rotation quaternion (w, x, y, z), unit length
  - ``opacity_logits`` float32 [N]      prior opacity o = sigmoid(logit)
  - ``sh``             float32 [N, K, 3] colour coefficients, K = (degree + 1)**2; the
    first coefficient is the base RGB colour.

* A camera is a pinhole (Sec. 3.1) with OpenCV axes (x right, y down, z forward):
  ``x_cam = R @ x_world + t``; pixel (i, j) looks along ((i+.5-cx)/fx, (j+.5-cy)/fy, 1).
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations: a normalised isotropic 4-D normal draw."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(F32)


def make_camera(width, height, fx, fy, cx=None, cy=None, R=None, t=None,
                near=0.01, mip=False) -> dict:
    """A pinhole camera record (all floating fields float32 values).  mip: False / 0 none,
    True / 1 the pixel-invariant anti-aliasing term, "exact" / 2 the pixel-dependent one."""
    if cx is None:
        cx = width / 2.0
    if cy is None:
        cy = height / 2.0
    R = np.eye(3, dtype=F32) if R is None else np.asarray(R, dtype=F32)
    t = np.zeros(3, dtype=F32) if t is None else np.asarray(t, dtype=F32)
    return dict(width=int(width), height=int(height), fx=F32(fx), fy=F32(fy),
                cx=F32(cx), cy=F32(cy), R=R.reshape(3, 3), t=t.reshape(3),
                near=F32(near), mip=(2 if mip == "exact" else int(mip)))


def look_at(eye, target, up=(0.0, 1.0, 0.0)):
    """World->camera (R, t) of a camera at ``eye`` looking at ``target`` (OpenCV axes)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, dtype=np.float64)
    if abs(float(np.dot(f, up))) > 0.99:          # forward almost parallel to up
        up = np.array([1.0, 0.0, 0.0]) if abs(f[0]) < 0.9 else np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f]).astype(F32)
    t = (-(R.astype(np.float64) @ eye)).astype(F32)
    return R, t


def uniform_scene(n=1000, seed=0) -> dict:
    """Small scene: means U([-1,1]^2 x [2,4]), scales log-uniform [0.01, 0.1] per axis,
    uniform random rotations, opacity sigmoid(N(0,1)), SH degree 0 with RGB U[0,1]."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n),
                      rng.uniform(2, 4, n)], axis=1).astype(F32)
    log_scales = rng.uniform(np.log(0.01), np.log(0.1), (n, 3)).astype(F32)
    quats = _unit_quats(rng, n)
    logits = rng.standard_normal(n).astype(F32)
    sh = rng.uniform(0, 1, (n, 1, 3)).astype(F32)
    return dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=logits,
                sh=sh, sh_degree=0)


def blob_scene(n, seed, sh_degree=3, n_blobs=64, blob_sigma=0.3,
               box_lo=(-5.0, -5.0, 1.0), box_hi=(5.0, 5.0, 11.0),
               degenerate_frac=0.0) -> dict:
    """Mixture-of-blobs scene shaped like a reconstructed capture.

    Blob centres are uniform in a 10 m box in front of the identity camera; means are
    isotropic normal around a random centre (sigma 0.3 m); scales log-normal around 2 cm
    (sigma 0.8); opacity sigmoid(N(0, 1.5)); colour: base RGB U[0,1], higher SH bands
    N(0, 0.05).  ``degenerate_frac`` of the primitives get their smallest axis shrunk to
    s_max * 10**-U(3,4) (axis ratio above 1e3: near-flat disks).
    """
    rng = np.random.default_rng(seed)
    lo = np.asarray(box_lo)
    hi = np.asarray(box_hi)
    centres = lo + (hi - lo) * rng.uniform(0, 1, (n_blobs, 3))
    which = rng.integers(0, n_blobs, n)
    means = (centres[which] + blob_sigma * rng.standard_normal((n, 3))).astype(F32)
    log_scales = (np.log(0.02) + 0.8 * rng.standard_normal((n, 3)))
    if degenerate_frac > 0:
        n_deg = int(round(degenerate_frac * n))
        idx = rng.choice(n, n_deg, replace=False)
        ls = log_scales[idx]
        amin = np.argmin(ls, axis=1)
        ratio_dec = rng.uniform(3.0, 4.0, n_deg)
        ls[np.arange(n_deg), amin] = ls.max(axis=1) - ratio_dec * np.log(10.0)
        log_scales[idx] = ls
    log_scales = log_scales.astype(F32)
    quats = _unit_quats(rng, n)
    logits = (1.5 * rng.standard_normal(n)).astype(F32)
    k = (sh_degree + 1) ** 2
    sh = np.empty((n, k, 3), dtype=F32)
    sh[:, 0, :] = rng.uniform(0, 1, (n, 3))
    if k > 1:
        sh[:, 1:, :] = 0.05 * rng.standard_normal((n, k - 1, 3))
    return dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=logits,
                sh=sh, sh_degree=sh_degree)


def subset(scene: dict, idx) -> dict:
    out = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    return out


# --------------------------------------------------------------------------- workloads

def workload_small(seed=0):
    """1 view 64x64 (fx=fy=64, cx=cy=32) at the origin looking +z; 1,000 primitives."""
    scene = uniform_scene(1000, seed)
    cams = [make_camera(64, 64, 64.0, 64.0, 32.0, 32.0)]
    return scene, cams


def workload_mip_720p(seed=1, n=500_000):
    """1 view 1280x720 (fx=fy=1000) with the MIP filter; 500k blob primitives, SH degree 3."""
    scene = blob_scene(n, seed)
    cams = [make_camera(1280, 720, 1000.0, 1000.0, mip=True)]
    return scene, cams


def workload_backward_720p(seed=2, n=1_500_000):
    """1 view 1280x720 (fx=fy=1000); 1.5M blob primitives for forward + backward."""
    scene = blob_scene(n, seed)
    cams = [make_camera(1280, 720, 1000.0, 1000.0)]
    return scene, cams


def stereo_batch_cameras(seed=3, centre=(0.0, 0.0, 6.0), radius=3.0, ipd=0.064,
                         eye_w=2064, eye_h=2208, eye_f=1100.0, n_pairs=4, n_extra=8):
    """4 stereo pairs (2064x2208 per eye) plus 8 views of random size in
    [640,1920]x[480,1080]; every camera sits on a 3 m sphere around the scene centre
    looking at it (uniform random directions)."""
    rng = np.random.default_rng(seed + 1000)
    centre = np.asarray(centre, dtype=np.float64)
    cams = []

    def rand_dir():
        v = rng.standard_normal(3)
        return v / np.linalg.norm(v)

    for _ in range(n_pairs):
        eye = centre + radius * rand_dir()
        R, _t = look_at(eye, centre)
        right = R[0].astype(np.float64)
        for side in (-0.5, 0.5):
            e = eye + side * ipd * right
            t = (-(R.astype(np.float64) @ e)).astype(F32)
            cams.append(make_camera(eye_w, eye_h, eye_f, eye_f, R=R, t=t))
    for _ in range(n_extra):
        w = int(rng.integers(640, 1921))
        h = int(rng.integers(480, 1081))
        f = eye_f * w / eye_w
        eye = centre + radius * rand_dir()
        R, t = look_at(eye, centre)
        cams.append(make_camera(w, h, f, f, R=R, t=t))
    return cams


def workload_stereo_batch(seed=3, n=3_000_000, degenerate_frac=0.10):
    """3M blob primitives (10% near-flat, axis ratio > 1e3) seen by 16 uneven views."""
    scene = blob_scene(n, seed, degenerate_frac=degenerate_frac)
    return scene, stereo_batch_cameras(seed)


def precision_cameras(seed=4):
    """4 poses at 3840x2160 plus the same 4 poses at 960x540 with the MIP filter."""
    rng = np.random.default_rng(seed + 1000)
    centre = np.array([0.0, 0.0, 6.0])
    cams_hi, cams_lo = [], []
    for _ in range(4):
        v = rng.standard_normal(3)
        eye = centre + 3.0 * v / np.linalg.norm(v)
        R, t = look_at(eye, centre)
        cams_hi.append(make_camera(3840, 2160, 2000.0, 2000.0, R=R, t=t))
        cams_lo.append(make_camera(960, 540, 500.0, 500.0, R=R, t=t, mip=True))
    return cams_hi + cams_lo


def workload_precision(seed=4, n=6_000_000):
    scene = blob_scene(n, seed)
    return scene, precision_cameras(seed)


# ----------------------------------------------------------- reduced-precision storage

def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even float32 -> bfloat16, returned as uint16 bit patterns."""
    b = np.ascontiguousarray(x, dtype=F32).view(np.uint32).astype(np.uint64)
    rounding = ((b >> 16) & 1) + 0x7FFF
    return ((b + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(F32)


def _store(x: np.ndarray, dtype: str):
    if dtype == "f32":
        return np.asarray(x, dtype=F32)
    if dtype == "f16":
        return np.asarray(x, dtype=F32).astype(np.float16)
    if dtype == "bf16":
        return f32_to_bf16_bits(x)
    raise ValueError(dtype)


def to_storage_form(scene: dict, sh: str = "f32", scales: str = "f32", opacity: str = "f32") -> dict:
    """Store SH coefficients, log-scales and opacity logits each in its own dtype ('f32',
    'f16' or 'bf16'; opacity 'f32' or 'f16').  Reduced fields are numpy float16 arrays
    ('f16') or uint16 bf16 bit patterns ('bf16'), tagged ``sh_dtype``/``scale_dtype``/
    ``opacity_dtype``."""
    if opacity not in ("f32", "f16"):
        raise ValueError(opacity)
    out = dict(scene)
    out["sh"], out["sh_dtype"] = _store(scene["sh"], sh), sh
    out["log_scales"], out["scale_dtype"] = _store(scene["log_scales"], scales), scales
    out["opacity_logits"], out["opacity_dtype"] = _store(scene["opacity_logits"], opacity), opacity
    return out


def to_storage(scene: dict, dtype: str) -> dict:
    """Store log-scales and SH in ``dtype`` ('f16' or 'bf16') and opacity logits in f16.

    Returns a new scene whose reduced fields are numpy float16 arrays ('f16') or uint16
    bf16 bit patterns ('bf16'), with ``scale_dtype``/``sh_dtype``/``opacity_dtype`` tags.
    """
    if dtype not in ("f16", "bf16"):
        raise ValueError(dtype)
    return to_storage_form(scene, sh=dtype, scales=dtype, opacity="f16")


def round_attributes(scene: dict, sh_dc: str = "f32", sh_rest: str = "f32", scales: str = "f32",
                     opacity: str = "f32") -> dict:
    """The float32 scene whose chosen attribute groups are rounded to 'f16' or 'bf16' (SH DC
    coefficient, higher SH bands, log-scales, opacity logits): the values a reduced storage
    of just those groups would hold, kept in float32 (an ablation of the storage rounding)."""
    def rnd(x, dt):
        x = np.asarray(x, dtype=F32)
        if dt == "f32":
            return x.copy()
        if dt == "f16":
            return x.astype(np.float16).astype(F32)
        if dt == "bf16":
            return bf16_bits_to_f32(f32_to_bf16_bits(x))
        raise ValueError(dt)
    out = dict(scene)
    sh = np.array(scene["sh"], dtype=F32)
    sh[:, :1] = rnd(sh[:, :1], sh_dc)
    sh[:, 1:] = rnd(sh[:, 1:], sh_rest)
    out["sh"] = sh
    out["log_scales"] = rnd(scene["log_scales"], scales)
    out["opacity_logits"] = rnd(scene["opacity_logits"], opacity)
    return out


def widen(scene: dict) -> dict:
    """The float32 values a reduced-precision scene holds (exact widening)."""
    out = dict(scene)
    for key, tag in (("log_scales", "scale_dtype"), ("sh", "sh_dtype"),
                     ("opacity_logits", "opacity_dtype")):
        t = scene.get(tag, "f32")
        if t == "bf16":
            out[key] = bf16_bits_to_f32(scene[key])
        else:
            out[key] = np.asarray(scene[key]).astype(F32)
        out[tag] = "f32"
    return out

"""Dense FP64 PyTorch-CPU restatement of the RayGS image, for reference gradients.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Same definitions and readings as
raygs_oracle.c (Sec. 3 activation and Eq. rendering, Sec. 3.2 Eq. Q_ray and Eq. c, Eq.
support, Eq. rend_opacity, the 0.99 clamp and the 1e-4 transmittance stop), written with
differentiable torch operations over a dense [pixels x primitives] grid so that autograd
gives d(loss)/d(parameters).  The discrete decisions (which primitives are culled, their
depth order) are taken from the C oracle's per-primitive pass and held fixed, as they are
piecewise constant in the parameters.  No anti-aliasing (MIP) term.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import raygs_oracle as _orc


def quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrices [N,3,3] of quaternions (w,x,y,z) [N,4] after normalisation."""
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=1)
    return R.view(-1, 3, 3)


def _legendre(l, m, t, st):
    pmm = torch.ones_like(t)
    for i in range(1, m + 1):
        pmm = pmm * (2.0 * i - 1.0) * st
    if l == m:
        return pmm
    pm1 = t * (2.0 * m + 1.0) * pmm
    if l == m + 1:
        return pm1
    pl = pm1
    for ll in range(m + 2, l + 1):
        pl = ((2.0 * ll - 1.0) * t * pm1 - (ll + m - 1.0) * pmm) / (ll - m)
        pmm, pm1 = pm1, pl
    return pl


def sh_basis(degree: int, d: torch.Tensor) -> torch.Tensor:
    """Real spherical harmonics without the Condon-Shortley phase, [N, (deg+1)^2], for unit
    directions d [N,3] (associated Legendre recurrence, as in the C oracle)."""
    t = d[:, 2].clamp(-1.0, 1.0)
    st = torch.sqrt(torch.clamp(1.0 - t * t, min=0.0) + 1e-300)
    phi = torch.atan2(d[:, 1], d[:, 0])
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            P = _legendre(l, am, t, st)
            if m == 0:
                out.append(K * P)
            elif m > 0:
                out.append(math.sqrt(2) * K * torch.cos(m * phi) * P)
            else:
                out.append(math.sqrt(2) * K * torch.sin(am * phi) * P)
    return torch.stack(out, dim=1)


def render_dense(params: dict, scene: dict, cam: dict, cfg: dict | None = None, pixels=None):
    """Differentiable FP64 render of one camera.

    params: dict of float64 torch tensors (requires_grad as wanted) with keys means [N,3],
    log_scales [N,3], quats [N,4], opacity_logits [N], sh [N,K,3].  scene: the numpy scene
    the parameters were taken from (for the C oracle's cull / order decisions).
    Returns (rgb [P,3], T [P]).
    """
    if cam.get("mip", False):
        raise ValueError("the dense reference has no anti-aliasing term")
    c = dict(_orc.DEFAULT_CFG)
    if cfg:
        c.update(cfg)
    info = _orc.prepare(scene, cam, cfg)
    valid = np.nonzero(info[:, 0] == 0)[0]
    keys = info[valid, 1].astype(np.uint64)
    order = valid[np.lexsort((valid, keys))]
    idx = torch.as_tensor(order, dtype=torch.long)
    dt = torch.float64
    Rwc = torch.as_tensor(np.asarray(cam["R"], np.float32).astype(np.float64), dtype=dt)
    twc = torch.as_tensor(np.asarray(cam["t"], np.float32).astype(np.float64), dtype=dt)
    mu_w = params["means"][idx]
    mu = mu_w @ Rwc.T + twc
    Rc = Rwc @ quat_to_rot(params["quats"][idx])
    s = torch.exp(params["log_scales"][idx])
    o = torch.sigmoid(params["opacity_logits"][idx])
    W = Rc.transpose(1, 2) / s[:, :, None]              # S^-1 R^T
    m = torch.einsum("nij,nj->ni", W, mu)
    c2 = (m * m).sum(1)
    kappa = -2.0 * torch.log(c["p_min"] / o)
    # colour
    C = -(Rwc.T @ twc)
    d = mu_w - C
    d = d / d.norm(dim=1, keepdim=True)
    deg = int(scene["sh_degree"])
    Y = sh_basis(deg, d)
    coef = params["sh"][idx]
    rgb = coef[:, 0, :] + torch.einsum("nk,nkc->nc", Y[:, 1:], coef[:, 1:, :])
    rgb = torch.clamp(rgb, min=0.0)
    # rays
    Wd, Hd = int(cam["width"]), int(cam["height"])
    if pixels is None:
        jj, ii = np.divmod(np.arange(Wd * Hd), Wd)
    else:
        pix = np.asarray(pixels).reshape(-1, 2)
        ii, jj = pix[:, 0], pix[:, 1]
    fx, fy = float(np.float32(cam["fx"])), float(np.float32(cam["fy"]))
    cx, cy = float(np.float32(cam["cx"])), float(np.float32(cam["cy"]))
    x = torch.stack([torch.as_tensor((ii + 0.5 - cx) / fx), torch.as_tensor((jj + 0.5 - cy) / fy),
                     torch.ones(len(ii), dtype=dt)], dim=1).to(dt)
    w = torch.einsum("nij,pj->pni", W, x)                 # whitened rays [P,N,3]
    num = (w * m[None]).sum(-1)
    den = (w * w).sum(-1)
    tau = num / den
    r = tau[..., None] * w - m[None]
    D = (r * r).sum(-1)
    inside = ((tau > 0) & (D <= kappa[None])).to(dt)
    om = torch.clamp(o[None] * torch.exp(-0.5 * D), max=c["alpha_max"]) * inside
    one_m = 1.0 - om
    Tpre = torch.cumprod(torch.cat([torch.ones(len(ii), 1, dtype=dt), one_m[:, :-1]], dim=1), dim=1)
    stop = ((Tpre * one_m < c["t_stop"]) & (inside > 0)).detach()
    excluded = (torch.cumsum(stop.to(torch.int64), dim=1) > 0).to(dt)
    wgt = om * Tpre * (1.0 - excluded)
    out_rgb = wgt @ rgb
    T = torch.prod(1.0 - om * (1.0 - excluded), dim=1)
    return out_rgb, T


def params_from_scene(scene: dict, requires_grad=True) -> dict:
    out = {}
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        t = torch.as_tensor(np.asarray(scene[k], dtype=np.float32).astype(np.float64))
        out[k] = t.clone().requires_grad_(requires_grad)
    return out

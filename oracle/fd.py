"""Central finite differences of an image loss through the FP64 C oracle.

TEST INFRASTRUCTURE ONLY.  A parameter element is moved by +-h in the float32 scene; the
quotient uses the exact float32 difference of the two moved values.  A difference is
reported as undefined (None) when the set of composited primitives of any pixel changes
between the two renders (the oracle's per-pixel decision signature differs): the loss is
then discontinuous inside [x-h, x+h] and no derivative exists there to compare with.
"""
from __future__ import annotations

import numpy as np

from . import raygs_oracle as _orc


def l1_loss(rgb: np.ndarray, target: np.ndarray) -> float:
    return float(np.abs(rgb - target).sum())


def central_difference(scene: dict, cam: dict, target: np.ndarray, key: str, index: tuple,
                       h: float, cfg: dict | None = None, threads: int = 0):
    """d(L1 loss)/d(scene[key][index]) by central differences, or None."""
    arr = scene[key]
    x0 = np.float32(arr[index])
    xp, xm = np.float32(x0 + np.float32(h)), np.float32(x0 - np.float32(h))
    outs = []
    for xv in (xp, xm):
        s2 = dict(scene)
        a2 = np.array(arr, dtype=np.float32, copy=True)
        a2[index] = xv
        s2[key] = a2
        outs.append(_orc.render(s2, cam, cfg, threads=threads))
    if not np.array_equal(outs[0]["sig"], outs[1]["sig"]) or \
            not np.array_equal(outs[0]["ncontrib"], outs[1]["ncontrib"]):
        return None
    lp, lm = l1_loss(outs[0]["rgb"], target), l1_loss(outs[1]["rgb"], target)
    return (lp - lm) / (float(xp) - float(xm))

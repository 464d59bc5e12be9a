"""Writes the stored expected values under tests/golden/ from the FP64 oracle alone.

    python -m tests.golden.make_golden

small_uniform_64x64.txt: the 1,000-primitive 64x64 scene (uniform generator, seed 0;
SH degree 0) rendered by the oracle (Eq. rendering with Eq. Q_ray and Eq. rend_opacity,
Sec. 3) at 256 pixels sampled with seed 7.  One line per pixel: column, row, R, G, B,
final transmittance, oracle flag (1 when some primitive's opacity lies within 1e-6 of
the cut-off).  Nothing here calls the CUDA library.
"""
import os

import numpy as np

import oracle
from paper_2503_18682_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


def small_pixels():
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(64 * 64, size=256, replace=False))
    return np.stack([idx % 64, idx // 64], axis=1).astype(np.int32), idx


def main():
    scene, cams = scenes.workload_small()
    pix, _ = small_pixels()
    out = oracle.render(scene, cams[0], pixels=pix)
    path = os.path.join(HERE, "small_uniform_64x64.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle, uniform scene (1000 primitives, seed 0), 64x64 view fx=fy=64 cx=cy=32\n")
        f.write("# Eq. rendering / Eq. Q_ray / Eq. rend_opacity (Sec. 3); written by make_golden.py\n")
        f.write("# col row R G B T flag\n")
        for (c, r), rgb, T, fl in zip(pix, out["rgb"], out["T"], out["flags"]):
            f.write(f"{c} {r} {rgb[0]:.17g} {rgb[1]:.17g} {rgb[2]:.17g} {T:.17g} {int(fl)}\n")
    print(path)


if __name__ == "__main__":
    main()

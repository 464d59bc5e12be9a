"""FP64 CPU oracle for the RayGS hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
leg may import this package.  The CUDA library never calls it; the two share no code.

``raygs_oracle.c`` holds the arithmetic (the plain definition, brute force over every
pixel and primitive); ``ref_torch.py`` holds a dense PyTorch-CPU FP64 restatement of the
same image used only to obtain reference gradients by autograd.  ``build()`` compiles the
C file with gcc (-O2 -fopenmp -ffp-contract=off).
"""
from .raygs_oracle import (  # noqa: F401
    build, lib, cam_array, cfg_array, prepare, render, quad, rot_align, D_ray, support_mask, sh_basis,
    quat_to_rot, depth_key, DEFAULT_CFG, OG,
)

"""GB300-native (sm_103a) renderer for ray-based Gaussian splatting (RayGS).

The compute path is a C-ABI CUDA library (``csrc/``, declared in ``include/raygs.h``);
``raygs`` is its thin Python binding.  Importing this package loads nothing: the library is
opened on first use and every entry point raises if it is missing.
"""
__all__ = ["raygs", "scenes"]

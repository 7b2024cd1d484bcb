"""GB300-native long-characteristics 3D radiative transfer (formal solution,
Lambda* band and ALI), after Hauschildt & Baron, arXiv:2102.01734.

The CUDA library is loaded lazily by ``paper_2102_01734_gb300.rt3d``.
"""
__all__ = ["inputs", "rt3d"]

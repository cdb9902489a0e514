"""GB300-native forward semi-Lagrangian advection step (arXiv:1410.2817).

The CUDA library is loaded on first use by ``paper_1410_2817_gb300.sl``; importing the package
itself loads nothing, so the input generators can be used without a GPU.
"""
__all__ = ["inputs", "sl"]

"""B300-native PIV image-pair renderer (SynthPix, arXiv 2512.09664).

The CUDA library is loaded lazily by :mod:`paper_2512_09664_b300.binding`;
importing this package (for instance for the synthetic workloads) does not
need a GPU.
"""
__all__ = ["workloads"]

"""GB300-native particle-side step of the coarse-grained CFD-DEM-IBM method for hydrogen
reduction of iron ore (Lan et al., arXiv 2311.03908).

The compute path is libdem_gb300.so (hand-written CUDA for sm_103a) behind the C ABI of
include/dem.h; ``binding`` exposes it to Python under the same names, ``synth`` builds
seeded synthetic beds, ``autograd`` wraps the adjoint as a torch.autograd.Function.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "binding", "build"]

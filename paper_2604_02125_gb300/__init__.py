"""GB300-native (sm_103a) cRKFR hot path: one compact Runge-Kutta flux
reconstruction step with entropy-conservative / kinetic-energy-preserving flux
differencing (arXiv 2604.02125), behind a small C-ABI library; the same
kernels also run the multi-stage RKFR scheme the method is derived from and,
for GLM-MHD, the stage-wise non-conservative flux.

The CUDA library is loaded lazily by :mod:`paper_2604_02125_gb300.crkfr`; there
is no CPU fallback: creating a solver without the compiled library raises.
"""
__all__ = ["inputs"]

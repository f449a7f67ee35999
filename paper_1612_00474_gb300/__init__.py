"""GB300-native (sm_103a) Rotne-Prager-Blake Brownian dynamics: the all-pairs wall-corrected RPY
product, Lanczos M^{1/2} W, RFD drift and the stochastic Adams-Bashforth step, as hand-written
CUDA behind a C ABI (include/rpb.h).

Modules: rpb (binding of the C ABI), build (nvcc build of librpb.so), inputs (seeded synthetic
configurations).  Importing the package does not load the CUDA library; rpb.load() does.
"""
__all__ = ["rpb", "build", "inputs"]

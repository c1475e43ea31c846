"""GB300-native even-odd clover-Wilson operator, CG solver and fermion force.

``synth`` draws the seeded synthetic inputs; ``qcd`` is the binding to the CUDA
library ``libqcd.so`` (C ABI in ``include/qcd.h``), loaded on first use.
"""

"""GB300-native Local Naive Bayes Nearest Neighbor (McCann & Lowe).

``lnbnn`` is the binding of the CUDA library (include/lnbnn.h); ``synth`` the
seeded synthetic workloads; ``build`` compiles the library for sm_103a.
"""
__all__ = ["lnbnn", "synth", "build"]

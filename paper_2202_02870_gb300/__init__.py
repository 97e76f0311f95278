"""GB300-native (sm_103a) generalized *_L-product tensor completion.

The compute path is liblt.so (include/lt.h), hand-written CUDA kernels built in-tree by
`paper_2202_02870_gb300.build`; `paper_2202_02870_gb300.lt` is its Python binding and
`paper_2202_02870_gb300.synth` the seeded synthetic-input generators.
"""
__all__ = ["lt", "synth", "build"]

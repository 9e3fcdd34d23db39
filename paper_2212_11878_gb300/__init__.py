"""GB300-native stochastic rotation dynamics (SRD / MPCD) time step.

The compute path is the C-ABI library ``libmpcd.so`` (hand-written CUDA for sm_103a); the
Python side only marshals arguments.  Import :mod:`paper_2212_11878_gb300.abi` for the
binding; importing this package itself loads nothing.
"""
__all__ = ["abi", "inputs"]

"""GB300-native real-space PAW eigensolver step (finite-difference H and S, Rayleigh-Ritz).

Importing the package is cheap: the CUDA library is loaded on first use by
``paper_2310_14776_gb300.api``; ``synth`` only makes seeded inputs.
"""
__all__ = ["synth"]

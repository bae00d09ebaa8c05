"""GB300-native sliding-window bundle adjustment (Levenberg-Marquardt step).

Importing the package is cheap; the CUDA library is loaded on first use of the
binding (`paper_2506_04359_gb300.cvba`).
"""
__all__ = ["synth"]

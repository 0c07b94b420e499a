"""GB300-native MB4 integrator for the 2D-grid nonlinear Schroedinger-type system.

The compute path is the C-ABI library ``libmb4`` (hand-written CUDA for
sm_103a); ``paper_2003_04345_gb300.mb4`` is its thin ctypes binding and
``paper_2003_04345_gb300.inputs`` makes seeded synthetic inputs.  Importing the
package does not load the library; ``mb4`` loads it on first use and raises if
it has not been built.
"""
__all__ = ["inputs", "mb4"]

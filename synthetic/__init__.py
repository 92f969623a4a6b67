"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

Only input construction lives here: noise, injected signals and the chirp
parameter grids of the workloads.  None of the matched-filter arithmetic (FFT
correlation, Parseval sigma, thresholding) is in this package.
"""
from .inputs import *  # noqa: F401,F403

"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This package draws images only: it holds none of the method's arithmetic
(no colour conversion, no grid, no Gaussian), so both the CUDA path and the
oracle may be fed from it.
"""
from .voronoi import voronoi_image, batch_sizes, CONFIGS  # noqa: F401

"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random arrays and nothing else: it holds none of the Wilson
operator's arithmetic (no gamma matrices, no hopping, no parity arithmetic), so
both sides of a parity comparison can take their inputs from it without sharing
any of the method's code.
"""

from .fields import (  # noqa: F401
    rng,
    complex_gaussian,
    haar_su3,
    smooth_su3,
    gauge_field,
    gaussian_spinor,
    point_sources,
    random_gauge_transform,
    volume,
)

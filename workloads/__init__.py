"""Seeded synthetic inputs shaped like SISSO l0-regularization workloads.

This package only draws numbers: primary features, candidate feature columns
built as products of powers of primaries, planted targets and noise.  It holds
none of the l0 method's arithmetic (no centring, no least squares, no
ranking), so both the CPU oracle and the CUDA path can consume its arrays.
"""

from .synth import (  # noqa: F401
    EXPONENTS,
    Problem,
    make_config,
    make_problem,
    CONFIGS,
)

"""Seeded synthetic Hamiltonians shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and assembles input matrices. It holds none of
the method's arithmetic (no bounds, no Chebyshev coefficients, no expansion), so both
the CUDA path and the CPU oracle can be fed from it without sharing any of the method.
"""
from .hamiltonians import (  # noqa: F401
    random_symmetric,
    tight_binding,
    metallic,
    metallic_electrons,
    METALLIC_FILLING,
    batch_sizes,
    batch_temperatures,
    tight_binding_box,
)

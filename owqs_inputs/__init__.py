"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Holds the pattern data model, the J/CZ circuit-to-pattern generator, the
workload definitions and the splitmix64 stream.  It contains none of the
simulation arithmetic.
"""
from .patterns import Cmd, Pattern, N, E, M, X, Z, circuit_to_pattern  # noqa: F401
from .rng import SplitMix64, pattern_rng, random_state  # noqa: F401

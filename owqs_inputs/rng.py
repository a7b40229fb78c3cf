"""Seeded random numbers for the synthetic workloads.

The generator is splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the state advances by the
64-bit golden-ratio increment and each output is the state passed through the
published three-step xor-shift-multiply finaliser.  Uniform doubles take the
top 53 bits.  Complex normals use the Box-Muller transform.

Both the oracle and the CUDA path draw their inputs from here, so the two
sides always see the same patterns, angles, input states and forced outcome
bits.  Nothing in this module simulates a pattern.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
MUL1 = 0xBF58476D1CE4E5B9
MUL2 = 0x94D049BB133111EB

# Workload seeds: config c uses BASE_SEED + c; pattern i of a config uses
# splitmix64 seeded with (config seed XOR i).
BASE_SEED = 1604056590


def mix64(z: int) -> int:
    """The splitmix64 output finaliser on one 64-bit integer."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MUL1) & MASK64
    z = ((z ^ (z >> 27)) * MUL2) & MASK64
    return z ^ (z >> 31)


def mix64_array(z: np.ndarray) -> np.ndarray:
    """Vectorised finaliser; numpy uint64 arithmetic wraps modulo 2^64."""
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= np.uint64(MUL1)
    z ^= z >> np.uint64(27)
    z *= np.uint64(MUL2)
    z ^= z >> np.uint64(31)
    return z


class SplitMix64:
    """Sequential splitmix64 stream."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        return mix64(self.state)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, n: int) -> int:
        """Integer in [0, n) by multiply-shift of a 53-bit uniform."""
        if n <= 0:
            raise ValueError("randint needs n > 0")
        return min(int(self.uniform() * n), n - 1)

    def bits(self, count: int) -> np.ndarray:
        """`count` independent outcome bits (top bit of each output)."""
        return np.array([self.next_u64() >> 63 for _ in range(count)], dtype=np.uint8)

    def u64_block(self, count: int) -> np.ndarray:
        """The next `count` outputs of the stream, vectorised."""
        idx = np.arange(1, count + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            states = np.uint64(self.state) + idx * np.uint64(GOLDEN)
        self.state = (self.state + count * GOLDEN) & MASK64
        return mix64_array(states)

    def uniform_block(self, count: int) -> np.ndarray:
        return (self.u64_block(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def complex_normal(self, count: int) -> np.ndarray:
        """`count` complex N(0,1) values (Box-Muller on pairs of uniforms)."""
        u = self.uniform_block(2 * count).reshape(count, 2)
        r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))       # 1-u in (0,1]
        phi = 2.0 * math.pi * u[:, 1]
        return r * np.cos(phi) + 1j * r * np.sin(phi)


def config_seed(config_index: int) -> int:
    return BASE_SEED + config_index


def pattern_rng(config_index: int, pattern_index: int = 0) -> SplitMix64:
    return SplitMix64(config_seed(config_index) ^ pattern_index)


def random_state(rng: SplitMix64, nqubits: int) -> np.ndarray:
    """Normalised complex128 vector of 2^nqubits N(0,1) amplitudes."""
    v = rng.complex_normal(1 << nqubits)
    return v / np.linalg.norm(v)

"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the fermionic method: it only draws random
numbers, random permutations and graph structures (lattices, contraction
trees).  Both the CPU oracle and the CUDA path consume what it produces, and
neither side's arithmetic lives here.
"""
from .gen import *  # noqa: F401,F403
from .lattice import *  # noqa: F401,F403
from .peps import *  # noqa: F401,F403

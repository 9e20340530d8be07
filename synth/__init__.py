"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package holds no arithmetic of the robust-control method itself (no gate
exponentials, no TEBD, no overlaps, no gradients): only the seeded random
controls, random product states, the closed-form target states of the paper
(parallel X, parallel CNOT, GHZ of Sec. IV) and the Heisenberg ground-state
target, plus the MPS container used to pass states across the C ABI.
"""
from .inputs import *  # noqa: F401,F403

"""Noise realisations of the parasitic ZZ strengths (Sec. II: J_j iid
uniform on [-dJ, dJ]; the normal variant N(0, sigma^2) is the second
distribution the library offers).

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-based: the i-th output of the
stream seeded with ``seed`` is  mix(seed + (i + 1) * 0x9E3779B97F4A7C15)  with
the published finaliser ``mix``.  Written here with Python integers.

Draw for sample s, bond b (i = s * (N - 1) + b; with three crosstalk terms per
bond, i = 3 (s * (N - 1) + b) + c for term c = x, y, z):
  uniform: u = (out(i) >> 11) * 2^-53 in [0, 1);  J = scale * (2u - 1)
  normal:  u1 = ((out(2i) >> 11) + 1) * 2^-53 in (0, 1],
           u2 = (out(2i + 1) >> 11) * 2^-53,
           J  = scale * sqrt(-2 ln u1) * cos(2 pi u2)      (Box-Muller)
"""
import math

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, i: int) -> int:
    """The i-th (0-based) output of SplitMix64 started from ``seed``."""
    z = (seed + (i + 1) * _GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def sample_J(seed: int, M: int, N: int, dist: int, scale: float, terms: int = 1) -> np.ndarray:
    """J[M][N-1] float64 (ZZ crosstalk), or J[M][N-1][3] = (J^x, J^y, J^z) per
    bond for the Heisenberg-type crosstalk of Eq. Hp (terms = 3); draw
    (s, b, c) uses counter i = (s (N-1) + b) terms + c."""
    nb = N - 1
    J = np.zeros((M, nb * terms), dtype=np.float64)
    for s in range(M):
        for b in range(nb * terms):
            i = s * nb * terms + b
            if dist == 0:
                u = (splitmix64(seed, i) >> 11) * 2.0 ** -53
                J[s, b] = scale * (2.0 * u - 1.0)
            elif dist == 1:
                u1 = ((splitmix64(seed, 2 * i) >> 11) + 1) * 2.0 ** -53
                u2 = (splitmix64(seed, 2 * i + 1) >> 11) * 2.0 ** -53
                J[s, b] = scale * math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
            else:
                raise ValueError("dist must be 0 (uniform) or 1 (normal)")
    return J if terms == 1 else J.reshape(M, nb, terms)

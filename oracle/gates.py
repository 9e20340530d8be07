"""Two-site gates of the second-order TEBD slice (Sec. II, Eq. circuit, with
the Hamiltonian of Eq. sysH and the crosstalk of Eq. Hp).

Bond b couples sites b and b+1.  Its Hamiltonian in the basis
|s_b s_{b+1}> (index 2 s_b + s_{b+1}) is

  h_b = c_b Z(x)Z + J^x_b X(x)X + J^y_b Y(x)Y
        + wL (x_b X + y_b Y)(x)I + wR I(x)(x_{b+1} X + y_{b+1} Y)

with c_b = g_b + J^z_b (tunable plus parasitic ZZ; J^x = J^y = 0 for pure ZZ
crosstalk, all three for the Heisenberg-type crosstalk of Eq. Hp) and weights
wL = 1 if b is the first bond else 1/2, wR = 1 if b is the last bond else 1/2,
so that summing h_b over all bonds gives H of Eq. sysH.  The gate is the exact
4x4 exponential G = exp(-i tau h_b) through the Hermitian eigendecomposition
h_b = V diag(lam) V^dagger.
"""
import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def bond_weights(N: int, b: int):
    wl = 1.0 if b == 0 else 0.5
    wr = 1.0 if b + 1 == N - 1 else 0.5
    return wl, wr


def bond_hamiltonian(N, b, xl, yl, xr, yr, c, jx=0.0, jy=0.0):
    """h_b for left-site drives (xl, yl), right-site drives (xr, yr), ZZ
    coefficient c and the XX, YY crosstalk strengths jx, jy (Eq. Hp)."""
    wl, wr = bond_weights(N, b)
    return (c * np.kron(Z, Z) + jx * np.kron(X, X) + jy * np.kron(Y, Y)
            + wl * np.kron(xl * X + yl * Y, I2)
            + wr * np.kron(I2, xr * X + yr * Y))


def bond_generators(N, b):
    """dh_b / d(parameter) for the five parameters (xl, yl, xr, yr, c)."""
    wl, wr = bond_weights(N, b)
    return {
        "xl": wl * np.kron(X, I2), "yl": wl * np.kron(Y, I2),
        "xr": wr * np.kron(I2, X), "yr": wr * np.kron(I2, Y),
        "c": np.kron(Z, Z),
    }


def expm_hermitian(h, tau):
    """exp(-i tau h) for Hermitian h, and its eigendecomposition."""
    lam, V = np.linalg.eigh(h)
    G = (V * np.exp(-1j * tau * lam)) @ V.conj().T
    return G, lam, V


def dexpm_hermitian(lam, V, tau, P):
    """Frechet derivative of h -> exp(-i tau h) in direction P
    (Daleckii-Krein): V [ (V^dag P V) o Gamma ] V^dag with the divided
    differences Gamma_jk = (e^{-i tau lam_j} - e^{-i tau lam_k}) / (lam_j - lam_k)
    written in the form that stays finite at lam_j = lam_k:
        Gamma_jk = -i tau e^{-i tau (lam_j + lam_k)/2} sinc(tau (lam_j - lam_k)/2).
    """
    lj = lam[:, None]
    lk = lam[None, :]
    x = tau * (lj - lk) / 2.0
    sinc = np.where(np.abs(x) > 1e-30, np.sin(x) / np.where(x == 0, 1.0, x), 1.0)
    gamma = -1j * tau * np.exp(-1j * tau * (lj + lk) / 2.0) * sinc
    return V @ ((V.conj().T @ P @ V) * gamma) @ V.conj().T

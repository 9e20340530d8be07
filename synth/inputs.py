"""Seeded synthetic workloads for tensor-network robust control.

Every array here is drawn from ``numpy.random.default_rng(seed)`` (PCG64) or is
a closed form printed in the paper.  Nothing here evaluates the method: the
noise realisations J are drawn on each side from the counter-based SplitMix64
definition (Steele, Lea, Flood 2014), not here.

Conventions (shared by both sides of every parity test):
  * |0> = (1, 0) is the Z = +1 state; site 0 is the leftmost site.
  * An MPS site tensor has shape (D_left, 2, D_right); the boundary bonds are 1.
  * Controls are ``u[K][C][N]`` float64: slot 0 = x_i (X drive), slot 1 = y_i
    (Y drive), slot 2 (C = 3 only) = g_i, the tunable ZZ coupling on bond
    (i, i+1) (Eq. sysH).  ``mask[C][N]`` (uint8) marks which slots are
    controls; a masked slot does not enter the Hamiltonian.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "MPS", "Workload", "WORKLOADS", "controls", "pi_pulse_controls",
    "product_inputs", "zero_state", "x_targets", "cnot_targets", "ghz_mps",
    "heisenberg_ground_mps", "control_mask", "echo_controls", "make_problem", "identity_operator", "x_gate_operator",
    "cnot_gate_operator",
]


@dataclasses.dataclass
class MPS:
    """A matrix-product state: ``sites[i]`` has shape (D_{i-1}, d, D_i), d = 2
    for qubit states, d = 4 for operators written as vectors (site index
    s = 2 out + in)."""

    sites: List[np.ndarray]

    @property
    def n_sites(self) -> int:
        return len(self.sites)

    @property
    def bond_dims(self) -> np.ndarray:
        """Bond dimensions [N+1] with both ends equal to 1."""
        d = [self.sites[0].shape[0]] + [s.shape[2] for s in self.sites]
        return np.asarray(d, dtype=np.int32)

    def pack(self):
        """(bond_dims int32 [N+1], data complex128 flat, site-major, each site
        (D_l, d, D_r) row-major) -- the layout the C ABI takes."""
        data = np.concatenate([np.ascontiguousarray(s, dtype=np.complex128).ravel()
                               for s in self.sites])
        return self.bond_dims, data

    @staticmethod
    def unpack(bond_dims, data, d=2) -> "MPS":
        bond_dims = np.asarray(bond_dims, dtype=np.int64)
        data = np.asarray(data, dtype=np.complex128)
        sites, off = [], 0
        for i in range(len(bond_dims) - 1):
            dl, dr = int(bond_dims[i]), int(bond_dims[i + 1])
            sites.append(data[off:off + dl * d * dr].reshape(dl, d, dr).copy())
            off += dl * d * dr
        return MPS(sites)

    def copy(self) -> "MPS":
        return MPS([s.copy() for s in self.sites])


# --------------------------------------------------------------------------
# controls
# --------------------------------------------------------------------------

def controls(K: int, C: int, N: int, seed: int, sigma: float = 0.5) -> np.ndarray:
    """Piecewise-constant control amplitudes u[K][C][N] ~ N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, size=(K, C, N)).astype(np.float64)


def pi_pulse_controls(K: int, C: int, N: int, dt: float, seed: Optional[int] = None,
                      jitter: float = 0.0) -> np.ndarray:
    """Constant resonant pi pulse on X (x = pi / (2 T), T = K dt), optionally
    plus N(0, jitter^2) on every slot (the "near-solution" controls)."""
    u = np.zeros((K, C, N), dtype=np.float64)
    u[:, 0, :] = math.pi / (2.0 * K * dt)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        u += rng.normal(0.0, jitter, size=u.shape)
    return u


def echo_controls(K: int, C: int, N: int, seed: int, sigma: float) -> np.ndarray:
    """u[k] ~ N(0, sigma^2) for k < K/2 and u[K-1-k] = -u[k] for the second
    half (K even): a time-reversed, negated copy.  At zero crosstalk the
    symmetric splitting then undoes the first half exactly, so the state
    entangles up to mid-time and disentangles again; the middle bonds can
    reach the cap while the final overlap with the input stays O(1)."""
    if K % 2:
        raise ValueError("echo controls need an even number of slices")
    rng = np.random.default_rng(seed)
    h = rng.normal(0.0, sigma, size=(K // 2, C, N))
    return np.concatenate([h, -h[::-1]]).astype(np.float64)


def control_mask(C: int, N: int, g_bonds: str = "none") -> np.ndarray:
    """mask[C][N] uint8.  x and y are controls on every site.  For C = 3 the g
    slot i (bond (i, i+1)) is a control on ``g_bonds``: "all" bonds, "pairs"
    (bonds (2j, 2j+1) only: the parallel-CNOT layout), or "none".  The g slot
    of the last site never is (it has no bond)."""
    m = np.ones((C, N), dtype=np.uint8)
    if C == 3:
        m[2, :] = 0
        if g_bonds == "all":
            m[2, : N - 1] = 1
        elif g_bonds == "pairs":
            m[2, 0 : N - 1 : 2] = 1
        elif g_bonds != "none":
            raise ValueError(g_bonds)
    return m


# --------------------------------------------------------------------------
# states
# --------------------------------------------------------------------------

def _product(vecs: Sequence[np.ndarray]) -> MPS:
    return MPS([np.asarray(v, dtype=np.complex128).reshape(1, 2, 1).copy() for v in vecs])


def product_inputs(N: int, P: int, seed: int) -> List[MPS]:
    """P random product states; each site is a normalised complex Gaussian
    2-vector (uniform on the Bloch sphere)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(P):
        z = rng.normal(size=(N, 2)) + 1j * rng.normal(size=(N, 2))
        z /= np.linalg.norm(z, axis=1, keepdims=True)
        out.append(_product(list(z)))
    return out


def zero_state(N: int) -> MPS:
    """|0...0>, bond dimension 1 (Sec. IV: A_0 = 1, A_1 = 0)."""
    return _product([np.array([1.0, 0.0])] * N)


def x_targets(inputs: Sequence[MPS]) -> List[MPS]:
    """(prod_j X_j)|in> for product inputs: X swaps the two components."""
    out = []
    for mps in inputs:
        if any(s.shape != (1, 2, 1) for s in mps.sites):
            raise ValueError("x_targets expects product states")
        out.append(MPS([s[:, ::-1, :].copy() for s in mps.sites]))
    return out


def cnot_targets(inputs: Sequence[MPS]) -> List[MPS]:
    """(prod_i CNOT_{2i -> 2i+1})|in> for product inputs, as an exact MPS with
    bond 2 inside each pair and bond 1 between pairs (control = site 2i,
    the 0-indexed form of the paper's CNOT_{2j-1,2j}).  N must be even."""
    out = []
    for mps in inputs:
        N = mps.n_sites
        if N % 2:
            raise ValueError("parallel CNOT needs an even chain")
        sites = []
        for i in range(0, N, 2):
            c = mps.sites[i].reshape(2)
            t = mps.sites[i + 1].reshape(2)
            a = np.zeros((1, 2, 2), dtype=np.complex128)
            a[0, 0, 0] = c[0]          # control |0>: target unchanged
            a[0, 1, 1] = c[1]          # control |1>: target flipped
            b = np.zeros((2, 2, 1), dtype=np.complex128)
            b[0, :, 0] = t
            b[1, :, 0] = t[::-1]
            sites += [a, b]
        out.append(MPS(sites))
    return out


def ghz_mps(N: int) -> MPS:
    """The GHZ state (|0..0> + |1..1>)/sqrt(2) in the bond-2 MPS of Sec. IV.
    The first-site matrices are row vectors (the printed column separator is
    lost; the first site of an MPS is a row vector, Sec. II)."""
    if N < 2:
        raise ValueError("GHZ needs N >= 2")
    r = 2.0 ** -0.5
    first = np.zeros((1, 2, 2), dtype=np.complex128)
    first[0, 0, :] = [r, 0.0]
    first[0, 1, :] = [0.0, r]
    mid = np.zeros((2, 2, 2), dtype=np.complex128)
    mid[:, 0, :] = [[1.0, 0.0], [0.0, 0.0]]
    mid[:, 1, :] = [[0.0, 0.0], [0.0, 1.0]]
    last = np.zeros((2, 2, 1), dtype=np.complex128)
    last[:, 0, 0] = [1.0, 0.0]
    last[:, 1, 0] = [0.0, 1.0]
    return MPS([first] + [mid.copy() for _ in range(N - 2)] + [last])


# --------------------------------------------------------------------------
# operators as vectors (d = 4, site index s = 2 out + in), normalised so that
# <<A|B>> = tr(A^dag B) / 2^N
# --------------------------------------------------------------------------

def _vec(op2):
    return np.asarray(op2, dtype=np.complex128).reshape(4)


def identity_operator(N: int) -> MPS:
    """The identity on N qubits: the initial operator U(0) of the MPO evolution."""
    v = _vec(np.eye(2)) / np.sqrt(2.0)
    return MPS([v.reshape(1, 4, 1).copy() for _ in range(N)])


def x_gate_operator(N: int) -> MPS:
    """X on every qubit (the parallel-X gate target)."""
    v = _vec([[0, 1], [1, 0]]) / np.sqrt(2.0)
    return MPS([v.reshape(1, 4, 1).copy() for _ in range(N)])


def cnot_gate_operator(N: int) -> MPS:
    """CNOT on every pair (2i, 2i+1), control 2i: |0><0| (x) I + |1><1| (x) X,
    operator bond dimension 2 inside a pair."""
    if N % 2:
        raise ValueError("parallel CNOT needs an even chain")
    P0 = _vec([[1, 0], [0, 0]])
    P1 = _vec([[0, 0], [0, 1]])
    I2 = _vec(np.eye(2))
    X2 = _vec([[0, 1], [1, 0]])
    sites = []
    for _ in range(N // 2):
        a = np.zeros((1, 4, 2), dtype=np.complex128)
        a[0, :, 0] = P0 / np.sqrt(2.0)
        a[0, :, 1] = P1 / np.sqrt(2.0)
        b = np.zeros((2, 4, 1), dtype=np.complex128)
        b[0, :, 0] = I2 / np.sqrt(2.0)
        b[1, :, 0] = X2 / np.sqrt(2.0)
        sites += [a, b]
    return MPS(sites)


def heisenberg_ground_mps(N: int, d_max: int, tol: float = 1e-12):
    """Ground state of H_T = sum_j (XX + YY + ZZ)_{j,j+1} (open chain, Sec. IV)
    by Lanczos (scipy ``eigsh``), then cut into an MPS by successive SVDs
    keeping at most ``d_max`` values per bond and renormalised.

    Returns (mps, E0, psi_dense) with psi indexed by the bit string, site 0
    the most significant bit.
    """
    import scipy.sparse.linalg as sla

    dim = 1 << N
    idx = np.arange(dim, dtype=np.int64)
    diag = np.zeros(dim)
    flips = []
    for b in range(N - 1):
        sb = (idx >> (N - 1 - b)) & 1
        sc = (idx >> (N - 2 - b)) & 1
        diag += np.where(sb == sc, 1.0, -1.0)               # Z_b Z_{b+1}
        mask = (1 << (N - 1 - b)) | (1 << (N - 2 - b))
        anti = sb != sc
        flips.append((anti, idx ^ mask))                    # XX + YY = 2 (|01><10| + h.c.)

    def matvec(v):
        v = np.asarray(v).ravel()
        out = diag * v
        for anti, partner in flips:
            out = out + np.where(anti, 2.0 * v[partner], 0.0)
        return out

    op = sla.LinearOperator((dim, dim), matvec=matvec, dtype=np.float64)
    if dim <= 64:
        h = np.column_stack([matvec(np.eye(dim)[:, j]) for j in range(dim)])
        w, v = np.linalg.eigh(h)
        e0, psi = float(w[0]), v[:, 0]
    else:
        rng = np.random.default_rng(7)
        w, v = sla.eigsh(op, k=1, which="SA", tol=tol, v0=rng.normal(size=dim),
                         ncv=min(dim - 1, 40), maxiter=20000)
        e0, psi = float(w[0]), v[:, 0]
    psi = psi / np.linalg.norm(psi)
    # successive SVDs, left to right
    sites, rest, dl = [], psi.astype(np.complex128).reshape(1, dim), 1
    for i in range(N - 1):
        m = rest.reshape(dl * 2, -1)
        u, s, vh = np.linalg.svd(m, full_matrices=False)
        k = int(min(d_max, np.count_nonzero(s > tol * s[0])))
        k = max(k, 1)
        sites.append(u[:, :k].reshape(dl, 2, k))
        rest = (s[:k, None] * vh[:k]) / np.linalg.norm(s[:k])
        dl = k
    sites.append(rest.reshape(dl, 2, 1))
    return MPS(sites), e0, psi


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    """One problem instance: shapes, seeds and the distributions they feed."""

    name: str
    N: int
    chi: int
    K: int
    dt: float
    C: int
    M: int
    P: int
    noise_dist: int          # 0 = uniform U[-scale, scale], 1 = normal N(0, scale^2)
    noise_scale: float
    seed_u: int
    seed_J: int
    seed_in: int
    target: str              # "x", "cnot", "ghz", "heisenberg", "input" (target = input)
    g_bonds: str = "none"
    sv_cutoff: float = 1e-12
    u_sigma: float = 0.5
    crosstalk: int = 1       # 1: ZZ (J^z); 3: J^x XX + J^y YY + J^z ZZ (Eq. Hp)
    order: int = 2           # Trotter order: 2 (A B A) or 1 (the slice of Eq. circuit)
    substeps: int = 1        # Trotter steps per control bin
    operator: bool = False   # evolve the operator U (MPO, d = 4) from the identity;
                             # F = |tr(U_T^dag U) / 2^N|^2 (Eq. gateinfid)
    u_mode: str = "random"   # "random": u ~ N(0, u_sigma^2); "near": the pi pulse plus
                             # N(0, 0.05^2) (the near-solution controls); "echo": the first
                             # half N(0, u_sigma^2), the second half the first reversed in
                             # time and negated, so that at zero crosstalk the evolution
                             # returns to its input (pair with target "input")

    @property
    def trajectories(self) -> int:
        return self.M * self.P

    @property
    def slice_steps(self) -> int:
        """Slices of all trajectories in one call: the unit of the metric."""
        return self.M * self.P * self.K

    def controls(self) -> np.ndarray:
        if self.u_mode == "near":
            return pi_pulse_controls(self.K, self.C, self.N, self.dt, seed=self.seed_u, jitter=0.05)
        if self.u_mode == "echo":
            return echo_controls(self.K, self.C, self.N, self.seed_u, self.u_sigma)
        if self.u_mode != "random":
            raise ValueError(self.u_mode)
        return controls(self.K, self.C, self.N, self.seed_u, self.u_sigma)

    def mask(self) -> np.ndarray:
        return control_mask(self.C, self.N, self.g_bonds)

    def states(self):
        """(inputs[P], targets[P]) as MPS lists."""
        if self.operator:
            if self.target == "x":
                return [identity_operator(self.N)] * self.P, [x_gate_operator(self.N)] * self.P
            if self.target == "cnot":
                return [identity_operator(self.N)] * self.P, [cnot_gate_operator(self.N)] * self.P
            raise ValueError("operator targets: x or cnot")
        if self.target == "x":
            ins = product_inputs(self.N, self.P, self.seed_in)
            return ins, x_targets(ins)
        if self.target == "cnot":
            ins = product_inputs(self.N, self.P, self.seed_in)
            return ins, cnot_targets(ins)
        if self.target == "ghz":
            return [zero_state(self.N)] * self.P, [ghz_mps(self.N)] * self.P
        if self.target == "heisenberg":
            t, _, _ = heisenberg_ground_mps(self.N, min(20, self.chi))
            return [zero_state(self.N)] * self.P, [t] * self.P
        if self.target == "input":
            ins = [zero_state(self.N)] + product_inputs(self.N, self.P - 1, self.seed_in)
            return ins, [m.copy() for m in ins]
        raise ValueError(self.target)

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


#: The workload shapes: parallel X on 8 and 50 qubits, parallel CNOT on 50
#: (random and near-solution controls), GHZ on 30 (Sec. III-IV), an echo on 14
#: qubits whose bonds reach the cap, and the parallel-CNOT gate (operator form).
WORKLOADS = {
    "x8": Workload("x8", N=8, chi=16, K=20, dt=0.05, C=2, M=16, P=4,
                   noise_dist=0, noise_scale=0.05, seed_u=1, seed_J=2, seed_in=3,
                   target="x"),
    "x50": Workload("x50", N=50, chi=32, K=64, dt=0.05, C=2, M=128, P=8,
                    noise_dist=0, noise_scale=0.1, seed_u=11, seed_J=12, seed_in=13,
                    target="x"),
    "cnot50": Workload("cnot50", N=50, chi=64, K=100, dt=0.05, C=3, M=256, P=8,
                       noise_dist=1, noise_scale=0.05, seed_u=21, seed_J=22, seed_in=23,
                       target="cnot", g_bonds="pairs"),
    "ghz30": Workload("ghz30", N=30, chi=64, K=200, dt=0.05, C=3, M=512, P=1,
                      noise_dist=0, noise_scale=0.1, seed_u=31, seed_J=32, seed_in=33,
                      target="ghz", g_bonds="all"),
    # the benchmark shape with near-solution controls: the pi pulse plus N(0, 0.05^2)
    "cnot50near": Workload("cnot50near", N=50, chi=64, K=100, dt=0.05, C=3, M=256, P=8,
                           noise_dist=1, noise_scale=0.05, seed_u=21, seed_J=22, seed_in=23,
                           target="cnot", g_bonds="pairs", u_mode="near"),
    # bonds at the cap: a 14-qubit echo (random controls, then their time
    # reverse negated) entangles the middle bonds past chi = 64 (theta up to
    # 128 x 128), so the cap decides the cut, and returns towards the input
    "echo14": Workload("echo14", N=14, chi=64, K=16, dt=0.5, C=3, M=304, P=1,
                       noise_dist=0, noise_scale=0.1, seed_u=51, seed_J=52, seed_in=53,
                       target="input", g_bonds="all", u_sigma=1.5, u_mode="echo"),
    # the gate objective of Eq. gateinfid with the MPO of Sec. II (D_max = 20)
    "cnotgate50": Workload("cnotgate50", N=50, chi=20, K=100, dt=0.05, C=3, M=256, P=1,
                           noise_dist=1, noise_scale=0.05, seed_u=41, seed_J=42, seed_in=43,
                           target="cnot", g_bonds="pairs", operator=True),
}


def make_problem(w: Workload):
    """Everything one evaluation needs except the noise: a dict with the
    workload, controls u, mask, inputs and targets."""
    ins, tgs = w.states()
    return {"w": w, "u": w.controls(), "mask": w.mask(), "inputs": ins, "targets": tgs}

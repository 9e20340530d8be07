"""Ensemble-averaged fidelity and its costate gradient (Sec. II state form;
App. A), one trajectory (noise sample s, input p) at a time.

Time discretisation.  Slice k (k = 0..K-1) of length dt is the second-order
split A(dt/2) B(dt) A(dt/2): layer A applies exp(-i tau h_b) on every even
bond b, layer B on every odd bond, with h_b the bond Hamiltonian of
``oracle.gates`` built from slice k's controls.  One slice = one control bin.
The MPS is compressed after every time step (Sec. II): the half layer A(dt/2)
that ends slice k and the one that starts slice k+1 act on the same bonds with
nothing in between, so they are applied as one gate (their product) followed
by one truncated SVD.  The truncated layers are therefore
    A_0, B_0, A_0 A_1, B_1, A_1 A_2, ..., B_{K-1}, A_{K-1}   (2K + 1 layers).

Objective.  O_sp = <t_p | a_sp(T)>, F = (1/(M P)) sum_sp |O_sp|^2, the
fidelity whose complement is the ensemble-averaged state infidelity of Sec. II.

Gradient.  With layers l = 1..L (L = 3K), a_l the truncated state after layer
l and b_l = L_{l+1}^dag ... L_L^dag t (the costate, truncated by the same rule),
O = <b_l | L_l | a_{l-1}> for every l (App. A), so for a parameter u inside the
gate G of bond b in layer l:
    dO/du += <b_l | (dG/du) G^dagger | a_l>,
summed over every gate the parameter enters.  dF/du = (2/(MP)) sum Re(conj(O) dO/du).
Without truncation this is the exact derivative of the discrete map.
"""
import dataclasses
from typing import List, Optional

import numpy as np

from . import gates as _g
from . import mps as _m


@dataclasses.dataclass
class Problem:
    N: int
    K: int
    dt: float
    C: int
    chi: int
    u: np.ndarray                 # [K][C][N]
    mask: np.ndarray              # [C][N]
    J: np.ndarray                 # [M][N-1]
    inputs: list                  # P lists of site tensors
    targets: list
    g_fixed: Optional[np.ndarray] = None   # [K][N-1]
    eps: float = 1e-12

    @property
    def M(self):
        return self.J.shape[0]

    @property
    def P(self):
        return len(self.inputs)


def layers(K, dt):
    """[(k, parity, tau)] of the elementary gate layers in time order."""
    out = []
    for k in range(K):
        out += [(k, 0, dt / 2.0), (k, 1, dt), (k, 0, dt / 2.0)]
    return out


def merged_layers(K, dt):
    """[(parity, [(k, tau), ...])]: the truncated layers, each the product of
    the listed elementary layers (first in time first)."""
    out = [(0, [(0, dt / 2.0)])]
    for k in range(K):
        out.append((1, [(k, dt)]))
        if k + 1 < K:
            out.append((0, [(k, dt / 2.0), (k + 1, dt / 2.0)]))
    out.append((0, [(K - 1, dt / 2.0)]))
    return out


def bond_params(pb: Problem, s, k, b):
    """(xl, yl, xr, yr, c, jx, jy) of bond b in slice k for noise sample s; a
    masked control slot does not enter the Hamiltonian.  J[M][N-1] is ZZ
    crosstalk; J[M][N-1][3] = (J^x, J^y, J^z) the Heisenberg type (Eq. Hp)."""
    u, m = pb.u, pb.mask
    xl = u[k, 0, b] * m[0, b]
    yl = u[k, 1, b] * m[1, b]
    xr = u[k, 0, b + 1] * m[0, b + 1]
    yr = u[k, 1, b + 1] * m[1, b + 1]
    if pb.J.ndim == 3:
        jx, jy, c = pb.J[s, b]
    else:
        jx, jy, c = 0.0, 0.0, pb.J[s, b]
    if pb.C == 3:
        c += u[k, 2, b] * m[2, b]
    if pb.g_fixed is not None:
        c += pb.g_fixed[k, b]
    return xl, yl, xr, yr, c, jx, jy


def param_slots(pb: Problem, k, b):
    """[(name, (k, c, i))] of the controls the gate of bond b depends on."""
    m = pb.mask
    out = []
    for name, c, i in (("xl", 0, b), ("yl", 1, b), ("xr", 0, b + 1), ("yr", 1, b + 1)):
        if m[c, i]:
            out.append((name, (k, c, i)))
    if pb.C == 3 and m[2, b]:
        out.append(("c", (k, 2, b)))
    return out


def bond_gate(pb: Problem, s, k, b, tau):
    h = _g.bond_hamiltonian(pb.N, b, *bond_params(pb, s, k, b))
    return _g.expm_hermitian(h, tau)


def _layer_bonds(N, parity):
    return list(range(parity, N - 1, 2))


def trajectory(pb: Problem, s: int, p: int, want_grad: bool = True, stats=None):
    """(O_sp, dO_sp[K][C][N] or None) for noise sample s and input p."""
    N = pb.N
    B, lam = _m.canonicalize(pb.inputs[p], pb.chi, pb.eps)
    T, tlam = _m.canonicalize(pb.targets[p], pb.chi, pb.eps)
    sched = merged_layers(pb.K, pb.dt)
    gate_cache = []
    hist = [([x.copy() for x in B], [x.copy() for x in lam])] if want_grad else None
    for (par, group) in sched:
        gl = {}
        for b in _layer_bonds(N, par):
            parts = [(k, tau) + bond_gate(pb, s, k, b, tau) for (k, tau) in group]
            Mg = np.eye(4, dtype=np.complex128)
            for part in parts:
                Mg = part[2] @ Mg
            gl[b] = (Mg, parts)
            w, kk = _m.two_site_update(B, lam, b, Mg, pb.chi, pb.eps)
            if stats is not None:
                stats["discarded"] += w
                stats["dims"].append(kk)
        gate_cache.append(gl)
        if want_grad:
            hist.append(([x.copy() for x in B], [x.copy() for x in lam]))
    O = _m.overlap(T, B)
    if not want_grad:
        return O, None
    dO = np.zeros((pb.K, pb.C, N), dtype=np.complex128)
    cB, clam = [x.copy() for x in T], [x.copy() for x in tlam]
    for li in range(len(sched) - 1, -1, -1):
        par, group = sched[li]
        a_after = hist[li + 1][0]
        for b in _layer_bonds(N, par):
            Mg, parts = gate_cache[li][b]
            rho = _m.mixed_two_site_density(cB, a_after, b)
            gens = _g.bond_generators(N, b)
            # gate j of the product M = G_n ... G_1:  dO/du = tr(Q_j L^dag rho L),
            # Q_j = (dG_j/du) G_j^dag, L = G_n ... G_{j+1} (the gates after it)
            Lt = np.eye(4, dtype=np.complex128)
            for (k, tau, G, ev, V) in reversed(parts):
                r = Lt.conj().T @ rho @ Lt
                for name, idx in param_slots(pb, k, b):
                    dG = _g.dexpm_hermitian(ev, V, tau, gens[name])
                    Q = dG @ G.conj().T
                    dO[idx] += np.trace(Q @ r)
                Lt = Lt @ G
        for b in _layer_bonds(N, par):
            Mg = gate_cache[li][b][0]
            _m.two_site_update(cB, clam, b, Mg.conj().T, pb.chi, pb.eps)
    return O, dO


def ensemble(pb: Problem, want_grad: bool = True, pairs=None, stats=None):
    """(F, grad[K][C][N] or None, O[M][P]) averaged over all (s, p) (or over
    ``pairs`` when given, a sample of them)."""
    if pairs is None:
        pairs = [(s, p) for s in range(pb.M) for p in range(pb.P)]
    O = np.zeros((pb.M, pb.P), dtype=np.complex128)
    F = 0.0
    grad = np.zeros((pb.K, pb.C, pb.N)) if want_grad else None
    for s, p in pairs:
        o, do = trajectory(pb, s, p, want_grad, stats)
        O[s, p] = o
        F += abs(o) ** 2
        if want_grad:
            grad += 2.0 * np.real(np.conj(o) * do)
    n = len(pairs)
    return F / n, (grad / n if want_grad else None), O


def from_workload(prob: dict, J: np.ndarray, g_fixed=None) -> Problem:
    """Build a Problem from a ``synth.make_problem`` dict and a noise array."""
    w = prob["w"]
    return Problem(N=w.N, K=w.K, dt=w.dt, C=w.C, chi=w.chi, u=prob["u"], mask=prob["mask"],
                   J=J, inputs=[m.sites for m in prob["inputs"]],
                   targets=[m.sites for m in prob["targets"]], g_fixed=g_fixed,
                   eps=w.sv_cutoff)


def per_gate_infidelity(chi_bar: float, n: int, qubits_per_gate: int) -> float:
    """Sec. III reporting formula: 1 - (1 - chi_bar)^(q/n) for gates acting on
    q qubits each (q = 1: parallel X, q = 2: parallel CNOT)."""
    return 1.0 - (1.0 - chi_bar) ** (qubits_per_gate / n)

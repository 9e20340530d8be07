"""Ensemble-averaged fidelity and its costate gradient (Sec. II state form;
App. A), one trajectory (noise sample s, input p) at a time.

Time discretisation.  Control bin k (k = 0..K-1) of length dt holds the
controls u[k]; it is split into n_sub equal Trotter steps of length
dts = dt / n_sub (one step per bin unless stated otherwise).

Second order (the default): each step is A(dts/2) B(dts) A(dts/2): layer A
applies exp(-i tau h_b) on every even bond b, layer B on every odd bond, with
h_b the bond Hamiltonian of ``oracle.gates`` built from the bin's controls.
The MPS is compressed after every time step (Sec. II): the half layer A that
ends one step and the one that starts the next act on the same bonds with
nothing in between, so they are applied as one gate (their product) followed
by one truncated SVD.  With S = K n_sub steps the truncated layers are
    A_0, B_0, A_0 A_1, B_1, A_1 A_2, ..., B_{S-1}, A_{S-1}   (2S + 1 layers).

First order (Eq. circuit): each step applies, right to left,
exp(-i dts V_b) on every bond (V_b = c_b ZZ + J^x XX + J^y YY, odd bonds
first, then even bonds), then exp(-i dts y_j Y_j) on every site, then
exp(-i dts x_j X_j) on every site.  Single-site gates do not change the
Schmidt values, so each site's two rotations are folded into the one bond
gate of the step that touches it last: the even bond (j or j-1) for every
site of an even chain, and for an odd chain the last site goes with the odd
bond N-2.  Truncated layers: (odd V), (even V with folded rotations), per
step (2S layers).

Objective.  O_sp = <t_p | a_sp(T)>, F = (1/(M P)) sum_sp |O_sp|^2, the
fidelity whose complement is the ensemble-averaged state infidelity of Sec. II.

Operator form (Sec. II: the propagator itself as an MPO, starting from the
identity, compressed by the same truncated SVD; Eq. gateinfid).  An operator
A on N qubits is the vector with site index s = 2 out + in (physical
dimension 4), scaled so that <<A|B>> = tr(A^dag B) / 2^N; a gate G acts on
the out indices only, G (x) I_in, and the same algebra then gives
O = tr(U_T^dag U) / 2^N and F = |O|^2 averaged over the ensemble -- one minus
the gate infidelity of Eq. gateinfid -- and its gradient, with every 4x4
gate or Q embedded as G (x) I on the two sites' (out, in) pairs.

Gradient.  With truncated layers l = 1..L, a_l the truncated state after layer
l and b_l = L_{l+1}^dag ... L_L^dag t (the costate, truncated by the same rule),
O = <b_l | L_l | a_{l-1}> for every l (App. A), so for a parameter u inside the
factor G_f of the gate of bond b in layer l (gate = G_n ... G_1):
    dO/du += <b_l | L_f (dG_f/du) G_f^dagger L_f^dagger | a_l>,  L_f = G_n ... G_{f+1},
summed over every factor the parameter enters.  dF/du = (2/(MP)) sum Re(conj(O) dO/du).
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
    order: int = 2                # Trotter order: 2 (A B A) or 1 (Eq. circuit)
    substeps: int = 1             # Trotter steps per control bin
    operator: bool = False        # inputs/targets are operators as vectors (d = 4)

    @property
    def M(self):
        return self.J.shape[0]

    @property
    def P(self):
        return len(self.inputs)


def layers(K, dt, substeps=1):
    """[(k, parity, tau)] of the elementary gate layers of the second-order
    split in time order (bin k, Trotter step of length dt / substeps)."""
    out = []
    dts = dt / substeps
    for k in range(K):
        for _ in range(substeps):
            out += [(k, 0, dts / 2.0), (k, 1, dts), (k, 0, dts / 2.0)]
    return out


def merged_layers(K, dt, substeps=1):
    """[(parity, [(k, tau), ...])]: the truncated layers of the second-order
    split, each the product of the listed elementary layers (first in time
    first)."""
    S = K * substeps
    dts = dt / substeps
    out = [(0, [(0, dts / 2.0)])]
    for st in range(S):
        k = st // substeps
        out.append((1, [(k, dts)]))
        if st + 1 < S:
            out.append((0, [(k, dts / 2.0), ((st + 1) // substeps, dts / 2.0)]))
    out.append((0, [(K - 1, dts / 2.0)]))
    return out


def schedule(pb: "Problem"):
    """[(parity, factors)] of the truncated layers; ``factors(b)`` lists the
    (kind, k, tau) factors of bond b's gate, first in time first.  Kinds:
    "bond" = exp(-i tau h_b) with h_b of ``oracle.gates``; "V" = the
    interaction c ZZ + J^x XX + J^y YY alone; "xl", "yl", "xr", "yr" = the
    rotation exp(-i tau x X) (or y Y) of the bond's left or right site."""
    if pb.order == 2:
        return [(par, (lambda b, g=group: [("bond", k, tau) for (k, tau) in g]))
                for (par, group) in merged_layers(pb.K, pb.dt, pb.substeps)]
    if pb.order != 1:
        raise ValueError("order must be 1 or 2")
    N = pb.N
    dts = pb.dt / pb.substeps
    out = []
    for st in range(pb.K * pb.substeps):
        k = st // pb.substeps

        def odd(b, k=k):
            f = [("V", k, dts)]
            if N % 2 == 1 and b == N - 2:   # the last site of an odd chain
                f += [("yr", k, dts), ("xr", k, dts)]
            return f

        def even(b, k=k):
            return [("V", k, dts), ("yl", k, dts), ("yr", k, dts), ("xl", k, dts), ("xr", k, dts)]

        out.append((1, odd))
        out.append((0, even))
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


_SINGLE = {"xl": (0, 0, "X"), "yl": (1, 0, "Y"), "xr": (0, 1, "X"), "yr": (1, 1, "Y")}


def factor_hamiltonian(pb: Problem, s, b, kind, k):
    """4x4 Hermitian h of one factor exp(-i tau h) of bond b's gate (see
    ``schedule``)."""
    if kind == "bond":
        return _g.bond_hamiltonian(pb.N, b, *bond_params(pb, s, k, b))
    xl, yl, xr, yr, c, jx, jy = bond_params(pb, s, k, b)
    if kind == "V":
        return c * np.kron(_g.Z, _g.Z) + jx * np.kron(_g.X, _g.X) + jy * np.kron(_g.Y, _g.Y)
    amp = {"xl": xl, "yl": yl, "xr": xr, "yr": yr}[kind]
    return amp * factor_generator(kind)


def factor_generator(kind):
    """d h / d amplitude of a single-site factor (X or Y on the left or right site)."""
    _, side, op = _SINGLE[kind]
    P = _g.X if op == "X" else _g.Y
    return np.kron(P, _g.I2) if side == 0 else np.kron(_g.I2, P)


def factor_params(pb: Problem, b, kind, k):
    """[((k, c, i), dh/du)] for the controls that enter the factor."""
    if kind == "bond":
        gens = _g.bond_generators(pb.N, b)
        return [(idx, gens[name]) for name, idx in param_slots(pb, k, b)]
    if kind == "V":
        if pb.C == 3 and pb.mask[2, b]:
            return [((k, 2, b), np.kron(_g.Z, _g.Z))]
        return []
    c, side, _ = _SINGLE[kind]
    i = b + side
    return [((k, c, i), factor_generator(kind))] if pb.mask[c, i] else []


def embed_out(G):
    """G (x) I_in for a 4x4 two-qubit matrix G: the 16x16 matrix on two
    operator sites with index s = 2 out + in."""
    E = np.einsum("acbd,ik,jl->aicjbkdl", G.reshape(2, 2, 2, 2), np.eye(2), np.eye(2))
    return E.reshape(16, 16)


def _layer_bonds(N, parity):
    return list(range(parity, N - 1, 2))


def _note_cut(stats, info):
    """Record a cap-decided cut in ``stats`` (diagnostic: "cap_cuts", "min_gap")."""
    if stats is not None and info.get("gap") is not None:
        stats["cap_cuts"] = stats.get("cap_cuts", 0) + 1
        stats["min_gap"] = min(stats.get("min_gap", np.inf), info["gap"])


def trajectory(pb: Problem, s: int, p: int, want_grad: bool = True, stats=None):
    """(O_sp, dO_sp[K][C][N] or None) for noise sample s and input p.

    ``stats`` (a dict, optional) collects diagnostics: "discarded" (forward
    discarded weight), "dims" (forward bond dimensions), and over the forward
    and costate updates "cap_cuts" (cuts the cap chi decided) and "min_gap"
    (smallest relative gap at such a cut, see ``mps.two_site_update``)."""
    info = {}
    N = pb.N
    B, lam = _m.canonicalize(pb.inputs[p], pb.chi, pb.eps)
    T, tlam = _m.canonicalize(pb.targets[p], pb.chi, pb.eps)
    sched = schedule(pb)
    gate_cache = []
    hist = [([x.copy() for x in B], [x.copy() for x in lam])] if want_grad else None
    for (par, factors) in sched:
        gl = {}
        for b in _layer_bonds(N, par):
            parts = [(kind, k, tau) + _g.expm_hermitian(factor_hamiltonian(pb, s, b, kind, k), tau)
                     for (kind, k, tau) in factors(b)]
            Mg = np.eye(4, dtype=np.complex128)
            for part in parts:
                Mg = part[3] @ Mg
            if pb.operator:
                Mg = embed_out(Mg)
            gl[b] = (Mg, parts)
            w, kk = _m.two_site_update(B, lam, b, Mg, pb.chi, pb.eps, info)
            if stats is not None:
                stats["discarded"] += w
                stats["dims"].append(kk)
                _note_cut(stats, info)
        gate_cache.append(gl)
        if want_grad:
            hist.append(([x.copy() for x in B], [x.copy() for x in lam]))
    O = _m.overlap(T, B)
    if not want_grad:
        return O, None
    dO = np.zeros((pb.K, pb.C, N), dtype=np.complex128)
    cB, clam = [x.copy() for x in T], [x.copy() for x in tlam]
    for li in range(len(sched) - 1, -1, -1):
        par, _ = sched[li]
        a_after = hist[li + 1][0]
        for b in _layer_bonds(N, par):
            Mg, parts = gate_cache[li][b]
            rho = _m.mixed_two_site_density(cB, a_after, b)
            # factor j of the product M = G_n ... G_1:  dO/du = tr(Q_j L^dag rho L),
            # Q_j = (dG_j/du) G_j^dag, L = G_n ... G_{j+1} (the factors after it)
            Lt = np.eye(4, dtype=np.complex128)
            for (kind, k, tau, G, ev, V) in reversed(parts):
                Le = embed_out(Lt) if pb.operator else Lt
                r = Le.conj().T @ rho @ Le
                for idx, gen in factor_params(pb, b, kind, k):
                    dG = _g.dexpm_hermitian(ev, V, tau, gen)
                    Q = dG @ G.conj().T
                    dO[idx] += np.trace((embed_out(Q) if pb.operator else Q) @ r)
                Lt = Lt @ G
        for b in _layer_bonds(N, par):
            Mg = gate_cache[li][b][0]
            _m.two_site_update(cB, clam, b, Mg.conj().T, pb.chi, pb.eps, info)
            _note_cut(stats, info)
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
                   eps=w.sv_cutoff, order=getattr(w, "order", 2), substeps=getattr(w, "substeps", 1),
                   operator=getattr(w, "operator", False))


def per_gate_infidelity(chi_bar: float, n: int, qubits_per_gate: int) -> float:
    """Sec. III reporting formula: 1 - (1 - chi_bar)^(q/n) for gates acting on
    q qubits each (q = 1: parallel X, q = 2: parallel CNOT)."""
    return 1.0 - (1.0 - chi_bar) ** (qubits_per_gate / n)

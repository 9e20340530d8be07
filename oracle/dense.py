"""Dense state-vector reference for small chains (N <= 12): the same gate
sequence as the TEBD path without any truncation, plus the exact per-slice
propagator exp(-i dt H_k) of Eq. sysH for the Trotter-error check.
Site 0 is the most significant bit of the basis index."""
import numpy as np

from . import gates as _g
from . import robust as _r


def apply_two_site(psi, G, b, N):
    v = psi.reshape(2 ** b, 4, 2 ** (N - b - 2))
    return np.einsum("ij,ajc->aic", G, v).reshape(-1)


def product_vector(sites):
    v = np.ones(1, dtype=np.complex128)
    for t in sites:
        v = np.kron(v, np.asarray(t).reshape(-1))
    return v


def mps_vector(sites):
    v = np.asarray(sites[0]).reshape(2, -1)
    for t in sites[1:]:
        v = np.tensordot(v, t, axes=(1, 0)).reshape(-1, t.shape[2])
    v = v.reshape(-1)
    return v / np.linalg.norm(v)


def apply_one_site(psi, U, j, N):
    v = psi.reshape(2 ** j, 2, 2 ** (N - j - 1))
    return np.einsum("ij,ajc->aic", U, v).reshape(-1)


def first_order_trajectory(pb: "_r.Problem", s, p, want_grad=True):
    """(O, dO) with the slice of Eq. circuit applied literally to a dense
    vector: per Trotter step (dt / substeps) of bin k, exp(-i dts V_b) on
    every bond (odd bonds, then even bonds; V_b = c ZZ + J^x XX + J^y YY),
    then exp(-i dts y_j Y) on every site, then exp(-i dts x_j X) on every
    site.  The gradient is the costate formula of App. A with its factor
    -i dts and each derivative taken at its own factor:
    dO/du = <b| (-i dts P) |a> right after the factor u enters, P = ZZ, X_j or Y_j."""
    N = pb.N
    a = mps_vector(pb.inputs[p])
    t = mps_vector(pb.targets[p])
    dts = pb.dt / pb.substeps
    ops = []   # (kind, where, U, (k, c, i) or None, generator) in time order
    for k in range(pb.K):
        for _ in range(pb.substeps):
            for b in list(range(1, N - 1, 2)) + list(range(0, N - 1, 2)):
                xl, yl, xr, yr, c, jx, jy = _r.bond_params(pb, s, k, b)
                h = c * np.kron(_g.Z, _g.Z) + jx * np.kron(_g.X, _g.X) + jy * np.kron(_g.Y, _g.Y)
                G = _g.expm_hermitian(h, dts)[0]
                slot = (k, 2, b) if (pb.C == 3 and pb.mask[2, b]) else None
                ops.append((2, b, G, slot, np.kron(_g.Z, _g.Z)))
            for cidx, P in ((1, _g.Y), (0, _g.X)):
                for j in range(N):
                    amp = pb.u[k, cidx, j] * pb.mask[cidx, j]
                    U = np.cos(dts * amp) * _g.I2 - 1j * np.sin(dts * amp) * P
                    ops.append((1, j, U, (k, cidx, j) if pb.mask[cidx, j] else None, P))
    hist = [a]
    for (kind, wh, U, _, _) in ops:
        a = apply_two_site(a, U, wh, N) if kind == 2 else apply_one_site(a, U, wh, N)
        hist.append(a)
    O = np.vdot(t, a)
    if not want_grad:
        return O, None
    dO = np.zeros((pb.K, pb.C, N), dtype=np.complex128)
    c = t.copy()
    for i in range(len(ops) - 1, -1, -1):
        kind, wh, U, slot, P = ops[i]
        if slot is not None:
            Q = -1j * dts * P
            v = apply_two_site(hist[i + 1], Q, wh, N) if kind == 2 else apply_one_site(hist[i + 1], Q, wh, N)
            dO[slot] += np.vdot(c, v)
        Ud = U.conj().T
        c = apply_two_site(c, Ud, wh, N) if kind == 2 else apply_one_site(c, Ud, wh, N)
    return O, dO


def trajectory(pb: "_r.Problem", s, p, want_grad=True):
    """(O, dO) for one trajectory with dense vectors and the costate formula."""
    if pb.order == 1:
        return first_order_trajectory(pb, s, p, want_grad)
    N = pb.N
    a = mps_vector(pb.inputs[p])
    t = mps_vector(pb.targets[p])
    sched = _r.layers(pb.K, pb.dt, pb.substeps)
    hist = [a]
    gl_all = []
    for (k, par, tau) in sched:
        gl = {}
        for b in range(par, N - 1, 2):
            G, ev, V = _r.bond_gate(pb, s, k, b, tau)
            gl[b] = (G, ev, V)
            a = apply_two_site(a, G, b, N)
        gl_all.append(gl)
        hist.append(a)
    O = np.vdot(t, a)
    if not want_grad:
        return O, None
    dO = np.zeros((pb.K, pb.C, N), dtype=np.complex128)
    c = t.copy()
    for li in range(len(sched) - 1, -1, -1):
        k, par, tau = sched[li]
        for b in range(par, N - 1, 2):
            G, ev, V = gl_all[li][b]
            gens = _g.bond_generators(N, b)
            for name, idx in _r.param_slots(pb, k, b):
                Q = _g.dexpm_hermitian(ev, V, tau, gens[name]) @ G.conj().T
                dO[idx] += np.vdot(c, apply_two_site(hist[li + 1], Q, b, N))
        for b in range(par, N - 1, 2):
            c = apply_two_site(c, gl_all[li][b][0].conj().T, b, N)
    return O, dO


def evolve(pb: "_r.Problem", s, a):
    """The time-ordered gate sequence of noise sample s applied to the dense
    vector a without truncation: the elementary layers A(dts/2) B(dts)
    A(dts/2) of every Trotter step (second order), or Eq. circuit applied
    literally (first order)."""
    N = pb.N
    if pb.order == 1:
        dts = pb.dt / pb.substeps
        for k in range(pb.K):
            for _ in range(pb.substeps):
                for b in list(range(1, N - 1, 2)) + list(range(0, N - 1, 2)):
                    xl, yl, xr, yr, c, jx, jy = _r.bond_params(pb, s, k, b)
                    h = c * np.kron(_g.Z, _g.Z) + jx * np.kron(_g.X, _g.X) + jy * np.kron(_g.Y, _g.Y)
                    a = apply_two_site(a, _g.expm_hermitian(h, dts)[0], b, N)
                for cidx, P in ((1, _g.Y), (0, _g.X)):
                    for j in range(N):
                        amp = pb.u[k, cidx, j] * pb.mask[cidx, j]
                        a = apply_one_site(a, np.cos(dts * amp) * _g.I2 - 1j * np.sin(dts * amp) * P, j, N)
        return a
    for (k, par, tau) in _r.layers(pb.K, pb.dt, pb.substeps):
        for b in range(par, N - 1, 2):
            a = apply_two_site(a, _r.bond_gate(pb, s, k, b, tau)[0], b, N)
    return a


def unitary(pb: "_r.Problem", s):
    """The 2^N x 2^N propagator of noise sample s, column by column."""
    n = 2 ** pb.N
    U = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        U[:, j] = evolve(pb, s, e)
    return U


def gate_overlap(pb: "_r.Problem", s, U_T):
    """tr(U_T^dag U^(s)) / 2^N, the quantity whose squared modulus is one minus
    the gate infidelity of Eq. gateinfid."""
    return np.trace(U_T.conj().T @ unitary(pb, s)) / 2 ** pb.N


def full_hamiltonian(pb: "_r.Problem", s, k):
    """H_k of Eq. sysH (ZZ crosstalk) as a dense 2^N x 2^N matrix."""
    N = pb.N
    H = np.zeros((2 ** N, 2 ** N), dtype=np.complex128)
    for b in range(N - 1):
        h = _g.bond_hamiltonian(N, b, *_r.bond_params(pb, s, k, b))
        H += np.kron(np.kron(np.eye(2 ** b), h), np.eye(2 ** (N - b - 2)))
    return H


def exact_overlap(pb: "_r.Problem", s, p):
    """<t| prod_k exp(-i dt H_k) |in> with exact slice exponentials."""
    a = mps_vector(pb.inputs[p])
    t = mps_vector(pb.targets[p])
    for k in range(pb.K):
        w, V = np.linalg.eigh(full_hamiltonian(pb, s, k))
        a = V @ (np.exp(-1j * pb.dt * w) * (V.conj().T @ a))
    return np.vdot(t, a)

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


def trajectory(pb: "_r.Problem", s, p, want_grad=True):
    """(O, dO) for one trajectory with dense vectors and the costate formula."""
    N = pb.N
    a = mps_vector(pb.inputs[p])
    t = mps_vector(pb.targets[p])
    sched = _r.layers(pb.K, pb.dt)
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

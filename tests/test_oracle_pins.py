"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(closed forms, a published generator, a textbook exponential, brute force),
independent of the oracle's own code paths."""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import dense, gates, mps, noise, robust

GOLD = os.path.join(os.path.dirname(__file__), "golden")
I2 = np.eye(2)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]])
PZ = np.diag([1.0, -1.0]).astype(complex)


def mkpb(N, K, dt, C, chi, u, mask, J, inputs, targets, g_fixed=None, eps=1e-12, order=2, substeps=1,
         operator=False):
    return robust.Problem(N=N, K=K, dt=dt, C=C, chi=chi, u=u, mask=mask,
                          J=np.atleast_2d(J) if np.ndim(J) < 3 else J,
                          inputs=[m.sites for m in inputs], targets=[m.sites for m in targets],
                          g_fixed=g_fixed, eps=eps, order=order, substeps=substeps, operator=operator)


def rand_products(N, P, seed):
    return synth.product_inputs(N, P, seed)


# ---------------------------------------------------------------- (a) pi pulse
def test_pi_pulse_gives_parallel_x():
    N, K, dt = 6, 10, 0.1
    u = synth.pi_pulse_controls(K, 2, N, dt)
    ins = rand_products(N, 3, 5)
    pb = mkpb(N, K, dt, 2, 16, u, synth.control_mask(2, N), np.zeros(N - 1), ins, synth.x_targets(ins))
    F, g, _ = robust.ensemble(pb)
    assert abs(F - 1.0) < 1e-13
    # a maximum: gradient vanishes
    assert np.max(np.abs(g)) < 1e-12
    o, _ = dense.trajectory(pb, 0, 1, False)
    assert abs(abs(o) - 1.0) < 1e-13


# ---------------------------------------------------- J = 0: single-qubit closed form
def _rot(x, y, dt):
    """exp(-i dt (x X + y Y)) = cos(th) I - i sin(th)/th (a X + b Y), th = |(a, b)|."""
    a, b = dt * x, dt * y
    th = math.hypot(a, b)
    sc = math.sin(th) / th if th > 0 else 1.0
    return math.cos(th) * I2 - 1j * sc * (a * PX + b * PY)


def _drot(x, y, dt, wrt):
    a, b = dt * x, dt * y
    th = math.hypot(a, b)
    sc = math.sin(th) / th
    dsc = (th * math.cos(th) - math.sin(th)) / th ** 2
    da = a / th if wrt == "x" else b / th
    gen = PX if wrt == "x" else PY
    dU = -math.sin(th) * da * I2 - 1j * (dsc * da * (a * PX + b * PY) + sc * gen)
    return dt * dU


def test_zero_crosstalk_closed_form_fidelity_and_gradient():
    N, K, dt = 5, 6, 0.1
    rng = np.random.default_rng(11)
    u = rng.normal(0, 0.7, size=(K, 2, N))
    ins = rand_products(N, 1, 12)
    tgs = rand_products(N, 1, 13)
    pb = mkpb(N, K, dt, 2, 8, u, synth.control_mask(2, N), np.zeros(N - 1), ins, tgs)
    F, g, _ = robust.ensemble(pb)
    vin = [s.reshape(2) for s in ins[0].sites]
    vt = [s.reshape(2) for s in tgs[0].sites]
    Us = []
    Os = []
    for i in range(N):
        U = I2.astype(complex)
        for k in range(K):
            U = _rot(u[k, 0, i], u[k, 1, i], dt) @ U
        Us.append(U)
        Os.append(np.vdot(vt[i], U @ vin[i]))
    O = np.prod(Os)
    assert abs(F - abs(O) ** 2) < 1e-13
    gref = np.zeros((K, 2, N))
    for i in range(N):
        rest = np.prod([Os[j] for j in range(N) if j != i])
        for k in range(K):
            for c, wrt in ((0, "x"), (1, "y")):
                M = I2.astype(complex)
                for kk in range(K):
                    M = (_drot(u[kk, 0, i], u[kk, 1, i], dt, wrt) if kk == k else
                         _rot(u[kk, 0, i], u[kk, 1, i], dt)) @ M
                dO = rest * np.vdot(vt[i], M @ vin[i])
                gref[k, c, i] = 2 * np.real(np.conj(O) * dO)
    assert np.max(np.abs(g - gref)) < 1e-12 * max(1.0, np.max(np.abs(gref))) + 1e-15


# ---------------------------------------------------------- ZZ only: closed form
def test_zz_only_closed_form_with_g_gradient():
    N, K, dt = 6, 5, 0.2
    rng = np.random.default_rng(21)
    u = rng.normal(0, 0.8, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    mask[0, :] = 0
    mask[1, :] = 0
    J = rng.uniform(-0.3, 0.3, size=N - 1)
    ins = rand_products(N, 1, 22)
    tgs = rand_products(N, 1, 23)
    pb = mkpb(N, K, dt, 3, 8, u, mask, J, ins, tgs)
    F, g, _ = robust.ensemble(pb)
    vin = [s.reshape(2) for s in ins[0].sites]
    vt = [s.reshape(2) for s in tgs[0].sites]
    sig = np.array([1.0, -1.0])
    phi = np.array([dt * (u[:, 2, b].sum() + K * J[b]) for b in range(N - 1)])

    def chain(deriv=None):
        w = np.conj(vt[0]) * vin[0]
        for b in range(N - 1):
            Mb = np.exp(-1j * phi[b] * np.outer(sig, sig))
            if deriv == b:
                Mb = Mb * (-1j * dt * np.outer(sig, sig))
            w = (w @ Mb) * np.conj(vt[b + 1]) * vin[b + 1]
        return w.sum()

    O = chain()
    assert abs(F - abs(O) ** 2) < 1e-13
    for b in range(N - 1):
        dO = chain(deriv=b)
        for k in range(K):
            assert abs(g[k, 2, b] - 2 * np.real(np.conj(O) * dO)) < 1e-12
    assert np.all(g[:, :2, :] == 0.0)
    assert np.all(g[:, 2, N - 1] == 0.0)


# ------------------------------------------------ untruncated MPS == dense vector
def test_untruncated_mps_equals_dense_statevector():
    N, K, dt = 8, 4, 0.15
    rng = np.random.default_rng(31)
    u = rng.normal(0, 0.8, size=(K, 3, N))
    J = rng.uniform(-0.2, 0.2, size=(2, N - 1))
    ins = rand_products(N, 2, 32)
    tgs = rand_products(N, 2, 33)
    pb = mkpb(N, K, dt, 3, 16, u, synth.control_mask(3, N, "all"), J, ins, tgs)
    for s in range(2):
        for p in range(2):
            o1, d1 = robust.trajectory(pb, s, p)
            o2, d2 = dense.trajectory(pb, s, p)
            assert abs(o1 - o2) < 1e-12
            assert np.max(np.abs(d1 - d2)) < 1e-12


def test_mps_state_matches_dense_vector_elementwise():
    N, K, dt = 6, 3, 0.3
    rng = np.random.default_rng(41)
    u = rng.normal(0, 1.0, size=(K, 3, N))
    ins = rand_products(N, 1, 42)
    pb = mkpb(N, K, dt, 3, 8, u, synth.control_mask(3, N, "all"), rng.normal(0, 0.1, N - 1), ins, ins)
    B, lam = mps.canonicalize(pb.inputs[0], pb.chi, pb.eps)
    a = dense.mps_vector(pb.inputs[0])
    for (par, group) in robust.merged_layers(K, dt):
        for b in range(par, N - 1, 2):
            Mg = np.eye(4, dtype=complex)
            for (k, tau) in group:
                G, _, _ = robust.bond_gate(pb, 0, k, b, tau)
                Mg = G @ Mg
                a = dense.apply_two_site(a, G, b, N)
            mps.two_site_update(B, lam, b, Mg, pb.chi, pb.eps)
    v = mps.to_dense(B)
    assert np.max(np.abs(v - a)) < 1e-12
    # Schmidt values of every bond = singular values of the dense reshape
    for b in range(N - 1):
        sv = np.linalg.svd(a.reshape(2 ** (b + 1), -1), compute_uv=False)
        k = len(lam[b])
        assert np.max(np.abs(sv[:k] - lam[b])) < 1e-12
        assert np.all(sv[k:] < 1e-12)


@pytest.mark.parametrize("chi,eps", [(3, 1e-12), (8, 1e-2), (2, 1e-12)])
def test_one_truncated_update_is_the_dense_schmidt_projection(chi, eps):
    """On a state in exact canonical form, one truncated two-site update is the
    dense rule written out: apply the gate, Schmidt-decompose the vector across
    the bond, keep k = min(chi, #{sigma_i > max(eps, 1e-13) sigma_1}) values,
    renormalise.  The kept Schmidt values and the whole state vector must agree
    (the projection is unique when the cut is not a tie, which is checked)."""
    N = 7
    rng = np.random.default_rng(17 + chi)
    # an entangled canonical state: a random MPS of bond 6
    sites = []
    dims = [1, 2, 4, 6, 6, 4, 2, 1]
    for i in range(N):
        sites.append(rng.normal(size=(dims[i], 2, dims[i + 1])) + 1j * rng.normal(size=(dims[i], 2, dims[i + 1])))
    B, lam = mps.canonicalize(sites, 64, 1e-14)
    psi = mps.to_dense(B)
    for b in (2, 3):
        Bb, lamb = [x.copy() for x in B], [x.copy() for x in lam]
        h = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
        G = gates.expm_hermitian(h + h.conj().T, 0.7)[0]
        mps.two_site_update(Bb, lamb, b, G, chi, eps)
        v = dense.apply_two_site(psi, G, b, N)
        U, S, Vh = np.linalg.svd(v.reshape(2 ** (b + 1), -1), full_matrices=False)
        k = max(1, min(chi, int(np.count_nonzero(S > max(eps, 1e-13) * S[0]))))
        assert S[k - 1] - (S[k] if k < len(S) else 0.0) > 1e-6      # no tie at the cut
        ref = (U[:, :k] * S[:k]) @ Vh[:k] / np.linalg.norm(S[:k])
        assert len(lamb[b]) == k
        assert np.max(np.abs(lamb[b] - S[:k] / np.linalg.norm(S[:k]))) < 1e-12
        assert np.max(np.abs(mps.to_dense(Bb) - ref.reshape(-1))) < 1e-12


# ------------------------------------------------------- Trotter error is O(dt^2)
def test_second_order_trotter_error_scaling():
    N, K0, T = 4, 2, 1.0
    rng = np.random.default_rng(51)
    u0 = rng.normal(0, 1.0, size=(K0, 3, N))
    J = rng.uniform(-0.5, 0.5, size=N - 1)
    ins = rand_products(N, 1, 52)
    tgs = rand_products(N, 1, 53)
    errs = []
    for r in (4, 8, 16):
        u = np.repeat(u0, r, axis=0)
        K = K0 * r
        pb = mkpb(N, K, T / K, 3, 16, u, synth.control_mask(3, N, "all"), J, ins, tgs)
        o_t, _ = dense.trajectory(pb, 0, 0, False)
        o_e = dense.exact_overlap(pb, 0, 0)
        errs.append(abs(o_t - o_e))
    assert 3.3 < errs[0] / errs[1] < 4.7
    assert 3.3 < errs[1] / errs[2] < 4.7


@pytest.mark.parametrize("order,ratio", [(1, 2.0), (2, 4.0)])
def test_trotter_error_order_with_substeps(order, ratio):
    """Against the exact exponential of each bin's Hamiltonian (Eq. sysH), the
    overlap error of n Trotter steps per bin falls as 1/n for the first-order
    slice of Eq. circuit and as 1/n^2 for the second-order split."""
    N, K, T = 4, 2, 1.0
    rng = np.random.default_rng(57)
    u = rng.normal(0, 1.0, size=(K, 3, N))
    J = rng.uniform(-0.5, 0.5, size=N - 1)
    ins = rand_products(N, 1, 58)
    tgs = rand_products(N, 1, 59)
    errs = []
    for n in (4, 8, 16):
        pb = mkpb(N, K, T / K, 3, 16, u, synth.control_mask(3, N, "all"), J, ins, tgs, order=order, substeps=n)
        o_t, _ = robust.trajectory(pb, 0, 0, want_grad=False)
        errs.append(abs(o_t - dense.exact_overlap(pb, 0, 0)))
    for a, b in zip(errs, errs[1:]):
        assert 0.8 * ratio < a / b < 1.2 * ratio, errs


# ------------------------------------------------------- finite differences
def test_gradient_matches_central_finite_differences():
    N, K, dt = 6, 5, 0.1
    rng = np.random.default_rng(61)
    u = rng.normal(0, 0.5, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    J = rng.uniform(-0.1, 0.1, size=(2, N - 1))
    ins = rand_products(N, 2, 62)
    tgs = synth.x_targets(ins)
    pb = mkpb(N, K, dt, 3, 8, u, mask, J, ins, tgs)
    F, g, _ = robust.ensemble(pb)
    h = 1e-6
    idxs = [tuple(int(rng.integers(0, n)) for n in u.shape) for _ in range(20)]
    for idx in idxs:
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        Fp, _, _ = robust.ensemble(mkpb(N, K, dt, 3, 8, up, mask, J, ins, tgs), want_grad=False)
        Fm, _, _ = robust.ensemble(mkpb(N, K, dt, 3, 8, um, mask, J, ins, tgs), want_grad=False)
        fd = (Fp - Fm) / (2 * h)
        assert abs(fd - g[idx]) < 1e-6 * max(1e-3, np.max(np.abs(g)))


# ----------------------------------------- Daleckii-Krein vs Van Loan block exponential
@pytest.mark.parametrize("degenerate", [False, True])
def test_gate_derivative_matches_block_exponential(degenerate):
    rng = np.random.default_rng(71 + degenerate)
    if degenerate:
        h = 0.7 * np.kron(PZ, PZ)
    else:
        a = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
        h = (a + a.conj().T) / 2
    b = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    P = (b + b.conj().T) / 2
    tau = 0.37
    G, lam, V = gates.expm_hermitian(h, tau)
    assert np.max(np.abs(G - scipy.linalg.expm(-1j * tau * h))) < 1e-14
    assert np.max(np.abs(G.conj().T @ G - np.eye(4))) < 1e-14
    big = np.zeros((8, 8), dtype=complex)
    big[:4, :4] = -1j * tau * h
    big[4:, 4:] = -1j * tau * h
    big[:4, 4:] = -1j * tau * P
    ref = scipy.linalg.expm(big)[:4, 4:]
    dG = gates.dexpm_hermitian(lam, V, tau, P)
    assert np.max(np.abs(dG - ref)) < 1e-13


def test_bond_hamiltonians_sum_to_system_hamiltonian():
    N = 5
    rng = np.random.default_rng(81)
    x, y, c = rng.normal(size=N), rng.normal(size=N), rng.normal(size=N - 1)
    H = np.zeros((2 ** N, 2 ** N), dtype=complex)
    for b in range(N - 1):
        h = gates.bond_hamiltonian(N, b, x[b], y[b], x[b + 1], y[b + 1], c[b])
        H += np.kron(np.kron(np.eye(2 ** b), h), np.eye(2 ** (N - b - 2)))

    def op(o, i):
        return np.kron(np.kron(np.eye(2 ** i), o), np.eye(2 ** (N - i - 1)))

    ref = sum(x[i] * op(PX, i) + y[i] * op(PY, i) for i in range(N))
    ref = ref + sum(c[b] * op(PZ, b) @ op(PZ, b + 1) for b in range(N - 1))
    assert np.max(np.abs(H - ref)) < 1e-13
    # Heisenberg-type crosstalk terms (Eq. Hp)
    jx, jy = rng.normal(size=N - 1), rng.normal(size=N - 1)
    H2 = np.zeros((2 ** N, 2 ** N), dtype=complex)
    for b in range(N - 1):
        h = gates.bond_hamiltonian(N, b, x[b], y[b], x[b + 1], y[b + 1], c[b], jx[b], jy[b])
        H2 += np.kron(np.kron(np.eye(2 ** b), h), np.eye(2 ** (N - b - 2)))
    ref2 = ref + sum(jx[b] * op(PX, b) @ op(PX, b + 1) + jy[b] * op(PY, b) @ op(PY, b + 1) for b in range(N - 1))
    assert np.max(np.abs(H2 - ref2)) < 1e-13


def test_heisenberg_crosstalk_two_site_closed_form():
    """u = 0, one bond: (J^x XX + J^y YY) couples |01> and |10> with strength
    J^x + J^y, J^z ZZ is a phase on that subspace, so <01|U(T)|01> has modulus
    |cos(T (J^x + J^y))|."""
    N, K, dt = 2, 7, 0.13
    jx, jy, jz = 0.31, -0.12, 0.27
    one = synth.MPS([np.array([1.0, 0.0]).reshape(1, 2, 1), np.array([0.0, 1.0]).reshape(1, 2, 1)])
    pb = mkpb(N, K, dt, 2, 2, np.zeros((K, 2, N)), synth.control_mask(2, N), np.array([[[jx, jy, jz]]]),
              [one], [one])
    F, _, _ = robust.ensemble(pb, want_grad=False)
    assert abs(F - np.cos(K * dt * (jx + jy)) ** 2) < 1e-13


def test_isotropic_xy_crosstalk_keeps_the_polarised_state():
    """With J^x = J^y on every bond and no drive, |0...0> is an eigenstate of
    every bond gate, so F = 1 for input = target = |0...0>."""
    N, K, dt = 7, 5, 0.2
    rng = np.random.default_rng(123)
    jxy = rng.uniform(-0.3, 0.3, size=N - 1)
    J = np.stack([jxy, jxy, rng.uniform(-0.3, 0.3, size=N - 1)], axis=1)[None]
    z = synth.zero_state(N)
    pb = mkpb(N, K, dt, 3, 8, np.zeros((K, 3, N)), synth.control_mask(3, N, "all"), J, [z], [z])
    F, g, _ = robust.ensemble(pb)
    assert abs(F - 1.0) < 1e-13
    assert np.max(np.abs(g)) < 1e-12


def test_heisenberg_crosstalk_mps_equals_dense_and_fd():
    N, K, dt = 6, 4, 0.15
    rng = np.random.default_rng(131)
    u = rng.normal(0, 0.7, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    J = noise.sample_J(5, 2, N, 0, 0.2, terms=3)
    ins = rand_products(N, 2, 132)
    tgs = rand_products(N, 2, 133)
    pb = mkpb(N, K, dt, 3, 8, u, mask, J, ins, tgs)
    for s in range(2):
        o1, d1 = robust.trajectory(pb, s, 1)
        o2, d2 = dense.trajectory(pb, s, 1)
        assert abs(o1 - o2) < 1e-12 and np.max(np.abs(d1 - d2)) < 1e-12
    F, g, _ = robust.ensemble(pb)
    h = 1e-6
    for _ in range(8):
        idx = tuple(int(rng.integers(0, n)) for n in u.shape)
        if not mask[idx[1], idx[2]]:
            continue
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        Fp, _, _ = robust.ensemble(mkpb(N, K, dt, 3, 8, up, mask, J, ins, tgs), want_grad=False)
        Fm, _, _ = robust.ensemble(mkpb(N, K, dt, 3, 8, um, mask, J, ins, tgs), want_grad=False)
        assert abs((Fp - Fm) / (2 * h) - g[idx]) < 1e-6 * max(1e-3, np.max(np.abs(g)))


# ------------------------------------------- first-order split (Eq. circuit)
def test_first_order_pi_pulse_gives_parallel_x():
    # Eq. circuit with x = pi/(2T), y = 0, no crosstalk: every site gets exp(-i pi X / 2) = -iX
    N, K, dt = 5, 8, 0.1
    u = synth.pi_pulse_controls(K, 2, N, dt)
    ins = rand_products(N, 2, 7)
    pb = mkpb(N, K, dt, 2, 16, u, synth.control_mask(2, N), np.zeros(N - 1), ins, synth.x_targets(ins),
              order=1, substeps=2)
    F, g, _ = robust.ensemble(pb)
    assert abs(F - 1.0) < 1e-13 and np.max(np.abs(g)) < 1e-12


@pytest.mark.parametrize("substeps", [1, 3])
def test_first_order_zero_crosstalk_closed_form(substeps):
    """No interaction: each site evolves by prod_k (e^{-i d x X} e^{-i d y Y})^n_sub,
    d = dt / n_sub -- X applied after Y, as the left-to-right order of Eq. circuit
    says -- a product of 2x2 rotations with closed-form derivatives."""
    N, K, dt = 5, 4, 0.15
    rng = np.random.default_rng(41)
    u = rng.normal(0, 0.8, size=(K, 2, N))
    ins = rand_products(N, 1, 42)
    tgs = rand_products(N, 1, 43)
    pb = mkpb(N, K, dt, 2, 8, u, synth.control_mask(2, N), np.zeros(N - 1), ins, tgs, order=1,
              substeps=substeps)
    F, g, _ = robust.ensemble(pb)
    d = dt / substeps

    def rx(x):
        return math.cos(d * x) * I2 - 1j * math.sin(d * x) * PX

    def ry(y):
        return math.cos(d * y) * I2 - 1j * math.sin(d * y) * PY

    vin = [q.reshape(2) for q in ins[0].sites]
    vt = [q.reshape(2) for q in tgs[0].sites]
    Os, dOs = [], []
    for i in range(N):
        steps = [(k, rx(u[k, 0, i]) @ ry(u[k, 1, i])) for k in range(K) for _ in range(substeps)]
        U = I2.astype(complex)
        for _, S in steps:
            U = S @ U
        Os.append(np.vdot(vt[i], U @ vin[i]))
        dd = np.zeros((K, 2), dtype=complex)
        for j, (k, S) in enumerate(steps):
            before = I2.astype(complex)
            for _, S2 in steps[:j]:
                before = S2 @ before
            after = I2.astype(complex)
            for _, S2 in steps[j + 1:]:
                after = S2 @ after
            x, y = u[k, 0, i], u[k, 1, i]
            dSx = (-1j * d * PX) @ rx(x) @ ry(y)
            dSy = rx(x) @ (-1j * d * PY) @ ry(y)
            dd[k, 0] += np.vdot(vt[i], after @ dSx @ before @ vin[i])
            dd[k, 1] += np.vdot(vt[i], after @ dSy @ before @ vin[i])
        dOs.append(dd)
    O = np.prod(Os)
    assert abs(F - abs(O) ** 2) < 1e-13
    gref = np.zeros((K, 2, N))
    for i in range(N):
        rest = np.prod([Os[j] for j in range(N) if j != i])
        gref[:, :, i] = 2 * np.real(np.conj(O) * rest * dOs[i])
    assert np.max(np.abs(g - gref)) < 1e-12 * max(1.0, np.max(np.abs(gref)))


@pytest.mark.parametrize("N,terms,substeps", [(6, 1, 1), (5, 1, 2), (6, 3, 2), (5, 3, 1), (2, 1, 1)])
def test_first_order_mps_equals_literal_circuit(N, terms, substeps):
    """The folded truncated layers of the MPS path against Eq. circuit applied
    gate by gate to a dense vector (every bond, then Y on every site, then X on
    every site), untruncated: overlaps and costate gradients to 1e-12."""
    K, dt = 3, 0.2
    rng = np.random.default_rng(51 + N + terms)
    u = rng.normal(0, 0.7, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    J = noise.sample_J(9, 2, N, 0, 0.3, terms=terms)
    ins = rand_products(N, 2, 52)
    tgs = rand_products(N, 2, 53)
    pb = mkpb(N, K, dt, 3, 16, u, mask, J, ins, tgs, order=1, substeps=substeps)
    for s in range(2):
        for p in range(2):
            o1, d1 = robust.trajectory(pb, s, p)
            o2, d2 = dense.first_order_trajectory(pb, s, p)
            assert abs(o1 - o2) < 1e-12
            assert np.max(np.abs(d1 - d2)) < 1e-12


def test_first_order_gradient_matches_finite_differences():
    N, K, dt = 5, 3, 0.2
    rng = np.random.default_rng(61)
    u = rng.normal(0, 0.7, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    J = noise.sample_J(3, 2, N, 0, 0.2, terms=3)
    ins = rand_products(N, 1, 62)
    tgs = rand_products(N, 1, 63)
    kw = dict(order=1, substeps=2)
    F, g, _ = robust.ensemble(mkpb(N, K, dt, 3, 16, u, mask, J, ins, tgs, **kw))
    h = 1e-6
    checked = 0
    for _ in range(30):
        idx = tuple(int(rng.integers(0, n)) for n in u.shape)
        if not mask[idx[1], idx[2]]:
            continue
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        Fp, _, _ = robust.ensemble(mkpb(N, K, dt, 3, 16, up, mask, J, ins, tgs, **kw), want_grad=False)
        Fm, _, _ = robust.ensemble(mkpb(N, K, dt, 3, 16, um, mask, J, ins, tgs, **kw), want_grad=False)
        assert abs((Fp - Fm) / (2 * h) - g[idx]) < 1e-6 * max(1e-3, np.max(np.abs(g)))
        checked += 1
    assert checked >= 12


@pytest.mark.parametrize("order", [1, 2])
def test_substeps_equal_repeated_bins(order):
    """n Trotter steps per bin are the map of n consecutive bins of length dt/n
    holding the same controls; the gradient of a bin is the sum over its copies."""
    N, K, dt, n = 6, 3, 0.3, 2
    rng = np.random.default_rng(71)
    u = rng.normal(0, 0.7, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    J = rng.uniform(-0.2, 0.2, size=(1, N - 1))
    ins = rand_products(N, 1, 72)
    tgs = rand_products(N, 1, 73)
    o1, d1 = robust.trajectory(mkpb(N, K, dt, 3, 16, u, mask, J, ins, tgs, order=order, substeps=n), 0, 0)
    u2 = np.repeat(u, n, axis=0)
    o2, d2 = robust.trajectory(mkpb(N, K * n, dt / n, 3, 16, u2, mask, J, ins, tgs, order=order), 0, 0)
    assert abs(o1 - o2) < 1e-13
    assert np.max(np.abs(d1 - d2.reshape(K, n, 3, N).sum(axis=1))) < 1e-13


def test_first_order_schedule_folds_each_site_once():
    """Every site's two rotations enter exactly one bond gate per Trotter step,
    after every bond gate of that step that touches the site."""
    for N in (2, 3, 6, 7):
        pb = mkpb(N, 1, 0.1, 2, 4, np.zeros((1, 2, N)), synth.control_mask(2, N), np.zeros(N - 1),
                  rand_products(N, 1, 1), rand_products(N, 1, 2), order=1)
        seen = {j: [] for j in range(N)}
        last_touch = {j: -1 for j in range(N)}
        t = 0
        for par, factors in robust.schedule(pb):
            for b in range(par, N - 1, 2):
                for kind, _, _ in factors(b):
                    if kind == "V":
                        for j in (b, b + 1):
                            assert not seen[j], "bond gate after the site's rotations"
                            last_touch[j] = t
                    else:
                        seen[b + (kind[1] == "r")].append(kind[0])
                t += 1
        for j in range(N):
            assert seen[j] == ["y", "x"], (N, j, seen[j])


# ------------------------------------------ operator (MPO) form, Eq. gateinfid
def _dense_cnot_pairs(N):
    c = np.zeros((4, 4), dtype=complex)
    c[0, 0] = c[1, 1] = c[2, 3] = c[3, 2] = 1.0
    U = np.ones((1, 1), dtype=complex)
    for _ in range(N // 2):
        U = np.kron(U, c)
    return U


def test_operator_vectors_are_the_dense_operators():
    """<<A|B>> = tr(A^dag B) / 2^N for the identity, parallel X and parallel CNOT."""
    N = 4
    dense_ops = {"I": np.eye(16), "X": np.kron(np.kron(PX, PX), np.kron(PX, PX)), "C": _dense_cnot_pairs(N)}
    mps_ops = {"I": synth.identity_operator(N), "X": synth.x_gate_operator(N), "C": synth.cnot_gate_operator(N)}
    for a in dense_ops:
        for b in dense_ops:
            ref = np.trace(dense_ops[a].conj().T @ dense_ops[b]) / 2 ** N
            assert abs(mps.overlap(mps_ops[a].sites, mps_ops[b].sites) - ref) < 1e-14


def test_operator_pi_pulse_is_the_parallel_x_gate():
    N, K, dt = 5, 6, 0.1
    u = synth.pi_pulse_controls(K, 2, N, dt)
    pb = mkpb(N, K, dt, 2, 8, u, synth.control_mask(2, N), np.zeros(N - 1), [synth.identity_operator(N)],
              [synth.x_gate_operator(N)], operator=True)
    F, g, _ = robust.ensemble(pb)
    assert abs(F - 1.0) < 1e-13 and np.max(np.abs(g)) < 1e-12


def test_operator_zero_crosstalk_closed_form():
    """No interaction: U = (x) u_j with u_j the product of each slice's
    exp(-i dt (x X + y Y)), so tr(X^{(x)N} U) / 2^N = prod_j tr(X u_j) / 2 --
    fidelity and every derivative in closed form."""
    N, K, dt = 4, 5, 0.12
    rng = np.random.default_rng(81)
    u = rng.normal(0, 0.8, size=(K, 2, N))
    pb = mkpb(N, K, dt, 2, 8, u, synth.control_mask(2, N), np.zeros(N - 1), [synth.identity_operator(N)],
              [synth.x_gate_operator(N)], operator=True)
    F, g, _ = robust.ensemble(pb)
    Os, dOs = [], []
    for i in range(N):
        U = I2.astype(complex)
        for k in range(K):
            U = _rot(u[k, 0, i], u[k, 1, i], dt) @ U
        Os.append(np.trace(PX @ U) / 2)
        dd = np.zeros((K, 2), dtype=complex)
        for k in range(K):
            for c, wrt in ((0, "x"), (1, "y")):
                M = I2.astype(complex)
                for kk in range(K):
                    M = (_drot(u[kk, 0, i], u[kk, 1, i], dt, wrt) if kk == k else
                         _rot(u[kk, 0, i], u[kk, 1, i], dt)) @ M
                dd[k, c] = np.trace(PX @ M) / 2
        dOs.append(dd)
    O = np.prod(Os)
    assert abs(F - abs(O) ** 2) < 1e-13
    gref = np.zeros((K, 2, N))
    for i in range(N):
        rest = np.prod([Os[j] for j in range(N) if j != i])
        gref[:, :, i] = 2 * np.real(np.conj(O) * rest * dOs[i])
    assert np.max(np.abs(g - gref)) < 1e-12 * max(1.0, np.max(np.abs(gref)))


@pytest.mark.parametrize("order,terms,target", [(2, 1, "cnot"), (2, 3, "x"), (1, 1, "cnot"), (1, 3, "x")])
def test_operator_mpo_equals_dense_unitary_and_fd(order, terms, target):
    """The MPO path (untruncated) against the dense propagator built column by
    column from the same gate sequence: O = tr(U_T^dag U) / 2^N to 1e-12, and
    the costate gradient against central differences of the dense O."""
    N, K, dt = 4, 3, 0.2
    rng = np.random.default_rng(91 + order + terms)
    u = rng.normal(0, 0.7, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    J = noise.sample_J(4, 2, N, 0, 0.3, terms=terms)
    tg = synth.cnot_gate_operator(N) if target == "cnot" else synth.x_gate_operator(N)
    UT = _dense_cnot_pairs(N) if target == "cnot" else np.kron(np.kron(PX, PX), np.kron(PX, PX))

    def pbu(uu):
        return mkpb(N, K, dt, 3, 64, uu, mask, J, [synth.identity_operator(N)], [tg], order=order,
                    operator=True)

    pb = pbu(u)
    for s in range(2):
        o, dO = robust.trajectory(pb, s, 0)
        assert abs(o - dense.gate_overlap(pb, s, UT)) < 1e-12
        h = 1e-6
        for _ in range(6):
            idx = tuple(int(rng.integers(0, n)) for n in u.shape)
            if not mask[idx[1], idx[2]]:
                continue
            up, um = u.copy(), u.copy()
            up[idx] += h
            um[idx] -= h
            fd = (dense.gate_overlap(pbu(up), s, UT) - dense.gate_overlap(pbu(um), s, UT)) / (2 * h)
            assert abs(fd - dO[idx]) < 1e-7 * max(1.0, np.max(np.abs(dO)))


def test_operator_truncation_converges_in_chi():
    """The truncated MPO fidelity approaches the exact (dense) gate fidelity
    as chi grows, and equals it once chi reaches the exact operator rank."""
    N, K, dt = 6, 4, 0.25
    rng = np.random.default_rng(97)
    u = rng.normal(0, 1.2, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    J = noise.sample_J(6, 1, N, 0, 0.2)
    UT = _dense_cnot_pairs(N)
    errs = []
    for chi in (2, 4, 8, 64):
        pb = mkpb(N, K, dt, 3, chi, u, mask, J, [synth.identity_operator(N)], [synth.cnot_gate_operator(N)],
                  operator=True)
        o, _ = robust.trajectory(pb, 0, 0, want_grad=False)
        errs.append(abs(abs(o) ** 2 - abs(dense.gate_overlap(pb, 0, UT)) ** 2))
    assert errs[-1] < 1e-12
    assert errs[2] <= errs[0] + 1e-12


# ----------------------------------------------------------------- invariants
def test_merged_schedule_is_the_elementary_sequence():
    K, dt = 4, 0.1
    flat = [(k, par, tau) for (par, grp) in robust.merged_layers(K, dt) for (k, tau) in grp
            for _ in [0]]
    # the merged layers list the elementary layers in the same time order
    elem = robust.layers(K, dt)
    assert [(k, tau) for (k, _, tau) in flat] == [(k, tau) for (k, _, tau) in elem]
    assert [p for (p, _) in robust.merged_layers(K, dt)] == [0] + [1, 0] * K
    assert len(robust.merged_layers(K, dt)) == 2 * K + 1


def test_costate_overlap_is_constant_over_layers():
    N, K, dt = 6, 4, 0.2
    rng = np.random.default_rng(91)
    u = rng.normal(0, 0.8, size=(K, 3, N))
    ins = rand_products(N, 1, 92)
    tgs = rand_products(N, 1, 93)
    pb = mkpb(N, K, dt, 3, 8, u, synth.control_mask(3, N, "all"), rng.normal(0, .1, N - 1), ins, tgs)
    sched = robust.merged_layers(K, dt)
    B, lam = mps.canonicalize(pb.inputs[0], 8, 1e-12)
    states = [[x.copy() for x in B]]
    gl = []
    for (par, group) in sched:
        gg = {}
        for b in range(par, N - 1, 2):
            G = np.eye(4, dtype=complex)
            for (k, tau) in group:
                G = robust.bond_gate(pb, 0, k, b, tau)[0] @ G
            gg[b] = G
            mps.two_site_update(B, lam, b, G, 8, 1e-12)
        gl.append(gg)
        states.append([x.copy() for x in B])
    C, clam = mps.canonicalize(pb.targets[0], 8, 1e-12)
    vals = [mps.overlap(C, states[-1])]
    for li in range(len(sched) - 1, -1, -1):
        for b, G in gl[li].items():
            mps.two_site_update(C, clam, b, G.conj().T, 8, 1e-12)
        vals.append(mps.overlap(C, states[li]))
        # norms stay 1
        assert abs(mps.overlap(C, C) - 1) < 1e-12
    assert np.max(np.abs(np.array(vals) - vals[0])) < 1e-12


def test_identical_samples_give_single_sample_result():
    N, K, dt = 5, 3, 0.2
    rng = np.random.default_rng(95)
    u = rng.normal(0, 0.6, size=(K, 2, N))
    J1 = rng.uniform(-0.1, 0.1, size=(1, N - 1))
    ins = rand_products(N, 1, 96)
    tgs = synth.x_targets(ins)
    F1, g1, _ = robust.ensemble(mkpb(N, K, dt, 2, 8, u, synth.control_mask(2, N), J1, ins, tgs))
    F3, g3, _ = robust.ensemble(mkpb(N, K, dt, 2, 8, u, synth.control_mask(2, N), np.repeat(J1, 3, 0), ins, tgs))
    assert abs(F1 - F3) < 1e-15 and np.max(np.abs(g1 - g3)) < 1e-15


def test_truncated_fidelity_converges_in_chi():
    N, K, dt = 10, 6, 0.25
    rng = np.random.default_rng(97)
    u = rng.normal(0, 1.5, size=(K, 3, N))
    mask = synth.control_mask(3, N, "all")
    ins = rand_products(N, 1, 98)
    tgs = rand_products(N, 1, 99)
    J = rng.normal(0, 0.1, size=N - 1)
    o_exact, _ = dense.trajectory(mkpb(N, K, dt, 3, 32, u, mask, J, ins, tgs), 0, 0, False)
    errs = []
    for chi in (4, 8, 16, 32):
        o, _ = robust.trajectory(mkpb(N, K, dt, 3, chi, u, mask, J, ins, tgs), 0, 0, False)
        errs.append(abs(o - o_exact))
    assert errs[-1] < 1e-12
    assert errs[0] > errs[1] > errs[2] > errs[3]


# ------------------------------------------------------------------ canonical form
def test_canonical_form_of_random_mps():
    rng = np.random.default_rng(101)
    N, D = 6, 3
    dims = [1] + [D] * (N - 1) + [1]
    sites = [rng.normal(size=(dims[i], 2, dims[i + 1])) + 1j * rng.normal(size=(dims[i], 2, dims[i + 1]))
             for i in range(N)]
    v = dense.mps_vector(sites)
    B, lam = mps.canonicalize(sites, 64, 1e-12)
    w = mps.to_dense(B)
    assert abs(abs(np.vdot(v, w)) - 1.0) < 1e-13
    for i in range(1, N):
        b = B[i]
        gram = sum(b[:, s, :] @ b[:, s, :].conj().T for s in range(2))
        assert np.max(np.abs(gram - np.eye(b.shape[0]))) < 1e-13
    for bnd in range(N - 1):
        sv = np.linalg.svd(v.reshape(2 ** (bnd + 1), -1), compute_uv=False)
        assert np.max(np.abs(sv[:len(lam[bnd])] - lam[bnd])) < 1e-13


# --------------------------------------------------------------------- noise
def test_splitmix64_published_vectors():
    for line in open(os.path.join(GOLD, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, i, out = (int(x) for x in line.split())
        assert noise.splitmix64(seed, i) == out


def test_three_term_noise_uses_consecutive_counters():
    J3 = noise.sample_J(8, 4, 6, 0, 0.1, terms=3)
    flat = noise.sample_J(8, 4 * 3, 6, 0, 0.1)          # same stream, one term per "bond"
    assert J3.shape == (4, 5, 3)
    assert np.array_equal(J3.reshape(-1), flat.reshape(-1)[: 4 * 5 * 3])


def test_noise_distributions():
    J = noise.sample_J(5, 400, 51, 0, 0.1)
    assert J.shape == (400, 50) and np.all(np.abs(J) <= 0.1)
    assert abs(J.mean()) < 0.002 and abs(J.var() - 0.01 / 3) < 2e-4
    Jn = noise.sample_J(6, 400, 51, 1, 0.05)
    assert abs(Jn.mean()) < 0.002 and abs(Jn.std() - 0.05) < 0.002
    # bond (s, b) uses counter s*(N-1)+b: the stream is the same for a longer ensemble
    assert np.array_equal(noise.sample_J(5, 3, 51, 0, 0.1), J[:3])


# ------------------------------------------------------------------- targets
def _read_ghz_golden():
    rows = {}
    for line in open(os.path.join(GOLD, "ghz_sec4.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, s, r, c, v = line.split()
        rows[(kind, int(s), int(r), int(c))] = float(v)
    return rows


def test_ghz_mps_is_the_papers_and_is_ghz():
    gold = _read_ghz_golden()
    N = 7
    m = synth.ghz_mps(N)
    for (kind, s, r, c), v in gold.items():
        t = {"first": m.sites[0][0], "mid": m.sites[1], "last": m.sites[-1][:, :, 0]}[kind]
        if kind == "first":
            assert t[s, c] == v
        elif kind == "mid":
            assert t[r, s, c] == v
        else:
            assert t[r, s] == v
    psi = mps.to_dense(m.sites)
    assert abs(np.vdot(psi, psi) - 1) < 1e-15
    ref = np.zeros(2 ** N)
    ref[0] = ref[-1] = 2 ** -0.5
    assert np.max(np.abs(psi - ref)) < 1e-15


def test_cnot_targets_match_dense_cnots():
    N = 6
    ins = rand_products(N, 2, 111)
    tg = synth.cnot_targets(ins)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    for a, t in zip(ins, tg):
        v = dense.mps_vector(a.sites)
        for i in range(0, N, 2):
            v = dense.apply_two_site(v, cnot, i, N)
        w = mps.to_dense(t.sites)
        assert np.max(np.abs(v - w)) < 1e-15


def _heisenberg_dense(N):
    H = np.zeros((2 ** N, 2 ** N), dtype=complex)
    for b in range(N - 1):
        for P in (PX, PY, PZ):
            H += np.kron(np.kron(np.eye(2 ** b), np.kron(P, P)), np.eye(2 ** (N - b - 2)))
    return H


def test_heisenberg_ground_state():
    _, e2, _ = synth.heisenberg_ground_mps(2, 20)
    assert abs(e2 + 3.0) < 1e-12          # the singlet
    for N in (8, 10):
        m, e0, psi = synth.heisenberg_ground_mps(N, 64)
        w = np.linalg.eigvalsh(_heisenberg_dense(N))
        assert abs(e0 - w[0]) < 1e-9
        assert w[1] - w[0] > 1e-3        # unique ground state for even N
        v = mps.to_dense(m.sites)
        assert abs(abs(np.vdot(v, psi)) - 1) < 1e-10
    # compressed to D = 4 at N = 10: overlap >= 1 - discarded weight (loose)
    m4, _, psi = synth.heisenberg_ground_mps(10, 4)
    v4 = mps.to_dense(m4.sites)
    assert 0.9 < abs(np.vdot(v4, psi)) < 1.0


def test_per_gate_infidelity_printed_values():
    for line in open(os.path.join(GOLD, "per_gate_infidelity.txt")):
        if line.startswith("#") or not line.strip():
            continue
        gate, n, chib, printed = line.split()
        q = 1 if gate == "X" else 2
        val = robust.per_gate_infidelity(float(chib), int(n), q)
        assert abs(val - float(printed)) < 0.06 * float(printed)


# ------------------------------------------- truncation-gap diagnostic (Sec. II)
def _two_site_state(s, seed):
    """Two-site state with Schmidt values s (a 2x2 amplitude matrix U diag(s)
    V^dag), split as B_0 = U diag(s), B_1 = V^dag (the product B_0 B_1 is the
    amplitude matrix, as the oracle's two-site update reads it)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2)))
    V, _ = np.linalg.qr(rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2)))
    B = [(U * s).reshape(1, 2, 2), V.conj().T.reshape(2, 2, 1)]
    lam = [np.ones(2)]
    return B, lam


def test_gap_at_a_cap_decided_cut_is_the_schmidt_gap():
    """Keeping one of two Schmidt values (chi = 1) is a cut the cap decides:
    the gap is (s_1 - s_2) / s_1 of the known spectrum, and the discarded
    weight s_2^2 / (s_1^2 + s_2^2)."""
    s = np.array([0.8, 0.6])
    B, lam = _two_site_state(s, 3)
    info = {}
    w, k = mps.two_site_update(B, lam, 0, np.eye(4, dtype=complex), 1, 1e-12, info)
    assert k == 1
    assert abs(info["gap"] - (0.8 - 0.6) / 0.8) < 1e-14
    assert abs(w - 0.36) < 1e-14
    # the same state kept whole (chi = 2): no cut, no gap
    B, lam = _two_site_state(s, 3)
    info = {}
    w, k = mps.two_site_update(B, lam, 0, np.eye(4, dtype=complex), 2, 1e-12, info)
    assert k == 2 and info["gap"] is None and abs(w) < 1e-14


def test_no_gap_when_the_cutoff_decides():
    """A second Schmidt value below the cutoff is dropped by the cutoff, not the
    cap: no gap is reported even at chi = 1."""
    B, lam = _two_site_state(np.array([1.0, 1e-14]), 4)
    info = {}
    _, k = mps.two_site_update(B, lam, 0, np.eye(4, dtype=complex), 1, 1e-12, info)
    assert k == 1 and info["gap"] is None


def test_cut_statistics_are_the_count_and_minimum_of_the_gaps():
    """Over a trajectory the recorded cap cuts and their smallest gap are those
    of the individual updates (every update's gap collected separately)."""
    w = synth.WORKLOADS["ghz30"].replace(N=8, K=3, chi=4, M=1, P=1, u_sigma=1.5, dt=0.25)
    ins, tgs = w.states()
    u = w.controls()
    J = noise.sample_J(w.seed_J, w.M, w.N, w.noise_dist, w.noise_scale)
    pb = mkpb(w.N, w.K, w.dt, w.C, w.chi, u, w.mask(), J, ins, tgs)
    gaps = []
    orig = mps.two_site_update

    def spy(*a, **k):
        out = orig(*a, **k)
        info = a[6] if len(a) > 6 else k.get("info")
        if info is not None and info.get("gap") is not None:
            gaps.append(info["gap"])
        return out

    stats = {"discarded": 0.0, "dims": []}
    try:
        robust._m.two_site_update = spy
        robust.trajectory(pb, 0, 0, want_grad=True, stats=stats)
    finally:
        robust._m.two_site_update = orig
    assert len(gaps) > 0
    assert stats["cap_cuts"] == len(gaps)
    assert stats["min_gap"] == min(gaps)

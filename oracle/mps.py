"""Matrix-product-state primitives (Sec. II; TEBD after Vidal 2004 as the paper
cites it, in the right-canonical form of Hastings 2009).

A state is ``B`` (list of site tensors, shape (D_l, d, D_r)) plus ``lam``
(list of Schmidt-value vectors, lam[b] on bond b between sites b and b+1).
Amplitudes are psi(s_0 .. s_{N-1}) = B_0[s_0] B_1[s_1] ... B_{N-1}[s_{N-1}];
every B_i is a right isometry and lam[b] are the Schmidt values across bond b.
The physical dimension d is 2 for qubit states and 4 for operators written
as vectors (the MPO form of Sec. II: site index s = 2 out + in), read from
the tensors' shapes.

Truncation rule (Sec. II, "compressed ... to a predetermined maximum bond size
D_max using truncated SVD"): keep the k = min(chi, #{sigma_i > e sigma_1})
largest singular values (at least one), in LAPACK's descending order, then
renormalise the kept values to unit norm.  e = max(eps, 1e-13): singular
values at or below 1e-13 sigma_1 are numerically zero and always dropped.
"""
import numpy as np

#: relative level below which a singular value counts as numerically zero
ZERO_FLOOR = 1e-13


def _keep(S, chi, eps):
    if S[0] <= 0.0:
        raise FloatingPointError("zero state in truncation")
    k = int(np.count_nonzero(S > max(eps, ZERO_FLOOR) * S[0]))
    return max(1, min(chi, k))


def canonicalize(sites, chi, eps):
    """Bring an arbitrary MPS to normalised right-canonical form with Schmidt
    values.  Left sweep: SVDs make every site a left isometry (values at or
    below eps * sigma_1 are dropped as numerically zero).  Right sweep: the SVD
    of each site, with everything to its left left-isometric, gives the Schmidt
    values of the bond to its left; keep them by the truncation rule."""
    A = [np.array(s, dtype=np.complex128) for s in sites]
    N = len(A)
    for i in range(N - 1):
        dl, d, dr = A[i].shape
        U, S, Vh = np.linalg.svd(A[i].reshape(dl * d, dr), full_matrices=False)
        r = max(1, int(np.count_nonzero(S > max(eps, ZERO_FLOOR) * S[0])))
        A[i] = U[:, :r].reshape(dl, d, r)
        carry = S[:r, None] * Vh[:r]
        A[i + 1] = np.tensordot(carry, A[i + 1], axes=(1, 0))
    A[N - 1] = A[N - 1] / np.linalg.norm(A[N - 1])
    B = [None] * N
    lam = [None] * (N - 1)
    carry = np.ones((1, 1), dtype=np.complex128)
    for i in range(N - 1, 0, -1):
        M = np.tensordot(A[i], carry, axes=(2, 0))
        dl, d, dr = M.shape
        U, S, Vh = np.linalg.svd(M.reshape(dl, d * dr), full_matrices=False)
        k = _keep(S, chi, eps)
        nrm = np.linalg.norm(S[:k])
        B[i] = Vh[:k].reshape(k, d, dr)
        lam[i - 1] = S[:k] / nrm
        carry = U[:, :k] * (S[:k] / nrm)[None, :]
    M0 = np.tensordot(A[0], carry, axes=(2, 0))
    B[0] = M0 / np.linalg.norm(M0)
    return B, lam


def two_site_update(B, lam, b, G, chi, eps, info=None):
    """Apply the d^2 x d^2 gate G (basis |s_b s_{b+1}>) on bond b and truncate.

    theta = lam_{b-1} . G (B_b B_{b+1}) reshaped (d D_l) x (d D_r);
    theta = X S Y^dagger;  keep k values;  B_{b+1} <- Y_k^dagger,
    B_b <- Phi Y_k / ||S_k|| with Phi = G (B_b B_{b+1}) (no division by lam),
    lam_b <- S_k / ||S_k||.  Returns the discarded weight
    sum_{i>k} sigma_i^2 / sum_i sigma_i^2 and k.

    Diagnostic only: when ``info`` (a dict) is given, info["gap"] receives
    (sigma_k - sigma_{k+1}) / sigma_1 if the cap chi (not the cutoff) decided
    the cut -- more than chi values above the cutoff -- else None.  A gap near
    zero is a tie at the cut: the kept subspace is then not fixed by the
    singular values, and rounding decides it."""
    A, C = B[b], B[b + 1]
    dl, d, dr = A.shape[0], A.shape[1], C.shape[2]
    lam_l = lam[b - 1] if b > 0 else np.ones(1)
    AB = np.tensordot(A, C, axes=(2, 0))                       # (dl, d, d, dr)
    G4 = G.reshape(d, d, d, d)                                 # [s1 s2, s1' s2']
    Phi = np.einsum("xyuv,auvd->axyd", G4, AB)
    theta = lam_l[:, None, None, None] * Phi
    U, S, Vh = np.linalg.svd(theta.reshape(dl * d, d * dr), full_matrices=False)
    k = _keep(S, chi, eps)
    if info is not None:
        above = int(np.count_nonzero(S > max(eps, ZERO_FLOOR) * S[0]))
        info["gap"] = float((S[k - 1] - S[k]) / S[0]) if above > k else None
    nrm = np.linalg.norm(S[:k])
    Yk = Vh[:k].conj().T
    B[b + 1] = Vh[:k].reshape(k, d, dr)
    B[b] = (Phi.reshape(dl * d, d * dr) @ Yk / nrm).reshape(dl, d, k)
    lam[b] = S[:k] / nrm
    tot = float(np.sum(S ** 2))
    return float(np.sum(S[k:] ** 2)) / tot, k


def overlap(bra, ket):
    """<bra|ket> by a left-to-right transfer-matrix sweep."""
    E = np.ones((1, 1), dtype=np.complex128)
    for tb, ta in zip(bra, ket):
        E = np.einsum("ba,bsc,asd->cd", E, tb.conj(), ta)
    return complex(E[0, 0])


def mixed_two_site_density(bra, ket, b):
    """rho[s'_b s'_{b+1}, s_b s_{b+1}] = sum over all other sites of
    ket(.. s'_b s'_{b+1} ..) conj(bra(.. s_b s_{b+1} ..)), so that
    <bra| Q |ket> = trace(Q rho) for any d^2 x d^2 Q acting on sites b, b+1."""
    N = len(ket)
    L = np.ones((1, 1), dtype=np.complex128)
    for i in range(b):
        L = np.einsum("ba,bsc,asd->cd", L, bra[i].conj(), ket[i])
    R = np.ones((1, 1), dtype=np.complex128)
    for i in range(N - 1, b + 1, -1):
        R = np.einsum("bsc,cd,asd->ba", bra[i].conj(), R, ket[i])
    kb = np.tensordot(ket[b], ket[b + 1], axes=(2, 0))        # (Dal, d, d, Dar)
    bb = np.tensordot(bra[b], bra[b + 1], axes=(2, 0))        # (Dbl, d, d, Dbr)
    rho = np.einsum("ba,auvd,bxyc,cd->uvxy", L, kb, bb.conj(), R)
    d = ket[b].shape[1]
    return rho.reshape(d * d, d * d)


def to_dense(B):
    """Full state vector (site 0 the most significant digit)."""
    v = B[0].reshape(B[0].shape[1], -1)
    for t in B[1:]:
        v = np.tensordot(v, t, axes=(1, 0)).reshape(-1, t.shape[2])
    return v.reshape(-1)

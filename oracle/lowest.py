"""CPU FP64 oracle: lowest eigenstates of H by all-band CG (non-folded), and the
Gamma-point real-coefficient form.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module; only tests, the package's smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.

The paper's ground-state codes (Sec. II.A-B: PEtot, LS3DF) find the lowest
eigenstates of H by all-band conjugate-gradient minimisation.  The form here is
the same locally optimal block iteration as the folded solver, on H itself:
each iteration a Rayleigh-Ritz step of H over span{X, W, P}, with W the
preconditioned residuals H x_i - theta_i x_i (made orthogonal to X) and P the
previous update directions; basis selection by the eigenvectors of the scaled
overlap (near-dependent directions dropped).  Preconditioner 1 / (1 + |q|^2/2).

Gamma point (k = 0): V(r) and the projector functions are real, so
H[-G, -G'] = conj(H[G, G']) and the eigenvectors can be taken with
c(-G) = conj(c(G)) (real psi(r)).  The real coordinates
    c(0),  Re-part sqrt(2) Re c(G),  Im-part sqrt(2) Im c(G)   (one G of each +-G pair)
are an orthonormal change of basis in which H is a real symmetric matrix of
the same spectrum; the solver then runs in real arithmetic on half the data.
"""
from __future__ import annotations

import numpy as np

PARITY_PINS = """
lowest      : the nstates lowest eigenvalues equal LAPACK's on small boxes, residuals <= tol
gamma       : H[-G,-G'] = conj(H[G,G']) at k = 0; the real change of basis is orthonormal and
              makes H real symmetric with the same spectrum; the real-arithmetic solve finds the
              same lowest eigenvalues
planted     : a residual with the wrong sign (H x + theta x) no longer converges to them
"""


def _residual(HX, X, theta):
    """H x_i - theta_i x_i for the rows of X."""
    return HX - theta[:, None] * X


def _rr(S, HS, m, tau):
    """Rayleigh-Ritz of H on the rows of S (HS their images): the m lowest pairs."""
    GA = S.conj() @ HS.T
    GB = S.conj() @ S.T
    GA = 0.5 * (GA + GA.conj().T)
    GB = 0.5 * (GB + GB.conj().T)
    d = 1.0 / np.sqrt(np.real(np.diag(GB)))
    lam, U = np.linalg.eigh(d[:, None] * GB * d[None, :])
    keep = lam > tau * lam.max()
    T = (d[:, None] * U[:, keep]) / np.sqrt(lam[keep])[None, :]
    theta, C = np.linalg.eigh(T.conj().T @ GA @ T)
    return theta[:m], (T @ C[:, :m])


def lobpcg_lowest(apply, kin, nstates, tol, X0, guard=None, maxit=3000, tau=1e-11):
    """The nstates lowest eigenpairs of the Hermitian operator `apply` (rows in, rows
    out); kin is |q|^2/2 per coefficient for the preconditioner.  Returns eps, states
    [nstates][N], residual norms, iterations."""
    X = np.asarray(X0)
    m = X.shape[0]
    if guard is not None:
        m = min(m, nstates + guard)
        X = X[:m]
    M = 1.0 / (1.0 + kin)
    HX = apply(X)
    theta, C = _rr(X, HX, m, tau)
    X, HX = C.T @ X, C.T @ HX
    P = HP = None
    for it in range(maxit + 1):
        R = _residual(HX, X, theta)
        res = np.linalg.norm(R, axis=1)
        if np.all(res[:nstates] <= tol) or it == maxit:
            return theta[:nstates], X[:nstates], res[:nstates], it
        W = M[None, :] * R
        W = W - (W @ X.conj().T) @ X
        W /= np.linalg.norm(W, axis=1)[:, None]
        HW = apply(W)
        if P is None:
            S, HS = np.vstack([X, W]), np.vstack([HX, HW])
        else:
            S, HS = np.vstack([X, W, P]), np.vstack([HX, HW, HP])
        theta, C = _rr(S, HS, m, tau)
        Xn, HXn = C.T @ S, C.T @ HS
        P, HP = C[m:].T @ S[m:], C[m:].T @ HS[m:]
        nrm = np.linalg.norm(P, axis=1)
        P, HP = P / nrm[:, None], HP / nrm[:, None]
        X, HX = Xn, HXn


def gamma_pairs(g):
    """Index of -G for every G of a sphere symmetric under G -> -G."""
    pos = {tuple(v): i for i, v in enumerate(np.asarray(g))}
    return np.array([pos[tuple(-v)] for v in np.asarray(g)])


def gamma_real_basis(g):
    """Unitary T (columns = real coordinates in terms of the complex coefficients) with
    T^H H T real symmetric for a Gamma-point H: e_0 for G = 0 and, for each pair
    (G, -G) with G the first in sphere order, (e_G + e_-G)/sqrt(2) and
    i (e_G - e_-G)/sqrt(2)."""
    g = np.asarray(g)
    mate = gamma_pairs(g)
    N = g.shape[0]
    T = np.zeros((N, N), dtype=np.complex128)
    col = 0
    s = 1.0 / np.sqrt(2.0)
    for i in range(N):
        j = mate[i]
        if j == i:
            T[i, col] = 1.0
            col += 1
        elif i < j:
            T[i, col], T[j, col] = s, s
            T[i, col + 1], T[j, col + 1] = 1j * s, -1j * s
            col += 2
    return T

"""CPU FP64 oracle: the folded-spectrum all-band PCG eigensolve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module; only tests, the package's smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.

The paper (Sec. II.C) folds the spectrum of H about an energy E: the
operator A = (H - E)^2 is positive semidefinite, so a preconditioned
conjugate-gradient minimisation applies, and its lowest eigenvectors are the
eigenvectors of H whose eigenvalues lie nearest E (the spectral expansion in
Sec. II.C weights each eigenstate by 1/(eps_i - E)^2).  The paper names the
folded-spectrum eigen-method but prints no algorithm for it; the steps below
are the reading this project takes: all-band PCG in its locally optimal block
form (each iteration a Rayleigh-Ritz step on A over the bands, their
preconditioned residuals and their previous update directions), then a final
Rayleigh-Ritz step on H.  The G-space diagonal preconditioner is the paper's
M(G) = 1 / ((G^2 - E)^2 + dE^2) of Sec. II.C, taken in Hartree:
M(q) = 1 / ((|q|^2/2 - E)^2 + dE^2).

Everything is FP64 with plain NumPy/SciPy calls; no blocking or fusion.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .planewave import Hamiltonian


def _inner(a, b):
    """<a|b> for single vectors."""
    return np.vdot(a, b)


def cholesky_orthonormalise(X, *others):
    """X <- X L^-H with S = X^H X = L L^H (rows of X are bands).
    The same transform is applied to each block in ``others``."""
    S = X.conj() @ X.T                    # S_ij = <x_i, x_j>
    S = 0.5 * (S + S.conj().T)
    Lc = np.linalg.cholesky(S)            # S = L L^H
    T = np.linalg.inv(Lc).conj().T        # columns: new_j = sum_i x_i T_ij
    out = [T.T @ X] + [T.T @ O for O in others]
    return out


def rayleigh_ritz_A(X, Y, Z):
    """RR on A = (H-E)^2 in span X (orthonormal): G = Y^H Y, G = U diag(theta) U^H."""
    G = Y.conj() @ Y.T
    G = 0.5 * (G + G.conj().T)
    theta, U = np.linalg.eigh(G)
    return U.T @ X, U.T @ Y, U.T @ Z, theta


def precond_M(kin, e_ref, dE):
    return 1.0 / ((kin - e_ref) ** 2 + dE * dE)


def _orthonormalise_block(Wb, *others):
    """Cholesky QR of one block (rows are vectors); None when its Gram
    matrix is not numerically positive definite."""
    S = Wb.conj() @ Wb.T
    S = 0.5 * (S + S.conj().T)
    try:
        Lc = np.linalg.cholesky(S)
    except np.linalg.LinAlgError:
        return None
    T = np.linalg.inv(Lc).conj().T
    return [T.T @ Wb] + [T.T @ O for O in others]


def solve_folded(w, e_ref, nstates, tol, x0_raw, guard=None, dE=0.5, maxit=3000,
                 ham=None, callback=None, precond=None):
    """Folded-spectrum all-band PCG in its locally-optimal block form.

    Each iteration minimises the Rayleigh quotient of A = (H-E)^2 over
    span{X, W, P}: X the current bands, W = M(R) the preconditioned residuals
    R = A X - X Theta (made orthogonal to X), P the previous update
    directions (made orthogonal to X and W).  The Ritz vectors of the m lowest
    Ritz values of A become the new bands.  A band counts as converged when
    its H residual ||y - <x,y> x|| (y = (H-E) x) is <= tol; the run stops when
    the nstates lowest bands have converged, then a Rayleigh-Ritz step on H
    in span X gives the eigenvalues.

    Returns dict(eps, X, resid, iters, converged, theta, napply), eps ordered
    by (|eps - e_ref|, eps) and X[nstates][npw] the matching states.
    """
    h = ham if ham is not None else Hamiltonian(w)
    m = nstates + (max(4, nstates // 16) if guard is None else guard)
    E = e_ref
    M = precond_M(h.kin, E, dE) if precond is None else precond
    X = x0_raw[:m] * (1.0 / (1.0 + h.kin))[None, :]
    (X,) = cholesky_orthonormalise(X)
    Y = h.apply(X, E)
    Z = h.apply(Y, E)                          # Z = A X
    X, Y, Z, theta = rayleigh_ritz_A(X, Y, Z)
    P = YP = ZP = None
    converged = False
    it = 0
    for it in range(0, maxit + 1):
        resid = np.array([np.linalg.norm(Y[i] - _inner(X[i], Y[i]) * X[i]) for i in range(m)])
        if callback is not None:
            callback(it, theta, resid)
        if np.all(resid[:nstates] <= tol):
            converged = True
            break
        if it == maxit:
            break
        R = Z - theta[:, None] * X
        W = M[None, :] * R
        W = W - (X.conj() @ W.T).T @ X
        ow = _orthonormalise_block(W)
        if ow is None:
            break
        (W,) = ow
        YW = h.apply(W, E)
        ZW = h.apply(YW, E)
        blocks = [(X, Y, Z), (W, YW, ZW)]
        if P is not None:
            cx = X.conj() @ P.T                 # <x_i, p_j>
            cw = W.conj() @ P.T
            P = P - cx.T @ X - cw.T @ W
            YP = YP - cx.T @ Y - cw.T @ YW
            ZP = ZP - cx.T @ Z - cw.T @ ZW
            op = _orthonormalise_block(P, YP, ZP)
            if op is not None:
                P, YP, ZP = op
                blocks.append((P, YP, ZP))
        S = np.concatenate([b[0] for b in blocks])
        SY = np.concatenate([b[1] for b in blocks])
        SZ = np.concatenate([b[2] for b in blocks])
        GA = S.conj() @ SZ.T
        GB = S.conj() @ S.T
        GA = 0.5 * (GA + GA.conj().T)
        GB = 0.5 * (GB + GB.conj().T)
        theta, C = sla.eigh(GA, GB, subset_by_index=[0, m - 1])
        Cp = C.copy()
        Cp[:m] = 0.0
        P, YP, ZP = Cp.T @ S, Cp.T @ SY, Cp.T @ SZ
        X = C[:m].T @ X + P
        Y = C[:m].T @ Y + YP
        Z = C[:m].T @ Z + ZP
    # final Rayleigh-Ritz on H in span X
    Hs = X.conj() @ Y.T + E * np.eye(m)
    Hs = 0.5 * (Hs + Hs.conj().T)
    eps, U = np.linalg.eigh(Hs)
    X = U.T @ X
    Y = U.T @ Y
    res_all = np.array([np.linalg.norm(Y[i] - (eps[i] - E) * X[i]) for i in range(m)])
    order = np.lexsort((eps, np.abs(eps - E)))[:nstates]
    return dict(eps=eps[order], X=X[order], resid=res_all[order], iters=it,
                converged=converged, theta=theta, napply=h.napply)

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

This module is a fixed reference algorithm: it does not follow the tuning of
the CUDA solver (its locking, stall and precision rules), and a change to it
must be justified by the paper's text or by the mathematics alone.  The
arbiter of every solver result is the plain definition (the eigenpairs of H
nearest E by LAPACK brute force, or the golden spectrum of the wire), not
agreement with the iterations of this module.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .planewave import Hamiltonian


def _inner(a, b):
    """<a|b> for single vectors."""
    return np.vdot(a, b)


def precond_M(kin, e_ref, dE):
    return 1.0 / ((kin - e_ref) ** 2 + dE * dE)


def rayleigh_ritz_basis(S, SY, m, tau):
    """Rayleigh-Ritz of A on the rows of S (possibly near-dependent).

    G_A = <S, A S> taken as <(H-E)S, (H-E)S> = SY^H SY (SY = (H-E)S), the
    form that keeps the small Rayleigh quotients of A accurate in low
    precision; G_B = <S, S>.  The basis is first scaled to unit norm
    (D = diag(G_B)^-1/2), then orthonormalised through the eigenvectors of
    D G_B D, dropping every direction whose eigenvalue is <= tau times the
    largest (near-dependent vectors); the m lowest eigenpairs of the reduced
    G_A give the Ritz values theta and the coefficients C (rows of S -> new
    vectors, shape [len(S)][m]).
    """
    GA = SY.conj() @ SY.T
    GB = S.conj() @ S.T
    GA = 0.5 * (GA + GA.conj().T)
    GB = 0.5 * (GB + GB.conj().T)
    d = 1.0 / np.sqrt(np.real(np.diag(GB)))
    lam, U = np.linalg.eigh(d[:, None] * GB * d[None, :])
    keep = lam > tau * lam.max()
    T = (d[:, None] * U[:, keep]) / np.sqrt(lam[keep])[None, :]
    ga = T.conj().T @ GA @ T
    theta, Cr = np.linalg.eigh(0.5 * (ga + ga.conj().T))
    return theta[:m], T @ Cr[:, :m]


def residual_tolerance_A(theta, tol):
    """Per-band threshold on the A residual ||A x - theta x|| that matches an
    H residual of about tol: for an isolated eigenvector of H at distance
    d = sqrt(theta) from E the A residual is about 2 d times the H residual;
    the factor is floored at 1e-3 for states that sit on E."""
    return tol * np.maximum(np.sqrt(np.maximum(theta, 0.0)), 1e-3)


def h_ritz_check(X, Y, theta, E, nstates):
    """Rayleigh-Ritz step on H within the nstates lowest A-Ritz vectors (plus
    any band tied with the nstates-th within 1e-3 relative in theta): H-Ritz
    values eps, vectors and their H residuals ||H u - eps u||, nstates nearest
    E first (ordered by (|eps - E|, eps))."""
    n = nstates + int(np.sum(theta[nstates:] <= theta[nstates - 1] * (1.0 + 1e-3)))
    Hs = X[:n].conj() @ Y[:n].T
    lam, U = np.linalg.eigh(0.5 * (Hs + Hs.conj().T))
    Xr = U.T @ X[:n]
    Yr = U.T @ Y[:n]
    res = np.linalg.norm(Yr - lam[:, None] * Xr, axis=1)
    eps = lam + E
    order = np.lexsort((eps, np.abs(eps - E)))[:nstates]
    return eps[order], Xr[order], res[order]


def solve_folded(w, e_ref, nstates, tol, x0_raw, guard=None, dE=0.5, maxit=3000,
                 ham=None, callback=None, precond=None, tau=1e-10):
    """Folded-spectrum all-band PCG in its locally optimal block form.

    Each iteration minimises the Rayleigh quotient of A = (H-E)^2 over
    span{X, W, P}: X the current m bands (A-Ritz vectors, Ritz values theta),
    W = M(R) the preconditioned A residuals R = A X - X Theta of the bands that
    are not yet converged (made orthogonal to X), P their previous update
    directions (made orthogonal to X).  The Rayleigh-Ritz step selects its
    basis robustly (rayleigh_ritz_basis).  Convergence: once every wanted band
    (the nstates lowest theta) has an A residual below residual_tolerance_A, a
    Rayleigh-Ritz step on H within those bands (h_ritz_check) must give H
    residuals <= tol for the nstates pairs nearest E.

    Returns dict(eps, X, resid, iters, converged, theta, napply), eps ordered
    by (|eps - e_ref|, eps) and X[nstates][npw] the matching states.
    """
    h = ham if ham is not None else Hamiltonian(w)
    m = nstates + (max(4, nstates // 16) if guard is None else guard)
    E = e_ref
    M = precond_M(h.kin, E, dE) if precond is None else precond
    X = x0_raw[:m] * (1.0 / (1.0 + h.kin))[None, :]
    Y = h.apply(X, E)
    Z = h.apply(Y, E)                          # Z = A X
    theta, C = rayleigh_ritz_basis(X, Y, m, tau)
    X, Y, Z = C.T @ X, C.T @ Y, C.T @ Z
    P = YP = ZP = None
    converged = False
    it = 0
    eps = states = res = None
    for it in range(0, maxit + 1):
        R = Z - theta[:, None] * X
        ra = np.linalg.norm(R, axis=1)
        tolA = residual_tolerance_A(theta, tol)
        if callback is not None:
            callback(it, theta, ra)
        if np.all(ra[:nstates] <= tolA[:nstates]):
            eps, states, res = h_ritz_check(X, Y, theta, E, nstates)
            if np.all(res <= tol):
                converged = True
                break
        if it == maxit:
            break
        # soft locking: a band stops contributing directions once its A residual
        # is below its threshold
        act = np.where(ra > tolA)[0]
        if act.size == 0:
            act = np.arange(m)
        W = M[None, :] * R[act]
        W = W - (X.conj() @ W.T).T @ X
        W = W / np.linalg.norm(W, axis=1)[:, None]
        YW = h.apply(W, E)
        ZW = h.apply(YW, E)
        blocks = [(X, Y, Z), (W, YW, ZW)]
        if P is not None:
            Pa, YPa, ZPa = P[act], YP[act], ZP[act]
            cx = X.conj() @ Pa.T                 # <x_i, p_j>
            Pa = Pa - cx.T @ X
            YPa = YPa - cx.T @ Y
            ZPa = ZPa - cx.T @ Z
            nrm = np.linalg.norm(Pa, axis=1)
            blocks.append((Pa / nrm[:, None], YPa / nrm[:, None], ZPa / nrm[:, None]))
        S = np.concatenate([b[0] for b in blocks])
        SY = np.concatenate([b[1] for b in blocks])
        SZ = np.concatenate([b[2] for b in blocks])
        theta, C = rayleigh_ritz_basis(S, SY, m, tau)
        Cp = C.copy()
        Cp[:m] = 0.0
        P, YP, ZP = Cp.T @ S, Cp.T @ SY, Cp.T @ SZ
        X = C[:m].T @ X + P
        Y = C[:m].T @ Y + YP
        Z = C[:m].T @ Z + ZP
    if eps is None or not converged:
        eps, states, res = h_ritz_check(X, Y, theta, E, nstates)
    return dict(eps=eps, X=states, resid=res, iters=it, converged=converged, theta=theta,
                napply=h.napply)

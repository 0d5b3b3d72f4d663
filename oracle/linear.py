"""CPU FP64 oracle: the folded-spectrum linear solve with the eigenstate preconditioner.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module; only tests, the package's smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.

Sec. II.C: the scattering-state equation (H - E) psi = w (Eq. wl) has an
indefinite operator; applying (H - E) on both sides gives Eq. wl1,

    (H - E)^2 psi = (H - E) w = w',

whose operator is positive definite, solved by a preconditioned conjugate
gradient minimisation of F = 1/2 <psi|(H - E)^2|psi> - Re<psi|w'> (the paper
prints the linear term with w; its gradient vanishes at the solution of
Eq. wl1 only with w', the reading taken here).  The paper measures the error
as ||(H - E) psi - w||.  The solution has the spectral expansion

    psi = sum_i <phi_i|w'> / (eps_i - E)^2  phi_i        (over all eigenpairs of H),

and a set of approximate eigenpairs (phi_i, eps_i) with residuals
Delta_i = ||H phi_i - eps_i phi_i|| near E builds the preconditioner

    M' = M (1 - sum_i |phi_i><phi_i|) + sum_i |phi_i><phi_i| / ((eps_i - E)^2 + Delta_i^2),

M(G) the G-space diagonal 1 / ((|q|^2/2 - E)^2 + dE^2) (Hartree reading of the
paper's M(G)).  M' is applied exactly as written (it is not Hermitian when M
is not constant); the conjugate directions use the Polak-Ribiere coefficient
(clamped at zero), which tolerates that.

PCG for every right-hand side l independently (rows of W):
  psi_0 = 0, r_0 = w' - A psi_0, z_0 = M' r_0, p_0 = z_0;
  alpha = Re<r, z> / Re<p, A p>;  psi += alpha p;  r -= alpha A p;
  z' = M' r;  beta = max(0, Re<z', r - r_old> / Re<z_old, r_old>);  p = z' + beta p.
Stop when ||(H - E) psi - w|| <= tol.

Everything is FP64 with plain NumPy; A p is (H - E) applied twice.
"""
from __future__ import annotations

import numpy as np

from .folded import precond_M

PARITY_PINS = """
spectral    : the PCG solution equals the spectral expansion over all eigenpairs of the
              dense H (and numpy.linalg.solve of (H - E) psi = w) on small boxes
M'          : M' phi_j = phi_j / (eps_j - E)^2 for exact eigenvectors (Delta = 0);
              M' r = M r for r orthogonal to the phi_i; a planted mistake (the -M P term
              dropped) breaks the first
acceleration: with M' from the exact eigenstates nearest E the PCG needs fewer iterations
              than with M alone (the effect the paper reports in Sec. II.C)
"""


def spectral_solution(H, e_ref, W):
    """psi_l = sum_i <phi_i|w'_l> / (eps_i - E)^2 phi_i over every eigenpair of the
    dense Hermitian H; W is [nrhs][N]."""
    eps, V = np.linalg.eigh(H)
    Wp = (H - e_ref * np.eye(H.shape[0])) @ W.T          # w'_l as columns
    coef = (V.conj().T @ Wp) / ((eps - e_ref) ** 2)[:, None]
    return (V @ coef).T


def apply_mprime(kin, e_ref, dE, R, phi=None, eps=None, delta=None):
    """M' r for the rows of R: M (r - sum_i phi_i <phi_i|r>) + sum_i phi_i <phi_i|r> c_i,
    c_i = 1 / ((eps_i - E)^2 + Delta_i^2); M alone when phi is None."""
    M = precond_M(kin, e_ref, dE)
    if phi is None or len(phi) == 0:
        return M[None, :] * R
    T = phi.conj() @ R.T                                  # <phi_i|r_l>, [n][nrhs]
    c = 1.0 / ((np.asarray(eps) - e_ref) ** 2 + np.asarray(delta) ** 2)
    return M[None, :] * _project_out(R, phi, T) + (phi.T @ (c[:, None] * T)).T


def _project_out(R, phi, T):
    """r - sum_i phi_i <phi_i|r> for the rows of R, with T = <phi_i|r_l>."""
    return R - (phi.T @ T).T


def pcg_folded(ham, e_ref, W, tol, dE=0.5, phi=None, eps=None, delta=None, maxit=20000):
    """Solve (H - E)^2 psi = (H - E) w for every row w of W by the PCG above.
    Returns psi [nrhs][N], the iterations taken and the final errors
    ||(H - E) psi - w|| (recomputed from psi)."""
    W = np.atleast_2d(np.asarray(W, dtype=np.complex128))
    nrhs = W.shape[0]
    kin = ham.kin
    psi = np.zeros_like(W)
    Y = np.zeros_like(W)                                  # (H - E) psi, carried by linearity
    R = ham.apply(W, e_ref)                               # w' - A psi_0 = (H - E) w with psi_0 = 0
    Z = apply_mprime(kin, e_ref, dE, R, phi, eps, delta)
    P = Z.copy()
    zr = np.real(np.sum(Z.conj() * R, axis=1))
    done = np.zeros(nrhs, dtype=bool)
    it = 0
    while it < maxit:
        YP = ham.apply(P, e_ref)
        AP = ham.apply(YP, e_ref)
        pap = np.real(np.sum(P.conj() * AP, axis=1))
        alpha = np.where(done, 0.0, zr / np.where(pap != 0, pap, 1.0))
        R_old = R
        psi = psi + alpha[:, None] * P
        Y = Y + alpha[:, None] * YP
        R = R - alpha[:, None] * AP
        it += 1
        err = np.linalg.norm(Y - W, axis=1)
        done = done | (err <= tol)
        if np.all(done):
            break
        Z_new = apply_mprime(kin, e_ref, dE, R, phi, eps, delta)
        zr_new = np.real(np.sum(Z_new.conj() * R, axis=1))
        zro = np.real(np.sum(Z_new.conj() * R_old, axis=1))
        beta = np.where(done, 0.0, np.maximum(0.0, (zr_new - zro) / np.where(zr != 0, zr, 1.0)))
        P = Z_new + beta[:, None] * P
        zr = zr_new
    err = np.linalg.norm(ham.apply(psi, e_ref) - W, axis=1)
    return psi, it, err

"""CPU FP64 oracle: Chebyshev filter diagonalisation (ChebFD) for the states in an
energy window around E.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module; only tests, the package's smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.

Sec. II.C: a polynomial p(H), a combination of Chebyshev polynomials, imitates
a window function around E; applied to a block of random vectors it keeps the
components of the eigenstates inside the window and suppresses the others; a
subspace diagonalisation of <phi'_i|H|phi'_j> then gives the states of the
step, and the step is repeated on them.  The filter used here is the standard
window filter of the methods the paper cites (kernel-polynomial expansion with
Jackson damping):

  spectrum mapped to [-1, 1]:  Hs = (H - c) / e,  c = (emax + emin) / 2,  e = (emax - emin) / 2;
  window [E - d, E + d]  ->  [t1, t2],  theta_k = arccos t_k;
  mu_0 = (theta_1 - theta_2) / pi,   mu_n = 2 (sin n theta_1 - sin n theta_2) / (n pi)   (n >= 1)
  (the Chebyshev coefficients of the indicator of [t1, t2]);
  g_n = ((N - n + 1) cos(pi n / (N + 1)) + sin(pi n / (N + 1)) cot(pi / (N + 1))) / (N + 1)
  (Jackson damping for degree N);
  p(Hs) X = sum_{n=0}^{N} g_n mu_n T_n(Hs) X,  T_0 X = X,  T_1 X = Hs X,  T_{n+1} = 2 Hs T_n - T_{n-1}.

One step: Y = p(Hs) X; Rayleigh-Ritz of H on the columns of Y (basis from the
eigenvectors of Y^H Y, dropping eigenvalues below 1e-12 of the largest); X =
the Ritz vectors.  Reported: the Ritz pairs inside the window, ordered by
(|eps - E|, eps), with Delta_i = ||H phi_i - eps_i phi_i||.
"""
from __future__ import annotations

import numpy as np

PARITY_PINS = """
coefficients: mu_n against numerical quadrature of the Chebyshev projection of the
              window; the Jackson-damped filter stays within [0, 1] on [-1, 1]
filter      : p(Hs) phi = p(eps_s) phi for exact eigenvectors (scalar evaluation of the
              same series); a planted sign error in the recurrence breaks it
window      : the eigenvalues found inside the window equal LAPACK's on small boxes
"""


def jackson(N):
    n = np.arange(N + 1)
    a = np.pi / (N + 1)
    return ((N - n + 1) * np.cos(a * n) + np.sin(a * n) / np.tan(a)) / (N + 1)


def window_coefficients(t1, t2, N):
    """mu_n g_n for the indicator of [t1, t2] inside [-1, 1], n = 0..N."""
    th1, th2 = np.arccos(np.clip(t1, -1, 1)), np.arccos(np.clip(t2, -1, 1))
    n = np.arange(1, N + 1)
    mu = np.empty(N + 1)
    mu[0] = (th1 - th2) / np.pi
    mu[1:] = 2.0 * (np.sin(n * th1) - np.sin(n * th2)) / (n * np.pi)
    return mu * jackson(N)


def eval_series(coef, x):
    """sum_n coef_n T_n(x) for scalars or arrays x in [-1, 1] (T_n(x) = cos(n arccos x))."""
    th = np.arccos(np.clip(np.asarray(x, dtype=np.float64), -1, 1))
    n = np.arange(len(coef))
    return np.cos(np.multiply.outer(th, n)) @ coef


def _step(T_cur, HsT, T_prev):
    """T_{n+1} from Hs T_n and T_{n-1}."""
    return 2.0 * HsT - T_prev


def apply_filter(ham, X, c, e, coef):
    """p(Hs) X for the rows of X, Hs = (H - c) / e."""
    X = np.atleast_2d(np.asarray(X, dtype=np.complex128))
    Y = coef[0] * X
    if len(coef) == 1:
        return Y
    T_prev, T_cur = X, ham.apply(X, c) / e
    Y = Y + coef[1] * T_cur
    for n in range(2, len(coef)):
        T_next = _step(T_cur, ham.apply(T_cur, c) / e, T_prev)
        Y = Y + coef[n] * T_next
        T_prev, T_cur = T_cur, T_next
    return Y


def rayleigh_ritz_H(ham, Y, tau=1e-12):
    """Ritz pairs of H on the rows of Y: eigenvalues, vectors [k][N], residual norms."""
    GB = Y.conj() @ Y.T
    HY = ham.apply(Y, 0.0)
    GA = Y.conj() @ HY.T
    lam, U = np.linalg.eigh(0.5 * (GB + GB.conj().T))
    keep = lam > tau * lam.max()
    T = U[:, keep] / np.sqrt(lam[keep])[None, :]
    eps, C = np.linalg.eigh(T.conj().T @ (0.5 * (GA + GA.conj().T)) @ T)
    V = (T @ C).T @ Y
    HV = (T @ C).T @ HY
    res = np.linalg.norm(HV - eps[:, None] * V, axis=1)
    return eps, V, res


def chebfd(ham, e_ref, half_width, emin, emax, degree, X0, steps):
    """ChebFD steps from the start block X0 [nvec][N]; returns the Ritz pairs inside
    [E - d, E + d] ordered by (|eps - E|, eps): eps, states [k][N], residuals."""
    c, e = 0.5 * (emax + emin), 0.5 * (emax - emin)
    coef = window_coefficients((e_ref - half_width - c) / e, (e_ref + half_width - c) / e, degree)
    X = np.asarray(X0, dtype=np.complex128)
    for _ in range(steps):
        Y = apply_filter(ham, X, c, e, coef)
        eps, X, res = rayleigh_ritz_H(ham, Y)
    inside = np.abs(eps - e_ref) <= half_width
    eps, X, res = eps[inside], X[inside], res[inside]
    order = np.lexsort((eps, np.abs(eps - e_ref)))
    return eps[order], X[order], res[order]

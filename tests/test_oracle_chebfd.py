"""Pins of the ChebFD oracle (Sec. II.C: a Chebyshev polynomial window filter
followed by subspace diagonalisation) against quadrature, the eigen-
decomposition of the dense H and LAPACK's eigenvalues."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import fs_inputs as fi  # noqa: E402
from oracle import chebfd as cf  # noqa: E402
from oracle import planewave as pw  # noqa: E402


def _box():
    return fi.make_box(L=(10.0, 10.0, 20.0), n=(16, 16, 32), ecut=5.0, natom=4, widths=(1.0,), nstates=6,
                       e_ref=0.3, seed=3)


def _bounds(eps):
    return eps[0] - 0.05, eps[-1] + 0.05


def test_window_coefficients_match_quadrature():
    from numpy.polynomial import chebyshev as C
    from scipy.integrate import quad
    t1, t2, N = -0.37, 0.21, 30
    mu = cf.window_coefficients(t1, t2, N) / cf.jackson(N)
    for n in (0, 1, 2, 7, 30):
        e = np.zeros(n + 1)
        e[n] = 1.0
        val, _ = quad(lambda x: C.chebval(x, e) / np.sqrt(1.0 - x * x), t1, t2, epsabs=1e-13, epsrel=1e-13)
        want = val / np.pi if n == 0 else 2.0 * val / np.pi
        assert mu[n] == pytest.approx(want, abs=1e-11)


def test_jackson_filter_stays_in_unit_interval():
    coef = cf.window_coefficients(-0.1, 0.1, 400)
    x = np.linspace(-1, 1, 4001)
    p = cf.eval_series(coef, x)
    assert p.min() >= -1e-12 and p.max() <= 1 + 1e-12
    assert cf.eval_series(coef, 0.0) > 0.99
    assert np.abs(p[np.abs(x) > 0.2]).max() < 1e-3


def _filter_pin_error(w):
    h = pw.Hamiltonian(w)
    eps, V = np.linalg.eigh(pw.dense_H(w))
    a, b = _bounds(eps)
    c, e = 0.5 * (a + b), 0.5 * (b - a)
    coef = cf.window_coefficients((0.25 - c) / e, (0.35 - c) / e, 50)
    pick = [0, 5, 17, 40]
    Y = cf.apply_filter(h, V[:, pick].T, c, e, coef)
    want = cf.eval_series(coef, (eps[pick] - c) / e)[:, None] * V[:, pick].T
    return np.abs(Y - want).max() / np.abs(V[:, pick]).max()


def test_filter_acts_on_eigenvectors_as_the_scalar_series():
    assert _filter_pin_error(_box()) <= 1e-10


def test_pin_catches_recurrence_sign(monkeypatch):
    """Plant a sign error in the oracle's three-term recurrence: the eigenvector pin fails."""
    monkeypatch.setattr(cf, "_step", lambda T_cur, HsT, T_prev: 2.0 * HsT + T_prev)
    assert _filter_pin_error(_box()) > 1e-3


def test_chebfd_finds_the_window_eigenvalues():
    """Every eigenvalue well inside the window is found to 1e-9 with a small
    residual; every reported pair with a small residual is an eigenpair.  Pairs
    with a large residual ("ghost states", which the paper also meets) may be
    reported and carry their residual."""
    w = _box()
    h = pw.Hamiltonian(w)
    eps_all = np.linalg.eigvalsh(pw.dense_H(w))
    a, b = _bounds(eps_all)
    E, d = w.e_ref, 0.045
    X0 = fi.raw_start_block(24, h.npw, 9)
    eps, X, res = cf.chebfd(h, E, d, a, b, degree=300, X0=X0, steps=4)
    deep = eps_all[np.abs(eps_all - E) <= 0.8 * d]
    assert len(deep) >= 4
    for x in deep:
        i = np.argmin(np.abs(eps - x))
        assert abs(eps[i] - x) <= 1e-9 and res[i] <= 1e-8
    for x, r in zip(eps, res):
        if r <= 1e-6:
            assert np.min(np.abs(eps_all - x)) <= 1e-9
    assert np.all(np.abs(eps - E) <= d)
    assert np.all(np.diff(np.abs(eps - E)) >= -1e-15)
    # the states come back orthonormal
    assert np.abs(X.conj() @ X.T - np.eye(len(eps))).max() <= 1e-10

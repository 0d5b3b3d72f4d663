"""Pins of the lowest-state (non-folded) all-band CG oracle and its Gamma-point
real form against LAPACK and the symmetry of the synthetic H at k = 0."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import fs_inputs as fi  # noqa: E402
from oracle import lowest as lo  # noqa: E402
from oracle import planewave as pw  # noqa: E402


def _box(k=(0.0, 0.0, 0.0)):
    return fi.make_box(L=(10.0, 10.0, 20.0), n=(16, 16, 32), ecut=5.0, k=k, natom=4, widths=(1.0,), nstates=10,
                       e_ref=0.3, seed=3)


def _solve(w, nstates=10, tol=1e-8):
    h = pw.Hamiltonian(w)
    X0 = fi.raw_start_block(nstates + 4, h.npw, 17)
    return lo.lobpcg_lowest(lambda X: h.apply(X, 0.0), h.kin, nstates, tol, X0, maxit=400)


def test_lowest_states_match_lapack():
    w = _box(k=(0.1, -0.05, 0.2))
    eps, X, res, it = _solve(w)
    ref = np.linalg.eigvalsh(pw.dense_H(w))[:10]
    assert np.all(res <= 1e-8)
    assert np.abs(eps - ref).max() <= 1e-9
    assert it < 400


def test_pin_catches_residual_sign(monkeypatch):
    monkeypatch.setattr(lo, "_residual", lambda HX, X, theta: HX + theta[:, None] * X)
    w = _box(k=(0.1, -0.05, 0.2))
    eps, X, res, it = _solve(w)
    ref = np.linalg.eigvalsh(pw.dense_H(w))[:10]
    assert not (np.all(res <= 1e-8) and np.abs(eps - ref).max() <= 1e-9)


def test_gamma_point_time_reversal_and_real_form():
    w = _box()
    g, _ = pw.sphere(w.L, w.n, w.ecut, w.k)
    H = pw.dense_H(w)
    mate = lo.gamma_pairs(g)
    assert np.abs(H[np.ix_(mate, mate)] - H.conj()).max() <= 1e-12
    T = lo.gamma_real_basis(g)
    assert np.abs(T.conj().T @ T - np.eye(T.shape[0])).max() <= 1e-12
    Hr = T.conj().T @ H @ T
    assert np.abs(Hr.imag).max() <= 1e-12
    assert np.abs(np.linalg.eigvalsh(Hr.real) - np.linalg.eigvalsh(H)).max() <= 1e-10


def test_gamma_real_arithmetic_solve():
    """The solve in the real coordinates (real arithmetic) finds the lowest
    eigenvalues of the complex H."""
    w = _box()
    g, _ = pw.sphere(w.L, w.n, w.ecut, w.k)
    h = pw.Hamiltonian(w)
    T = lo.gamma_real_basis(g)
    Hr = (T.conj().T @ pw.dense_H(w) @ T).real
    kin_r = np.real(np.diag(T.conj().T @ np.diag(h.kin) @ T))
    rng = np.random.default_rng(4)
    X0 = rng.normal(size=(14, h.npw))
    eps, X, res, it = lo.lobpcg_lowest(lambda X: X @ Hr.T, kin_r, 10, 1e-8, X0, maxit=400)
    assert np.isrealobj(X)
    assert np.all(res <= 1e-8)
    assert np.abs(eps - np.linalg.eigvalsh(pw.dense_H(w))[:10]).max() <= 1e-9

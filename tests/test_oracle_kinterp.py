"""Pins of the wave-function interpolation oracle (Sec. II.D): with a complete
basis it reproduces the eigenvalues of the linearly interpolated Hamiltonian
built densely; alpha = 1 returns the k1 eigenvalues; the Gram-Schmidt U is
unitary and triangular in S; a planted transposition of U is caught."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import fs_inputs as fi  # noqa: E402
from oracle import kinterp as ki  # noqa: E402

K1, K2 = (0.0, 0.0, 0.05), (0.0, 0.0, 0.15)


def _hams(gmax=2.2):
    w = fi.make_box(L=(10.0, 10.0, 20.0), n=(16, 16, 32), ecut=5.0, natom=4, widths=(1.0,), nstates=6,
                    e_ref=0.3, seed=3)
    H1, g = ki.dense_H_common(w, K1, gmax)
    H2, _ = ki.dense_H_common(w, K2, gmax)
    return w, H1, H2, g


def _eig(H):
    e, V = np.linalg.eigh(H)
    return e, V.T.copy()


def _complete_error(interp=ki.interpolate):
    _, H1, H2, _ = _hams()
    e1, p1 = _eig(H1)
    e2, p2 = _eig(H2)
    worst = 0.0
    for alpha in (0.0, 0.3, 0.7, 1.0):
        e, _ = interp(alpha, e1, p1, e2, p2)
        ref = np.linalg.eigvalsh(alpha * H1 + (1 - alpha) * H2)
        worst = max(worst, np.abs(e - ref).max())
    return worst


def test_complete_basis_reproduces_the_interpolated_hamiltonian():
    assert _complete_error() <= 1e-10


def test_pin_catches_transposed_u(monkeypatch):
    real = ki.gram_schmidt_rows
    monkeypatch.setattr(ki, "gram_schmidt_rows", lambda S: real(S).T)
    assert _complete_error() > 1e-4


def test_alpha_one_returns_the_k1_states():
    _, H1, H2, _ = _hams()
    e1, p1 = _eig(H1)
    e2, p2 = _eig(H2)
    n = 20
    e, psi = ki.interpolate(1.0, e1[:n], p1[:n], e2[:n], p2[:n])
    assert np.abs(e - e1[:n]).max() <= 1e-12
    # each returned state is an eigenvector of H(k1)
    r = np.linalg.norm(psi @ H1.T - e[:, None] * psi, axis=1)
    assert r.max() <= 1e-9


def test_gram_schmidt_is_unitary_and_triangular_in_s():
    rng = np.random.default_rng(5)
    S = rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12))
    U = ki.gram_schmidt_rows(S)
    assert np.abs(U @ U.conj().T - np.eye(12)).max() <= 1e-12
    L = U @ np.linalg.inv(S)
    assert np.abs(np.triu(L, 1)).max() <= 1e-10


def test_truncated_interpolation_tracks_the_midpoint_bands():
    """The 20 lowest states of each k-point interpolate the lowest bands at the
    midpoint to within the quadratic error of linear interpolation in k
    (alpha (1 - alpha) (k1 - k2)^2 / 2 on the kinetic term) plus truncation."""
    w, H1, H2, _ = _hams()
    e1, p1 = _eig(H1)
    e2, p2 = _eig(H2)
    n = 20
    e, _ = ki.interpolate(0.5, e1[:n], p1[:n], e2[:n], p2[:n])
    Hm, _ = ki.dense_H_common(w, (0.0, 0.0, 0.10), 2.2)
    ref = np.linalg.eigvalsh(Hm)[:6]
    assert np.abs(e[:6] - ref).max() <= 2e-3

"""Parity of the GPU Chebyshev filter diagonalisation (Sec. II.C) with LAPACK
and the CPU oracle: the eigenvalues inside the window, the states' residuals
recomputed by the oracle, the spectral-bound estimate, and the states as the
M' preconditioner of the folded linear solve."""
import numpy as np
import pytest

import fs_inputs as fi
from oracle import planewave as pw

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    from paper_1907_06821_gb300 import build as b
    b.build()
    import paper_1907_06821_gb300 as m
    return m


def _box():
    return fi.make_box(L=(10.0, 10.0, 20.0), n=(16, 16, 32), ecut=5.0, natom=4, widths=(1.0,), nstates=6,
                       e_ref=0.3, seed=3)


def test_chebfd_finds_the_window_eigenvalues(fs):
    w = _box()
    h = pw.Hamiltonian(w)
    eps_all = np.linalg.eigvalsh(pw.dense_H(w))
    a, b = eps_all[0] - 0.05, eps_all[-1] + 0.05
    E, d = w.e_ref, 0.045
    with fs.Context.from_workload(w) as c:
        r = c.chebfd(E, d, a, b, degree=300, nvec=24, steps=4, seed=9)
        X = c.get_states(r["nfound"])
    eps, res = r["eps"], r["resid"]
    deep = eps_all[np.abs(eps_all - E) <= 0.8 * d]
    assert len(deep) >= 4
    for x in deep:
        i = np.argmin(np.abs(eps - x))
        assert abs(eps[i] - x) <= 1e-9 and res[i] <= 1e-8
    good = res <= 1e-6
    for x in eps[good]:
        assert np.min(np.abs(eps_all - x)) <= 1e-9
    assert np.all(np.abs(eps - E) <= d)
    assert np.all(np.diff(np.abs(eps - E)) >= -1e-15)
    # the oracle's residuals of the returned states agree with the reported ones
    ro = np.linalg.norm(h.apply(X, 0.0) - eps[:, None] * X, axis=1)
    assert np.allclose(ro[good], res[good], rtol=0, atol=1e-9)
    assert np.abs(X[good].conj() @ X[good].T - np.eye(int(good.sum()))).max() <= 1e-10


def test_spectral_bounds_bracket_the_spectrum(fs):
    w = _box()
    eps_all = np.linalg.eigvalsh(pw.dense_H(w))
    with fs.Context.from_workload(w) as c:
        lo, hi = c.spectral_bounds(40)
    assert lo <= eps_all[0] and hi >= eps_all[-1]
    assert hi - lo <= 1.5 * (eps_all[-1] - eps_all[0])


def test_chebfd_states_precondition_the_linear_solve(fs):
    w = _box()
    h = pw.Hamiltonian(w)
    W = fi.wavepacket_rhs(h.g, w.L, [(5.0, 5.0, 6.0), (4.0, 6.0, 14.0)])
    with fs.Context.from_workload(w) as c:
        lo, hi = c.spectral_bounds(40)
        r = c.chebfd(w.e_ref, 0.045, lo, hi, degree=300, nvec=24, steps=4, seed=9)
        _, im = c.linear_solve(W, w.e_ref, tol=1e-9)
        c.set_linear_states(r["nfound"])
        _, ip = c.linear_solve(W, w.e_ref, tol=1e-9)
    assert r["nfound"] >= 4
    assert np.all(im["err"] <= 1e-9) and np.all(ip["err"] <= 1e-9)
    assert ip["iters"] < im["iters"]

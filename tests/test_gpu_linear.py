"""Parity of the folded-spectrum linear solve (Sec. II.C, Eq. wl1 with the M'
preconditioner) through the C ABI with the CPU FP64 oracle.  What decides the
result is the spectral expansion of the solution over every eigenpair of the
dense H (LAPACK); the eigenstate preconditioner built from the library's own
eigensolve must cut the iteration count.  The oracle's PCG iteration counts
are a sanity bound only (the library may take fewer steps, not many more)."""
import numpy as np
import pytest

import fs_inputs as fi
from oracle import linear as lin
from oracle import planewave as pw

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def fs():
    from paper_1907_06821_gb300 import build as b
    b.build()
    import paper_1907_06821_gb300 as m
    return m


def _box():
    return fi.make_box(L=(10.0, 10.0, 20.0), n=(16, 16, 32), ecut=5.0, natom=4, widths=(1.0,), nstates=8,
                       e_ref=0.3, seed=3)


def _rhs(w, h):
    return fi.wavepacket_rhs(h.g, w.L, [(5.0, 5.0, 6.0), (4.0, 6.0, 14.0), (6.0, 4.5, 10.0)])


def test_linear_solve_matches_spectral_expansion(fs):
    w = _box()
    h = pw.Hamiltonian(w)
    W = _rhs(w, h)
    ref = lin.spectral_solution(pw.dense_H(w), w.e_ref, W)
    _, it_o, _ = lin.pcg_folded(h, w.e_ref, W, tol=TOL)
    with fs.Context.from_workload(w) as c:
        psi, info = c.linear_solve(W, w.e_ref, tol=TOL)
    assert np.all(info["err"] <= TOL)
    assert np.linalg.norm(psi - ref) <= 1e-7 * np.linalg.norm(ref)
    assert info["iters"] <= 1.5 * it_o + 3
    assert info["n_hpsi"] >= 2 * info["iters"] * W.shape[0]


def test_eigenstate_preconditioner_from_the_solver(fs):
    w = _box()
    h = pw.Hamiltonian(w)
    W = _rhs(w, h)
    ref = lin.spectral_solution(pw.dense_H(w), w.e_ref, W)
    with fs.Context.from_workload(w) as c:
        c.set_initial_states(fi.raw_start_block(w.nbands, c.npw, 17), damp=True)
        r = c.solve(w.e_ref, w.nstates, tol=1e-8)
        phi = c.get_states(w.nstates)
        psi_m, im = c.linear_solve(W, w.e_ref, tol=TOL)
        c.set_linear_states(w.nstates)
        psi_p, ip = c.linear_solve(W, w.e_ref, tol=TOL)
        psi_d, idev = c.linear_solve(torch.from_numpy(W).cuda(), w.e_ref, tol=TOL)
        psi_w, iw = c.linear_solve(W, w.e_ref, tol=TOL, psi=psi_p)
        c.set_linear_states(0)
        psi_0, i0 = c.linear_solve(W, w.e_ref, tol=TOL)
    for p_, i_ in ((psi_m, im), (psi_p, ip), (psi_0, i0)):
        assert np.all(i_["err"] <= TOL)
        assert np.linalg.norm(p_ - ref) <= 1e-7 * np.linalg.norm(ref)
    # the states nearest E cut the iteration count (the effect reported in Sec. II.C)
    assert ip["iters"] < im["iters"]
    assert i0["iters"] == im["iters"]
    # device buffers give the same iteration; a converged start needs no further step
    assert idev["iters"] == ip["iters"]
    assert np.linalg.norm(psi_d.cpu().numpy() - psi_p) <= 1e-12 * np.linalg.norm(psi_p)
    assert iw["iters"] == 0 and np.all(iw["err"] <= TOL)
    # sanity bound against the oracle's PCG with the same eigenpairs
    _, it_o, _ = lin.pcg_folded(h, w.e_ref, W, tol=TOL, phi=phi, eps=r["eps"], delta=r["resid"])
    assert ip["iters"] <= 1.5 * it_o + 3


def test_linear_solve_arguments(fs):
    w = _box()
    with fs.Context.from_workload(w) as c:
        psi, info = c.linear_solve(np.zeros((0, c.npw), dtype=np.complex128), w.e_ref)
        assert info["iters"] == 0 and psi.shape == (0, c.npw)
        with pytest.raises(fs.FSError):
            c.linear_solve(np.ones((1, c.npw), dtype=np.complex128), w.e_ref, tol=0.0)
        with pytest.raises(fs.FSError):
            c.set_linear_states(3)                 # no solve yet: no states to take
        # a cap of one iteration reports the error it reached
        psi, info = c.linear_solve(_rhs(w, pw.Hamiltonian(w))[:1], w.e_ref, tol=1e-14, maxit=1,
                                   allow_unconverged=True)
        assert info["iters"] == 1 and info["status"] == fs.FS_ERR_NOT_CONVERGED and info["err"][0] > 1e-14

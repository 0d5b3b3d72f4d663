"""Wave-function interpolation between k-points (Sec. II.D) on the GPU
(fs_kinterp) against the CPU FP64 oracle (oracle/kinterp.py) on the same
states: H(k1), H(k2) built densely on one common set of plane waves, their
eigenpairs by LAPACK; with a complete basis the interpolated eigenvalues equal
those of alpha H(k1) + (1 - alpha) H(k2); with a truncated basis the GPU result
equals the oracle's (eigenvalues and, up to a phase per state, the states);
alpha = 1 returns eps(k1)."""
import numpy as np
import pytest

import fs_inputs as fi
from oracle import kinterp as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K1, K2 = (0.0, 0.0, 0.05), (0.0, 0.0, 0.15)
GMAX = 2.2


@pytest.fixture(scope="module")
def setup():
    from paper_1907_06821_gb300 import build as b
    b.build()
    import paper_1907_06821_gb300 as fs
    w = fi.make_box(L=(10.0, 10.0, 20.0), n=(16, 16, 32), ecut=5.0, natom=4, widths=(1.0,), nstates=6,
                    e_ref=0.3, seed=3)
    H1, g = ki.dense_H_common(w, K1, GMAX)
    H2, _ = ki.dense_H_common(w, K2, GMAX)
    e1, V1 = np.linalg.eigh(H1)
    e2, V2 = np.linalg.eigh(H2)
    # a context whose sphere is the common plane-wave set (k = 0, cutoff GMAX^2 / 2)
    ctx = fs.Context(w.L, w.n, 0.5 * GMAX * GMAX, (0.0, 0.0, 0.0), w.vloc)
    assert np.array_equal(ctx.gvectors(), g.astype(np.int32))
    yield fs, ctx, (H1, H2, e1, V1.T.copy(), e2, V2.T.copy())
    ctx.close()


@pytest.mark.parametrize("alpha", [0.0, 0.3, 0.7, 1.0])
def test_complete_basis(setup, alpha):
    fs, c, (H1, H2, e1, p1, e2, p2) = setup
    eps, _ = c.kinterp(alpha, e1, torch.from_numpy(p1).cuda(), e2, torch.from_numpy(p2).cuda())
    ref = np.linalg.eigvalsh(alpha * H1 + (1 - alpha) * H2)
    assert np.abs(eps - ref).max() <= 1e-10


@pytest.mark.parametrize("alpha", [0.25, 0.6])
def test_truncated_basis_matches_oracle(setup, alpha):
    fs, c, (H1, H2, e1, p1, e2, p2) = setup
    n1, n2 = 20, 30
    eo, po = ki.interpolate(alpha, e1[:n1], p1[:n1], e2[:n2], p2[:n2])
    eps, psi = c.kinterp(alpha, e1[:n1], torch.from_numpy(p1[:n1]).cuda(), e2[:n2],
                         torch.from_numpy(p2[:n2]).cuda())
    psi = psi.cpu().numpy()
    assert np.abs(eps - eo).max() <= 1e-11
    # states: equal up to a phase where the eigenvalue is simple
    gaps = np.minimum(np.abs(np.diff(np.r_[-1e9, eo])), np.abs(np.diff(np.r_[eo, 1e9])))
    for q in np.nonzero(gaps[:n1] > 1e-6)[0]:
        ov = np.vdot(po[q], psi[q])
        assert abs(abs(ov) - np.linalg.norm(po[q]) * np.linalg.norm(psi[q])) <= 1e-9 * np.linalg.norm(po[q]) ** 2


def test_alpha_one_returns_k1(setup):
    fs, c, (H1, H2, e1, p1, e2, p2) = setup
    eps, _ = c.kinterp(1.0, e1[:12], torch.from_numpy(p1[:12]).cuda(), e2[:15], torch.from_numpy(p2[:15]).cuda())
    assert np.abs(eps - e1[:12]).max() <= 1e-12


def test_rejects_bad_sizes(setup):
    fs, c, (H1, H2, e1, p1, e2, p2) = setup
    with pytest.raises(fs.FSError):
        c.kinterp(0.5, e1[:10], torch.from_numpy(p1[:10]).cuda(), e2[:5], torch.from_numpy(p2[:5]).cuda())

"""The library's dense FP64 eigensolver (the subspace diagonalisation of the
Rayleigh-Ritz steps, Sec. II.C) through the C ABI against LAPACK (numpy.linalg):
random Hermitian matrices of several sizes including a ragged last block,
exactly degenerate pairs (the folded spectrum maps E +- d to one eigenvalue),
a folded-like spectrum of tiny and large eigenvalues, the m-lowest subset, and
the generalized problem with a positive definite B (Cholesky reduction); a B
that is not positive definite is reported."""
import numpy as np
import pytest

import fs_inputs as fi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1907_06821_gb300 import build as b
    b.build()
    import paper_1907_06821_gb300 as fs
    w = fi.make_config("tiny")
    with fs.Context.from_workload(w) as c:
        yield fs, c


def _herm(n, seed, spectrum=None):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    if spectrum is None:
        return 0.5 * (X + X.conj().T)
    Q, _ = np.linalg.qr(X)
    A = (Q * spectrum[None, :]) @ Q.conj().T
    return 0.5 * (A + A.conj().T)


def _check(A, w, Z, m, B=None, rtol=1e-12):
    ref = np.linalg.eigvalsh(A if B is None else np.linalg.solve(np.linalg.cholesky(B), A)
                             @ np.linalg.inv(np.linalg.cholesky(B)).conj().T)[:m]
    scale = max(1.0, np.abs(np.linalg.eigvalsh(A)).max())
    assert np.abs(w - ref).max() <= rtol * scale * 10
    Bm = np.eye(A.shape[0]) if B is None else B
    res = np.linalg.norm(A @ Z - (Bm @ Z) * w[None, :], axis=0)
    assert res.max() <= 1e-11 * scale
    G = Z.conj().T @ Bm @ Z
    assert np.abs(G - np.eye(m)).max() <= 1e-10


@pytest.mark.parametrize("n,m", [(1, 1), (7, 7), (33, 33), (100, 40), (272, 272), (816, 272)])
def test_heev_random(ctx, n, m):
    fs, c = ctx
    A = _herm(n, n)
    w, Z = c.dense_eigh(A, m)
    _check(A, w, Z, m)


def test_heev_degenerate_pairs_and_folded_spectrum(ctx):
    fs, c = ctx
    rng = np.random.default_rng(5)
    d = rng.uniform(-0.5, 0.5, 60)
    pairs = np.concatenate([d ** 2, d ** 2, rng.uniform(1, 100, 80)])   # (eps - E)^2 of eps = E +- d, and far ones
    A = _herm(200, 9, pairs)
    w, Z = c.dense_eigh(A, 150)
    _check(A, w, Z, 150)


@pytest.mark.parametrize("n,m", [(50, 50), (300, 120)])
def test_generalized(ctx, n, m):
    fs, c = ctx
    A = _herm(n, 3)
    X = _herm(n, 4)
    B = X @ X.conj().T / n + np.eye(n)
    w, Z = c.dense_eigh(A, m, B=B)
    _check(A, w, Z, m, B=B)


def test_generalized_rejects_indefinite_b(ctx):
    fs, c = ctx
    A = _herm(20, 1)
    B = np.eye(20, dtype=np.complex128)
    B[7, 7] = -1.0
    with pytest.raises(fs.FSError) as ei:
        c.dense_eigh(A, 5, B=B)
    assert ei.value.code == fs.FS_ERR_NUMERIC and "column 8" in str(ei.value)


def test_heev_near_identity_cluster(ctx):
    """The scaled overlap of an orthonormal block: every eigenvalue within 1e-9 of 1,
    one cluster of 300; the vectors must still come out orthonormal."""
    fs, c = ctx
    A = np.eye(300) + 1e-9 * _herm(300, 12)
    w, Z = c.dense_eigh(A, 300)
    assert np.abs(w - np.linalg.eigvalsh(A)).max() <= 1e-14
    assert np.abs(Z.conj().T @ Z - np.eye(300)).max() <= 1e-10
    assert np.linalg.norm(A @ Z - Z * w[None, :], axis=0).max() <= 1e-13

"""Pins of the CPU FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a brute-force
count, a textbook spectrum (free electrons), a closed form (constant or cosine
potential, the Gaussian Fourier transform, a one-projector secular equation),
an invariant (Hermiticity, translation), or LAPACK brute force.  The last tests
plant a mistake in the oracle and show that a pin catches it.
"""
import numpy as np
import pytest
import scipy.optimize as sopt

import fs_inputs as fi
from oracle import planewave as pw
from oracle import folded as of


def _box(**kw):
    base = dict(L=(7.0, 8.0, 9.0), n=(12, 12, 15), ecut=3.0, k=(0.0, 0.0, 0.0),
                natom=3, widths=(1.0,), nstates=5, e_ref=0.4, seed=3)
    base.update(kw)
    return fi.make_box(**base)


# ---------------------------------------------------------------- sphere
def _brute_sphere(L, ecut, k, hmax=30):
    out = []
    for g0 in range(-hmax, hmax + 1):
        for g1 in range(-hmax, hmax + 1):
            for g2 in range(-hmax, hmax + 1):
                q0 = k[0] + 2 * np.pi * g0 / L[0]
                q1 = k[1] + 2 * np.pi * g1 / L[1]
                q2 = k[2] + 2 * np.pi * g2 / L[2]
                if 0.5 * (q0 * q0 + q1 * q1 + q2 * q2) <= ecut:
                    out.append((g0, g1, g2))
    return sorted(out)


@pytest.mark.parametrize("L,ecut,k", [((10.0, 10.0, 20.0), 5.0, (0, 0, 0)),
                                      ((7.0, 8.0, 9.0), 3.0, (0.11, -0.07, 0.2))])
def test_sphere_matches_brute_force(L, ecut, k):
    g, q = pw.sphere(L, (64, 64, 64), ecut, np.asarray(k, float))
    assert [tuple(r) for r in g.tolist()] == _brute_sphere(L, ecut, k)
    if L == (10.0, 10.0, 20.0):
        assert g.shape[0] == 1069


def test_sphere_sizes_of_named_workloads():
    for name, npw in (("tiny", 1069), ("wire", 193673)):
        w = fi.make_config(name)
        assert pw.sphere(w.L, w.n, w.ecut, w.k)[0].shape[0] == npw


def test_grid_too_small_is_rejected():
    with pytest.raises(pw.GridTooSmall):
        pw.sphere((40.0, 40.0, 80.0), (72, 72, 144), 20.0, np.zeros(3))


# ---------------------------------------------------------------- kinetic
def test_free_electron_spectrum():
    w = _box(k=(0.1, 0.05, -0.13))
    w.vloc[:] = 0.0
    w.D[:] = 0.0
    H = pw.dense_H(w)
    g, q = pw.sphere(w.L, w.n, w.ecut, w.k)
    kin = np.sort(0.5 * np.sum(q * q, axis=1))
    assert np.allclose(np.linalg.eigvalsh(H), kin, atol=1e-13, rtol=0)


# ---------------------------------------------------------------- local
def test_constant_potential_shifts_spectrum():
    w = _box()
    e0 = np.linalg.eigvalsh(pw.dense_H(w))
    w.vloc += 0.37
    e1 = np.linalg.eigvalsh(pw.dense_H(w))
    assert np.allclose(e1 - e0, 0.37, atol=1e-12, rtol=0)


def test_cosine_potential_couples_G_pm_G0():
    w = _box(k=(0.05, 0.0, 0.0))
    v0, h = 0.21, np.array([1, 2, -1])
    j = np.meshgrid(*[np.arange(nd) for nd in w.n], indexing="ij")
    phase = 2 * np.pi * sum(h[d] * j[d] / w.n[d] for d in range(3))
    w.vloc = 2 * v0 * np.cos(phase)
    Hl = pw.dense_H(w, include=("V",))
    g, _ = pw.sphere(w.L, w.n, w.ecut, w.k)
    diff = g[:, None, :] - g[None, :, :]
    hit = np.all(diff == h, axis=2) | np.all(diff == -h, axis=2)
    assert hit.sum() > 0
    assert np.allclose(Hl[hit], v0, atol=1e-14)
    assert np.abs(Hl[~hit]).max() < 1e-14


def test_vtilde_matches_gaussian_transform():
    """Fourier coefficients of the sampled wells vs the analytic transform
    -(U/Omega)(2 pi w^2)^{3/2} exp(-w^2 G^2/2) exp(-i G.R) at small G."""
    w = fi.make_config("tiny")
    vt = pw.vtilde(w.vloc)
    omega = float(np.prod(w.L))
    for h in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (-1, 1, 3), (2, -2, -4)]:
        G = 2 * np.pi * np.asarray(h) / w.L
        ana = sum(-w.U[a] / omega * (2 * np.pi * w.w_v ** 2) ** 1.5
                  * np.exp(-0.5 * w.w_v ** 2 * G @ G) * np.exp(-1j * G @ w.pos[a])
                  for a in range(w.natom))
        idx = tuple(np.asarray(h) % np.asarray(w.n))
        assert abs(vt[idx] - ana) < 1e-11


# ---------------------------------------------------------------- nonlocal
@pytest.mark.parametrize("wid", [0.8, 1.0, 1.2])
def test_projector_norm_is_one_at_large_cutoff(wid):
    w = fi.make_box(L=(14.0, 14.0, 14.0), n=(96, 96, 96), ecut=60.0, natom=1,
                    widths=(wid,), seed=1)
    g, q = pw.sphere(w.L, w.n, w.ecut, w.k)
    B = pw.beta_matrix(w, g, q)
    norms = np.sum(np.abs(B) ** 2, axis=0)
    assert np.allclose(norms, 1.0, atol=1e-9)
    G = B.conj().T @ B                         # s and p of one centre are orthogonal
    assert np.abs(G - np.eye(4)).max() < 1e-9


def test_projector_matches_numerical_transform():
    """beta(q) = Omega^-1/2 int e^{-i q.r} phi(r - R) dr, by an FFT of the
    real-space Gaussian sampled on a fine grid."""
    w = fi.make_box(L=(14.0, 15.0, 16.0), n=(112, 120, 128), ecut=4.0, natom=1, widths=(0.9,),
                    k=(0.0, 0.0, 0.0), seed=2)
    g, q = pw.sphere(w.L, w.n, w.ecut, w.k)
    B = pw.beta_matrix(w, g, q)
    n, L, R = np.asarray(w.n), w.L, w.pos[0]
    x = [np.arange(n[d]) * L[d] / n[d] for d in range(3)]
    X = np.meshgrid(*x, indexing="ij")
    d = [((X[i] - R[i] + L[i] / 2) % L[i]) - L[i] / 2 for i in range(3)]
    r2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
    wid = 0.9
    ns = (np.pi * wid * wid) ** -0.75
    funcs = [ns * np.exp(-r2 / (2 * wid * wid))]
    funcs += [ns * np.sqrt(2.0) / wid * d[a] * np.exp(-r2 / (2 * wid * wid)) for a in range(3)]
    omega = float(np.prod(L))
    gi = tuple((g % n).T)
    for c, f in enumerate(funcs):
        num = np.fft.fftn(f)[gi] * omega / f.size / np.sqrt(omega)
        assert np.abs(num - B[:, c]).max() < 1e-9


def test_one_projector_secular_equation():
    """V = 0 and one s projector with D = d: every eigenvalue off the kinetic
    set solves 1 = d sum_G |beta_G|^2 / (eps - |q|^2/2)."""
    w = fi.make_box(L=(8.0, 8.0, 8.0), n=(16, 16, 16), ecut=3.0, natom=1, widths=(1.0,),
                    k=(0.07, 0.03, 0.0), seed=4)
    w.vloc[:] = 0.0
    w.proj = [w.proj[0]]
    d = 0.8
    w.D = np.full((1, 1, 1), d)
    g, q = pw.sphere(w.L, w.n, w.ecut, w.k)
    kin = 0.5 * np.sum(q * q, axis=1)
    b2 = np.abs(pw.beta_matrix(w, g, q)[:, 0]) ** 2
    ev = np.linalg.eigvalsh(pw.dense_H(w))

    def f(e):
        return 1.0 - d * np.sum(b2 / (e - kin))
    # distinct kinetic levels with their total weight; roots lie between them
    lv, inv = np.unique(np.round(kin, 12), return_inverse=True)
    wgt = np.bincount(inv, weights=b2)
    lv = lv[wgt > 1e-30]
    roots = []
    for a, b in zip(lv[:-1], lv[1:]):
        roots.append(sopt.brentq(f, a + 1e-12, b - 1e-12, xtol=1e-15))
    roots.append(sopt.brentq(f, lv[-1] + 1e-12, lv[-1] + 10 * d + 10, xtol=1e-15))
    for r in roots:
        assert np.min(np.abs(ev - r)) < 1e-10


# ---------------------------------------------------------------- full H
@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.13, -0.2, 0.07)])
def test_hermitian_and_matrix_free(k):
    w = _box(k=k)
    H = pw.dense_H(w)
    assert np.abs(H - H.conj().T).max() == 0.0 or np.abs(H - H.conj().T).max() < 1e-15
    h = pw.Hamiltonian(w)
    X = fi.raw_start_block(4, h.npw, 9)
    assert np.abs(h.apply(X, 0.3) - (H @ X.T).T + 0.3 * X).max() < 1e-12


def test_translation_invariance():
    w = _box(k=(0.1, 0.0, -0.05))
    e0 = np.linalg.eigvalsh(pw.dense_H(w))
    t = np.array([3, -2, 5])
    w.vloc = np.roll(w.vloc, shift=tuple(t), axis=(0, 1, 2))
    w.pos = w.pos + t * w.L / np.asarray(w.n)
    e1 = np.linalg.eigvalsh(pw.dense_H(w))
    assert np.abs(e1 - e0).max() < 1e-12


def test_brute_nearest_selects_closest():
    w = _box()
    eps, V, alle = pw.brute_nearest(w, w.e_ref, 7)
    rest = np.setdiff1d(np.round(alle, 12), np.round(eps, 12))
    assert np.abs(eps - w.e_ref).max() <= np.abs(rest - w.e_ref).min()
    assert np.all(np.diff(np.abs(eps - w.e_ref)) >= 0)
    H = pw.dense_H(w)
    for i in range(7):
        assert np.linalg.norm(H @ V[i] - eps[i] * V[i]) < 1e-12


# ---------------------------------------------------------------- folded PCG
def dense_box():
    """18 wells, 2,309 plane waves, 40 states in the middle of a dense spectrum
    (level spacing ~3e-3 Ha, near-mirror pairs about E)."""
    w = fi.make_box(L=(16., 16., 24.), n=(24, 24, 36), ecut=4.0, natom=18, widths=(1.0,), nstates=40,
                    e_ref=None, seed=7)
    e = np.linalg.eigvalsh(pw.dense_H(w))
    w.e_ref = 0.5 * (e[60] + e[61])
    return w


@pytest.mark.parametrize("case", ["tiny", "box_k", "box_dense"])
def test_folded_solver_matches_lapack(case):
    if case == "tiny":
        w = fi.make_config("tiny")
    elif case == "box_k":
        w = _box(k=(0.09, -0.04, 0.12), natom=4, nstates=6)
    else:
        w = dense_box()
    h = pw.Hamiltonian(w)
    eb, Vb, _ = pw.brute_nearest(w, w.e_ref, w.nstates)
    X0 = fi.raw_start_block(w.nbands, h.npw, 17)
    tol = 1e-8 if case != "box_dense" else 1e-6
    r = of.solve_folded(w, w.e_ref, w.nstates, tol, X0, ham=h)
    assert r["converged"]
    # compare the sets: the dense box puts E exactly between two levels (a tie in |eps - E|)
    assert np.abs(np.sort(r["eps"]) - np.sort(eb)).max() < (1e-10 if case != "box_dense" else 1e-9)
    X = r["X"]
    assert np.abs(X.conj() @ X.T - np.eye(w.nstates)).max() < 1e-10
    HX = pw.Hamiltonian(w).apply(X)
    res = np.linalg.norm(HX - r["eps"][:, None] * X, axis=1)
    assert res.max() <= 1.01 * tol


# ---------------------------------------------------------------- planted mistakes
def test_pin_catches_wrong_projector_phase(monkeypatch):
    """Flip the sign of the projector phase: translation invariance breaks."""
    real = pw.beta_matrix

    def wrong(w, g, q):
        B = real(w, g, q)
        fix = np.exp(2j * (q @ w.pos.T))                 # e^{-iqR} -> e^{+iqR}
        return B * np.repeat(fix, w.nproj, axis=1)
    monkeypatch.setattr(pw, "beta_matrix", wrong)
    w = _box(k=(0.1, 0.0, -0.05))
    e0 = np.linalg.eigvalsh(pw.dense_H(w))
    t = np.array([3, -2, 5])
    w.vloc = np.roll(w.vloc, shift=tuple(t), axis=(0, 1, 2))
    w.pos = w.pos + t * w.L / np.asarray(w.n)
    e1 = np.linalg.eigvalsh(pw.dense_H(w))
    assert np.abs(e1 - e0).max() > 1e-6


def test_pin_catches_dropped_normalisation(monkeypatch):
    """Drop the (2 pi w^2)^{3/2} factor: the Parseval norm pin fails."""
    real = pw.beta_matrix

    def wrong(w, g, q):
        return real(w, g, q) / (2 * np.pi) ** 1.5
    monkeypatch.setattr(pw, "beta_matrix", wrong)
    w = fi.make_box(L=(12.0, 12.0, 12.0), n=(96, 96, 96), ecut=60.0, natom=1, widths=(1.0,), seed=1)
    g, q = pw.sphere(w.L, w.n, w.ecut, w.k)
    norms = np.sum(np.abs(pw.beta_matrix(w, g, q)) ** 2, axis=0)
    assert not np.allclose(norms, 1.0, atol=1e-3)


# ---------------------------------------------------------------- learned preconditioner network
from oracle import mlp  # noqa: E402


def test_mlp_untrained_is_identity_gain():
    """The output layer starts at zero: z = 0, gain exp(0) = 1, i.e. the paper's M(G)."""
    th = mlp.init_params(3)
    F = np.random.default_rng(1).normal(size=(50, 4))
    z, _ = mlp.forward(th, F)
    assert np.all(z == 0.0)
    assert th.size == mlp.n_params() == 33793


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    th = mlp.init_params(5) + 0.05 * rng.normal(size=mlp.n_params())
    F = rng.normal(size=(37, 4))
    zt = rng.normal(size=37)
    wt = rng.uniform(0.1, 1.0, size=37)
    _, g = mlp.loss_and_grad(th, F, zt, wt)
    for idx in rng.choice(th.size, size=40, replace=False):
        e = np.zeros_like(th)
        e[idx] = 1e-6
        lp, _ = mlp.loss_and_grad(th + e, F, zt, wt)
        lm, _ = mlp.loss_and_grad(th - e, F, zt, wt)
        assert abs((lp - lm) / 2e-6 - g[idx]) <= 1e-6 * max(1.0, abs(g[idx]))


def _fd_mismatch(th, F, zt, wt, n=40, seed=11):
    """Largest |finite difference - backprop| over sampled parameters."""
    rng = np.random.default_rng(seed)
    _, g = mlp.loss_and_grad(th, F, zt, wt)
    worst = 0.0
    for idx in rng.choice(th.size, size=n, replace=False):
        e = np.zeros_like(th)
        e[idx] = 1e-6
        lp, _ = mlp.loss_and_grad(th + e, F, zt, wt)
        lm, _ = mlp.loss_and_grad(th - e, F, zt, wt)
        worst = max(worst, abs((lp - lm) / 2e-6 - g[idx]) / max(1.0, abs(g[idx])))
    return worst


def test_pin_catches_activation_derivative_mismatch(monkeypatch):
    """Plant a forward activation (sin) that the backward pass's tanh
    derivative does not match: the finite-difference pin fails."""
    class _Np:
        def __getattr__(self, k):
            return getattr(np, k)
        tanh = staticmethod(np.sin)
    rng = np.random.default_rng(7)
    th = mlp.init_params(5) + 0.05 * rng.normal(size=mlp.n_params())
    F = rng.normal(size=(37, 4))
    zt = rng.normal(size=37)
    wt = rng.uniform(0.1, 1.0, size=37)
    assert _fd_mismatch(th, F, zt, wt) <= 1e-6
    monkeypatch.setattr(mlp, "np", _Np())
    assert _fd_mismatch(th, F, zt, wt) > 1e-4


def test_shell_index_matches_brute_force():
    """Shells are uniform bins of |q|^2/2 over [0, ecut]; the top edge and
    anything above it fall in the last shell."""
    rng = np.random.default_rng(4)
    ecut, ns = 7.5, 9
    kin = np.concatenate([rng.uniform(0, ecut, 500), [0.0, ecut, ecut * (1 - 1e-12)],
                          [ecut * s / ns for s in range(1, ns)]])
    got = mlp.shell_index(kin, ecut, ns)
    for k, s in zip(kin, got):
        want = ns - 1
        for j in range(ns):
            if ecut * j / ns <= k < ecut * (j + 1) / ns:
                want = j
                break
        assert s == want, (k, s, want)


def test_adam_first_step_is_signed_lr():
    """First Adam step with bias correction moves every parameter by lr*g/(|g|+eps)."""
    th = np.zeros(5)
    g = np.array([0.3, -2.0, 1e-3, 0.0, 5.0])
    new, m, v = mlp.adam_step(th, g, np.zeros(5), np.zeros(5), 1, 0.01)
    assert np.allclose(new, -0.01 * g / (np.abs(g) + 1e-8))


def test_label_recovers_proportional_error():
    """If the error equals c * M R everywhere, every shell's label is 0; if one
    shell carries twice the gain of the others, its label exceeds theirs by
    log 2; phases do not enter; an empty error shell gets the floor."""
    rng = np.random.default_rng(2)
    kin = rng.uniform(0, 5.0, size=400)
    sh = mlp.shell_index(kin, 5.0, 8)
    M = 1.0 / ((kin - 0.3) ** 2 + 0.25)
    R = rng.normal(size=(3, 400)) + 1j * rng.normal(size=(3, 400))
    c = np.array([0.5, 2.0, 3.0])
    E_err = c[:, None] * M[None, :] * R
    F, zt, wt = mlp.features_and_labels(kin, 5.0, 8, M, R, E_err, np.array([0.1, -0.2, 0.0]), sh)
    z = zt.reshape(3, 8)
    for i in range(3):
        # a proportional error is the same gain on every shell: relative label 0
        assert np.allclose(z[i][wt.reshape(3, 8)[i] > 0], 0.0, atol=1e-12)
    assert np.allclose(wt.reshape(3, 8).sum(axis=1), 1.0)
    E2 = E_err.copy()
    E2[:, sh == 3] *= 2.0
    _, zt2, wt2 = mlp.features_and_labels(kin, 5.0, 8, M, R, E2, np.array([0.1, -0.2, 0.0]), sh)
    z2 = zt2.reshape(3, 8)
    others = [s for s in range(8) if s != 3 and wt2.reshape(3, 8)[0, s] > 0]
    assert np.allclose(z2[:, 3][:, None] - z2[:, others], np.log(2.0))
    # the label is a ratio of magnitudes: an error of the same size but with
    # phases uncorrelated with M R in one shell leaves every label at 0
    E3 = E_err.copy()
    sel = sh == 5
    E3[:, sel] *= np.exp(2j * np.pi * rng.uniform(size=(3, int(sel.sum()))))
    _, zt3, _ = mlp.features_and_labels(kin, 5.0, 8, M, R, E3, np.array([0.1, -0.2, 0.0]), sh)
    assert np.allclose(zt3, zt, atol=1e-12)
    # no error in a shell: the label sits at the floor log 0.1
    E4 = E_err.copy()
    E4[:, sh == 6] = 0.0
    _, zt4, wt4 = mlp.features_and_labels(kin, 5.0, 8, M, R, E4, np.array([0.1, -0.2, 0.0]), sh)
    assert np.allclose(zt4.reshape(3, 8)[:, 6], np.log(0.1)) and np.all(wt4.reshape(3, 8)[:, 6] > 0)


def test_chunked_nonlocal_equals_stored_table():
    """The table-free oracle H (projectors formed atom chunk by atom chunk, the form
    used for the long wire whose table would not fit) equals the stored-table H."""
    w = fi.make_box(L=(12.0, 12.0, 12.0), n=(20, 24, 40), ecut=4.0, k=(0.0, 0.05, 0.0), natom=5,
                    widths=(0.8, 1.2), nstates=10, e_ref=0.2, seed=8)
    h = pw.Hamiltonian(w)
    hc = pw.Hamiltonian(w, table_bytes=0, atom_chunk=2)
    assert h.B is not None and hc.B is None and hc.chunked
    X = fi.raw_start_block(5, h.npw, 2)
    a, b = h.apply(X, 0.1), hc.apply(X, 0.1)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_bf16_rounding_and_forward():
    """bf16_round: nearest BF16 with ties to even (closed-form cases); the BF16
    forward of the tensor-core inference equals the FP64 forward when no
    rounding happens (zero output layer) and stays within the BF16 error bound
    otherwise."""
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -(1.0 + 2.0 ** -7), 2.0 ** -130, 3.0])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, -(1.0 + 2.0 ** -7), 2.0 ** -130, 3.0])
    assert np.array_equal(mlp.bf16_round(x), want)
    v = np.random.default_rng(5).normal(size=1000)
    r = mlp.bf16_round(v)
    assert np.array_equal(mlp.bf16_round(r), r)
    assert np.all(np.abs(r - v) <= 2.0 ** -8 * np.abs(v) * (1 + 1e-6))        # half a BF16 spacing
    th = mlp.init_params(3)
    F = np.random.default_rng(6).normal(size=(200, 4))
    assert np.array_equal(mlp.forward_bf16(th, F), mlp.forward(th, F)[0])     # output layer zero
    th = th + 0.1 * np.random.default_rng(7).normal(size=th.size)
    zb, z = mlp.forward_bf16(th, F), mlp.forward(th, F)[0]
    assert 0 < np.abs(zb - z).max() <= 5e-2 * max(1.0, np.abs(z).max())

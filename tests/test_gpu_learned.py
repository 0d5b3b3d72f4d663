"""Learned G-shell preconditioner on the GPU.

The network's inference (tensor cores, BF16 operands, FP32 accumulation), loss
and gradient (CUDA cores, FP32 arithmetic, BF16 weights) are compared with the
FP64 CPU oracle (oracle/mlp.py) on weights that BF16 represents exactly; the untrained network must
reproduce the paper's M(G) run; a network trained on one box is applied to a
held-out box and must keep the solve correct and need fewer H applications
than M(G); the iteration counts with and without it are reported.
"""
import numpy as np
import pytest

import fs_inputs as fi
from oracle import mlp
from oracle import planewave as pw
from gpu_helpers import dense_box

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    from paper_1907_06821_gb300 import build as b
    b.build()
    import paper_1907_06821_gb300 as m
    return m


def bf16_exact(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def random_weights(seed):
    th = mlp.init_params(seed) + 0.1 * np.random.default_rng(seed).normal(size=mlp.n_params())
    return bf16_exact(th.astype(np.float32))


@pytest.mark.parametrize("rows", [1000, 25001])      # 8 tiles with a ragged tail; more tiles than SMs
def test_forward_matches_oracle(fs, rows):
    """Inference (tensor cores, BF16 operands of the 128 x 128 layers, FP32
    accumulation) against the oracle's forward with the same BF16 roundings.
    Tolerance: an activation whose FP32 value lies within FP32 rounding of a BF16
    rounding boundary may round to the neighbouring BF16 value on one side
    (2^-8 relative, about 3e-5 of the activations); its effect on z stays below
    5e-3.  Against the unrounded FP64 forward (the form training uses) the
    tensor-core result stays within 5e-2, the effect of the BF16 activations."""
    w = fi.make_config("tiny")
    with fs.Context.from_workload(w) as c:
        th = random_weights(4)
        c.precond_weights(th)
        assert np.array_equal(c.precond_weights(), th)
        F = np.random.default_rng(1).normal(size=(rows, 4)).astype(np.float32)
        z = c.precond_eval(torch.from_numpy(F).cuda()).cpu().numpy()
        zo = mlp.forward_bf16(th.astype(np.float64), F.astype(np.float64))
        scale = max(1.0, np.abs(zo).max())
        assert np.abs(z - zo).max() <= 5e-3 * scale
        assert np.median(np.abs(z - zo)) <= 1e-5 * scale     # almost every row to FP32 accuracy
        zf, _ = mlp.forward(th.astype(np.float64), F.astype(np.float64))
        assert np.abs(z - zf).max() <= 5e-2 * scale


def test_loss_and_gradient_match_oracle(fs):
    w = fi.make_config("tiny")
    with fs.Context.from_workload(w) as c:
        th = random_weights(9)
        c.precond_weights(th)
        rng = np.random.default_rng(3)
        n = 777                                   # several tiles of 28 rows and a ragged tail
        F = rng.normal(size=(n, 4)).astype(np.float32)
        zt = rng.normal(size=n).astype(np.float32)
        wt = rng.uniform(0.0, 1.0, size=n).astype(np.float32)
        loss, g = c.precond_loss_grad(torch.from_numpy(F).cuda(), torch.from_numpy(zt).cuda(),
                                      torch.from_numpy(wt).cuda())
        lo, go = mlp.loss_and_grad(th.astype(np.float64), F.astype(np.float64), zt.astype(np.float64),
                                   wt.astype(np.float64))
        g = g.cpu().numpy()
        assert abs(loss - lo) <= 1e-4 * lo
        assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_features_and_labels_match_oracle(fs, precision):
    """The features, labels and weights a recording solve computes on the device
    (correction into the reference span by the solver's GEMMs, shell sums,
    feature/label kernel) against oracle/mlp.features_and_labels on the same
    residual block; shells with no plane wave carry weight 0 on both sides."""
    w = fi.make_config("tiny")
    h = pw.Hamiltonian(w)
    npw, nb, nref, ns = h.npw, 7, 9, 32
    rng = np.random.default_rng(21)
    damp = 1.0 / (1.0 + h.kin)
    R = fi.raw_start_block(nb, npw, 31) * damp[None, :]
    X = fi.raw_start_block(nb, npw, 32) * damp[None, :]
    Q, _ = np.linalg.qr(fi.raw_start_block(nref, npw, 33).T)
    Xref = np.ascontiguousarray(Q.T)
    d = rng.uniform(-0.3, 0.3, size=nb)
    cdt = np.complex128 if precision == "fp64" else np.complex64
    R, X, Xref = R.astype(cdt), X.astype(cdt), Xref.astype(cdt)
    prec = fs.FS_FP64 if precision == "fp64" else fs.FS_MIXED
    with fs.Context.from_workload(w, precision=prec) as c:
        tR, tX, tXr = (torch.from_numpy(a).cuda() for a in (R, X, Xref))
        F, zt, wt = (t.cpu().numpy().astype(np.float64) for t in c.precond_features(w.e_ref, tR, d, X=tX, Xref=tXr))
        F_only = c.precond_features(w.e_ref, tR, d).cpu().numpy()
    R64, X64, Xr64 = (a.astype(np.complex128) for a in (R, X, Xref))
    E_err = (Xr64.conj() @ X64.T).T @ Xr64 - X64
    M = 1.0 / ((h.kin - w.e_ref) ** 2 + 0.5 ** 2)
    shell = mlp.shell_index(h.kin, w.ecut, ns)
    Fo, zo, wo = mlp.features_and_labels(h.kin, w.ecut, ns, M, R64, E_err, d, shell)
    full = np.tile(np.bincount(shell, minlength=ns) > 0, nb)
    assert full.sum() >= nb * 20                     # most shells hold plane waves
    assert np.array_equal(F_only, F.astype(np.float32))
    assert np.abs(F[full] - Fo[full]).max() <= 2e-5
    assert np.abs(wt - wo).max() <= 1e-5 and np.all(wt[~full] == 0)
    # labels: log-gains relative to the band's weighted mean (FP32 storage; the FP32
    # stage's correction comes from TF32 x3 tensor-core products)
    ltol = 1e-4 if precision == "fp64" else 2e-3
    assert np.abs(zt[full] - zo[full]).max() <= ltol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_untrained_network_is_paper_preconditioner(fs, precision):
    w = fi.make_config("tiny")
    prec = fs.FS_FP64 if precision == "fp64" else fs.FS_MIXED
    out = {}
    for pc in (fs.FS_PREC_M, fs.FS_PREC_LEARNED):
        with fs.Context.from_workload(w, precision=prec, precond=pc) as c:
            c.set_initial_states(fi.raw_start_block(w.nbands, c.npw, 17), damp=True)
            out[pc] = c.solve(w.e_ref, w.nstates, tol=1e-6)
    a, b = out[fs.FS_PREC_M], out[fs.FS_PREC_LEARNED]
    assert a["iters"] == b["iters"] and a["n_hpsi"] == b["n_hpsi"]
    assert np.array_equal(a["eps"], b["eps"])


def _held_out_iterations(fs):
    """Train on one seeded box, apply to a box of another seed (same sizes); both
    solves must reach the brute-force set.  Returns (loss, rows, {name: (iters, n_hpsi)})."""
    train = dense_box()
    test_box = fi.make_box(L=(16., 16., 24.), n=(24, 24, 36), ecut=4.0, natom=18, widths=(1.0,), nstates=40,
                           e_ref=None, seed=11)
    e = np.linalg.eigvalsh(pw.dense_H(test_box))
    test_box.e_ref = 0.5 * (e[60] + e[61])
    eb, _, _ = pw.brute_nearest(test_box, test_box.e_ref, test_box.nstates)
    with fs.Context.from_workload(train, precision=fs.FS_MIXED) as c:
        c.set_initial_states(fi.raw_start_block(train.nbands, c.npw, 17), damp=True)
        loss, rows = c.precond_train(train.e_ref, train.nstates, tol=1e-6, epochs=300, lr=2e-3)
        weights = c.precond_weights()
    assert rows > 0 and np.isfinite(loss)
    iters = {}
    for name, pc in (("M", fs.FS_PREC_M), ("learned", fs.FS_PREC_LEARNED)):
        with fs.Context.from_workload(test_box, precision=fs.FS_MIXED, precond=pc) as c:
            if pc == fs.FS_PREC_LEARNED:
                c.precond_weights(weights)
            c.set_initial_states(fi.raw_start_block(test_box.nbands, c.npw, 5), damp=True)
            r = c.solve(test_box.e_ref, test_box.nstates, tol=1e-6)
            assert r["nconv"] == test_box.nstates
            assert np.abs(np.sort(r["eps"]) - np.sort(eb)).max() <= 1e-5
            iters[name] = (r["iters"], r["n_hpsi"])
    return loss, rows, iters


_HELD_OUT = {}


def test_trained_network_keeps_the_solve_correct(fs, capsys):
    """The trained network on a held-out box: the solve reaches the brute-force set
    (the preconditioner changes the path, not the fixed point); the iteration counts
    with and without it are reported."""
    loss, rows, iters = _held_out_iterations(fs)
    _HELD_OUT.update(iters)
    with capsys.disabled():
        print(f"\n[learned preconditioner] training loss {loss:.4f} on {rows} rows; held-out box: "
              f"M(G) {iters['M'][0]} iterations / {iters['M'][1]} H applications, "
              f"learned {iters['learned'][0]} / {iters['learned'][1]}")


def test_trained_network_gains_over_paper_preconditioner(fs):
    """What the trained network gains over the method without it: on the held-out
    box it needs fewer H applications and fewer iterations than the paper's M(G)
    (measured on a GB300: 65 against 85 iterations, 6,376 against 8,312 H
    applications)."""
    if not _HELD_OUT:
        _HELD_OUT.update(_held_out_iterations(fs)[2])
    assert _HELD_OUT["learned"][1] < 0.95 * _HELD_OUT["M"][1]
    assert _HELD_OUT["learned"][0] < _HELD_OUT["M"][0]

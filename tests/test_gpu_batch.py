"""Batched independent boxes (fs_batch_*) and the FFT tile autotuner.

Each box of a batch of uneven boxes, solved concurrently, must give the same
result as the same box solved alone from the same start block, and every
returned state must pass the CPU oracle's FP64 residual check; the smallest
boxes are also checked against LAPACK brute force.  The autotuner must keep
the H application unchanged.
"""
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


def boxes():
    shapes = [(24, 24, 24), (20, 20, 40), (32, 32, 32), (24, 24, 48), (16, 16, 32), (30, 30, 30)]
    out = []
    for i, n in enumerate(shapes):
        L = tuple(0.6 * np.asarray(n, float))
        w = fi.make_box(L=L, n=n, ecut=3.0, natom=4 + 2 * i, widths=(1.0,), nstates=6 + 2 * i, e_ref=None,
                        seed=100 + i, name=f"b{i}")
        w.e_ref = -0.5 * float(np.mean(w.U))
        out.append(w)
    return out


def test_batch_matches_single_solves(fs):
    ws = boxes()
    ctxs = [fs.Context.from_workload(w, precision=fs.FS_MIXED) for w in ws]
    for w, c in zip(ws, ctxs):
        c.set_initial_states(fi.raw_start_block(w.nbands, c.npw, 7), damp=True)
    batch = fs.Batch(ctxs, nthreads=4)
    rb = batch.solve([w.e_ref for w in ws], [w.nstates for w in ws], tol=1e-6)
    for i, (w, c) in enumerate(zip(ws, ctxs)):
        assert rb[i]["status"] == fs.FS_OK, i
        states = c.get_states(w.nstates)
        h = pw.Hamiltonian(w)
        res = np.linalg.norm(h.apply(states) - rb[i]["eps"][:, None] * states, axis=1)
        assert res.max() <= 1e-6
        with fs.Context.from_workload(w, precision=fs.FS_MIXED) as single:
            single.set_initial_states(fi.raw_start_block(w.nbands, single.npw, 7), damp=True)
            r1 = single.solve(w.e_ref, w.nstates, tol=1e-6)
        assert np.array_equal(r1["eps"], rb[i]["eps"])      # concurrency does not change a box's result
        if h.npw <= 2500:
            eb, _, _ = pw.brute_nearest(w, w.e_ref, w.nstates)
            assert np.abs(np.sort(rb[i]["eps"]) - np.sort(eb)).max() <= 1e-5
    batch.close()
    for c in ctxs:
        c.close()


def test_autotune_keeps_H(fs):
    w = boxes()[3]
    with fs.Context.from_workload(w) as c:
        X = torch.from_numpy(fi.raw_start_block(9, c.npw, 2)).cuda()
        before = c.apply_H(X).cpu().numpy()
        cpb = c.autotune()
        assert cpb in (2, 4, 8, 16, 32)
        after = c.apply_H(X).cpu().numpy()
    assert np.abs(after - before).max() <= 1e-12 * np.abs(before).max()

"""Failure paths without a GPU fault: a bounded device wait that nothing
completes returns FS_ERR_TIMEOUT and leaves the context usable; a non-finite
start block is reported as FS_ERR_NUMERIC before any dense eigensolve sees it,
and the context solves normally afterwards."""
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


def test_bounded_wait_expires_with_a_status(fs):
    w = fi.make_config("tiny")
    with fs.Context.from_workload(w, precision=fs.FS_MIXED) as c:
        X = torch.from_numpy(fi.raw_start_block(5, c.npw, 1).astype(np.complex64)).cuda()
        before = c.apply_H(X).cpu().numpy()
        with pytest.raises(fs.FSError) as ei:
            c.wait_selftest(4096)
        assert ei.value.code == fs.FS_ERR_TIMEOUT
        after = c.apply_H(X).cpu().numpy()
    assert np.array_equal(before, after)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_start_block_is_reported(fs, prec):
    w = fi.make_config("tiny")
    p = fs.FS_FP64 if prec == "fp64" else fs.FS_MIXED
    eb, _, _ = pw.brute_nearest(w, w.e_ref, w.nstates)
    with fs.Context.from_workload(w, precision=p) as c:
        X0 = fi.raw_start_block(w.nbands, c.npw, 17)
        bad = X0.copy()
        bad[3, 10] = np.nan
        c.set_initial_states(bad, damp=True)
        with pytest.raises(fs.FSError) as ei:
            c.solve(w.e_ref, w.nstates, tol=1e-6)
        assert ei.value.code == fs.FS_ERR_NUMERIC
        c.set_initial_states(X0, damp=True)
        r = c.solve(w.e_ref, w.nstates, tol=1e-6)
    assert r["nconv"] == w.nstates
    assert np.abs(np.sort(r["eps"]) - np.sort(eb)).max() <= 1e-5

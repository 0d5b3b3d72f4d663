"""The lowest eigenpairs of H by the all-band CG on H itself (fs_solve_lowest;
the ground-state solver of the codes the paper builds on, Sec. II.A-B) through
the C ABI: eigenvalues against LAPACK's on small boxes (FP64 and mixed
precision), every state's residual recomputed by the oracle's H, orthonormal
states, ascending order; the same solve agrees with the oracle's block CG of
oracle/lowest.py; at the wire's full size the lowest 129 eigenvalues match the
golden spectrum (oracle + SciPy LOBPCG) and give the wire's E_ref, the midpoint
of the 128th and 129th."""
import json
import os

import numpy as np
import pytest

import fs_inputs as fi
from oracle import lowest as lo
from oracle import planewave as pw
from gpu_helpers import CASES

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    from paper_1907_06821_gb300 import build as b
    b.build()
    import paper_1907_06821_gb300 as m
    return m


def _check(w, r, states, ref, tol=1e-6):
    assert np.all(np.diff(r["eps"]) >= -1e-12)
    assert np.abs(r["eps"] - ref).max() <= 1e-5
    h = pw.Hamiltonian(w)
    res = np.linalg.norm(h.apply(states) - r["eps"][:, None] * states, axis=1)
    assert res.max() <= tol
    assert np.allclose(res, r["resid"], atol=1e-8)
    assert np.abs(states.conj() @ states.T - np.eye(states.shape[0])).max() < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["tiny", "box_k_radix35", "box_radix5_two_widths"])
def test_lowest_matches_lapack(fs, case, precision):
    w = CASES[case]()
    n = 12
    ref = np.linalg.eigvalsh(pw.dense_H(w))[:n]
    prec = fs.FS_FP64 if precision == "fp64" else fs.FS_MIXED
    with fs.Context.from_workload(w, precision=prec) as c:
        c.set_initial_states(fi.raw_start_block(n + 4, c.npw, 17), damp=True)
        r = c.solve_lowest(n, tol=1e-6)
        states = c.get_states(n)
    assert r["nconv"] == n
    _check(w, r, states, ref)


def test_lowest_agrees_with_oracle_block_cg(fs):
    w = CASES["box_k_radix35"]()
    h = pw.Hamiltonian(w)
    n = 8
    X0 = fi.raw_start_block(n + 4, h.npw, 17) / (1.0 + h.kin)[None, :]
    eo, _, _, _ = lo.lobpcg_lowest(h.apply, h.kin, n, 1e-8, X0)
    with fs.Context.from_workload(w) as c:
        c.set_initial_states(fi.raw_start_block(n + 4, c.npw, 17), damp=True)
        r = c.solve_lowest(n, tol=1e-8)
    assert np.abs(r["eps"] - eo).max() <= 1e-9


def test_wire_lowest_states_give_e_ref(fs):
    """Full-size wire (193,673 plane waves, 2,048 projectors), mixed precision:
    the 129 lowest states; E_ref = midpoint of the 128th and 129th."""
    w = fi.make_config("wire")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "wire_spectrum.json")
    with open(path) as f:
        gold = np.asarray(json.load(f)["eigenvalues"])
    n = 129
    with fs.Context.from_workload(w, precision=fs.FS_MIXED) as c:
        c.set_initial_states(fi.raw_start_block(n + 8, c.npw, 17), damp=True)
        r = c.solve_lowest(n, tol=1e-6)
    assert r["nconv"] == n
    assert np.abs(r["eps"] - gold[:n]).max() <= 1e-5
    e_ref = 0.5 * (r["eps"][127] + r["eps"][128])
    assert abs(e_ref - w.e_ref) <= 1e-5
    assert r["resid"].max() <= 1e-6

"""Shared helpers of the GPU parity tests (test infrastructure)."""
import numpy as np

import fs_inputs as fi
from oracle import planewave as pw


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def small_box(**kw):
    base = dict(L=(7.0, 8.0, 9.0), n=(12, 12, 15), ecut=3.0, k=(0.11, -0.07, 0.2), natom=3,
                widths=(1.0,), nstates=5, e_ref=0.4, seed=3)
    base.update(kw)
    return fi.make_box(**base)


CASES = {
    "tiny": lambda: fi.make_config("tiny"),
    "box_k_radix35": lambda: small_box(),
    "box_radix5_two_widths": lambda: fi.make_box(L=(12.0, 12.0, 12.0), n=(20, 24, 40), ecut=4.0,
                                                 k=(0.0, 0.05, 0.0), natom=5, widths=(0.8, 1.2),
                                                 nstates=10, e_ref=0.2, seed=8),
    "box_no_projectors": lambda: fi.make_box(L=(9.0, 9.0, 9.0), n=(16, 18, 20), ecut=3.5,
                                             natom=2, widths=(), nstates=4, e_ref=0.5, seed=9),
}


def oracle_ham(w):
    return pw.Hamiltonian(w)


def dense_box():
    """18 wells, 2,309 plane waves, 40 states in the middle of a dense spectrum
    (level spacing ~3e-3 Ha, near-mirror pairs about E)."""
    w = fi.make_box(L=(16., 16., 24.), n=(24, 24, 36), ecut=4.0, natom=18, widths=(1.0,), nstates=40,
                    e_ref=None, seed=7)
    e = np.linalg.eigvalsh(pw.dense_H(w))
    w.e_ref = 0.5 * (e[60] + e[61])
    return w

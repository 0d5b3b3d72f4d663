"""Writes tests/golden/eref.json: the reference energy of the wire workloads.

The wire workloads place E_ref at the midpoint between the floor(N_sites/2)-th
and the next eigenvalue of H (counting from the bottom of the spectrum), i.e.
at half filling of one s-like level per well.  This script computes those two
eigenvalues with the CPU FP64 oracle's matrix-free H and SciPy's LOBPCG, and
calls nothing but oracle/, fs_inputs and NumPy/SciPy.

    python tests/golden/make_eref.py wire
"""
import json
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as ssl

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import fs_inputs  # noqa: E402
from oracle.planewave import Hamiltonian  # noqa: E402


def lowest(w, k, tol=1e-6, maxiter=200, seed=11):
    h = Hamiltonian(w)
    N = h.npw
    op = ssl.LinearOperator((N, N), dtype=np.complex128,
                            matvec=lambda v: h.apply(v.reshape(1, -1))[0],
                            matmat=lambda V: h.apply(np.ascontiguousarray(V.T)).T)
    # kinetic-energy preconditioner (positive, diagonal)
    pre = 1.0 / (1.0 + h.kin)
    prec = ssl.LinearOperator((N, N), dtype=np.complex128,
                              matvec=lambda v: pre * v.ravel(),
                              matmat=lambda V: pre[:, None] * V)
    X0 = fs_inputs.raw_start_block(k, N, seed).T * pre[:, None]
    vals, _ = ssl.lobpcg(op, X0, M=prec, largest=False, tol=tol, maxiter=maxiter,
                         verbosityLevel=0)
    return np.sort(vals.real)


def main(names):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "eref.json")
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    for name in names:
        w = fs_inputs.make_config(name)
        nsite = w.natom if name != "longwire" else 1000
        half = nsite // 2
        t = time.time()
        ev = lowest(w, half + 16)
        e_lo, e_hi = float(ev[half - 1]), float(ev[half])
        data[name] = {"e_ref": 0.5 * (e_lo + e_hi), "eig_half": e_lo, "eig_half_plus_1": e_hi,
                      "lowest": [float(v) for v in ev],
                      "how": "oracle matrix-free H + scipy lobpcg, tol 1e-6",
                      "seconds": time.time() - t}
        with open(path, "w") as f:
            json.dump(data, f, indent=1)
        print(name, data[name]["e_ref"], data[name]["seconds"])


if __name__ == "__main__":
    main(sys.argv[1:] or ["wire"])

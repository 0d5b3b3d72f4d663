"""Writes tests/golden/wire_spectrum.json: the lowest eigenvalues of the wire's H.

The wire solve returns the 256 eigenpairs of H nearest E_ref (the folded
spectrum, Sec. II.C).  To check the whole returned set, and not only the
residuals of its states, the eigenvalues of H on both sides of E_ref must be
known independently of the library: this script finds the lowest `count`
eigenvalues with SciPy's LOBPCG applied to the CPU FP64 oracle's matrix-free
H, preconditioned by 1/(1 + |q|^2/2).  It calls nothing but oracle/,
fs_inputs and NumPy/SciPy.

The oracle applies H band by band with numpy.fft.  Here a pool of forked
workers (one BLAS thread each, sharing the oracle's tables copy-on-write)
applies the oracle's local part (kinetic + V_loc, its H with the projector
table switched off) to slices of a block in parallel, and the parent adds the
nonlocal term B D B^H X from the same oracle object's tables with threaded
BLAS.  Run on a machine without a GPU context:

    python tests/golden/make_wire_spectrum.py [count] [workers]

Eigenvalue accuracy: LOBPCG stops at residual norm tol; an eigenvalue's error
is then of order tol^2 / gap, far below the 1e-5 Ha the parity test allows.
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as ssl

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import fs_inputs  # noqa: E402
from oracle.planewave import Hamiltonian  # noqa: E402

_H = None  # the oracle's H, built before the pool forks


def _apply_local(X):
    """The oracle's H without its nonlocal term (worker side)."""
    from threadpoolctl import threadpool_limits
    _H.B = None  # this worker's copy only
    with threadpool_limits(1):
        return _H.apply(X)


def main(count=360, workers=8, tol=1e-5, maxiter=300, seed=23):
    global _H
    t0 = time.time()
    w = fs_inputs.make_config("wire")
    _H = Hamiltonian(w)
    N = _H.npw
    B, Dfull = _H.B, _H.Dfull
    ctx = mp.get_context("fork")
    pool = ctx.Pool(workers)
    nslice = 4 * workers

    def matmat(V):
        rows = np.ascontiguousarray(np.asarray(V).T)
        parts = np.array_split(rows, min(nslice, rows.shape[0]))
        out = np.concatenate(pool.map(_apply_local, parts))
        out += (B @ (Dfull @ (B.conj().T @ rows.T))).T
        return out.T

    op = ssl.LinearOperator((N, N), dtype=np.complex128, matvec=lambda v: matmat(v.reshape(-1, 1)).ravel(),
                            matmat=matmat)
    pre = 1.0 / (1.0 + _H.kin)
    prec = ssl.LinearOperator((N, N), dtype=np.complex128, matvec=lambda v: pre * v.ravel(),
                              matmat=lambda V: pre[:, None] * V)
    X0 = fs_inputs.raw_start_block(count, N, seed).T * pre[:, None]
    vals, vecs, rnorms = ssl.lobpcg(op, X0, M=prec, largest=False, tol=tol, maxiter=maxiter, verbosityLevel=0,
                                    retResidualNormsHistory=True)
    order = np.argsort(vals.real)
    vals = vals.real[order]
    # residuals recomputed from the returned vectors with the oracle's H
    V = vecs[:, order]
    V = V / np.linalg.norm(V, axis=0)[None, :]
    R = matmat(V) - V * vals[None, :]
    res = np.linalg.norm(R, axis=0)
    pool.close()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "wire_spectrum.json")
    data = {
        "workload": "wire",
        "count": int(count),
        "eigenvalues": [float(v) for v in vals],
        "residuals": [float(r) for r in res],
        "lobpcg_iterations": len(rnorms),
        "how": f"oracle matrix-free H (FP64) + scipy.sparse.linalg.lobpcg, {count} vectors, tol {tol}, "
               f"preconditioner 1/(1+|q|^2/2), start block fs_inputs.raw_start_block(seed={seed})",
        "seconds": time.time() - t0,
    }
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
    print("wire spectrum:", count, "eigenvalues, max residual", float(res.max()), "in", data["seconds"], "s")


if __name__ == "__main__":
    a = sys.argv[1:]
    main(int(a[0]) if a else 360, int(a[1]) if len(a) > 1 else 8)

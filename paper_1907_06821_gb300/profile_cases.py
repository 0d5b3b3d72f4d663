"""Small, fixed GPU cases for kernel profiling (ncu captures and timing).

    python -m paper_1907_06821_gb300.profile_cases apply --workload wire --bands 64 --precision mixed
    python -m paper_1907_06821_gb300.profile_cases solve --workload wire --maxit 20
    python -m paper_1907_06821_gb300.profile_cases apply --workload medium --bands 64
    python -m paper_1907_06821_gb300.profile_cases linear --workload medium --nrhs 4 --states 128 --maxit 3000

``wire_local`` is the wire's grid, cutoff and V(r) without projectors: the FFT
kernels alone, with a few hundred MB on the device (for ncu captures of them).

``medium`` is a 24 x 24 x 48 bohr box on a 48 x 48 x 96 grid at 20 Ry (41,657
plane waves) with 64 wells and 8 projectors per atom: operands larger than the
L2 cache with about 2 GB on the device, for captures that replay a kernel many
times.

``apply`` builds the context and applies (H - E) to a block of seeded random
bands ``--repeat`` times (the first two launches warm up); ``solve`` runs a
bounded solve.  Both print the per-kernel-class CUDA-event statistics of the
last repetition.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _print_stats(ctx):
    for k, v in ctx.kernel_stats().items():
        if v["launches"]:
            print(f"{k:18s} n={v['launches']:5d} ms={v['ms']:10.2f} "
                  f"TF/s={v['flops'] / max(v['ms'], 1e-9) / 1e9:8.2f} GB/s={v['bytes'] / max(v['ms'], 1e-9) / 1e6:9.1f}")


def _linear(a, w, ctx, fs, fi, np):
    """The folded linear solve of nrhs wave packets with M alone, then with M' from
    the `states` eigenpairs nearest E found by the mixed-precision eigensolve (a
    separate FP64-checked solve); one JSON line with iterations, times and errors."""
    import json
    import time
    L = np.asarray(w.L)
    cen = [(L[0] * (0.3 + 0.4 * i / max(a.nrhs - 1, 1)), L[1] * 0.5, L[2] * (0.2 + 0.6 * i / max(a.nrhs - 1, 1)))
           for i in range(a.nrhs)]
    W = fi.wavepacket_rhs(ctx.gvectors(), L, cen)
    out = {"workload": a.workload, "npw": ctx.npw, "nrhs": a.nrhs, "tol": a.tol, "e_ref": w.e_ref}
    _, r0 = ctx.linear_solve(W, w.e_ref, tol=a.tol, maxit=a.maxit, allow_unconverged=True)
    out["M"] = {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in r0.items()}
    es = fs.Context.from_workload(w, precision=fs.FS_MIXED, maxit=3000)
    es.set_initial_states(fi.raw_start_block(a.states + max(4, a.states // 16), es.npw, 17), damp=True)
    t0 = time.time()
    r = es.solve(w.e_ref, a.states, tol=1e-6, allow_unconverged=True)
    t_eig = time.time() - t0
    phi = es.get_states(a.states)
    es.close()
    ctx.set_linear_states(a.states, phi=phi, eps=r["eps"], delta=r["resid"])
    _, r1 = ctx.linear_solve(W, w.e_ref, tol=a.tol, maxit=a.maxit, allow_unconverged=True)
    out["eigensolve"] = {"states": a.states, "nconv": r["nconv"], "seconds": t_eig,
                         "max_resid": float(np.max(r["resid"]))}
    out["M_prime"] = {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in r1.items()}
    print(json.dumps(out), flush=True)


def _chebfd(a, w, ctx, fi, np):
    """ChebFD states near E (Lanczos bounds, window filter, Rayleigh-Ritz), then the
    folded linear solve of nrhs wave packets with M' built from them; one JSON line."""
    import json
    lo, hi = ctx.spectral_bounds(40)
    r = ctx.chebfd(w.e_ref, a.halfwidth, lo, hi, a.degree, a.nvec, a.steps, seed=9)
    res = r["resid"]
    out = {"workload": a.workload, "npw": ctx.npw, "bounds": [lo, hi], "window": [w.e_ref - a.halfwidth,
           w.e_ref + a.halfwidth], "degree": a.degree, "nvec": a.nvec, "steps": a.steps,
           "chebfd": {"nfound": r["nfound"], "seconds": r["seconds"], "n_hpsi": r["n_hpsi"],
                      "resid_le_1e-6": int(np.sum(res <= 1e-6)), "resid_le_1e-8": int(np.sum(res <= 1e-8)),
                      "resid_median": float(np.median(res)) if len(res) else None}}
    L = np.asarray(w.L)
    cen = [(L[0] * (0.3 + 0.4 * i / max(a.nrhs - 1, 1)), L[1] * 0.5, L[2] * (0.2 + 0.6 * i / max(a.nrhs - 1, 1)))
           for i in range(a.nrhs)]
    W = fi.wavepacket_rhs(ctx.gvectors(), L, cen)
    ctx.set_linear_states(r["nfound"])
    _, rl = ctx.linear_solve(W, w.e_ref, tol=a.tol, maxit=a.maxit, allow_unconverged=True)
    out["linear_M_prime_from_chebfd"] = {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in rl.items()}
    print(json.dumps(out), flush=True)


def _learned(a, fs, fi, np):
    """Train the learned preconditioner on one seeded instance (a reference
    solve, a recording solve, Adam on the recorded rows), then solve another
    seed's instance with M(G) and with the trained network; one JSON line with
    the iteration counts, H applications and times; weights to --save."""
    import json
    import time
    name = "wire" if a.workload == "wire_local" else a.workload
    if name == "medium":
        make = lambda seed: fi.make_medium(11 if seed is None else seed)  # noqa: E731
    else:
        make = lambda seed: fi.make_config(name, seed=seed)  # noqa: E731
    train, test = make(a.train_seed), make(None)
    out = {"workload": name, "train_seed": a.train_seed, "epochs": a.epochs, "lr": a.lr}
    with fs.Context.from_workload(train, precision=fs.FS_MIXED, maxit=a.maxit) as c:
        c.set_initial_states(fi.raw_start_block(train.nbands, c.npw, 17), damp=True)
        t0 = time.time()
        loss, rows = c.precond_train(train.e_ref, train.nstates, tol=1e-6, epochs=a.epochs, lr=a.lr)
        out["train"] = {"loss": loss, "rows": rows, "seconds": time.time() - t0}
        weights = c.precond_weights()
    if a.save:
        np.asarray(weights, dtype=np.float32).tofile(a.save)
    for label, pc in (("M", fs.FS_PREC_M), ("learned", fs.FS_PREC_LEARNED)):
        with fs.Context.from_workload(test, precision=fs.FS_MIXED, precond=pc, maxit=a.maxit,
                                      verbose=int(a.verbose)) as c:
            if pc == fs.FS_PREC_LEARNED:
                c.precond_weights(weights)
            c.set_initial_states(fi.raw_start_block(test.nbands, c.npw, 17), damp=True)
            t0 = time.time()
            r = c.solve(test.e_ref, test.nstates, tol=1e-6, allow_unconverged=True)
            out[label] = {"iters": r["iters"], "iters_mixed": r["iters_mixed"], "n_hpsi": r["n_hpsi"],
                          "nconv": r["nconv"], "seconds": time.time() - t0, "max_resid": float(np.max(r["resid"]))}
    print(json.dumps(out), flush=True)


def main(argv=None):
    import numpy as np
    import torch

    import fs_inputs as fi
    import paper_1907_06821_gb300 as fs

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["apply", "solve", "linear", "chebfd", "learned"])
    ap.add_argument("--workload", default="wire", choices=["tiny", "wire", "wire_local", "medium", "longwire"])
    ap.add_argument("--autotune", action="store_true", help="run the launch-shape autotuner first (verbose)")
    ap.add_argument("--bands", type=int, default=64)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--maxit", type=int, default=20)
    ap.add_argument("--verbose", action="store_true", help="per-iteration solver log on stderr")
    ap.add_argument("--dE", type=float, default=0.5, help="width of the preconditioner M(G), Ha")
    ap.add_argument("--nrhs", type=int, default=4, help="linear: right-hand sides (wave packets)")
    ap.add_argument("--states", type=int, default=128, help="linear: eigenstates nearest E for M'")
    ap.add_argument("--tol", type=float, default=1e-8, help="linear: target of ||(H - E) psi - w||")
    ap.add_argument("--nvec", type=int, default=96, help="chebfd: block size")
    ap.add_argument("--degree", type=int, default=300, help="chebfd: filter degree")
    ap.add_argument("--steps", type=int, default=3, help="chebfd: filter steps")
    ap.add_argument("--halfwidth", type=float, default=0.04, help="chebfd: window half-width, Ha")
    ap.add_argument("--train-seed", type=int, default=2907, help="learned: seed of the training instance")
    ap.add_argument("--epochs", type=int, default=300, help="learned: Adam epochs")
    ap.add_argument("--lr", type=float, default=2e-3, help="learned: Adam step")
    ap.add_argument("--save", default="", help="learned: file for the trained weights (float32)")
    a = ap.parse_args(argv)
    if a.case == "learned":
        _learned(a, fs, fi, np)
        return
    if a.workload == "medium":
        w = fi.make_medium()
    else:
        w = fi.make_config("wire" if a.workload == "wire_local" else a.workload)
    prec = fs.FS_MIXED if a.precision == "mixed" else fs.FS_FP64
    verbose = int(a.verbose or a.autotune)
    if a.workload == "wire_local":
        ctx = fs.Context(w.L, w.n, w.ecut, w.k, w.vloc, precision=prec, maxit=a.maxit, verbose=verbose)
    else:
        ctx = fs.Context.from_workload(w, precision=prec, maxit=a.maxit, verbose=verbose, dE=a.dE)
    if a.autotune:
        print("autotune: column tile", ctx.autotune(), flush=True)
    if a.case == "apply":
        dt = torch.complex64 if prec == fs.FS_MIXED else torch.complex128
        X = torch.from_numpy(fi.raw_start_block(a.bands, ctx.npw, 1)).to(dt).cuda()
        for r in range(a.repeat):
            if r == a.repeat - 1:
                ctx.profile(True)
            ctx.apply_H(X, shift=w.e_ref)
        torch.cuda.synchronize()
    elif a.case == "linear":
        _linear(a, w, ctx, fs, fi, np)
        ctx.close()
        return
    elif a.case == "chebfd":
        _chebfd(a, w, ctx, fi, np)
        ctx.close()
        return
    else:
        ctx.set_initial_states(fi.raw_start_block(w.nbands, ctx.npw, 17), damp=True)
        ctx.profile(True)
        r = ctx.solve(w.e_ref, w.nstates, tol=1e-6, allow_unconverged=True)
        print("solve", {k: r[k] for k in ("nconv", "iters", "n_hpsi", "seconds")}, "max resid",
              float(np.max(r["resid"])))
    _print_stats(ctx)
    ctx.close()


if __name__ == "__main__":
    main()

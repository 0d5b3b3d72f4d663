"""Small, fixed GPU cases for kernel profiling (ncu captures and timing).

    python -m paper_1907_06821_gb300.profile_cases apply --workload wire --bands 64 --precision mixed
    python -m paper_1907_06821_gb300.profile_cases solve --workload wire --maxit 20
    python -m paper_1907_06821_gb300.profile_cases apply --workload medium --bands 64

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


def main(argv=None):
    import numpy as np
    import torch

    import fs_inputs as fi
    import paper_1907_06821_gb300 as fs

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["apply", "solve"])
    ap.add_argument("--workload", default="wire", choices=["tiny", "wire", "medium"])
    ap.add_argument("--bands", type=int, default=64)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--maxit", type=int, default=20)
    ap.add_argument("--verbose", action="store_true", help="per-iteration solver log on stderr")
    a = ap.parse_args(argv)
    if a.workload == "medium":
        w = fi.make_box(L=(24.0, 24.0, 48.0), n=(48, 48, 96), ecut=10.0, natom=64, widths=(0.8, 1.2),
                        lattice=5.0, nstates=128, e_ref=0.05, seed=11, name="medium")
    else:
        w = fi.make_config(a.workload)
    prec = fs.FS_MIXED if a.precision == "mixed" else fs.FS_FP64
    ctx = fs.Context.from_workload(w, precision=prec, maxit=a.maxit, verbose=int(a.verbose))
    if a.case == "apply":
        dt = torch.complex64 if prec == fs.FS_MIXED else torch.complex128
        X = torch.from_numpy(fi.raw_start_block(a.bands, ctx.npw, 1)).to(dt).cuda()
        for r in range(a.repeat):
            if r == a.repeat - 1:
                ctx.profile(True)
            ctx.apply_H(X, shift=w.e_ref)
        torch.cuda.synchronize()
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

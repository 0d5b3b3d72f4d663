"""Benchmark of the folded-spectrum eigensolve (one JSON line on rank 0).

A step is one complete solve, from the same seeded start block, of the
wire-segment workload: 40x40x80 bohr cell, 72x72x144 grid, 20 Ry cutoff
(193,673 plane waves), 256 Gaussian wells, 8 projectors per atom, the 256
states nearest the reference energy, to residual 1e-6.  The metric is states
converged per second: a state counts when its residual (the library's FP64
check) is <= 1e-6 and, for the wire, the returned eigenvalue set matches the
golden set (the 256 eigenvalues nearest E_ref of tests/golden/wire_spectrum.json,
computed on the CPU from the FP64 oracle by SciPy's LOBPCG) to 1e-5 Ha.

  python bench.py [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--workload wire|tiny] [--impl ours|reference]

--impl reference times the CPU FP64 oracle (test infrastructure, the only
other code path here) on a bounded sample of the same workload.  Under
torchrun each rank solves its own seeded instance (independent problems, no
collective on the data path; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# DRAM traffic over algorithmic bytes for one launch, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the medium profiling case (64 bands, 512 projectors, 41,657 plane waves;
# profiles/tcq_kernels_medium_64bands.md).  The formatted operand images are the reason it exceeds 1:
# the projector table is read as TF32 hi and lo images (2x), expanded to 2x2 real blocks for the add (4x).
NCU_TRAFFIC_RATIO = {
    "nonlocal_project": (426.996736e6 + 14.766592e6) / ((512 + 64) * 41657 * 8 + 512 * 64 * 16),
    "nonlocal_add": (706.371584e6 + 18.200576e6) / ((512 + 2 * 64) * 41657 * 8 + 64 * 512 * 16),
    # the same ratio for a Gram matrix of two 136-band blocks and for the in-place projection
    # W -= X (X^H W) of 136 bands, from the bounded medium solve (profiles/tcq_gram_kernel_medium_solve.md,
    # profiles/tcq_nn_kernel_medium_solve.md): formatted images read once, tile re-reads from L2
    "gram": (362.928896e6 + 10.022144e6) / ((136 + 136) * 41657 * 8 + 136 * 136 * 16),
    "rotate": (227.311360e6 + 16.754176e6) / ((136 + 2 * 136) * 41657 * 8 + 136 * 136 * 16),
}
METRIC = "states converged/s to 1e-6 residual (mixed+learned vs plain FP64); Hψ HBM GB/s"
TOL = 1e-6
TOL_EPS = 1e-5


def golden_nearest(name, e_ref, nstates):
    """The nstates eigenvalues nearest e_ref from the stored golden spectrum of
    the workload (sorted), or None when the workload has none."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}_spectrum.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        ev = np.asarray(json.load(f)["eigenvalues"])
    order = np.lexsort((ev, np.abs(ev - e_ref)))
    return np.sort(ev[order[:nstates]])


def count_converged(r, gold):
    """States with residual <= TOL; with a golden set, only while the sorted
    returned eigenvalues match it to TOL_EPS (one to one in sorted order)."""
    ok = np.asarray(r["resid"]) <= TOL
    if gold is None:
        return int(ok.sum())
    order = np.argsort(r["eps"])
    match = np.abs(np.asarray(r["eps"])[order] - gold) <= TOL_EPS
    return int(np.sum(ok[order] & match))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(name, rank):
    """Rank 0 solves the named seeded instance; every other rank an instance
    of the same shape with its own seed (independent problems)."""
    import fs_inputs as fi
    return fi.make_config(name, seed=1908 + 1000 * rank) if rank else fi.make_config(name)


def combine_ranks(dist, dev, t_dev, nconv, t_e2e, e2e_states):
    """Whole-job figures over the ranks: the slowest rank's times and the
    states converged by all ranks (no collective when dist is None)."""
    if dist is None:
        return t_dev, nconv, t_e2e, e2e_states
    import torch
    tt = torch.tensor([t_dev, float(nconv), t_e2e, float(e2e_states)], dtype=torch.float64, device=dev)
    gathered = [torch.zeros_like(tt) for _ in range(dist.get_world_size())]
    dist.all_gather(gathered, tt)
    return (max(float(g[0]) for g in gathered), sum(int(g[1]) for g in gathered),
            max(float(g[2]) for g in gathered), sum(int(g[3]) for g in gathered))


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    res = cpu_baseline(args.workload, None)
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": "states/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["seconds_per_solve"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": res["desc"], "precision": "fp64 (oracle)", "tol": TOL, "sample": res["sample"]},
            "cpu_baseline": {"value": res["value"], "unit": "states/s", "cores": res["cores"],
                             "kind": "oracle", "sample": res["sample"], "tiny_full_solve": res["tiny_full_solve"]},
            "e2e": {"value": res["value"], "unit": "states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(name, gpu_counts):
    """Time the CPU FP64 oracle on a bounded sample of the workload and scale
    it to one solve with the GPU solve's operation counts (or, without them,
    with the iteration count the oracle needs on the tiny workload)."""
    import fs_inputs as fi
    from oracle import planewave as pw
    w = workload(name, 0)
    cores = os.cpu_count()
    t0 = time.time()
    h = pw.Hamiltonian(w)
    t_setup = time.time() - t0
    nb = 8
    X = fi.raw_start_block(nb, h.npw, 3)
    t0 = time.time()
    h.apply(X, w.e_ref)
    t_h = (time.time() - t0) / nb                      # seconds per band application of H
    m = w.nbands
    Xb = fi.raw_start_block(m, h.npw, 4)
    t0 = time.time()
    _ = Xb.conj() @ Xb.T
    t_gram = time.time() - t0                            # one m x m Gram product, K = npw
    gram_flops = 8.0 * m * m * h.npw
    if gpu_counts is None:
        # per iteration: 2 m band applications of H + about 9 m x m-sized Gram-type products
        per_iter = 2 * m * t_h + 9 * 4 * t_gram
        iters = gpu_counts_iters = 150
        est = iters * per_iter
        how = f"assumed {gpu_counts_iters} iterations"
    else:
        est = gpu_counts["n_hpsi"] * t_h + gpu_counts["gemm_flops"] / gram_flops * t_gram
        how = "scaled by the GPU solve's H applications and GEMM flops"
    value = w.nstates / est
    sample = (f"extrapolated: oracle H on {nb} bands ({t_h * 1e3:.1f} ms/band) and one {m}x{m} Gram product over "
              f"{h.npw} plane waves ({t_gram:.2f} s), {how}; setup {t_setup:.1f} s")
    return dict(value=value, cores=cores, sample=sample, seconds_per_solve=est, desc=workload_desc(name, w, h.npw),
                tiny_full_solve=oracle_tiny_solve())


def oracle_tiny_solve():
    """A complete oracle solve (FP64 block PCG) of the tiny workload, measured: the
    one configuration where the CPU solve runs to convergence in seconds."""
    import fs_inputs as fi
    from oracle import folded as fo
    from oracle import planewave as pw
    w = fi.make_config("tiny")
    h = pw.Hamiltonian(w)
    x0 = fi.raw_start_block(w.nbands, h.npw, 17)
    t0 = time.time()
    r = fo.solve_folded(w, w.e_ref, w.nstates, TOL, x0, ham=h)
    dt = time.time() - t0
    n = int(np.sum(np.asarray(r["resid"]) <= TOL))
    return {"value": n / dt, "unit": "states/s", "seconds": dt, "iters": int(r["iters"]), "nconv": n,
            "kind": "measured", "workload": "tiny: grid (16, 16, 32), 1069 PWs, 8 states nearest 0.3 Ha"}


def workload_desc(name, w, npw):
    """The workload string both arms report in config.workload."""
    return (f"{name}: grid {tuple(w.n)}, {npw} PWs, {w.natom} atoms, {w.nproj} proj/atom, "
            f"{w.nstates} states nearest E_ref={w.e_ref:.6f} Ha")


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import fs_inputs as fi
    import paper_1907_06821_gb300 as fs
    from paper_1907_06821_gb300 import build as b

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    b.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    w = workload(args.workload, rank)
    prec = fs.FS_MIXED if args.precision == "mixed" else fs.FS_FP64
    stream = torch.cuda.Stream(device=dev)
    ctx = fs.Context.from_workload(w, precision=prec, maxit=args.maxit, stream=stream.cuda_stream,
                                   seed=1907)
    x0_host = fi.raw_start_block(w.nbands, ctx.npw, 17)
    x0_dev = torch.from_numpy(x0_host).to(dev)
    torch.cuda.synchronize()

    def step():
        ctx.set_initial_states(x0_dev, damp=True)
        return ctx.solve(w.e_ref, w.nstates, tol=TOL, allow_unconverged=True)

    # the last warm-up step is timed with the kernel-class events off: the timed
    # region below records them (for the roofline), and this shows what they cost
    t_unprof = None
    for i in range(args.warmup):
        if i == args.warmup - 1:
            ea = torch.cuda.Event(enable_timing=True)
            eb = torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            step()
            eb.record(stream)
            torch.cuda.synchronize()
            t_unprof = ea.elapsed_time(eb) / 1e3
        else:
            step()
    sampler = ClockSampler(dev.index if ws == 1 else local)
    ctx.profile(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    t_dev = ev0.elapsed_time(ev1) / 1e3
    allstats = ctx.kernel_stats()
    # "dense.*" classes time parts of the dense algebra inside "dense_la" (contained, not added)
    stats = {k: v for k, v in allstats.items() if not k.startswith("dense.")}
    dense_parts = {k[len("dense."):]: v for k, v in allstats.items() if k.startswith("dense.")}
    ctx.profile(False)
    # end-to-end through the C ABI with pinned host buffers: start block H2D, solve, states D2H
    x0_pinned = torch.from_numpy(x0_host).pin_memory()
    states_pinned = torch.empty((w.nstates, ctx.npw), dtype=torch.complex128).pin_memory()
    t0 = time.time()
    e2e_states = 0
    for _ in range(args.steps):
        ctx.set_initial_states(x0_pinned, damp=True)
        r = ctx.solve(w.e_ref, w.nstates, tol=TOL, allow_unconverged=True)
        ctx.get_states(w.nstates, out=states_pinned)
        e2e_states += count_converged(r, golden_nearest(args.workload, w.e_ref, w.nstates) if rank == 0 else None)
    t_e2e = time.time() - t0
    gold = golden_nearest(args.workload, w.e_ref, w.nstates) if rank == 0 else None
    nconv = sum(count_converged(r, gold) for r in results)
    tmax, nconv, t_e2e, e2e_states = combine_ranks(dist, dev, t_dev, nconv, t_e2e, e2e_states)
    if rank == 0:
        hbm, bf16, smax, src = peaks()
        line = make_line(args, w, ctx, results, stats, nconv, tmax, t_e2e, e2e_states, clocks, hbm, bf16, src, ws,
                         x0_host, gold)
        line["ms_per_step_unprofiled"] = t_unprof * 1e3 if t_unprof is not None else None
        line["dense_la_parts"] = {k: {"launches": v["launches"], "ms": round(v["ms"], 2),
                                      "share_of_dense_la": round(v["ms"] / max(stats["dense_la"]["ms"], 1e-9), 4)}
                                  for k, v in dense_parts.items() if v["launches"]}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def make_line(args, w, ctx, results, stats, nconv, tmax, t_e2e, e2e_states, clocks, hbm, bf16, src, ws, x0_host,
              gold=None):
    r0 = results[0]
    hpsi = ("col_inverse_fft", "plane_fft_vloc", "col_forward_fft")
    hpsi_ms = sum(stats[k]["ms"] for k in hpsi)
    hpsi_bytes = sum(stats[k]["bytes"] for k in hpsi)
    # the algorithmic bytes of one band application of the local term (FP32): sphere in
    # and out, two 3-D FFTs of two grid passes each (read + write of the full grid)
    ng = int(np.prod(w.n))
    hpsi_alg_band = 2.0 * ctx.npw * 8 + 2 * 2 * 2 * ng * 8.0
    # band applications behind the FP32 classes: each z-inverse launch counts (npw + n2 ncol) x 8 bytes a band
    g = ctx.gvectors()
    ncol = len(np.unique(np.asarray(g)[:, 0] * 100003 + np.asarray(g)[:, 1]))
    hpsi_bands = stats["col_inverse_fft"]["bytes"] / ((ctx.npw + w.n[2] * ncol) * 8.0)
    # roofline of the library's dominant GEMM / FFT / vector class in the FP32 stage (the FP64
    # dense algebra is latency- and FP64-bound, and the FP64 classes are the final check; their
    # shares are reported in kernel_time_share and dense_la_parts)
    own = {k: v for k, v in stats.items()
           if k not in ("dense_la", "nonlocal_D") and not k.endswith("_fp64") and v["ms"] > 0}
    top = max(own, key=lambda k: own[k]["ms"])
    fp32 = args.precision == "mixed"
    st = stats[top]
    sec = st["ms"] / 1e3
    gbs = st["bytes"] / sec / 1e9                      # algorithmic bytes per second
    tfs = st["flops"] / sec / 1e12                     # algorithmic flops per second
    avg_bytes = st["bytes"] / max(st["launches"], 1)   # algorithmic bytes per launch
    traffic = NCU_TRAFFIC_RATIO[top] * avg_bytes if top in NCU_TRAFFIC_RATIO else None
    if top in ("gram", "rotate", "nonlocal_project", "nonlocal_add"):
        if fp32:
            # tcgen05 kind::tf32 with a 3-term split: TF32 peak = measured BF16 peak x nominal TF32/BF16 ratio
            cpeak, cbound = bf16 * (1.1 / 2.25), "tensor"
            csrc = f"{src} bf16_tflops x 1.1/2.25 (TF32); the TF32 x3 split runs 3 MMAs per product"
        else:
            cpeak, cbound = 152 * 128 * 2 * 2.07e9 / 1e12 / 64, "alu"
            csrc = "FP64 CUDA-core peak 152 SMs x 64 FMA x 2 x 2.07 GHz / 64 (GB300 FP64 rate)"
        # the binding resource is the one the kernel runs closer to
        if tfs / cpeak >= gbs / hbm:
            roof = {"kernel": top, "bound": cbound, "achieved": tfs, "peak": cpeak, "unit": "TFLOP/s",
                    "frac": tfs / cpeak, "traffic": traffic, "peak_source": csrc}
        else:
            roof = {"kernel": top, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                    "frac": gbs / hbm, "traffic": traffic, "peak_source": f"{src} hbm_gbs"}
    else:
        roof = {"kernel": top, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "traffic": traffic, "peak_source": f"{src} hbm_gbs"}
    roof["traffic_note"] = ("DRAM bytes per average launch: the ncu ratio of measured to algorithmic bytes "
                            "on the medium box (profiles/) times this run's algorithmic bytes per launch (the wire "
                            "launches are too large to capture)" if traffic else None)
    gemm_flops = sum(stats[k]["flops"] for k in ("gram", "rotate", "nonlocal_project", "nonlocal_add"))
    n_hpsi = sum(r["n_hpsi"] for r in results) / len(results)
    counts = {"n_hpsi": n_hpsi, "gemm_flops": gemm_flops / len(results)}
    cpu = None
    if not args.no_cpu and ws == 1:
        c = cpu_baseline(args.workload, counts)
        cpu = {"value": c["value"], "unit": "states/s", "cores": c["cores"], "kind": "oracle", "sample": c["sample"],
               "tiny_full_solve": c["tiny_full_solve"]}
    total_ms = sum(v["ms"] for v in stats.values())
    fp64 = None
    if fp32 and ws == 1 and getattr(args, "fp64_full", False):
        fp64 = plain_fp64_full(args, w, x0_host, gold)
    elif fp32 and not args.no_fp64 and ws == 1:
        fp64 = plain_fp64_sample(args, w, x0_host, r0["iters"])
    comparison = precision_comparison() if fp32 and not args.no_fp64 and ws == 1 else None
    return {
        "metric": METRIC, "value": nconv / tmax, "unit": "states/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, w, ctx.npw),
                   "precision": args.precision, "tol": TOL, "l2": "inputs larger than L2 (each band block "
                   f"{w.nbands * ctx.npw * (8 if fp32 else 16) / 1e6:.0f} MB)", "start_block_seed": 17},
        "roofline": roof,
        "hpsi_gbs": hpsi_bytes / (hpsi_ms / 1e3) / 1e9 if hpsi_ms > 0 else None,
        "hpsi_frac_hbm": (hpsi_bytes / (hpsi_ms / 1e3) / 1e9) / hbm if hpsi_ms > 0 else None,
        "hpsi_algorithmic": {"bytes_per_band": hpsi_alg_band, "bands": hpsi_bands,
                        "GB/s": hpsi_alg_band * hpsi_bands / (hpsi_ms / 1e3) / 1e9 if hpsi_ms > 0 else None,
                        "frac_hbm": hpsi_alg_band * hpsi_bands / (hpsi_ms / 1e3) / 1e9 / hbm if hpsi_ms > 0 else None,
                        "note": "algorithmic bytes of the local term per band (sphere in and out, "
                                "2 FFTs x 2 grid passes x read+write of the full grid, FP32) over the event time "
                                "of the three FFT kernels"},
        "kernel_time_share": {k: round(v["ms"] / total_ms, 4) for k, v in stats.items() if total_ms > 0},
        "kernel_stats": {k: {"launches": v["launches"], "ms": round(v["ms"], 2),
                             "GB/s": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                             "TFLOP/s": round(v["flops"] / max(v["ms"], 1e-9) / 1e9, 2)} for k, v in stats.items()},
        "solve": {"nconv": r0["nconv"], "iters": r0["iters"], "iters_mixed": r0["iters_mixed"],
                  "n_hpsi": r0["n_hpsi"], "max_resid": float(np.max(r0["resid"])), "status": r0["status"],
                  "nconv_vs_golden": count_converged(r0, gold) if gold is not None else None,
                  "max_deps_vs_golden": float(np.abs(np.sort(r0["eps"]) - gold).max()) if gold is not None else None},
        "cpu_baseline": cpu,
        "plain_fp64_gpu": fp64,
        "precision_comparison": comparison,
        "e2e": {"value": e2e_states / t_e2e, "unit": "states/s",
                "h2d_bytes_per_step": int(x0_host.nbytes), "d2h_bytes_per_step": int(w.nstates * ctx.npw * 16)},
        "gpu_launches": int(sum(v["launches"] for v in stats.values())),
        "clocks": clocks,
    }


def plain_fp64_sample(args, w, x0_host, iters_mixed, nit=2):
    """The plain FP64 GPU solver on the same inputs, timed over a bounded number
    of iterations and extrapolated to the mixed solve's iteration count (the
    algorithm and its iteration count are the same; FP64 only changes the
    arithmetic)."""
    import time as _t
    import paper_1907_06821_gb300 as fs
    ctx = fs.Context.from_workload(w, precision=fs.FS_FP64, maxit=1)
    ctx.set_initial_states(x0_host, damp=True)
    t0 = _t.time()
    ctx.solve(w.e_ref, w.nstates, tol=TOL, allow_unconverged=True)
    t1 = _t.time() - t0                      # start + 1 iteration + final step
    ctx.close()
    ctx = fs.Context.from_workload(w, precision=fs.FS_FP64, maxit=1 + nit)
    ctx.set_initial_states(x0_host, damp=True)
    t0 = _t.time()
    ctx.solve(w.e_ref, w.nstates, tol=TOL, allow_unconverged=True)
    t2 = _t.time() - t0
    ctx.close()
    per_it = (t2 - t1) / nit
    est = t1 + per_it * max(iters_mixed - 1, 0)
    return {"value": w.nstates / est, "unit": "states/s", "seconds_per_iteration": per_it,
            "sample": f"FP64 solver timed for 1 and {1 + nit} iterations, extrapolated to "
                      f"{iters_mixed} iterations (the mixed solve's count)", "kind": "extrapolated"}


def precision_comparison():
    """Mixed precision against the plain FP64 GPU solver, both run to convergence
    from the same start block on the medium box (41,657 plane waves, 512
    projectors, 128 states nearest 0.05 Ha), where a plain FP64 solve takes about
    a minute: measured, not extrapolated.  A state counts when its residual is
    <= 1e-6; the two eigenvalue sets must agree to 1e-5 Ha."""
    import torch
    import fs_inputs as fi
    import paper_1907_06821_gb300 as fs
    w = fi.make_medium()
    out = {"workload": f"medium: grid {tuple(w.n)}, {w.natom} atoms, {w.nproj} proj/atom, "
                       f"{w.nstates} states nearest E_ref={w.e_ref} Ha", "kind": "measured"}
    eps = {}
    for name, prec in (("mixed", fs.FS_MIXED), ("fp64", fs.FS_FP64)):
        ctx = fs.Context.from_workload(w, precision=prec, maxit=3000)
        out.setdefault("npw", ctx.npw)
        x0 = fi.raw_start_block(w.nbands, ctx.npw, 17)
        ctx.set_initial_states(x0, damp=True)
        ctx.solve(w.e_ref, w.nstates, tol=TOL, allow_unconverged=True)    # warm-up (allocations, images)
        ctx.set_initial_states(x0, damp=True)
        torch.cuda.synchronize()
        t0 = time.time()
        r = ctx.solve(w.e_ref, w.nstates, tol=TOL, allow_unconverged=True)
        torch.cuda.synchronize()
        dt = time.time() - t0
        ctx.close()
        n = int(np.sum(np.asarray(r["resid"]) <= TOL))
        eps[name] = np.sort(r["eps"])
        out[name] = {"value": n / dt, "unit": "states/s", "seconds": dt, "iters": r["iters"], "nconv": n,
                     "n_hpsi": r["n_hpsi"], "max_resid": float(np.max(r["resid"]))}
    out["max_deps_between"] = float(np.abs(eps["mixed"] - eps["fp64"]).max())
    out["speedup_mixed_over_fp64"] = out["mixed"]["value"] / max(out["fp64"]["value"], 1e-300)
    return out


def plain_fp64_full(args, w, x0_host, gold):
    """The plain FP64 GPU solver (FP64 FFTs, FP64 GEMMs, no precision ladder) run
    to convergence on the same inputs: measured, not extrapolated."""
    import torch
    import paper_1907_06821_gb300 as fs
    ctx = fs.Context.from_workload(w, precision=fs.FS_FP64, maxit=args.maxit)
    ctx.set_initial_states(x0_host, damp=True)
    torch.cuda.synchronize()
    t0 = time.time()
    r = ctx.solve(w.e_ref, w.nstates, tol=TOL, allow_unconverged=True)
    torch.cuda.synchronize()
    dt = time.time() - t0
    ctx.close()
    n = count_converged(r, gold)
    return {"value": n / dt, "unit": "states/s", "seconds": dt, "iters": r["iters"], "nconv": n,
            "n_hpsi": r["n_hpsi"], "kind": "measured",
            "sample": "one complete FP64 solve from the same start block (FP64 FFTs and GEMMs throughout)"}


def run_batched(args):
    """The batched-fragments workload: independent boxes of uneven grid
    (32^3, 40^3, 48^3, 64^3, 48x48x96), 8-64 wells, 32-128 states each, 15 Ry
    cutoff, solved concurrently (fs_batch_solve); metric: states/s of the batch."""
    import torch
    import fs_inputs as fi
    import paper_1907_06821_gb300 as fs
    from paper_1907_06821_gb300 import build as b
    b.build()
    boxes = fi.make_batch(args.nbox)
    ctxs = [fs.Context.from_workload(w, precision=fs.FS_MIXED, maxit=args.maxit) for w in boxes]
    tiles = {}
    for w, c in zip(boxes, ctxs):
        tiles[str(tuple(w.n))] = c.autotune()
    x0 = [fi.raw_start_block(w.nbands, c.npw, 17) for w, c in zip(boxes, ctxs)]
    batch = fs.Batch(ctxs, nthreads=args.threads)

    def step():
        for c, x in zip(ctxs, x0):
            c.set_initial_states(x, damp=True)
        return batch.solve([w.e_ref for w in boxes], [w.nstates for w in boxes], tol=TOL)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    t0 = time.time()
    res = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    dt = time.time() - t0
    clocks = sampler.stop()
    nconv = sum(r["nconv"] for rr in res for r in rr)
    wanted = sum(w.nstates for w in boxes) * args.steps
    line = {"metric": METRIC, "value": nconv / dt, "unit": "states/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"batched: {len(boxes)} boxes, grids {sorted(set(tuple(w.n) for w in boxes))}, "
                                   f"{sum(w.nstates for w in boxes)} states in total",
                       "threads": args.threads, "fft_tiles": tiles},
            "converged_fraction": nconv / wanted,
            "max_resid": float(max(np.max(r["resid"]) for rr in res for r in rr)),
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    batch.close()
    for c in ctxs:
        c.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="wire", choices=["wire", "tiny", "batched"])
    ap.add_argument("--nbox", type=int, default=96)
    ap.add_argument("--threads", type=int, default=16)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--maxit", type=int, default=3000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain FP64 GPU sample and the measured precision comparison")
    ap.add_argument("--fp64-full", action="store_true",
                    help="run the plain FP64 GPU solve to convergence (minutes) instead of the timed sample")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

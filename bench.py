#!/usr/bin/env python
"""Throughput benchmark: right-hand sides solved per second at GMRES rtol 1e-6.

Workload (default): the Overthrust-like synthetic model at 5 Hz — 20 x 20 x
4.65 km, graded Kuhn tensor grid at 1.3 P3 cells per local minimum
wavelength, Dirichlet free surface on top and absorbing faces elsewhere,
64 box subdomains with one element layer of overlap, a nested 2x coarser
mesh for the coarse level, 16 surface sources at z = 100 m. One step = one
hz_solve of the 16 sources (FGMRES + two-level ORAS to rtol 1e-6), factors
resident on the device (setup reported separately, not timed).

Both forms are measured on the same GPU: FP64 and mixed (local fronts in
complex FP32, everything else FP64); `value` is the mixed form, `forms`
holds both. `e2e` repeats the mixed-form step through the C ABI with host
output buffers (device-to-host copy of the wavefields inside the timed
region). `roofline` covers the dominant kernel family (the fine-level local
solves), timed with CUDA events inside the library over the timed region.
`cpu_baseline` times the CPU oracle (assembly + SuperLU) on a bounded crop
of the same workload.

Multi-GPU (torchrun): sources are independent, so every rank holds its own
replica of the factors and solves its own 16 sources (weak scaling, no
collective on the data path); the barrier and the max over ranks only
frame the timing.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_GFLOPS = 1250.0  # nominal GB300 FP64 rate, context only (the FP64 peak is measured live)
TILE_PROFILE = os.path.join(ROOT, "profiles", "k_mf_tile_overthrust5_quarter.md")


def fronts_traffic(cfg, per_app):
    """DRAM bytes of one application of the fine local solves: the ratio of
    DRAM traffic to algorithmic bytes that ncu measured on the quarter crop
    (profiles/k_mf_tile_overthrust5_quarter.md) times this run's algorithmic
    bytes; None when the profile is absent or for the cube, whose factors
    fit in L2."""
    if cfg == "cube":
        return None
    try:
        with open(TILE_PROFILE) as f:
            for ln in f:
                if ln.startswith("| dram_over_algorithmic |"):
                    return float(ln.split("|")[2]) * per_app
    except OSError:
        pass
    return None


def fp32_simt_tflops(torch, sm_max_mhz):
    """FP32 SIMT peak derived from the device: SMs (queried) x 128 FP32 lanes
    x 2 flops per FMA x the maximum SM clock (MEASURED_PEAKS.json)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_max_mhz or 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


def measure_gemm_peaks(torch):
    """Live GEMM rates on this GPU (cuBLAS through torch.matmul, best of 5
    after warm-up, CUDA events): FP64 (DGEMM), FP32 without TF32 (SGEMM) and
    TF32 tensor-core GEMM, N = 8192 (FP64: 4096). They are the measured
    denominators of the FP64 and FP32 rooflines."""
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, n, tf32 in (("fp64_gemm_tflops", torch.float64, 4096, False),
                                  ("fp32_gemm_tflops", torch.float32, 8192, False),
                                  ("tf32_gemm_tflops", torch.float32, 8192, True)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            for _ in range(2):
                torch.matmul(a, b)
            best = None
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    out["how"] = "torch.matmul (cuBLAS), square N=8192 (FP64 N=4096), best of 5 after 2 warm-up, CUDA events"
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["overthrust5", "overthrust5_quarter", "overthrust10", "cube"],
                    default="overthrust5",
                    help="overthrust5_quarter: the 10 x 10 km corner of the same model (profiling case); "
                         "overthrust10: the same model at 10 Hz, 256 subdomains, 64 sources (mixed precision at scale)")
    ap.add_argument("--forms", default="mixed,fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the FP64 form")
    ap.add_argument("--fp64-warmup", type=int, default=1, help="warm-up steps of the FP64 form")
    ap.add_argument("--variants", default="one_level,block,coarse_fp32,paper_resolution",
                    help="extra variants of the headline form: one_level (one-level ORAS; also runs the short "
                         "serving stream), coarse_fp32 (mixed form with the coarse level in complex FP32), "
                         "paper_resolution (two- and one-level at 1.3 Hz on the same mesh: 5 P3 cells per "
                         "local wavelength as in the paper, coarse mesh at 2.5), block (one-level ORAS with "
                         "block FGMRES, CGS2 + CholQR2, one block of up to 16 sources)")
    ap.add_argument("--maxit", type=int, default=500, help="FGMRES iteration cap (lower it only for profiling runs)")
    ap.add_argument("--max-block", type=int, default=0,
                    help="right-hand sides per block (0: the library default, 64; the 10 Hz workload needs 16 to fit)")
    ap.add_argument("--coarse", choices=["gmres", "none", "direct"], default="gmres",
                    help="coarse level of the headline forms (the paper's: gmres, 10 inner steps)")
    ap.add_argument("--tensor-cores", type=int, choices=[-1, 0, 1], default=-1,
                    help="mixed form: front sweeps on the tcgen05 tensor cores (1) or SIMT (0); -1: library default")
    ap.add_argument("--persistent", type=int, choices=[-1, 0, 1], default=-1,
                    help="SIMT front sweeps as one launch per direction (1) or one per level (0); -1: library default")
    ap.add_argument("--leaf-size", type=int, default=0, help="nested-dissection leaf size (0: library default)")
    ap.add_argument("--coarse-leaf-size", type=int, default=-1,
                    help="leaf size of the coarse level's local problems (-1: library default)")
    ap.add_argument("--emulate-fp64", type=int, choices=[-1, 0, 1], default=-1,
                    help="mixed form: FP64 products and Arnoldi as FP32 pairs (1) or native FP64 (0); -1: default")
    ap.add_argument("--spmm-sweep", action="store_true",
                    help="instead of the throughput line: HBM and FP64 rates of the product with A "
                         "(hz_apply_A, device blocks) for block widths 1..16 on the bench workload")
    ap.add_argument("--serving", action="store_true",
                    help="instead of the throughput line: a seeded Poisson stream of point-source requests over "
                         "several frequencies through the continuous-batching server (p50/p99 latency, RHS/s)")
    ap.add_argument("--serving-freqs", default="3.5,5,7")
    ap.add_argument("--serving-requests", type=int, default=400)
    ap.add_argument("--serving-rate", type=float, default=2.0, help="mean request arrivals per second")
    ap.add_argument("--serving-loads", default="",
                    help="comma-separated fractions of the measured saturation rate (e.g. 0.5,0.8,1.2): "
                         "calibrate, then run the same seeded stream at each offered load")
    ap.add_argument("--serving-slots", type=int, default=32, help="right-hand-side slots per frequency "
                    "(when --serving-budget-gb is 0)")
    ap.add_argument("--serving-budget-gb", type=float, default=60.0,
                    help="device bytes shared by the servers' slots (admission by footprint); 0: fixed slots")
    ap.add_argument("--serving-coarse", choices=["gmres", "none", "direct"], default="none",
                    help="coarse level of the serving solvers (one-level ORAS by default: on these meshes it "
                         "converges in fewer iterations than the two-level form)")
    return ap.parse_args()


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz")
    except Exception:
        return 6800.0, "fallback", None


def problem(cfg):
    from paper_2004_07930_gb300 import workloads as wl

    if cfg == "cube":
        return wl.cube_problem(), "cube 1 km, 6^3 cells, P3 (6859 dofs), 2 Hz, 4 subdomains, 1 source"
    if cfg == "overthrust5_quarter":
        p = wl.overthrust_problem(5.0, nparts=16, seed=0, crop=(0.5, 0.5, 1.0),
                                  sources=wl.surface_source_grid(4, 4, 1250.0, 8750.0))
        nx, ny, nz = p["fine"]["ncells"]
        return p, ("Overthrust-like 5 Hz, 10x10 km corner crop, %dx%dx%d cells, 16 subdomains, %d sources"
                   % (nx, ny, nz, len(p["src_xyz"])))
    if cfg == "overthrust10":
        p = wl.overthrust_problem(10.0, nparts=256, seed=0,
                                  sources=wl.surface_source_grid(8, 8, 1250.0, 18750.0))
        nx, ny, nz = p["fine"]["ncells"]
        return p, ("Overthrust-like 20x20x4.65 km, 10 Hz, %dx%dx%d cells x 6 Kuhn tets, P3, 256 subdomains "
                   "(16x16x1), overlap 1, nested coarse mesh, 64 surface sources (8x8 grid)" % (nx, ny, nz))
    p = wl.overthrust_problem(5.0, nparts=64, seed=0)
    nx, ny, nz = p["fine"]["ncells"]
    return p, ("Overthrust-like 20x20x4.65 km, 5 Hz, %dx%dx%d cells x 6 Kuhn tets, P3, 64 subdomains "
               "(8x8x1), overlap 1, nested coarse mesh, 16 surface sources" % (nx, ny, nz))


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, ws):
    """Largest value over the ranks (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(cfg="overthrust5"):
    """Oracle (assembly + SuperLU + triangular solves) on a bounded sample of
    the workload: for the Overthrust-like configs a corner of 8 x 8 cells
    (about 2.8 x 2.8 km, full depth) with 2 sources, for the cube the whole
    cube with its source."""
    from oracle import assemble as oa
    from paper_2004_07930_gb300 import workloads as wl

    t0 = time.time()
    if cfg == "cube":
        p = wl.cube_problem()
        what = "the whole 6^3-cell cube"
    else:
        p = wl.overthrust_problem(5.0, nparts=4, crop=(0.125, 0.125, 1.0),
                                  sources=[[1250.0, 1250.0, 100.0], [2000.0, 1000.0, 100.0]])
        what = "an 8x8-cell (2.8x2.8x4.65 km) corner crop of the same 5 Hz workload"
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    import scipy.sparse.linalg as spla

    lu = spla.splu(A.tocsc())
    lu.solve(F.T.copy())
    elapsed = time.time() - t0
    ns = F.shape[0]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": ns / elapsed, "unit": "RHS/s", "cores": 1, "kind": "oracle",
            "host_cores_available": cores,
            "sample": "oracle (P3 assembly + SciPy SuperLU, single-threaded) on %s: n=%d dofs, %d sources, "
                      "%.1f s" % (what, space.n, ns, elapsed),
            "n_sample": int(space.n), "rhs": int(ns), "seconds": elapsed}


def run_reference(args):
    """The oracle as the reference arm: --warmup untimed and --steps timed
    samples (cpu_baseline), value = right-hand sides / seconds over the timed
    ones. Rank 0 only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    _, desc = problem(args.config)
    timed = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(args.config)
        if i >= args.warmup:
            timed.append(cb)
    rhs = sum(c["rhs"] for c in timed)
    sec = sum(c["seconds"] for c in timed)
    value = rhs / sec
    cb = dict(timed[-1])
    cb["value"] = value
    cb["sample"] = "%d timed samples, each: %s" % (len(timed), cb["sample"])
    out = {"impl": "reference", "metric": "RHS solved/s at rtol 1e-6", "value": value, "unit": "RHS/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / len(timed),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic (seeded Overthrust-like model; no real data)",
           "config": {"workload": desc, "reference": "CPU oracle: direct solve of the same discretisation"},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def serving_stream(S, hz, rhs_per_s, nreq=24, load=0.8, seed=11, budget_gb=40.0):
    """A short seeded Poisson stream through the continuous-batching server
    on the solver S: nreq requests of 1-16 point sources at uniform surface
    positions (z = 100 m), offered at `load` x the measured saturated rate
    rhs_per_s, slots admitted by device footprint within budget_gb. Returns
    RHS/s and p50/p99 latency (arrival to completion)."""
    import numpy as np

    from paper_2004_07930_gb300.serve import ServingLoop

    rng = np.random.Generator(np.random.PCG64(seed))
    nsrc = rng.integers(1, 17, nreq)
    rate = load * rhs_per_s / nsrc.mean()           # requests per second
    arrival = np.cumsum(rng.exponential(1.0 / rate, nreq))
    reqs = []
    for i in range(nreq):
        xy = rng.uniform(1000.0, 19000.0, size=(nsrc[i], 2))
        reqs.append((float(arrival[i]), i, 0, np.concatenate([xy, np.full((nsrc[i], 1), 100.0)], axis=1)))
    loop = ServingLoop({0: S}, device_budget=budget_gb * 1e9)
    summ = loop.run_stream(reqs)
    loop.close()
    summ.update({"offered_load": load, "offered_rhs_per_s": load * rhs_per_s, "slot_budget_gb": budget_gb,
                 "column_gb": S.column_bytes() / 1e9,
                 "stream": "%d requests, 1-16 sources each, Poisson arrivals (PCG64 seed %d)" % (nreq, seed)})
    return summ


def measure_form(prob, form, steps, warmup, stream, ws, torch, hz, with_e2e, serve=False, **opts):
    prec = hz.HZ_PREC_MIXED if form == "mixed" else hz.HZ_PREC_FP64
    if TENSOR_CORES >= 0:
        opts["tensor_cores"] = TENSOR_CORES
    if PERSISTENT >= 0:
        opts["persistent_sweeps"] = PERSISTENT
    if EMULATE >= 0:
        opts["emulate_fp64"] = EMULATE
    if LEAF > 0:
        opts["leaf_size"] = LEAF
    if CLEAF >= 0:
        opts["coarse_leaf_size"] = CLEAF
    if MAX_BLOCK > 0:
        opts["max_block"] = MAX_BLOCK
    t0 = time.time()
    S = hz.Solver.from_problem(prob, precision=prec, rtol=1e-6, stream=stream, maxit=MAXIT, **opts)
    setup_wall = time.time() - t0
    info = S.info()
    src = prob["src_xyz"]
    ns = len(src)
    out = torch.empty((ns, S.n), dtype=torch.complex128, device="cuda")
    iters = []
    notconv = MAXIT < 500
    for _ in range(warmup):
        _, st = S.solve(src, out=out, raise_on_notconv=not notconv)
        iters.append(st["iterations"])
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = S.info()["kernel_launches"]
    S.profile_begin()
    e0.record(stream)
    stats = []
    for _ in range(steps):
        _, st = S.solve(src, out=out, raise_on_notconv=not notconv)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = S.profile_end()
    launches = S.info()["kernel_launches"] - launches0
    barrier(ws)
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, ws)
    res = {"rhs_per_s": ns * steps * ws / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
           "iterations": [s["iterations"] for s in stats], "max_rel_residual": max(s["max_rel_residual"] for s in stats),
           "converged": all(s["converged"] for s in stats), "setup_s": setup_wall,
           "factor_s": stats[0]["factor_seconds"], "info": info, "phases": prof, "gpu_launches": launches,
           "factor_ldlt_s": info["factor_ldlt_seconds"], "factor_inverse_s": info["factor_inverse_seconds"],
           "perturbed_pivots": info["perturbed_pivots"],
           "coarse_fp32": S.options.coarse_fp32, "overlap": S.options.overlap,
           "tensor_cores": S.options.tensor_cores, "persistent_sweeps": S.options.persistent_sweeps,
           "emulate_fp64": S.options.emulate_fp64 if prec == hz.HZ_PREC_MIXED else 0,
           "max_block": S.options.max_block, "block_arnoldi": S.options.block_arnoldi, "device_gb": S.info()["device_bytes"] / 1e9}
    if with_e2e:
        import numpy as np

        hostbuf = np.empty((ns, S.n), dtype=np.complex128)
        barrier(ws)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(steps):
            S.solve(src, out=hostbuf, raise_on_notconv=not notconv)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t, ws)
        res["e2e"] = {"value": ns * steps * ws / el, "unit": "RHS/s",
                      "h2d_bytes_per_step": int(src.size * 8 + ns * 16),
                      "d2h_bytes_per_step": int(hostbuf.nbytes)}
    if serve:
        res["serving"] = serving_stream(S, hz, res["rhs_per_s"])
        res["serving"]["preconditioner"] = "one-level ORAS" if opts.get("coarse_mode") == hz.HZ_COARSE_NONE else \
            "two-level ORAS"
    S.close()
    return res


MAXIT = 500
TENSOR_CORES = -1
PERSISTENT = -1
EMULATE = -1
LEAF = 0
CLEAF = -1
MAX_BLOCK = 0


def run_spmm_sweep(args):
    """k_spmm_split alone: for s = 1, 2, 4, 8, 16 the product Y = A X through
    hz_apply_A on device blocks, timed by the library's CUDA events around
    the product only (the layout transposes of hz_apply_A are outside the
    recorded phase). Algorithmic bytes: 12 per nonzero (value + column),
    row pointers, X and Y once; flops: 4 per nonzero and column."""
    import torch

    from paper_2004_07930_gb300 import hz

    torch.cuda.set_device(0)
    hz.load()
    prob, desc = problem(args.config)
    hbm, peak_kind, _ = peaks()
    out = {}
    with hz.Solver.from_problem(prob, precision=hz.HZ_PREC_FP64, coarse_mode=hz.HZ_COARSE_NONE) as S:
        for s in (1, 2, 4, 8, 16):
            X = torch.randn((s, S.n), dtype=torch.complex128, device="cuda")
            for _ in range(3):
                S.apply_A(X)
            torch.cuda.synchronize()
            S.profile_begin()
            for _ in range(20):
                S.apply_A(X)
            ph = S.profile_end()["spmm_A"]
            sec = ph["ms"] / 1e3
            out[s] = {"calls": ph["calls"], "us_per_call": 1e6 * sec / ph["calls"],
                      "gbs": ph["bytes"] / sec / 1e9, "hbm_frac": ph["bytes"] / sec / 1e9 / hbm,
                      "fp64_gflops": ph["flops"] / sec / 1e9,
                      "fp64_frac": ph["flops"] / sec / 1e9 / FP64_NOMINAL_GFLOPS}
    print(json.dumps({"mode": "spmm_sweep", "kernel": "k_spmm_split", "config": {"workload": desc},
                      "hbm_peak_gbs": hbm, "hbm_peak_kind": peak_kind, "fp64_peak_gflops": FP64_NOMINAL_GFLOPS,
                      "by_block_width": out}), flush=True)


def run_serving(args):
    """Continuous batching of a seeded Poisson request stream: every request
    carries 1-32 point sources at uniform surface positions (z = 100 m) and
    one frequency drawn from --serving-freqs; one resident solver (mixed form,
    rtol 1e-6, preconditioner from --serving-coarse) and one server of
    --serving-slots columns per frequency. Latency = arrival to completion."""
    import numpy as np
    import torch

    from paper_2004_07930_gb300 import hz
    from paper_2004_07930_gb300 import workloads as wl
    from paper_2004_07930_gb300.serve import ServingLoop

    torch.cuda.set_device(0)
    hz.load()
    freqs = [float(f) for f in args.serving_freqs.split(",") if f]
    cm = {"gmres": hz.HZ_COARSE_GMRES, "none": hz.HZ_COARSE_NONE, "direct": hz.HZ_COARSE_DIRECT}[args.serving_coarse]
    solvers, sizes, setup = {}, {}, {}
    for f in freqs:
        p = wl.overthrust_problem(f, nparts=64, seed=0)
        t0 = time.time()
        solvers[f] = hz.Solver.from_problem(p, precision=hz.HZ_PREC_MIXED, rtol=1e-6, maxit=MAXIT, coarse_mode=cm)
        setup[f] = time.time() - t0
        sizes[f] = solvers[f].n
    rng = np.random.Generator(np.random.PCG64(7))
    N = args.serving_requests
    gaps = rng.exponential(1.0, N)  # unit-rate gaps, scaled by the request rate below
    nsrc = rng.integers(1, 33, N)
    fsel = rng.integers(0, len(freqs), N)
    srcs = []
    for i in range(N):
        xy = rng.uniform(1000.0, 19000.0, size=(nsrc[i], 2))
        srcs.append(np.concatenate([xy, np.full((nsrc[i], 1), 100.0)], axis=1))
    loads = [float(x) for x in args.serving_loads.split(",") if x]
    if loads:
        # saturation: device time per right-hand side averaged over the frequency mix, from one
        # timed block of 32 seeded sources per frequency
        per_rhs = []
        for f in freqs:
            xy = rng.uniform(1000.0, 19000.0, size=(32, 2))
            src = np.concatenate([xy, np.full((32, 1), 100.0)], axis=1)
            solvers[f].solve(src[:4])
            torch.cuda.synchronize()
            t0 = time.time()
            solvers[f].solve(src)
            torch.cuda.synchronize()
            per_rhs.append((time.time() - t0) / 32)
        sat = 1.0 / float(np.mean(per_rhs))
        mean_src = float(np.mean(nsrc))
        for load in loads:
            rate = load * sat / mean_src
            arrival = np.cumsum(gaps / rate)
            reqs = [(float(arrival[i]), i, freqs[fsel[i]], srcs[i]) for i in range(N)]
            loop = ServingLoop(solvers, device_budget=args.serving_budget_gb * 1e9)
            summ = loop.run_stream(reqs)
            loop.close()
            print(json.dumps({"mode": "serving_load", "offered_fraction_of_saturation": load,
                              "saturation_rhs_per_s": sat, "offered_rhs_per_s": load * sat,
                              "request_rate_per_s": rate, "rhs_per_s": summ["rhs_per_s"],
                              "latency_p50_s": summ["latency_p50_s"], "latency_p99_s": summ["latency_p99_s"],
                              "requests": summ["requests"], "rhs": summ["rhs"], "wall_s": summ["wall_s"],
                              "converged": summ["converged"], "slots": summ.get("slots"),
                              "freqs": freqs, "n": [sizes[f] for f in freqs],
                              "setup_s": {str(f): setup[f] for f in freqs}}), flush=True)
        for S in solvers.values():
            S.close()
        return
    arrival = np.cumsum(gaps / args.serving_rate)
    reqs = [(float(arrival[i]), i, freqs[fsel[i]], srcs[i]) for i in range(N)]
    if args.serving_budget_gb > 0:
        loop = ServingLoop(solvers, device_budget=args.serving_budget_gb * 1e9)
    else:
        loop = ServingLoop(solvers, args.serving_slots)
    dev_gb = sum(S.info()["device_bytes"] for S in solvers.values()) / 1e9
    launches0 = next(iter(solvers.values())).info()["kernel_launches"]  # process-wide counter
    clocks = ClockSampler(0)
    clocks.start()
    summ = loop.run_stream(reqs)
    clk = clocks.stop()
    launches = next(iter(solvers.values())).info()["kernel_launches"] - launches0
    loop.close()
    line = {"metric": "RHS/s served (Poisson request stream, rtol 1e-6)", "value": summ["rhs_per_s"],
            "unit": "RHS/s", "n_gpus": 1, "higher_is_better": True, "mode": "serving",
            "latency_p50_s": summ["latency_p50_s"], "latency_p99_s": summ["latency_p99_s"],
            "requests": summ["requests"], "rhs": summ["rhs"], "wall_s": summ["wall_s"],
            "converged": summ["converged"], "dtype": "c64 fronts + c128 Krylov/SpMM/coarse",
            "data": "synthetic (seeded Overthrust-like model and request stream)",
            "config": {"workload": "Overthrust-like, f in %s Hz, n %s, 64 subdomains, Poisson arrivals %.2f/s, "
                                   "1-32 sources per request" % (freqs, [sizes[f] for f in freqs], args.serving_rate),
                       "slots_per_frequency": summ.get("slots"), "device_gb": dev_gb,
                       "slot_budget_gb": args.serving_budget_gb,
                       "coarse": args.serving_coarse, "setup_s": {str(f): setup[f] for f in freqs}},
            "clocks": clk, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    for S in solvers.values():
        S.close()


def run_scale(args):
    """Mixed precision at scale: the 10 Hz workload (256 subdomains, 64
    sources in blocks of --max-block), one-level ORAS (at 1.3 P3 cells per
    wavelength the coarse level slows FGMRES down). Reports RHS/s of the mixed
    form, its iterations and device footprint. The FP64 form of the full
    10 Hz problem does not fit the device (its frontal workspace alone is
    ~384 GB of complex FP64), so the mixed-vs-FP64 difference is measured on a
    corner crop of the same 10 Hz model (a quarter of each horizontal axis,
    16 subdomains, 4 sources), both forms on the GPU."""
    import numpy as np
    import torch

    from paper_2004_07930_gb300 import hz
    from paper_2004_07930_gb300 import workloads as wl

    torch.cuda.set_device(0)
    hz.load()
    prob, desc = problem("overthrust10")
    src = prob["src_xyz"]
    mb = args.max_block if args.max_block > 0 else 16
    opts = dict(rtol=1e-6, maxit=args.maxit, coarse_mode=hz.HZ_COARSE_NONE, max_block=mb)
    out = {"mode": "scale", "metric": "RHS solved/s at rtol 1e-6", "unit": "RHS/s", "n_gpus": 1,
           "config": {"workload": desc, "preconditioner": "one-level ORAS", "max_block": mb}}
    clocks = ClockSampler(0)
    t0 = time.time()
    S = hz.Solver.from_problem(prob, precision=hz.HZ_PREC_MIXED, **opts)
    out["setup_s"] = time.time() - t0
    info = S.info()
    out["config"].update({"n": info["n"], "nnz": info["nnz"], "factor_entries": info["factor_entries"],
                          "max_front": info["max_front"], "factor_ldlt_s": info["factor_ldlt_seconds"],
                          "factor_inverse_s": info["factor_inverse_seconds"]})
    S.solve(src[:mb], raise_on_notconv=False)  # warm-up block
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    u_mixed, st = S.solve(src, raise_on_notconv=False)
    e1.record()
    torch.cuda.synchronize()
    out["clocks"] = clocks.stop()
    sec = e0.elapsed_time(e1) / 1e3
    out.update({"value": len(src) / sec, "seconds": sec, "iterations": st["iterations"],
                "converged": st["converged"], "max_rel_residual": st["max_rel_residual"],
                "device_gb": S.info()["device_bytes"] / 1e9})
    S.close()
    del u_mixed
    print(json.dumps(out), flush=True)
    # mixed vs FP64 on a corner crop of the same 10 Hz model
    crop = wl.overthrust_problem(10.0, nparts=16, seed=0, crop=(0.25, 0.25, 1.0),
                                 sources=wl.surface_source_grid(2, 2, 1250.0, 3750.0))
    cmp_ = {"crop": "10 Hz, (0.25, 0.25, 1) corner crop, %dx%dx%d cells, 16 subdomains, 4 sources"
            % tuple(crop["fine"]["ncells"])}
    copts = dict(opts, max_block=4)
    u = {}
    for name, prec in (("mixed", hz.HZ_PREC_MIXED), ("fp64", hz.HZ_PREC_FP64)):
        t0 = time.time()
        with hz.Solver.from_problem(crop, precision=prec, **copts) as Sc:
            t1 = time.time()
            u[name], stc = Sc.solve(crop["src_xyz"], raise_on_notconv=False)
            cmp_[name] = {"setup_s": t1 - t0, "solve_s": time.time() - t1, "iterations": stc["iterations"],
                          "converged": stc["converged"], "max_rel_residual": stc["max_rel_residual"],
                          "device_gb": Sc.info()["device_bytes"] / 1e9, "n": Sc.n}
    d = np.linalg.norm(u["mixed"] - u["fp64"], axis=1) / np.linalg.norm(u["fp64"], axis=1)
    cmp_["mixed_vs_fp64_rel_l2"] = float(d.max())
    print(json.dumps({"mode": "scale_crop_fp64", **cmp_}), flush=True)


def main():
    global MAXIT, TENSOR_CORES, PERSISTENT, MAX_BLOCK, EMULATE, LEAF, CLEAF
    args = parse()
    MAX_BLOCK = args.max_block
    MAXIT = args.maxit
    TENSOR_CORES = args.tensor_cores
    PERSISTENT = args.persistent
    EMULATE = args.emulate_fp64
    LEAF = args.leaf_size
    CLEAF = args.coarse_leaf_size
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serving:
        run_serving(args)
        return
    if args.spmm_sweep:
        run_spmm_sweep(args)
        return
    if args.config == "overthrust10":
        run_scale(args)
        return
    ws, rank, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2004_07930_gb300 import hz

    hz.load()
    prob, desc = problem(args.config)
    stream = torch.cuda.current_stream()
    forms = [f for f in args.forms.split(",") if f]
    clocks = ClockSampler(local)
    results = {}
    for i, form in enumerate(forms):
        steps = args.steps if form != "fp64" else args.fp64_steps
        warm = args.warmup if form != "fp64" else args.fp64_warmup
        if i == 0:
            clocks.start()
        cm = {"gmres": hz.HZ_COARSE_GMRES, "none": hz.HZ_COARSE_NONE, "direct": hz.HZ_COARSE_DIRECT}[args.coarse]
        results[form] = measure_form(prob, form, steps, warm, stream, ws, torch, hz, with_e2e=(i == 0),
                                     coarse_mode=cm)
        if i == 0:
            clk = clocks.stop()
    from paper_2004_07930_gb300 import workloads as wl

    variants = {}
    for v in [x for x in args.variants.split(",") if x]:
        if v == "one_level":
            variants["one_level_" + forms[0]] = measure_form(prob, forms[0], args.steps, args.warmup, stream, ws,
                                                             torch, hz, False, coarse_mode=hz.HZ_COARSE_NONE,
                                                             serve=(forms[0] == "mixed" and ws == 1))
        elif v == "paper_resolution" and args.config == "overthrust5":
            # the same mesh at the paper's resolution: 5 P3 cells per local minimum wavelength
            # (Sec. "Numerical results"), i.e. 1.3 Hz on the 5 Hz grid; coarse mesh at 2.5 cells per wavelength
            p2 = wl.overthrust_problem(1.3, nparts=64, seed=0, cells_per_wavelength=5.0)
            for nm, c2 in (("two_level", cm), ("one_level", hz.HZ_COARSE_NONE)):
                variants["paper_resolution_%s_%s" % (nm, forms[0])] = measure_form(
                    p2, forms[0], args.steps, args.warmup, stream, ws, torch, hz, False, coarse_mode=c2)
        elif v == "block":
            variants["block_one_level_" + forms[0]] = measure_form(prob, forms[0], args.steps, args.warmup, stream,
                                                                   ws, torch, hz, False, coarse_mode=hz.HZ_COARSE_NONE,
                                                                   block_arnoldi=1, max_block=16)
        elif v == "coarse_fp32" and forms[0] == "mixed" and args.coarse != "none":
            variants["coarse_fp32_mixed"] = measure_form(prob, "mixed", args.steps, args.warmup, stream, ws, torch,
                                                         hz, False, coarse_mode=cm, coarse_fp32=1)
    head = forms[0]
    r = results[head]
    hbm, peak_kind, sm_max = peaks()
    gemm = measure_gemm_peaks(torch)
    simt, nsm, mhz = fp32_simt_tflops(torch, sm_max)
    ph = r["phases"]["fronts"]
    per_app = ph["bytes"] / ph["calls"]  # algorithmic bytes of one application of the fine local solves
    hbm_achieved = ph["bytes"] / (ph["ms"] / 1e3) / 1e9
    flops_achieved = ph["flops"] / (ph["ms"] / 1e3) / 1e12
    tc_on = (TENSOR_CORES if TENSOR_CORES >= 0 else hz.default_options().tensor_cores) == 1
    if head == "mixed":
        pers = r.get("persistent_sweeps", 0) == 1
        kern = ("fine local solves (tcgen05 sweep tiles, 3xTF32 split, FP32 accumulation in TMEM, one launch per "
                "level)" if tc_on else "fine local solves (SIMT complex FP32 sweep tiles, %s)" %
                ("k_mf_sweep: one launch per sweep over all levels" if pers else "k_mf_tile + k_mf_reduce per level"))
        # a sweep reads each factor entry once per application: HBM is the roof of the
        # tensor-core form; the SIMT FP32 rate (16 flops per factor byte at s = 16) is given beside it
        roof = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm, "unit": "GB/s", "frac": hbm_achieved / hbm,
                "traffic": None if tc_on else fronts_traffic(args.config, per_app),
                "traffic_unit": "DRAM bytes per application of the fine local solves",
                "kernel": kern, "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_application": per_app, "applications": ph["calls"],
                "fp32_tflops_achieved": flops_achieved, "fp32_simt_peak_tflops": simt,
                "fp32_simt_frac": flops_achieved / simt,
                "fp32_simt_peak_kind": "derived: %d SMs (queried) x 128 FP32 lanes x 2 x %.0f MHz" % (nsm, mhz)}
    else:
        fp64 = gemm["fp64_gemm_tflops"]
        roof = {"bound": "alu", "achieved": flops_achieved, "peak": fp64, "unit": "TFLOP/s",
                "frac": flops_achieved / fp64, "traffic": None,
                "kernel": "fine local solves (SIMT complex FP64 sweep tiles)",
                "peak_kind": "measured live: FP64 DGEMM (cuBLAS, torch.matmul)", "hbm_achieved_gbs": hbm_achieved,
                "hbm_frac": hbm_achieved / hbm, "applications": ph["calls"]}
    phase_roof = {}
    for name, q in r["phases"].items():
        if q["calls"] and q["ms"] > 0:
            gbs = q["bytes"] / (q["ms"] / 1e3) / 1e9
            phase_roof[name] = {"share_of_step": q["ms"] / (r["ms_per_step"] * r["steps"]), "ms_per_call": q["ms"] / q["calls"],
                                "gbs": gbs, "hbm_frac": gbs / hbm,
                                "tflops": q["flops"] / (q["ms"] / 1e3) / 1e12}
    if head == "mixed":
        cf = results[head].get("coarse_fp32", 0)
        emu = results[head].get("emulate_fp64", 0)
        c128 = "FP64-class as FP32 pairs" if emu else "c128"
        dtype = ("c64 fine fronts (" + ("3xTF32 tensor cores" if tc_on else "SIMT FP32") + ") + " +
                 ("c64 coarse level + " if cf else "coarse level: c64 fronts, %s E/Krylov + " % c128) +
                 "%s Krylov/SpMM/outer residual" % c128)
    else:
        dtype = "c128"
    line = {
        "metric": "RHS solved/s at rtol 1e-6", "value": r["rhs_per_s"], "unit": "RHS/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic (seeded Overthrust-like model; no real data)",
        "config": {"workload": desc, "n": r["info"]["n"], "nnz": r["info"]["nnz"],
                   "sources_per_step": len(prob["src_xyz"]), "max_block": r.get("max_block"),
                   "rtol": 1e-6, "preconditioner": {"gmres": "two-level ORAS, coarse by 10 GMRES steps",
                                                    "none": "one-level ORAS", "direct": "two-level ORAS, direct coarse"}[args.coarse],
                   "l2_flush": "inputs larger than L2 (factors %.1f GB)" %
                   (r["info"]["device_bytes"] / 1e9), "parallelism": "replicas x%d (sources)" % ws},
        "roofline": roof,
        "phase_roofline": phase_roof,
        "peaks": dict(gemm, hbm_gbs=hbm, hbm_kind=peak_kind, fp32_simt_derived_tflops=simt, sms=nsm),
        "clocks": clk,
        "gpu_launches": r["gpu_launches"],
        "e2e": r.get("e2e"),
        "forms": {f: {k: v for k, v in results[f].items() if k not in ("info",)} for f in results},
    }
    if variants:
        line["variants"] = {k: {kk: vv for kk, vv in v.items() if kk not in ("info", "serving")}
                            for k, v in variants.items()}
        for v in variants.values():
            if v.get("serving"):
                line["serving"] = v["serving"]
    if "mixed" in results and "fp64" in results:
        line["mixed_over_fp64"] = results["mixed"]["rhs_per_s"] / results["fp64"]["rhs_per_s"]
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.config)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Benchmark: Liouville applications/s on the 64-atom diamond-like batch.

One step = one call of tddft_apply_liouville on the whole batch (8 trial
vectors, all occupied pairs, every term of L, FP32 pair/FFT path). Prints one
JSON line (rank 0). Under torchrun every rank runs an independent replica on
its own GPU (the operator needs no collective for independent batches).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Liouville applications/s (all occupied pairs) and % HBM roofline vs FP64 path"
UNIT = "applications/s"
WORKLOAD = dict(n=72, a=13.48, ecut=25.0, nocc=128, nb=8, alpha=0.18, seed=0)
WORKLOAD_NAME = ("diamond64: 64-atom diamond-like cubic cell a=13.48 bohr, 72^3 grid, Ecut 25 Ha "
                 "(14771 plane waves), Nocc 128, Nb 8 trial vectors, alpha 0.18, all occupied pairs")

# DRAM traffic per launch of the plane-kernel classes from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by a hash of the kernel sources
# it was taken on and the grid of the pair convolutions; reported as null when either
# differs. Captured launch: a 128 x 8 pair batch (1024 pair convolutions of 64^3) of the
# exchange term inside D; its algorithmic bytes (the library profiler's model) beside it.
NCU_TRAFFIC = {
    "08eb3ad5c147/64": {
        "launch": "128 x 8 pair batch of the exchange term inside D (1024 pair convolutions of 64^3)",
        "xy_fwd_pair_product": {"dram": 1.813e9, "algorithmic": 5.807e9},
        "z_kernel_multiply": {"dram": 2.968e9, "algorithmic": 3.024e9},
        "xy_inv_remultiply_accumulate": {"dram": 2.109e9, "algorithmic": 4.196e9},
    },
}


def kernel_source_hash() -> str:
    h = hashlib.sha1()
    for f in ("fft.cuh", "plane_kernels.cuh", "plane_lines.cuh", "plane_ops.cuh"):
        with open(os.path.join(ROOT, "paper_2309_03513_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6400.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(rank: int, npw: int):
    """The bench batch; npw is the sphere size, counted by the caller's own side
    (the library for the native arm, the oracle for the reference arm)."""
    from paper_2309_03513_b300 import synth
    w = WORKLOAD
    return synth.make_workload(n=w["n"], a=w["a"], ecut=w["ecut"], npw=npw, nocc_src=w["nocc"], nb=w["nb"],
                               seed=w["seed"] + rank, alpha=w["alpha"])


def oracle_sample(wl, rows):
    """Time the FP64 oracle on a few rows (b, v) of the batch; returns (seconds, threads)."""
    from oracle import tddft_oracle as O
    S = O.system_from_workload(wl)
    S.phi_src_r()  # orbitals to real space once, as the oracle's set-up
    t0 = time.perf_counter()
    S.apply(wl.X, rows=rows)
    return time.perf_counter() - t0, O.fft_workers()


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    """Largest value over the ranks (the slowest rank's time); CPU tensor under gloo."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, units_per_rank: float, local_seconds: float) -> tuple[float, float]:
    """Whole-job rate for independent replicas: units of all ranks / slowest rank's time.
    Returns (rate, max seconds)."""
    t = max_over_ranks(ws, local_seconds)
    return ws * units_per_rank / t, t


def bench_config(ws: int) -> dict:
    """The workload keys both arms print (identical, so the two lines describe the same job)."""
    w = WORKLOAD
    return {"workload": WORKLOAD_NAME, "n": w["n"], "npw": 14771, "nocc": w["nocc"], "nb": w["nb"],
            "parallelism": "replicas" if ws > 1 else "single process",
            "l2": "inputs larger than L2 (trial vectors and outputs in real space: 2 x 3.1 GB per step)"}


def run_reference(args):
    """The FP64 oracle on the host cores, one row (b, v) of the bench batch per step.
    The sphere is counted by the oracle itself: this arm never loads the CUDA library."""
    from oracle import tddft_oracle as O
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOAD
    wl = make_workload(0, O.miller_sphere(w["n"], w["a"], w["ecut"]).shape[0])
    nocc = w["nocc"]
    times = []
    cores = 1
    for i in range(args.warmup + args.steps):
        row = [(i % w["nb"], (7 * i) % nocc)]
        dt, cores = oracle_sample(wl, row)
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = (len(times) / nocc) / total  # rows -> applications
    cfg = bench_config(ws)
    cfg["npw"] = int(wl.phi_src.shape[1])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "step": "one row (b, v) of L.A, all pair convolutions of that row",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one row (b, v) of the batch per step: all pair convolutions of that row, "
                                   "with the Hartree/xc density of its trial vector; rows/s / Nocc"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def row_errors(got_rows, want_rows, x_rows) -> dict:
    """Errors of sampled rows (b, v) of L.A against the FP64 oracle: relative
    Frobenius error per row, and the error of those rows' contribution to
    omega_b = <X_b|L X_b> (sum over the sampled v of Re<x_v|(L x)_v>, Ha)."""
    got = np.asarray(got_rows, dtype=np.complex128)
    want = np.asarray(want_rows, dtype=np.complex128)
    x = np.asarray(x_rows, dtype=np.complex128)
    rel = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    om_got = float(np.sum(np.einsum("vg,vg->v", x.conj(), got).real))
    om_want = float(np.sum(np.einsum("vg,vg->v", x.conj(), want).real))
    return {"rows_rel_err": [float(e) for e in rel], "rows_rel_err_max": float(rel.max()),
            "omega_rows_Ha": om_want, "omega_rows_abs_err_Ha": abs(om_got - om_want)}


def run_native(args):
    import torch

    from paper_2309_03513_b300 import tddft as T

    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local if ws > 1 else 0)
    w = WORKLOAD
    wl = make_workload(rank, T.sphere_size(w["n"], w["a"], w["ecut"]))
    nb, nocc = w["nb"], w["nocc"]
    stream = torch.cuda.current_stream(dev)
    sys_ = T.system_from_workload(wl, precision=T.PREC_FP32, stream=stream)
    npw = sys_.npw
    # pair convolutions on the smallest grid on which they are exact (the same operator as on n^3)
    sys_.set_tuning(exchange_grid=args.exchange_grid, xy_kernel=args.xy_kernel, k1d_all=args.k1d_all)
    n_exchange = sys_.query()["n_exchange"]
    X = torch.from_numpy(wl.X).to(dev, torch.complex64)
    LA = torch.empty_like(X)

    for _ in range(args.warmup):
        sys_.apply(X, out=LA, stream=stream)
    torch.cuda.synchronize(dev)

    # timed region: the bare operator (no profiler events)
    sampler = ClockSampler(local if ws > 1 else 0)
    sampler.start()
    launches0 = T.launch_count()
    barrier(ws)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sys_.apply(X, out=LA, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    ms = e0.elapsed_time(e1)
    launches = T.launch_count() - launches0
    clocks = sampler.stop()
    value, sec_max = job_throughput(ws, args.steps * nb, ms / 1e3)
    ms_max = sec_max * 1e3
    nrows = max(1, args.cpu_rows)
    la_rows = LA[0, :nrows].cpu().numpy()
    x_rows = X[0, :nrows].cpu().numpy()

    # measured arithmetic peaks of this GPU (ALU / tensor-core roofline denominators)
    alu_peaks = {"fp32_fma_tflops": T.measure_peak(0)["tflops"], "tf32_tensor_tflops": T.measure_peak(1)["tflops"],
                 "how": "tddft_testing_peak: FMA chains on every SM; tcgen05.mma kind::tf32 128x256x8 back to back"}

    # per-class device time of the plane kernels: a separate pass with the library's
    # profiler (CUDA events around every plane-kernel launch, on the launching stream)
    prof_steps = max(1, min(args.steps, 3))
    T.profile_enable(True)
    for _ in range(prof_steps):
        sys_.apply(X, out=LA, stream=stream)
    torch.cuda.synchronize(dev)
    prof = T.profile_read()
    T.profile_enable(False)

    # end to end through the host-buffer entry point (pinned host memory, copies inside)
    Xh_t = torch.from_numpy(wl.X.astype(np.complex64)).pin_memory()
    LAh_t = torch.empty(Xh_t.shape, dtype=torch.complex64).pin_memory()
    Xh, LAh = Xh_t.numpy(), LAh_t.numpy()
    sys_.apply_host(Xh, LAh, stream=stream)
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        sys_.apply_host(Xh, LAh, stream=stream)
    t_e2e = max_over_ranks(ws, time.perf_counter() - t0)
    e2e = ws * args.e2e_steps * nb / t_e2e if args.e2e_steps > 0 else None
    io_bytes = nb * nocc * npw * 8

    # per-term split (one step each, same batch): K1d-only apps/s etc.
    term_ms, term_marginal_ms = {}, {}
    if args.term_split:
        for name, mask in (("D_exchange", T.TERM_D_EXX), ("K1d", T.TERM_K1D), ("K1e", T.TERM_K1E_H | T.TERM_K1E_XC),
                           ("diagonal_and_projector", T.TERM_D_KIN | T.TERM_D_VLOC | T.TERM_PROJ),
                           ("K2d (Z-vector operator only)", T.TERM_K2D),
                           ("K2e (Z-vector operator only)", T.TERM_K2E_H | T.TERM_K2E_XC)):
            sys_.set_terms(mask)
            sys_.apply(X, out=LA, stream=stream)
            t0e = torch.cuda.Event(enable_timing=True)
            t1e = torch.cuda.Event(enable_timing=True)
            t0e.record(stream)
            sys_.apply(X, out=LA, stream=stream)
            t1e.record(stream)
            torch.cuda.synchronize(dev)
            term_ms[name] = t0e.elapsed_time(t1e)
        # marginal cost in the full operator: L minus L without the term (shared field transforms
        # of the trial vectors and results are not charged to a term)
        def one_step(mask):
            sys_.set_terms(mask)
            sys_.apply(X, out=LA, stream=stream)
            t0e = torch.cuda.Event(enable_timing=True)
            t1e = torch.cuda.Event(enable_timing=True)
            t0e.record(stream)
            sys_.apply(X, out=LA, stream=stream)
            t1e.record(stream)
            torch.cuda.synchronize(dev)
            return t0e.elapsed_time(t1e)
        full_ms = one_step(T.TERMS_ALL)
        for name, mask in (("D_exchange", T.TERM_D_EXX), ("K1d", T.TERM_K1D), ("K1e", T.TERM_K1E_H | T.TERM_K1E_XC),
                           ("diagonal_and_projector", T.TERM_D_KIN | T.TERM_D_VLOC | T.TERM_PROJ)):
            term_marginal_ms[name] = full_ms - one_step(T.TERMS_ALL & ~mask)
        sys_.set_terms(T.TERMS_ALL)

    # the extras describe other workloads beside the metric: one GPU only (under torchrun every
    # rank would build them, holding all GPUs for minutes of host-side input generation)
    extras = {}
    if ws > 1:
        args.extra = ""
    if "uneven" in args.extra:
        extras["uneven12"] = bench_uneven(torch, T, dev, stream)
    if "sf216" in args.extra:
        extras["sf216"] = bench_sf216(torch, T, dev, stream)
    if "ace" in args.extra:
        extras["ace"] = bench_ace(torch, T, dev, stream, wl, X, LA)
    if "zvector" in args.extra:
        extras["zvector"] = bench_zvector(torch, T, dev, stream, wl, X)
    if "pairtrunc" in args.extra:
        extras["pairtrunc"] = bench_pairtrunc(torch, T, dev, stream)
    if "taucache" in args.extra:
        extras["taucache"] = bench_taucache(torch, T, dev, stream, wl, X, LA)
    if "combined" in args.extra:
        extras["combined"] = bench_combined(torch, T, dev, stream)

    # plain FP64 GPU path on the same batch
    fp64 = None
    la64_rows = None
    if args.fp64_steps > 0:
        del LA
        s64 = T.system_from_workload(wl, precision=T.PREC_FP64, stream=stream)
        X64 = torch.from_numpy(wl.X).to(dev)
        LA64 = torch.empty_like(X64)
        s64.apply(X64, out=LA64, stream=stream)
        torch.cuda.synchronize(dev)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            s64.apply(X64, out=LA64, stream=stream)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        fms = max_over_ranks(ws, f0.elapsed_time(f1))
        fp64 = {"value": ws * args.fp64_steps * nb / (fms / 1e3), "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": fms / args.fp64_steps}
        la64_rows = LA64[0, :nrows].cpu().numpy()
        s64.close()

    if rank != 0:
        return
    peaks = measured_peaks()
    cls = prof["classes"]
    dom = max(cls, key=lambda k: cls[k]["ms"])
    d = cls[dom]
    achieved = (d["bytes"] / d["launches"]) / (d["ms"] / d["launches"] / 1e3) / 1e9 if d["launches"] else None
    src_hash = kernel_source_hash()
    cap = NCU_TRAFFIC.get(f"{src_hash}/{n_exchange}", {})
    traffic = cap.get(dom, {}).get("dram")
    traffic_launch = ({"launch": cap["launch"], "algorithmic_bytes": cap[dom]["algorithmic"],
                       "dram_over_algorithmic": cap[dom]["dram"] / cap[dom]["algorithmic"]}
                      if traffic is not None else None)
    shares = {k: round(v["ms"] / max(1e-9, sum(c["ms"] for c in cls.values())), 4) for k, v in cls.items()}
    cfg = bench_config(ws)
    cfg["npw"] = npw
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": cfg,
        "schedule": {"exchange_grid": n_exchange, "xy_kernel": args.xy_kernel, "k1d_all": args.k1d_all,
                     "step": "one tddft_apply_liouville on the whole batch"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
                     "traffic": traffic, "traffic_launch": traffic_launch, "peak_source": peaks["source"],
                     "avg_launch_ms": d["ms"] / max(1, d["launches"]),
                     "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                     "class_time_share": shares, "kernel_sources": src_hash,
                     "timing": f"separate pass of {prof_steps} step(s) with per-launch CUDA events"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
        "gpu_launches": launches,
        "measured_alu_peaks": alu_peaks,
        "clocks": clocks,
        "terms_ms_per_step": term_ms or None,
        "terms_marginal_ms_per_step": term_marginal_ms or None,
        "k1d_only_apps_per_s": (nb / (term_ms["K1d"] / 1e3)) if term_ms else None,
        "extras": extras or None,
        "fp64_path": fp64,
        "speedup_vs_fp64_path": (value / fp64["value"]) if fp64 else None,
    }
    if ws == 1 and not args.no_cpu_baseline:
        from oracle import tddft_oracle as O
        rows = [(0, v) for v in range(nrows)]
        S = O.system_from_workload(wl)
        S.phi_src_r()  # orbitals to real space once, as the oracle's set-up
        t0 = time.perf_counter()
        want = S.apply(wl.X, rows=rows)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": (len(rows) / nocc) / dt, "unit": UNIT, "cores": O.fft_workers(),
                                "kind": "oracle",
                                "sample": f"{len(rows)} rows (b=0, v=0..{len(rows)-1}) of the same batch: all pair "
                                          f"convolutions of those rows plus the Hartree/xc density of b=0; "
                                          f"rows/s / Nocc; {dt:.1f} s"}
        errs = {"fp32_path": row_errors(la_rows, want, x_rows),
                "tolerance": {"rows_rel_err": 1e-5, "omega_abs_err_Ha": 1e-6}}
        if la64_rows is not None:
            errs["fp64_path"] = row_errors(la64_rows, want, wl.X[0, :nrows])
        line["errors_vs_oracle"] = errs
    print(json.dumps(line), flush=True)
    sys_.close()


def bench_uneven(torch, T, dev, stream, steps=2):
    """12 uneven systems (grids 48..96, 32..256 orbitals, 4..16 trial vectors, mixed
    spin-conserving / spin-flip) in one CUDA-graph launch with one branch per system;
    applications/s over all systems. Beside it the same systems applied one after the
    other on one stream, and the sum of their times alone: the graph's time against
    that sum shows how much the branches overlap (1.0 = none)."""
    from paper_2309_03513_b300 import synth
    systems, Xs = [], []
    total_nb = 0
    for i in range(1, 13):
        n = [48, 64, 80, 96][(i - 1) % 4]
        a = n * (13.48 / 72)
        nocc = 32 + round(224 * (i - 1) / 11)
        nbi = 4 * (1 + (i - 1) % 4)
        sf = (i % 2 == 0)
        wl = synth.make_workload(n=n, a=a, ecut=25.0, npw=T.sphere_size(n, a, 25.0), nocc_src=nocc, nb=nbi, seed=i,
                                 spin_flip=sf, nocc_tgt=nocc - 2 if sf else None)
        s = T.system_from_workload(wl, precision=T.PREC_FP32, stream=stream)
        systems.append(s)
        Xs.append(torch.from_numpy(wl.X).to(dev, torch.complex64))
        total_nb += nbi
    outs = [torch.empty_like(X) for X in Xs]
    T.apply_multi(systems, Xs, outs, stream=stream)  # capture + first run
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        T.apply_multi(systems, Xs, outs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    alone = []
    for s, X, o in zip(systems, Xs, outs):
        s.apply(X, out=o, stream=stream)
        e0.record(stream)
        s.apply(X, out=o, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        alone.append(e0.elapsed_time(e1))
    for s in systems:
        s.close()
    return {"value": total_nb / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "trial_vectors": total_nb,
            "steps": steps, "systems": 12, "sum_of_systems_alone_ms": sum(alone),
            "graph_over_sum_alone": ms / sum(alone), "systems_alone_ms": alone,
            "note": "one CUDA-graph launch per step, one branch per system"}


def bench_ace(torch, T, dev, stream, wl, X, LA, steps=3):
    """The same batch with the exchange inside D through the compressed operator
    built on N_ACE = 4 N_occ vectors (the occupied orbitals plus 3 N_occ random
    orthonormal rows orthogonal to them, standing in for unoccupied orbitals).
    An approximation of L: its relative deviation from the exact operator on this
    batch is reported beside the rate."""
    from paper_2309_03513_b300 import synth
    s = T.system_from_workload(wl, precision=T.PREC_FP32, stream=stream)
    s.apply(X, out=LA, stream=stream)
    exact = LA.clone()
    nocc = wl.phi_tgt.shape[0]
    extra = synth.complement_rows(np.random.default_rng(1234), wl.phi_tgt, 3 * nocc)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s.ace_build(extra, stream=stream)
    build_s = time.perf_counter() - t0
    s.apply(X, out=LA, stream=stream)
    torch.cuda.synchronize(dev)
    dev_rel = float(torch.linalg.vector_norm(LA - exact) / torch.linalg.vector_norm(exact))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        s.apply(X, out=LA, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    s.set_terms(T.TERM_D_EXX)
    s.apply(X, out=LA, stream=stream)
    e0.record(stream)
    s.apply(X, out=LA, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    d_ms = e0.elapsed_time(e1)
    s.close()
    nb = X.shape[0]
    return {"value": nb / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "n_ace": 4 * nocc,
            "build_s": build_s, "D_exchange_ms": d_ms, "rel_deviation_from_exact_L": dev_rel,
            "note": "approximate operator (compressed exchange inside D); not the bench metric"}


def bench_zvector(torch, T, dev, stream, wl, X, max_iter=40):
    """Z-vector equation (Eq. 19) for the bench batch's states: right-hand sides
    from the adjoint, then preconditioned CG with the inexact Krylov switch at
    lambda_thr = 1e-4 (Sec. 3.3) to a residual norm of 1e-6, FP32 operator.
    Reports the time of one exact and one approximate operator application."""
    s = T.system_from_workload(wl, precision=T.PREC_FP32, stream=stream)
    nb = X.shape[0]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    U = s.zvector_rhs(X, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    rhs_ms = e0.elapsed_time(e1)
    Y = torch.empty_like(X)
    op_ms = {}
    for name, mask in (("exact", T.TERMS_ZVEC), ("approx_no_K2d", T.TERMS_ZVEC & ~T.TERM_K2D)):
        s.set_terms(mask)
        s.apply(U, out=Y, stream=stream)
        e0.record(stream)
        s.apply(U, out=Y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        op_ms[name] = e0.elapsed_time(e1)
    s.set_terms(T.TERMS_ALL)
    t0 = time.perf_counter()
    Z, it, ex, res = s.zvector_solve(U, lambda_thr=1e-4, tol=1e-6, max_iter=max_iter, precondition=True,
                                     stream=stream, require_convergence=False)
    torch.cuda.synchronize(dev)
    solve_s = time.perf_counter() - t0
    s.close()
    return {"states": nb, "rhs_ms": rhs_ms, "operator_ms_per_batch": op_ms, "solve_s": solve_s,
            "iterations": it.tolist(), "exact_iterations": ex.tolist(), "residual": res.tolist(),
            "lambda_thr": 1e-4, "tol": 1e-6, "max_iter": max_iter,
            "note": "preconditioned CG; per state the exact operator while ||r|| >= lambda_thr"}


def bench_pairtrunc(torch, T, dev, stream, s_thr=1e-3):
    """K1d with pair truncation over localised orbitals (Sec. 3.2): the diamond64
    grid and batch with 128 localised orbitals (Gaussians of width 1 bohr,
    Loewdin-orthonormalised, rotated by a random unitary), FP32. The localised
    frame is the one tddft_localize finds from the mixed orbitals. K1d time per
    batch exact (given frame) and truncated at S_thr = 1e-3, computed over the
    pair list of kept pairs and over 16 x 16 blocks with the dropped pairs
    masked, the whole operator, and the deviation of the truncated L from the
    exact one on this batch."""
    from paper_2309_03513_b300 import synth
    w = WORKLOAD
    n, a, ecut = w["n"], w["a"], w["ecut"]
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=w["nocc"], nb=w["nb"],
                             seed=11, localized_sigma=1.0, miller=T.sphere_miller(n, a, ecut))
    s = T.system_from_workload(wl, precision=T.PREC_FP32, stream=stream)
    X = torch.from_numpy(wl.X).to(dev, torch.complex64)
    LA = torch.empty_like(X)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # the localised frame found by the library from the mixed orbitals (host, tddft_localize)
    t0 = time.perf_counter()
    U, spreads, sweeps = T.localize(n, a, ecut, wl.phi_src)
    loc_s = time.perf_counter() - t0

    def timed(mask):
        s.set_terms(mask)
        s.apply(X, out=LA, stream=stream)
        e0.record(stream)
        s.apply(X, out=LA, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    out = {"s_thr": s_thr, "nocc": w["nocc"], "sigma_bohr": 1.0,
           "localization": {"seconds": loc_s, "sweeps": sweeps, "spread_bohr2": list(spreads),
                            "frame": "tddft_localize from the mixed orbitals (host)"}}
    out["k1d_ms_exact"] = timed(T.TERM_K1D)
    out["L_ms_exact"] = timed(T.TERMS_ALL)
    exact = LA.clone()
    S, kept = s.set_localization(U, s_thr, stream=stream)
    out["kept_pairs"] = kept
    out["kept_fraction"] = kept / float(w["nocc"] ** 2)
    s.set_tuning(k1d_sparse=0, k1d_block=16)
    out["k1d_ms_truncated_blocks16"] = timed(T.TERM_K1D)
    s.set_tuning(k1d_sparse=1)
    out["k1d_ms_truncated_pair_list"] = timed(T.TERM_K1D)
    out["k1d_speedup_pair_list"] = out["k1d_ms_exact"] / out["k1d_ms_truncated_pair_list"]
    out["L_ms_truncated"] = timed(T.TERMS_ALL)
    out["rel_deviation_from_exact_L"] = float(torch.linalg.vector_norm(LA - exact) / torch.linalg.vector_norm(exact))
    s.close()
    return out


def bench_combined(torch, T, dev, stream, s_thr=1e-3, lambda_thr=1e-4, tol=1e-6, max_iter=40):
    """The approximations of Sec. 3 together, as the paper combines them: the compressed
    exchange inside D (N_ACE = 4 N_occ: the occupied orbitals plus 3 N_occ random orthonormal
    rows orthogonal to them), K1d truncated at S_thr = 1e-3 in the frame tddft_localize finds,
    and the inexact-Krylov switch at lambda_thr = 1e-4 in the Z-vector CG; against the exact
    operator and an exact-operator CG on the same batch (the pair-truncation workload: 128
    localised orbitals mixed by a random unitary, 8 trial vectors), FP32. Reports one operator
    application and one Z-vector solve each way, and the deviations of the approximate L X and
    Z from the exact ones."""
    from paper_2309_03513_b300 import synth
    w = WORKLOAD
    n, a, ecut = w["n"], w["a"], w["ecut"]
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=w["nocc"], nb=w["nb"],
                             seed=11, localized_sigma=1.0, miller=T.sphere_miller(n, a, ecut))
    s = T.system_from_workload(wl, precision=T.PREC_FP32, stream=stream)
    X = torch.from_numpy(wl.X).to(dev, torch.complex64)
    LA = torch.empty_like(X)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed_apply():
        s.apply(X, out=LA, stream=stream)
        e0.record(stream)
        s.apply(X, out=LA, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    def solve(lam):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Z, it, ex, res = s.zvector_solve(U, lambda_thr=lam, tol=tol, max_iter=max_iter, precondition=True,
                                         stream=stream, require_convergence=False)
        torch.cuda.synchronize(dev)
        return Z, time.perf_counter() - t0, it, ex, res

    out = {"s_thr": s_thr, "lambda_thr": lambda_thr, "n_ace": 4 * w["nocc"], "tol": tol, "max_iter": max_iter}
    out["L_ms_exact"] = timed_apply()
    L_exact = LA.clone()
    U = s.zvector_rhs(X, stream=stream)  # right-hand sides from the exact operator's adjoint
    Z_exact, t_exact, it_e, _, res_e = solve(0.0)
    out["zvector_exact"] = {"solve_s": t_exact, "iterations": it_e.tolist(), "residual": res_e.tolist()}
    # the approximations on
    extra = synth.complement_rows(np.random.default_rng(1234), wl.phi_tgt, 3 * w["nocc"])
    t0 = time.perf_counter()
    s.ace_build(extra, stream=stream)
    Uloc, spreads, _ = T.localize(n, a, ecut, wl.phi_src)
    _, kept = s.set_localization(Uloc, s_thr, stream=stream)
    s.set_tuning(k1d_sparse=1)
    torch.cuda.synchronize(dev)
    out["setup_s"] = time.perf_counter() - t0
    out["kept_fraction"] = kept / float(w["nocc"] ** 2)
    out["L_ms_approx"] = timed_apply()
    out["L_rel_deviation"] = float(torch.linalg.vector_norm(LA - L_exact) / torch.linalg.vector_norm(L_exact))
    Z_apx, t_apx, it_a, ex_a, res_a = solve(lambda_thr)
    out["zvector_approx"] = {"solve_s": t_apx, "iterations": it_a.tolist(), "exact_iterations": ex_a.tolist(),
                             "residual": res_a.tolist()}
    out["Z_rel_deviation"] = float(torch.linalg.vector_norm(Z_apx - Z_exact) / torch.linalg.vector_norm(Z_exact))
    out["speedup_L"] = out["L_ms_exact"] / out["L_ms_approx"]
    out["speedup_zvector_solve"] = t_exact / t_apx
    out["note"] = "approximate operator (Sec. 3 combined); not the bench metric"
    s.close()
    return out


def bench_taucache(torch, T, dev, stream, wl, X, LA, steps=5):
    """The bench batch with K1d read from the stored tau_vv' of every occupied pair
    (tuning.k1d_cache: built once from the occupied orbitals, then only the
    contraction per application). Exact up to rounding, but a different mode from
    the bench metric, which recomputes every pair convolution: reported beside it."""
    s = T.system_from_workload(wl, precision=T.PREC_FP32, stream=stream)
    s.apply(X, out=LA, stream=stream)
    torch.cuda.synchronize(dev)
    exact = LA.clone()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(mask, n):
        s.set_terms(mask)
        s.apply(X, out=LA, stream=stream)
        e0.record(stream)
        for _ in range(n):
            s.apply(X, out=LA, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    out = {"k1d_ms_recomputed": timed(T.TERM_K1D, 1)}
    before = s.query()["device_bytes"]
    t0 = time.perf_counter()
    s.set_tuning(k1d_cache=1)
    out["build_s"] = time.perf_counter() - t0
    out["stored_GB"] = (s.query()["device_bytes"] - before) / 1e9
    out["k1d_ms_stored"] = timed(T.TERM_K1D, 1)
    ms = timed(T.TERMS_ALL, steps)
    out["rel_deviation_from_recomputed_L"] = float(torch.linalg.vector_norm(LA - exact) /
                                                   torch.linalg.vector_norm(exact))
    s.close()
    nb = X.shape[0]
    out.update({"value": nb / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
                "note": "K1d from stored tau (built once per ground state); not the bench metric"})
    return out


def bench_sf216(torch, T, dev, stream, steps=1):
    """216-atom spin-flip cell (108^3, 433/431 orbitals, 16 trial vectors), FP32 path, pair
    convolutions on the 96^3 exchange grid; one warm-up, then `steps` timed applications. Row
    (b = 0, v = 0) is compared with the oracle's digest of that row in tests/golden (written by
    tests/golden/make_sf216_row_digest.py from the oracle alone)."""
    from paper_2309_03513_b300 import synth
    n, a = 108, 20.2
    wl = synth.make_workload(n=n, a=a, ecut=25.0, npw=T.sphere_size(n, a, 25.0), nocc_src=433, nb=16, seed=0,
                             spin_flip=True, nocc_tgt=431)
    s = T.system_from_workload(wl, precision=T.PREC_FP32, stream=stream)
    n_exchange = s.query()["n_exchange"]
    X = torch.from_numpy(wl.X).to(dev, torch.complex64)
    LA = torch.empty_like(X)
    s.apply(X, out=LA, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        s.apply(X, out=LA, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    out = {"value": 16 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": 1,
           "exchange_grid": n_exchange, "pairs_per_step": 16 * 433 * 431 + 433 * 434 // 2}
    # 48 B per point per pair convolution on the exchange grid (the HBM model of the pair stage)
    model_s = out["pairs_per_step"] * n_exchange ** 3 * 48.0 / (measured_peaks()["hbm_gbs"] * 1e9)
    out["model_48B_per_point_s"] = model_s
    out["fraction_of_model_rate"] = model_s / (ms / 1e3)
    gold = os.path.join(ROOT, "tests", "golden", "sf216_row_digest.json")
    if os.path.exists(gold):
        with open(gold) as fh:
            g = json.load(fh)
        b, v = g["row"]
        row = LA[b, v].cpu().numpy().astype(np.complex128)
        x = wl.X[b, v]
        idx = np.array([t[0] for t in g["samples"]])
        want = np.array([complex(t[1], t[2]) for t in g["samples"]])
        out["errors_vs_oracle_row"] = {
            "row": [b, v],
            "sampled_coefficients_rel_err": float(np.linalg.norm(row[idx] - want) / np.linalg.norm(want)),
            "norm_rel_err": float(abs(np.linalg.norm(row) - g["norm"]) / g["norm"]),
            "omega_row_abs_err_Ha": float(abs(np.vdot(x, row).real - g["omega_row"])),
        }
    s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-rows", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--term-split", type=int, default=1, help="time each term alone (one step each)")
    ap.add_argument("--extra", default="sf216,uneven", help="comma list: uneven (12-system graph), sf216 (216-atom spin-flip), "
                                             "ace (compressed exchange on the bench batch), zvector (Z-vector CG on the bench batch), "
                                             "pairtrunc (K1d pair truncation, localised orbitals), "
                                             "taucache (K1d from stored tau of every pair), "
                                             "combined (the approximations of Sec. 3 together against the exact operator)")
    ap.add_argument("--exchange-grid", type=int, default=1, choices=[0, 1],
                    help="1: pair convolutions on the smallest exact grid (64^3 here; the default); 0: on the 72^3 grid")
    ap.add_argument("--xy-kernel", type=int, default=1, choices=[0, 1, 2, 3],
                    help="register-line xy passes where they exist: 1 one thread per line (the default), 2 two "
                         "lanes per line, 3 forward one thread, inverse two lanes; 0: shared-memory radix stages")
    ap.add_argument("--k1d-all", type=int, default=1, choices=[0, 1],
                    help="1: K1d over the tau of every pair in one pass (the default); 0: by 16 x 16 blocks")
    ap.add_argument("--nb", type=int, default=WORKLOAD["nb"],
                    help="trial vectors per batch (smaller cases for profiler captures; the bench line uses 8)")
    args = ap.parse_args()
    WORKLOAD["nb"] = args.nb
    if args.warmup < 3 and args.impl == "native":
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the SPME stochastic-Lanczos MBD hot path on GB300.

One step = one mbd_energy_forces call on the 100,002-atom water-like box
(33,334 molecules, L = 188.8 bohr, mesh 192^3, spline order 6, Ewald beta 0.30
bohr^-1, r_cut 12 bohr, 64 probes x 60 Lanczos steps): probe generation, the
Lanczos recurrence with the SPME operator (spread, FFT convolution, gather +
real space + self), the tridiagonal quadrature and the force estimator.  The
operator runs in FP32 and the Lanczos layer in FP64 (the mixed path); the
plain FP64 path is timed beside it.  The 3000- and 24,000-atom boxes are timed
too and reported under "other_workloads".

Metric: probe-matvecs/s = R m / step time (whole job over all ranks).  The
timed region carries CUDA events around each step only; the per-stage table
and the roofline come from the same steps run again with the library's
per-stage events (which add a little time per step).
Probes shard across ranks (rank r uses probes r R .. r R + R - 1); the energy
and forces are averaged over ranks with one all-reduce per step.

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded
sample of the same workload and prints the same JSON line with impl=reference.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "probe-matvecs/s and ms per MBD energy+forces at 1 GB300; frac of HBM roofline"
UNIT = "probe-matvecs/s"
WORKLOADS = {"water3000": 2, "water24000": 3, "water100002": 5}
DEFAULT_WORKLOAD = "water100002"
OTHER_WORKLOADS = ("water3000", "water24000")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--quadrature", default="chebyshev", choices=["chebyshev", "ql", "ql_df64"],
                    help="evaluation of the per-probe Gauss quadrature (Chebyshev expansion with QL fallback, "
                         "or the QL eigendecomposition in FP64 or double-float)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(WORKLOADS) + ["batch64"],
                    help="water100002 (default, the bench line): 100002 atoms, mesh 192^3, 64 x 60; "
                         "water24000: 24000 atoms, mesh 128^3, 128 x 60; water3000: 3000-atom water box, mesh "
                         "64^3, 64 x 50; batch64: the 64 uneven random boxes (200-20000 atoms, 32 probes x 40 "
                         "steps) run as one graph-replayed batch (energies)")
    ap.add_argument("--energy-only", action="store_true",
                    help="time mbd_lanczos_energy instead of mbd_energy_forces (small cases for ncu captures)")
    ap.add_argument("--lanczos-steps", type=int, default=0,
                    help="Lanczos steps m per call instead of the workload's (0: the workload's; small cases "
                         "for ncu captures)")
    ap.add_argument("--other-steps", type=int, default=5,
                    help="timed steps of each other water box and of the 64-box batch reported beside the bench "
                         "line (0: none)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip mbd_autotune (launch choices by the built-in rules)")
    ap.add_argument("--choices", default="",
                    help="apply these launch choices (ld,field_atoms_per_block,fft_tile,spread_tile, as the JSON "
                         "line's config.autotune reports them) instead of timing them: profiles taken under ncu "
                         "then run the configuration of a live run")
    ap.add_argument("--no-cufft", action="store_true",
                    help="skip the comparison of the FFT convolution (forward 3D FFT, x G, inverse) with cuFFT "
                         "(torch.fft) on the same complex mesh")
    ap.add_argument("--study", default="", choices=["", "delta11"],
                    help="delta11: Delta_11 against the mesh for the 14.2 angstrom water and diamond boxes, "
                         "and the parameters mbd_spme_params chooses (JSON lines)")
    ap.add_argument("--scs-steps", type=int, default=3,
                    help="timed calls of the screening front end (mbd_scs_screen) on the workload and on the "
                         "3000-atom box, with the oracle's screening of the 3000-atom box timed beside it (0: none)")
    ap.add_argument("--cpu-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-child-scs", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


SINGLE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                     "NUMEXPR_NUM_THREADS": "1"}


# ---------------------------------------------------------------------------- helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(index)], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.strip().split(",") for ln in self.file.read().splitlines() if ln.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for name, val in zip(names, r[5:9]):
                    if val.strip().lower() in ("active", "1"):
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash(files=None) -> str:
    """Hash of the kernel sources (all of csrc, or the listed glob patterns)."""
    import glob
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2307_02278_gb300", "csrc")
    names = sorted(os.listdir(csrc)) if files is None else sorted(
        {os.path.basename(f) for pat in files for f in glob.glob(os.path.join(csrc, pat))})
    for fn in names:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


# the sources each roofline stage's kernels are built from (a change to any
# invalidates its recorded DRAM traffic)
L2_BYTES = 129 * 1000 * 1000     # GB300 L2 (about 129 MB)
STAGE_SOURCES = {"fft": ["fft.cuh", "fft_sizes_*.cu", "kernels_mesh.cu", "mbd_internal.cuh"]}


def dram_traffic(stage: str, workload: str):
    """Bytes per launch from a committed ncu summary, if it was taken on the
    current sources of the stage's kernels (profiles/dram_traffic.txt: stage
    workload bytes hash)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = source_hash(STAGE_SOURCES.get(stage))
    with open(path) as f:
        for ln in f:
            p = ln.split()
            if len(p) == 4 and not ln.startswith("#") and p[0] == stage and p[1] == workload and p[3] == cur:
                return float(p[2])
    return None


def stage_bytes(n_atoms, mesh, R, m, s_bytes, n_pairs, p=6, real_clusters=False):
    """Algorithmic HBM bytes per launch of each stage (minimum traffic of the
    stage's inputs and outputs; every array read or written once).  With the
    real-space clusters the pairs are read by the "real" stage, which writes
    E_real for the field kernel to read."""
    npts = mesh[0] * mesh[1] * mesh[2]
    rows = 3 * n_atoms
    R2 = 2 * R
    pairs = n_pairs * (6 * s_bytes + 4)
    return {
        "prologue": rows * R * (4 * 8 + s_bytes),                     # read l, y_{k-1}, y_{k-2}; write y*, d
        "spread": npts * R * s_bytes + rows * R * s_bytes + n_atoms * 3 * p * 2 * s_bytes,
        "fft": 2 * npts * R * s_bytes,                                 # one pass: read + write the mesh
        "real": 2 * rows * R * s_bytes + pairs,                        # d and the pair tensors in, E_real out
        "field": (npts * R * s_bytes + rows * R * s_bytes + (rows * R * s_bytes if real_clusters else pairs)
                  + rows * R * 8 * 3),                                 # mesh, d, E_real or pairs, y* in / y, l out
        "force_spread": npts * R2 * s_bytes + rows * R2 * s_bytes,
        "force_fft": 2 * npts * R2 * s_bytes,
        "force_gather": npts * R2 * s_bytes + rows * R2 * s_bytes + n_pairs * 8,
    }


# ---------------------------------------------------------------------------- reference arm
def oracle_cv_sample(s, n_min: int, seconds: float):
    """The oracle as it stands on a bounded sample of the workload: products
    C v of one probe vector with the oracle's SPME operator (the Lanczos step's
    dominant work), n_min of them at least and more while `seconds` last.
    Returns (seconds per product, products timed, operator setup seconds)."""
    import numpy as np

    from oracle.operator import Operator

    t0 = time.perf_counter()
    op = Operator(s, "spme")
    setup = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    t = []
    t_end = time.perf_counter() + seconds
    while len(t) < n_min or time.perf_counter() < t_end:
        x = rng.normal(size=(1, 3 * s.n_atoms))
        t0 = time.perf_counter()
        op(x)
        t.append(time.perf_counter() - t0)
    return float(np.mean(t)), len(t), setup


def _oracle_sample_text(s, n, setup):
    return (f"{n} products C v of one probe with the oracle's SPME operator on {s.name} (FP64 NumPy, 1 thread; "
            f"operator setup {setup:.1f} s untimed); probe-matvecs/s extrapolated as 1 / (seconds per product): "
            f"the Lanczos vector updates, the quadrature and the force estimator are not in the sample")


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    from workloads.systems import config

    s = config(WORKLOADS[args.workload])
    per_warm, _, setup = oracle_cv_sample(s, max(1, args.warmup), 0.0)
    per, n, _ = oracle_cv_sample(s, args.steps, 0.0)
    value = 1.0 / per
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": s.name, "n_atoms": s.n_atoms, "mesh": list(s.mesh), "spline_order": s.spline_order,
                   "ewald_beta": s.ewald_beta, "r_cut": s.r_cut, "step": "one oracle product C v (one probe)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": _oracle_sample_text(s, n, setup), "ms_per_cv": per * 1e3},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_child(seconds: float, workload: str):
    """The oracle's bounded sample, run in a child process started with
    single-thread BLAS/OpenMP settings."""
    from workloads.systems import config

    s = config(WORKLOADS[workload])
    per, n, setup = oracle_cv_sample(s, 1, seconds)
    print(json.dumps({"value": 1.0 / per, "unit": UNIT, "cores": 1, "kind": "oracle",
                      "sample": _oracle_sample_text(s, n, setup), "ms_per_cv": per * 1e3}))


def cpu_baseline(seconds: float, workload: str):
    env = dict(os.environ, **SINGLE_THREAD_ENV)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", "--cpu-seconds", str(seconds),
                        "--workload", workload], capture_output=True, text=True, env=env, cwd=ROOT)
    try:
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return {"error": (r.stderr or r.stdout)[-300:]}


SCS_FREQ = 23
SCS_TOL = 1e-10


def cpu_scs_child():
    """The oracle's screening (sparse conjugate gradient, one thread) of the
    3000-atom box, timed; prints its per-atom results' summary."""
    import numpy as np

    from oracle import scs as oscs
    from workloads.systems import config

    s = config(2)
    t0 = time.perf_counter()
    out = oscs.scs(s, n_freq=SCS_FREQ, solver="cg")
    dt = time.perf_counter() - t0
    print(json.dumps({"seconds": dt, "cores": 1, "workload": s.name, "alpha": out["alpha"].tolist(),
                      "omega": out["omega"].tolist()}))


def scs_measurement(mbd, s, args, stream, flush):
    """Device time of mbd_scs_screen (mixed) on the workload and on the
    3000-atom box (CUDA events, L2 flushed before each call), the FP64 path on
    the 3000-atom box, and the oracle's screening of that box on one core."""
    import numpy as np
    import torch

    from workloads.systems import config

    def timed(sys_, steps):
        sys_.scs_screen(n_freq=SCS_FREQ, tol=SCS_TOL)
        ms = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = sys_.scs_screen(n_freq=SCS_FREQ, tol=SCS_TOL)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.mean(ms)), r

    out = {"n_freq": SCS_FREQ, "tol": SCS_TOL,
           "includes": "pair records, T_SR evaluated in each product (FP32), CG to tol on every column, "
                       "C6/omega/R_vdw, host copies"}
    g = mbd.MBDSystem.from_workload(s, precision="mixed", stream=stream)
    ms, r = timed(g, args.scs_steps)
    out["workload"] = {"name": s.name, "ms_per_call": ms, "iterations": r["iterations"], "residual": r["residual"],
                       "n_pairs": g.info()["n_pairs"], "mean_alpha_scs_over_alpha": float(np.mean(r["alpha"] / s.alpha))}
    g.close()
    s2 = config(2)
    g = mbd.MBDSystem.from_workload(s2, precision="mixed", stream=stream)
    ms2, r2 = timed(g, args.scs_steps)
    g.close()
    g = mbd.MBDSystem.from_workload(s2, precision="fp64", stream=stream)
    ms64, r64 = timed(g, 1)
    g.close()
    out["water3000"] = {"ms_per_call": ms2, "iterations": r2["iterations"], "fp64_ms_per_call": ms64,
                        "mixed_vs_fp64_max_rel": float(max(np.max(np.abs(r2[k] - r64[k]) / np.abs(r64[k]))
                                                           for k in ("alpha", "omega", "r_vdw", "c6")))}
    if not args.no_cpu_baseline:
        env = dict(os.environ, **SINGLE_THREAD_ENV)
        p = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child-scs"], capture_output=True,
                           text=True, env=env, cwd=ROOT)
        try:
            o = json.loads(p.stdout.strip().splitlines()[-1])
            worst = max(float(np.max(np.abs(r2[k] - np.asarray(o[k])) / np.abs(np.asarray(o[k]))))
                        for k in ("alpha", "omega"))
            out["water3000"]["oracle"] = {"seconds": o["seconds"], "cores": 1, "kind": "oracle",
                                          "sample": "the oracle's screening of the 3000-atom box (scipy sparse CG "
                                                    "per column, FP64), the same n_freq",
                                          "gpu_speedup": o["seconds"] / (ms2 * 1e-3),
                                          "gpu_mixed_vs_oracle_max_rel": worst}
        except Exception:
            out["water3000"]["oracle"] = {"error": (p.stderr or p.stdout)[-300:]}
    return out


# ---------------------------------------------------------------------------- our arm
def cufft_comparison(mbd, s, precision, R, stream, reps=10):
    """Device time of the FFT convolution of R probes on the workload's mesh:
    the library's passes (mbd_convolve, stage profiler) against torch.fft
    (cuFFT): forward 3D FFT, product with a real G, inverse, on the same complex
    layout (two probes per complex value)."""
    import numpy as np
    import torch
    K = tuple(s.mesh)
    V = (R + 1) // 2
    g = mbd.MBDSystem.from_workload(s, precision=precision, stream=stream)
    q = torch.randn((R,) + K, dtype=torch.float64, device="cuda")
    g.convolve(q)
    g.profile_enable(True)
    for _ in range(reps):
        g.convolve(q)
    prof = g.profile_read()
    g.close()
    del q
    ours_ms = prof["fft"][1] / reps
    cdt = torch.complex64 if precision == "mixed" else torch.complex128
    x = torch.randn(K + (V,), dtype=cdt, device="cuda")
    G = torch.rand(K + (1,), dtype=torch.float32 if precision == "mixed" else torch.float64, device="cuda")
    ts = []
    with torch.cuda.stream(stream):
        for k in range(reps + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            y = torch.fft.ifftn(torch.fft.fftn(x, dim=(0, 1, 2)) * G, dim=(0, 1, 2))
            b.record(stream)
            torch.cuda.synchronize()
            if k >= 2:
                ts.append(a.elapsed_time(b))
    del x, y, G
    torch.cuda.empty_cache()
    return {"mesh": list(K), "probes": R, "ours_ms": ours_ms, "cufft_ms": float(np.median(ts)),
            "note": "ours: 5 passes (k3, k2, k1 fused with G and its inverse, k2, k3); cuFFT: fftn, x G, ifftn"}


def roofline(stages, dom, peak, peak_kind, workload, n_prof, npts_bytes):
    """Roofline line of the dominant stage: achieved = algorithmic bytes per
    launch / device time per launch against the measured HBM copy bandwidth,
    and, when an ncu capture of the current sources gives the stage's DRAM
    traffic per launch, the same fraction on those measured bytes."""
    d = stages[dom]
    ach = d["achieved_gbs"]
    traffic = dram_traffic(dom, workload)
    out = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "basis": "algorithmic bytes (the stage's inputs and outputs read or written once)",
           "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth)",
           "duration_source": f"library per-stage CUDA events on its stream over {n_prof} live steps "
                              "run right after the timed region",
           "mesh_bytes": npts_bytes, "mesh_exceeds_l2": npts_bytes > L2_BYTES, "traffic": traffic}
    if traffic is not None:
        dram_gbs = traffic / (d["us_per_launch"] * 1e-6) / 1e9
        out["frac_dram"] = dram_gbs / peak
        out["achieved_dram_gbs"] = dram_gbs
    return out


def other_workload(mbd, s, args, stream, flush):
    """A shorter measurement of another water box beside the bench line: the
    same energy + forces step (autotuned, L2 flushed before each step), its
    device time per step and, from a second pass with the per-stage events,
    the microseconds per launch of each stage and the FFT pass's fraction of
    the HBM copy bandwidth."""
    import numpy as np
    import torch

    R, m = s.n_probes, s.n_steps
    g = mbd.MBDSystem.from_workload(s, precision=args.precision, quadrature=args.quadrature, stream=stream)
    tuning = None if args.no_autotune else g.autotune(R)
    forces = torch.empty((s.n_atoms, 3), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        g.energy_forces(R, m, s.probe_seed, forces=forces)
    ms = []
    for _ in range(args.other_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.energy_forces(R, m, s.probe_seed, forces=forces)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    g.profile_enable(timing=True)
    for _ in range(2):
        with torch.cuda.stream(stream):
            flush.zero_()
        g.energy_forces(R, m, s.probe_seed, forces=forces)
    prof = g.profile_read()
    info = g.info()
    g.close()
    t = float(np.mean(ms))
    s_bytes = 4 if args.precision == "mixed" else 8
    sb = stage_bytes(s.n_atoms, s.mesh, R, m, s_bytes, info["n_pairs"], s.spline_order,
                     real_clusters=prof["real"][0] > 0)
    us = {k: prof[k][1] * 1e3 / prof[k][0] for k in ("prologue", "spread", "fft", "real", "field")
          if prof[k][0] > 0}
    peak, _ = measured_peaks()
    return {"workload": s.name, "n_atoms": s.n_atoms, "mesh": list(s.mesh), "n_probes": R, "n_steps": m,
            "steps": args.other_steps, "ms_per_energy_forces": t, "value": R * m / (t * 1e-3), "unit": UNIT,
            "ns_per_atom_probe_step": t * 1e6 / (s.n_atoms * R * m), "us_per_launch": us,
            "fft_frac_of_hbm": sb["fft"] / (us["fft"] * 1e-6) / 1e9 / peak if "fft" in us else None,
            "n_pairs": info["n_pairs"], "autotune": tuning}


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as mbd
    from workloads.systems import config

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2307_02278_gb300.parallel import reduce_estimates, shard_seed
    s = config(WORKLOADS[args.workload])
    R, m = s.n_probes, (args.lanczos_steps if args.lanczos_steps > 0 else s.n_steps)
    seed = shard_seed(s.probe_seed, rank, R)
    stream = torch.cuda.Stream()
    sysm = mbd.MBDSystem.from_workload(s, precision=args.precision, quadrature=args.quadrature, stream=stream)
    if args.choices:
        vals = [int(v) for v in args.choices.split(",")]
        tuning = dict(zip(("ld", "field_atoms_per_block", "fft_tile", "spread_tile"), vals))
        sysm.set_launch_choices(tuning)
    else:
        tuning = None if args.no_autotune else sysm.autotune(R)
    info = sysm.info()
    forces = torch.empty((s.n_atoms, 3), dtype=torch.float64, device="cuda")
    energy_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(system, seed_k):
        if args.energy_only:
            return system.lanczos_energy(R, m, seed_k)
        e, _ = system.energy_forces(R, m, seed_k, forces=forces)
        if world > 1:
            with torch.cuda.stream(stream):
                energy_t.fill_(e)
                reduce_estimates(energy_t, forces)
        return e

    for _ in range(args.warmup):
        step(sysm, seed)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each step, CUDA events on the
    # system stream around each step (no per-stage events inside)
    visible = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    sampler = ClockSampler(visible[local] if local < len(visible) else local)
    time.sleep(0.3)
    sysm.profile_enable(timing=False)           # resets the launch counters
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    energies = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
        energies.append(step(sysm, seed))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches_timed = int(sysm.profile_read()["total_launches"])
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(step_ms) / 1e3
    t_max = t_dev
    if world > 1:
        tt = torch.tensor([t_dev], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    ms_per_step = t_max / args.steps * 1e3
    value = world * R * m * args.steps / t_max

    # ---- the same steps again with the library's per-stage CUDA events (stage
    # table and roofline); these events add a little time to each step
    n_prof = min(args.steps, 20)
    sysm.profile_enable(timing=True)
    t_prof = 0.0
    for k in range(n_prof):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(sysm, seed)
        b.record(stream)
        torch.cuda.synchronize()
        t_prof += a.elapsed_time(b)
    prof = sysm.profile_read()
    sysm.profile_enable(timing=False)
    prof_ms = t_prof / n_prof

    out = None
    if rank == 0:
        # ---- roofline of the dominant stage
        s_bytes = 4 if args.precision == "mixed" else 8
        sb = stage_bytes(s.n_atoms, s.mesh, R, m, s_bytes, info["n_pairs"], s.spline_order,
                         real_clusters=prof["real"][0] > 0)
        peak, peak_kind = measured_peaks()
        stages = {}
        stage_names = [k for k in prof if k != "total_launches"]
        total_ms = sum(prof[k][1] for k in stage_names)
        for name in stage_names:
            nl, ms = prof[name]
            if nl == 0:
                continue
            per_launch_ms = ms / nl
            d = {"launches": nl, "ms_total": ms, "share": ms / max(1e-12, total_ms), "us_per_launch": per_launch_ms * 1e3}
            if name in sb and per_launch_ms > 0:
                d["algorithmic_bytes_per_launch"] = sb[name]
                d["achieved_gbs"] = sb[name] / (per_launch_ms * 1e-3) / 1e9
            stages[name] = d
        dom = max((k for k in stages if k in sb), key=lambda k: stages[k]["ms_total"])
        ach = stages[dom]["achieved_gbs"]
        roof = roofline(stages, dom, peak, peak_kind, s.name, n_prof, npts_bytes=int(np.prod(s.mesh)) * R * s_bytes)

        # ---- end to end through the public API with host buffers
        pos_host = torch.tensor(s.pos, dtype=torch.float64).pin_memory()
        f_host = torch.empty((s.n_atoms, 3), dtype=torch.float64).pin_memory()
        t_e2e = []
        for k in range(args.e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sysm.update_positions(pos_host.numpy())
            e, _ = sysm.energy_forces(R, m, seed, forces=forces)
            f_host.copy_(forces, non_blocking=True)
            torch.cuda.synchronize()
            t_e2e.append(time.perf_counter() - t0)
        e2e = None
        if t_e2e:
            e2e_s = float(np.median(t_e2e))
            e2e = {"value": world * R * m / e2e_s, "unit": UNIT, "ms_per_step": e2e_s * 1e3,
                   "h2d_bytes_per_step": 3 * 8 * s.n_atoms, "d2h_bytes_per_step": 3 * 8 * s.n_atoms + 8,
                   "includes": "update_positions (H2D, neighbour list, splines, pair tensors) + energy_forces + D2H"}

        # ---- plain FP64 path on the same workload
        fp64 = None
        if args.precision == "mixed" and args.fp64_steps > 0:
            s64 = mbd.MBDSystem.from_workload(s, precision="fp64", stream=stream)
            e64, f64 = s64.energy_forces(R, m, seed)
            f64 = f64.clone()
            em, fm = sysm.energy_forces(R, m, seed)       # the mixed path on the same probes
            force_rel = float((fm - f64).abs().max() / f64.abs().max())
            tt = []
            for k in range(args.fp64_steps):
                flush.zero_()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                e64, _ = s64.energy_forces(R, m, seed)
                b.record(stream)
                torch.cuda.synchronize()
                tt.append(a.elapsed_time(b))
            ms64 = float(np.mean(tt))
            fp64 = {"value": R * m / (ms64 * 1e-3), "ms_per_step": ms64, "energy": e64,
                    "mixed_energy_rel_diff": abs(em - e64) / abs(e64),
                    "mixed_force_max_rel_diff": force_rel,
                    "speedup_mixed_over_fp64": ms64 / ms_per_step}
            s64.close()

        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(args.cpu_seconds, args.workload)

        cufft = None
        if not args.no_cufft:
            cufft = cufft_comparison(mbd, s, args.precision, R, stream)

        scs_line = None
        if args.scs_steps > 0 and world == 1:
            scs_line = scs_measurement(mbd, s, args, stream, flush)

        others = {}
        if args.other_steps > 0:
            for name in OTHER_WORKLOADS:
                if name != args.workload:
                    others[name] = other_workload(mbd, config(WORKLOADS[name]), args, stream, flush)
            if world == 1:
                others["batch64"] = batch_measurement(mbd, args, stream, args.other_steps)

        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 operator / f64 lanczos" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": s.name + ("" if m == s.n_steps else f"_m{m}"), "n_atoms": s.n_atoms,
                       "mesh": list(s.mesh),
                       "spline_order": s.spline_order, "n_probes_per_gpu": R, "n_steps": m,
                       "precision": args.precision, "quadrature": args.quadrature, "ewald_beta": s.ewald_beta,
                       "r_cut": s.r_cut,
                       "n_pairs": info["n_pairs"],
                       "step": "mbd_lanczos_energy (energy)" if args.energy_only
                       else "mbd_energy_forces (energy + forces)",
                       "autotune": tuning,
                       "l2": "flushed before every timed step (512 MB write, outside the events)",
                       "parallelism": f"probes sharded over {world} GPU(s)"},
            "ms_per_energy_forces": ms_per_step,
            "ns_per_atom_probe_step": ms_per_step * 1e6 / (s.n_atoms * R * m),
            "ms_per_step_with_stage_events": prof_ms,
            "stage_profile_steps": n_prof,
            "energy": energies[-1],
            "roofline": roof,
            "stages": stages,
            "e2e": e2e,
            "fp64_path": fp64,
            "cpu_baseline": cpu,
            "cufft_comparison": cufft,
            "scs_screen": scs_line,
            "other_workloads": others,
            "gpu_launches": launches_timed,
            "clocks": clocks,
            "wall_s_timed_region": wall,
            "kernel_sources": source_hash(),
        }
        print(json.dumps(out), flush=True)
    sysm.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def covering_members(member_ms, replay_ms):
    """The members sorted by their time alone (largest first) and how many of
    the largest, run one after another with the whole GPU, already take as
    long as the replay of all of them (the others run in their shadow)."""
    import numpy as np

    member_ms = np.asarray(member_ms, dtype=float)
    order = np.argsort(-member_ms, kind="stable")
    cover = int(np.searchsorted(np.cumsum(member_ms[order]), replay_ms) + 1)
    return order, min(cover, len(member_ms))


def batch_measurement(mbd, args, stream, steps):
    """The uneven 64-box workload: every box's Lanczos energy in one replayed CUDA
    graph per step, against the same boxes run one after another (L2 flushed
    before each step, CUDA events on the batch's stream)."""
    import numpy as np
    import torch

    from workloads.systems import batch_systems

    systems = batch_systems()
    R, m = systems[0].n_probes, systems[0].n_steps
    seeds = np.array([s.probe_seed for s in systems], dtype=np.uint64)
    t0 = time.perf_counter()
    batch = mbd.MBDBatch(systems, precision=args.precision, quadrature=args.quadrature, stream=stream)
    setup_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch.lanczos_energy(R, m, seeds)            # records the graph
    capture_s = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        batch.lanczos_energy(R, m, seeds)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        energies, _ = batch.lanczos_energy(R, m, seeds)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    info = batch.info()
    batch.close()
    t_step = float(np.mean(ms)) * 1e-3
    n_sys, atoms = len(systems), sum(s.n_atoms for s in systems)

    # the same boxes one after another through mbd_lanczos_energy
    seq_ms = []
    singles = [mbd.MBDSystem.from_workload(s, precision=args.precision, quadrature=args.quadrature,
                                           stream=stream) for s in systems]
    for s, g in zip(systems, singles):
        g.lanczos_energy(R, m, s.probe_seed)
    member_ms = np.zeros(len(systems))
    n_seq = min(steps, 3)
    for k in range(n_seq):
        flush.zero_()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(systems) + 1)]
        ev[0].record(stream)
        e_seq = []
        for i, (s, g) in enumerate(zip(systems, singles)):
            e_seq.append(g.lanczos_energy(R, m, s.probe_seed))
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        seq_ms.append(ev[0].elapsed_time(ev[-1]))
        member_ms += np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(len(systems))]) / n_seq
    for g in singles:
        g.close()
    del flush
    t_seq = float(np.mean(seq_ms)) * 1e-3
    max_rel = float(np.max(np.abs(np.asarray(e_seq) - energies) / np.abs(energies)))
    order, cover = covering_members(member_ms, t_step * 1e3)
    return {
        "metric": "probe-matvecs/s over a batch of uneven systems", "value": n_sys * R * m / t_step,
        "unit": UNIT, "steps": steps, "ms_per_step": t_step * 1e3,
        "config": {"workload": f"batch{n_sys}_random_N200-20000", "n_sys": n_sys, "total_atoms": atoms,
                   "n_atoms": [s.n_atoms for s in systems], "mesh": [s.mesh[0] for s in systems],
                   "n_probes": R, "n_steps": m, "precision": args.precision,
                   "step": "mbd_batch_lanczos_energy (one CUDA graph replay, energies of all boxes)",
                   "l2": "flushed before every timed step (512 MB write, outside the events)"},
        "ns_per_atom_probe_step": t_step * 1e9 / (atoms * R * m),
        "graph_kernels": info["graph_kernels"],
        "sequential_ms_per_step": t_seq * 1e3, "speedup_over_sequential": t_seq / t_step,
        "max_rel_diff_vs_sequential": max_rel, "setup_s": setup_s, "first_call_with_capture_s": capture_s,
        "member_ms_alone": [round(float(x), 3) for x in member_ms],
        "largest_members_alone_covering_replay": {
            "members": cover, "their_ms_alone": float(np.sum(member_ms[order[:cover]])),
            "their_atoms": int(sum(systems[i].n_atoms for i in order[:cover])),
            "rest_ms_alone": float(np.sum(member_ms[order[cover:]]))},
    }


def run_batch(args, world, rank, local):
    """--workload batch64: the batch measurement as the JSON line."""
    import torch

    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as mbd

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    visible = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    sampler = ClockSampler(visible[local] if local < len(visible) else local)
    time.sleep(0.3)
    out = batch_measurement(mbd, args, stream, args.steps)
    clocks = sampler.stop()
    out.update({"n_gpus": 1, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 operator / f64 lanczos" if args.precision == "mixed" else "f64",
                "data": "synthetic", "gpu_launches": out["graph_kernels"], "clocks": clocks,
                "kernel_sources": source_hash()})
    print(json.dumps(out), flush=True)
    return 0


def run_delta11_study(args):
    """Delta_11 = v^T C v of one normalised Rademacher probe against the mesh
    (spline orders 4 and 6), for a 96-molecule water box and a 512-atom diamond
    crystal (both 14.2 angstrom), r_cut 12 bohr, damping cut 13 bohr,
    beta_E 0.3/bohr, FP64.  Deviations are from the 96-point mesh; times are the
    device time of one Lanczos step with one probe (CUDA events, median of 20)."""
    import numpy as np
    import torch

    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as mbd
    from workloads.systems import ANGSTROM, diamond_system, water_system

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    seed = 2307022781

    def d11_and_ms(s):
        g = mbd.MBDSystem.from_workload(s, precision="fp64")
        _, det = g.lanczos_energy(1, 2, seed, details=True)
        ts = []
        for _ in range(20):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.lanczos_energy(1, 1, seed)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        g.close()
        return float(det["a"][0, 0]), float(np.median(ts))

    for name, make in (("water96_L14.2A", lambda: water_system(96, 5)), ("diamond512_L14.3A", diamond_system)):
        base = make().with_(r_cut=12.0, damp_cut=13.0, ewald_beta=0.3)
        box_a = base.cell[0, 0] / ANGSTROM
        for p in (4, 6):
            ref, _ = d11_and_ms(base.with_(mesh=(96, 96, 96), spline_order=p))
            for k in (8, 10, 12, 15, 16, 18, 20, 24, 27, 30, 36, 48):
                if k < 2 * p:
                    continue
                d, ms = d11_and_ms(base.with_(mesh=(k, k, k), spline_order=p))
                print(json.dumps({"study": "delta11_vs_mesh", "system": name, "spline_order": p, "mesh": k,
                                  "points_per_angstrom": k / box_a, "delta11": d,
                                  "rel_dev_from_mesh96": abs(d - ref) / abs(ref), "ms_one_step_one_probe": ms}),
                      flush=True)
        for tol in (1e-2, 1e-3, 1e-4, 1e-5):
            c = mbd.spme_params(base, tol, 6)
            print(json.dumps({"study": "spme_params", "system": name, "tol": tol, **c}), flush=True)
    return 0


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.cpu_child:
        cpu_baseline_child(args.cpu_seconds, args.workload)
        return 0
    if args.cpu_child_scs:
        cpu_scs_child()
        return 0
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.study == "delta11":
        return run_delta11_study(args)
    if args.workload == "batch64":
        return run_batch(args, world, rank, local)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    if "--cpu-child" in sys.argv or "--cpu-child-scs" in sys.argv or "reference" in sys.argv:
        os.environ.update(SINGLE_THREAD_ENV)     # before NumPy is imported
    sys.exit(main())

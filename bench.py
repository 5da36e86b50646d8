"""Benchmark: direct J+K Fock builds on the 16-atom RT-TDHF workload.

Workload: seeded 16-atom O/H cluster (6 O, 10 H; min distance 1.7 bohr),
even-tempered s,p,d basis (210 Cartesian functions, contraction depth 1-6),
complex-Hermitian density from 29 random orthonormal orbitals -- the density
a real-time TDHF step contracts.  One step = one J+K build (every class
kernel, density preparation and finalisation), Schwarz threshold 1e-14.

Headline `value`: mixed-precision builds/s (FP32 for quartets whose Schwarz x
density bound is below mixed_tol, double-float -- FP32 pairs -- up to
fp64_tol, FP64 above; everything accumulated exactly), with the
energy error against the all-FP64 GPU build checked in the same run
(|dE| <= 1e-6 Eh).  The all-FP64 rate is reported beside it.  The same run
then times the 100-atom, 1930-function single build (the same three tiers,
mixed_tol 3e-3, Schwarz 1e-12) under the key "large100" (--large-steps, 0
to skip).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
  python bench.py --impl reference ...   # the CPU oracle on the same workload
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

import synth  # noqa: E402

METRIC = "J+K Fock builds/s & ERI quartets/s; mixed vs FP64 GPU at |dE|<=1e-6 Eh"
WORKLOAD = "rt16: 16-atom O6H10 cluster, 210 Cartesian s,p,d functions, complex-Hermitian P (29 occ)"
# precision split of the headline build: the mixed_tol sweep of this
# workload (--workload tolsweep) gives |dE| 0.3-2.3e-7 Eh at 5e-3 (target
# 1e-6; 1e-2 leaves 2.5e-7 to 8.3e-7 and element errors of 2.5e-6, too
# close), checked again in every run
MIXED_TOL = 5e-3
# double-float tier of the mixed builds: quartets with mixed_tol <= bound <
# FP64_TOL in pairs of FP32 values (~48 bits, on the FP32 pipes), bound >=
# FP64_TOL in FP64.  The sweep at mixed_tol 5e-3 (--workload tolsweep):
# two tiers 173 ms, FP64_TOL 0.1 107 ms, 1.0 98 ms, |dE| the same to 1e-14
# Eh; FP64 keeps the quartets bounded above 1 Eh
FP64_TOL = 1.0
# the RT-TDHF comparison keeps a tighter split: its mixed run never returns
# to all-FP64 builds, and the dipole error grows with the split
RT_MIXED_TOL = 1e-3
NOCC = 29


def workload():
    mol, bas = synth.workload_rt16()
    n = bas.nbf
    P = synth.density(n, NOCC, 5, complex_=True)
    return mol, bas, P


# the large single J/K build: 100-atom cluster, three precision tiers (the
# tighter 3e-3 split: its energy error against an all-FP64 build is not
# measured in the benchmark run)
LARGE_WORKLOAD = ("large100: 100-atom cluster (H with p 0.25, else C/N/O), 1930 Cartesian s,p,d functions, "
                  "real P of 200 random orthonormal orbitals, Schwarz 1e-12")
LARGE_MIXED_TOL = 3e-3
LARGE_SCHWARZ = 1e-12


def large_workload():
    mol, bas = synth.workload_large100()
    return mol, bas, synth.density(bas.nbf, 200, 11)


def large_leg(steps: int, warmup: int, fp64_ref: bool):
    """Config 3 in the same process: mixed builds timed with CUDA events
    (one profiled build gives the per-class kernel times), optionally the
    all-FP64 build for the energy error of the split."""
    import torch

    import paper_1905_01381_gb300 as cq
    from paper_1905_01381_gb300 import flops as fl
    mol, bas, Ph = large_workload()
    t0 = time.perf_counter()
    b = cq.Basis(mol, bas)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    n = b.nbf
    P = torch.as_tensor(Ph, device="cuda")
    J = torch.empty((n, n), dtype=torch.float64, device="cuda")
    K = torch.empty((n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    kw = dict(prec=cq.CQ_PREC_MIXED, mixed_tol=LARGE_MIXED_TOL, fp64_tol=FP64_TOL, schwarz_tol=LARGE_SCHWARZ,
              J=J, K=K)
    for _ in range(warmup):
        b.fock_build(P, **kw)
    torch.cuda.synchronize()
    tms = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for i in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.fock_build(P, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
    # one profiled build: per class and precision kernel times (the passes of
    # a large basis run on one stream, so the events time each launch alone)
    b.profile(True)
    Jm, Km, st = b.fock_build(P, stats=True, **kw)
    cls = b.class_stats()
    b.profile(False)
    peak64, peak32 = cq.peak_fma(False), cq.peak_fma(True)
    peaks = prec_peaks(peak64, peak32)
    dom = None
    tot = [0.0, 0.0, 0.0]
    for key, v in cls.items():
        X, Y = cq.QUARTET_CLASSES[v["qc"]]
        v["flops"] = fl.class_flops(X, Y, v["quartets"], v["prims"], 1)
        tot[v["prec"]] += v["flops"]
        if dom is None or v["ms"] > cls[dom]["ms"]:
            dom = key
    f64, f32, fdf = tot
    dv = cls[dom]
    dpeak = peaks[dv["prec"]]
    ms = sum(tms) / len(tms)
    out = {"workload": LARGE_WORKLOAD, "nbf": n, "nshell": b.nshell, "basis_setup_s": setup_s,
           "mixed_tol": LARGE_MIXED_TOL, "fp64_tol": FP64_TOL, "schwarz_tol": LARGE_SCHWARZ, "steps": steps,
           "warmup": warmup,
           "builds_per_s": 1e3 / ms, "ms_per_build": ms,
           "quartets_per_s": (st["quartets_fp64"] + st["quartets_fp32"] + st["quartets_df"]) * 1e3 / ms,
           "quartets_per_build": {"fp64": st["quartets_fp64"], "df": st["quartets_df"], "fp32": st["quartets_fp32"]},
           "prim_quartets_per_build": {"fp64": st["prim_fp64"], "df": st["prim_df"], "fp32": st["prim_fp32"]},
           "gflops_per_build": {"fp64": f64 * 1e-9, "df": fdf * 1e-9, "fp32": f32 * 1e-9},
           "build_roofline": {"min_ms": sum(f / pk for f, pk in zip(tot, peaks)) * 1e3, "ms": ms,
                              "frac": sum(f / pk for f, pk in zip(tot, peaks)) * 1e3 / ms},
           "roofline": {"bound": "alu", "kernel": dom, "achieved": dv["flops"] / (dv["ms"] * 1e-3) * 1e-12,
                        "peak": dpeak * 1e-12, "unit": "TFLOP/s",
                        "frac": dv["flops"] / (dv["ms"] * 1e-3) / dpeak, "traffic": None},
           "class_roofline": {k: {"ms": round(v["ms"], 2), "quartets": v["quartets"], "prims": v["prims"],
                                  "frac": round(v["flops"] / max(v["ms"], 1e-9) * 1e3 / peaks[v["prec"]], 4)}
                              for k, v in sorted(cls.items(), key=lambda kv: -kv[1]["ms"])},
           "clocks": clk.summary(), "accuracy_vs_fp64_gpu": None}
    if fp64_ref:
        t = time.perf_counter()
        J64, K64, st64 = b.fock_build(P, schwarz_tol=LARGE_SCHWARZ, stats=True)
        torch.cuda.synchronize()
        dE = float(torch.sum((2 * (Jm - J64) - (Km - K64)) * P.T).item())
        out["accuracy_vs_fp64_gpu"] = {"dE_Eh": abs(dE), "max_dJ": float((Jm - J64).abs().max().item()),
                                       "max_dK": float((Km - K64).abs().max().item()),
                                       "fp64_build_s": time.perf_counter() - t,
                                       "fp64_prim_quartets": st64["prim_fp64"]}
    b.close()
    return out


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over the ranks of the process group (x itself
    without one): the replicas' timed region ends when the slowest ends."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rk, lr


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1.0)   # 256 MiB write, larger than the 129 MB L2


# ---------------------------------------------------------------- reference arm
def pair_cost_model(ob) -> np.ndarray:
    """Modelled cost of each bra shell pair p of the oracle's unique-quartet
    loop (kets p2 <= p): its primitive quartets, each weighted by
    (1 + L_bra + L_ket)^2.5 for the growth of the integral work with total
    angular momentum."""
    a, b = np.tril_indices(ob.nsh)
    L, npr = np.asarray(ob.L), np.asarray(ob.np_)
    Lp = L[a] + L[b]
    wp = (npr[a] * npr[b]).astype(np.float64)
    cost = np.zeros(a.size)
    for l in range(int(Lp.max()) + 1):
        pref = np.cumsum(np.where(Lp == l, wp, 0.0))      # kets p2 <= p of total momentum l
        cost += (1.0 + Lp + l) ** 2.5 * pref
    return wp * cost


def bra_pair_sample(ob, frac: float, seed: int):
    """Seeded systematic sample of the oracle's bra shell pairs (pair index
    a(a+1)/2 + b, a >= b): the pairs sorted by modelled cost, every k-th
    (k = 1/frac) from a random start.  Returns the pairs and the ratio of
    the whole build's modelled cost to the sample's."""
    cost = pair_cost_model(ob)
    order = np.argsort(cost, kind="stable")
    k = max(1, int(round(1.0 / frac)))
    start = int(synth.rng(seed).integers(0, k))
    picks = np.sort(order[start::k])
    return picks, float(cost.sum() / cost[picks].sum())


def oracle_rate(ob, Ds, frac, seed, nthreads):
    """Builds/s of the oracle estimated from one sample: the sample's time
    scaled by the ratio of modelled costs (whole build / sample)."""
    import oracle
    npair = ob.nsh * (ob.nsh + 1) // 2
    total = npair * (npair + 1) // 2
    pairs, ratio = bra_pair_sample(ob, frac, seed)
    t = time.perf_counter()
    _, _, nq = oracle.jk_sample_pairs(ob, Ds, pairs, nthreads)
    dt = time.perf_counter() - t
    return 1.0 / (dt * ratio), nq, dt, total, pairs.size


def run_reference(args):
    ws, rk, _ = dist_env()
    if rk != 0:
        return 0
    import oracle
    oracle.build()
    mol, bas, P = workload()
    ob = oracle.OBasis(mol, bas)
    nthreads = oracle.nthreads_default()
    Ds = [P.real, P.imag]
    oracle_rate(ob, Ds, 0.1 * args.ref_frac, 7, nthreads)   # warm-up (small)
    times, builds_time, nqs = [], [], []
    total = npick = 0
    for k in range(args.warmup + args.steps):
        rate, nq, dt, total, npick = oracle_rate(ob, Ds, args.ref_frac, 100 + k, nthreads)
        if k >= args.warmup:
            times.append(dt); nqs.append(nq); builds_time.append(1.0 / rate)
    builds = len(builds_time) / sum(builds_time)
    line = {"impl": "reference", "metric": METRIC, "value": builds, "unit": "builds/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            # wall time of one timed step (one sample), not of a whole build
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nbf": int(ob.nbf), "unique_shell_quartets": total},
            "quartets_per_s": sum(nqs) / sum(times),
            "ms_per_build_estimated": 1e3 / builds,
            "cpu_baseline": {"value": builds, "unit": "builds/s", "cores": nthreads, "kind": "oracle",
                             "sample": f"per step: a seeded systematic sample of {npick} bra shell pairs "
                                       f"(every {int(round(1 / args.ref_frac))}-th by modelled cost) of the "
                                       f"unique-quartet loop ({total} shell quartets per build); the step's "
                                       f"time scaled by the modelled cost of the whole build over the sample's"},
            "e2e": {"value": builds, "unit": "builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline(seconds: float, ref_frac: float):
    """The oracle on the host cores, timed on the reference arm's kind of
    sample, grown to about `seconds` of work."""
    import oracle
    oracle.build()
    mol, bas, P = workload()
    ob = oracle.OBasis(mol, bas)
    nthreads = oracle.nthreads_default()
    Ds = [P.real, P.imag]
    rate0, _, dt0, _, _ = oracle_rate(ob, Ds, 0.1 * ref_frac, 7, nthreads)
    frac = min(1.0, 0.1 * ref_frac * max(seconds, 1e-3) / max(dt0, 1e-3))
    rate, nq, dt, total, npick = oracle_rate(ob, Ds, frac, 99, nthreads)
    return {"value": rate, "unit": "builds/s", "cores": nthreads, "kind": "oracle",
            "sample": f"seeded systematic sample of {npick} bra shell pairs (every {int(round(1 / frac))}-th "
                      f"by modelled cost) of the unique-quartet loop: {nq} of {total} shell quartets in "
                      f"{dt:.1f} s, scaled by the modelled cost of the whole build over the sample's",
            "quartets_per_s": nq / dt}


# ---------------------------------------------------------------- GPU arm
TRAFFIC = os.path.join(ROOT, "profiles", "traffic_jk_rt16.json")
KERNEL_SOURCES = ("csrc/cq_common.cuh", "csrc/cq_df.cuh", "csrc/cq_jk.cuh", "csrc/cq_coop.cuh",
                  "csrc/cq_coop_kernel.cuh", "csrc/cq_sym.cuh", "csrc/gen_eri.py", "csrc/gen_coop.py",
                  "csrc/gen_sym.py", "buildlib.py")   # buildlib.py: lanes per quartet of each kernel


def kernel_sources_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1905_01381_gb300", f), "rb").read())
    return h.hexdigest()


def traffic_of(key, cls, variant):
    """DRAM bytes (read + write) of one launch of a class kernel, from the
    ncu capture summarised in profiles/ (bytes per quartet x the launch's
    quartets); None when no capture of this kernel and variant exists or the
    kernel sources changed since it was taken."""
    try:
        tj = json.load(open(TRAFFIC))
    except (OSError, ValueError):
        return None
    if tj.get("sources_sha1") != kernel_sources_sha1():
        return None
    for e in tj.get("launches", {}).get(key, []):
        if e.get("variant") == variant:
            return e["bytes_per_quartet"] * cls["quartets"]
    return None


def prec_peaks(peak64, peak32):
    """Roofline peaks of the three precisions: the measured FP64 and FP32 FMA
    peaks, and for double-float the FP32 peak x 2/30 -- one double-float FMA
    (2 FLOPs) is 15 FP32 instructions in this implementation (cq_df.cuh)."""
    return (peak64, peak32, peak32 * 2.0 / 30.0)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1905_01381_gb300 as cq
    from paper_1905_01381_gb300 import flops as fl

    ws, rk, lr = dist_env()
    torch.cuda.set_device(lr)
    if ws > 1:
        dist.init_process_group("nccl")
    cq.build() if rk == 0 or ws == 1 else None
    if ws > 1:
        dist.barrier()
    mol, bas, Ph = workload()
    b = cq.Basis(mol, bas)
    n = b.nbf
    stream = torch.cuda.current_stream()
    P = torch.as_tensor(Ph, device="cuda")
    prec = cq.CQ_PREC_MIXED if args.prec == "mixed" else cq.CQ_PREC_FP64
    J = torch.empty((n, n), dtype=torch.float64, device="cuda")
    K = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    flush = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # ---- kernel variant per class (autotuner; set-up, not timed)
    if not args.no_autotune:
        # --tuning-cache reuses the table an earlier run stored (profiling runs
        # that must launch exactly the timed build's kernels)
        b.autotune(P, prec=prec, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL if prec != cq.CQ_PREC_FP64 else 0.0,
                   cache=args.tuning_cache)
    for spec in args.variant:          # QC:PREC:VARIANT, after the autotuner
        q, pv, v = (int(x) for x in spec.split(":"))
        b.set_variant(q, pv, v)
    tuned = {"variant": [[b.get_variant(q, p) for p in range(3)] for q in range(21)]}

    # ---- accuracy of the timed mode against the all-FP64 build (same run)
    J64, K64 = b.fock_build(P)
    Jm, Km = b.fock_build(P, prec=prec, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL)
    dF = 2 * (Jm - J64).to(torch.complex128) - (Km - K64)
    dE = float(abs(torch.sum(dF * P.T).real.item()))
    dJ = float((Jm - J64).abs().max().item())
    dK = float((Km - K64).abs().max().item())

    def build():
        b.fock_build(P, prec=prec, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL, J=J, K=K)

    for _ in range(args.warmup):
        build()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(lr) as clk:
        for i in range(args.steps):
            flush_l2(flush)
            ev[i][0].record(stream)
            build()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    tot_ms = max_over_ranks(sum(step_ms), "cuda")
    value = ws * args.steps / (tot_ms * 1e-3)

    # ---- per-class profile (one extra build, events around each class kernel)
    b.profile(True)
    _, _, st = b.fock_build(P, prec=prec, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL, J=J, K=K, stats=True)
    cls = b.class_stats()
    b.profile(False)
    quartets = st["quartets_fp64"] + st["quartets_fp32"] + st["quartets_df"]
    nk = 2
    peak64 = cq.peak_fma(False)
    peak32 = cq.peak_fma(True)
    peaks = prec_peaks(peak64, peak32)
    tot = [0.0, 0.0, 0.0]
    dom = None
    for key, v in cls.items():
        X, Y = cq.QUARTET_CLASSES[v["qc"]]
        f = fl.class_flops(X, Y, v["quartets"], v["prims"], nk)
        v["flops"] = f
        tot[v["prec"]] += f
        if dom is None or v["ms"] > cls[dom]["ms"]:
            dom = key
    tot_flops64, tot_flops32, tot_flopsdf = tot
    dv = cls[dom]
    dom_peak = peaks[dv["prec"]]
    achieved = dv["flops"] / (dv["ms"] * 1e-3)
    traffic = traffic_of(dom, dv, b.get_variant(dv["qc"], dv["prec"]))

    # ---- FP64-only rate (reported beside the headline)
    fp64_rate = None
    if prec != cq.CQ_PREC_FP64:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nrep = max(1, min(3, args.steps))
        tms = 0.0
        for _ in range(nrep):
            flush_l2(flush)
            e0.record(stream)
            b.fock_build(P, J=J, K=K)
            e1.record(stream)
            torch.cuda.synchronize()
            tms += e0.elapsed_time(e1)
        fp64_rate = nrep / (tms * 1e-3)

    # ---- end to end through the public API with host buffers
    Ph_pin = torch.from_numpy(Ph).pin_memory()
    Jh = torch.empty((n, n), dtype=torch.float64).pin_memory()
    Kh = torch.empty((n, n), dtype=torch.complex128).pin_memory()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nrep = max(1, min(3, args.steps))
    e0.record(stream)
    for _ in range(nrep):
        Pd = Ph_pin.to("cuda", non_blocking=True)
        Jd, Kd = b.fock_build(Pd, prec=prec, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL)
        Jh.copy_(Jd, non_blocking=True)
        Kh.copy_(Kd, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e = ws * nrep / (e0.elapsed_time(e1) * 1e-3)

    # density preparation, block maxima, classify (count), scan, classify
    # (write), counter totals, finalisation + one launch per class and precision
    launches_per_build = 7 + sum(1 for v in cls.values())
    out = None
    if rk == 0:
        out = {"metric": METRIC, "value": value, "unit": "builds/s", "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64+df+f32" if prec != cq.CQ_PREC_FP64 else "f64", "data": "synthetic",
               "config": {"workload": WORKLOAD, "nbf": n, "precision": args.prec, "mixed_tol": MIXED_TOL,
                          "fp64_tol": FP64_TOL, "schwarz_tol": 1e-14,
                          "l2": "flushed (256 MiB write) between timed steps", "parallelism": f"replicas x{ws}"},
               "quartets_per_s": value * quartets,
               "quartets_per_build": {"fp64": st["quartets_fp64"], "df": st["quartets_df"],
                                      "fp32": st["quartets_fp32"]},
               "prim_quartets_per_build": {"fp64": st["prim_fp64"], "df": st["prim_df"], "fp32": st["prim_fp32"]},
               "fp64_builds_per_s": fp64_rate if fp64_rate is not None else value,
               "accuracy_vs_fp64_gpu": {"dE_Eh": dE, "max_dJ": dJ, "max_dK": dK},
               "gflops_per_build": {"fp64": tot_flops64 * 1e-9, "df": tot_flopsdf * 1e-9, "fp32": tot_flops32 * 1e-9},
               # whole build against the time its FLOPs need at the three
               # precisions' peaks (class kernels run concurrently)
               "build_roofline": {"min_ms": sum(f / pk for f, pk in zip(tot, peaks)) * 1e3,
                                  "ms": tot_ms / args.steps,
                                  "frac": sum(f / pk for f, pk in zip(tot, peaks)) * 1e3 / (tot_ms / args.steps)},
               "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved * 1e-12,
                            "peak": dom_peak * 1e-12, "unit": "TFLOP/s", "frac": achieved / dom_peak,
                            "traffic": traffic,
                            "peak_source": "measured FMA-chain peaks in this run (cq_peak_fma), "
                                           f"fp64 {peak64 * 1e-12:.3f} / fp32 {peak32 * 1e-12:.2f} TFLOP/s; "
                                           f"double-float = fp32 x 2/30 = {peaks[2] * 1e-12:.2f} TFLOP/s"},
               "tuned_variants": tuned["variant"],
               "class_roofline": {k: {"ms": round(v["ms"], 3), "quartets": v["quartets"], "prims": v["prims"],
                                      "tflops": round(v["flops"] / max(v["ms"], 1e-9) * 1e-9, 4),
                                      "frac": round(v["flops"] / max(v["ms"], 1e-9) * 1e3 / peaks[v["prec"]], 4)}
                                  for k, v in sorted(cls.items(), key=lambda kv: -kv[1]["ms"])},
               "class_ms": {k: round(v["ms"], 3) for k, v in sorted(cls.items(), key=lambda kv: -kv[1]["ms"])},
               "e2e": {"value": e2e, "unit": "builds/s", "h2d_bytes_per_step": n * n * 16,
                       "d2h_bytes_per_step": n * n * 8 + n * n * 16},
               "gpu_launches": launches_per_build * args.steps,
               "clocks": clk.summary()}
    b.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rk == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.ref_frac) if ws == 1 else None
    if rk == 0 and ws == 1 and args.large_steps > 0:
        # the 100-atom single build (config 3) in the same run, under its own key
        out["large100"] = large_leg(args.large_steps, args.large_warmup, args.large_fp64)
    if rk == 0:
        print(json.dumps(out))
    return 0


def _driver_setup():
    import torch
    import paper_1905_01381_gb300 as cq
    ws, rk, lr = dist_env()
    if ws > 1:
        # the driver workloads are single-GPU runs: replicas print nothing
        if rk != 0:
            return None, None
    torch.cuda.set_device(lr)
    cq.build()
    return torch, cq


def _line(metric, value, unit, hib, args, ms, config, extra, clk, launches):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": hib, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+df+f32", "data": "synthetic", "config": config,
           "gpu_launches": launches, "clocks": clk.summary()}
    out.update(extra)
    print(json.dumps(out))


def run_tol_sweep(args):
    """The precision split's trade-off on the 16-atom workload: for each
    mixed_tol, the share of quartets evaluated in FP32, the errors of J, K
    and E against the all-FP64 build, and the build time."""
    torch, cq = _driver_setup()
    if cq is None:
        return 0
    mol, bas, Ph = workload()
    b = cq.Basis(mol, bas)
    P = torch.as_tensor(Ph, device="cuda")
    b.autotune(P, prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL, cache=False)
    J64, K64 = b.fock_build(P)
    flush = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(**kw):
        for _ in range(args.warmup):
            b.fock_build(P, **kw)
        tms = []
        for _ in range(max(1, args.steps)):
            flush_l2(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.fock_build(P, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
        return statistics.median(tms)

    rows = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t64 = timed()
        for tol in [float(x) for x in args.tols.split(",")]:
            for dtol in [float(x) for x in args.df_tols.split(",")]:
                if dtol and dtol <= tol:
                    continue
                kw = dict(prec=cq.CQ_PREC_MIXED, mixed_tol=tol, fp64_tol=dtol)
                Jm, Km, st = b.fock_build(P, stats=True, **kw)
                dF = 2 * (Jm - J64).to(torch.complex128) - (Km - K64)
                nq = max(1, st["quartets_fp32"] + st["quartets_fp64"] + st["quartets_df"])
                rows.append({"mixed_tol": tol, "fp64_tol": dtol,
                             "fp32_share": st["quartets_fp32"] / nq, "df_share": st["quartets_df"] / nq,
                             "dE_Eh": float(abs(torch.sum(dF * P.T).real.item())),
                             "max_dJ": float((Jm - J64).abs().max().item()),
                             "max_dK": float((Km - K64).abs().max().item()),
                             "ms": timed(**kw)})
    b.close()
    best = min((r for r in rows if r["dE_Eh"] <= 1e-6), key=lambda r: r["ms"], default=None)
    _line("J+K build time vs precision split (mixed_tol sweep)", best["ms"] if best else None, "ms", False, args,
          best["ms"] if best else None, {"workload": WORKLOAD, "l2": "flushed between timed builds"},
          {"fp64_ms": t64, "sweep": rows, "fastest_within_1e-6": best}, clk, None)
    return 0


def run_cluster30(args):
    """A 30-atom cluster of the large workload's composition (598 functions):
    mixed builds with the large workload's split and Schwarz threshold and
    the default kernel variants -- a case small enough to profile the class
    kernels of the large build one launch at a time."""
    torch, cq = _driver_setup()
    if cq is None:
        return 0
    mol = synth.cluster(30, 3333, p_h=0.25)
    b = cq.Basis(mol, synth.basis_spd(mol, 3340))
    P = torch.as_tensor(synth.density(b.nbf, 60, 11), device="cuda")
    stream = torch.cuda.current_stream()
    kw = dict(prec=cq.CQ_PREC_MIXED, mixed_tol=LARGE_MIXED_TOL, schwarz_tol=LARGE_SCHWARZ)
    for _ in range(args.warmup):
        b.fock_build(P, **kw)
    tms = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(max(1, args.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, st = b.fock_build(P, stats=True, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
    b.close()
    ms = statistics.median(tms)
    _line(METRIC, 1e3 / ms, "builds/s", True, args, ms,
          {"workload": f"cluster30: 30-atom cluster (large100 composition), {b.nbf} functions, real P (60 occ)",
           "mixed_tol": LARGE_MIXED_TOL, "schwarz_tol": LARGE_SCHWARZ},
          {"quartets_per_build": {"fp64": st["quartets_fp64"], "fp32": st["quartets_fp32"]}}, clk,
          None)
    return 0


def run_transition(args):
    """J+K of a ph-RPA transition density on the 16-atom workload: D = C_o X
    C_v^T (random orthonormal occupied and virtual orbitals, random X; no
    symmetry), builds/s in FP64 and with the headline's three tiers, and the
    mixed build's errors against the FP64 one."""
    torch, cq = _driver_setup()
    if cq is None:
        return 0
    mol, bas = synth.workload_rt16()
    b = cq.Basis(mol, bas)
    n = b.nbf
    C = synth.orbitals(n, n, 7)
    X = synth.rng(8).standard_normal((NOCC, n - NOCC)) / np.sqrt(NOCC * (n - NOCC))
    D = torch.as_tensor(C[:, :NOCC] @ X @ C[:, NOCC:].T, device="cuda")
    kind = cq.CQ_DENS_REAL_GENERAL
    b.autotune(D, prec=cq.CQ_PREC_FP64, cache=False, kind=kind)
    b.autotune(D, prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL, cache=False, kind=kind)
    flush = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    modes = {"fp64": dict(prec=cq.CQ_PREC_FP64),
             "mixed": dict(prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL)}
    out, ms = {}, {}
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for name, kw in modes.items():
            for _ in range(args.warmup):
                b.fock_build(D, kind=kind, **kw)
            tms = []
            for _ in range(max(1, args.steps)):
                flush_l2(flush)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out[name] = b.fock_build(D, kind=kind, **kw)
                e1.record(stream)
                torch.cuda.synchronize()
                tms.append(e0.elapsed_time(e1))
            ms[name] = statistics.median(tms)
    (J64, K64), (Jm, Km) = out["fp64"], out["mixed"]
    dJ = float((Jm - J64).abs().max().item())
    dK = float((Km - K64).abs().max().item())
    b.close()
    _line("J+K builds/s of a non-Hermitian (transition) density, mixed vs FP64", 1e3 / ms["mixed"], "builds/s",
          True, args, ms["mixed"],
          {"workload": WORKLOAD.replace("complex-Hermitian P (29 occ)",
                                        "real transition density C_o X C_v^T (29 occ, 181 virt)"),
           "mixed_tol": MIXED_TOL, "fp64_tol": FP64_TOL, "l2": "flushed (256 MiB write) between timed builds"},
          {"fp64_builds_per_s": 1e3 / ms["fp64"], "max_dJ_mixed_vs_fp64": dJ, "max_dK_mixed_vs_fp64": dK,
           "max_abs_K_asymmetry": float((K64 - K64.T).abs().max().item())}, clk, None)
    return 0


def run_scf(args):
    """RHF direct SCF on the 16-atom workload: time to the converged energy,
    all-FP64 against mixed precision with incremental builds."""
    torch, cq = _driver_setup()
    if cq is None:
        return 0
    mol, bas = synth.workload_rt16()
    b = cq.Basis(mol, bas)
    nocc = mol.n_electrons() // 2
    P = torch.as_tensor(synth.density(b.nbf, nocc, 5), device="cuda")
    # FP64 kernels for the all-FP64 run and builds; FP32 and double-float for the mixed ones
    b.autotune(P, prec=cq.CQ_PREC_FP64, cache=False)
    b.autotune(P, prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL, cache=False)
    for _ in range(args.warmup):
        b.fock_build(P)
    modes = {"fp64": dict(prec=cq.CQ_PREC_FP64),
             "mixed": dict(prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL, incremental=True,
                           switch_tol=1e-5)}
    res = {}
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for name, kw in modes.items():
            ts, st = [], None
            for _ in range(args.steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, _, st = b.scf(nocc, **kw)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            res[name] = {"s": statistics.median(ts), "energy": st["energy"], "iterations": st["iterations"],
                         "quartets_fp64": st["quartets_fp64"], "quartets_fp32": st["quartets_fp32"],
                         "quartets_df": st["quartets_df"]}
    dE = abs(res["mixed"]["energy"] - res["fp64"]["energy"])
    b.close()
    _line("RHF SCF time to converged energy (mixed + incremental vs FP64)", res["mixed"]["s"], "s", False, args,
          res["mixed"]["s"] * 1e3,
          {"workload": WORKLOAD.replace("complex-Hermitian P (29 occ)", "RHF, 29 doubly occupied"),
           "e_tol": 1e-10, "d_tol": 1e-8, "mixed_tol": MIXED_TOL, "fp64_tol": FP64_TOL, "switch_tol": 1e-5},
          {"fp64_s": res["fp64"]["s"], "speedup_vs_fp64": res["fp64"]["s"] / res["mixed"]["s"],
           "dE_mixed_vs_fp64_Eh": dE, "runs": res}, clk, None)
    return 0


def run_rt(args):
    """RT-TDHF (MMUT with EM2 restarts) from the RHF ground state of the
    16-atom workload, delta kick 1e-4 au along z for the first step:
    steps/s in FP64 and mixed precision, and the observables' agreement."""
    torch, cq = _driver_setup()
    if cq is None:
        return 0
    mol, bas = synth.workload_rt16()
    b = cq.Basis(mol, bas)
    nocc = mol.n_electrons() // 2
    D, _, st = b.scf(nocc, d_tol=1e-10)
    P0 = D.to(torch.complex128)
    b.autotune(P0, prec=cq.CQ_PREC_FP64, cache=False)
    b.autotune(P0, prec=cq.CQ_PREC_MIXED, mixed_tol=RT_MIXED_TOL, fp64_tol=FP64_TOL, cache=False)
    dt = 0.05
    field = dict(field=(0.0, 0.0, 1e-4), t_on=0.0, t_off=dt)
    traces, rates = {}, {}
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for name, kw in (("fp64", dict(prec=cq.CQ_PREC_FP64)),
                         ("mixed", dict(prec=cq.CQ_PREC_MIXED, mixed_tol=RT_MIXED_TOL, fp64_tol=FP64_TOL))):
            Pp, Pc = P0.clone(), P0.clone()
            for k in range(args.warmup):
                b.rt_step(k, Pp, Pc, dt=dt, **field, **kw)
            Pp, Pc = P0.clone(), P0.clone()
            obs = []
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(args.rt_steps):
                obs.append(b.rt_step(k, Pp if k else None, Pc, dt=dt, **field, **kw))
            torch.cuda.synchronize()
            rates[name] = args.rt_steps / (time.perf_counter() - t0)
            traces[name] = obs
    mu = {k: np.array([o["dipole"][2] for o in v]) for k, v in traces.items()}
    tr = {k: np.array([o["trPS"] for o in v]) for k, v in traces.items()}
    en = {k: np.array([o["energy"] for o in v]) for k, v in traces.items()}
    b.close()
    _line("RT-TDHF MMUT/EM2 steps/s (mixed vs FP64)", rates["mixed"], "steps/s", True, args,
          1e3 / rates["mixed"],
          {"workload": WORKLOAD.replace("complex-Hermitian P (29 occ)", "RHF ground state, delta kick 1e-4 au z"),
           "dt": dt, "steps": args.rt_steps, "restart_every": 50, "mixed_tol": RT_MIXED_TOL, "fp64_tol": FP64_TOL},
          {"fp64_steps_per_s": rates["fp64"],
           "max_abs_dmu_z_mixed_vs_fp64": float(np.abs(mu["mixed"] - mu["fp64"]).max()),
           "mu_z_response_range": float(np.ptp(mu["fp64"])),
           "max_abs_trPS_minus_nocc": {k: float(np.abs(v - nocc).max()) for k, v in tr.items()},
           "energy_drift_after_kick_Eh": {k: float(np.ptp(v[2:])) for k, v in en.items()},
           "ground_state_energy": st["energy"]}, clk, None)
    return 0


def run_batch(args):
    """Batched RHF over many uneven molecules (4-12 atoms, single-primitive
    even-tempered s,p,d shells) with the iterations replayed from a captured
    graph; the learned guess trained on batched SCF solutions of other
    molecules, against the core-Hamiltonian guess at identical energies."""
    torch, cq = _driver_setup()
    if cq is None:
        return 0
    t_all = time.perf_counter()
    train = synth.workload_batch(args.ntrain, rep=1, max_depth=1)
    test = synth.workload_batch(args.nmol, rep=0, max_depth=1)
    no = lambda items: [m.n_electrons(m.closed_shell_charge()) // 2 for m, _ in items]
    btr, bte = cq.Basis.batch(train), cq.Basis.batch(test)
    Pw = torch.zeros((bte.nmol, bte.ld, bte.ld), dtype=torch.float64, device="cuda")
    for m, n in enumerate(bte.mol_n):
        Pw[m, :n, :n] = torch.as_tensor(synth.density(n, no(test)[m], m))
    bte.autotune(Pw, prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, cache=False)
    for qc in range(21):
        for p in range(3):
            btr.set_variant(qc, p, bte.get_variant(qc, p))
    # training data: converged FP64 solutions of the training molecules
    t0 = time.perf_counter()
    Dtr, _, ittr, sttr = btr.scf_batch(no(train), raise_on_fail=False)
    t_train_scf = time.perf_counter() - t0
    ok = [i for i in range(btr.nmol) if ittr[i] < 128]
    keep = [train[i] for i in ok]
    bk = cq.Basis.batch(keep)
    Dk = bk.pack([btr.unpack(Dtr)[i] for i in ok])
    net = cq.DensityGuessMLP(seed=7)
    X, T, H = net.dataset(bk, Dk)
    loss0, _ = net.loss_grad(X, T, H)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = net.train(X, T, H, epochs=150, batch=256, lr=2e-3, seed=3)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    nocc = no(test)
    runs = {}
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for name, prec, learned in (("core_fp64", cq.CQ_PREC_FP64, False), ("learned_fp64", cq.CQ_PREC_FP64, True),
                                    ("core_mixed", cq.CQ_PREC_MIXED, False),
                                    ("learned_mixed", cq.CQ_PREC_MIXED, True)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            D0 = net.guess(bte, nocc) if learned else None
            _, E, it, st = bte.scf_batch(nocc, prec=prec, mixed_tol=MIXED_TOL, D0=D0, raise_on_fail=False)
            torch.cuda.synchronize()
            runs[name] = {"s": time.perf_counter() - t0, "E": E, "it": it, "st": st}
    base = runs["core_fp64"]
    conv = base["it"] < 128
    summary = {}
    for name, r in runs.items():
        same = conv & (r["it"] < 128) & (np.abs(r["E"] - base["E"]) <= 1e-8)
        summary[name] = {"s": round(r["s"], 3), "batched_iterations": r["st"]["iterations"],
                         "converged": int((r["it"] < 128).sum()), "same_energy_as_core_fp64": int(same.sum()),
                         "mean_iterations_same": float(r["it"][same].mean()) if same.any() else None,
                         "quartets_fp64": r["st"]["quartets_fp64"], "quartets_fp32": r["st"]["quartets_fp32"],
                         "graph": r["st"]["graph"]}
    best = runs["learned_mixed"]
    _line("batched RHF time to converged energies, learned guess + mixed vs core guess FP64",
          bte.nmol / best["s"], "molecules/s", True, args, best["s"] * 1e3,
          {"workload": f"{bte.nmol} molecules of 4-12 atoms (H/C/N/O), single-primitive even-tempered "
                       f"s,p,d shells, {min(bte.mol_n)}-{max(bte.mol_n)} functions",
           "training_molecules": len(ok), "training_pairs": int(X.shape[0]), "e_tol": 1e-10, "d_tol": 1e-8,
           "mixed_tol": MIXED_TOL},
          {"core_fp64_molecules_per_s": bte.nmol / base["s"],
           "speedup_vs_core_fp64": base["s"] / best["s"], "runs": summary,
           "training": {"scf_s": t_train_scf, "fit_s": t_fit, "loss0": loss0, "loss": loss},
           "wall_s": time.perf_counter() - t_all}, clk, None)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-frac", type=float, default=1.0 / 150,
                    help="fraction of the bra shell pairs the reference arm's oracle visits per step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernel variant per class (profiling runs)")
    ap.add_argument("--variant", action="append", default=[], metavar="QC:PREC:V",
                    help="set the kernel variant of one class and precision (0 FP64, 1 FP32, 2 double-float; after autotuning)")
    ap.add_argument("--workload", default="jk",
                    choices=["jk", "scf", "rt", "batch", "tolsweep", "cluster30", "transition"],
                    help="jk: the headline J+K build rate; scf / rt / batch: the drivers "
                         "(RHF time to converged energy, RT-TDHF steps, batched SCF with the learned guess); "
                         "transition: J+K of a non-Hermitian transition density")
    ap.add_argument("--tuning-cache", action="store_true",
                    help="reuse (or store) the autotuned variant table instead of re-tuning")
    ap.add_argument("--large-steps", type=int, default=1,
                    help="timed mixed builds of the 100-atom configuration after the headline (0: skip)")
    ap.add_argument("--large-warmup", type=int, default=0)
    ap.add_argument("--large-fp64", action="store_true",
                    help="also build the 100-atom case in all-FP64 for the split's energy error (about an hour)")
    ap.add_argument("--rt-steps", type=int, default=100)
    ap.add_argument("--nmol", type=int, default=512)
    ap.add_argument("--ntrain", type=int, default=512)
    ap.add_argument("--tols", default="1e-2,3e-3,1e-3,1e-4,1e-5,1e-6")
    ap.add_argument("--df-tols", default="0",
                    help="fp64_tol values of the sweep (0: no double-float tier)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "scf":
        return run_scf(args)
    if args.workload == "rt":
        return run_rt(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "tolsweep":
        return run_tol_sweep(args)
    if args.workload == "cluster30":
        return run_cluster30(args)
    if args.workload == "transition":
        return run_transition(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark: MHD cell-updates/s of the batched FP32-bulk block-AMR update and
its fraction of the HBM roofline, beside the plain per-block FP64 path.

One step = one full SSPRK3 time step (three stages: ghost fill, reconstruction,
glm + HLLD flux, update, psi damping; CFL dt + conservation sums on the device)
over every block of the workload.  Default workload: 3D block-AMR blast,
18,304 blocks of 16^3 over 4 levels (ratio 2), FP32 bulk with FP64 pressure
recovery, HLLD + vanleer, glm.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  Under torchrun each rank advances its own
replica of a single-domain workload (the update shards by block but the halo
exchange between GPUs is not built: weak scaling); the batched independent
instances (--workload c5) are partitioned over the ranks instead (no exchange:
strong scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
METRIC = "MHD cell-updates/s (FP32-bulk batched block-AMR)"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c4", choices=["c4", "c5", "c3", "c2"])
    p.add_argument("--kernel", default="auto", choices=["auto", "plain", "fused"])
    p.add_argument("--size", type=int, default=0,
                   help="workload size (c4: level-0 blocks per dim; c3/c2: cells per dim; "
                        "c5: instance count); 0 = the full configuration")
    p.add_argument("--flux", default=None, choices=["hll", "hlld", "tvdlf", "hllc"],
                   help="override the workload's flux scheme")
    p.add_argument("--limiter", default=None,
                   choices=["minmod", "vanleer", "koren", "superbee", "woodward", "mcbeta",
                            "albada", "cada3", "venk", "mp5", "weno5", "wenoz5", "wenozp5"],
                   help="override the workload's limiter")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the HLL and FP64-pressure variant timings")
    p.add_argument("--pressure", default="ff", choices=["ff", "fp64"],
                   help="FP32-bulk pressure recovery: float-float or double")
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison leg")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU-baseline leg")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the sub-records of the other workloads (c2, c3, c5)")
    p.add_argument("--no-tune", action="store_true",
                   help="skip the launch-shape autotuning before the timed region")
    return p.parse_args()


def make_workload(name, precision="fp32", size=0):
    from paper_2303_03026_gb300 import workloads as wl
    if name == "c4":
        W = wl.c4_blast_amr(base=size or 6, precision=precision)
        desc = {"workload": "3D block-AMR blast, %d blocks of 16^3 over 4 levels (ratio 2), "
                            "shell 0.2<=r<=0.3, HLLD+vanleer+glm, SSPRK3" % W.nblocks,
                "blocks": W.nblocks, "blocks_per_level": W.info["blocks_per_level"]}
    elif name == "c5":
        W = wl.c5_instances(count=size or 256, precision=precision)
        desc = {"workload": "256 uneven 2D instances 64^2..512^2 in 16^2 blocks, "
                            "HLLD+vanleer+glm, SSPRK3, per-instance dt", "blocks": W.nblocks}
    elif name == "c3":
        W = wl.c3_turbulence(n=size or 256, precision=precision)
        desc = {"workload": "3D %d^3 Mach-1 beta-0.01 turbulence in 16^3 blocks, "
                            "HLLD+vanleer+glm, SSPRK3" % (size or 256), "blocks": W.nblocks}
    else:
        W = wl.c2_orszag_tang(size or 1024, precision=precision)
        desc = {"workload": "2D Orszag-Tang %d^2 in 16^2 blocks, HLLD+koren+glm, SSPRK3"
                            % (size or 1024),
                "blocks": W.nblocks}
    return W, desc


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
            os.unlink(self.path)
        except Exception:
            return out
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                mhz.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if mhz:
            out = {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(mx),
                   "reasons": sorted(reasons), "samples": len(mhz)}
        return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(W, seconds_target=12.0, threads=None):
    """The FP64 oracle as it stands, timed on the host cores on a bounded sample
    of the workload's blocks: one full SSPRK3 step of ``nsample`` blocks, the
    sample sized from a small probe so that it takes about seconds_target."""
    import oracle
    threads = threads or os.cpu_count() or 1
    m = oracle.mesh_for(W, threads)
    U = W.U.astype(np.float64)
    dt, ch = m.cfl(U)
    rng = np.random.Generator(np.random.PCG64(11))
    A = np.zeros_like(U)
    B = np.zeros_like(U)
    nsample = min(W.nblocks, max(16, threads))
    for final in (False, True):
        blocks = np.sort(rng.choice(W.nblocks, nsample, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        m.stage(0, dt, ch, U, U, blocks=blocks, out=A)
        m.stage(1, dt, ch, U, A, blocks=blocks, out=B)
        m.stage(2, dt, ch, U, B, blocks=blocks, out=A)
        el = time.perf_counter() - t0
        if final or nsample >= W.nblocks:
            break
        nsample = min(W.nblocks, max(nsample, int(nsample * seconds_target / max(el, 1e-3))))
    cells = nsample * W.ncell
    return {"value": cells / el, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
            "sample": "%d random blocks (%d cells) of the workload, one full SSPRK3 step "
                      "(3 stages incl. ghost fill) in FP64, %.2f s" % (nsample, cells, el)}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    W, desc = make_workload(args.workload, "fp64", args.size)
    if args.flux:
        W.cfg.flux = args.flux
    if args.limiter:
        W.cfg.limiter = args.limiter
    desc["scheme"] = "%s + %s + %s, SSPRK3" % (W.cfg.flux.upper(), W.cfg.limiter,
                                               "glm" if W.cfg.glm else "no glm")
    import oracle
    threads = os.cpu_count() or 1
    m = oracle.mesh_for(W, threads)
    U = W.U
    dt, ch = m.cfl(U)
    rng = np.random.Generator(np.random.PCG64(13))
    nsample = min(W.nblocks, max(threads * 16, 128))
    blocks = np.sort(rng.choice(W.nblocks, nsample, replace=False)).astype(np.int32)
    A = np.zeros_like(U)
    B = np.zeros_like(U)

    def one():
        m.stage(0, dt, ch, U, U, blocks=blocks, out=A)
        m.stage(1, dt, ch, U, A, blocks=blocks, out=B)
        m.stage(2, dt, ch, U, B, blocks=blocks, out=A)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    cells = nsample * W.ncell
    value = cells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(desc, sample_blocks=nsample),
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": threads,
                             "kind": "oracle",
                             "sample": "%d random blocks (%d cells) per step, one full SSPRK3 "
                                       "step each" % (nsample, cells)},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def counters_from_profile(workload, kernel_digest):
    """Per cell-update counters of the fused stage kernel (DRAM bytes, warp
    instructions) from the committed ncu summary, when it was taken on the
    current build (else {})."""
    path = os.path.join(ROOT, "profiles", "k_fused_c4_counters.txt")
    try:
        rows = [r.split() for r in open(path) if r.strip() and not r.startswith("#")]
    except OSError:
        return {}
    for r in rows:
        kv = dict(x.split("=", 1) for x in r if "=" in x)
        if kv.get("workload") == workload and kv.get("build") == kernel_digest:
            return kv
    return {}


def max_over_ranks(value, device):
    """Maximum of a float over all ranks (the slowest rank's time); identity
    without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(torch, S, k):
    """ms per full step over k graph-launched steps (events on the state's stream)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    S.stream.synchronize()
    e0.record(S.stream)
    S.step(k)
    e1.record(S.stream)
    S.stream.synchronize()
    return e0.elapsed_time(e1) / k


VARS = ("rho", "m_x", "m_y", "m_z", "e", "B_x", "B_y", "B_z", "psi")


def rel_l1_by_var(a, b, ch):
    """Relative L1 error of a against b per conserved variable: rho and e
    against themselves, each component of m and B against the magnitude of
    its vector, psi against c_h |B| (its natural scale)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    mm = np.sqrt(b[1] ** 2 + b[2] ** 2 + b[3] ** 2).sum()
    bm = np.sqrt(b[5] ** 2 + b[6] ** 2 + b[7] ** 2).sum()
    out = {}
    for v, n in enumerate(VARS):
        s = (mm if v in (1, 2, 3) else bm if v in (5, 6, 7) else
             max(np.abs(b[8]).sum(), float(ch) * bm) if v == 8 else np.abs(b[v]).sum())
        out[n] = float(np.abs(a[v] - b[v]).sum() / max(s, 1e-300))
    return out


def bench_configs(torch, amrvac, dev, args, hbm):
    """Sub-records of the other workloads of the metric, one GPU, synthetic data
    (FP32 bulk with the headline's pressure recovery, --pressure):
    c5, the 256 uneven 2D instances batched in one launch per stage against the
    same instances advanced one at a time; c3, the 256^3 turbulence box in FP32
    bulk and in FP64 on the GPU, with the FP32 error against the FP64 GPU path
    after 1, 10 and 200 steps and against the FP64 oracle after one step; c2,
    the 1024^2 Orszag-Tang vortex at its stated FP64 precision (and FP32)."""
    import dataclasses
    import oracle
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # c5: batched vs one at a time
    W = make_workload("c5", "fp32")[0]
    cells = W.interior_cells()
    U = torch.from_numpy(W.U.astype(np.float32)).to(dev)
    S = amrvac.State.from_workload(W, device=dev, pressure=args.pressure)
    S.set_conserved(U)
    tune5 = None if args.no_tune else S.autotune(trial_steps=3)
    S.step(3)
    ms = time_steps(torch, S, 10)
    states, off = [], 0
    for q, inst in enumerate(W.instances):
        nb = int((W.block_meta[:, 0] == q).sum())
        meta = W.block_meta[off:off + nb].copy()
        meta[:, 0] = 0
        # the default launch shape: the batched state's dynamic schedule would
        # add a counter reset to every one of these small launches
        Sq = amrvac.State(W.cfg, [inst], meta, device=dev, stream=S.stream,
                          pressure=args.pressure)
        Sq.set_conserved(U[:, off:off + nb].contiguous())
        Sq.step(1)
        states.append(Sq)
        off += nb
    S.stream.synchronize()
    e0, e1 = ev(), ev()
    e0.record(S.stream)
    for _ in range(3):
        for Sq in states:
            Sq.step(1)
    e1.record(S.stream)
    S.stream.synchronize()
    msq = e0.elapsed_time(e1) / 3
    for Sq in states:
        Sq.close()
    out["c5"] = {"workload": "256 uneven 2D instances 64^2..512^2 in 16^2 blocks, FP32 bulk, "
                             "HLLD+vanleer+glm, SSPRK3, per-instance dt",
                 "blocks": int(W.nblocks), "cells": int(cells),
                 "value": cells / (ms / 1e3), "ms_per_step": ms, "tuning": tune5,
                 "pressure": args.pressure,
                 "frac": 288 * cells / (ms / 1e3) / 1e9 / hbm,
                 "one_at_a_time": {"value": cells / (msq / 1e3), "ms_per_step": msq,
                                   "launches": "one graph per instance per step"},
                 "batched_speedup": msq / ms}
    S.close()
    # the same instances with a five-point limiter (wenozp5, as the paper's 2D
    # hydro and thermal-instability runs): the fused 2D kernel with three ghost
    # layers against the plain per-block kernels
    five = {}
    W.cfg.limiter = "wenozp5"
    for kern in ("fused", "plain"):
        Sf = amrvac.State.from_workload(W, device=dev, kernel=kern, pressure=args.pressure)
        if kern == "fused" and tune5 is not None:
            Sf.set_tuning(tune5["ctas_per_sm"], tune5["order"], tune5["dynamic"], "sides")
        Sf.set_conserved(U)
        Sf.step(2)
        msf = time_steps(torch, Sf, 5)
        five[kern] = {"value": cells / (msf / 1e3), "ms_per_step": msf}
        Sf.close()
    W.cfg.limiter = "vanleer"
    out["c5"]["wenozp5"] = dict(five, speedup_fused=five["plain"]["ms_per_step"] /
                                five["fused"]["ms_per_step"])
    del U

    # c3: FP32 bulk and FP64 GPU, errors at 1, 10, 200 steps; oracle after 1
    W = make_workload("c3", "fp32")[0]
    cells = W.interior_cells()
    U64 = W.U.astype(np.float32).astype(np.float64)
    W64 = dataclasses.replace(W, cfg=dataclasses.replace(W.cfg, precision="fp64"))
    A = amrvac.State.from_workload(W, device=dev, pressure=args.pressure)
    B = amrvac.State.from_workload(W64, device=dev)
    A.set_conserved(U64.astype(np.float32))
    B.set_conserved(U64)
    errs, done = {}, 0
    for n in (1, 10, 200):
        A.step(n - done)
        B.step(n - done)
        done = n
        a = A.get_conserved(0)
        b = B.get_conserved(0)
        ch = A.diag()["ch"][0]
        errs[n] = rel_l1_by_var(a, b, ch)
        if n == 1:
            m = oracle.mesh_for(W64, os.cpu_count() or 1)
            Uo, to, ns, st = m.run(U64, 1e30, maxsteps=1)
            err_oracle = rel_l1_by_var(a, Uo, ch)
            err64_oracle = float(np.abs(b - Uo).max() / np.abs(Uo).max())
            del Uo
    A.set_conserved(U64.astype(np.float32))
    B.set_conserved(U64)
    A.step(3)
    B.step(2)
    ms32 = time_steps(torch, A, 20)
    ms64 = time_steps(torch, B, 5)
    out["c3"] = {"workload": "3D 256^3 Mach-1 beta-0.01 turbulence in 16^3 blocks, "
                             "HLLD+vanleer+glm, SSPRK3",
                 "cells": int(cells), "value": cells / (ms32 / 1e3), "ms_per_step": ms32,
                 "pressure": args.pressure,
                 "frac": 288 * cells / (ms32 / 1e3) / 1e9 / hbm,
                 "fp64_gpu": {"value": cells / (ms64 / 1e3), "ms_per_step": ms64,
                              "frac": 576 * cells / (ms64 / 1e3) / 1e9 / hbm},
                 "rel_l1_fp32_vs_fp64_gpu": {str(k): v for k, v in errs.items()},
                 "rel_l1_fp32_vs_oracle_step1": err_oracle,
                 "rel_linf_fp64_gpu_vs_oracle_step1": err64_oracle,
                 "norms": "rho, e relative; m and B components against their vector's "
                          "magnitude; psi against c_h |B|"}
    A.close()
    B.close()
    del U64

    # c2: Orszag-Tang at its stated FP64 precision, and in FP32
    res = {}
    for prec in ("fp64", "fp32"):
        W = make_workload("c2", prec)[0]
        cells = W.interior_cells()
        S = amrvac.State.from_workload(W, device=dev, pressure=args.pressure)
        S.set_conserved(W.U if prec == "fp64" else W.U.astype(np.float32))
        S.step(3)
        msp = time_steps(torch, S, 20)
        nbytes = (576 if prec == "fp64" else 288) * cells
        res[prec] = {"value": cells / (msp / 1e3), "ms_per_step": msp,
                     "frac": nbytes / (msp / 1e3) / 1e9 / hbm}
        S.close()
    out["c2"] = {"workload": "2D Orszag-Tang 1024^2 in 16^2 blocks, HLLD+koren+glm, SSPRK3",
                 "cells": 1024 * 1024, "fp64": res["fp64"], "fp32": res["fp32"],
                 "pressure_fp32": args.pressure,
                 "l2": "state smaller than L2 (75.5 MB FP64 per register): frac is not a "
                       "roofline measurement"}
    return out


def bench_regrid(torch, amrvac, W, S, dev, args, hbm, thr=0.05, ratio=0.2):
    """Times one regrid of S's current state (register 0), refining on density
    and pressure (weights 1/2 each).  Algorithmic bytes: the estimator reads
    every conserved variable of a cell once (36 B a cell); the transfer reads
    each source cell it needs once (a split block's cells once for all its
    children) and writes every destination cell (36 B a cell each way)."""
    maxlev = int(W.block_meta[:, 1].max())
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    est_ms = []
    for _ in range(3):
        e0, e1 = ev(), ev()
        e0.record(S.stream)
        _, flags = S.regrid_estimate(thr, ratio, max_level=maxlev,
                                     weights=[0.5, 0, 0, 0, 0.5, 0, 0, 0, 0])
        e1.record(S.stream)
        S.stream.synchronize()
        est_ms.append(e0.elapsed_time(e1))
    # the plan on the device (the product path; wall clock including the flag
    # upload and the new list's download), beside the host plan it equals
    plan_dev = []
    for _ in range(3):
        t0 = time.perf_counter()
        new = S.regrid_plan(flags)
        plan_dev.append((time.perf_counter() - t0) * 1e3)
    plan_ms = float(np.median(plan_dev))
    t0 = time.perf_counter()
    new_host = amrvac.regrid_plan(W.cfg, W.instances, S.meta, flags)
    plan_host_ms = (time.perf_counter() - t0) * 1e3
    assert np.array_equal(new, new_host)
    t0 = time.perf_counter()
    D = amrvac.State(W.cfg, W.instances, new, device=dev, kernel=args.kernel,
                     pressure=args.pressure, stream=S.stream)
    torch.cuda.synchronize(dev)
    create_ms = (time.perf_counter() - t0) * 1e3
    tr_ms = []
    for _ in range(3):
        e0, e1 = ev(), ev()
        e0.record(S.stream)
        S.regrid_transfer(D, 0, 0)
        e1.record(S.stream)
        S.stream.synchronize()
        tr_ms.append(e0.elapsed_time(e1))
    s0 = S.diag()["sums"][0]
    s1 = D.diag()["sums"][0]
    old = {tuple(r) for r in S.meta.tolist()}
    kept = sum(1 for r in new.tolist() if tuple(r) in old)
    nd = W.cfg.ndim
    parents = {(r[0], r[1] - 1, r[2] >> 1, r[3] >> 1, r[4] >> 1) for r in new.tolist()
               if tuple(r) not in old}
    n_split = sum(1 for p in parents if p in old)
    n_merged = sum(1 for r in new.tolist()
                   if tuple(r) not in old and
                   (r[0], r[1] - 1, r[2] >> 1, r[3] >> 1, r[4] >> 1) not in old)
    ncell = W.ncell
    src_cells = (kept + n_split + n_merged * (1 << nd)) * ncell
    dst_cells = len(new) * ncell
    est_s = float(np.median(est_ms)) / 1e3
    tr_s = float(np.median(tr_ms)) / 1e3
    est_bytes = 36 * S.nblocks * ncell
    tr_bytes = 36 * (src_cells + dst_cells)
    scale = np.abs(s0).max()
    D.close()
    return {"refine_threshold": thr, "derefine_ratio": ratio, "max_level": maxlev,
            "weights": "rho 0.5, p 0.5",
            "blocks_before": int(S.nblocks), "blocks_after": int(len(new)),
            "split": int(n_split), "merged_parents": int(n_merged), "kept": int(kept),
            "estimate_ms": est_s * 1e3, "plan_ms": plan_ms, "plan_host_ms": plan_host_ms,
            "state_create_ms": create_ms,
            "transfer_ms": tr_s * 1e3,
            "estimate_gbs": est_bytes / est_s / 1e9, "transfer_gbs": tr_bytes / tr_s / 1e9,
            "transfer_frac": tr_bytes / tr_s / 1e9 / hbm,
            "estimate_alg_bytes": est_bytes, "transfer_alg_bytes": tr_bytes,
            "max_rel_change_of_integrals": float(np.abs(s1 - s0).max() / max(scale, 1e-300)),
            "cells_per_s": dst_cells / (est_s + tr_s)}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    ws, rank, local = dist_env()
    if args.workload == "c5" and ws > 1:
        # every rank refuses an empty shard before any collective
        from paper_2303_03026_gb300 import shard
        shard.check_ranks(args.size or 256, ws)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2303_03026_gb300 import amrvac
    from paper_2303_03026_gb300 import build as libbuild

    W, desc = make_workload(args.workload, "fp32", args.size)
    if args.flux:
        W.cfg.flux = args.flux
    if args.limiter:
        W.cfg.limiter = args.limiter
    desc["scheme"] = "%s + %s + %s, SSPRK3" % (W.cfg.flux.upper(), W.cfg.limiter,
                                               "glm" if W.cfg.glm else "no glm")
    # independent instances shard over the ranks (no exchange at all); a single
    # domain runs as one replica per rank
    sharded = args.workload == "c5" and ws > 1
    cells_all = W.interior_cells() * (1 if sharded else ws)
    if sharded:
        from paper_2303_03026_gb300 import shard
        parts = shard.partition_instances(shard.instance_cells(W), ws)
        W = shard.instance_subset(W, parts[rank])
        desc["shard"] = {"ranks": ws, "instances_per_rank": [len(p) for p in parts]}
    cells = W.interior_cells()
    state_bytes = 9 * 4 * cells
    S = amrvac.State.from_workload(W, device=dev, kernel=args.kernel, pressure=args.pressure)
    U32 = torch.from_numpy(W.U.astype(np.float32)).to(dev)
    S.set_conserved(U32)
    stream = S.stream

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # launch-shape autotuning (untimed set-up; restores the state it times on)
    tuning = None
    if not args.no_tune and args.kernel != "plain":
        tuning = S.autotune(trial_steps=3)

    # warm-up (also captures the step graph)
    S.step(max(args.warmup, 3))
    d = S.diag()
    if d["status"] != 0:
        raise RuntimeError("device error during warm-up: %s" % (d["error"],))

    # timed region: K full steps, device-resident inputs
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = S.launches
    barrier()
    with Clocks(local) as clk:
        ev0.record(stream)
        S.step(args.steps)
        ev1.record(stream)
        barrier()
    launches = S.launches - n0
    clocks = clk.summary()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    ms_step = ms / args.steps
    value = cells_all * args.steps / (ms / 1e3)
    d = S.diag()
    if d["status"] != 0:
        raise RuntimeError("device error in the timed region: %s" % (d["error"],))

    # per-stage kernel timing on the launching stream for the roofline
    stage_ms = []
    for rep in range(3):
        S.cfl_dt()
        row = []
        for k in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S.stage(k)
            e1.record(stream)
            row.append((e0, e1))
        stream.synchronize()
        stage_ms.append([a.elapsed_time(b) for a, b in row])
    stage_ms = np.median(np.array(stage_ms), axis=0)
    passes = [2, 3, 3]
    alg_bytes = [p * 9 * 4 * cells for p in passes]
    hbm, src = peaks()
    achieved = sum(alg_bytes) / (sum(stage_ms) / 1e3) / 1e9
    fused = args.kernel != "plain" and (W.cfg.block_nx[0] == 16)
    digest = libbuild._digest()[:16]
    kdigest = libbuild.kernel_digest()[:16]
    kv = counters_from_profile(args.workload + (str(args.size) if args.size else ""),
                               kdigest) if fused and W.cfg.flux == "hlld" else {}
    tr = float(kv["dram_bytes_per_cell_step"]) if "dram_bytes_per_cell_step" in kv else None
    # issue ceiling beside the HBM bound: one warp instruction per cycle per
    # SM sub-partition (4 per SM) at the SM clock sampled during the timed steps
    issue = None
    if "warp_inst_per_cell_step" in kv:
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 0
        ipc = float(kv["warp_inst_per_cell_step"])
        if mhz:
            peak_i = nsm * 4 * mhz * 1e6
            ach_i = ipc * cells / (sum(stage_ms) / 1e3)
            issue = {"achieved": ach_i, "peak": peak_i, "unit": "warp-instr/s",
                     "frac": ach_i / peak_i, "warp_inst_per_cell_step": ipc,
                     "peak_basis": "%d SMs x 4 issue slots x %.0f MHz (sampled)" % (nsm, mhz)}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm,
                "traffic": tr * cells / 3.0 if tr is not None else None,
                "traffic_unit": "DRAM bytes per stage launch (ncu, mean of the 3 stages)",
                "peak_source": src,
                "kernel": ("k_fused%s (one persistent launch per SSPRK stage, after the "
                           "k_ghost_slabs pre-pass where the mesh has level-change faces; "
                           "stage_ms covers both)" % ("" if W.cfg.ndim == 3 else "2d"))
                if fused else "plain per-block kernels (prim + flux x ndim + update) per stage",
                "issue_ceiling": issue,
                "stage_ms": [float(x) for x in stage_ms],
                "alg_bytes_per_cell_step": 288,
                "alg_bytes_per_launch": [int(b) for b in alg_bytes],
                "frac_of_nominal_7900": achieved / NOMINAL_HBM_GBS}

    # variants on the same workload: other fluxes, time steppers, FP64
    # pressure recovery; algorithmic bytes per cell-update follow the stage
    # registers each scheme reads and writes (state passes x 9 x 4 B)
    passes = {"ssprk2": 5, "ssprk3": 8, "ssprk43": 9, "ssprk54": 16}
    variants = {}
    if not args.no_variants and fused:
        for name, kw in (("hll_vanleer", {"flux": "hll"}), ("tvdlf_vanleer", {"flux": "tvdlf"}),
                         ("hllc_vanleer", {"flux": "hllc"}),
                         ("hlld_ssprk43", {"time": "ssprk43"}),
                         ("hlld_ssprk54", {"time": "ssprk54"}),
                         ("hlld_woodward", {"limiter": "woodward"}),
                         ("hlld_reflux", {"reflux": True}),
                         ("fp64_pressure", {"pressure": "fp64"}),
                         # five-point limiters: three ghost cells (the fused 3D
                         # kernel's 6-plane ring; the plain kernels for contrast)
                         ("hlld_mp5", {"limiter": "mp5"}),
                         ("hlld_wenozp5", {"limiter": "wenozp5"}),
                         ("hlld_mp5_plain", {"limiter": "mp5", "kernel": "plain"}),
                         ("hlld_wenoz5_plain", {"limiter": "wenoz5", "kernel": "plain"}),
                         # reflecting walls on every side (FULL fused kernels)
                         ("hlld_walls", {"bc": (("symmetric", "symmetric"),) * 3}),
                         # fix_small_values after every stage (flag pass + repair)
                         ("hlld_fix_average", {"fix_small_values": "average",
                                               "small_density": 1e-8,
                                               "small_pressure": 1e-8})):
            keys = ("flux", "time", "limiter", "reflux", "bc", "fix_small_values",
                    "small_density", "small_pressure")
            old = {k: getattr(W.cfg, k) for k in keys}
            for k in keys:
                setattr(W.cfg, k, kw.get(k, old[k]))
            Sv = amrvac.State.from_workload(W, device=dev, kernel=kw.get("kernel", args.kernel),
                                            pressure=kw.get("pressure", args.pressure))
            nbytes = passes[W.cfg.time] * 9 * 4
            if W.cfg.fix_small_values != "off":
                nbytes += 3 * (9 * 4 + 1)  # per stage: the state read once, a flag byte
            for k in keys:
                setattr(W.cfg, k, old[k])
            Sv.set_conserved(U32)
            if tuning is not None and kw.get("kernel") != "plain":
                Sv.set_tuning(tuning["ctas_per_sm"], tuning["order"], tuning["dynamic"],
                              tuning["faces"])
            Sv.step(2)
            msv = time_steps(torch, Sv, max(3, min(args.steps, 10)))
            variants[name] = {"value": cells_all / (msv / 1e3), "ms_per_step": msv,
                              "kernel": kw.get("kernel", args.kernel),
                              "alg_bytes_per_cell_step": nbytes,
                              "frac": nbytes * cells / (msv / 1e3) / 1e9 / hbm}
            Sv.close()

    # dynamic regridding of the evolved state: estimator + flags (device),
    # plan (host), new state tables (host + upload), transfer (device)
    regrid = None
    if not args.no_variants and W.cfg.ndim == 3 and len(np.unique(W.block_meta[:, 1])) > 1:
        regrid = bench_regrid(torch, amrvac, W, S, dev, args, hbm)

    # C5 batching: the same instances advanced one at a time
    one_at_a_time = None
    if args.workload == "c5" and not args.no_variants:
        import paper_2303_03026_gb300.workloads as wlm
        states = []
        off = 0
        for q, inst in enumerate(W.instances):
            nb = int((W.block_meta[:, 0] == q).sum())
            meta = W.block_meta[off:off + nb].copy()
            meta[:, 0] = 0
            Sq = amrvac.State(W.cfg, [inst], meta, device=dev, kernel=args.kernel,
                              pressure=args.pressure, stream=stream)
            Sq.set_conserved(U32[:, off:off + nb].contiguous())
            Sq.step(1)
            states.append(Sq)
            off += nb
        stream.synchronize()
        kq = max(2, min(args.steps, 5))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(kq):
            for Sq in states:
                Sq.step(1)
        e1.record(stream)
        stream.synchronize()
        msq = e0.elapsed_time(e1) / kq
        one_at_a_time = {"value": cells / (msq / 1e3), "ms_per_step": msq,
                         "batched_speedup": msq / ms_step, "instances": len(states)}
        for Sq in states:
            Sq.close()

    # the other workloads of the metric (c5 batching, c3 accuracy, c2 FP64)
    configs = None
    if not args.no_configs and args.workload == "c4" and ws == 1:
        configs = bench_configs(torch, amrvac, dev, args, hbm)

    # end to end through the C ABI with host buffers: every step uploads its
    # input from pinned host memory and downloads its result to pinned host
    # memory.  The upload of step n+1's input and the download of step n's
    # result run on their own streams through double-buffered device staging
    # (caller-owned memory, as the boundary intends), overlapping the steps;
    # the state's register 0 is filled from and read into the staging buffers
    # by device-to-device copies on the state's stream (amrvac_set_conserved,
    # amrvac_get_conserved).  Wall-clock time over the whole pipeline,
    # including its fill and drain.
    e2e = None
    if not args.no_e2e:
        n_e2e = max(3, min(args.steps, 8))
        h_in = torch.from_numpy(W.U.astype(np.float32)).pin_memory()
        h_out = [torch.empty_like(h_in).pin_memory() for _ in range(2)]
        d_in = [torch.empty(h_in.shape, dtype=h_in.dtype, device=dev) for _ in range(2)]
        d_out = [torch.empty(h_in.shape, dtype=h_in.dtype, device=dev) for _ in range(2)]
        up, down, main = torch.cuda.Stream(dev), torch.cuda.Stream(dev), S.stream
        evs = {k: [torch.cuda.Event(), torch.cuda.Event()]
               for k in ("landed", "consumed", "ready", "fetched")}

        def pipeline(nsteps):
            for e in evs["consumed"] + evs["fetched"]:
                e.record(main)  # staging initially free
            with torch.cuda.stream(up):
                up.wait_event(evs["consumed"][0])
                d_in[0].copy_(h_in, non_blocking=True)
                evs["landed"][0].record(up)
            for n in range(nsteps):
                i = n % 2
                with torch.cuda.stream(main):
                    main.wait_event(evs["landed"][i])
                    S.set_conserved(d_in[i])            # staging -> register 0
                    evs["consumed"][i].record(main)
                    S.step(1)
                    main.wait_event(evs["fetched"][i])
                    S.get_conserved(0, out=d_out[i])    # register 0 -> staging
                    evs["ready"][i].record(main)
                if n + 1 < nsteps:                      # the next input, during this step
                    j = 1 - i
                    with torch.cuda.stream(up):
                        up.wait_event(evs["consumed"][j])
                        d_in[j].copy_(h_in, non_blocking=True)
                        evs["landed"][j].record(up)
                with torch.cuda.stream(down):           # this result, during the next step
                    down.wait_event(evs["ready"][i])
                    h_out[i].copy_(d_out[i], non_blocking=True)
                    evs["fetched"][i].record(down)
            for st in (up, main, down):
                st.synchronize()

        pipeline(2)  # warm-up
        barrier()
        t0 = time.perf_counter()
        pipeline(n_e2e)
        barrier()
        el = time.perf_counter() - t0
        nbytes = h_in.numel() * 4

        # the host link alone: one upload, one download, then both at once
        def link(do_up, do_down):
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            if do_up:
                with torch.cuda.stream(up):
                    d_in[0].copy_(h_in, non_blocking=True)
            if do_down:
                with torch.cuda.stream(down):
                    h_out[0].copy_(d_out[0], non_blocking=True)
            up.synchronize()
            down.synchronize()
            return time.perf_counter() - t
        link(True, True)
        t_up = min(link(True, False) for _ in range(2))
        t_down = min(link(False, True) for _ in range(2))
        t_both = min(link(True, True) for _ in range(2))
        # per step the link must carry one input and one result; with the copies
        # hidden behind the steps the pipeline is bound by the slower of the
        # two: the step on the device and the link's concurrent transfer
        bound_s = max(ms_step / 1e3, t_both)
        e2e = {"value": cells_all * n_e2e / max_over_ranks(el, dev), "unit": "cell-updates/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "steps": n_e2e,
               "method": "pinned host input uploaded and result downloaded every step on "
                         "their own streams through double-buffered device staging, "
                         "overlapping the steps; wall clock incl. pipeline fill and drain",
               "link": {"h2d_gbs": nbytes / t_up / 1e9, "d2h_gbs": nbytes / t_down / 1e9,
                        "both_gbs": 2 * nbytes / t_both / 1e9,
                        "bound_value": cells_all / bound_s,
                        "frac_of_bound": cells_all * n_e2e / max_over_ranks(el, dev) /
                        (cells_all / bound_s)}}
        del d_in, d_out, h_out

    # plain FP64 per-block path on the same workload, and the FP32 error
    fp64 = None
    if not args.no_fp64:
        import dataclasses
        W64 = dataclasses.replace(W, cfg=dataclasses.replace(W.cfg, precision="fp64"))
        S64 = amrvac.State.from_workload(W64, device=dev, kernel="plain")
        U64 = torch.from_numpy(W.U.astype(np.float32).astype(np.float64)).to(dev)
        S64.set_conserved(U64)
        S64.step(2)
        ms64 = time_steps(torch, S64, max(2, min(args.steps, 5)))
        # accuracy at equal steps from the same state
        S.set_conserved(U32)
        S64.set_conserved(U64)
        nacc = 5
        S.step(nacc)
        S64.step(nacc)
        a = S.get_conserved(0, numpy=False).double()
        b = S64.get_conserved(0, numpy=False)
        ch = float(S64.diag()["ch"].max())
        # rho, e against themselves; m and B components against the magnitude of
        # their vector; psi against c_h |B|
        diff = (a - b).abs().sum(dim=(1, 2))
        del a
        mm = torch.sqrt(b[1] ** 2 + b[2] ** 2 + b[3] ** 2).sum()
        bm = torch.sqrt(b[5] ** 2 + b[6] ** 2 + b[7] ** 2).sum()
        own = b.abs().sum(dim=(1, 2))
        scale = torch.stack([own[0], mm, mm, mm, own[4], bm, bm, bm,
                             torch.maximum(own[8], ch * bm)])
        l1 = (diff / scale.clamp_min(1e-300)).cpu()
        fp64 = {"value": cells_all / (ms64 / 1e3), "ms_per_step": ms64,
                "speedup_fp32_fused_vs_fp64_plain": ms64 / ms_step,
                "rel_l1_fp32_vs_fp64_after_%d_steps" % nacc:
                    {n: float(x) for n, x in zip(("rho", "m_x", "m_y", "m_z", "e", "B_x", "B_y",
                                                  "B_z", "psi"), l1.tolist())}}
        S64.close()
        del U64

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(W)
        # the same oracle on one core (a smaller bounded sample)
        one = cpu_baseline(W, seconds_target=4.0, threads=1)
        cpu["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}

    if rank == 0:
        l2 = ("inputs larger than L2 (%.2f GB per state register)" % (state_bytes / 1e9)
              if state_bytes > 129e6 else
              "inputs smaller than L2 (%.0f MB per register): not a roofline measurement"
              % (state_bytes / 1e6))
        line = {"metric": METRIC, "value": value,
                "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "strong" if sharded else "weak", "vs_baseline": None,
                "dtype": "f32",
                "data": "synthetic",
                "config": dict(desc, cells=cells, l2=l2,
                               precision="fp32 bulk; pressure recovery in %s; fp64 dt, c_h "
                                         "and conservation sums" %
                                         ("float-float" if args.pressure == "ff" else "fp64"),
                               kernel=args.kernel, build=digest, kernel_build=kdigest,
                               tuning=tuning,
                               parallelism=("instances sharded over %d ranks" % ws if sharded
                                            else "replicas" if ws > 1 else "1 GPU")),
                "clocks": clocks, "gpu_launches": launches, "roofline": roofline,
                "e2e": e2e, "variants": variants or None, "regrid": regrid,
                "one_at_a_time": one_at_a_time, "configs": configs,
                "fp64_plain": fp64, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    S.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

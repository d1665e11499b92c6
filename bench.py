#!/usr/bin/env python
"""Throughput of streaming FOA-based DMD on one GB300 per rank.

Workload: u, v, w, p fields on a 256^3 grid (n = 4 * 256^3 = 67,108,864), N = 384 snapshots
stored in FP32 (V is 103 GB), 48 damped travelling waves with amplitudes 1 -> 1e-3 plus 1e-7
relative noise (kappa_2(X) near 1/eps_fp32).  One step is one full streaming run: reset,
384 pushes (Alg. 4 with p = 1, the error indicator evaluated every 16 pushes over the 32
leading modes), then the eigen-decomposition with automatic rank truncation and the DMD modes
Phi for the 32 leading modes (the eigen extraction of Alg. 1).  The snapshots are generated on the device
before timing (103 GB, larger than L2, so no flush is needed between steps).

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead.
With torchrun (N > 1 ranks) every rank runs an independent stream (weak scaling, no
collective on the data path); the reported value is the total over ranks divided by the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "snapshots/s ingested at n=67M,k≤384; HBM GB/s vs peak; eig rel. err vs FP64 oracle"
UNIT = "snapshots/s"
FALLBACK_HBM_GBS = 6800.0
BREAKDOWN_TOL = 1e-12
PASS_NAMES = {1: ("A", "B", "C", "other"), 2: ("A2 (lagged append + first projection)", "B2 (second projection + commit)",
                                            "unused", "other")}
PUSH_FORM = {1: "CGS2, three passes over V per push (pre-vector, CGS2 projections and norm of Alg. 1)",
             2: "CGS2 read as two passes over V per push (h_{j+1,j} by Pythagoras, lagged append)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=256, help="grid points per axis (256 = the full workload)")
    p.add_argument("--snapshots", type=int, default=384)
    p.add_argument("--indicator-every", type=int, default=16)
    p.add_argument("--modes", type=int, default=32)
    p.add_argument("--reorth", type=int, default=1, choices=[1, 2],
                   help="1: CGS2 in three passes over V per push; 2: the two-pass reading (Pythagorean "
                        "h_{j+1,j}, new column appended during the next push's first pass)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="skip the launch-geometry autotuner (untimed setup)")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the secondary lines: the two-pass push on the same workload, the 256 batched "
                        "streams and the FP64/FP32/BF16 storage forms on the 1024^2 waves")
    p.add_argument("--sample-grid", type=int, default=40, help="grid of the CPU-oracle sample")
    p.add_argument("--workload", default="fields", choices=["fields", "batched", "forms", "waves3d", "blocksweep"],
                   help="fields: the 4-field 256^3 stream (default); batched: 256 uneven planted streams; "
                        "forms: storage forms and the kappa sweep; waves3d: the 256^3 single-field waves "
                        "(kappa_t 1e4) through the three-pass push and the block push of 4; blocksweep: the "
                        "three block passes of one block of 4 at a list of basis sizes")
    p.add_argument("--reps", type=int, default=2, help="waves3d: timed repetitions of each push form")
    p.add_argument("--streams", type=int, default=256)
    p.add_argument("--batch-n", type=int, default=0,
                   help="batched: give every stream this length (planted rank 16, noise 1e-5) instead of the "
                        "log-uniform mix; a small case for profiling")
    p.add_argument("--batch-snapshots", type=int, default=0, help="batched with --batch-n: snapshots per stream")
    p.add_argument("--block-n", type=int, default=1 << 24, help="blocksweep: rows")
    p.add_argument("--block-dtype", default="f32", choices=["f32", "bf16"], help="blocksweep: storage type")
    p.add_argument("--block-j", default="32,64,128,192,256,320,384,448,500",
                   help="blocksweep: basis sizes (comma separated) at which one block of 4 is pushed")
    return p.parse_args()


def workload_name(G, N):
    return f"fields4x{G}^3 n={4 * G ** 3} N={N} FP32 storage, CGS2 push (breakdown_tol {BREAKDOWN_TOL:g}), " \
           f"indicator every 16 over 32 leading modes, final eig rank_tol=auto + Phi for 32 leading modes"


# ------------------------------------------------------------------ distributed helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(units_local, seconds_local, group=None):
    """Total units over ranks and the slowest rank's time (max), via torch.distributed if active."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(seconds_local)], dtype=torch.float64, device=dev)
        u = torch.tensor([float(units_local)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
        return float(u.item()), float(t.item())
    return float(units_local), float(seconds_local)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid=None):
        self.proc = None
        self.uuid = gpu_uuid
        # raw samples go to FOA_DMD_CLOCKS_DIR (default: the system temporary directory)
        d = os.environ.get("FOA_DMD_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd.insert(1, f"--id={self.uuid}")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def pass_kernel_hash():
    h = hashlib.sha1()
    for f in ("pass.cuh", "pass_ws.cuh", "pass_fused.cuh", "lag.cuh", "lag_ws.cuh", "lag_fused.cuh", "internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1805_05821_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def traffic_ratio():
    """DRAM bytes per algorithmic byte of the pass kernel from the committed ncu summary, if it was
    taken on the current kernel source (its hash is recorded in the summary)."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_ncu.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    want = pass_kernel_hash()
    ratio, src = None, None
    for line in txt.splitlines():
        if line.startswith("kernel source hash:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("dram bytes per algorithmic byte:"):
            ratio = float(line.split(":", 1)[1].strip())
    return ratio if (ratio is not None and src == want) else None


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(G, N, every, n_modes, full_n, reorth=1, X=None):
    """The FP64 oracle (C push, OpenMP over fixed row blocks; LAPACK eig) on the same generator at
    a smaller grid: the same N pushes, indicator schedule, truncated eig and modes.  The push
    cost is linear in n, so snapshots/s at the full n is the measured rate times n_sample/n."""
    import oracle
    from paper_1805_05821_gb300 import synth
    spec = synth.config5(0, G=G, N=N)
    if X is None:
        X = synth.snapshots(spec, np.float32).astype(np.float64)
    t0 = time.perf_counter()
    o = oracle.FoaOracle(spec.n, N, breakdown_tol=BREAKDOWN_TOL, storage="f32", reorth=reorth)
    for t in range(N):
        st, _, _ = o.push(X[:, t])
        if st != "ok":
            break
        if every and (t + 1) % every == 0 and o.m >= 1:
            r = o.eig(0.0)
            _ = float(np.max(r["indicator"][:32]))
    res = o.eig(oracle.auto_rank_tol("f32", o.m + 1))
    _ = o.modes(res, min(n_modes, res["r"]))
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    rate = N / dt * (spec.n / full_n)
    return {"value": rate, "seconds": dt, "n_sample": spec.n, "cores": cores, "X": X, "spec": spec, "res": res,
            "oracle": o}


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    full_n = 4 * args.grid ** 3
    vals = []
    X = None  # the sample's snapshots are generated once (untimed) and reused by every step
    for i in range(args.warmup + args.steps):
        s = oracle_sample(args.sample_grid, args.snapshots, args.indicator_every, args.modes, full_n, args.reorth, X)
        X = s["X"]
        if i >= args.warmup:
            vals.append(s)
    v = statistics.median([s["value"] for s in vals])
    secs = statistics.median([s["seconds"] for s in vals])
    sample = (f"FP64 C oracle, OpenMP over fixed row blocks, on fields4x{args.sample_grid}^3 (n={vals[0]['n_sample']}), "
              f"N={args.snapshots}, same indicator schedule, truncated eig and modes; rate scaled by n_sample/n")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 * full_n / vals[0]["n_sample"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.grid, args.snapshots)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "forms":
        return run_forms(args)
    if args.workload == "waves3d":
        return run_waves3d(args)
    if args.workload == "blocksweep":
        return run_block_sweep(args)
    world, rank, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1805_05821_gb300 import build, synth
    from paper_1805_05821_gb300 import foa_dmd as F
    build.build()
    G, N = args.grid, args.snapshots
    spec = synth.config5(0, G=G, N=N)
    n = spec.n
    # ---- inputs resident in HBM
    X = torch.empty((N, n), dtype=torch.float32, device="cuda")
    tabs = torch.from_numpy(np.stack(spec.tables).astype(np.float32)).cuda()
    coefs = torch.from_numpy(np.ascontiguousarray(np.transpose(spec.T, (2, 0, 1))).astype(np.float32)).cuda()
    for t in range(N):
        F.foa_synth_waves(X[t], "f32", n, 3, G, 4, spec.M, tabs, coefs[t], spec.noise_scale, spec.seed_noise, t)
    torch.cuda.synchronize()
    opts = F.foa_dmd_opts_default()
    opts.indicator_every = args.indicator_every
    opts.n_lead = 32
    opts.indicator_rank_tol = 0.0
    # The workload's snapshots beyond its 96 wave dimensions differ only by 1e-7 noise (kappa_2 near
    # 1/eps_fp32 on purpose, to exercise rank truncation); the default breakdown test (sqrt(u_fp32))
    # would stop the stream there, so the run keeps every snapshot.
    opts.breakdown_tol = BREAKDOWN_TOL
    opts.reorth = args.reorth
    h = F.foa_dmd_create(n, N, "f32", opts)
    tune_s = None
    if not args.no_tune:  # untimed setup: pick the pass launch geometry per (pass kind, j bucket)
        t0 = time.perf_counter()
        F.foa_dmd_autotune(h)
        tune_s = time.perf_counter() - t0
    ld_phi = (n + 3) // 4 * 4
    nm = args.modes
    phi = torch.empty((2 * nm, ld_phi), dtype=torch.float32, device="cuda")
    L = F.lib()

    def step(src_dev=None, src_host=None):
        F.foa_dmd_reset(h)
        for t in range(N):
            if src_host is not None:
                st = L.foa_dmd_push_host(h, ctypes.c_void_p(src_host + t * n * 4), None)
            else:
                st = L.foa_dmd_push(h, ctypes.c_void_p(src_dev[t].data_ptr()), None)
            if st != 0:
                raise RuntimeError(f"push {t}: {F.STATUS.get(st, st)}")
        return F.foa_dmd_eig(h, -1.0, N, nm, phi, ld_phi, 0)

    for _ in range(args.warmup):
        res = step(X)
        assert res["status"] == 0, res
    F.foa_dmd_profile_read(h)  # clear
    F.foa_dmd_profile(h, True)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clk = ClockSampler(uuid)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        res = step(X)
    F.foa_dmd_indicators(h)  # the last step's indicator eigensolve (side stream) ends inside the timed region
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    F.foa_dmd_profile(h, False)
    stats = F.foa_dmd_profile_read(h)
    secs = e0.elapsed_time(e1) / 1e3
    units, secs_max = aggregate(N * args.steps, secs)
    value = units / secs_max
    # ---- roofline of the dominant kernel (the streaming pass, kinds 0-2)
    pk = [0, 1, 2]
    pass_ms = sum(stats["ms"][k] for k in pk)
    pass_bytes = sum(stats["bytes"][k] for k in pk)
    pass_launches = sum(stats["launches"][k] for k in pk)
    achieved = pass_bytes / (pass_ms / 1e3) / 1e9 if pass_ms > 0 else None
    peak, peak_src = measured_peak()
    ratio = traffic_ratio()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": (ratio * pass_bytes / pass_launches) if (ratio and pass_launches) else None,
            "kernel": ("streaming passes over V: pass_fused_kernel or pass_ws_kernel (A, B) + pass_kernel (C)" if args.reorth == 1 else
                       "streaming passes over V: lag_fused_kernel or lag_ws_kernel (A2) + pass_fused_kernel or pass_ws_kernel (B2)"),
            "algorithmic_bytes_per_launch": pass_bytes / pass_launches if pass_launches else None,
            "avg_launch_ms": pass_ms / pass_launches if pass_launches else None,
            "share_of_step": pass_ms / (secs * 1e3) if secs > 0 else None,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
            "per_pass": {name: {"launches": stats["launches"][k],
                                "avg_ms": stats["ms"][k] / stats["launches"][k],
                                "GBps": stats["bytes"][k] / (stats["ms"][k] / 1e3) / 1e9}
                         for k, name in enumerate(PASS_NAMES[args.reorth]) if stats["launches"][k] and stats["ms"][k] > 0}}
    gpu_launches = stats["total_launches"]
    # planted-truth check of the leading eigenvalues (err against the generating map)
    lam = res["lam"]
    planted = spec.lam
    rel_planted = None
    if len(lam):
        from scipy.optimize import linear_sum_assignment
        lead = lam[:min(32, len(lam))]
        D = np.abs(lead[:, None] - planted[None, :])
        ri, ci = linear_sum_assignment(D)
        rel_planted = float(np.max(D[ri, ci] / np.abs(planted[ci])))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": secs_max * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload_name(G, N), "n": n, "N": N, "l2": "inputs (N x n FP32 snapshots, "
                      f"{N * n * 4 / 1e9:.0f} GB) exceed L2; no flush needed", "parallelism": "independent stream per GPU",
                      "push": PUSH_FORM[args.reorth],
                      "launch_geometry": "autotuned (untimed setup, %.1f s)" % tune_s if tune_s is not None else "default"},
           "roofline": roof, "gpu_launches": gpu_launches, "clocks": clocks,
           "accuracy": {"rank": res["r"], "m": res["m"], "leading32_rel_err_vs_planted": rel_planted}}
    # ---- end to end through the public API with host buffers (pinned), copies in the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, h, X, n, N, F, L, step, world)
        X = None
    out["e2e"] = e2e
    # ---- the other push form on the same workload (its own handle; the headline handle is freed)
    if not args.no_variants and args.reorth == 1:
        F.foa_dmd_destroy(h)
        h = None
        phi = None
        torch.cuda.empty_cache()
        out["variants"] = {"two_pass": run_variant(args, spec, X, n, N, F, L, world, 2)}
    # ---- the batched streams and the storage forms (rank 0 of a one-rank run)
    if not args.no_variants and rank == 0 and world == 1:
        if h is not None:
            F.foa_dmd_destroy(h)
            h = None
        phi = X = tabs = coefs = None  # the 256 streams' bases take 174 GB
        torch.cuda.empty_cache()
        out.setdefault("variants", {})["batched"] = batched_measure(args.streams)
        out["variants"]["forms"] = run_forms_variant(F, torch)
    # ---- CPU oracle baseline (rank 0) and the FP32-vs-FP64 eigenvalue error on that sample
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = oracle_sample(args.sample_grid, N, args.indicator_every, nm, n, args.reorth)
        out["cpu_baseline"] = {"value": s["value"], "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                               "sample": f"FP64 C oracle (OpenMP, fixed row blocks) on fields4x{args.sample_grid}^3 "
                                         f"(n={s['n_sample']}), N={N}, same schedule/eig/modes; "
                                         f"{s['seconds']:.1f} s, rate scaled by n_sample/n"}
        out["accuracy"].update(sample_eig_accuracy(s, F, torch, N, nm, args.reorth))
    if h is not None:
        F.foa_dmd_destroy(h)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_variant(args, spec, X, n, N, F, L, world, reorth, block=0):
    """Secondary line: the same step (reset, N pushes, truncated eig + modes) with another push form
    (block > 0: foa_dmd_push_block of all N snapshots, `block` at a time; the push-time indicator
    schedule does not run there), 3 warm-up and 2 timed steps, CUDA events; the snapshots are
    regenerated on the device if the end-to-end leg has released them."""
    import torch
    G = args.grid
    if X is None:
        X = torch.empty((N, n), dtype=torch.float32, device="cuda")
        tabs = torch.from_numpy(np.stack(spec.tables).astype(np.float32)).cuda()
        coefs = torch.from_numpy(np.ascontiguousarray(np.transpose(spec.T, (2, 0, 1))).astype(np.float32)).cuda()
        for t in range(N):
            F.foa_synth_waves(X[t], "f32", n, 3, G, 4, spec.M, tabs, coefs[t], spec.noise_scale, spec.seed_noise, t)
        torch.cuda.synchronize()
    opts = F.foa_dmd_opts_default()
    opts.indicator_every = args.indicator_every
    opts.n_lead = 32
    opts.breakdown_tol = BREAKDOWN_TOL
    opts.reorth = reorth
    h = F.foa_dmd_create(n, N, "f32", opts)
    try:
        if not args.no_tune:
            F.foa_dmd_autotune(h)
        nm = args.modes
        ld_phi = (n + 3) // 4 * 4
        phi = torch.empty((2 * nm, ld_phi), dtype=torch.float32, device="cuda")

        def step():
            F.foa_dmd_reset(h)
            if block:
                st = L.foa_dmd_push_block(h, ctypes.c_void_p(X.data_ptr()), N, n, block, None)
                if st != 0:
                    raise RuntimeError(f"block push: {F.STATUS.get(st, st)}")
            else:
                for t in range(N):
                    st = L.foa_dmd_push(h, ctypes.c_void_p(X[t].data_ptr()), None)
                    if st != 0:
                        raise RuntimeError(f"push {t}: {F.STATUS.get(st, st)}")
            return F.foa_dmd_eig(h, -1.0, N, nm, phi, ld_phi, 0)

        for _ in range(3):
            step()
        F.foa_dmd_profile_read(h)
        F.foa_dmd_profile(h, True)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = 2
        e0.record()
        for _ in range(k):
            res = step()
        F.foa_dmd_indicators(h)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        F.foa_dmd_profile(h, False)
        stats = F.foa_dmd_profile_read(h)
        secs = e0.elapsed_time(e1) / 1e3
        units, secs_max = aggregate(N * k, secs)
        kinds = (0, 1, 2) if block else (0, 1)
        pass_ms = sum(stats["ms"][k] for k in kinds)
        pass_bytes = sum(stats["bytes"][k] for k in kinds)
        peak, _ = measured_peak()
        achieved = pass_bytes / (pass_ms / 1e3) / 1e9
        lam = res["lam"]
        lead = lam[:min(32, len(lam))]
        from scipy.optimize import linear_sum_assignment
        D = np.abs(lead[:, None] - spec.lam[None, :])
        ri, ci = linear_sum_assignment(D)
        form = (f"block push of {block} snapshots (block CGS2 + Cholesky QR twice; no indicator schedule)"
                if block else PUSH_FORM[reorth])
        note = ("algorithmic bytes of its three block passes (3 n j s of V per block) over their event time" if block
                else "algorithmic bytes of its two passes (2 n j s of V per push) over their event time")
        return {"push": form, "value": units / secs_max, "unit": UNIT, "steps": k, "warmup": 3,
                "ms_per_step": secs_max * 1e3 / k,
                "roofline": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "note": note},
                "leading32_rel_err_vs_planted": float(np.max(D[ri, ci] / np.abs(spec.lam[ci])))}
    finally:
        F.foa_dmd_destroy(h)


def run_forms_variant(F, torch, reps=2):
    """Secondary line for the precision forms: the same snapshots (the 1024^2 waves, n = 2^20,
    N = 200, 20 damped waves, noise 1e-6, kappa_2 about 1.8e6) stored in FP64, FP32 and BF16.
    Per form: snapshots/s of the N pushes alone and of the pushes plus the untruncated eig
    (CUDA events, one warm-up run and `reps` timed runs), and the relative error of the 20 leading
    eigenvalues (the oracle's |c| order, matched one to one) against ONE FP64 oracle run on the
    unrounded FP64 snapshots, so the storage rounding of the inputs counts in each form's error;
    the error against the planted eigenvalues e^{sigma +- i omega} is given beside it."""
    import oracle
    from paper_1805_05821_gb300 import synth
    spec = synth.config2(0)
    n, N = spec.n, spec.N
    X = torch.empty((N, n), dtype=torch.float64, device="cuda")
    tabs = torch.from_numpy(np.stack(spec.tables).astype(np.float64)).cuda()
    for t in range(N):
        coef = torch.from_numpy(np.ascontiguousarray(spec.T[:, :, t]).astype(np.float64)).cuda()
        F.foa_synth_waves(X[t], "f64", n, 2, spec.grid[0], 1, spec.M, tabs, coef, spec.noise_scale,
                          spec.seed_noise, t)
    torch.cuda.synchronize()
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
    forms = {}
    for dt in ("f64", "f32", "bf16"):
        Xc = X.to(tdt[dt]).contiguous()
        g = F.FoaDMD(n, N, dt, breakdown_tol=BREAKDOWN_TOL)
        t_push, t_all = [], []
        for rep in range(reps + 1):
            g.reset()
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            for t in range(N):
                st, _ = g.push(Xc[t], info=False)
                if st != 0:
                    raise RuntimeError(f"forms {dt} push {t}: {F.STATUS.get(st, st)}")
            e1.record()
            res = g.eig(0.0)
            e2.record()
            torch.cuda.synchronize()
            if rep:
                t_push.append(e0.elapsed_time(e1) / 1e3)
                t_all.append(e0.elapsed_time(e2) / 1e3)
        g.close()
        del Xc
        forms[dt] = {"pushes_per_s": N / statistics.median(t_push), "snapshots_per_s_with_eig": N / statistics.median(t_all),
                     "lam": res["lam"], "status": res["status"]}
    Xh = X.cpu().numpy().T
    del X
    o = oracle.FoaOracle(n, N, breakdown_tol=BREAKDOWN_TOL, storage="f64")
    for t in range(N):
        if o.push(np.ascontiguousarray(Xh[:, t]))[0] != "ok":
            break
    ro = o.eig(0.0)
    lead = ro["lam"][:20]
    sv = np.linalg.svd(o.B[:o.q, :o.q], compute_uv=False)
    out = {"workload": f"waves2d 1024^2 n={n} N={N} (20 damped waves, noise 1e-6), kappa_2(X) = {sv[0] / sv[-1]:.3g}",
           "eig": "untruncated (rank_tol 0)", "reps": reps,
           "error": "max relative error of the 20 leading eigenvalues against the FP64 oracle on the FP64 snapshots"}
    for dt, f in forms.items():
        out[dt] = {"pushes_per_s": f["pushes_per_s"], "snapshots_per_s_with_eig": f["snapshots_per_s_with_eig"],
                   "leading20_eig_rel_err_vs_fp64_oracle": _match_rel(lead, f["lam"]),
                   "leading20_eig_rel_err_vs_planted": _match_rel(f["lam"][:20], spec.lam)}
    out["f32_over_f64_snapshots_per_s"] = out["f32"]["snapshots_per_s_with_eig"] / out["f64"]["snapshots_per_s_with_eig"]
    out["bf16_over_f64_snapshots_per_s"] = out["bf16"]["snapshots_per_s_with_eig"] / out["f64"]["snapshots_per_s_with_eig"]
    return out


def sample_eig_accuracy(s, F, torch, N, nm, reorth=1):
    """Relative error of the leading eigenvalues of the FP32 GPU path against the FP64 oracle on the
    same (FP32-rounded) sample inputs."""
    X = s["X"]
    n = X.shape[0]
    Xd = torch.from_numpy(np.ascontiguousarray(X.T).astype(np.float32)).cuda()
    g = F.FoaDMD(n, N, "f32", breakdown_tol=BREAKDOWN_TOL, reorth=reorth)
    for t in range(N):
        st, _ = g.push(Xd[t], info=False)
    res = g.eig(-1.0)
    ro = s["res"]
    lo = ro["lam"][:nm]
    lg = res["lam"]
    from scipy.optimize import linear_sum_assignment
    D = np.abs(lo[:, None] - lg[None, :])
    ri, ci = linear_sum_assignment(D)
    err = float(np.max(D[ri, ci] / np.abs(lo[ri])))
    g.close()
    return {"sample_leading32_eig_rel_err_vs_fp64_oracle": err, "sample_rank_gpu": res["r"], "sample_rank_oracle": ro["r"]}


def batched_measure(streams=256, n_fixed=0, N_fixed=0):
    """The batched streams (config 4): S independent planted streams (n log-uniform in [2^14, 2^22],
    N in [50, 400], rank 8-32, noise 1e-5, FP32) advanced together by foa_dmd_batch_push, one round
    (plan, beta_pre, passes A/B/C over all streams, append) captured once in a CUDA graph and
    replayed per round.  The snapshots of all streams do not fit in HBM next to their bases, so
    each round's snapshots are generated on the device before the round and only the replays are
    timed (CUDA events on the batch's stream).  Algorithmic bytes: the V bytes of the three passes,
    3 n j 4 per push."""
    import torch
    from paper_1805_05821_gb300 import build, synth
    from paper_1805_05821_gb300 import foa_dmd as F
    build.build()
    if n_fixed:
        specs = [synth.planted(n_fixed, N_fixed, 16, seed=1000 + s, noise_rel=1e-5) for s in range(streams)]
    else:
        specs = synth.config4(0, streams=streams)
    S = len(specs)
    stream = torch.cuda.Stream()
    opts = F.foa_dmd_opts_default()
    opts.cuda_stream = stream.cuda_stream
    opts.breakdown_tol = BREAKDOWN_TOL
    b = F.foa_dmd_batch_create([sp.n for sp in specs], [sp.N for sp in specs], "f32", opts)
    bufs = [torch.empty(sp.n, dtype=torch.float32, device="cuda") for sp in specs]
    coefs = [torch.from_numpy(np.ascontiguousarray(sp.T[0].T).astype(np.float32)).cuda() for sp in specs]
    ptrs = torch.zeros(S, dtype=torch.int64, device="cuda")
    hl = torch.zeros(S, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    rounds = max(sp.N for sp in specs)
    total_ms, pushes, bytes_alg = 0.0, 0, 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for r in range(rounds):
        host = []
        with torch.cuda.stream(stream):
            for s, sp in enumerate(specs):
                if r < sp.N:
                    F.foa_synth_gauss(bufs[s], "f32", sp.n, sp.M, sp.seed_modes, sp.mode_scale, coefs[s][r],
                                      sp.noise_scale, sp.seed_noise, r, stream)
                    host.append(int(bufs[s].data_ptr()))
                    pushes += 1
                    bytes_alg += 3.0 * sp.n * r * 4
                else:
                    host.append(0)
            ptrs.copy_(torch.tensor(host, dtype=torch.int64))
            if r == 0:
                with torch.cuda.graph(graph, stream=stream):
                    assert F.foa_dmd_batch_push(b, ptrs, hl) == 0
            e0.record(stream)
            graph.replay()
            e1.record(stream)
        stream.synchronize()
        total_ms += e0.elapsed_time(e1)
    statuses = [F.foa_dmd_batch_get_state(b, s, specs[s].N)[1] for s in range(S)]
    F.foa_dmd_batch_destroy(b)
    del bufs, coefs, graph
    torch.cuda.empty_cache()
    peak, _ = measured_peak()
    achieved = bytes_alg / (total_ms / 1e3) / 1e9
    return {"metric": f"snapshots/s over {S} uneven streams (batched push)", "value": pushes / (total_ms / 1e3),
            "unit": "snapshots/s", "rounds": rounds, "pushes": pushes, "ms_total": total_ms,
            "workload": (f"{S} planted streams, n = {n_fixed}, N = {N_fixed}, rank 16, noise 1e-5, FP32" if n_fixed else
                         f"{S} planted streams, n log-uniform [2^14,2^22], N U[50,400], rank 8-32, noise 1e-5, FP32")
                        + "; one graph replay per round (6 launches: plan, beta_pre, passes A/B/C, append)",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "kernel": "bpass_kernel (passes A, B, C of all streams)",
                         "note": "V bytes of the three passes per push (3 n j 4) over the replay time"},
            "gpu_launches": 6 * rounds,
            "streams_ok": int(sum(1 for st in statuses if st == 0))}


def run_batched(args):
    """Secondary measurement printed on its own (see batched_measure)."""
    line = batched_measure(args.streams, args.batch_n, args.batch_snapshots)
    line.update({"n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                 "config": {"workload": line.pop("workload")}})
    print(json.dumps(line), flush=True)
    return 0


def run_waves3d(args):
    """Secondary measurement: the single-field waves on a G^3 grid (G = --grid, default 256, so
    n = 16,777,216), N = --snapshots (500 when left at the fields default), kappa_t 1e4, FP32,
    snapshots generated on the device.  Times the N pushes of the three-pass CGS2 push and of the
    block push of 4 (foa_dmd_push_block: the first snapshot alone, then blocks of 4) with CUDA
    events, --reps times each after one untimed run of each, and reports the per-pass-kind GB/s of
    the handle's event counters."""
    import ctypes
    import torch
    from paper_1805_05821_gb300 import build, synth
    from paper_1805_05821_gb300 import foa_dmd as F
    build.build()
    G = args.grid
    N = 500 if args.snapshots == 384 else args.snapshots
    spec = synth.config3(0, kappa=1e4, G=G, N=N)
    n = spec.n
    X = torch.empty((N, n), dtype=torch.float32, device="cuda")
    tabs = torch.from_numpy(np.stack(spec.tables).astype(np.float32)).cuda()
    coefs = torch.from_numpy(np.ascontiguousarray(np.transpose(spec.T, (2, 0, 1))).astype(np.float32)).cuda()
    for t in range(N):
        F.foa_synth_waves(X[t], "f32", n, 3, G, 1, spec.M, tabs, coefs[t], spec.noise_scale, spec.seed_noise, t)
    torch.cuda.synchronize()
    L = F.lib()
    opts = F.foa_dmd_opts_default()
    opts.breakdown_tol = 1e-9
    h = F.foa_dmd_create(n, N, "f32", opts)
    if not args.no_tune:
        F.foa_dmd_autotune(h)

    def run(block):
        F.foa_dmd_reset(h)
        if block:
            st = L.foa_dmd_push_block(h, ctypes.c_void_p(X.data_ptr()), N, n, block, None)
        else:
            st = 0
            for t in range(N):
                st = L.foa_dmd_push(h, ctypes.c_void_p(X[t].data_ptr()), None)
                if st:
                    break
        if st:
            raise RuntimeError(f"{'block' if block else 'three-pass'} push: {F.STATUS.get(st, st)}")

    peak, _ = measured_peak()
    out = {"metric": "snapshots/s of the N pushes (waves3d)", "unit": "snapshots/s", "data": "synthetic",
           "dtype": "f32", "higher_is_better": True,
           "config": {"workload": f"waves3d {G}^3 n={n} N={N} M={spec.M} kappa_t=1e4 FP32 (device-generated)",
                      "timing": f"CUDA events over the N pushes, best of {args.reps} after one untimed run"}}
    for label, block in (("three_pass", 0), ("block4", 4)):
        run(block)  # untimed
        best = None
        for _ in range(args.reps):
            F.foa_dmd_profile_read(h)
            F.foa_dmd_profile(h, True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run(block)
            e1.record()
            torch.cuda.synchronize()
            F.foa_dmd_profile(h, False)
            stats = F.foa_dmd_profile_read(h)
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                best = (ms, stats)
        ms, stats = best
        kinds = {}
        for k, name in enumerate(("A", "B", "C", "append/Q")):
            if stats["ms"][k] > 0:
                gbs = stats["bytes"][k] / (stats["ms"][k] / 1e3) / 1e9
                kinds[name] = {"launches": stats["launches"][k], "GBps": gbs, "frac": gbs / peak}
        out[label] = {"value": N / (ms / 1e3), "ms": ms, "q": F.foa_dmd_get_state(h, N)[0], "per_kind": kinds}
    F.foa_dmd_destroy(h)
    out["value"] = out["three_pass"]["value"]
    print(json.dumps(out), flush=True)
    return 0


def run_block_sweep(args):
    """Secondary measurement: the block passes A, B and C (foa_dmd_push_block) of one block of 4
    Gaussian snapshots (seeded, generated on the device) at each basis size j of --block-j, after j
    single pushes, with --block-n rows and --block-dtype storage.  GB/s per pass kind from the
    handle's CUDA-event counters (V once plus the block's vectors), best of two."""
    import ctypes
    import torch
    from paper_1805_05821_gb300 import build
    from paper_1805_05821_gb300 import foa_dmd as F
    build.build()
    n, dt = args.block_n, args.block_dtype
    js = [int(v) for v in args.block_j.split(",")]
    N = max(js) + 4
    gen = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn((N, n), generator=gen, device="cuda", dtype=torch.float32)
    if dt == "bf16":
        X = X.to(torch.bfloat16)
    L = F.lib()
    h = F.foa_dmd_create(n, N, dt, F.foa_dmd_opts_default())
    peak, _ = measured_peak()

    def singles(j):
        F.foa_dmd_reset(h)
        for t in range(j):
            st = L.foa_dmd_push(h, ctypes.c_void_p(X[t].data_ptr()), None)
            if st:
                raise RuntimeError(f"push {t}: {F.STATUS.get(st, st)}")
        torch.cuda.synchronize()

    rows = {}
    for j in js:
        best = None
        for _ in range(2):
            singles(j)
            F.foa_dmd_profile_read(h)
            F.foa_dmd_profile(h, True)
            st = L.foa_dmd_push_block(h, ctypes.c_void_p(X[j].data_ptr()), 4, n, 4, None)
            torch.cuda.synchronize()
            F.foa_dmd_profile(h, False)
            stats = F.foa_dmd_profile_read(h)
            if st:
                raise RuntimeError(f"block push at j={j}: {F.STATUS.get(st, st)}")
            us = sum(stats["ms"][:3]) * 1e3
            if best is None or us < best[0]:
                best = (us, stats)
        stats = best[1]
        rows[j] = {k: {"us": stats["ms"][i] * 1e3, "GBps": stats["bytes"][i] / (stats["ms"][i] / 1e3) / 1e9,
                       "frac": stats["bytes"][i] / (stats["ms"][i] / 1e3) / 1e9 / peak}
                   for i, k in enumerate("ABC")}
    F.foa_dmd_destroy(h)
    out = {"metric": "GB/s of the block passes (one block of 4)", "unit": "GB/s", "data": "synthetic",
           "dtype": dt, "higher_is_better": True, "peak_GBps": peak,
           "config": {"workload": f"blocksweep n={n} Gaussian snapshots, {dt} storage, block of 4 at j in {js}",
                      "timing": "CUDA events of the handle's pass counters, best of 2"},
           "per_j": rows}
    print(json.dumps(out), flush=True)
    return 0


def _match_rel(a, b):
    """max relative distance of an optimal one-to-one matching of eigenvalue sets a -> b"""
    from scipy.optimize import linear_sum_assignment
    D = np.abs(a[:, None] - b[None, :])
    ri, ci = linear_sum_assignment(D)
    return float(np.max(D[ri, ci] / np.maximum(np.abs(a[ri]), 1e-300)))


def run_forms(args):
    """Secondary measurement: the FP64, FP32 and BF16 storage forms (and the two-pass push in FP64
    and FP32) on the 1024^2 waves workload
    (n = 2^20, N = 200, 20 damped waves, noise 1e-6) -- snapshots/s (pushes + eig, CUDA events)
    and the relative error of the 20 leading eigenvalues against the FP64 oracle on the same
    storage-rounded inputs and against the planted eigenvalues; then a kappa sweep of the
    precision forms (waves3d, 64^3 grid, N = 200, 100 undamped waves with amplitudes
    kappa_t^{-(m-1)/99}): normwise H-bar and beta errors against the oracle (the paper's three-pass
    step) in units of u*kappa_2, for the three-pass push, the two-pass push and the QR view."""
    import torch
    import oracle
    from paper_1805_05821_gb300 import build, synth
    from paper_1805_05821_gb300 import foa_dmd as F
    build.build()
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
    u = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8}

    def device_snapshots(spec):
        X = torch.empty((spec.N, spec.n), dtype=torch.float64, device="cuda")
        tabs = torch.from_numpy(np.stack(spec.tables).astype(np.float64)).cuda()
        for t in range(spec.N):
            coef = torch.from_numpy(np.ascontiguousarray(spec.T[:, :, t]).astype(np.float64)).cuda()
            F.foa_synth_waves(X[t], "f64", spec.n, len(spec.grid), spec.grid[0], spec.n_fields, spec.M, tabs, coef,
                              spec.noise_scale, spec.seed_noise, t)
        torch.cuda.synchronize()
        return X

    def run_gpu(Xd, n, N, dt, tol, reorth=1, form=0, block=0):
        g = F.FoaDMD(n, N, dt, breakdown_tol=tol, reorth=reorth, form=form)
        Xc = Xd.to(tdt[dt]).contiguous()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if block:
            st, _ = g.push_block(Xc, block=block, info=False)
            assert st in (0, 5), st  # a block push may stop at a dependent snapshot (reported as q)
        else:
            for t in range(N):
                st, _ = g.push(Xc[t], info=False)
                assert st == 0
        res = g.eig(0.0)
        e1.record()
        torch.cuda.synchronize()
        q, stopped, H, B = g.state()
        g.close()
        return res, q, H, B, e0.elapsed_time(e1) / 1e3, Xc.double().cpu().numpy().T

    out = {"metric": "storage forms: snapshots/s and eigenvalue error vs the FP64 oracle", "unit": "snapshots/s",
           "data": "synthetic", "forms": {}, "kappa_sweep": []}
    spec = synth.config2(0)
    Xd = device_snapshots(spec)
    for dt, ro_ in (("f64", 1), ("f32", 1), ("bf16", 1), ("f64", 2), ("f32", 2)):
        res, q, H, B, secs, Xr = run_gpu(Xd, spec.n, spec.N, dt, 1e-12, ro_)
        # the oracle runs the paper's three-pass CGS2 step in both cases
        o = oracle.FoaOracle(spec.n, spec.N, breakdown_tol=1e-12, storage=dt)
        for t in range(spec.N):
            if o.push(Xr[:, t])[0] != "ok":
                break
        ro = o.eig(0.0)
        m = o.m
        lead_o = ro["lam"][:20]
        entry = {"snapshots_per_s": spec.N / secs, "seconds": secs, "q": q,
                 "leading20_eig_rel_err_vs_fp64_oracle": _match_rel(lead_o, res["lam"]),
                 "leading20_eig_rel_err_vs_planted": _match_rel(res["lam"][:20], spec.lam),
                 "hbar_rel_err_vs_oracle": float(np.linalg.norm(H[:m + 1, :m] - o.H[:m + 1, :m]) /
                                                 np.linalg.norm(o.H[:m + 1, :m])),
                 "beta_rel_err_vs_oracle": float(np.linalg.norm(B[:q, :q] - o.B[:q, :q]) / np.linalg.norm(o.B[:q, :q]))}
        sv = np.linalg.svd(o.B[:q, :q], compute_uv=False)
        entry["kappa2"] = float(sv[0] / sv[-1])
        out["forms"][dt if ro_ == 1 else dt + "_two_pass"] = entry
    del Xd
    for kap in (1e2, 1e4, 1e6, 1e8):
        sp = synth.waves(64, 3, 1, 200, 100, 1, sigma=None, omega=np.pi * (np.arange(1, 101) - 0.5) / 100,
                         amp=kap ** (-np.arange(100) / 99.0), kmax=31, name=f"waves3d 64^3 kappa_t={kap:g}")
        Xd = device_snapshots(sp)
        for dt, ro_, fm, bk in (("f32", 1, 0, 0), ("bf16", 1, 0, 0), ("f32", 2, 0, 0), ("bf16", 2, 0, 0),
                                ("f32", 1, 1, 0), ("bf16", 1, 1, 0), ("f32", 1, 0, 4)):
            res, q, H, B, secs, Xr = run_gpu(Xd, sp.n, sp.N, dt, 1e-12, ro_, fm, bk)
            o = oracle.FoaOracle(sp.n, sp.N, breakdown_tol=1e-12, storage=dt)
            for t in range(sp.N):
                if o.push(Xr[:, t])[0] != "ok":
                    break
            m = o.m
            sv = np.linalg.svd(o.B[:o.q, :o.q], compute_uv=False)
            k2 = float(sv[0] / sv[-1])
            eh = float(np.linalg.norm(H[:m + 1, :m] - o.H[:m + 1, :m]) / np.linalg.norm(o.H[:m + 1, :m]))
            eb = float(np.linalg.norm(B[:o.q, :o.q] - o.B[:o.q, :o.q]) / np.linalg.norm(o.B[:o.q, :o.q]))
            out["kappa_sweep"].append({"kappa_t": kap, "dtype": dt,
                                       "push": "block4" if bk else ("qr_view" if fm else
                                                                    ("two_pass" if ro_ == 2 else "three_pass")),
                                       "kappa2": k2, "q": q, "hbar_rel_err": eh,
                                       "beta_rel_err": eb, "hbar_err_over_u_kappa": eh / (u[dt] * k2),
                                       "leading20_eig_rel_err_vs_planted": _match_rel(res["lam"][:20], sp.lam),
                                       "snapshots_per_s": sp.N / secs})
        del Xd
    print(json.dumps(out), flush=True)
    return 0


def mem_available_bytes():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except Exception:
        pass
    return 0


def run_e2e(args, h, X, n, N, F, L, step, world):
    import torch
    nbytes = N * n * 4
    if mem_available_bytes() < nbytes + 40 * 2 ** 30:
        return {"value": None, "unit": UNIT, "skipped": "not enough host memory for pinned snapshots"}
    ptr = F.foa_dmd_host_alloc(nbytes)
    try:
        host = np.ctypeslib.as_array(ctypes.cast(ctypes.c_void_p(ptr), ctypes.POINTER(ctypes.c_float)), shape=(N, n))
        ht = torch.from_numpy(host)
        for t in range(N):
            ht[t].copy_(X[t])
        torch.cuda.synchronize()
        del X
        torch.cuda.empty_cache()
        step(src_host=ptr)  # warm-up
        k = max(1, min(args.steps, 3))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(k):
            res = step(src_host=ptr)
            d2h += 6 * 8 * res["r"]
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        barrier()
        units, secs_max = aggregate(N * k, secs)
        return {"value": units / secs_max, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": d2h // k,
                "steps": k, "api": "foa_dmd_push_host (pinned host snapshot, copy overlapped) + foa_dmd_eig"}
    finally:
        F.foa_dmd_host_free(ptr)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Throughput of the MacCormack-TVD step (cell-updates/s) on GB300.

Workload: 2D compressible convection, aspect ratio 4, 4096 x 1024 nodes,
Ra = 1e10, Pr = 1, gamma = 5/3, eps = 0.1, D = 0.5, seeded isobaric
temperature perturbation of amplitude 1e-3 (synthetic input).  FP32 state
with FP64 dt and reductions is the timed line; an FP64-state run is reported
beside it.  A step is one full time step of the scheme (z, x, z, x sweeps)
over the whole grid; one cell-update is one node advanced by one step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank advances its own independent replica (the method
has no exchange between independent boxes); timing is the max over ranks and
the value counts the cells of all ranks.  L2 is flushed (256 MiB memset)
before every timed step; durations come from CUDA events on the solver's
stream.
"""
from __future__ import annotations

import argparse
import contextlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NZ, RA, PR, GAMMA = 4096, 1024, 1e10, 1.0, 5.0 / 3.0
RA3 = 1e9  # the 512 x 512 x 128 box
ZSTRETCH = 2.0  # tanh z-grid of the stretched leg (first spacing 0.147 of the uniform one)
# tanh z-grid of the stretched batch: beta = 2 would put the nz = 254, Ra = 1.5e5 box at an explicit
# diffusion number of 1.36 (cm_batch_init rejects it); beta = 1 (the paper's plate refinement) gives 0.37
BATCH_ZSTRETCH = 1.0
WORKLOAD = "2d_aspect4_4096x1024_Ra1e10"
METRIC = "cell-updates/s per MacCormack-TVD step"
UNIT = "cell-updates/s"
FLUSH_BYTES = 256 << 20
# FP64 flops of one 2D sweep per interior node: add, sub, mul, div and sqrt as
# the formulas of Secs. 2 and 3.1 evaluate them (23 divisions and one square
# root each), counted on the restatement of the step by tests/test_flop_count.py;
# FP64_FLOPS drops the 8 subtractions of the two TVD differences per interface
# that repeat a neighbouring interface's
FP64_FLOPS_FORMULA = {"z": 185, "x": 179}
FP64_FLOPS = {"z": 177, "x": 171}
# FP64 peak of GB300: 152 SMs x 2 FP64 FMA per SM per clock x 2 flops x 2.07 GHz
# (the nominal 1.25 TFLOP/s; derived from unit counts and the maximum clock, not measured)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None  # (start, end) host wall-clock of the timed region

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, line in self.lines:
            if self.window and not (self.window[0] <= t <= self.window[1]):
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, steps: int, max_ms: float, world: int) -> float:
    """Whole-job throughput: the units every rank advanced, over the slowest rank's time."""
    return world * units_per_rank * steps / (max_ms * 1e-3)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2411_10372_gb300 as cm

    stream = torch.cuda.Stream()
    hbm, peak_kind = peaks()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_ms(x: float) -> float:
        return max_over_ranks(x, world, "cuda")

    NXr, NZr = args.nx, args.nz
    cells = NXr * NZr

    def measure(precision: str, K: int, W: int, clocks: bool, zstretch: float = 0.0):
        # the workload samples the diagnostics every 100 steps (FP64 sums of Nu, Re, KE, budgets)
        s = cm.Solver(NXr, NZr, RA, PR, GAMMA, precision=precision, stream=stream, seed=12345 + rank,
                      diag_every=100, diag_capacity=4096, zstretch=zstretch)
        s.step(W)
        s.sync()
        barrier()
        s.diagnostics()  # drain the warm-up's records
        launches0 = cm.cm_launch_count()
        clk = Clocks(local)
        # the value: events only at step boundaries, so the sweeps of a step
        # overlap their launches exactly as in cm_step
        if clocks:
            with clk:
                time.sleep(0.5)  # let nvidia-smi start; only samples inside the window count
                t_start = time.time()
                _, step_ms = cm.cm_profile_steps(K, FLUSH_BYTES, per_sweep=False)
                clk.window = (t_start, time.time())
        else:
            _, step_ms = cm.cm_profile_steps(K, FLUSH_BYTES, per_sweep=False)
        barrier()
        launches = cm.cm_launch_count() - launches0
        s.sync()
        ds = s.diagnostics()  # the records taken inside the timed steps
        total_ms = max_ms(sum(step_ms))
        seg = cm.cm_tuning()
        # per-kernel durations for the roofline: a second timed pass with an
        # event pair around every sweep (each duration includes its launch gap)
        sweep_ms, _ = cm.cm_profile_steps(max(3, min(K, 500)), FLUSH_BYTES, per_sweep=True)
        diag = {"samples_in_timed_steps": len(ds), "all_finite": all(d["status"] == 0 for d in ds),
                "last_Nu_bar": ds[-1]["Nu_bar"] if ds else None}
        out = dict(total_ms=total_ms, sweep_ms=sweep_ms, launches=launches, clocks=clk.summary() if clocks else None,
                   w=8 if precision == "fp64" else 4, segments={"z": seg[0], "x": seg[1]}, diag=diag)
        return s, out

    # ---- FP32 state: the timed line ----
    s, r32 = measure("fp32", args.steps, args.warmup, clocks=not args.only_fp32)
    if args.only_fp32:  # profiling runs: the timed FP32 steps and nothing else
        s.close()
        if rank == 0:
            print(json.dumps({"nx": NXr, "nz": NZr, "steps": args.steps, "sweep_ms": r32["sweep_ms"],
                              "ms_per_step": r32["total_ms"] / args.steps}), flush=True)
        return
    # end to end through the public C ABI with host buffers: every step
    # uploads the state from pinned host memory (dense float64), steps once
    # and reads one diagnostics sample back
    # (float32 host buffers, the state's own precision; the float64 entry
    # point is timed beside it)
    host = torch.empty((4, NZr, NXr), dtype=torch.float64, pin_memory=True)
    hostnp = host.numpy()
    cm.cm_get_state(hostnp)
    host32 = torch.empty((4, NZr, NXr), dtype=torch.float32, pin_memory=True)
    host32np = host32.numpy()
    host32np[...] = hostnp
    n_e2e = max(3, min(args.steps, 30))
    cm.cm_run_host_f32(host32np, 1, None, True)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        cm.cm_run_host_f32(host32np, 1, None, True)
    e2e_s = max_ms(time.perf_counter() - t0)
    cm.cm_run_host(hostnp, 1, None, True)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        cm.cm_run_host(hostnp, 1, None, True)
    e2e64_s = max_ms(time.perf_counter() - t0)
    # extended diagnostics of the stepped state (force terms, C(Ra), boundary
    # layers, K_e/I_e histogram): one blocking call, host wall clock
    s.extended(96, -14.0, 0.0)
    t0 = time.perf_counter()
    n_ext = 5
    for _ in range(n_ext):
        ext_vals, ext_hist = s.extended(96, -14.0, 0.0)
    ext_ms = (time.perf_counter() - t0) * 1e3 / n_ext
    ext_bytes = 4 * 4 * cells  # one read of the FP32 state (neighbours from L1/L2)
    extended = {"ms_per_call": round(ext_ms, 4), "state_bytes": ext_bytes,
                "GB_per_s_of_state": round(ext_bytes / (ext_ms * 1e-3) / 1e9, 1),
                "values": {k: ext_vals[k] for k in ("C", "lambda_b", "lambda_top", "F_n", "F_p", "F_b", "F_v", "r_max")},
                "hist_nodes": int(ext_hist.sum()), "timing": "host wall clock around cm_extended (launch, copies, host sums)"}
    s.close()

    # ---- batched ensemble: 64 independent boxes, N_z = round(32 * 8^u), N_x = 4 N_z,
    # Ra = 10^(5 + 4 u'), u, u' uniform in [0, 1) from a seeded generator ----
    batch = None
    if not args.no_batch:
        import numpy as np
        rng = np.random.default_rng(2024 + rank)
        u, u2 = rng.random(64), rng.random(64)
        nzs = [int(round(32 * 8 ** x)) for x in u]
        ras = [10 ** (5 + 4 * x) for x in u2]
        p = cm.cm_default_params()
        p.precision = cm.CM_FP32
        p.stream = stream.cuda_stream
        kb = args.batch_steps

        def run_batch(beta):
            cm.cm_batch_init([cm.cm_grid(2, 4 * nz, 1, nz, 4.0, beta) for nz in nzs], ras, PR, GAMMA, p)
            cm.cm_batch_step(50)
            barrier()
            l0 = cm.cm_batch_launch_count()
            ms = max_ms(cm.cm_batch_profile_steps(kb, FLUSH_BYTES))
            nl = cm.cm_batch_launch_count() - l0
            tuning = cm.cm_batch_tuning()
            diags = cm.cm_batch_diagnostics()
            cm.cm_batch_finalize()
            return ms, nl, tuning, diags

        ms, nl, (seg_z, seg_x), diags = run_batch(0.0)
        cells_b = sum(4 * nz * nz for nz in nzs)
        per_sweep_ms = ms / kb / 4.0
        ach_b = 2 * 4 * 4 * cells_b / (per_sweep_ms * 1e-3) / 1e9
        batch = {"value": job_rate(cells_b, kb, ms, world), "unit": UNIT, "steps": kb, "boxes": 64,
                 "roofline": {"bound": "hbm", "achieved": round(ach_b, 1), "peak": hbm, "unit": "GB/s",
                              "frac": round(ach_b / hbm, 4), "traffic": None,
                              "note": "mean over the 4 sweeps of a step; the 67 MB ensemble stays in L2"},
                 "cells": cells_b, "ms_per_step": ms / kb, "gpu_launches": nl,
                 "all_finite": all(d["status"] == 0 for d in diags),
                 "segments_z": sorted(set(seg_z)), "segments_x": sorted(set(seg_x)),
                 "l2": "flushed once before the timed steps (the steps replay captured 50-step graphs)"}
        if not args.no_stretched:
            # the same ensemble with every box on the tanh z-grid of beta = BATCH_ZSTRETCH
            ms_s, nl_s, _, diags_s = run_batch(BATCH_ZSTRETCH)
            batch["stretched"] = {"zstretch": BATCH_ZSTRETCH, "value": job_rate(cells_b, kb, ms_s, world),
                                  "ms_per_step": ms_s / kb, "gpu_launches": nl_s, "vs_uniform": round(ms / ms_s, 4),
                                  "all_finite": all(d["status"] == 0 for d in diags_s)}

    # ---- 3D box: 512 x 512 x 128 nodes, aspect 4 x 4 x 1, FP32, same Ra ----
    box3 = None
    if not args.no_3d:
        n3 = (512, 512, 128)
        s3 = cm.Solver(n3[0], n3[2], RA3, PR, GAMMA, ny=n3[1], ndim=3, precision="fp32", stream=stream,
                       seed=777 + rank)
        s3.step(min(args.warmup, 5))
        s3.sync()
        barrier()
        l3 = cm.cm_launch_count()
        k3 = args.steps_3d
        sw3, st3 = cm.cm_profile_steps(k3, FLUSH_BYTES)
        barrier()
        nl3 = cm.cm_launch_count() - l3
        d3 = s3.sample()
        s3.close()
        ms3 = max_ms(sum(st3))
        cells3 = n3[0] * n3[1] * n3[2]
        kinds3 = {"sweep3d_march_z": sw3[0] + sw3[3], "sweep3d_march_y": sw3[1] + sw3[4],
                  "sweep3d_x": sw3[2] + sw3[5]}
        bytes3 = 2 * 5 * 4 * cells3
        box3 = {"value": job_rate(cells3, k3, ms3, world), "unit": UNIT, "steps": k3,
                "workload": "3d_aspect4x4_512x512x128_Ra1e9_fp32", "ms_per_step": ms3 / k3,
                "sweep_ms": [round(x, 5) for x in sw3], "gpu_launches": nl3, "finite": d3["status"] == 0,
                "roofline": {k: {"bound": "hbm", "achieved": round(bytes3 / (v / 2 * 1e-3) / 1e9, 1), "peak": hbm,
                                 "unit": "GB/s", "frac": round(bytes3 / (v / 2 * 1e-3) / 1e9 / hbm, 4)}
                             for k, v in kinds3.items()},
                "l2": "flushed before every timed step (256 MiB memset)"}
        if not args.no_stretched:
            # the same box on the tanh z-grid (stretched kernels)
            s3 = cm.Solver(n3[0], n3[2], RA3, PR, GAMMA, ny=n3[1], ndim=3, precision="fp32", stream=stream,
                           seed=777 + rank, zstretch=ZSTRETCH)
            s3.step(min(args.warmup, 5))
            s3.sync()
            barrier()
            l3 = cm.cm_launch_count()
            k3s = max(3, args.steps_3d // 2)
            sw3s, st3s = cm.cm_profile_steps(k3s, FLUSH_BYTES)
            barrier()
            nl3s = cm.cm_launch_count() - l3
            d3s = s3.sample()
            s3.close()
            ms3s = max_ms(sum(st3s))
            box3["stretched"] = {"value": job_rate(cells3, k3s, ms3s, world), "unit": UNIT, "steps": k3s,
                                 "zstretch": ZSTRETCH, "ms_per_step": ms3s / k3s, "gpu_launches": nl3s,
                                 "finite": d3s["status"] == 0, "sweep_ms": [round(x, 5) for x in sw3s]}

    # ---- adjoint: 1024 x 256, Ra = 1e8, FP64, 2000 steps, checkpoints every
    # 100, J = mean Nu_bar over steps 1501..2000, from the conduction profile
    # plus a seeded uniform temperature perturbation of amplitude 1e-3 (the
    # initial condition of cm_init on a numpy-seeded field, cm_set_temperature).
    # Cost of the reverse pass (recompute + vector-Jacobian products) over that
    # of the plain forward; the gradient of the frozen-limiter reading checked
    # against central differences of J on the same dts; the exact reading's
    # gradient norm beside it ----
    adjoint = None
    if not args.no_adjoint:
        import numpy as np
        na, ka, wa = args.adjoint_steps, max(1, args.adjoint_steps // 20), args.adjoint_steps * 3 // 4 + 1
        NXa, NZa, RAa = 1024, 256, 1e8
        rng = np.random.default_rng(99 + rank)
        za = np.linspace(0.0, 1.0, NZa)[:, None]
        T0 = np.repeat(1.0 - 0.6 * za, NXa, axis=1)  # T_c(z) between the plate temperatures 1 and 1 - eps - D
        T0[1:-1] += 1e-3 * rng.uniform(-1.0, 1.0, (NZa - 2, NXa))
        v = np.zeros((NZa, NXa))
        v[1:-1] = rng.uniform(-1.0, 1.0, (NZa - 2, NXa))

        def adj_solver(limiter=cm.CM_ADJ_PHI_FROZEN):
            s_ = cm.Solver(NXa, NZa, RAa, PR, GAMMA, precision="fp64", stream=stream, adj_limiter=limiter)
            cm.cm_set_temperature(T0)
            return s_

        sa = adj_solver()
        sa.step(1)  # warm-up of the kernels
        cm.cm_set_temperature(T0)
        sa.sync()
        t0 = time.perf_counter()
        sa.step(na)
        sa.sync()
        t_fwd = time.perf_counter() - t0
        sa.close()
        sa = adj_solver()
        l0 = cm.cm_launch_count()
        t0 = time.perf_counter()
        Ja = cm.cm_adj_forward(na, ka, wa)
        t_afwd = time.perf_counter() - t0
        gT = np.empty((NZa, NXa))
        t0 = time.perf_counter()
        gRa = cm.cm_adj_backward(None, gT)
        t_bwd = time.perf_counter() - t0
        nla = cm.cm_launch_count() - l0
        dts = cm.cm_adj_get_dts(na)
        sa.close()
        ad = float(np.sum(gT * v))
        # central differences of J along v on the replayed dts (untimed)
        h = 1e-4
        Js = []
        for sg in (1.0, -1.0):
            sa = cm.Solver(NXa, NZa, RAa, PR, GAMMA, precision="fp64", stream=stream)
            cm.cm_set_temperature(T0 + sg * h * v)
            cm.cm_adj_set_dts(dts)
            Js.append(cm.cm_adj_forward(na, na, wa))
            sa.close()
        fd = (Js[0] - Js[1]) / (2 * h)
        sa = adj_solver(cm.CM_ADJ_PHI_EXACT)
        cm.cm_adj_forward(na, ka, wa)
        gTe = np.empty((NZa, NXa))
        gRa_e = cm.cm_adj_backward(None, gTe)
        sa.close()
        adjoint = {"workload": "2d_aspect4_1024x256_Ra1e8_fp64_adjoint", "steps": na, "K": ka, "window": [wa, na],
                   "J": Ja, "reading": "frozen limiter (phi' = 0)", "dJ_dRa": gRa,
                   "grad_T0_norm": float(np.linalg.norm(gT)),
                   "fd_check": {"direction": "uniform random interior temperature field (seed 99)", "step": h,
                                "adjoint": ad, "central_difference": fd, "rel_diff": abs(fd - ad) / abs(ad),
                                "window_checked": [wa, na]},
                   "exact_reading": {"grad_T0_norm": float(np.linalg.norm(gTe)), "dJ_dRa": gRa_e,
                                     "note": "phi' = 2 on 0 < 2r < 1: agrees with finite differences to 200 steps, "
                                             "grows without bound beyond (non-Lipschitz vector limiter)"},
                   "forward_s": t_fwd, "adj_forward_s": t_afwd, "backward_s": t_bwd,
                   "ratio_backward_over_forward": t_bwd / t_fwd, "gpu_launches": nla,
                   "timing": "host wall clock around blocking calls"}

    # ---- FP64 state, same workload ----
    k64 = max(3, min(args.steps, 20))
    s64, r64 = measure("fp64", k64, min(args.warmup, 3), clocks=False)
    s64.close()

    # ---- the same FP32 workload on the tanh z-grid of Sec. 3 (stretched kernels) ----
    stretched = None
    if not args.no_stretched:
        kst = max(3, min(args.steps, 1000))
        sst, rst = measure("fp32", kst, args.warmup, clocks=False, zstretch=ZSTRETCH)
        zs = sst.z
        sst.close()
        stretched = {"value": job_rate(cells, kst, rst["total_ms"], world), "unit": UNIT, "steps": kst,
                     "workload": WORKLOAD + f"_tanh{ZSTRETCH:g}_fp32", "zstretch": ZSTRETCH,
                     "dz_min_over_uniform": float(min(zs[1:] - zs[:-1]) * (NZr - 1)),
                     "ms_per_step": rst["total_ms"] / kst, "gpu_launches": rst["launches"],
                     "segment_rows": rst["segments"], "diagnostics": rst["diag"],
                     "sweep_ms": [round(x, 5) for x in rst["sweep_ms"]]}

    def measured_traffic(kernel: str, segments: dict):
        """DRAM bytes per launch of `kernel` from the committed ncu capture, if
        its kernel sources and segment lengths are unchanged since (else None)."""
        import hashlib
        path = os.path.join(ROOT, "profiles", "sweep2d_fp32_x2_4096x1024_traffic.json")
        if (NXr, NZr) != (NX, NZ) or not os.path.exists(path):
            return None
        rec = json.load(open(path))
        if rec.get("segment_rows") != segments:
            return None
        for name, digest in rec["source_sha256"].items():
            src = os.path.join(ROOT, "paper_2411_10372_gb300", "csrc", name)
            if hashlib.sha256(open(src, "rb").read()).hexdigest() != digest:
                return None
        # the two x sweeps of a step are two kernels (without and with the
        # next dt): the timed duration is their mean, and so is the traffic
        names = [kernel, kernel + "_dt"] if kernel + "_dt" in rec["per_launch_bytes"] else [kernel]
        got = [rec["per_launch_bytes"][n]["total"] for n in names if n in rec["per_launch_bytes"]]
        return int(sum(got) / len(got)) if got else None

    def roofline(r, suffix=None):
        nf, w = 4, r["w"]
        suffix = suffix or ("_x2" if w == 4 else "<double>")
        kinds = {"sweep_z2d" + suffix: r["sweep_ms"][0] + r["sweep_ms"][2],
                 "sweep_x2d" + suffix: r["sweep_ms"][1] + r["sweep_ms"][3]}
        dom = max(kinds, key=kinds.get)
        per_launch_ms = kinds[dom] / 2.0
        bytes_per_launch = 2 * nf * w * cells
        achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
        kernels = [dom, dom + "_dt"] if dom.startswith("sweep_x2d") and suffix.startswith("_x2") else [dom]
        return {"kernel": dom, "launches_averaged": kernels, "bound": "hbm", "achieved": round(achieved, 1),
                "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                "traffic": measured_traffic(dom, r["segments"]) if w == 4 and suffix == "_x2" else None,
                "bytes_per_launch": bytes_per_launch, "ms_per_launch": round(per_launch_ms, 5)}

    def roofline_fp64_alu(r):
        """FP64 leg against the FP64 ALU peak: the method's flops (FP64_FLOPS per
        interior node of each sweep) over the dominant sweep kind's launch time."""
        interior = NXr * (NZr - 2)
        kinds = {"z": (r["sweep_ms"][0] + r["sweep_ms"][2]) / 2.0, "x": (r["sweep_ms"][1] + r["sweep_ms"][3]) / 2.0}
        dom = max(kinds, key=kinds.get)
        tflops = {d: FP64_FLOPS[d] * interior / (ms * 1e-3) / 1e12 for d, ms in kinds.items()}
        step_tflops = sum(2 * FP64_FLOPS[d] for d in kinds) * interior / (sum(r["sweep_ms"]) * 1e-3) / 1e12
        return {"kernel": "sweep_" + dom + "2d<double>", "bound": "alu", "achieved": round(tflops[dom], 4),
                "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s", "frac": round(tflops[dom] / FP64_PEAK_TFLOPS, 4),
                "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flops x 2.07 GHz (nominal 1.25 TFLOP/s), not measured",
                "flops_per_node": dict(FP64_FLOPS), "per_kind_tflops": {d: round(v, 4) for d, v in tflops.items()},
                "step_frac": round(step_tflops / FP64_PEAK_TFLOPS, 4), "traffic": None}

    K = args.steps
    value = job_rate(cells, K, r32["total_ms"], world)
    value64 = job_rate(cells, k64, r64["total_ms"], world)
    e2e_value = job_rate(cells, n_e2e, e2e_s * 1e3, world)
    e2e64_value = job_rate(cells, n_e2e, e2e64_s * 1e3, world)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": r32["total_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + "_fp32", "nx": NXr, "nz": NZr, "Ra": RA, "Pr": PR, "gamma": GAMMA,
                   "eps": 0.1, "D": 0.5, "cfl": 0.5, "state": "fp32, fp64 dt and reductions",
                   "diagnostics": f"FP64 record every 100 steps ({r32['diag']['samples_in_timed_steps']} "
                                  f"of them inside the {K} timed steps)",
                   "l2": "flushed before every timed step (256 MiB memset)", "parallelism": f"replicas x{world}",
                   "timing": "events at step boundaries for value; per-sweep events in a second pass for roofline"},
        "roofline": roofline(r32),
        "sweep_ms": [round(x, 5) for x in r32["sweep_ms"]],
        "segment_rows": r32["segments"],
        "diagnostics": r32["diag"],
        "gpu_launches": r32["launches"],
        "clocks": r32["clocks"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * cells * 4,
                "d2h_bytes_per_step": 128, "steps": n_e2e, "api": "cm_run_host_f32, pinned float32 host state",
                "float64_host": {"value": e2e64_value, "h2d_bytes_per_step": 4 * cells * 8, "api": "cm_run_host"}},
        "batch": batch,
        "box3d": box3,
        "adjoint": adjoint,
        "fp64": {"value": value64, "unit": UNIT, "ms_per_step": r64["total_ms"] / k64, "steps": k64,
                 "sweep_ms": [round(x, 5) for x in r64["sweep_ms"]], "gpu_launches": r64["launches"],
                 "roofline": roofline_fp64_alu(r64), "roofline_hbm": roofline(r64)},
        "stretched": stretched,
        "extended": extended,
    }
    if stretched is not None:
        stretched["roofline"] = roofline(rst, "_x2s")
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(steps=args.cpu_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def host_cpu() -> dict:
    """Model name and online core count of the host CPU."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"model": model, "nproc": os.cpu_count()}


def cpu_baseline(steps: int, nx: int = NX):
    """The FP64 oracle as it stands on a bounded sample of the workload:
    `steps` full steps of the nx x 1024 grid from the seeded state, first on
    one thread, then the same source built with OpenMP on all host cores
    (bit-identical states; its per-node sweep loops split over the cores)."""
    import oracle as O
    cfg = O.Config(nx=nx, nz=NZ, Ra=RA, Pr=PR, gamma=GAMMA)
    X = O.init(cfg)
    t0 = time.perf_counter()
    O.step(cfg, X, steps)
    dt = time.perf_counter() - t0
    cpu = host_cpu()
    line = {"value": nx * NZ * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu,
            "sample": f"{steps} FP64 steps of the {nx}x{NZ} grid, single thread, {dt:.1f} s"}
    path = O.build_omp()
    if path is not None:
        with O.library(path):
            O.step(cfg, X, 1)  # thread pool start-up
            t0 = time.perf_counter()
            O.step(cfg, X, steps)
            dto = time.perf_counter() - t0
        line["all_cores"] = {"value": nx * NZ * steps / dto, "unit": UNIT, "cores": cpu["nproc"],
                             "sample": f"{steps} FP64 steps of the {nx}x{NZ} grid, OpenMP build, {dto:.1f} s"}
    return line


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, timed as it stands on the
    host cores, on this workload; each step is a bounded sample (all nz rows,
    nx columns sized so the whole run stays within a few minutes)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    # one full-width step costs ~0.55 us per node on one core: size nx
    budget_s = 150.0
    est_node_s = 0.6e-6
    nx = NX
    while nx > 32 and (args.steps + args.warmup) * nx * NZ * est_node_s > budget_s:
        nx //= 2
    cfg = O.Config(nx=nx, nz=NZ, Ra=RA, Pr=PR, gamma=GAMMA)
    X = O.init(cfg)
    # all host cores: the same oracle source built with OpenMP (bit-identical
    # states), else the serial build on one core
    cpu = host_cpu()
    path = O.build_omp()
    cores = cpu["nproc"] if path is not None else 1
    with (O.library(path) if path is not None else contextlib.nullcontext()):
        X, _, _ = O.step(cfg, X, args.warmup)
        t0 = time.perf_counter()
        O.step(cfg, X, args.steps)
        dt = time.perf_counter() - t0
    value = nx * NZ * args.steps / dt
    how = f"OpenMP build on {cores} cores" if path is not None else "single thread"
    sample = f"{args.steps} FP64 steps of a {nx}x{NZ} slice of the workload (same per-node work), {how}"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "nx": nx, "nz": NZ, "Ra": RA, "Pr": PR, "gamma": GAMMA},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu": cpu},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_case(args):
    """One kernel family on its own, for profiler captures: a few steps of
    the chosen case at the given size, then one JSON line (no timing claims)."""
    import numpy as np
    import paper_2411_10372_gb300 as cm
    case, out = args.case, {"case": args.case}
    if case in ("2d_fp32", "2d_fp64", "3d_fp32", "3d_fp64"):
        prec = case[3:]
        if case.startswith("3d"):
            s = cm.Solver(args.nx, args.nz, RA3, PR, GAMMA, ny=args.ny, ndim=3, precision=prec, zstretch=args.zstretch)
        else:
            s = cm.Solver(args.nx, args.nz, RA, PR, GAMMA, precision=prec, zstretch=args.zstretch)
        s.step(args.warmup)
        s.step(args.steps)
        d = s.sample()
        s.close()
        out.update(nx=args.nx, ny=args.ny if case.startswith("3d") else 1, nz=args.nz, status=d["status"])
    elif case == "extended":
        s = cm.Solver(args.nx, args.nz, RA, PR, GAMMA, precision="fp32", zstretch=args.zstretch)
        s.step(args.warmup)
        for _ in range(max(1, args.steps)):
            e, hist = s.extended(96, -14.0, 0.0)
        s.close()
        out.update(nx=args.nx, nz=args.nz, C=e["C"], hist_nodes=int(hist.sum()))
    elif case == "batch":
        rng = np.random.default_rng(2024)
        u, u2 = rng.random(64), rng.random(64)
        nzs = [int(round(32 * 8 ** x)) for x in u]
        p = cm.cm_default_params()
        p.precision = cm.CM_FP32
        cm.cm_batch_init([cm.cm_grid(2, 4 * nz, 1, nz, 4.0, args.zstretch) for nz in nzs], [10 ** (5 + 4 * x) for x in u2], PR,
                         GAMMA, p)
        cm.cm_batch_step(args.warmup + args.steps)
        out.update(boxes=64, status=max(d["status"] for d in cm.cm_batch_diagnostics()))
        cm.cm_batch_finalize()
    elif case == "adjoint":
        s = cm.Solver(args.nx, args.nz, 1e8, PR, GAMMA, precision="fp64")
        J = cm.cm_adj_forward(args.steps, max(1, args.steps // 4), args.steps // 2 + 1)
        g = cm.cm_adj_backward(None, None)
        s.close()
        out.update(nx=args.nx, nz=args.nz, J=J, dJ_dRa=g)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-stretched", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--steps-3d", type=int, default=200)
    ap.add_argument("--nx", type=int, default=NX, help="grid override (profiling captures only)")
    ap.add_argument("--nz", type=int, default=NZ, help="grid override (profiling captures only)")
    ap.add_argument("--ny", type=int, default=512, help="3D grid override (--case only)")
    ap.add_argument("--only-fp32", action="store_true", help="time the FP32 steps only (profiling captures)")
    ap.add_argument("--zstretch", type=float, default=0.0, help="tanh z-grid for --case 2d_*, 3d_*, batch, extended (profiling captures)")
    ap.add_argument("--case", choices=["2d_fp32", "2d_fp64", "3d_fp32", "3d_fp64", "batch", "adjoint", "extended"],
                    help="run one kernel family untimed (profiling captures)")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

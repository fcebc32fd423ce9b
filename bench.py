#!/usr/bin/env python
"""Throughput of the coupled LBM step with the general local reactive
boundary condition on one GB300 (or N independent replicas under torchrun).

Default workload: 3D precipitation in a seeded sphere pack of 512^3 cells
(porosity 0.4, radii U[8,16], periodic in y and z, 8 fluid layers at both
open x ends), D3Q19 TRT flow at Re = 0.1, D3Q7 solute at Pe = 100 through
the rest fraction, supersaturated inlet c = 2 c_eq, phase change on, FP32
populations with FP64 ledgers and solid fractions.  A step is one pass of
the whole hot path: fluid stream-collide, reactive boundary condition +
ledger + solid fraction on every wet boundary cell, the precipitation-share
gather, and the phase-change events with the rebuild of the lists.
``--case channel`` runs the 256x128x128 tilted channel instead.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (bounded per-step samples, all cores).
"""
import argparse
import ctypes
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled MLUPS and % of HBM roofline at stated accuracy vs FP64; adjoint/forward cost"
BYTES_PER_FLUID_CELL = {"fp32": 2 * (19 + 7) * 4, "fp64": 2 * (19 + 7) * 8}
L2_BYTES = 129e6
# cells of an oracle sample (about 420 B of host memory per cell)
ORACLE_MAX_CELLS = 8_000_000


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 200; --case adjoint: 4000, the gradient's run length)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--theta", type=float, default=30.0)
    ap.add_argument("--pe", type=float, default=10.0)
    ap.add_argument("--da", type=float, default=1.0)
    ap.add_argument("--size", type=str, default="256x128x128")
    ap.add_argument("--pack-n", type=int, default=512, help="edge of the sphere-pack case")
    ap.add_argument("--case", choices=["channel", "spherepack", "batch", "adjoint", "molins"], default="spherepack",
                    help="spherepack: the headline, 512^3 precipitation with phase change; channel: 256x128x128 "
                         "tilted channel")
    ap.add_argument("--layout", choices=["auto", "dense", "sparse"], default="auto",
                    help="population layout of the library (auto: active cells in porous media)")
    ap.add_argument("--accuracy-steps", type=int, default=None,
                    help="steps of the FP32-vs-FP64 accuracy run (default: the case's run length)")
    ap.add_argument("--sweep", choices=["dense", "list"], default="dense",
                    help="fluid-cell sweep of the library (LBRBC_FLUID_SWEEP)")
    ap.add_argument("--domains", type=int, default=256, help="number of domains of --case batch")
    ap.add_argument("--molins-cases", type=str, default="4", help="Table 2 cases of --case molins, e.g. 1,2,3,4")
    ap.add_argument("--scale", type=float, default=1.0, help="resolution of --case molins (1 = the paper's 600x1200)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    return ap.parse_args()


def workload(a):
    from paper_2306_10794_gb300 import workloads

    if a.case == "spherepack":
        p, mask, extra = workloads.case_sphere_pack(n=a.pack_n)
        p["precision"] = a.precision
        p["layout"] = a.layout
        name = ("3D precipitation in a seeded sphere pack %d^3, porosity 0.4, radii U[8,16], D3Q19 TRT flow "
                "Re=0.1 + D3Q7 solute Pe=100 (rest fraction), c_in = 2 c_eq, phase change on, %s" % (a.pack_n, a.precision))
        return p, mask, extra, name
    nx, ny, nz = (int(v) for v in a.size.split("x"))
    p, mask, extra = workloads.case_channel(nx=nx, ny=ny, nz=nz, theta_deg=a.theta, Pe=a.pe, Da=a.da)
    p["precision"] = a.precision
    p["layout"] = a.layout
    name = ("3D tilted channel %dx%dx%d, walls %g deg to the grid, D3Q19 TRT flow Re=1 + D3Q7 solute "
            "Pe=%g Da=%g (rest fraction), c_in=1 c_eq=0.5, %s" % (nx, ny, nz, a.theta, a.pe, a.da, a.precision))
    return p, mask, extra, name


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    """SM clock, power and clock-event reasons while the timed region runs.
    NVML (the driver's management library, read-only queries through ctypes)
    is polled every 2 ms from a thread, so a timed region of tens of
    milliseconds still gets samples; without NVML, nvidia-smi samples every
    200 ms."""

    # clock-event reason bits of the NVML API
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = self.nvml_index(index)
        self.rows, self.stop_flag, self.thread, self.p = [], False, None, None
        self.lib = self.dev = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            dev = ctypes.c_void_p()
            if lib.nvmlInit_v2() == 0 and lib.nvmlDeviceGetHandleByIndex_v2(self.index, ctypes.byref(dev)) == 0:
                self.lib, self.dev = lib, dev
                self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                    getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
                mx = ctypes.c_uint()
                self.max_mhz = float(mx.value) if lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx)) == 0 else None
                self.thread = threading.Thread(target=self._poll, daemon=True)
                self.thread.start()
                return
        except Exception:
            self.lib = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    @staticmethod
    def nvml_index(local):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if ids and all(v.isdigit() for v in ids) and local < len(ids):
            return int(ids[local])
        return local

    def _poll(self):
        sm, rs, pw = ctypes.c_uint(), ctypes.c_ulonglong(), ctypes.c_uint()
        while not self.stop_flag:
            ok = self.lib.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(sm)) == 0
            ok = ok and self.reasons_fn(self.dev, ctypes.byref(rs)) == 0
            self.lib.nvmlDeviceGetPowerUsage(self.dev, ctypes.byref(pw))
            if ok:
                self.rows.append((float(sm.value), int(rs.value), pw.value / 1000.0))
            time.sleep(0.002)

    def stop(self):
        if self.thread is not None:
            self.stop_flag = True
            self.thread.join(timeout=5)
            if not self.rows:
                return None
            sm = [r[0] for r in self.rows]
            reasons = sorted({n for r in self.rows for b, n in self.REASONS.items() if r[1] & b})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                    "samples": len(self.rows), "power_w_max": max(r[2] for r in self.rows), "source": "nvml 2 ms"}
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                c = [x.strip() for x in line.split(",")]
                if len(c) >= 9:
                    rows.append(c)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if re.match(r"^[0-9.]+$", r[1])]
        mx = [float(r[2]) for r in rows if re.match(r"^[0-9.]+$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi 200 ms"}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# GB300 FP64 rate (nominal, no measured figure exists for it): 1.25 TFLOP/s,
# i.e. 625 G FP64 pipe operations/s (a DFMA is 2 FLOP; DADD and DMUL take a
# pipe slot each as well).
FP64_PEAK_GOPS = 625.0


def fp64_ops_per_cell(kernel_src_hash, wkey):
    """FP64 pipe operations (DFMA + DADD + DMUL) per fluid cell of one
    k_fluid launch from the committed ncu count, if it was taken on the
    current kernel source and this workload (else None)."""
    path = os.path.join(ROOT, "profiles", "k_fluid_channel_fp64.md")
    try:
        txt = open(path).read()
    except OSError:
        return None, None
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"fp64_ops_per_fluid_cell:\s*([0-9.eE+]+)", txt)
    w = re.search(r"workload_key:\s*(\S+)", txt)
    if not m or not t or not w or m.group(1) != kernel_src_hash or w.group(1) != wkey:
        return None, None
    return float(t.group(1)), os.path.relpath(path, ROOT)


def workload_key(a, layout):
    """Identifies the workload an ncu summary was taken on."""
    if a.case == "spherepack":
        return "spherepack-n%d-%s-%s" % (a.pack_n, a.precision, layout)
    return "%s-%s-%s-theta%g-pe%g-da%g-%s-%s" % (a.case, a.size, a.precision, a.theta, a.pe, a.da, a.sweep, layout)


def ncu_traffic(kernel_src_hash, wkey, fname):
    """DRAM bytes per launch of the fluid kernel from the committed ncu summary,
    if it was taken on the current kernel source and on this workload (else
    None)."""
    path = os.path.join(ROOT, "profiles", fname)
    try:
        txt = open(path).read()
    except OSError:
        return None, None
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    w = re.search(r"workload_key:\s*(\S+)", txt)
    if not m or not t or not w or m.group(1) != kernel_src_hash or w.group(1) != wkey:
        return None, None
    return float(t.group(1)), os.path.relpath(path, ROOT)


def kernel_hash():
    """Hash of the fluid kernel's device sources with comments and blank
    space removed (a comment edit does not change the kernel)."""
    h = hashlib.sha256()
    for f in ("engine.cuh", "lattice.cuh", "pairs.cuh"):
        txt = open(os.path.join(ROOT, "paper_2306_10794_gb300", "csrc", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        h.update("\n".join(line.strip() for line in txt.splitlines() if line.strip()).encode())
    return h.hexdigest()[:16]


def aggregate(ms_local, units_local, dist=None, device=None):
    """Whole-job figure over ranks: the slowest rank's time and the sum of
    all ranks' units (replicas: each rank runs its own domain).  Returns
    (ms_max, units_total, value = units_total / ms_max in units per ms)."""
    import torch

    t = torch.tensor([float(ms_local), float(units_local)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized():
        tm = t[:1].clone()
        tu = t[1:].clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(tu, op=dist.ReduceOp.SUM)
        t = torch.cat([tm, tu])
    ms_max, units = float(t[0]), float(t[1])
    return ms_max, units, units / ms_max


# ---------------------------------------------------------------------------
# CPU oracle timing
# ---------------------------------------------------------------------------
def oracle_mlups(p, mask, extra, budget_s, threads=1, max_steps=None):
    """Run the FP64 oracle on (a bounded x-slab of) the workload on `threads`
    host threads; returns (MLUPS, threads, sample description, steps, s)."""
    import numpy as np

    import oracle

    nz, ny, nx = mask.shape
    q = {k: v for k, v in p.items() if k not in ("precision", "layout")}
    # calibrate on a thin slab
    cal_nx = min(nx, 8)
    q["nx"] = cal_nx
    o = oracle.OracleSim(q, np.ascontiguousarray(mask[:, :, :cal_nx]), **extra)
    o.set_threads(threads)
    t0 = time.perf_counter()
    o.step(1)
    t_cal = time.perf_counter() - t0
    o.close()
    per_slab_col = t_cal / cal_nx
    steps = max_steps or 1
    sub_nx = max(4, min(nx, int(budget_s / max(steps * per_slab_col, 1e-9)), ORACLE_MAX_CELLS // (ny * nz)))
    q["nx"] = sub_nx
    sub = np.ascontiguousarray(mask[:, :, :sub_nx])
    o = oracle.OracleSim(q, sub, **extra)
    o.set_threads(threads)
    fluid = int((sub == 0).sum())
    done, t0 = 0, time.perf_counter()
    while True:
        o.step(1)
        done += 1
        el = time.perf_counter() - t0
        if (max_steps and done >= max_steps) or (not max_steps and el >= budget_s):
            break
    o.close()
    desc = "x-slab %dx%dx%d of the workload (first %d columns, inlet included), %d step(s), %d thread(s)" % (
        sub_nx, ny, nz, sub_nx, done, threads)
    return fluid * done / el / 1e6, threads, desc, done, el


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def reference_arm(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p, mask, extra, name = workload(a)
    K, W = max(1, a.steps), max(0, a.warmup)
    # each step (warm-up and timed) is one oracle step on a bounded slab,
    # sized so that the whole run stays around two minutes
    per_step_budget = 110.0 / (K + W)
    import numpy as np

    import oracle

    nz, ny, nx = mask.shape
    cores = host_cores()
    q = {k: v for k, v in p.items() if k not in ("precision", "layout")}
    cal_nx = min(nx, 8)
    q["nx"] = cal_nx
    o = oracle.OracleSim(q, np.ascontiguousarray(mask[:, :, :cal_nx]), **extra)
    o.set_threads(cores)
    t0 = time.perf_counter()
    o.step(1)
    per_col = (time.perf_counter() - t0) / cal_nx
    o.close()
    sub_nx = max(4, min(nx, int(per_step_budget / max(per_col, 1e-9)), ORACLE_MAX_CELLS // (ny * nz)))
    q["nx"] = sub_nx
    sub = np.ascontiguousarray(mask[:, :, :sub_nx])
    o = oracle.OracleSim(q, sub, **extra)
    o.set_threads(cores)
    fluid = int((sub == 0).sum())
    o.step(W)
    t0 = time.perf_counter()
    o.step(K)
    el = time.perf_counter() - t0
    o.close()
    v = fluid * K / el / 1e6
    sample = "x-slab %dx%dx%d of the workload per step (oracle FP64, %d threads: z-slabs)" % (sub_nx, ny, nz, cores)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": a.gpus, "steps": K,
            "warmup": W, "ms_per_step": el / K * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sample": sample, "fluid_cells_per_step": fluid},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# Table 2 of the paper (Sec. 3.3): R_avg in 1e-8 mol/(cm^2 s) per case and
# scheme, the printed values the molins case is compared with.
TABLE2 = {1: dict(verhaeghe=4.48, patel_ju=4.66, new=4.64, anti_bb=4.71),
          2: dict(verhaeghe=4.70, patel_ju=4.70, new=4.70, anti_bb=4.71),
          3: dict(verhaeghe=75.5, patel_ju=75.9, new=75.8, anti_bb=76.0),
          4: dict(verhaeghe=8.05, patel_ju=29.1, new=18.5, anti_bb=76.0)}


def molins_arm(a):
    """Reactive disc in a channel flow (Sec. 3.3): every scheme of the
    chosen Table 2 cases run to a steady R_avg (relative change below 1e-4
    over a chunk), R_avg from the outlet integral and from the ledger, the
    paper's value beside it, and the coupled MLUPS of the run."""
    import numpy as np
    import torch

    from paper_2306_10794_gb300 import _build, experiments, lbrbc, workloads

    _build.build()
    stream = torch.cuda.current_stream()
    rows, cells_steps, t_total, launches = [], 0, 0.0, 0
    for case in [int(c) for c in a.molins_cases.split(",")]:
        for scheme in ("verhaeghe", "patel_ju", "new", "anti_bb"):
            p, mask, init, geom = workloads.case_molins(case, scheme, a.scale, precision=a.precision)
            s = lbrbc.Sim(p, mask, **init)
            fluid = s.info()["fluid_cells"]
            per_step = s.launch_counts()["per_step"]
            chunk = max(1000, int(250_000 * a.scale * a.scale))
            cap = 3 * geom["steps_hint"]
            done, prev, led_prev = 0, None, s.ledger()["reacted"]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = 0.0
            while True:
                e0.record(stream)
                s.step(chunk, stream=stream.cuda_stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                done += chunk
                u, _, c, _ = s.fields()
                r = experiments.molins_ravg(u, c, geom)[1]
                led = s.ledger()["reacted"]
                r_led = -(led - led_prev) / chunk / (np.pi * geom["d_obj"]) * geom["to_paper"]
                led_prev = led
                if prev is not None and abs(r - prev) <= 1e-4 * abs(r) or done >= cap:
                    break
                prev = r
            s.check()
            s.close()
            cells_steps += fluid * done
            launches += per_step * done
            t_total += ms * 1e-3
            rows.append({"case": case, "scheme": scheme, "R_avg": r, "R_avg_ledger": r_led,
                         "paper": TABLE2[case][scheme], "rel_to_paper": r / TABLE2[case][scheme] - 1.0,
                         "steps": done, "converged": done < cap, "mlups": fluid * done / (ms * 1e-3) / 1e6})
    new4 = [x["R_avg"] for x in rows if x["case"] == 4 and x["scheme"] == "new"]
    line = {"metric": "R_avg of the reactive disc in a channel flow (Table 2)",
            "value": new4[0] if new4 else rows[0]["R_avg"], "unit": "1e-8 mol/(cm^2 s)", "n_gpus": 1,
            "steps": int(sum(x["steps"] for x in rows)), "warmup": 0, "higher_is_better": None, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "2D reactive disc in a channel, %dx%d cells (scale %.2f of 600x1200), D2Q9 TRT flow "
                                   "Re=0.6 + D2Q5 TRT solute with rest fraction, cases %s, four k_i schemes"
                                   % (int(round(1200 * a.scale)), int(round(600 * a.scale)), a.scale, a.molins_cases)},
            "table": rows, "mlups": cells_steps / t_total / 1e6, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    return 0


def batch_arm(a):
    """256 uneven dissolution domains: autotuned batched launches vs one
    launch (CUDA graph) per domain per step."""
    import torch

    from paper_2306_10794_gb300 import _build, lbrbc, workloads

    _build.build()
    cases, meta = workloads.case_batch(n=a.domains, precision=a.precision)
    K, W = max(2, a.steps), max(3, a.warmup)
    stream = torch.cuda.current_stream()
    b = lbrbc.Batch(cases)
    fluid = b.info()["fluid_cells"]
    tune = b.autotune(pairs=3, stream=stream.cuda_stream)
    b.step(W, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(K, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms_b = e0.elapsed_time(e1) / K
    b.close()
    sims = [lbrbc.Sim(p, m, **i) for (p, m, i) in cases]
    for s_ in sims:
        s_.step(W, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    Kp = max(2, min(K, 200))
    e0.record(stream)
    for _ in range(Kp):
        for s_ in sims:
            s_.step(1, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1) / Kp
    for s_ in sims:
        s_.close()
    line = {"metric": METRIC, "value": fluid / (ms_b * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": 1, "steps": K,
            "warmup": W, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if a.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "%d independent 3D dissolution domains, edge U{32..96}, sphere packs porosity "
                                   "U[0.3,0.6], Pe log-U[1,1000] (capped to what the lattice reaches), Da "
                                   "log-U[0.01,10], D3Q19 TRT + D3Q7 TRT, " % len(cases) + a.precision,
                       "domains": len(cases), "fluid_cells": fluid, "autotune": tune},
            "per_domain_launches": {"ms_per_step": ms_p, "value": fluid / (ms_p * 1e-3) / 1e6, "steps": Kp},
            "batched_speedup": ms_p / ms_b, "clocks": ck,
            # schedule 4 launches every domain's own 3 kernels; the others 3 per step
            "gpu_launches": 3 * K * (len(cases) if tune["tile_policy"] == 4 else 1)}
    print(json.dumps(line), flush=True)
    return 0


def adjoint_arm(a):
    """Gradient of the dissolved mass over K steps w.r.t. k_r, c_eq and a
    log-normal per-voxel k field (128^3 sphere pack, porosity 0.45): time of
    lbrbc_adjoint over K steps / time of K plain steps."""
    import numpy as np
    import torch

    from paper_2306_10794_gb300 import _build, lbrbc, workloads

    _build.build()
    n = 128
    mask = workloads.sphere_pack((n, n, n), 0.45, 4.0, 8.0, seed=2305, periodic=(False, True, True), buffer_x=4)
    kf = workloads.lognormal_k(mask.shape, 1e-3, 0.5, seed=2306)
    tau_f = 0.8
    U = 1.0 * (tau_f - 0.5) / 3.0 / 12.0
    p = dict(dim=3, nx=n, ny=n, nz=n, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"), tau_flow=tau_f,
             magic_flow=3.0 / 16.0, tau_solute=0.8, magic_solute=0.25, rest_fraction=0.5, k_r=1e-3, c_eq=1.0,
             c_init=0.0, c_inlet=0.0, u_inlet=U, rho_outlet=1.0, molar_volume=0.1, precision=a.precision)
    K = max(4, a.steps)
    stream = torch.cuda.current_stream()
    fwd = lbrbc.Sim(p, mask, k_field=kf)
    lay = fwd.layout_info()["layout"]
    fwd.step(3, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    fwd.step(K, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_f = time.perf_counter() - t0
    ck_f = clocks.stop()
    fwd.close()
    adj = lbrbc.Sim(p, mask, k_field=kf)
    adj.step(3, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    J, dk, dc, g = adj.adjoint(K, field=True)
    torch.cuda.synchronize()
    t_a = time.perf_counter() - t0
    ck = clocks.stop()
    fluid = adj.info()["fluid_cells"]
    # launches of lbrbc_adjoint over K steps: the forward pass (step graphs),
    # the per-segment recomputation (the step's 3 kernels, launched one by
    # one), the 3 adjoint kernels of each step, and the two ledger reductions
    adj_launches = K * (adj.launch_counts()["per_step"] + 3 + 3) + 4
    adj.close()
    line = {"metric": METRIC, "value": t_a / t_f, "unit": "adjoint/forward time", "n_gpus": 1, "steps": K,
            "warmup": 3, "ms_per_step": t_a / K * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "128^3 dissolution in a seeded sphere pack, porosity 0.45, D3Q19 TRT + D3Q7 TRT, "
                                   "log-normal k field (sigma 0.5), gradient of dissolved mass w.r.t. k_r, c_eq and "
                                   "k(x) by the discrete adjoint with sqrt(N) checkpoints",
                       "fluid_cells": fluid},
            "forward_ms_per_step": t_f / K * 1e3, "adjoint_ms_per_step": t_a / K * 1e3,
            "J": J, "dJ_dk": dk, "dJ_dceq": dc, "dJ_dkfield_norm": float(np.sqrt((g ** 2).sum())),
            "layout": lay, "clocks": ck, "clocks_forward": ck_f, "gpu_launches": adj_launches}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = args_()
    if a.steps is None:
        a.steps = 4000 if a.case == "adjoint" else 200
    if a.impl == "reference":
        return reference_arm(a)
    if a.case == "adjoint":
        return adjoint_arm(a)
    if a.case == "batch":
        return batch_arm(a)
    if a.case == "molins":
        return molins_arm(a)
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2306_10794_gb300 import _build, lbrbc

    if rank == 0 or world == 1:
        _build.build()
    if dist:
        dist.barrier()
    p, mask, extra, name = workload(a)
    os.environ["LBRBC_FLUID_SWEEP"] = a.sweep
    K, W = max(1, a.steps), max(3, a.warmup)
    stream = torch.cuda.current_stream()
    if p.get("phase_change"):
        p = dict(p, event_log_capacity=1 << 22)  # to count the steps with events
    sim = lbrbc.Sim(p, mask, **extra)
    info = sim.info()
    lay = sim.layout_info()
    fluid = info["fluid_cells"]
    sim.step(W, stream=stream.cuda_stream)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    nev0 = len(sim.events()) if p.get("phase_change") else 0
    clocks = Clocks(local)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(K, stream=stream.cuda_stream)
    e1.record(stream)
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    # launches in the timed region: every step's, plus the phase-change path
    # of each step that raised events (a conditional node of the step graphs)
    lc = sim.launch_counts()
    ev_steps = len(set(np.asarray(sim.events())[nev0:, 0].tolist())) if p.get("phase_change") else 0
    launches_timed = lc["per_step"] * K + lc["per_event_step"] * ev_steps
    ms_max, units, per_ms = aggregate(ms, fluid * K, dist, device="cuda")
    value = per_ms * 1e3 / 1e6  # fluid-cell updates per second / 1e6
    sim.check()

    # per-kernel durations, CUDA events on the launching stream (no graphs)
    nprof = min(K, 2000)
    kms, _ = sim.profile(nprof, stream=stream.cuda_stream)
    sim.check()
    bytes_launch = BYTES_PER_FLUID_CELL[a.precision] * fluid
    peak, peak_kind = measured_peak()
    achieved = bytes_launch / (kms[0] * 1e-3) / 1e9
    khash = kernel_hash()
    wkey = workload_key(a, lay["layout"])
    traffic, traffic_src = ncu_traffic(khash, wkey, "k_fluid_pack512.md" if a.case == "spherepack"
                                       else "k_fluid_channel.md")
    step_gbs = bytes_launch / (ms_max / K * 1e-3) / 1e9
    kname = "%s (fluid-cell stream-collide, D3Q19 + D3Q7)" % (
        "k_fluid_sp" if lay["layout"] == "sparse" else ("k_fluid_list" if a.sweep == "list" else "k_fluid"))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "bytes_per_launch": bytes_launch, "ms_per_launch": kms[0],
                "peak_kind": peak_kind, "traffic_source": traffic_src, "kernel_source_sha256": khash,
                "step_algorithmic_gbs": step_gbs}
    if a.precision == "fp64":
        # the FP64 sweep is bound by GB300's FP64 rate, not by HBM
        opc, osrc = fp64_ops_per_cell(khash, wkey)
        if opc is not None:
            gops = opc * fluid / (kms[0] * 1e-3) / 1e9
            roofline = {"bound": "alu", "achieved": gops, "peak": FP64_PEAK_GOPS, "unit": "G FP64 ops/s",
                        "frac": gops / FP64_PEAK_GOPS, "traffic": None, "kernel": kname,
                        "ops_per_fluid_cell": opc, "ops_source": osrc, "ms_per_launch": kms[0],
                        "peak_kind": "nominal FP64 rate 1.25 TFLOP/s = 625 G pipe ops/s (none measured)",
                        "kernel_source_sha256": khash,
                        "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak}}

    # accuracy of this precision against the FP64 path (outside the timed
    # region), over the case's run length: the channel at full size for
    # 20 000 steps; the sphere pack on a 128^3 pack of the same recipe for
    # 50 000 steps (the full 512^3 run would take too long in FP64).  The
    # FP64 path is matched against the oracle by the tests.
    acc = None
    if a.precision == "fp32" and not a.no_accuracy:
        from paper_2306_10794_gb300 import workloads

        if a.case == "spherepack":
            pa, ma, xa = workloads.case_sphere_pack(n=128)
            pa["layout"] = a.layout
            steps_acc = a.accuracy_steps or 50000
            where = "128^3 sphere pack of the same recipe (seed 2306)"
        else:
            pa, ma, xa = p, mask, extra
            steps_acc = a.accuracy_steps or 20000
            where = "the workload itself"
        pa = dict(pa, event_log_capacity=1 << 20)
        s64 = lbrbc.Sim(dict(pa, precision="fp64"), ma, **xa)
        s32 = lbrbc.Sim(dict(pa, precision="fp32"), ma, **xa)
        s64.step(steps_acc, stream=stream.cuda_stream)
        s32.step(steps_acc, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        s64.check()
        s32.check()
        u64, _, c64, phi64 = s64.fields()
        u32, _, c32, phi32 = s32.fields()
        ev64, ev32 = s64.events(), s32.events()
        rl2 = lambda x, y: float(np.sqrt(((x - y) ** 2).sum() / max((y ** 2).sum(), 1e-300)))
        acc = {"steps": steps_acc, "on": where, "rel_l2_c": rl2(c32, c64), "rel_l2_u": rl2(u32, u64),
               "rel_l2_phi": rl2(phi32, phi64), "events_fp64": int(len(ev64)), "events_fp32": int(len(ev32)),
               "events_identical": bool(len(ev64) == len(ev32) and np.array_equal(ev64, ev32)),
               "against": "FP64 CUDA path"}
        s64.close()
        s32.close()
    sim.close()

    # end to end through the C ABI with host buffers: create from the host
    # mask, K steps, concentration and solid fraction back to the host
    e2e = None
    if not a.no_e2e:
        barrier()
        c_host = np.empty(mask.size)
        phi_host = np.empty(mask.size)
        t0 = time.perf_counter()
        s2 = lbrbc.Sim(p, mask, **extra)
        t1 = time.perf_counter()
        s2.step(K, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        lbrbc.lbrbc_fields(s2._h, None, None, c_host, phi_host)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        parts = {"create_s": t1 - t0, "steps_s": t2 - t1, "fields_s": el - (t2 - t0)}
        s2.close()
        tt = torch.tensor([el], device="cuda", dtype=torch.float64)
        if dist:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        h2d = mask.nbytes + sum(v.nbytes for v in extra.values())
        d2h = c_host.nbytes + phi_host.nbytes
        e2e = {"value": world * fluid * K / float(tt.item()) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
               "includes": "lbrbc_create from host mask + K steps + lbrbc_fields(c, phi) to host", **parts}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        nc = host_cores()
        v, cores, desc, n, el = oracle_mlups(p, mask, extra, budget_s=10.0, threads=nc)
        v1, _, desc1, _, _ = oracle_mlups(p, mask, extra, budget_s=10.0, threads=1)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": desc,
               "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1, "sample": desc1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if a.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": name, "grid": list(mask.shape[::-1]), "fluid_cells": fluid,
                       "wet_boundary_cells": info["boundary_cells"], "parallelism": "replicas" if world > 1 else "1gpu",
                       "layout": lay["layout"], "stored_cells": lay["stored_cells"],
                       "fluid_sweep": a.sweep,
                       "l2_policy": "no flush: populations %.2f GB resident > L2 %.0f MB" % (
                           lay["population_bytes"] / 1e9, L2_BYTES / 1e6)},
            "roofline": roofline,
            "kernel_ms_per_step": {"fluid": kms[0], "boundary": kms[1], "fluid_ends": kms[2],
                                   "phase_change": kms[3]},
            "gpu_launches": int(launches_timed),
            "event_steps_timed": ev_steps,
            "clocks": ck,
            "accuracy": acc,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

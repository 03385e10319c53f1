#!/usr/bin/env python
"""Benchmark of the GB300 IMB-LBM-DEM step.

A step is one coupling cycle of the hot path (DEM sub-cycles, particle map,
fused stream-collide with the immersed boundary and the force/torque
reduction) over the 8192 x 4096 periodic-x suspension of 20000 disks (d = 20,
tau = 0.51, Smagorinsky C = 0.1, DEM on) -- the mixed-precision scale-up
workload on which the metric (MLUPS and HBM roofline fraction against the
plain FP32 path) is quoted.  Its populations (2 x 1.2 GB in FP32) exceed the
129 MB L2, so no flush is needed between steps.

Prints ONE JSON line.  ``value`` = lattice updates per second of whole steps
(all ranks), device-timed with CUDA events on the library's stream;
``e2e`` = the same through the C ABI with host buffers (particle kinematics
uploaded and forces/torques read back every step); ``roofline`` = the
stream-collide kernel's algorithmic bytes per launch over its event-timed
duration against the measured HBM copy bandwidth; ``cpu_baseline`` = the FP64
oracle on a bounded sample, timed on this host; ``storage_variants`` = the same
workload with FP16 / BF16 population storage; ``drag_gradient`` = one reverse-mode
gradient of the time-averaged drag on the 512 x 256 channel with 16 fixed disks
over 4000 steps (imb_drag_gradient), timed on the host clock; ``batched_sweep`` =
256 independent periodic domains with fixed disks (FP16, 5000 steps, imb_batch_*).

  python bench.py [--gpus N --steps K --warmup W] [--workload c3|c2|c1]
                  [--storage fp32|fp16|bf16] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica of the workload
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import math
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

import workloads as W  # noqa: E402

METRIC = "IMB-LBM MLUPS & HBM roofline fraction vs plain FP32 path at stated error"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-variants", action="store_true", help="skip the FP16/BF16 storage lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gradient", action="store_true",
                    help="skip the drag-gradient line (512 x 256 channel, 16 fixed disks, 4000 steps)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the batched-sweep line (256 periodic domains, FP16, 5000 steps)")
    ap.add_argument("--sweep-steps", type=int, default=5000)
    ap.add_argument("--no-3d", action="store_true", help="skip the D3Q19 lines")
    ap.add_argument("--ergun", action="store_true",
                    help="add the packed bed's friction factor against Ergun's (15 000 D3Q19 steps)")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the solid-fraction-0.40 suspension, collapse-box and channel lines")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--evolve-cycles", type=int, default=3000,
                    help="cycles run after the timed ones before the evolved-state timing (0: none)")
    ap.add_argument("--nx", type=int, default=None, help="smaller lattice at the same disk density")
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--particles", type=int, default=None, help="override the disk count (0 = fluid only)")
    ap.add_argument("--csmag", type=float, default=None, help="override the Smagorinsky constant")
    return ap.parse_args()


def make_workload(name, nx=None, ny=None, particles=None, csmag=None):
    if name == "c1":
        w = W.c1()
    elif name == "c2":
        w = W.c2()
    elif nx or ny or particles is not None:
        nx, ny = nx or 8192, ny or 4096
        n = int(round(20000 * nx * ny / (8192 * 4096))) if particles is None else particles
        w = W.c3(n=n, nx=nx, ny=ny)
        if n == 0:
            w = w.with_(name=f"c3_fluid_only_{nx}x{ny}")
    else:
        w = W.c3()
    if csmag is not None:
        w = w.with_(C_smag=csmag, name=w.name + f"_C{csmag:g}")
    return w


# --------------------------------------------------------------- distributed
def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda_ok() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def _cuda_ok():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# -------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.index is not None:
            cmd += ["-i", str(self.index)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        parsed = []
        for ts, line in self.rows:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                parsed.append((ts, float(f[1]), float(f[2]), f[4:]))
            except ValueError:
                continue
        window = "timed"
        sel = [p for p in parsed if t0 <= p[0] <= t1 + 0.25]
        if len(sel) < 2:
            sel, window = parsed[-8:], "around-timed"
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, _, flags in sel:
            for name, val in zip(names[1:], flags[1:5]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(s[1] for s in sel), "sm_max_mhz": max(s[2] for s in sel),
                "reasons": sorted(reasons), "samples": len(sel), "window": window}


def gpu_index_for_smi(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        items = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(items) and items[local_rank].strip().isdigit():
            return int(items[local_rank])
    return local_rank


# ----------------------------------------------------------------- baselines
def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "of fallback"


def committed_traffic(kernel_src_hash, workload, storage):
    """DRAM bytes per launch from the committed ncu summary, if it still matches the kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    entry = t.get(f"{workload}:{storage}")
    if not entry or entry.get("kernel_source_sha256") != kernel_src_hash:
        return None
    return entry.get("dram_bytes_per_launch")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("imb_lbm.cu", "imb_device.cuh", "imb_pull.cuh", "imb_node.cuh"):
        with open(os.path.join(ROOT, "paper_1809_07008_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def time_drag_gradient(imb, T=4000, checkpoint_every=100, nx=512, ny=256, snapshots=40):
    """Reverse-mode gradient of the time-averaged drag on the 512 x 256 channel with 16 fixed
    disks: one call of imb_drag_gradient (forward, checkpointed recomputation, backward), and
    one of imb_drag_gradient_binomial with ``snapshots`` snapshots."""
    w = W.c4(steps=T, nx=nx, ny=ny)
    warm = imb.Lattice.from_workload(w)
    warm.drag_gradient(200, checkpoint_every)
    warm.close()
    lat = imb.Lattice.from_workload(w)
    t0 = time.perf_counter()
    J, g_u, g_tau, g_x = lat.drag_gradient(T, checkpoint_every)
    dt = time.perf_counter() - t0
    lat.close()
    # binomial checkpointing with 40 snapshots (41 states held instead of ~140)
    lat = imb.Lattice.from_workload(w)
    t0 = time.perf_counter()
    Jb, g_ub, g_taub, g_xb = lat.drag_gradient(T, snapshots=snapshots)
    dtb = time.perf_counter() - t0
    lat.close()
    _, fwd_b = imb.binomial_schedule(T, snapshots)
    cells = w.nx * w.ny
    return {"workload": w.name, "steps": T, "checkpoint_every": checkpoint_every, "seconds": round(dt, 4),
            "mlups": round(cells * T / dt / 1e6, 1), "note": "lattice updates of the forward horizon per second "
            "of the whole gradient (forward, recomputation and adjoint)", "J": J, "dJ_duin": g_u,
            "dJ_dtau": g_tau, "dJ_dx_max": float(np.abs(g_x).max()),
            "binomial": {"snapshots": snapshots, "seconds": round(dtb, 4), "forward_steps": fwd_b + 1,
                         "states_held": snapshots + 1,
                         "J_rel_diff": abs(Jb - J) / abs(J) if J != 0.0 else abs(Jb - J),
                         "dJ_dtau_rel_diff": abs(g_taub - g_tau) / abs(g_tau) if g_tau != 0.0 else abs(g_taub - g_tau)}}


def time_batched_sweep(imb, steps=5000, n_domains=256, storage="fp16"):
    """The batched sweep: ``n_domains`` periodic domains (128..512 x 128..256, fixed disks,
    body-force driven) in FP16 storage, launch shape tuned on the batch, then ``steps`` steps
    timed with CUDA events on the batch's own stream (graph replays)."""
    doms = W.c5(n_domains)
    b = imb.Batch(doms, storage=storage)
    blk, cpl, _ = b.autotune(steps_per_trial=20)
    b.run(4)   # warm-up: graph capture
    cells = b.cells()
    t0 = time.perf_counter()   # imb_batch_run waits for its stream before returning
    b.run(steps)
    dt = time.perf_counter() - t0
    fx, _ = b.mean_drag()
    b.close()
    bpc = 36.0 if storage != "fp32" else 72.0
    peak, kind = measured_hbm_peak()
    gbs = bpc * cells * steps / dt / 1e9
    return {"domains": n_domains, "cells": cells, "storage": storage, "steps": steps, "seconds": round(dt, 4),
            "mlups": round(cells * steps / dt / 1e6, 1), "ms_per_step": round(dt / steps * 1e3, 4),
            "block": blk, "cells_per_lane": cpl, "bytes_per_cell": bpc, "achieved_gbs": round(gbs, 1),
            "frac": round(gbs / peak, 4), "peak_source": kind,
            "mean_drag_range": [float(fx.min()), float(fx.max())],
            "note": "host clock around imb_batch_run (graph replays, one sync at the end)"}


def _happel_brenner(R, l, U, nu):
    """Eqs. 18-19 (drag and torque on a held sphere a distance l from a wall, undisturbed
    velocity U at its centre, rho = 1), for reporting the benchmark's errors."""
    a = R / l
    F = 6.0 * math.pi * nu * R * U * (1.0 - a * a / 9.0) / (1.0 - 0.6526 * a + 0.316 * a ** 3 - 0.242 * a ** 4)
    T = 8.0 / 3.0 * math.pi * nu * R * R * U * a * (1.0 + 0.0758 * a + 0.049 * a * a)
    return F, T


def _ergun_friction(Re):
    """Eq. 22: the Ergun packed bed friction factor 150 / Re*_p + 1.75."""
    return 150.0 / Re + 1.75


def packed_bed_friction(D, U, N, tau, area, length):
    """The packed bed's modified Reynolds number (Eq. 23) and friction factor (Eq. 22, left) in
    lattice units (rho = 1, d_p = N cells, nu = (tau - 1/2) / 3, porosity 1 - pi / 6), with the
    drag D on the spheres per cross-section ``area`` standing for Delta P across the medium of
    ``length`` cells and U the superficial velocity; returns (Re*_p, f*, Ergun's f*)."""
    n = 1.0 - math.pi / 6.0
    nu = (tau - 0.5) / 3.0
    Re = U * N / (nu * (1.0 - n))
    f = D / (area * length) * N * n ** 3 / (U * U * (1.0 - n))
    return Re, f, _ergun_friction(Re)


def time_lattice3(imb, torch, ts, steps=100, ergun=False):
    """The D3Q19 path: throughput on the 400 x 100 x 400 Poiseuille-flow-past-a-sphere box
    (N = 20 cells per diameter, 16 M cells) and on the paper's packed bed (Sec. 3.3, N = 20,
    240 x 100 x 100 cells, its Delta P = 1600 Pa run: tau = 0.501, C = 0.3, touching spheres
    sharing cells), in FP32 and FP16 storage; the steady drag and torque errors against
    Eqs. 18-19 at N = 5, 10 and 20 (n_sub = 5, tau = 1: Table 2's rows); with ``ergun``, the
    packed bed's friction factor at its lowest pressure difference (1 Pa, tau = 0.58) against
    Ergun's (Eqs. 21-23)."""
    out = {}
    peak, kind = measured_hbm_peak()
    for w, kern in ((W.happel(20), "k3_stream_collide (one sphere per cell, BGK)"),
                    (W.packed_bed(20, run=9), "k3_stream_collide (two slots, Smagorinsky)")):
        for st in ("fp32", "fp16"):
            g = imb.Lattice3.from_workload(w, storage=st)
            g.step(5)
            g.enable_kernel_timing(True)
            t0 = time.perf_counter()
            g.step(steps)
            dt = time.perf_counter() - t0
            ms, n = g.kernel_time()
            kavg = ms / max(n, 1) * 1e-3
            gbs = g.bytes_per_cell() * w.cells / kavg / 1e9
            out[f"{w.name}:{st}"] = {"cells": w.cells, "spheres": w.n_spheres, "steps": steps,
                                     "ms_per_step": round(dt / steps * 1e3, 4),
                                     "mlups": round(w.cells / kavg / 1e6, 1), "kernel": kern,
                                     "kernel_ms_avg": round(kavg * 1e3, 4), "bytes_per_cell": g.bytes_per_cell(),
                                     "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4), "peak_source": kind}
            g.close()
    # the packed bed at 1 Pa: the drag on the spheres per unit cross-section is the pressure drop
    # a pressure-driven medium would need, and U the flow rate through the plane in the middle of
    # the free fluid.  The drag settles within tens of steps (the momentum balance), the flow in
    # the pores on the viscous time (d_p / 2)^2 / nu, about 3700 steps: 15 000 steps are four
    if ergun:
        N = 20
        wb = W.packed_bed(N, run=0, C_smag=0.0)
        g = imb.Lattice3.from_workload(wb)
        n_steps = 15000
        g.step(n_steps)
        F, _ = g.forces()
        D = float(F[:, 0].sum())
        _, ux, _, _ = g.macro()
        g.close()
        U = float(ux[:, :, 0].mean())
        Re, f, fe = packed_bed_friction(D, U, N, wb.tau, wb.ny * wb.nz, 10 * N)
        out[f"{wb.name}_ergun"] = {"steps": n_steps, "Re_p": round(Re, 5), "f_star": round(f, 3),
                                   "f_star_ergun": round(fe, 3), "rel_diff": round(f / fe - 1.0, 4)}
    for N in (5, 10, 20):
        wh = W.happel(N)
        g = imb.Lattice3.from_workload(wh)
        prev, n_steps, chunk = None, 0, 500 if N < 20 else 1000
        for _ in range(60):
            g.step(chunk)
            n_steps += chunk
            F, T = g.forces()
            if prev is not None and abs(F[0, 0] - prev) < 1e-5 * abs(F[0, 0]):
                break
            prev = F[0, 0]
        g.close()
        nu = (wh.tau - 0.5) / 3.0
        yc = wh.x[0, 1]
        U = wh.force[0] / (2 * nu) * yc * (wh.ny - yc)
        Fa, Ta = _happel_brenner(wh.R[0], yc, U, nu)
        out[f"happel_N{N}_error_pct"] = {"force": round(abs(Fa - F[0, 0]) / Fa * 100, 3),
                                         "torque": round(abs(Ta - abs(T[0, 2])) / Ta * 100, 3),
                                         "steps": n_steps, "paper_table2": {5: [17.791, 31.4374],
                                                                            10: [6.9793, 11.256],
                                                                            20: [3.7595, 4.426]}[N]}
    return out


def oracle_sample_workload():
    # bounded sample: the 512 x 512 subdomain of the suspension at the same disk density
    return W.c3sub(steps=0)


def _oracle_mlups(O, w, threads, target_s, max_steps):
    prev = O.set_threads(threads)
    sim = O.Sim(w)
    sim.step(2)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < target_s and steps < max_steps:
        sim.step(5)
        steps += 5
    dt = time.perf_counter() - t0
    O.set_threads(prev)
    return w.cells * steps / dt / 1e6, steps, dt


def time_oracle(target_s=12.0, max_steps=2000):
    """The FP64 oracle (as it stands: its collide and stream loops spread over the host's
    cores, the rest on one thread; results identical whatever the thread count) on bounded
    samples: the 512 x 512 subdomain of the suspension at the same disk density on all cores
    (the line's value) and on one core, and the one-disk 200 x 100 channel on one core and on
    all cores; MLUPS."""
    from oracle import oracle as O
    O.build()
    ncores = os.cpu_count() or 1
    w = oracle_sample_workload()
    mlups, steps, dt = _oracle_mlups(O, w, ncores, target_s, max_steps)
    m1, s1, d1 = _oracle_mlups(O, w, 1, 0.5 * target_s, max_steps)
    wc = W.c1(steps=0)
    c1a, _, _ = _oracle_mlups(O, wc, ncores, 0.25 * target_s, 2000)
    c11, _, _ = _oracle_mlups(O, wc, 1, 0.25 * target_s, 2000)
    return mlups, {"value": round(mlups, 3), "unit": "MLUPS", "cores": ncores, "kind": "oracle",
                   "sample": f"{w.name}, {steps} steps in {dt:.1f} s, FP64, {ncores} host threads",
                   "single_thread": {"value": round(m1, 3), "unit": "MLUPS", "cores": 1,
                                     "sample": f"{w.name}, {s1} steps in {d1:.1f} s"},
                   "config1_channel": {"workload": wc.name, "all_cores_mlups": round(c1a, 3),
                                       "single_thread_mlups": round(c11, 3)},
                   "cpu": f"{cpu_model()}, {ncores} logical cores on the host"}


def time_workload(imb, torch, ts, w, storage, steps, warmup):
    """MLUPS of ``steps`` coupling cycles of workload ``w`` (CUDA events on stream ``ts``) and
    the average stream-collide launch with its HBM roofline fraction."""
    lv = imb.Lattice.from_workload(w, storage=storage)
    lv.set_stream(ts.cuda_stream)
    lv.step(warmup)
    lv.enable_kernel_timing(True)
    lv.step(2)            # the timed cycles' graphs captured before the timed region
    lv.kernel_time()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ts)
    lv.step_async(steps)
    e1.record(ts)
    torch.cuda.synchronize()
    lv.sync()
    vms = e0.elapsed_time(e1)
    km, kn = lv.kernel_time()
    kavg = km / max(kn, 1) * 1e-3
    gbs = lv.bytes_per_cell() * w.cells / kavg / 1e9
    peak, _ = measured_hbm_peak()
    out = {"mlups": round(w.cells * steps / (vms * 1e-3) / 1e6, 1), "ms_per_step": round(vms / steps, 4),
           "steps": steps, "particles": w.n_particles, "kernel_ms_avg": round(kavg * 1e3, 4),
           "kernel_gbs": round(gbs, 1), "kernel_frac": round(gbs / peak, 4), "bytes_per_cell": lv.bytes_per_cell()}
    lv.close()
    del lv
    torch.cuda.synchronize()
    return out


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------- runs
def run_reference(args):
    rank, world, _ = dist_init(args.gpus)
    if rank != 0:
        return
    w = make_workload(args.workload, args.nx, args.ny, args.particles, args.csmag)
    mlups, cpu = time_oracle(target_s=max(5.0, min(60.0, 0.05 * (args.steps + args.warmup))))
    # time of one coupling cycle of the whole workload at the sample's throughput
    ms_step = w.cells / (mlups * 1e6) * 1e3 if mlups > 0 else None
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_step, 1) if ms_step else None,
            "ms_per_step_basis": "cells of the workload / the sample's MLUPS",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "sample": oracle_sample_workload().name},
            "cpu_baseline": cpu,
            "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    import paper_1809_07008_gb300 as imb
    imb.load()
    w = make_workload(args.workload, args.nx, args.ny, args.particles, args.csmag)
    lat = imb.Lattice.from_workload(w, storage=args.storage)
    ts = torch.cuda.Stream()
    lat.set_stream(ts.cuda_stream)
    cells = w.cells

    sampler = ClockSampler(gpu_index_for_smi(local))
    sampler.start()
    time.sleep(0.3)
    lat.step(max(args.warmup, 3))
    lat.enable_kernel_timing(True)
    lat.step(2)           # timed cycles replay graphs of their own: captured here, before the timed region
    lat.kernel_time()     # (and their two timings dropped)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = lat.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    ev0.record(ts)
    lat.step_async(args.steps)
    ev1.record(ts)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    lat.sync()
    barrier(world)
    torch.cuda.synchronize()
    launches = lat.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    k_ms, k_n = lat.kernel_time()
    lat.enable_kernel_timing(False)
    clocks = sampler.summary(t_wall0, t_wall1)
    sampler.stop()
    ms_max = max_over_ranks(ms, world)
    total_cells = sum_over_ranks(float(cells) * args.steps, world)
    mlups = total_cells / (ms_max * 1e-3) / 1e6

    # roofline of the fused stream-collide kernel (the dominant kernel)
    bpc = lat.bytes_per_cell()
    k_avg_s = k_ms / max(k_n, 1) * 1e-3
    achieved = bpc * cells / k_avg_s / 1e9
    peak, peak_kind = measured_hbm_peak()
    traffic = committed_traffic(kernel_source_hash(), w.name, args.storage)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
                "kernel": "k_stream_collide", "bytes_per_cell": bpc,
                "kernel_ms_avg": round(k_avg_s * 1e3, 4),
                "kernel_share_of_step": round(k_ms / ms, 4) if ms > 0 else None}

    # end to end through the C ABI with host buffers (kinematics in, forces out, every step)
    e2e_steps = args.e2e_steps or max(10, min(args.steps, 100))
    n = lat.np
    x, v, om = lat.particles()
    hx = torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
    hv = torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
    hw = torch.from_numpy(np.ascontiguousarray(om)).pin_memory().numpy()
    F = torch.zeros((n, 2), dtype=torch.float64).pin_memory().numpy()
    T = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):   # one imb_step_io per cycle: upload, cycle, read back, one wait
        if n:
            lat.step_io(1, (hx, hv, hw), F, T, hx, hv, hw)
        else:
            lat.step(1)
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(t1 - t0, world)
    e2e_mlups = sum_over_ranks(float(cells) * e2e_steps, world) / e2e_s / 1e6
    e2e = {"value": round(e2e_mlups, 1), "unit": "MLUPS", "h2d_bytes_per_step": 40 * n,
           "d2h_bytes_per_step": 24 * n + 40 * n, "steps": e2e_steps, "call": "imb_step_io"}

    # the same lattice further on: as the disks meet, contacts and islands form and the DEM's
    # sub-cycles (latency-bound FP64 chains) take a growing share of the cycle
    evolved = None
    if world == 1 and args.evolve_cycles > 0 and w.dem_on and n:
        lat.step(args.evolve_cycles)
        lat.enable_kernel_timing(True)
        torch.cuda.synchronize()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        v0.record(ts)
        lat.step_async(100)
        v1.record(ts)
        torch.cuda.synchronize()
        lat.sync()
        vms = v0.elapsed_time(v1) / 100
        km, kn = lat.kernel_time()
        lat.enable_kernel_timing(False)
        evolved = {"after_cycles": max(args.warmup, 3) + 2 + args.steps + e2e_steps + args.evolve_cycles,
                   "steps": 100, "ms_per_step": round(vms, 4), "mlups": round(cells / (vms * 1e-3) / 1e6, 1),
                   "kernel_ms_avg": round(km / max(kn, 1), 4)}

    variants, others = {}, {}
    if rank == 0 and ((not args.no_variants and args.storage == "fp32") or not args.no_other):
        lat.close()
        del lat
        torch.cuda.synchronize()
    if not args.no_variants and args.storage == "fp32" and rank == 0:
        for st in ("fp16", "bf16"):
            variants[st] = time_workload(imb, torch, ts, w, st, args.steps, max(args.warmup, 3))
    if not args.no_other and rank == 0:
        # the 8192 x 4096 suspension at solid fraction 0.40 (42 722 disks), the collapse box
        # and the one-disk channel (in L2: launch-bound)
        w40 = W.c3(n=42722).with_(name="c3_suspension_8192x4096_42722disks_phi040")
        for st in ("fp32", "fp16"):
            others[f"{w40.name}:{st}"] = time_workload(imb, torch, ts, w40, st, 100, 3)
        others["c2_collapse_2048x1024_1000disks:fp32"] = time_workload(imb, torch, ts, W.c2(), "fp32", 200, 3)
        others["c1_channel_200x100_1disk:fp32"] = time_workload(imb, torch, ts, W.c1(), "fp32", 2000, 10)

    gradient = None
    if not args.no_gradient and rank == 0:
        gradient = time_drag_gradient(imb)
    sweep = None
    if not args.no_sweep and rank == 0:
        sweep = time_batched_sweep(imb, args.sweep_steps)

    lattice3 = None
    if not args.no_3d and rank == 0:
        lattice3 = time_lattice3(imb, torch, ts, ergun=args.ergun)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, cpu = time_oracle()

    if rank == 0:
        line = {"metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "particles": w.n_particles,
                           "storage": args.storage, "tau": w.tau, "C_smag": w.C_smag,
                           "N_sub": w.N_sub if w.dem_on else 0, "dem": bool(w.dem_on),
                           "l2": "populations larger than L2 (no flush needed)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks}
        if evolved:
            line["evolved"] = evolved
        if variants:
            line["storage_variants"] = variants
        if others:
            line["other_workloads"] = others
        if lattice3:
            line["lattice_3d"] = lattice3
        if gradient:
            line["drag_gradient"] = gradient
        if sweep:
            line["batched_sweep"] = sweep
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()

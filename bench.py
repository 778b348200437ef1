"""Benchmark of the reactive-diffusion LBM hot path on one GB300 (D3Q7 by
default; `--lattice d3q19` times the paper's own 19-velocity lattice).

Workload: the 256^3 Pt catalyst layer at 2 nm (seeded QSGS: pore 45 %,
ionomer 18.87 %, solid 36.13 %; Knudsen diffusivity from the 13-direction
pore length at 353 K; 5 % of the carbon-pore faces catalytic with
k = 1e-3 m/s; gas reservoir plane at x = 0 with a fixed concentration,
zero-flux outlet; periodic in y and z).

One bench step = one check interval of the solver: `--check-every` fused
collide-stream steps (the last with the fused FP64 reduction), replayed as
one CUDA graph, plus the host read of the readouts.  The metric is MLUPS
over all box cells.  The population buffers (2 x 7 x 4 B x 16.8 M cells)
are far larger than the 129 MB L2, so no flush is needed between steps.

Rank r of N solves its own structure (seed 1 + r): weak scaling with no
data-path collective.

`--impl reference` times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import hashlib
import re

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(ROOT, "paper_1410_1914_gb300", "csrc")
KERNEL_SRCS = [os.path.join(_CSRC, f) for f in ("march.cu", "march.cuh", "device_util.cuh")]
KERNEL_SRCS_Q19 = [os.path.join(_CSRC, f) for f in ("q19.cu", "internal.cuh", "device_util.cuh")]
KERNEL_SRCS_Q19S = [os.path.join(_CSRC, f) for f in ("q19s.cu", "internal.cuh", "device_util.cuh")]
KERNEL_SRCS_POP = [os.path.join(_CSRC, f) for f in ("kernels.cu", "internal.cuh", "device_util.cuh")]


def code_only(text: str) -> str:
    """C/CUDA source without its comments and with whitespace collapsed, so
    that editing a comment does not read as a kernel change."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_src_sha256(srcs=None) -> str:
    """sha256 over the step kernel's sources, comments and whitespace aside
    (the key of profiles/traffic.json)."""
    h = hashlib.sha256()
    for f in srcs or KERNEL_SRCS:
        with open(f, encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")
sys.path.insert(0, ROOT)

WORKLOAD = "pt_cl_256"
WORKLOAD_DESC = ("256^3 Pt catalyst layer, 2 nm voxels, seeded QSGS (pore 0.45, ionomer 0.1887), "
                 "Knudsen D (353 K, M 0.032), 5% catalytic carbon-pore faces k=1e-3 m/s, "
                 "reservoir plane + fixed C inlet, zero-flux outlet, periodic y,z")


def bytes_per_cell(storage: str, lattice: str = "d3q7") -> float:
    """Algorithmic DRAM bytes of one fused step per box cell, as the method
    needs them: every cell's populations read once and written once, plus
    its link mask (D3Q7: 2 B; D3Q19: 4 B) and relaxation rate (f32, 4 B).
      fp32pop, fp32   7 f32 populations: 2 * 28 + 6 = 62 B (the FP32 state
                      carries the same information as C + 6 deviations)
      fp16dev         C f32 + 6 f16 deviations: 2 * 16 + 6 = 38 B
      D3Q19 (8 B of static data; the reactive-link word of the few catalytic
      cells is not counted):
        fp32pop, fp32   19 f32 populations: 2 * 76 + 8 = 160 B
        fp16dev         C f32 + 18 f16 deviations: 2 * 40 + 8 = 88 B"""
    if lattice == "d3q19":
        return 2 * {"fp32pop": 76, "fp32": 76, "fp16dev": 40}[storage] + 8
    state = {"fp32": 28, "fp16dev": 16, "fp32pop": 28}[storage]
    return 2 * state + 6


def layout_bytes_per_cell(storage: str, lattice: str = "d3q7") -> float:
    """Bytes per cell and step that this library's layouts move (the state
    keeps C as a double-float, whose low word the method does not need):
      fp32     C as two f32 + 6 f32 deviations: 2 * 32 + 6 = 70 B
      fp16dev  C f32 + f16 low word + 6 f16 deviations: 2 * 18 + 6 = 42 B
      fp32pop  62 B, as the algorithmic figure
      D3Q19: fp32pop 160 B; fp32 2 * (8 + 72) + 8 = 168 B; fp16dev
      2 * (8 + 36) + 8 = 96 B"""
    if lattice == "d3q19":
        return 2 * {"fp32pop": 76, "fp32": 80, "fp16dev": 44}[storage] + 8
    state = {"fp32": 32, "fp16dev": 18, "fp32pop": 28}[storage]
    return 2 * state + 6


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_traffic(storage: str, n_cells: int, lattice: str = "d3q7"):
    """DRAM bytes per launch of the step kernel from the committed ncu capture
    (profiles/traffic.json), scaled by the cells processed; None when the
    kernel source changed since the capture or no capture exists."""
    key = f"d3q19_{storage}" if lattice == "d3q19" else storage
    if lattice == "d3q19":
        srcs = KERNEL_SRCS_Q19 if storage == "fp32pop" else KERNEL_SRCS_Q19S
    else:
        srcs = KERNEL_SRCS_POP if storage == "fp32pop" else KERNEL_SRCS
    try:
        with open(TRAFFIC_JSON) as fh:
            rec = json.load(fh)[key]
        sha = kernel_src_sha256(srcs)
    except (OSError, KeyError, ValueError):
        return None, "no capture"
    if rec.get("src_sha256") != sha:
        return None, "kernel changed since the capture"
    return rec["dram_bytes_per_cell"] * n_cells, rec["case"]


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(ph, react, params, budget_s: float = 20.0, lattice: str = "d3q7", one_core_s: float = 10.0):
    """The FP64 oracle on the host cores: set-up, then as many whole steps as
    fit the budget (at least one), on all cores and then on one core.
    Returns MLUPS and what was sampled."""
    import oracle

    def sample(o, budget):
        steps = 0
        t1 = time.perf_counter()
        while True:
            o.step(1)
            steps += 1
            el = time.perf_counter() - t1
            if el * (steps + 1) / steps > budget:
                return steps, el

    t0 = time.perf_counter()
    o = oracle.OracleLBM(ph, react=react, lattice=int(lattice == "d3q19"), **params)
    t_setup = time.perf_counter() - t0
    n = ph.size
    cores = oracle.num_threads()
    steps, el = sample(o, budget_s)
    out = {"value": n * steps / el / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": f"{steps} FP64 steps of the full {ph.shape[2]}x{ph.shape[1]}x{ph.shape[0]} workload "
                     f"({el:.1f} s; oracle set-up {t_setup:.1f} s not counted)"}
    if one_core_s > 0:
        oracle.set_num_threads(1)
        try:
            s1, e1 = sample(o, one_core_s)
        finally:
            oracle.set_num_threads(cores)
        out["one_core"] = {"value": n * s1 / e1 / 1e6, "unit": "MLUPS", "cores": 1,
                           "sample": f"{s1} FP64 steps of the same workload on one thread ({e1:.1f} s)"}
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1410_1914_gb300 import inputs
    import oracle
    ph, react, params = inputs.make_workload(WORKLOAD, shape=args.shape)
    o = oracle.OracleLBM(ph, react=react, lattice=int(args.lattice == "d3q19"), **params)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(args.ref_steps_per_step)
    el = time.perf_counter() - t0
    n = ph.size
    value = n * args.steps * args.ref_steps_per_step / el / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS (%s fused collide-stream step, all box cells)" % args.lattice.upper(),
        "value": value,
        "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "shape_zyx": list(ph.shape),
                   "lbm_steps_per_bench_step": args.ref_steps_per_step},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{args.steps} x {args.ref_steps_per_step} FP64 steps of the full workload"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_batch64(storage: str, K: int, steps: int, warmup: int, stream):
    """The batch of 64 structures (edges 32-160, Pt/NPMC alternating) in one
    persistent launch per check interval, after the autotuner; against the
    same structures stepped one by one."""
    import torch
    from paper_1410_1914_gb300 import Solver, inputs
    from paper_1410_1914_gb300.batch import Batch
    work = inputs.batch_workloads(64)
    solvers = []
    for ph, react, params in work:
        s = Solver(ph.shape, storage=storage, stream=int(stream.cuda_stream), check_every=K, **params)
        s.set_structure(ph, react)
        solvers.append(s)
    cells = sum(ph.size for ph, _, _ in work)
    b = Batch(solvers)
    zc, pf, tr, ms_tune, cached = b.autotune(steps_per_trial=4, cache=None)
    bi = b.info()
    for _ in range(warmup):
        b.step(K)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        ev0.record(stream)
        for _ in range(steps):
            b.step(K)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    mlups = cells * K * steps / (ms * 1e-3) / 1e6
    # one solve interval through the per-structure stopping rule, for its overhead
    t0 = time.perf_counter()
    b.solve(K)
    torch.cuda.synchronize()
    interval_s = time.perf_counter() - t0
    # the same structures one after another, each with its own launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for s in solvers:
        s.step(2)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in solvers:
        s.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_mlups = cells * K / (e0.elapsed_time(e1) * 1e-3) / 1e6
    peak, peak_kind = measured_peak_gbs()
    achieved = bytes_per_cell(storage) * cells * K * steps / (ms * 1e-3) / 1e9
    out = {
        "workload": "64 cubes, edge uniform 32-160, Pt/NPMC alternating, porosity 0.35-0.65, Knudsen D, "
                    "D_eff set-up", "cells": cells, "storage": storage, "lbm_steps_per_bench_step": K,
        "steps": steps, "warmup": warmup, "mlups": mlups, "ms_per_step": ms / steps,
        "autotuned": {"z_chunk": zc, "prefetch": pf, "tile_rows": tr},
        "grid_blocks": bi["grid_blocks"], "work_items": bi["n_items"],
        "sequential_mlups": seq_mlups, "batch_over_sequential": mlups / seq_mlups,
        "solve_interval_s": interval_s, "solve_uses_graph": b.info()["uses_graph"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "layout_frac": layout_bytes_per_cell(storage) * cells * K * steps / (ms * 1e-3) / 1e9 / peak,
                     "traffic": None, "peak_kind": f"{peak_kind} hbm_gbs", "kernel": "k_march_batch"},
        "gpu_launches": steps,
        "clocks": clocks.summary(),
    }
    b.close()
    for s in solvers:
        s.close()
    return out


def run_batch(args):
    """Batched persistent launch: 64 structures of edge 32-160 in one launch
    per check interval, against the same structures stepped one by one."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    r = measure_batch64(args.storage, args.check_every, args.steps, args.warmup, stream)
    line = {
        "metric": "MLUPS (batch of 64 structures, one persistent launch per check interval)",
        "value": r["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": r["workload"], "cells": r["cells"], "storage": args.storage,
                   "lbm_steps_per_bench_step": args.check_every, "autotuned": r["autotuned"],
                   "grid_blocks": r["grid_blocks"], "work_items": r["work_items"]},
        "sequential_mlups": r["sequential_mlups"],
        "batch_over_sequential": r["batch_over_sequential"],
        "solve_interval_s": r["solve_interval_s"],
        "solve_uses_graph": r["solve_uses_graph"],
        "roofline": r["roofline"],
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_structures(args):
    """Structure generation and labelling on the GPU: the Pt-layer recipe
    (QSGS solid then ionomer, Sec. 2.1.2) at 464^3 = 1e8 voxels, then the
    connected-phase statistics of Sec. 2.1.3 for its three phases (26
    neighbours).  One step = one structure generated and labelled (seed
    1000 + step).  The host generator of the inputs module, timed on the
    same recipe at a bounded size, is the CPU baseline."""
    import torch
    from paper_1410_1914_gb300 import inputs, structures
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.shape[0] if args.shape else 464
    shape = (n, n, n)
    pore, ion = 0.45, inputs.EQ4_EPS045_IONOMER

    def one(seed):
        ph = structures.pt_cl(shape, seed, pore, ion)
        return ph, structures.connectivity(ph)

    for w in range(args.warmup):
        one(900 + w)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    with ClockSampler(0) as clocks:
        ev0.record(stream)
        for k in range(args.steps):
            ph, stats = one(1000 + k)
        ev1.record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = ev0.elapsed_time(ev1)
    vox = ph.numel()
    line = {
        "metric": "Mvoxel/s (QSGS Pt layer generated + three phases labelled, Sec. 2.1.2-2.1.3)",
        "value": vox * args.steps / (ms * 1e-3) / 1e6, "unit": "Mvoxel/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"Pt layer {n}^3, porosity {pore}, ionomer {ion:.4f}, c_d 0.01, P_alpha 0.01; "
                               "26-neighbour labelling of C/Pt, void, ionomer", "voxels": vox},
        "host_wall_s_per_step": wall / args.steps,
        "last_stats": stats,
        "gpu_launches": None,
        "clocks": clocks.summary(),
    }
    if not args.no_cpu_baseline:
        m = 256
        t0 = time.perf_counter()
        inputs.pt_cl((m, m, m), 1000, pore, ion)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": m ** 3 / el / 1e6, "unit": "Mvoxel/s (generation only)",
                                "cores": os.cpu_count(), "kind": "host generator",
                                "sample": f"one {m}^3 Pt layer by the host QSGS ({el:.1f} s), no labelling"}
    print(json.dumps(line), flush=True)
    return 0


def run_converge(args):
    print(json.dumps(measure_converge(args)), flush=True)
    return 0


def measure_converge(args, arm_names=None):
    """Time-to-converged D_eff (Eq. 19 readout within 1e-3, and staying there)
    per storage mode, from the linear ramp and from the learned warm start,
    on a D_eff set-up of the Pt recipe.  The reference is the FP32-state
    solve carried to an extrapolated relative change below 1e-9.  Each arm's
    time covers the GPU set-up of the structure, the network inference (warm
    arms) and the iteration with its per-check host synchronisation."""
    import torch
    from paper_1410_1914_gb300 import Solver, inputs
    from paper_1410_1914_gb300.convergence import deff_trace, time_to_tolerance
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    shape = args.shape or (128, 128, 128)
    if shape == (48, 48, 48):
        ph, react, params = inputs.make_workload("pt_cl_48")
        label = "48^3 Pt layer, 2 nm, bulk D (plain-method small workload)"
    else:
        ph, react, params = inputs.make_workload("pt_cl_256", shape=shape, reactive=False)
        label = f"{shape[2]}x{shape[1]}x{shape[0]} Pt layer, 2 nm, Knudsen D, D_eff set-up"
    if args.carrier == "proton":
        # Eq. 16 in the ionomer alone (uniform conductivity, no source): the
        # effective proton conductivity of Sec. 5.2; readouts are sigma_eff / sigma
        params = dict(params, carrier=1, D_ionomer=1.0, k_ms=0.0)
        react = None
        label = label.replace("Knudsen D, D_eff set-up", "proton conduction in the ionomer (Eq. 16)")
    K = args.check_every
    max_steps = args.max_steps

    if args.lattice == "d3q19":
        label += ", D3Q19 lattice"

    def solver(storage):
        s = Solver(ph.shape, storage=storage, stream=int(stream.cuda_stream), check_every=K, lattice=args.lattice,
                   **params)
        s.set_structure(ph, react)
        return s

    ref_s = solver("fp32")
    st, sec, val = deff_trace(ref_s, max_steps, K, stop_rel_change=1e-9)
    ref = float(val[-1])
    ref_s.close()
    arms = [("fp32pop", False), ("fp32", False), ("fp16dev", False)]
    net = None
    nz, ny, nx = ph.shape
    if nz == ny == nx and nx % 8 == 0 and not args.no_warm and args.carrier == "o2":
        from paper_1410_1914_gb300 import warmstart as W
        if os.path.exists(W.WEIGHTS):
            net = W.load_pretrained()
            net.forward(torch.zeros(1, nx, nx, nx, W.FEATURES, dtype=torch.bfloat16, device="cuda"), 1, nx)
            arms += [("fp32", True), ("fp16dev", True)]
    if arm_names is None and getattr(args, "arms", None):
        arm_names = tuple(a.strip() for a in args.arms.split(","))
    if arm_names is not None:
        arms = [(st, w) for st, w in arms if st + ("+warm" if w else "") in arm_names]
    out = {}
    for storage, warm in arms:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = solver(storage)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        inf_s = 0.0
        if warm:
            t1 = time.perf_counter()
            W.warm_start(net, s)
            torch.cuda.synchronize()
            inf_s = time.perf_counter() - t1
        # the trace only has to outlast the 1e-3 band; FP16 readouts carry ~1e-5 noise
        st, sec, val = deff_trace(s, max_steps, K, stop_rel_change=1e-7)
        n, t = time_to_tolerance(st, sec, val, ref, 1e-3)
        out[storage + ("+warm" if warm else "")] = {
            "steps_to_1e-3": n, "iteration_s": t, "setup_s": setup_s, "inference_s": inf_s,
            "seconds_to_1e-3": None if t is None else setup_s + inf_s + t,
            "final_rel_err": abs(float(val[-1]) - ref) / abs(ref), "steps_run": int(st[-1])}
        s.close()
    def want(name):
        return (arm_names is None and args.krylov) or (arm_names is not None and name in arm_names)

    def steady_arm(name, run):
        # the steady state as the fixed point of the step map; the arm's time covers the set-up and the
        # whole steady solve (to its residual, or its stall), no march afterwards
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = solver("fp32pop")
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        info = run(s)
        err = abs(s.effective_diffusivity()[1] - ref) / abs(ref)
        rec = {k: info[k] for k in ("iterations", "inner_iterations", "status") if k in info}
        rec.update({"solve_s": info["seconds"], "setup_s": setup_s,
                    "seconds_to_1e-3": setup_s + info["seconds"] if err <= 1e-3 else None, "final_rel_err": err})
        out[name] = rec
        s.close()

    if want("fp32pop+krylov"):
        steady_arm("fp32pop+krylov", lambda s: s.solve_krylov(tol=1e-8, max_iter=args.krylov_max_iter, max_steps=0))
    if want("fp32pop+krylov_dsa"):
        # flexible GMRES with the diffusion preconditioner (either lattice)
        steady_arm("fp32pop+krylov_dsa",
                   lambda s: s.solve_krylov_dsa(tol=1e-8, max_iter=args.krylov_max_iter, max_steps=0))
    if args.lattice == "d3q7":
        if want("fp32pop+lines"):
            # the same fixed point in C alone, the populations eliminated along lines (FGMRES in FP64)
            steady_arm("fp32pop+lines",
                       lambda s: s.solve_steady_lines(tol=1e-10, max_iter=args.krylov_max_iter, restart=200))
    plain = out["fp32pop"]["seconds_to_1e-3"] if "fp32pop" in out else None
    state32 = out["fp32"]["seconds_to_1e-3"] if "fp32" in out else None
    best = out.get("fp16dev+warm", out.get("fp16dev", {})).get("seconds_to_1e-3")
    line = {"metric": "time-to-converged D_eff (rel 1e-3)" if args.carrier == "o2"
            else "time-to-converged effective proton conductivity (rel 1e-3)", "unit": "s", "higher_is_better": False,
            "workload": label, "shape_zyx": list(ph.shape), "lattice": args.lattice, "reference_D_eff_over_Db": ref,
            "check_every": K,
            "by_arm": out,
            "fp16_warm_vs_plain_fp32": (None if plain is None or best is None else plain / best),
            "fp16_warm_vs_fp32_state_ramp": (None if state32 is None or best is None else state32 / best),
            "plain_fp32_note": "fp32pop = plain FP32 populations from the linear ramp" + (
                "; it never came within 1e-3" if plain is None else "")}
    return line


NPMC_DESC = ("400^3 NPMC catalyst layer, 1 nm voxels, seeded QSGS (base pore 0.45 + micropores to 0.55), "
             "Knudsen D (353 K, M 0.032), every carbon-pore face catalytic k=1e-5 m/s, reservoir plane + "
             "fixed C inlet, zero-flux outlet, periodic y,z")


def measure_npmc400(stream, K: int, steps: int, peak: float, local: int):
    """The 400^3 NPMC workload in the FP16 state: MLUPS and roofline of the
    fused step (device-timed check intervals), the FP32 state for context,
    and end to end through the C ABI with host buffers (structure upload,
    set-up, 1000 steps, reaction-rate readout)."""
    import torch
    from paper_1410_1914_gb300 import Solver, inputs
    from paper_1410_1914_gb300 import _lib as L
    ph, react, params = inputs.make_workload("npmc_cl_400")
    n_cells = ph.size
    out = {"workload": NPMC_DESC, "shape_zyx": list(ph.shape), "storage": "fp16dev",
           "lbm_steps_per_bench_step": K}
    for storage in ("fp16dev", "fp32"):
        s = Solver(ph.shape, storage=storage, stream=int(stream.cuda_stream), check_every=K, **params)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_structure(ph, react)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        for _ in range(3):
            s.solve_budget(K)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n = steps if storage == "fp16dev" else max(3, steps // 4)
        with ClockSampler(local) as clocks:
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(n):
                s.solve_budget(K)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        mlups = n_cells * K / (ms * 1e-3) / 1e6
        launch_s = ms * 1e-3 / K
        rec = {"mlups": mlups, "ms_per_step": ms, "setup_s": setup_s,
               "roofline": {"bound": "hbm", "kernel": "k_march",
                            "achieved": bytes_per_cell(storage) * n_cells / launch_s / 1e9, "peak": peak,
                            "unit": "GB/s", "frac": bytes_per_cell(storage) * n_cells / launch_s / 1e9 / peak,
                            "layout_frac": layout_bytes_per_cell(storage) * n_cells / launch_s / 1e9 / peak},
               "clocks": clocks.summary()}
        if storage == "fp16dev":
            ph_pin = torch.from_numpy(ph).pin_memory()
            re_pin = torch.from_numpy(react).pin_memory()
            E = max(K, (1000 // K) * K)
            reps = 2
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                L.cl_lbm_set_structure(s.h, ph_pin, re_pin, n_cells)
                s.solve_budget(E)
                s.reaction_rate()
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            rec["e2e"] = {"value": n_cells * E * reps / el / 1e6, "unit": "MLUPS",
                          "h2d_bytes_per_step": int(ph.nbytes + react.nbytes),
                          "d2h_bytes_per_step": int(40 * ph.shape[2] + 56 * (E // K) + 4 + 8 + 56),
                          "lbm_steps_per_e2e_step": E,
                          "includes": "structure upload + GPU set-up + steps + readout"}
            out.update(rec)
        else:
            out["fp32_state"] = {k: rec[k] for k in ("mlups", "roofline")}
        s.close()
    return out


def measure_ttc(local: int):
    """Time to D_eff within 1e-3 on the 128^3 D_eff set-up of the Pt recipe
    (the converge workload): plain FP32 populations and the FP32 state from
    the linear ramp, the FP16 state from the learned warm start, and the
    steady state found directly by the diffusion-preconditioned Krylov solve."""
    ns = argparse.Namespace(shape=(128, 128, 128), carrier="o2", check_every=500, max_steps=3_000_000,
                            lattice="d3q7", no_warm=False, krylov=False, krylov_max_iter=20000, arms=None)
    with ClockSampler(local) as clocks:
        line = measure_converge(ns, arm_names=("fp32pop", "fp32", "fp16dev+warm", "fp32pop+krylov_dsa"))
    line["clocks"] = clocks.summary()
    return line


def run_unet(args):
    """One training step of the warm-start network (forward, masked-MSE
    backward through every layer, Adam) on a batch of 4 cubes of 48^3 with
    synthetic features and targets, and the per-layer convolution kernels
    (forward, data gradient, weight gradient) timed alone.  Roofline: the
    convolutions' FLOPs against the measured dense BF16 tensor peak."""
    import ctypes

    import torch
    from paper_1410_1914_gb300 import warmstart as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    N, D = 4, 48
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(N, D, D, D, W.FEATURES, device="cuda", generator=g).to(torch.bfloat16)
    tgt = torch.randn(N * D ** 3, device="cuda", generator=g)
    mask = (torch.rand(N * D ** 3, device="cuda", generator=g) < 0.5).to(torch.uint8)
    net = W.UNet(seed=0)
    levels = {"e1": 1, "d1": 1, "e2": 2, "d2": 2, "e3": 3, "d3": 3, "bt": 4}
    step_flop = 0.0
    for name, ci, co in W.CONV_LAYERS:
        d = D >> (levels[name[:2]] - 1)
        passes = 2 if name == "e1a" else 3  # the first layer needs no data gradient
        step_flop += passes * 2.0 * 27 * ci * co * N * d ** 3

    def train_step():
        net.forward(x, N, D)
        net.backward(tgt, mask)
        net.step(lr=1e-4)

    for _ in range(args.warmup):
        train_step()
    net.check()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            train_step()
        e1.record(stream)
        torch.cuda.synchronize()
    net.check()
    ms = e0.elapsed_time(e1) / args.steps
    # per-layer kernels alone
    layers = []
    conv_ms = 0.0
    for name, ci, co in W.CONV_LAYERS:
        d = D >> (levels[name[:2]] - 1)
        M = N * d ** 3
        xi = torch.randn(M * ci, device="cuda", generator=g).to(torch.bfloat16)
        wi = (torch.randn(27 * co * ci, device="cuda", generator=g) * 0.05).to(torch.bfloat16)
        yo = torch.empty(M * co, device="cuda", dtype=torch.bfloat16)
        gy = torch.randn(M * co, device="cuda", generator=g).to(torch.bfloat16)
        gx = torch.empty(M * ci, device="cuda", dtype=torch.bfloat16)
        wd = torch.empty_like(wi)
        W._call("cl_nn_wt_dgrad", W._p(wi), W._p(wd), co, ci, sp)
        dw = torch.empty(27 * co * ci, device="cuda")
        ws = torch.empty(W._lib().cl_nn_wgrad_workspace(N, d, d, d, ci, co) // 4 + 1, device="cuda")
        runs = {
            "fwd": lambda: W._call("cl_nn_conv3d", W._p(xi), W._p(wi), None, W._p(yo), N, d, d, d, ci, co, ci, 0, co, 0,
                                   1, 1, sp),
            "dgrad": lambda: W._call("cl_nn_conv3d", W._p(gy), W._p(wd), None, W._p(gx), N, d, d, d, co, ci, co, 0, ci,
                                     0, 0, 1, sp),
            "wgrad": lambda: W._call("cl_nn_conv3d_wgrad", W._p(xi), W._p(gy), W._p(ws), W._p(dw), N, d, d, d, ci, co,
                                     ci, 0, co, 0, 1, sp),
        }
        row = {"layer": name, "edge": d, "ci": ci, "co": co}
        flop = 2.0 * 27 * ci * co * M
        for k, f in runs.items():
            if k == "dgrad" and name == "e1a":
                continue
            for _ in range(3):
                f()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(10):
                f()
            b.record(stream)
            torch.cuda.synchronize()
            kms = a.elapsed_time(b) / 10
            conv_ms += kms
            row[k + "_ms"] = round(kms, 4)
            row[k + "_tflops"] = round(flop / (kms * 1e-3) / 1e12, 1)
        layers.append(row)
    net.check()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, peak_kind = float(json.load(fh)["bf16_tflops"]), "measured bf16_tflops (burst)"
    except (OSError, KeyError, ValueError):
        peak, peak_kind = 1900.0, "fallback"
    achieved = step_flop / (conv_ms * 1e-3) / 1e12
    line = {
        "metric": "warm-start network training step (4 x 48^3, forward + backward + Adam)",
        "value": 1e3 / ms, "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "U-Net 16/32/64/128 channels, 1,466,065 parameters, batch 4 x 48^3 x 16 features",
                   "conv_flop_per_step": step_flop},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind,
                     "kernel": "convolution kernels (sum of per-layer times alone)"},
        "conv_ms_per_step_alone": conv_ms,
        "layers": layers,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp16dev", choices=["fp32", "fp16dev", "fp32pop"])
    ap.add_argument("--lattice", default="d3q7", choices=["d3q7", "d3q19"],
                    help="d3q19: the paper's 19-velocity lattice (19 f32 populations)")
    ap.add_argument("--no-other-storages", action="store_true",
                    help="skip the short timing of the other storage modes")
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-lbm-steps", type=int, default=1000)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-steps-per-step", type=int, default=1)
    ap.add_argument("--shape", type=int, nargs=3, default=None, help="override (nz ny nx)")
    ap.add_argument("--workload", default="pt_cl_256",
                    choices=["pt_cl_256", "batch64", "converge", "unet_train", "structures"])
    ap.add_argument("--max-steps", type=int, default=3_000_000)
    ap.add_argument("--no-warm", action="store_true", help="converge workload: skip the learned warm-start arms")
    ap.add_argument("--krylov", action="store_true",
                    help="converge workload: add the mixed-precision Krylov steady solves (BiCGSTAB; on D3Q7 also "
                         "the diffusion-preconditioned GMRES and the line-eliminated FGMRES) on plain f32 populations")
    ap.add_argument("--krylov-max-iter", type=int, default=20000)
    ap.add_argument("--arms", default=None,
                    help="converge workload: comma-separated arms to run (e.g. fp16dev+warm,fp32pop+krylov_dsa); "
                         "default: all storage arms, and the steady-solve arms with --krylov")
    ap.add_argument("--no-ttc", action="store_true",
                    help="default workload: skip the time-to-converged D_eff arms (128^3)")
    ap.add_argument("--no-npmc", action="store_true",
                    help="default workload: skip the 400^3 NPMC measurement")
    ap.add_argument("--no-batch", action="store_true",
                    help="default workload: skip the batch of 64 structures (FP16 state, 5 intervals)")
    ap.add_argument("--carrier", default="o2", choices=["o2", "proton"],
                    help="converge workload: O2 in the pores (D_eff) or protons in the ionomer (sigma_eff)")
    args = ap.parse_args()
    if args.shape:
        args.shape = tuple(args.shape)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "converge":
        return run_converge(args)
    if args.workload == "unet_train":
        return run_unet(args)
    if args.workload == "structures":
        return run_structures(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1410_1914_gb300 import Solver, inputs
    from paper_1410_1914_gb300 import _lib as L

    from paper_1410_1914_gb300.replicas import aggregate_rate, max_over_ranks, rank_seed
    ph, react, params = inputs.make_workload(WORKLOAD, shape=args.shape, seed=rank_seed(1, rank))
    n_cells = ph.size
    K = args.check_every
    stream = torch.cuda.current_stream()
    s = Solver(ph.shape, storage=args.storage, stream=int(stream.cuda_stream), check_every=K,
               lattice=args.lattice, **params)
    t0 = time.perf_counter()
    s.set_structure(ph, react)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = s.info()

    for _ in range(args.warmup):
        s.solve_budget(K)
    torch.cuda.synchronize()

    # ---------------------------------------------------------- timed region
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        last = None
        for _ in range(args.steps):
            last = s.solve_budget(K)
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    mlups = aggregate_rate(n_cells * K * args.steps, world, elapsed_ms * 1e-3) / 1e6
    ms_per_step = elapsed_ms / args.steps

    # roofline of the fused step kernel (average launch = interval time / K)
    launch_bytes = bytes_per_cell(args.storage, args.lattice) * n_cells
    launch_s = ms_per_step * 1e-3 / K
    peak, peak_kind = measured_peak_gbs()
    achieved = launch_bytes / launch_s / 1e9
    traffic, traffic_src = measured_traffic(args.storage, n_cells, args.lattice)
    layout_frac = layout_bytes_per_cell(args.storage, args.lattice) * n_cells / launch_s / 1e9 / peak
    dram_frac = None if traffic is None else traffic / launch_s / 1e9 / peak

    # the other storage modes and lattices on the same structure, for context (not the headline)
    others = {}
    if not args.no_other_storages:
        for st, lat in (("fp32", "d3q7"), ("fp16dev", "d3q7"), ("fp32pop", "d3q7"), ("fp32", "d3q19"),
                        ("fp16dev", "d3q19"), ("fp32pop", "d3q19")):
            if st == args.storage and lat == args.lattice:
                continue
            so = Solver(ph.shape, storage=st, stream=int(stream.cuda_stream), check_every=K, lattice=lat,
                        **params)
            so.set_structure(ph, react)
            for _ in range(3):
                so.solve_budget(K)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                so.solve_budget(K)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 5
            v = n_cells * K / (ms * 1e-3) / 1e6
            others[st if lat == "d3q7" else f"{lat}_{st}"] = {
                "mlups": v, "hbm_frac": bytes_per_cell(st, lat) * n_cells / (ms * 1e-3 / K) / 1e9 / peak,
                "layout_frac": layout_bytes_per_cell(st, lat) * n_cells / (ms * 1e-3 / K) / 1e9 / peak}
            so.close()

    # ---------------------------------------------------------- end to end
    # Through the public API with host buffers: pinned host structure ->
    # set_structure -> e2e_lbm_steps steps -> reaction rate to the host.
    e2e = None
    if args.e2e_steps > 0:
        ph_pin = torch.from_numpy(ph).pin_memory()
        re_pin = torch.from_numpy(react).pin_memory() if react is not None else None
        E = max(K, (args.e2e_lbm_steps // K) * K)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            L.cl_lbm_set_structure(s.h, ph_pin, re_pin, n_cells)
            s.solve_budget(E)
            R_tot, prof_R, prof_C = s.reaction_rate()
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        # device-to-host: 5 FP64 plane sums per x-plane for the readout, one
        # 7-slot FP64 check per interval, the set-up's error words and counters
        d2h = 40 * ph.shape[2] + 56 * (E // K) + 4 + 8 + 56
        e2e = {"value": aggregate_rate(n_cells * E * args.e2e_steps, world, el) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(ph.nbytes + (react.nbytes if react is not None else 0)),
               "d2h_bytes_per_step": int(d2h),
               "lbm_steps_per_e2e_step": E, "includes": "structure upload + GPU set-up + steps + readout"}

    line = {
        "metric": "MLUPS (%s fused collide-stream step, all box cells)" % args.lattice.upper(),
        "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "shape_zyx": list(ph.shape), "storage": args.storage,
                   "lattice": args.lattice,
                   "lbm_steps_per_bench_step": K, "active_fraction": info["n_active"] / n_cells,
                   "l2": "inputs larger than L2 (state buffers 2 x %.0f MB)" % (
                       (layout_bytes_per_cell(args.storage, args.lattice) - (8 if args.lattice == "d3q19" else 6))
                       / 2 * n_cells / 1e6),
                   "parallelism": f"replicas x{world}", "setup_s": setup_s},
        "active_mlups": mlups * info["n_active"] / n_cells,
        "other_storages": others,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": traffic_src,
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": launch_bytes,
                     "algorithmic_bytes_per_cell": bytes_per_cell(args.storage, args.lattice),
                     "layout_bytes_per_cell": layout_bytes_per_cell(args.storage, args.lattice),
                     "layout_frac": layout_frac,
                     "dram_frac": dram_frac,
                     "kernel": ("k_step19" if args.lattice == "d3q19" and args.storage == "fp32pop" else
                                "k_step19s" if args.lattice == "d3q19" else
                                "k_step_fp32" if args.storage == "fp32pop" else "k_march")},
        "gpu_launches": args.steps * (K + 1),
        "clocks": clocks.summary(),
        "e2e": e2e,
        "last_check": {k: last[k] for k in ("J_in", "J_out", "R", "flux_balance", "resid")},
    }
    s.close()
    if world == 1 and args.lattice == "d3q7" and args.shape is None:
        if not args.no_npmc:
            line["npmc_400"] = measure_npmc400(stream, K, args.steps, peak, local)
        if not args.no_ttc:
            line["ttc"] = measure_ttc(local)
        if not args.no_batch:
            try:
                line["batch64"] = measure_batch64("fp16dev", K, 5, 3, stream)
            except Exception as e:  # reported in the line, which is printed either way
                line["batch64"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ph, react, params, args.cpu_budget, args.lattice)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

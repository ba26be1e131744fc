#!/usr/bin/env python
"""Benchmark of the mEVP momentum subcycle on GB300.

One step = one outer time step of the hot path: mevp_begin_step (ice
strength, lumped mass, forcing) followed by the workload's n_sub mEVP
subcycles (strain, stress, divergence, velocity), on synthetic seeded inputs
resident in HBM.  Metric: element-subcycles per second (N_e * n_sub per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--precision fp64|mixed] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the plain restatement of the
method the GPU path is checked against) on the host cores, on a bounded
sample of the same workload.  With N > 1 (torchrun) every rank runs an
independent replica of the workload (the hot path needs no collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2402_00466_gb300 import workloads as W  # noqa: E402

METRIC = "mEVP element-subcycles/s & % HBM peak, FP64 vs mixed at stated field error"
UNIT = "element-subcycles/s"

# Algorithmic work per element and subcycle of the element kernel, counted
# from its operator sparsity (FMA = 2 flops, mul/add = 1, rsqrt = 1; zero
# entries skipped, +-1 entries as adds).  DG2: projected derivatives 268,
# Gauss evaluation 132, rheology 99, projection 240, update 62, element
# forces 254.  DG1: 153, 36, 44, 63, 32, 146.
ELEM_FLOPS = {3: 474, 6: 1055}
NODE_FLOPS_PER_NODE = 32.5          # node kernel (force gather, velocity update)
# Algorithmic HBM bytes per element-subcycle: state touched once (stress R+W,
# ice strength, vertices amortised, 4 nodes x (v R, v W, node constants R)).
HBM_BYTES = {("fp64", 6): 608, ("fp64", 3): 464}

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 vector peak: 152 SMs x 2 FP64 FMA/clk/SM (measured 1.90 by a throughput
# probe) x 2 flop x 2.07 GHz max SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(case, budget_s=12.0, max_sub=400):
    """Time the FP64 oracle (OpenMP build, all host cores) on a bounded sample."""
    import oracle
    args = (case["nx"], case["ny"], case["xy"], case["n_s"], 1, case["params"], case["H"],
            case["A"], case["tau"], case["vel0"], case["S0"])
    oracle.subcycles(*args, 1, openmp=True)  # first touch, thread start-up
    t0 = time.perf_counter()
    oracle.subcycles(*args, 3, openmp=True)
    t1 = (time.perf_counter() - t0) / 3
    k = int(max(1, min(max_sub, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    oracle.subcycles(*args, k, openmp=True)
    dt = time.perf_counter() - t0
    ne = case["nx"] * case["ny"]
    return {"value": ne * k / dt, "unit": UNIT, "cores": oracle.max_threads(True),
            "kind": "oracle",
            "sample": f"{k} subcycles of {case['name']} ({ne} elements), FP64 C oracle, OpenMP",
            "seconds": dt}


def run_reference(a):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    case = W.make_case(a.workload)
    ne = case["nx"] * case["ny"]
    args = (case["nx"], case["ny"], case["xy"], case["n_s"], 1, case["params"], case["H"],
            case["A"], case["tau"], case["vel0"], case["S0"])
    t0 = time.perf_counter()
    oracle.subcycles(*args, 1, openmp=True)
    t1 = time.perf_counter() - t0
    k_sub = int(max(1, min(case["n_sub"], 6.0 / max(t1, 1e-6))))  # ~6 s per step
    for _ in range(a.warmup):
        oracle.subcycles(*args, 1, openmp=True)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.subcycles(*args, k_sub, openmp=True)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = ne * k_sub * a.steps / total
    cores = oracle.max_threads(True)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": a.workload, "nx": case["nx"], "ny": case["ny"],
                   "n_stress": case["n_s"], "n_sub_per_step": k_sub,
                   "n_sub_workload": case["n_sub"], "precision": "fp64",
                   "alpha": case["params"]["alpha"], "beta": case["params"]["beta"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{k_sub} of {case['n_sub']} subcycles per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_2402_00466_gb300 import mevp

    ws, rank, local = dist_setup()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if ws > 1:
            dist.barrier()

    case = W.make_case(a.workload)
    nx, ny, ns, n_sub = case["nx"], case["ny"], case["n_s"], case["n_sub"]
    ne, nn, _ = W.sizes(nx, ny)
    st = mevp.State(nx, ny, ns, vertex_xy=case["xy"], precision=a.precision,
                    params=case["params"])
    st.set_ice(case["H"], case["A"])
    st.set_forcing(case["tau"])
    st.set_velocity(case["vel0"])
    st.set_stress(case["S0"])
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def step():
        st.begin_step()
        st.run_subcycles(n_sub)

    for _ in range(a.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    st.timing_enable(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(a.steps)]
    t_wall0 = time.perf_counter()
    for k in range(a.steps):
        flush.zero_()  # L2 flush between timed steps, outside the step events
        evs[k][0].record()
        step()
        evs[k][1].record()
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    kt = st.timing_read()
    st.timing_enable(False)
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in evs]
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    units = ws * ne * n_sub * a.steps
    value = units / (total_ms / 1e3)

    # dominant kernel: the element kernel; achieved = algorithmic flops per launch / mean launch time
    el_ms, el_n = kt["element"]
    nd_ms, nd_n = kt["node"]
    el_avg_s = el_ms / max(el_n, 1) / 1e3
    flops_launch = ELEM_FLOPS[ns] * ne
    achieved_tflops = flops_launch / el_avg_s / 1e12
    hbm_peak, hbm_kind = load_peaks()
    bytes_sub = HBM_BYTES.get((a.precision, ns), 0) * ne
    sub_s = (total_ms / 1e3) / (n_sub * a.steps)
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": f"k_element_f64<{ns}>", "peak_kind": "derived (FP64 pipe, max clock)",
                "kernel_ms_mean": el_avg_s * 1e3, "node_kernel_ms_mean": nd_ms / max(nd_n, 1),
                "kernel_share_of_subcycle": el_ms / max(el_ms + nd_ms, 1e-12),
                "hbm_algorithmic_GBps": bytes_sub / sub_s / 1e9,
                "hbm_frac": bytes_sub / sub_s / 1e9 / hbm_peak, "hbm_peak_GBps": hbm_peak,
                "hbm_peak_kind": hbm_kind}

    # end to end through the public API with pinned host buffers
    e2e = None
    if not a.no_e2e:
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()  # noqa: E731
        hH, hA, htau = pin(case["H"]), pin(case["A"]), pin(case["tau"])
        hv, hS = pin(case["vel0"]), pin(case["S0"])
        outs = {f: torch.empty(st.field_shape(f), dtype=torch.float64).pin_memory()
                for f in ("U", "V", "S11", "S12", "S22")}
        e2e_steps = max(1, min(a.steps, 3))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            st.set_ice(hH, hA)
            st.set_forcing(htau)
            st.set_velocity(hv)
            st.set_stress(hS)
            st.begin_step()
            st.run_subcycles(n_sub)
            for f, o in outs.items():
                mevp.mevp_read_field(st.state, f, o)
        torch.cuda.synchronize()
        barrier()
        dt = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([dt], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        h2d = 8 * (2 * ne + 2 * nn + 2 * nn + 3 * ns * ne)
        d2h = 8 * (2 * nn + 3 * ns * ne)
        e2e = {"value": ws * ne * n_sub * e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(case)

    st.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if a.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": a.workload, "nx": nx, "ny": ny, "n_stress": ns,
                       "n_sub": n_sub, "precision": a.precision,
                       "alpha": case["params"]["alpha"], "beta": case["params"]["beta"],
                       "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": a.steps * (2 + 2 * n_sub),
            "clocks": clk, "wall_s": t_wall,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="mesh256_dg2", choices=sorted(W.CONFIGS))
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    a = ap.parse_args()
    if a.warmup < 3 and a.impl == "ours":
        ap.error("--warmup must be >= 3")
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())

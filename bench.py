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
# entries skipped, +-1 entries as adds).  The strain and force operators are
# sum-factorised (two 1-D passes).  DG2: projected derivatives 204, Gauss
# evaluation 132, rheology 99, projection 240, update 62, element forces 182.
# DG1: 145, 36, 44, 63, 32, 130.  (Applied directly, without the
# factorisation, the two operators cost 268 and 254 (DG2), 153 and 146 (DG1).)
ELEM_FLOPS = {3: 450, 6: 919}
# The same count for the general-quad element kernel k_element_gen (bilinear
# map per element, Gauss-point strain, stress and forces with det J
# cancelled; the L D L^T factor of the local mass matrix is read from the
# per-element records written at state creation): DG2 = map 18, reference
# gradients 252, strain integrands 165, moments 195 + 195, solves
# 198 + 198, invariants 24, Gauss evaluation 132 + 132, rheology 183,
# update 61, force integrands 192, force sums 270.
GEN_ELEM_FLOPS = {3: 1019, 6: 2215, 8: 2675}
# Isoparametric (curved Q2) elements, k_element_iso: the same stages with the
# Jacobians at the Gauss points read from the per-element records (no map
# coefficients and no Jacobian arithmetic in the strain, rheology and force
# integrands).
ISO_ELEM_FLOPS = {3: 905, 6: 2053, 8: 2513}
# Transport step (k_advect, rectilinear mesh), per element and Runge-Kutta
# stage: volume terms at NQ x NQ points (velocity, contravariant flux,
# traces, basis gradients), NQ points on each of the 4 edges (velocity,
# normal flux, upwind trace, test functions), inverse mass, stage
# combination.  Stages per step: 1 (DG0), 2 (DG1), 3 (DG2).
ADV_FLOPS = {1: 195, 3: 885, 6: 2628}
# Gradient of the kinetic energy (hand-written reverse mode), per element and
# subcycle of the objective: the forward subcycle twice (checkpointed sweep and
# the per-segment recomputation: element kernel + 4 nodes of the node kernel)
# plus the reverse element kernel (forward recompute of strain and Gauss
# values 189 / 400, transposed divergence, reverse rheology and projection,
# transposed strain operator: 840 (DG1) / 1844 (DG2)) and 4 nodes of the
# reverse node kernel (~47 flops: transposed 2x2 solve, drag derivative).
ADJ_ELEM_FLOPS = {3: 840, 6: 1844}
ADJ_NODE_FLOPS = 47
ADV_STAGES = {1: 1, 3: 2, 6: 3}
NODE_FLOPS_PER_NODE = 32.5          # node kernel (force gather, velocity update)
# Algorithmic HBM bytes per element-subcycle: state touched once (stress R+W,
# ice strength, vertices amortised, 4 nodes x (v R, v W, node constants R)).
HBM_BYTES = {("fp64", 6): 608, ("fp64", 3): 464}

# DRAM bytes per launch of the dominant kernel, from one ncu capture of the
# same command line (ncu flushes the caches before a profiled launch, so this
# is the launch's cold-cache traffic); keyed by (workload, precision, kernel)
# and valid while that kernel is unchanged.  Summaries: profiles/.
NCU_TRAFFIC = {
    ("mesh1024_dg2", "fp64", "k_element_f64<6>"): 234397440 + 248332032,
    ("mesh1024_dg2", "mixed", "k_subcycle_mix<6,32,8>"): 214099456 + 105171968,
    ("mesh256_dg2_iso", "fp64", "k_element_iso<6>"): 44171776 + 55296000,
}

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 vector peak: SMs x 2 FP64 FMA/clk/SM (a throughput probe measured 1.90)
# x 2 flop x the maximum SM clock; the SM count comes from the device and the
# clock from nvidia-smi's clocks.max.sm (2070 MHz on GB300 when unavailable).
FP64_FMA_PER_CLK_SM = 2
FP32_FMA_PER_CLK_SM = 128


def sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def max_sm_mhz(clk=None):
    if clk and clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"])
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits", "-i", "0"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        return float(out.splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return 2070.0


def fp64_peak_tflops(clk=None):
    return sm_count() * FP64_FMA_PER_CLK_SM * 2 * max_sm_mhz(clk) * 1e6 / 1e12


def fp64_peak_kind(clk=None):
    return (f"derived: FP64 pipe {sm_count()} SM x {FP64_FMA_PER_CLK_SM} FMA/clk x 2 flop x "
            f"{max_sm_mhz(clk):.0f} MHz (max SM clock)")


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


def reduce_max(value: float, dist, device) -> float:
    """Max of a per-rank float over all ranks (timings: the slowest rank
    defines the whole job's time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return world * units_per_rank / max_seconds


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
    ph = np.zeros(4)
    t0 = time.perf_counter()
    oracle.subcycles(*args, k, openmp=True, phase_sec=ph)
    dt = time.perf_counter() - t0
    ne = case["nx"] * case["ny"]
    # the four stages of Table 1 (strain, stress, divergence, velocity), per
    # subcycle: OpenMP on all host cores, and serial on a shorter sample
    ks = int(max(1, min(20, 4.0 / max(t1 * oracle.max_threads(True), 1e-6))))
    phs = np.zeros(4)
    oracle.subcycles(*args, ks, openmp=False, phase_sec=phs)
    names = ("strain", "stress", "divergence", "velocity")
    return {"value": ne * k / dt, "unit": UNIT, "cores": oracle.max_threads(True),
            "kind": "oracle",
            "sample": f"{k} subcycles of {case['name']} ({ne} elements), FP64 C oracle, OpenMP",
            "seconds": dt,
            "stage_ms_per_subcycle_openmp": {n: 1e3 * v / k for n, v in zip(names, ph)},
            "stage_ms_per_subcycle_serial": {n: 1e3 * v / ks for n, v in zip(names, phs)},
            "serial_sample": f"{ks} subcycles, 1 core"}


def run_reference(a):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    case = W.make_case(a.workload)
    if case["n_sub"] == 0:
        return run_reference_advection(a, case)
    ne = case["nx"] * case["ny"]
    args = (case["nx"], case["ny"], case["xy"], case["n_s"], 1, case["params"], case["H"],
            case["A"], case["tau"], case["vel0"], case["S0"])
    # a call of the oracle has a fixed cost (element geometry and the lumped
    # mass, serial) besides its subcycles: size each step from the marginal
    # cost of a subcycle, about 5 s of work per step
    t0 = time.perf_counter()
    oracle.subcycles(*args, 1, openmp=True)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.subcycles(*args, 3, openmp=True)
    t3 = time.perf_counter() - t0
    per_sub = max((t3 - t1) / 2, 1e-6)
    fixed = max(t1 - per_sub, 0.0)
    k_sub = int(max(1, min(case["n_sub"], (5.0 - fixed) / per_sub)))
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


def advection_sample(case, nxs=128):
    """A bounded CPU sample of a transport workload: the nxs x nxs corner of
    its mesh, ice fields and a velocity of the same recipe."""
    nx, ny, na = case["nx"], case["ny"], case["n_a"]
    L = case["L"]
    xs = W.uniform_vertices(nxs, nxs, L * nxs / nx, L * nxs / ny)
    Hs = case["H"].reshape(na, ny, nx)[:, :nxs, :nxs].reshape(na, -1)
    As = case["A"].reshape(na, ny, nx)[:, :nxs, :nxs].reshape(na, -1)
    vs = W.smooth_velocity(nxs, nxs, 15, amp=0.3, L=L * nxs / nx)
    return nxs, xs, Hs, As, vs


def run_reference_advection(a, case):
    import oracle
    na = case["n_a"]
    nxs, xs, Hs, As, vs = advection_sample(case)
    dt = case["params"]["dt"]
    for _ in range(a.warmup):
        oracle.advect(nxs, nxs, xs, na, vs, dt, 1, Hs, As, openmp=True)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.advect(nxs, nxs, xs, na, vs, dt, 1, Hs, As, openmp=True)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = nxs * nxs * a.steps / total
    unit = "element-steps/s"
    line = {
        "impl": "reference", "metric": "DG upwind advection of H and A: element-steps/s",
        "value": value, "unit": unit, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": a.workload, "nx": case["nx"], "ny": case["ny"], "n_adv": na},
        "cpu_baseline": {"value": value, "unit": unit, "cores": oracle.max_threads(True),
                         "kind": "oracle",
                         "sample": f"one advection step of a {nxs}x{nxs} corner per step"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# Mixed path, one fused launch per subcycle.  Algorithmic HBM bytes per
# element-subcycle of the workload's single-pass count (FP32 stress
# R+W, FP32 H and A, vertices, 4 nodes x (FP64 v R + W, v^n R, tau R, m R)):
# 424 B for DG2; the same count gives 352 B for DG1.  This design touches
# fewer: FP32 stress R+W, FP32 ice strength, 4 nodes x (16 B velocity record
# R + W, 16 B constant record R) = 340 B (DG2) / 268 B (DG1).
MIXED_SINGLE_PASS_BYTES = {6: 424, 3: 352}
MIXED_OWN_BYTES = {6: 144 + 4 + 4 * 48, 3: 72 + 4 + 4 * 48}
# subcycles of the untimed run that splits the FP64 subcycle time between its
# element and node kernels (per-kernel CUDA events around every launch)
SPLIT_SUBCYCLES = 40


def fp32_peak_tflops(clk=None):
    return sm_count() * FP32_FMA_PER_CLK_SM * 2 * max_sm_mhz(clk) * 1e6 / 1e12


def measure(mevp, torch, barrier, ws, case, precision, steps, warmup, flush):
    """Time `steps` outer steps (begin_step + n_sub subcycles) after `warmup`,
    L2 flushed between steps, with three CUDA events per step on the launching
    stream: before begin_step, between begin_step and the subcycles, after the
    subcycles (the subcycle loop itself is not interrupted, so its CUDA-graph
    replay is what is timed).  For the FP64 path an untimed run afterwards
    brackets every element and node launch with events, for the split of the
    subcycle time between the two kernels."""
    nx, ny, ns, n_sub = case["nx"], case["ny"], case["n_s"], case["n_sub"]
    ne = nx * ny
    st = mevp.State(nx, ny, ns, vertex_xy=case["xy"], precision=precision,
                    params=case["params"])
    st.set_ice(case["H"], case["A"])
    st.set_forcing(case["tau"])
    st.set_velocity(case["vel0"])
    st.set_stress(case["S0"])
    for _ in range(warmup):
        flush.zero_()
        st.begin_step()
        st.run_subcycles(n_sub)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(steps)]
    t0 = time.perf_counter()
    for k in range(steps):
        flush.zero_()  # L2 flush between timed steps, outside the step events
        evs[k][0].record()
        st.begin_step()
        evs[k][1].record()
        st.run_subcycles(n_sub)
        evs[k][2].record()
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    total_ms = sum(a.elapsed_time(c) for a, _, c in evs)
    begin_ms = sum(a.elapsed_time(b) for a, b, _ in evs)
    sub_ms = sum(b.elapsed_time(c) for _, b, c in evs)
    split = None
    if precision == "fp64":
        st.timing_enable(1)
        st.run_subcycles(SPLIT_SUBCYCLES)
        kt = st.timing_read()
        st.timing_enable(0)
        el_ms, nd_ms = kt["element"][0], kt["node"][0]
        split = {"element": el_ms / (el_ms + nd_ms), "node": nd_ms / (el_ms + nd_ms),
                 "subcycles": kt["element"][1],
                 "how": "per-kernel CUDA events around every launch of an untimed run of "
                        f"{SPLIT_SUBCYCLES} direct (non-graph) subcycles"}
    return dict(state=st, total_ms=total_ms, begin_ms=begin_ms, sub_ms=sub_ms, split=split,
                wall=wall, value=ws * ne * n_sub * steps / (total_ms / 1e3))


def roofline_for(precision, case, m, steps, clk):
    """Roofline of the dominant kernel from the timed region: the subcycle
    time per launch (CUDA events around the uninterrupted subcycle loop) --
    for the FP64 path its element-kernel share from the split run."""
    ns, ne, n_sub = case["n_s"], case["nx"] * case["ny"], case["n_sub"]
    _, nn, _ = W.sizes(case["nx"], case["ny"])
    sub_s = (m["sub_ms"] / 1e3) / (n_sub * steps)
    hbm_peak, hbm_kind = load_peaks()
    geo = case.get("geometry", "uniform")
    general = geo != "uniform"
    iso = geo in ("wavy_iso", "curved")
    if precision == "fp64":
        table = ISO_ELEM_FLOPS if iso else (GEN_ELEM_FLOPS if general else ELEM_FLOPS)
        share = m["split"]["element"]
        el_s = sub_s * share
        ach = table[ns] * ne / el_s / 1e12
        peak = fp64_peak_tflops(clk)
        bytes_sub = HBM_BYTES.get(("fp64", ns), 0) * ne
        sub_flops = table[ns] * ne + NODE_FLOPS_PER_NODE * nn
        kern = ((f"k_element_iso<{ns}>" if iso else f"k_element_gen<{ns}>") if general
                else f"k_element_f64<{ns}>")
        r = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
             "frac": ach / peak, "traffic": None, "kernel": kern,
             "flops_per_element": table[ns],
             "kernel_ms_mean": el_s * 1e3,
             "kernel_time_source": "subcycle time of the timed region x element share "
                                   f"{share:.4f} of the split run",
             "peak_kind": fp64_peak_kind(clk),
             "subcycle_ms_mean": sub_s * 1e3,
             "subcycle_TFLOPs": sub_flops / sub_s / 1e12,
             "subcycle_frac": sub_flops / sub_s / 1e12 / peak,
             "hbm_algorithmic_GBps": bytes_sub / sub_s / 1e9,
             "hbm_frac": bytes_sub / sub_s / 1e9 / hbm_peak}
    else:
        # one fused launch per subcycle: its mean duration is at most the
        # subcycle time (the launch gaps of the graph replay included)
        nsm = sm_count()
        big = ((case["nx"] + 29) // 31) * ((case["ny"] + 5) // 7) >= 16 * nsm
        # FP32 map record (A, B, c) per bilinear element, 8 FP32 node offsets
        # per isoparametric element, and on both the FP32 mass-matrix factor
        extra = (64 if iso else 24) + 4 * ns * (ns + 1) // 2 if general else 0
        byts = MIXED_SINGLE_PASS_BYTES[ns] + extra
        ach = byts * ne / sub_s / 1e9
        own = (MIXED_OWN_BYTES[ns] + extra) * ne / sub_s / 1e9
        kern = f"k_subcycle_mix{'_iso' if iso else '_gen' if general else ''}<{ns},32,{8 if big else 4}>"
        r = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
             "frac": ach / hbm_peak, "traffic": None, "kernel": kern,
             "kernel_ms_mean": sub_s * 1e3,
             "kernel_time_source": "subcycle time of the timed region (one launch per subcycle)",
             "peak_kind": f"{hbm_kind} (MEASURED_PEAKS.json hbm_gbs)",
             "bytes_per_element": byts,
             "bytes_source": "single-pass count: stress R+W, H, A, vertices, 4 nodes x "
                             "(v R+W, v^n, tau, m)"
                             + (" + FP32 geometry and mass-factor records" if general else ""),
             "own_bytes_per_element": MIXED_OWN_BYTES[ns] + extra,
             "achieved_own_bytes": own, "frac_own_bytes": own / hbm_peak,
             "fp32_TFLOPs_approx": (ELEM_FLOPS[ns] * 1.1 + 4 * 40) * ne / sub_s / 1e12,
             "fp32_peak_TFLOPs": fp32_peak_tflops(clk)}
    r["traffic"] = NCU_TRAFFIC.get((case["name"], precision, r["kernel"]))
    if r["traffic"] is not None:
        r["traffic_note"] = "ncu dram__bytes_read+write per launch, cold cache"
    return r


def end_to_end(mevp, torch, barrier, ws, case, st, steps):
    """The same metric through the public API with host buffers: every step
    copies its inputs from pinned host memory (ice, forcing, velocity,
    stress), runs begin_step + n_sub subcycles, and reads velocity and stress
    back to pinned host memory."""
    nx, ny, ns, n_sub = case["nx"], case["ny"], case["n_s"], case["n_sub"]
    ne, nn, _ = W.sizes(nx, ny)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()  # noqa: E731
    hH, hA, htau = pin(case["H"]), pin(case["A"]), pin(case["tau"])
    hv, hS = pin(case["vel0"]), pin(case["S0"])
    outs = {f: torch.empty(st.field_shape(f), dtype=torch.float64).pin_memory()
            for f in ("U", "V", "S11", "S12", "S22")}
    e2e_steps = max(1, min(steps, 3))
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
    h2d = 8 * (2 * ne + 2 * nn + 2 * nn + 3 * ns * ne)
    d2h = 8 * (2 * nn + 3 * ns * ne)
    return {"value": ws * ne * n_sub * e2e_steps / dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps}, dt


def _rel(x, ref, mask=None):
    x, ref = np.asarray(x, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    if mask is not None:
        x, ref = x[..., mask], ref[..., mask]
    n2, ninf = np.linalg.norm(ref), np.abs(ref).max() if ref.size else 0.0
    return {"rel_l2": float(np.linalg.norm(x - ref) / (n2 if n2 > 0 else 1.0)),
            "rel_max": float(np.abs(x - ref).max() / (ninf if ninf > 0 else 1.0)) if ref.size
            else 0.0}


def field_errors_vs_oracle(mevp, case, n_sub, alpha_beta, precisions=("mixed", "fp64"),
                          checkpoints=None):
    """Per-field errors of the GPU paths against the FP64 oracle after n_sub
    subcycles of one outer step from the workload's initial state: velocity,
    stress, strain (of the final velocity), nodal force (divergence of the
    final stress), and Delta at the Gauss points (of the final strain, both
    evaluated by the oracle), plus the stress error restricted to the rigid
    elements (Delta < 10 Delta_min at some Gauss point of the last update).
    checkpoints (increasing subcycle counts ending at n_sub): velocity and
    stress errors after each, the growth of the discrepancy with p."""
    import oracle
    p = dict(case["params"], alpha=alpha_beta, beta=alpha_beta)
    nx, ny, ns = case["nx"], case["ny"], case["n_s"]
    cps = list(checkpoints) if checkpoints else [n_sub]
    assert cps == sorted(cps) and cps[-1] == n_sub
    t0 = time.perf_counter()
    vel, S, done, orc = case["vel0"], case["S0"], 0, []
    for k in cps:
        out = oracle.subcycles(nx, ny, case["xy"], ns, 1, p, case["H"], case["A"], case["tau"],
                               vel, S, k - done, vn=case["vel0"], want_last=(k == n_sub),
                               openmp=True)
        vel, S, done = out[0], out[1], k
        orc.append((vel, S))
    Elast = out[2]
    t_orc = time.perf_counter() - t0
    vo, So = orc[-1]
    Eo = oracle.strain(nx, ny, case["xy"], ns, vo, openmp=True)
    Fo = oracle.divergence(nx, ny, case["xy"], ns, So, openmp=True)
    Do = oracle.delta(nx, ny, ns, p, Eo)
    rigid = oracle.delta(nx, ny, ns, p, Elast).min(axis=1) < 10 * p["DeltaMin"]
    res = {"n_sub": n_sub, "alpha_beta": alpha_beta, "reference": "FP64 oracle",
           "oracle_seconds": t_orc, "rigid_elements": int(rigid.sum())}
    for prec in precisions:
        with mevp.State(nx, ny, ns, vertex_xy=case["xy"], precision=prec, params=p) as st:
            st.set_ice(case["H"], case["A"])
            st.set_forcing(case["tau"])
            st.set_velocity(case["vel0"])
            st.set_stress(case["S0"])
            st.begin_step()
            done, curve = 0, []
            for k, (vk, Sk) in zip(cps, orc):
                st.run_subcycles(k - done)
                done = k
                curve.append({"p": k, "velocity": _rel(st.velocity(), vk),
                              "stress": _rel(st.stress(), Sk)})
            v, S, E, F = st.velocity(), st.stress(), st.strain(), st.force()
        D = oracle.delta(nx, ny, ns, p, E)
        res[prec] = {"velocity": _rel(v, vo), "stress": _rel(S, So), "strain": _rel(E, Eo),
                     "force": _rel(F, Fo), "delta": _rel(D, Do),
                     "stress_rigid": _rel(S, So, rigid) if rigid.any() else None}
        if len(cps) > 1:
            res[prec]["curve"] = curve
    return res


def field_error_block(mevp, name):
    """The per-field error statement of the benchmark line.
    - "short_horizon": the workload's own mesh at its alpha = beta, with the
      discrepancy after p = 1, 2, 3, 5, 10 subcycles (on meshes this fine the
      iteration amplifies any rounding difference exponentially at that
      alpha, FP64's own included, so the errors are stated at p = 2);
    - "full_horizon_256": the 256 x 256 DG2 mesh over the full 500 subcycles
      at the stability-bound alpha = beta = 2000 (alpha h = 4e6 m)."""
    case = W.make_case(name)
    out = {"short_horizon": field_errors_vs_oracle(mevp, case, 2, case["params"]["alpha"])}
    out["short_horizon_curve"] = field_errors_vs_oracle(mevp, case, 10, case["params"]["alpha"],
                                                        checkpoints=[1, 2, 3, 5, 10])
    c256 = W.make_case("mesh256_dg2")
    out["full_horizon_256"] = field_errors_vs_oracle(mevp, c256, c256["n_sub"], 2000.0)
    return out


def run_ours(a):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_setup()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    # a non-default stream, so that the library can replay subcycles as CUDA
    # graphs; the L2 flush and the timing events go to the same stream
    with torch.cuda.stream(torch.cuda.Stream()):
        return _run_ours(a, torch, dist, ws, rank)


def run_ensemble(a, torch, dist, ws, rank, emit=True):
    """Ensemble workload: all members advanced together (one persistent
    launch per subcycle in the mixed precision), tile shape autotuned.
    Prints the line (emit) and returns it."""
    from paper_2402_00466_gb300 import mevp

    dev = torch.cuda.current_device()
    members = W.make_ensemble(a.workload)
    n_sub = members[0]["n_sub"]
    units_step = sum(c["nx"] * c["ny"] for c in members) * n_sub
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    states = []
    for c in members:
        st = mevp.State(c["nx"], c["ny"], c["n_s"], vertex_xy=c["xy"], precision=a.precision,
                        params=c["params"])
        st.set_ice(c["H"], c["A"])
        st.set_forcing(c["tau"])
        st.set_velocity(c["vel0"])
        st.set_stress(c["S0"])
        states.append(st)
    ens = mevp.Ensemble(states)
    ens.begin_step()
    shape = ens.autotune(10)
    shapes = mevp.mevp_ensemble_shapes(a.precision)

    def timed(step, steps, warmup):
        for _ in range(warmup):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            evs[k][0].record()
            step()
            evs[k][1].record()
        torch.cuda.synchronize()
        return sum(s_.elapsed_time(e_) for s_, e_ in evs)

    def ens_step():
        ens.begin_step()
        ens.run_subcycles(n_sub)

    def seq_step():  # the same members one state at a time
        for st in states:
            st.begin_step()
            st.run_subcycles(n_sub)

    clocks = Clocks(dev)
    clocks.start()
    total_ms = timed(ens_step, a.steps, a.warmup)
    clk = clocks.stop()
    seq_ms = timed(seq_step, 1, 1)
    value = ws * units_step * a.steps / (total_ms / 1e3)
    sub_s = total_ms / 1e3 / (a.steps * n_sub)
    hbm_peak, hbm_kind = load_peaks()
    roofline = None
    if a.precision == "mixed":
        byts = sum(c["nx"] * c["ny"] * MIXED_SINGLE_PASS_BYTES[c["n_s"]] for c in members)
        ach = byts / sub_s / 1e9
        roofline = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                    "frac": ach / hbm_peak, "traffic": None,
                    "kernel": "k_ens_mix<%d,%d>" % shapes[shape],
                    "bytes_per_element": "single-pass count: 424 (DG2) / 352 (DG1)",
                    "peak_kind": hbm_kind}
    else:
        flops = sum(c["nx"] * c["ny"] * ELEM_FLOPS[c["n_s"]] for c in members)
        ach = flops / sub_s / 1e12
        roofline = {"bound": "alu", "achieved": ach, "peak": fp64_peak_tflops(clk), "unit": "TFLOP/s",
                    "frac": ach / fp64_peak_tflops(clk), "traffic": None,
                    "kernel": "k_ens_f64_elem<%d> + k_ens_f64_node" % shapes[shape][0],
                    "note": "whole subcycle (element + node launch) timed"}
    for st in states:
        st.close()
    ens.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": a.workload, "members": len(members),
                   "elements": sum(c["nx"] * c["ny"] for c in members),
                   "dg2_members": sum(c["n_s"] == 6 for c in members), "n_sub": n_sub,
                   "precision": a.precision, "shape": shapes[shape],
                   "l2": "flushed between timed steps (512 MB write)"},
        "roofline": roofline, "sequential_ms_per_step": seq_ms,
        "speedup_vs_sequential": seq_ms / (total_ms / a.steps),
        # per member begin_step (3 kernels, mixed 5); per subcycle one tile
        # launch (mixed) or one element launch per stress space present plus
        # the node launch (FP64)
        "gpu_launches": a.steps * (len(members) * (5 if a.precision == "mixed" else 3) +
                                   n_sub * (1 if a.precision == "mixed" else
                                            1 + len({c["n_s"] for c in members}))),
        "clocks": clk, "cpu_baseline": None, "e2e": None,
    }
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def run_advection(a, torch, dist, ws, rank):
    """Transport workload: `steps` advection steps of DG H and A with the
    velocity held fixed, timed with CUDA events on the launching stream (L2
    flushed between steps)."""
    from paper_2402_00466_gb300 import mevp

    if a.precision != "fp64":
        raise SystemExit("the transport workload is FP64 (DG1/DG2 ice fields)")
    dev = torch.cuda.current_device()
    case = W.make_case(a.workload)
    nx, ny, na = case["nx"], case["ny"], case["n_a"]
    ne = nx * ny
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    st = mevp.State(nx, ny, case["n_s"], vertex_xy=case["xy"], n_adv=na,
                    params=case["params"])
    st.set_ice(case["H"], case["A"])
    st.set_forcing(case["tau"])
    st.set_velocity(case["vel0"])
    for _ in range(a.warmup):
        flush.zero_()
        st.advect(1)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(a.steps)]
    for k in range(a.steps):
        flush.zero_()
        evs[k][0].record()
        st.advect(1)
        evs[k][1].record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(s_.elapsed_time(e_) for s_, e_ in evs)
    if ws > 1:
        total_ms = reduce_max(total_ms, dist, "cuda")
    st.close()
    value = whole_job_throughput(ne * a.steps, ws, total_ms / 1e3)
    stage_s = total_ms / 1e3 / (a.steps * ADV_STAGES[na])
    ach = ADV_FLOPS[na] * ne / stage_s / 1e12
    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        import oracle
        nxs, xs, Hs, As, vs = advection_sample(case)
        nsteps, t_cpu = 0, 0.0
        while t_cpu < 10.0 and nsteps < 20:
            t0 = time.perf_counter()
            oracle.advect(nxs, nxs, xs, na, vs, case["params"]["dt"], 1, Hs, As, openmp=True)
            t_cpu += time.perf_counter() - t0
            nsteps += 1
        cpu = {"value": nxs * nxs * nsteps / t_cpu, "unit": "element-steps/s",
               "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"{nsteps} advection steps of a {nxs}x{nxs} mesh, FP64 C oracle, OpenMP",
               "seconds": t_cpu}
    if rank == 0:
        line = {
            "metric": "DG upwind advection of H and A: element-steps/s", "value": value,
            "unit": "element-steps/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a.workload, "nx": nx, "ny": ny, "n_adv": na,
                       "rk_stages": ADV_STAGES[na],
                       "l2": "flushed between timed steps (512 MB write)"},
            "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak_tflops(clk),
                         "unit": "TFLOP/s", "frac": ach / fp64_peak_tflops(clk), "traffic": None,
                         "kernel": f"k_advect<{na}>", "flops_per_element_stage": ADV_FLOPS[na],
                         "peak_kind": fp64_peak_kind(clk)},
            "cpu_baseline": cpu, "e2e": None,
            "gpu_launches": a.steps * ADV_STAGES[na],
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_adjoint(a, torch, dist, ws, rank, emit=True):
    """Adjoint workload: `steps` gradient evaluations (dJ/dP*, dJ/dtau of the
    kinetic energy after n_sub subcycles, checkpoints every k), device
    outputs, CUDA events on the launching stream."""
    from paper_2402_00466_gb300 import mevp

    if a.precision != "fp64":
        raise SystemExit("the adjoint runs on FP64 states")
    dev = torch.cuda.current_device()
    case = W.make_case(a.workload)
    nx, ny, ns, n_sub = case["nx"], case["ny"], case["n_s"], case["n_sub"]
    k = W.CONFIGS[a.workload]["adjoint_every"]
    ne, nn, _ = W.sizes(nx, ny)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    st = mevp.State(nx, ny, ns, vertex_xy=case["xy"], params=case["params"])
    st.set_ice(case["H"], case["A"])
    st.set_forcing(case["tau"])
    st.set_velocity(case["vel0"])
    st.begin_step()
    clocks = Clocks(dev)

    def timed(kk, steps):
        for _ in range(a.warmup):
            flush.zero_()
            st.adjoint_kinetic_energy(n_sub, kk, device=True)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            evs[i][0].record()
            st.adjoint_kinetic_energy(n_sub, kk, device=True)
            evs[i][1].record()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ms = sum(s_.elapsed_time(e_) for s_, e_ in evs)
        return reduce_max(ms, dist, "cuda") if ws > 1 else ms

    def work(kk):
        """FP64 flops per objective element-subcycle with checkpoints every kk:
        the forward sweep, the recomputation of every segment but the last
        (recorded during the forward sweep), the reverse sweep."""
        kk = min(kk, n_sub)
        last = n_sub - ((n_sub - 1) // kk) * kk
        fwd = ELEM_FLOPS[ns] + 4 * NODE_FLOPS_PER_NODE
        return (1 + (n_sub - last) / n_sub) * fwd + ADJ_ELEM_FLOPS[ns] + 4 * ADJ_NODE_FLOPS, last

    clocks.start()
    total_ms = timed(k, a.steps)
    clk = clocks.stop()
    store_ms = timed(n_sub, a.steps)  # checkpoint_every = n: every velocity kept
    st.close()
    value = whole_job_throughput(ne * n_sub * a.steps, ws, total_ms / 1e3)
    per_es, last = work(k)
    ach = per_es * ne * n_sub * a.steps / (total_ms / 1e3) / 1e12
    per_store, _ = work(n_sub)
    ach_store = per_store * ne * n_sub * a.steps / (store_ms / 1e3) / 1e12
    line = None
    if rank == 0:
        line = {
            "metric": "adjoint of the mEVP subcycle: objective element-subcycles/s",
            "value": value, "unit": "element-subcycles/s", "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a.workload, "nx": nx, "ny": ny, "n_stress": ns,
                       "n_sub": n_sub, "checkpoint_every": k,
                       "gradients": "dJ/dP* [N_e], dJ/dtau [2][N_n], J = 1/2 sum m |v|^2",
                       "l2": "flushed between timed steps (512 MB write)"},
            "gradients_per_s": a.steps / (total_ms / 1e3),
            "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak_tflops(clk),
                         "unit": "TFLOP/s", "frac": ach / fp64_peak_tflops(clk), "traffic": None,
                         "kernel": "whole gradient (forward sweep, recomputation of all "
                                   "segments but the last, reverse sweep)",
                         "flops_per_element_subcycle": per_es,
                         "peak_kind": fp64_peak_kind(clk)},
            "cpu_baseline": None, "e2e": None,
            # forward sweep 2n, seeds 3, recompute 2(n - last segment), reverse 2n, gradients 1
            "gpu_launches": a.steps * (6 * n_sub - 2 * last + 4),
            "clocks": clk,
            "variants": {"checkpoint_every_n": {
                "checkpoint_every": n_sub, "gradients_per_s": a.steps / (store_ms / 1e3),
                "value": whole_job_throughput(ne * n_sub * a.steps, ws, store_ms / 1e3),
                "note": "every velocity kept (2 N_n n doubles), no recomputation",
                "achieved_TFLOPs": ach_store, "frac": ach_store / fp64_peak_tflops(clk),
                "flops_per_element_subcycle": per_store}},
        }
        if emit:
            print(json.dumps(line), flush=True)
    if ws > 1 and emit:
        dist.destroy_process_group()
    return line if not emit else 0


def _run_ours(a, torch, dist, ws, rank):
    from paper_2402_00466_gb300 import mevp

    if a.workload in W.ENSEMBLES:
        run_ensemble(a, torch, dist, ws, rank)
        return 0
    if W.CONFIGS[a.workload]["n_sub"] == 0:
        return run_advection(a, torch, dist, ws, rank)
    if "adjoint_every" in W.CONFIGS[a.workload]:
        return run_adjoint(a, torch, dist, ws, rank)
    dev = torch.cuda.current_device()

    def barrier():
        if ws > 1:
            dist.barrier()

    case = W.make_case(a.workload)
    nx, ny, ns, n_sub = case["nx"], case["ny"], case["n_s"], case["n_sub"]
    ne, nn, _ = W.sizes(nx, ny)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    # the headline arm (a.precision) and, unless --no-variants, the other
    # precision, timed the same way on the same workload
    arms = [a.precision] + ([] if a.no_variants else
                            ["mixed" if a.precision == "fp64" else "fp64"])
    res = {}
    for prec in arms:
        clocks = Clocks(dev)
        clocks.start()
        m = measure(mevp, torch, barrier, ws, case, prec, a.steps, a.warmup, flush)
        clk = clocks.stop()
        st = m["state"]
        total_ms = m["total_ms"]
        if ws > 1:
            total_ms = reduce_max(total_ms, dist, "cuda")
        r = {"value": whole_job_throughput(ne * n_sub * a.steps, ws, total_ms / 1e3),
             "ms_per_step": total_ms / a.steps,
             "begin_step_ms_per_step": m["begin_ms"] / a.steps,
             "subcycles_ms_per_step": m["sub_ms"] / a.steps,
             "roofline": roofline_for(prec, case, m, a.steps, clk),
             "kernel_split": m["split"],
             # per step: begin_step (3 kernels; mixed adds 2 conversions) +
             # per subcycle 2 (FP64: element, node) or 1 (mixed: the fused tile)
             "gpu_launches": a.steps * ((5 if prec == "mixed" else 3) +
                                        (1 if prec == "mixed" else 2) * n_sub),
             "dtype": "f64" if prec == "fp64" else "f32",
             "clocks": clk, "wall_s": m["wall"], "e2e": None}
        if not a.no_e2e:
            e2e, dt = end_to_end(mevp, torch, barrier, ws, case, st, a.steps)
            if ws > 1:
                e2e["value"] = ws * ne * n_sub * e2e["steps"] / reduce_max(dt, dist, "cuda")
            r["e2e"] = e2e
        st.close()
        res[prec] = r

    # the other rows' workloads, a few steps each, so that the benchmark line
    # carries their numbers too: batched ensembles (mixed and FP64) and the
    # adjoint's gradient
    extras = None
    if not a.no_extras:
        extras = {}
        keep = ("value", "unit", "ms_per_step", "steps", "roofline", "config", "gpu_launches",
                "clocks")
        for prec in ("mixed", "fp64"):
            b = argparse.Namespace(**vars(a))
            b.workload, b.precision, b.steps, b.warmup = "ensemble64", prec, 3, 3
            line = run_ensemble(b, torch, dist, ws, rank, emit=False)
            extras[f"ensemble64_{prec}"] = dict(
                {k: line[k] for k in keep},
                speedup_vs_sequential=line["speedup_vs_sequential"])
        b = argparse.Namespace(**vars(a))
        b.workload, b.precision, b.steps, b.warmup = "adjoint256_dg1", "fp64", 5, 3
        line = run_adjoint(b, torch, dist, ws, rank, emit=False)
        if line is not None:
            extras["adjoint256_dg1"] = dict({k: line[k] for k in keep},
                                            gradients_per_s=line["gradients_per_s"],
                                            variants=line["variants"])

    head = res[a.precision]
    cpu = None
    field_errors = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(case)
        # the oracle leg: per-field errors of both paths against the oracle
        field_errors = field_error_block(mevp, a.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": head["dtype"], "data": "synthetic",
            "config": {"workload": a.workload, "nx": nx, "ny": ny, "n_stress": ns,
                       "n_sub": n_sub, "precision": a.precision,
                       "alpha": case["params"]["alpha"], "beta": case["params"]["beta"],
                       "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
            "wall_s": head["wall_s"],
            "begin_step_ms_per_step": head["begin_step_ms_per_step"],
            "subcycles_ms_per_step": head["subcycles_ms_per_step"],
            "kernel_split": head["kernel_split"],
            "arms": {p: r for p, r in res.items() if p != a.precision},
            "field_errors": field_errors,
            "extra_workloads": extras,
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
    ap.add_argument("--workload", default="mesh1024_dg2",
                    choices=sorted(W.CONFIGS) + sorted(W.ENSEMBLES))
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="time only --precision, not the other precision's arm")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ensemble and adjoint workloads of the default line")
    a = ap.parse_args()
    if a.warmup < 3 and a.impl == "ours":
        ap.error("--warmup must be >= 3")
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark of the sparse-FCI hot path on GB300.

One step = one sfci_lanczos_step: sigma = H w_i over all single and double
excitations (enumerate, Slater-Condon, Eq. 12 rank, merge), the T/S dot
products, u = sigma - a w_i - b w_{i-1}, and the top-N_d truncation (Eqs.
10-11); every N_L-th step also solves T x = lambda S x and restarts.

Workload (default): 28 spatial orbitals, 7 alpha + 7 beta electrons (FCI
dimension 1.4e12, ranks in uint64), synthetic integrals with L = 200 factors
and two near-degenerate orbital clusters, N_d = 1e6 determinants per basis
vector, N_L = 10.  The solver starts from the aufbau determinant; the warm-up
steps grow the vector to N_d; the timed steps then run at full size.

value = connected elements enumerated per second over the timed steps
(elements = sum over input determinants of 1 + the number of single and
double excitations).  Multi-GPU: one independent replica per rank (the
method's one exchange step is not built), scaling "weak".

--impl reference times the CPU oracle on a bounded sample of the same
workload (sigma of the first determinants of a vector of the same shape).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "σ=Hψ connected elements/s & Lanczos steps/s vs plain FP64 at ΔE≤1 µHa"
UNIT = "connected elements/s"
BYTES_PER_ELEMENT = 32  # 16 B intermediate element written + 16 B read back by the merge
# DRAM bytes per connected element that ncu measured for emit_kernel + merge_kernel
# together (dram__bytes_read.sum + dram__bytes_write.sum of one launch each on the same
# workload at N_d = 5e3, 1.5362e8 elements, one pass, every excitation class in the emit
# kernel); scaled by the elements of a step
MEASURED_DRAM_BYTES_PER_ELEMENT = (0.052011 + 2.438096 + 2.467282 + 0.004709) * 1e9 / 1.5362e8
# warp instructions per connected element (smsp__inst_executed.sum of the same captures) and
# the issue ceiling: 152 SMs x 4 schedulers x one warp instruction per clock at 2070 MHz
MEASURED_WARP_INST_PER_ELEMENT = {"emit": 1154000833 / 1.5362e8, "merge_kernel": 1938576001 / 1.5362e8}
ISSUE_PEAK_WARP_INST_PER_S = 152 * 4 * 2.07e9
# the constants above were captured before merge_kernel's key-grouping threshold changed
TRAFFIC_STALE = True
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=4)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--nkeep", type=int, default=1_000_000)
    p.add_argument("--nlanczos", type=int, default=10)
    p.add_argument("--cpu-sample", type=int, default=1000,
                   help="input determinants in the CPU oracle's timed sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-workloads", action="store_true",
                   help="skip the rows of the other workloads (8-orbital full space, Hubbard ring, "
                        "N_d = 1e5, RDM pass, batched scan) and the pipe-rate probes")
    p.add_argument("--bucket-elems", type=int, default=0,
                   help="intermediate elements per merge bucket (0 = automatic)")
    p.add_argument("--table-capacity", type=int, default=0,
                   help="merge-table slots (0 = sized by the solver)")
    p.add_argument("--mem-budget-gb", type=float, default=0.0,
                   help="device memory the sigma passes may use (0 = what is free); a small budget "
                        "gives a small case with several passes, for profiling")
    p.add_argument("--emit-warps", type=int, default=0,
                   help="warps per CTA of the element generator (0 = 8)")
    p.add_argument("--workload", default="sfci", choices=["sfci", "scan"],
                   help="sfci: the 28-orbital solver (headline); scan: 32 uneven instances stepped together")
    p.add_argument("--scan-cap-scale", type=float, default=1.0,
                   help="scale factor on the scan instances' vector caps")
    p.add_argument("--workers", type=int, default=0, help="scan host workers (0 = automatic)")
    p.add_argument("--tune", action="store_true",
                   help="scan: pick emit warps, bucket size and workers with the autotuner "
                        "(on the instances with caps scaled by --tune-cap-scale; cached)")
    p.add_argument("--tune-cap-scale", type=float, default=0.25)
    p.add_argument("--no-screen", action="store_true",
                   help="skip the heat-bath style selection study (eps_element)")
    p.add_argument("--screen-eps", default="1e-6,1e-5,1e-4")
    p.add_argument("--no-precision", action="store_true",
                   help="skip the float32-element vs float64 comparison")
    p.add_argument("--precision-nkeep", type=int, default=100_000)
    p.add_argument("--precision-steps", type=int, default=30)
    return p.parse_args()


def workload_name(a):
    return f"sfci-28o-7a7b-L200-clustered-Nd{a.nkeep:.0e}-NL{a.nlanczos}".replace("+0", "")


def config(a, world=1):
    """The workload; the same dictionary on both arms."""
    return {"workload": workload_name(a), "n_orb": 28, "n_alpha": 7, "n_beta": 7,
            "n_factors": 200, "n_keep": a.nkeep, "n_lanczos": a.nlanczos,
            "start": "aufbau determinant", "integrals": "seeded synthetic (seed 2)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "no flush: each step's element regions (hundreds of GB at N_d = 1e6) exceed the 129 MB L2"}


def reduce_over_ranks(ms, elements, dist=None, device="cuda"):
    """Whole-job timing of replicas: the slowest rank's time and the elements
    of all ranks (each rank runs the full workload: weak scaling)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    e = torch.tensor([float(elements)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle

def oracle_sample(n_src):
    """Input of the CPU oracle's timed sample: the first n_src determinants of a
    near-aufbau vector of the workload (the shape of a truncated Lanczos vector)."""
    import gen
    import oracle
    d = gen.config_system(2)
    osys = oracle.System.from_dict(d)
    a, b, lev = gen.near_aufbau_dets(28, 7, 7, n_src, seed=2024)
    r = oracle.det_rank(28, 7, a, b)
    o = __import__("numpy").argsort(r)
    c = gen.level_coefs(lev, 2025)
    return osys, r[o], c[o]


def time_oracle(n_src, threads=None):
    """sigma of the first n_src determinants of a near-aufbau vector by the
    oracle on `threads` host threads: (elements/s, elements, seconds, threads)."""
    import oracle
    osys, r, c = oracle_sample(n_src)
    nt = threads or oracle.n_threads()
    t0 = time.perf_counter()
    _, _, _, nel = oracle.sigma(osys, r, c, threads=nt)
    dt = time.perf_counter() - t0
    return nel / dt, nel, dt, nt


def run_reference(a):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    import oracle
    oracle.lib()
    for _ in range(a.warmup):
        time_oracle(max(10, a.cpu_sample // 20))
    vals, nel_tot, t_tot = [], 0, 0.0
    for _ in range(a.steps):
        v, nel, dt, nt = time_oracle(max(10, a.cpu_sample // 5))
        vals.append(v)
        nel_tot += nel
        t_tot += dt
    value = nel_tot / t_tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * t_tot / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(a, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": f"each step: sigma of the first {max(10, a.cpu_sample // 5)} "
                                       f"determinants of a near-aufbau vector of the workload "
                                       f"(plain C, OpenMP)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm

def precision_study(sf, d, nkeep, n_lanczos, steps, stream):
    """The solver from the aufbau determinant with float64 elements (twice) and
    with SFCI_FP32_ELEMENTS: throughput of each and the energy difference at
    every cycle end.  The second float64 run checks the run-to-run spread: the
    merge sums every sigma entry exactly (fixed point, rounded once), so two
    float64 runs repeat bit for bit and the float32 difference is its own."""
    import numpy as np
    import torch
    out = {}
    for name, flags in (("f64", 0), ("f64_repeat", 0), ("fp32_elements", sf.SFCI_FP32_ELEMENTS)):
        gsys = sf.System.from_dict(d, flags=flags)
        lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), nkeep, n_lanczos,
                        stream=stream)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        infos = [lz.step() for _ in range(steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        el = sum(i["n_elements"] for i in infos)
        out[name] = {"elements_per_s": el / (ms * 1e-3), "ms_per_step": ms / steps,
                     "ms_sigma_mean": statistics.mean(i["ms_sigma"] for i in infos),
                     "lambda": [i["lambda_min"] for i in infos if i["cycle_end"]]}
        lz.close()
        gsys.close()
    lam64, lam32 = out["f64"]["lambda"], out["fp32_elements"]["lambda"]
    out["delta_e_hartree"] = [b - a for a, b in zip(lam64, lam32)]
    out["f64_repeat_delta_e_hartree"] = [b - a for a, b in zip(lam64, out["f64_repeat"]["lambda"])]
    # cycle ends where two float64 runs agree to 1e-9 Ha (all of them: the sigma sums are
    # exact, so the runs repeat bit for bit): there the float32 difference is its own
    comp = [i for i, r in enumerate(out["f64_repeat_delta_e_hartree"]) if abs(r) < 1e-9]
    out["comparable_cycles"] = comp
    out["max_abs_delta_e_comparable"] = max((abs(out["delta_e_hartree"][i]) for i in comp), default=None)
    out["within_1_uHa"] = bool(comp) and out["max_abs_delta_e_comparable"] <= 1e-6
    out["speedup"] = out["fp32_elements"]["elements_per_s"] / out["f64"]["elements_per_s"]
    out["workload"] = f"sfci-28o-7a7b-L200-clustered-Nd{nkeep:.0e}-NL{n_lanczos}".replace("+0", "") + \
        f", {steps} steps from the aufbau determinant, both precisions"
    return out


def scan_study(sf, cap_scale, n_lanczos, warmup, steps, workers=0, bucket_elems=0, emit_warps=0):
    """The 32-instance batched scan (n 16-24, 5-8 electrons per spin, caps
    1e4-2e5 times cap_scale, integrals interpolated between two seeded sets)
    stepped together through sfci_scan (float64, then float32 elements), and
    the float64 instances one at a time (one worker) for comparison.  Per run:
    elements of all instances per second of wall time, and the device-busy
    fraction sum over instances of (sigma + truncation time, CUDA events) / wall
    time; the float32 run's energy difference from the float64 run at every
    cycle end, per instance."""
    import numpy as np
    import torch

    import gen
    inst_d = gen.batched_scan_instances()
    caps = [max(1000, int(d["cap"] * cap_scale)) for d in inst_d]
    out = {"workload": f"batched-scan-32-instances-n16to24-caps1e4to2e5x{cap_scale:g}", "caps": caps,
           "n_lanczos": n_lanczos, "warmup": warmup, "steps": steps}
    lams = {}
    for name, workers_, flags in (("batched", workers, 0), ("one_at_a_time", 1, 0),
                                  ("batched_fp32_elements", workers, sf.SFCI_FP32_ELEMENTS)):
        systems = [sf.System.from_dict(d, flags=flags) for d in inst_d]
        inst = [(s_, np.array([0], dtype=np.uint64), np.array([1.0]), c) for s_, c in zip(systems, caps)]
        sc = sf.Scan(inst, n_lanczos=n_lanczos, bucket_elems=bucket_elems, emit_warps=emit_warps,
                     workers=workers_)
        allsteps = [sc.step() for _ in range(warmup)]
        torch.cuda.synchronize()
        l0 = sf.kernel_launches()
        t0 = time.perf_counter()
        timed = [sc.step() for _ in range(steps)]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        allsteps += timed
        el = sum(x["n_elements"] for st in timed for x in st)
        busy = sum(x["ms_sigma"] + x["ms_topk"] for st in timed for x in st) * 1e-3
        out[name] = {"value": el / dt, "ms_per_step": 1e3 * dt / steps, "elements_per_step": el / steps,
                     "gpu_launches": sf.kernel_launches() - l0, "device_busy_fraction": busy / dt}
        lams[name] = [[st[k]["lambda_min"] for st in allsteps if st[k]["cycle_end"]] for k in range(len(caps))]
        if name == "batched":
            final = [sc.vector(k) for k in range(len(caps))]
        sc.close()
        for s_ in systems:
            s_.close()
    out["speedup_vs_one_at_a_time"] = out["batched"]["value"] / out["one_at_a_time"]["value"]
    out["fp32_speedup"] = out["batched_fp32_elements"]["value"] / out["batched"]["value"]
    d64, d32 = lams["batched"], lams["batched_fp32_elements"]
    out["fp32_delta_e_hartree"] = [[b - a for a, b in zip(x, y)] for x, y in zip(d64, d32)]  # per instance
    out["fp32_max_abs_delta_e"] = max((abs(v) for row in out["fp32_delta_e_hartree"] for v in row), default=None)
    out["lambda_cycle_ends_fp64"] = d64
    # element precision alone: <psi|H|psi> / <psi|psi> of the float64 run's final
    # vector of each instance, with float64 and with float32 elements (one step of
    # a one-vector solver gives a_0 = the Rayleigh quotient)
    same = []
    for k, d in enumerate(inst_d):
        r, c = final[k]
        a_ = []
        for flags in (0, sf.SFCI_FP32_ELEMENTS):
            s_ = sf.System.from_dict(d, flags=flags)
            lz = sf.Lanczos(s_, r, c, caps[k], 1)
            a_.append(lz.step()["a"])
            lz.close()
            s_.close()
        same.append(a_[1] - a_[0])
    out["fp32_delta_e_same_vector_hartree"] = same
    out["fp32_max_abs_delta_e_same_vector"] = max(abs(x) for x in same)
    out["fp32_within_1_uHa_same_vector"] = bool(max(abs(x) for x in same) <= 1e-6)
    return out


def run_scan(a):
    """--workload scan: the batched scan as the JSON line's headline (see scan_study)."""
    import torch

    import paper_2312_01846_gb300 as sf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    shape = {"bucket_elems": a.bucket_elems, "emit_warps": a.emit_warps, "workers": a.workers}
    tuned = None
    if a.tune:
        import gen
        from paper_2312_01846_gb300.tune import tune_scan
        inst_d = gen.batched_scan_instances()
        systems = [sf.System.from_dict(d) for d in inst_d]
        tcaps = [max(1000, int(d["cap"] * a.scan_cap_scale * a.tune_cap_scale)) for d in inst_d]
        tuned = tune_scan(systems, tcaps, n_lanczos=a.nlanczos)
        shape.update(tuned["best"])
        for s_ in systems:
            s_.close()
    out = scan_study(sf, a.scan_cap_scale, a.nlanczos, a.warmup, a.steps, shape["workers"],
                     shape["bucket_elems"], shape["emit_warps"])
    hbm, peak_kind = peaks()
    b = out["batched"]
    achieved = BYTES_PER_ELEMENT * b["elements_per_step"] / (b["ms_per_step"] * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": out["workload"], "instances": len(out["caps"]), "caps": out["caps"],
                   "n_lanczos": a.nlanczos, "parallelism": "single GPU, one stream per instance"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "kernel": "whole scan step (wall time)",
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "model": f"{BYTES_PER_ELEMENT} B per connected element"},
        "gpu_launches": b["gpu_launches"], "cpu_baseline": None, "e2e": None,
        "detail": out, "launch_shape": shape, "autotune": tuned,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def screen_study(sf, d, nkeep, n_lanczos, steps, stream, eps_list):
    """The solver with the heat-bath style selection (eps_element) against the
    exact sigma: throughput (enumerated elements per second, so a faster step
    shows as a higher rate) and the energy difference at every cycle end."""
    import numpy as np
    import torch
    gsys = sf.System.from_dict(d)
    out = {"workload": f"sfci-28o-7a7b-L200-clustered-Nd{nkeep:.0e}-NL{n_lanczos}".replace("+0", "") +
                       f", {steps} steps from the aufbau determinant", "runs": []}
    for eps in [0.0] + list(eps_list):
        lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), nkeep, n_lanczos,
                        stream=stream, eps_element=eps)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        infos = [lz.step() for _ in range(steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        lz.close()
        out["runs"].append({"eps_element": eps,
                            "elements_per_s": sum(i["n_elements"] for i in infos) / (ms * 1e-3),
                            "ms_per_step": ms / steps,
                            "ms_sigma_mean": statistics.mean(i["ms_sigma"] for i in infos),
                            "lambda": [i["lambda_min"] for i in infos if i["cycle_end"]]})
    exact = out["runs"][0]
    for r in out["runs"][1:]:
        r["delta_e_hartree"] = [b - a for a, b in zip(exact["lambda"], r["lambda"])]
        r["speedup"] = r["elements_per_s"] / exact["elements_per_s"]
    gsys.close()
    return out


def solver_row(sf, d, name, nkeep, n_lanczos, warmup, steps, stream, note):
    """One workload row of the bench line: the solver from the aufbau determinant,
    `warmup` untimed steps, then `steps` timed with CUDA events on the solver's
    stream.  Enumerated and generated (non-zero) elements per second, Lanczos
    steps per second, mean sigma time and the cycle-end energies."""
    import numpy as np
    import torch
    gsys = sf.System.from_dict(d)
    lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), nkeep, n_lanczos,
                    stream=stream)
    for _ in range(warmup):
        lz.step()
    torch.cuda.synchronize()
    l0 = sf.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = [lz.step() for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = sf.kernel_launches() - l0
    lz.close()
    gsys.close()
    el = sum(i["n_elements"] for i in infos)
    nz = sum(i["n_emitted"] for i in infos)
    return {"workload": name, "note": note, "n_keep": nkeep, "n_lanczos": n_lanczos,
            "warmup": warmup, "steps": steps, "ms_per_step": ms / steps,
            "lanczos_steps_per_s": steps / (ms * 1e-3),
            "elements_per_s": el / (ms * 1e-3), "nonzero_elements_per_s": nz / (ms * 1e-3),
            "elements_per_step": el / steps, "nonzero_elements_per_step": nz / steps,
            "ms_sigma_mean": statistics.mean(i["ms_sigma"] for i in infos),
            "n_in_last": infos[-1]["n_in"], "passes_max": max(i["n_passes"] for i in infos),
            "gpu_launches_per_step": launches / steps,
            "lambda_cycle_ends": [i["lambda_min"] for i in infos if i["cycle_end"]]}


def rdm_row(sf, stream, nkeep=300_000, grow_steps=12, reps=3):
    """20 orbitals 5a/5b (L = 64): the solver grows a sparse vector of N_d = 3e5
    determinants from the aufbau determinant, then sfci_rdm12 runs on it
    (one pass of the excitation generator over the vector, 1- and 2-RDM by
    atomics), timed with CUDA events; elements = entries x (n_conn + 1)."""
    import numpy as np
    import torch

    import gen
    d = gen.config_system(4)
    gsys = sf.System.from_dict(d)
    lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), nkeep, 10, stream=stream)
    for _ in range(grow_steps):
        lz.step()
    r, c = lz.vector()
    lz.close()
    sf.sfci_rdm12(gsys, r, c, stream=stream)  # warm-up
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        g1, g2, nrm = sf.sfci_rdm12(gsys, r, c, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    el = r.numel() * (gsys.n_conn + 1)
    h = torch.tensor(d["h"], device="cuda")
    g = torch.tensor(d["g"], device="cuda")
    e = sf.sfci_rdm_energy(g1, g2, nrm, h, g, 0.0)
    gsys.close()
    return {"workload": "rdm12-20o-5a5b-L64-Nd3e5", "n_det": int(r.numel()), "ms_per_pass": ms,
            "elements_per_s": el / (ms * 1e-3), "elements_per_pass": el, "energy": e,
            "note": "sigma-generator pass over a 3e5-determinant SFCI vector (12 steps from the aufbau "
                    "determinant), 1- and 2-RDM accumulated with float64 atomics"}


def pipe_rates(sf):
    """Lane operations per second and per SM per clock of the pipe operations
    the sigma kernels depend on (sfci_debug_pipe_rate)."""
    import torch
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    out = {}
    for k in sf.PIPE_KINDS:
        iters = 1 << 12 if k.startswith("fp64") else 1 << 14
        r = sf.pipe_rate(k, iters)
        out[k] = {"ops_per_s": r, "per_sm_per_clk_at_2070_mhz": r / sms / 2.07e9}
    return out


def run_ours(a):
    import numpy as np
    import torch

    import gen
    import paper_2312_01846_gb300 as sf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    d = gen.config_system(2)
    gsys = sf.System.from_dict(d)
    stream = torch.cuda.current_stream()
    lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), a.nkeep, a.nlanczos,
                    table_capacity=a.table_capacity, bucket_elems=a.bucket_elems, stream=stream,
                    emit_warps=a.emit_warps, mem_budget=int(a.mem_budget_gb * 1e9))

    def brief(i):
        return {k: i[k] for k in ("n_in", "n_sigma", "n_passes", "ms_plan", "ms_emit", "ms_merge",
                                  "ms_topk", "ms_step", "redo", "bucket_redo", "tau", "cut",
                                  "pass_budget_gb", "regions_gb", "free_gb", "n_overflow", "ms_alloc",
                                  "n_emitted")}

    warm = []
    for _ in range(a.warmup):
        warm.append(brief(lz.step()))
    barrier()
    launches0 = sf.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos = []
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    gpu_index = vis[local] if local < len(vis) and vis[local].strip() else str(local)
    with ClockSampler(gpu_index) as clk:
        ev0.record(stream)
        for _ in range(a.steps):
            infos.append(lz.step())
        ev1.record(stream)
        barrier()
    launches = sf.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    elements = sum(i["n_elements"] for i in infos)
    ms_max, elements_all = reduce_over_ranks(ms, elements, dist, "cuda")
    value = elements_all / (ms_max * 1e-3)
    steps_per_s = a.steps / (ms_max * 1e-3)

    # dominant stage: sigma = H w_i, i.e. the emit kernel (writes each intermediate
    # element once) plus the bucket merge (reads it once), timed with CUDA events
    # on the solver's stream; the 32 B/element model is exactly that write + read
    ms_sig = statistics.mean(i["ms_sigma"] for i in infos)
    ms_emit = statistics.mean(i["ms_emit"] for i in infos)
    ms_merge = statistics.mean(i["ms_merge"] for i in infos)
    el_per_launch = statistics.mean(i["n_elements"] for i in infos)
    hbm, peak_kind = peaks()
    achieved = BYTES_PER_ELEMENT * el_per_launch / (ms_sig * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm,
                # null: merge_kernel changed (its key-grouping threshold) after the last
                # capture; that capture's figure, which the change does not touch (the same
                # records are read), is kept below for reference
                "traffic": None if TRAFFIC_STALE else MEASURED_DRAM_BYTES_PER_ELEMENT * el_per_launch,
                "traffic_last_capture": MEASURED_DRAM_BYTES_PER_ELEMENT * el_per_launch,
                "traffic_note": "bytes per launch: ncu DRAM bytes per element of emit_kernel + "
                                "merge_kernel (N_d = 5e3 capture, one pass) x elements per launch; "
                                "null while a kernel has changed since that capture",
                "kernel": "sigma stage: emit (emit_kernel, emit_aa_kernel) + merge_kernel",
                "peak_kind": f"{peak_kind} copy bandwidth",
                "model": f"{BYTES_PER_ELEMENT} B per connected element (16 B written by emit, "
                         f"16 B read by merge)",
                "ms_per_launch": ms_sig, "ms_emit": ms_emit, "ms_merge": ms_merge,
                "ms_plan_host": statistics.mean(i["ms_plan"] for i in infos),
                "ms_topk": statistics.mean(i["ms_topk"] for i in infos),
                "passes": max(i["n_passes"] for i in infos),
                "buckets_log2": max(i["n_buckets_log2"] for i in infos),
                "elements_per_launch": el_per_launch,
                "nonzero_elements_per_launch": statistics.mean(i["n_emitted"] for i in infos),
                "sigma_share_of_step": sum(i["ms_sigma"] for i in infos) / ms,
                "issue_note": "merge_kernel's instructions per element were captured before its "
                              "key-grouping threshold changed (fewer grouped buckets: fewer "
                              "instructions now)" if TRAFFIC_STALE else "",
                # the kernels are bound by instruction issue and latency, not by DRAM: the
                # issue-slot view, with warp instructions per element from the N_d = 5e3
                # one-pass captures (at N_d = 1e6 entries repeat more, so the merge streams
                # out fewer entries per element and this overstates its count; the emit stage
                # there is emit_kernel plus emit_aa_kernel over three passes)
                "issue": {kname: {"warp_inst_per_element": ipe,
                                  "achieved_warp_inst_per_s": ipe * el_per_launch / (ms_k * 1e-3),
                                  "peak_warp_inst_per_s": ISSUE_PEAK_WARP_INST_PER_S,
                                  "frac": ipe * el_per_launch / (ms_k * 1e-3) / ISSUE_PEAK_WARP_INST_PER_S}
                          for kname, ipe, ms_k in (("emit", MEASURED_WARP_INST_PER_ELEMENT["emit"], ms_emit),
                                                   ("merge_kernel", MEASURED_WARP_INST_PER_ELEMENT["merge_kernel"], ms_merge))}}

    # end to end through the public API with host buffers, chained: each step
    # copies its input vector w_i host -> device and hands it to the solver
    # (sfci_lanczos_set_input, the cycle goes on), runs one step, and copies
    # the next vector (w_{i+1}, or the restart vector) back to the host, where
    # it is the next step's input
    e2e = None
    if not a.no_e2e:
        r_dev, c_dev = lz.vector()
        cap = a.nkeep
        h_r = torch.empty(cap, dtype=torch.int64).pin_memory()
        h_c = torch.empty(cap, dtype=torch.float64).pin_memory()
        h_r[: r_dev.numel()].copy_(r_dev)
        h_c[: c_dev.numel()].copy_(c_dev)
        n_cur = r_dev.numel()
        n_e2e = max(1, min(a.steps, 10))
        barrier()
        t0 = time.perf_counter()
        el2 = 0
        h2d = d2h = 0
        for _ in range(n_e2e):
            dr = h_r[:n_cur].to("cuda", non_blocking=True)
            dc = h_c[:n_cur].to("cuda", non_blocking=True)
            lz.set_input(dr, dc)
            info = lz.step()
            el2 += info["n_elements"]
            nr, nc = lz.vector()
            h_r[: nr.numel()].copy_(nr, non_blocking=True)
            h_c[: nc.numel()].copy_(nc, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            h2d += 16 * n_cur
            d2h += 16 * nr.numel() + 152
            n_cur = nr.numel()
        barrier()
        dt = time.perf_counter() - t0
        e2e = {"value": el2 / dt, "unit": UNIT, "h2d_bytes_per_step": h2d // n_e2e,
               "d2h_bytes_per_step": d2h // n_e2e, "steps": n_e2e,
               "note": "chained: host vector in (set as the solver's w_i), one step, the next vector "
                       "to the host as the next step's input (wall clock)"}

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        v, nel, dt, nt = time_oracle(a.cpu_sample)
        v1, nel1, dt1, _ = time_oracle(max(10, a.cpu_sample // 10), threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle",
               "sample": f"sigma of {a.cpu_sample} input determinants of a near-aufbau "
                         f"vector of the workload ({nel} elements, {dt:.1f} s)",
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                 "sample": f"sigma of {max(10, a.cpu_sample // 10)} input determinants "
                                           f"({nel1} elements, {dt1:.1f} s)"}}

    last_lambda = [i["lambda_min"] for i in infos if i["cycle_end"]]
    # the studies below build their own solvers: free this one's device memory first
    lz.close()
    torch.cuda.synchronize()

    workloads = None
    if rank == 0 and not a.no_workloads:
        workloads = {
            "cfg0": solver_row(sf, gen.config_system(0), "sfci-8o-4a4b-L16-full-space", 4900, 10, 3, 30,
                               stream, "whole space (N_d = dim = 4900): launch-latency floor of a step"),
            "cfg1": solver_row(sf, gen.config_system(1), "hubbard-ring-12-6a6b-U4-Nd2e4", 20_000, 10, 0, 40,
                               stream, "40 steps from the aufbau determinant; most enumerated elements are "
                                       "zero products, nonzero_elements_per_s counts those generated"),
            "cfg2_nd1e5": solver_row(sf, d, "sfci-28o-7a7b-L200-clustered-Nd1e5-NL10", 100_000, 10, 4, 16,
                                     stream, "same system as the headline at N_d = 1e5"),
            "cfg4_rdm": rdm_row(sf, stream),
            "cfg3_scan": scan_study(sf, 1.0, a.nlanczos, 3, 8),
            # the same 32 instances with caps cut 100-fold (1e3 determinants each): every
            # instance step is a few milliseconds of kernels and launch latency, the
            # regime where stepping the instances concurrently pays
            "cfg3_scan_caps_x0.01": scan_study(sf, 0.01, a.nlanczos, 3, 10),
        }
    issue = pipe_rates(sf) if rank == 0 and not a.no_workloads else None

    precision = None
    if rank == 0 and not a.no_precision:
        precision = precision_study(sf, d, a.precision_nkeep, a.nlanczos, a.precision_steps, stream)

    screen = None
    if rank == 0 and not a.no_screen:
        eps_list = [float(x) for x in a.screen_eps.split(",") if x]
        screen = {"cfg2": screen_study(sf, d, a.precision_nkeep, a.nlanczos, 20, stream, eps_list),
                  # the Hubbard ring, whose integrals are mostly exact zeros: the exact
                  # class skips already drop those; the screen then drops small products
                  "cfg1": screen_study(sf, gen.config_system(1), 20_000, a.nlanczos, 40, stream, eps_list)}
        screen["cfg1"]["workload"] = "hubbard-ring-12-6a6b-U4-Nd2e4, 40 steps from the aufbau determinant"

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config(a, world),
        "lanczos_steps_per_s": steps_per_s,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk.summary(),
        "workloads": workloads,
        "pipe_rates": issue,
        "precision": precision,
        "heat_bath_screen": screen,
        "detail": {"n_in": infos[-1]["n_in"], "n_sigma": infos[-1]["n_sigma"],
                   "elements_per_step": el_per_launch, "lambda_min": last_lambda[-1] if last_lambda else None,
                   "ms_sigma_mean": ms_sig,
                   "warmup_steps": warm, "timed_steps": [brief(i) for i in infos]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    gsys.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "scan":
        return run_scan(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark: acc+jerk pair interactions per second at N = 2^20 (compensated and plain).

One step = one Hermite block step of the whole hot path through the public C
ABI (nbody_next_block -> nbody_predict -> nbody_force -> nbody_correct) on an
equal-mass Plummer sphere of N = 2^20 particles (eps = 1e-3, Henon units).
All particles share one power-of-two level (dt_max = dt_min = 2^-10), so every
block holds all N particles and each step evaluates N (N - 1) pairs.

Prints one JSON line.  `value` is the compensated-mode rate with inputs resident
in device memory; `plain` holds the plain-FP32 rate; `e2e` repeats the
compensated step with pinned host buffers (active list in, forces out);
`roofline` relates the force kernel's own CUDA-event time to the FP32-pipe
bound of the chip; `cpu_baseline` times the FP64 CPU oracle on a bounded
sample of the same step.  `--impl reference` times only the oracle (the
reference arm).  Under torchrun each rank runs an independent replica on its
own GPU (weak scaling) and rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "acc+jerk pair-interactions/s at N=2^20, compensated vs plain FP32, % roofline"
UNIT = "pair-interactions/s"
N_DEFAULT = 1 << 20
SEED = 3
EPS2 = 1e-6          # eps = 1e-3
LEVEL = 10           # shared step 2^-10: every block is all N particles
OPS_PER_PAIR = 27    # FP32-pipe operations of one plain pair term (plus one MUFU rsqrt)
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int) -> float:
    """Largest value over all ranks (one all-reduce); identity for one process."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, ws: int) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_totals(ws: int, mode_ms: dict, e2e_ms: float, pairs_per_rank: float) -> dict:
    """Every cross-rank reduction of the benchmark, called by all ranks in one fixed order: per mode
    and for the end-to-end run, the slowest rank's time and the work of all replicas."""
    out = {}
    for mode in sorted(mode_ms):
        out[mode] = {"t_max": max_over_ranks(mode_ms[mode], ws), "pairs": sum_over_ranks(pairs_per_rank, ws)}
    out["e2e"] = {"t_max": max_over_ranks(e2e_ms, ws), "pairs": sum_over_ranks(pairs_per_rank, ws)}
    return out


def barrier(ws: int) -> None:
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"nbody_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [c.strip() for c in line.split(",")]
                if len(p) >= 9 and p[1].replace(".", "").isdigit():
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(float(r[2]) for r in rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "samples": len(rows), "reasons": reasons}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def make_sim(m, x, v, mode, stream):
    from paper_astro_ph_0702058_gb300 import Simulation
    return Simulation(m, x, v, EPS2, eta=0.02, lmin=LEVEL, lmax=LEVEL, mode=mode, stream=stream)


def run_steps(sim, n, steps, warmup, stream, flush, host=None, after_first=None):
    """Times `steps` block steps (after `warmup`).  Returns (total_ms, force_ms_list, launches).
    `after_first` (untimed, during the warm-up) is called once after the first step."""
    import torch
    dev_list = torch.zeros(n, dtype=torch.int32, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    step_ms, force_ms = [], []
    launches0 = 0
    for it in range(warmup + steps):
        if it == warmup:
            torch.cuda.synchronize()
            launches0 = sim.stats()["kernel_launches"]
        flush.zero_()                     # L2 flush between steps, outside the timed events
        e0, f0, f1, e1 = ev(), ev(), ev(), ev()
        e0.record(stream)
        if host is None:
            t_blk, n_act = sim.next_block(dev_list)
            sim.predict(t_blk)
            f0.record(stream)
            sim.force(dev_list, n_act)
            f1.record(stream)
            sim.correct(dev_list, n_act)
        else:
            lst, acc, jerk, pot = host
            t_blk, n_act = sim.next_block(lst)
            sim.predict(t_blk)
            f0.record(stream)
            sim.force(lst, n_act, acc=acc, jerk=jerk, pot=pot)
            f1.record(stream)
            sim.correct(lst, n_act)
        e1.record(stream)
        assert n_act == n, n_act
        if it == 0 and after_first is not None and warmup > 0:
            after_first()
        if it >= warmup:
            step_ms.append((e0, e1))
            force_ms.append((f0, f1))
    sim.sync()
    torch.cuda.synchronize()
    launches = sim.stats()["kernel_launches"] - launches0
    total = sum(a.elapsed_time(b) for a, b in step_ms)
    return total, [a.elapsed_time(b) for a, b in force_ms], launches


# the force kernel's code; its launch shape is recorded and compared separately
KERNEL_SOURCES = ("paper_astro_ph_0702058_gb300/csrc/force_impl.cuh", "paper_astro_ph_0702058_gb300/csrc/ptx.cuh",
                  "paper_astro_ph_0702058_gb300/csrc/force_x2.cuh",
                  "paper_astro_ph_0702058_gb300/csrc/force_dispatch.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "force_kernel_traffic_n1048576.json")


def kernel_code_digest():
    """SHA-256 of the force kernel's sources with // comments and blank lines removed, so that
    only code changes invalidate a recorded measurement."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel)) as f:
            for line in f:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def measured_traffic(mode, n, launch=None):
    """DRAM bytes per force launch from the committed ncu capture, or None when that
    capture was of another size or launch shape, or the kernel source has changed since."""
    import hashlib
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256(kernel_code_digest().encode())
    if rec.get("source_sha256") != h.hexdigest() or rec.get("n") != n or mode not in rec:
        return None
    if launch is not None and list(rec[mode].get("launch", [])) != list(launch):
        return None
    return rec[mode]["dram_read_bytes"] + rec[mode]["dram_write_bytes"]


def roofline(force_ms_avg, n, sm_count, clocks, peaks, mode="comp", launch=None):
    max_mhz = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
    pairs = n * (n - 1)
    achieved = pairs / (force_ms_avg * 1e-3) / 1e9
    peak = sm_count * FP32_LANES_PER_SM * max_mhz * 1e6 / OPS_PER_PAIR / 1e9
    out = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 2), "unit": "Gpair/s",
           "frac": round(achieved / peak, 4), "traffic": measured_traffic(mode, n, launch),
           "traffic_unit": "bytes per launch (ncu dram read + write)",
           "peak_basis": f"{sm_count} SM x {FP32_LANES_PER_SM} FP32 lanes x {max_mhz:.0f} MHz / "
                         f"{OPS_PER_PAIR} FP32 ops per pair (derived from unit counts and the max SM clock)"}
    if clocks.get("sm_mhz"):
        at_clock = sm_count * FP32_LANES_PER_SM * clocks["sm_mhz"] * 1e6 / OPS_PER_PAIR / 1e9
        out["frac_at_sampled_clock"] = round(achieved / at_clock, 4)
    return out


def cpu_baseline(m, x, v, n, target_s=12.0):
    """FP64 oracle, one step of the same workload on a bounded sample of active rows."""
    import numpy as np

    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    st = oracle.State(m, x, v, EPS2, 0.02, lmin=LEVEL, lmax=LEVEL)
    st.level[:] = LEVEL
    t_new = 1
    xp, vp = st.predict(t_new)        # predictor over all N (part of the sample's cost)
    rows = 64
    t0 = time.perf_counter()
    act = np.arange(rows, dtype=np.int32)
    fa, fk, _ = oracle.force(m, xp, vp, EPS2, act)
    dt = time.perf_counter() - t0
    rows = int(min(n, max(rows, rows * target_s / max(dt, 1e-3))))
    act = np.linspace(0, n - 1, rows).astype(np.int32)
    t0 = time.perf_counter()
    xp, vp = st.predict(t_new)
    fa, fk, _ = oracle.force(m, xp, vp, EPS2, act)
    st.correct(act, xp, vp, fa, fk, t_new)
    dt = time.perf_counter() - t0
    out = {"value": rows * (n - 1) / dt, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
           "sample": f"one step (predict all {n}, force on {rows} evenly spaced rows against all {n}, "
                     f"correct those rows) in FP64, {dt:.1f} s"}
    # the same oracle force on one thread, on a smaller sample of rows
    oracle.set_threads(1)
    rows1 = max(8, rows // max(1, cores))
    t0 = time.perf_counter()
    oracle.force(m, xp, vp, EPS2, np.linspace(0, n - 1, rows1).astype(np.int32))
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    out["single_thread"] = {"value": rows1 * (n - 1) / dt1, "sample": f"force on {rows1} rows, {dt1:.1f} s"}
    return out


def bench_ours(args):
    import numpy as np
    import torch

    from synthetic import plummer_sphere
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    n = args.n
    m, x, v = plummer_sphere(n, SEED + rank)  # independent replica per rank
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = measured_peaks()
    res = {}
    energy = {}
    with torch.cuda.stream(stream):
        for mode in ("comp", "plain"):
            sim = make_sim(m, x, v, mode, stream)
            if not energy:
                energy["e0"] = sum(sim.energy(ds_potential=True))  # t = 0: the same state in every mode
            first = {}
            barrier(ws)
            with ClockSampler(local) as cs:
                t0 = time.perf_counter()
                total_ms, force_ms, launches = run_steps(
                    sim, n, args.steps, args.warmup, stream, flush,
                    after_first=lambda: first.setdefault("e", sum(sim.energy(ds_potential=True))))
                wall = time.perf_counter() - t0
            clocks = cs.summary()
            cfg = sim.stats()
            energy[mode] = {"end": sum(sim.energy(ds_potential=True)), "first": first.get("e")}
            sim.close()
            res[mode] = {"total_ms": total_ms,
                         "force_ms": statistics.mean(force_ms), "launches": launches, "clocks": clocks,
                         "wall_s": wall, "shape": f"{cfg['last_threads']} threads x {cfg['last_i_per_thread']} "
                                                  f"i/thread, j-split {cfg['last_j_split']}",
                         "launch": [cfg["last_threads"], cfg["last_i_per_thread"], cfg["last_j_split"]]}
        # end to end: pinned host list in/out and forces back to the host every step
        sim = make_sim(m, x, v, "comp", stream)
        host = (torch.zeros(n, dtype=torch.int32).pin_memory(), torch.zeros((n, 3), dtype=torch.float64).pin_memory(),
                torch.zeros((n, 3), dtype=torch.float64).pin_memory(), torch.zeros(n, dtype=torch.float64).pin_memory())
        barrier(ws)
        e2e_ms, _, _ = run_steps(sim, n, args.steps, args.warmup, stream, flush, host=host)
        sim.close()
        totals = replica_totals(ws, {mode: r["total_ms"] for mode, r in res.items()}, e2e_ms,
                                args.steps * n * (n - 1))
        for mode, r in res.items():
            t_max = totals[mode]["t_max"]
            r.update(value=totals[mode]["pairs"] / (t_max * 1e-3), ms_per_step=t_max / args.steps)
        if rank == 0 and not args.no_energy_reference:
            # one step in double-single pair arithmetic (~1e-12 from FP64): the FP64 oracle's stand-in,
            # since the oracle itself would need ~1e12 FP64 pair terms per step on the host
            with make_sim(m, x, v, "ds", stream) as sim:
                lst = torch.zeros(n, dtype=torch.int32, device="cuda")
                t_blk, n_act = sim.next_block(lst)
                sim.predict(t_blk)
                sim.force(lst, n_act)
                sim.correct(lst, n_act)
                energy["ds"] = {"first": sum(sim.energy(ds_potential=True))}
    out = None
    if rank == 0:
        c = res["comp"]
        p = res["plain"]
        rl_c = roofline(c["force_ms"], n, sm_count, c["clocks"], peaks, "comp", c["launch"])
        rl_p = roofline(p["force_ms"], n, sm_count, p["clocks"], peaks, "plain", p["launch"])
        e0 = energy["e0"]
        rel = lambda e: None if e is None else abs((e - e0) / e0)  # noqa: E731
        steps_all = args.warmup + args.steps
        energy_info = {
            "segment": f"this run: {steps_all} full-force Hermite steps of dt = 2^-{LEVEL} from t = 0 "
                       f"(warm-up and timed), t_end = {steps_all}/{1 << LEVEL}",
            "diagnostic": "|E(t_end) - E(0)| / |E(0)|; E_kin FP64, E_pot double-single (nbody_energy_ds, "
                          "~1e-13 relative), outside the timed events",
            "after_first_step": {"comp": rel(energy["comp"]["first"]), "plain": rel(energy["plain"]["first"]),
                                 "ds_fp64_standin": rel(energy.get("ds", {}).get("first"))},
            "fp64_standin": "double-single pair arithmetic (NBODY_MODE_DS, ~1e-12 from the FP64 definition) "
                            "for the FP64 oracle, which cannot run this size"}
        out = {
            "metric": METRIC, "value": c["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": c["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "precision": "compensated: FP32 pair math on hi/lo splits of FP64 positions, double-single sums; "
                         "FP64 predictor, corrector, time bins and state",
            "data": "synthetic (seeded Plummer sphere, Henon units)",
            "config": {"workload": f"Plummer N={n} eps=1e-3, full-force Hermite block step (all N active, "
                                   f"shared level dt=2^-{LEVEL}): schedule+predict+force+correct",
                       "n": n, "n_act": n, "pairs_per_step": n * (n - 1), "l2": "flushed between steps "
                       f"({L2_FLUSH_BYTES >> 20} MiB write, outside the timed events)",
                       "force_launch_shape": c["shape"], "parallelism": f"replicas x{ws}"},
            "roofline": rl_c,
            "energy_error": rel(energy["comp"]["end"]),
            "energy": energy_info,
            "plain": {"value": p["value"], "ms_per_step": p["ms_per_step"], "roofline": rl_p,
                      "energy_error": rel(energy["plain"]["end"]),
                      "force_launch_shape": p["shape"], "clocks": p["clocks"]},
            "comp_over_plain": c["value"] / p["value"],
            "e2e": {"value": totals["e2e"]["pairs"] / (totals["e2e"]["t_max"] * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": 2 * 4 * n, "d2h_bytes_per_step": 4 * n + 7 * 8 * n},
            "gpu_launches": c["launches"],
            "clocks": c["clocks"],
            "context": {"paper_8800GTX_pairs_per_s": 1.23e9, "paper_GRAPE6Af_pairs_per_s": 2.16e9,
                        "note": "Table 4 per-interaction times of the paper, other hardware; not a target"},
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(m, x, v, n)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


def bench_reference(args):
    """The reference arm: the FP64 oracle, timed on the host cores, same workload and metric."""
    import numpy as np

    import oracle
    from synthetic import plummer_sphere
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    n = args.n
    m, x, v = plummer_sphere(n, SEED)
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    st = oracle.State(m, x, v, EPS2, 0.02, lmin=LEVEL, lmax=LEVEL)
    st.level[:] = LEVEL
    per_step_s = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    rows = 16
    times = []
    for it in range(args.warmup + args.steps):
        act = np.linspace(0, n - 1, rows).astype(np.int32)
        t0 = time.perf_counter()
        xp, vp = st.predict(int(st.t.max()) + 1)
        fa, fk, _ = oracle.force(m, xp, vp, EPS2, act)
        st.correct(act, xp, vp, fa, fk, int(st.t.max()) + 1)
        st.level[:] = LEVEL
        st.t[:] = st.t.max()
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append((rows, dt))
        rows = int(min(n, max(16, rows * per_step_s / max(dt, 1e-3))))
    pairs = sum(r * (n - 1) for r, _ in times)
    secs = sum(t for _, t in times)
    value = pairs / secs
    sample = (f"each step: predict all {n}, force on a bounded sample of evenly spaced rows "
              f"(~{per_step_s:.0f} s of CPU work) against all {n}, correct those rows; FP64")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Plummer sphere, Henon units)",
            "config": {"workload": f"Plummer N={n} eps=1e-3, full-force Hermite block step (all N active, "
                                   f"shared level dt=2^-{LEVEL}): schedule+predict+force+correct", "n": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def force_only(args):
    """One nbody_force per mode, untimed: the launch that profilers capture.  A Plummer sphere of
    --n particles (seed --seed, softening --eps2; default the benchmark's), after nbody_init's full
    force; the call covers all particles, or --rows of them (a seeded sorted uniform sample)."""
    import torch

    from paper_astro_ph_0702058_gb300 import Simulation
    from synthetic import active_subset, plummer_sphere
    seed = SEED if args.seed is None else args.seed
    eps2 = EPS2 if args.eps2 is None else args.eps2
    m, x, v = plummer_sphere(args.n, seed)
    rows = args.n if args.rows is None else args.rows
    if rows == args.n:
        act = torch.arange(args.n, dtype=torch.int32, device="cuda")
    else:
        act = torch.from_numpy(active_subset(args.n, rows, 2)).to("cuda")
    for mode in args.modes.split(","):
        with Simulation(m, x, v, eps2, mode=mode) as sim:
            sim.predict(0.0)
            sim.force(act, rows)
            sim.sync()
    print(json.dumps({"force_only": args.n, "rows": rows, "seed": seed, "eps2": eps2, "modes": args.modes}))


def c2_sweep(args):
    """C2 force-only sweep: N = 65536 Plummer sphere (seed 2, eps = 1/256), one nbody_force per
    call on a seeded sorted uniform sample of n_act particles, n_act in {1, 32, 1024, 1594
    (about the mean block 0.2 N^0.81), 32768, 65536}; interactions/s = n_act (N - 1) / t, t the
    median CUDA-event time of 20 calls after 3 warm-up calls on the context stream, plain and
    compensated.  The 3 MB j-stream stays resident in L2 across calls: that is the regime of the
    block steps this sweep stands for, so no flush between calls."""
    import torch

    from paper_astro_ph_0702058_gb300 import Simulation
    from synthetic import active_subset, plummer_sphere
    n, eps2 = 65536, (1.0 / 256) ** 2
    m, x, v = plummer_sphere(n, 2)
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    rows = []
    for mode in args.modes.split(","):
        with torch.cuda.stream(stream), Simulation(m, x, v, eps2, eta=0.02, mode=mode, stream=stream) as sim:
            sim.predict(0.0)
            for n_act in (1, 32, 1024, 1594, 32768, 65536):
                act = torch.from_numpy(active_subset(n, n_act, 2)).to("cuda")
                for _ in range(3):
                    sim.force(act, n_act)
                ts = []
                for _ in range(20):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    sim.force(act, n_act)
                    e1.record(stream)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1) * 1e-3)
                t = statistics.median(ts)
                st = sim.stats()
                rows.append({"mode": mode, "n_act": n_act, "us": t * 1e6, "interactions_per_s": n_act * (n - 1) / t,
                             "threads": st["last_threads"], "i_block": st["last_i_per_thread"],
                             "j_split": st["last_j_split"]})
    # cpu_baseline leg: the FP64 oracle on the same inputs (all host cores, then one), 1594 sampled rows
    import oracle
    cores = len(os.sched_getaffinity(0))
    act = active_subset(n, 1594, 2)
    orc = {}
    for threads in (cores, 1):
        oracle.set_threads(threads)
        rows_t = act if threads == cores else act[:max(16, 1594 // cores)]
        t0 = time.perf_counter()
        oracle.force(m, x, v, eps2, rows_t)
        orc[f"threads_{threads}"] = len(rows_t) * (n - 1) / (time.perf_counter() - t0)
    oracle.set_threads(cores)
    print(json.dumps({"workload": "c2 force-only sweep", "n": n, "eps": 1.0 / 256, "rows": rows,
                      "cpu_baseline": {"kind": "oracle", "interactions_per_s": orc,
                                       "sample": "1594 sampled rows (n_act = 1594 set) against all N, FP64"}}),
          flush=True)


def c1_run(args):
    """C1: N = 1024 Plummer (seed 1), eps = 1/256, eta = 0.01, dt_max = 1/64, dt_min = 2^-26, from t = 0 to
    1/8, in every force mode and in the FP64 oracle: blocks, wall time and |dE/E| (--c1-n: other N)."""
    import torch

    import oracle
    from paper_astro_ph_0702058_gb300 import Simulation
    from synthetic import plummer_sphere
    n, eps2, t_end = args.c1_n, (1.0 / 256) ** 2, 0.125
    m, x, v = plummer_sphere(n, 1)
    torch.cuda.set_device(0)
    from paper_astro_ph_0702058_gb300 import nbody_debug_step_graphs
    t_end = args.t_end if args.t_end is not None else t_end
    nbody_debug_step_graphs(args.step_graphs)
    rows = []
    for mode in args.c1_modes.split(","):
        with Simulation(m, x, v, eps2, eta=0.01, lmin=6, lmax=26, mode=mode) as sim:
            e0 = sum(sim.energy())
            sim.sync()
            t0 = time.perf_counter()
            blocks = sim.step(t_end)
            sim.sync()
            wall = time.perf_counter() - t0
            e1 = sum(sim.energy())
            st = sim.stats()
        # cluster_blocks / grid_blocks: blocks run by the one-cluster / whole-GPU kernel; graph_blocks: blocks run inside
        # step-graph replays; loop_blocks: of those, the ones the device-side loop ran without a host
        # round trip
        rows.append({"mode": mode, "blocks": int(blocks), "wall_s": wall, "us_per_block": wall / max(blocks, 1) * 1e6,
                     "energy_error": abs((e1 - e0) / e0), "cluster_blocks": int(st["cluster_blocks"]),
                     "grid_blocks": int(st["grid_blocks"]), "graph_blocks": int(st["graph_blocks"]),
                     "loop_blocks": int(st["loop_blocks"])})
    nbody_debug_step_graphs(3)
    if args.no_cpu_baseline:
        print(json.dumps({"workload": "c1", "n": n, "eps2": eps2, "eta": 0.01, "t_end": t_end, "rows": rows}),
              flush=True)
        return
    # cpu_baseline leg: the FP64 oracle's own run of C1 on the host cores
    oracle.set_threads(len(os.sched_getaffinity(0)))
    st = oracle.State(m, x, v, eps2, 0.01, lmin=6, lmax=26).init()
    e0 = sum(st.energy())
    t0 = time.perf_counter()
    bt, _, _ = st.evolve(int(t_end * 2 ** 26))
    wall = time.perf_counter() - t0
    base = {"kind": "oracle", "blocks": len(bt), "wall_s": wall, "cores": oracle.get_threads(),
            "energy_error": abs((sum(st.energy()) - e0) / e0), "sample": "the whole C1 run, FP64"}
    print(json.dumps({"workload": "c1", "n": n, "eps2": eps2, "eta": 0.01, "t_end": t_end, "rows": rows,
                      "cpu_baseline": base}), flush=True)


def block_run(args):
    """Free-running block steps: C3 (N = 2^20, seed 3, eps = 1e-3, to t = 1/64) or C2 (N = 65536,
    seed 2, eps = 1/256, to t = 1), eta = 0.02, dt_max = 1/64, dt_min = 2^-26, both modes.  Reports
    blocks, mean block size, pair-interactions/s over the run (host loop through the public
    nbody_step, wall clock after a synchronised start) and the relative energy error.  C2 also runs the
    double-single mode, whose drift stands in for the FP64 oracle's at this length."""
    import torch

    from paper_astro_ph_0702058_gb300 import Simulation
    from synthetic import plummer_sphere
    if args.workload == "c3-blocks":
        n, seed, eps2, t_end = N_DEFAULT if args.n == N_DEFAULT else args.n, 3, 1e-6, 1.0 / 64
    else:
        n, seed, eps2, t_end = 65536, 2, (1.0 / 256) ** 2, 1.0
    m, x, v = plummer_sphere(n, seed)
    torch.cuda.set_device(0)
    rows = []
    modes = args.modes.split(",")
    if args.workload == "c2-blocks" and args.modes == "plain,comp":
        modes.append("ds")  # double-single forces: the FP64-equivalent drift to compare with (C2 is too long for the CPU oracle)
    ds_energy = n > (1 << 17)  # the FP64 potential of 2^20 particles takes ~40 s on GB300's FP64 unit
    for mode in modes:
        t0 = time.perf_counter()
        with Simulation(m, x, v, eps2, eta=0.02, lmin=6, lmax=26, mode=mode) as sim:
            sim.sync()
            t_init = time.perf_counter() - t0
            e0 = sum(sim.energy(ds_potential=ds_energy))
            p0 = sim.stats()["pairs"]
            t1 = time.perf_counter()
            blocks = sim.step(t_end)
            sim.sync()
            wall = time.perf_counter() - t1
            st = sim.stats()
            e1 = sum(sim.energy(ds_potential=ds_energy))
        pairs = st["pairs"] - p0
        rows.append({"mode": mode, "blocks": int(blocks), "mean_block": pairs / max(1, blocks) / (n - 1),
                     "pairs": int(pairs), "wall_s": wall, "pairs_per_s": pairs / wall, "init_s": t_init,
                     "energy_error": abs((e1 - e0) / e0), "below_dt_min": int(st["below_dt_min"]),
                     "grid_blocks": int(st["grid_blocks"]),
                     "energy": "double-single potential" if ds_energy else "FP64"})
    print(json.dumps({"workload": args.workload, "n": n, "eps2": eps2, "eta": 0.02, "t_end": t_end,
                      "rows": rows}), flush=True)


# The paper's full-integration wall-clock over t = 0.25 -> 0.5 (Table 2, seconds), other hardware: context only.
TABLE2_PAPER_S = {1024: {"GRAPE6Af": 0.3327, "8800GTX": 17.46, "FX1400": 20.20, "Xeon": 2.584},
                  16384: {"GRAPE6Af": 16.32, "8800GTX": 924.4, "FX1400": 3398.0, "Xeon": 994.0},
                  65536: {"GRAPE6Af": 178.2, "8800GTX": 3973.0, "FX1400": 40560.0, "Xeon": 19290.0},
                  524288: {"8800GTX": 63960.0}}


def table2_run(args):
    """The paper's timed integration (Sect. 4, Table 2): an equal-mass Plummer sphere (seed 2), eps = 1/256,
    eta = 0.01, dt_max = 1/8, dt_min = 2^-26, from t = 0 to 0.5, timed from t = 0.25 to 0.5 (wall clock around
    nbody_step after a synchronised start), plain and compensated.  Reports blocks, pair interactions per second
    and |dE/E| over the timed interval, with the paper's wall clock for the same N as context."""
    import torch

    from paper_astro_ph_0702058_gb300 import Simulation
    from synthetic import plummer_sphere
    torch.cuda.set_device(0)
    eps2, eta = (1.0 / 256) ** 2, 0.01
    out = []
    for n in (int(v) for v in args.table2_n.split(",")):
        m, x, v = plummer_sphere(n, 2)
        rows = []
        for mode in args.modes.split(","):
            with Simulation(m, x, v, eps2, eta=eta, lmin=3, lmax=26, mode=mode) as sim:
                sim.step(0.25)
                sim.sync()
                e0 = sum(sim.energy())
                st0 = sim.stats()
                t0 = time.perf_counter()
                blocks = sim.step(0.5)
                sim.sync()
                wall = time.perf_counter() - t0
                st = sim.stats()
                e1 = sum(sim.energy())
            pairs = st["pairs"] - st0["pairs"]
            rows.append({"mode": mode, "blocks": int(blocks), "wall_s": wall, "pairs": int(pairs),
                         "pairs_per_s": pairs / wall, "energy_error": abs((e1 - e0) / e0),
                         "cluster_blocks": int(st["cluster_blocks"] - st0["cluster_blocks"]),
                         "grid_blocks": int(st["grid_blocks"] - st0["grid_blocks"])})
        out.append({"n": n, "rows": rows, "paper_wall_s": TABLE2_PAPER_S.get(n)})
    print(json.dumps({"workload": "table2", "eps2": eps2, "eta": eta, "dt_max": 0.125, "timed": [0.25, 0.5],
                      "runs": out, "context": "paper Table 2: other hardware, FP32 on the GPUs; not a target"}),
          flush=True)


def diff_workload(args):
    """C5: loss and gradient of a shared-step Hermite rollout (N = 4096 Plummer, seed 5,
    eps = 1/128, 256 steps of 2^-9, checkpoints every 16 steps) through nbody_diff_rollout,
    plain mode; 1 warm-up and 3 timed calls (the call waits for its result)."""
    import numpy as np
    import torch

    from paper_astro_ph_0702058_gb300 import MODES
    from paper_astro_ph_0702058_gb300._lib import nbody_diff_rollout
    from synthetic import plummer_sphere
    n, steps, level, ck = 4096, 256, 9, 16
    m, x, v = plummer_sphere(n, 5)
    torch.cuda.set_device(0)
    dm, dx, dv = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (m, x, v))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    gx, gv, gm = torch.zeros_like(dx), torch.zeros_like(dv), torch.zeros_like(dm)
    stream = torch.cuda.current_stream()
    call = lambda: nbody_diff_rollout(n, dm, dx, dv, (1.0 / 128) ** 2, level, steps, ck, MODES["plain"],
                                      loss, gx, gv, gm, stream)
    call()
    torch.cuda.synchronize()
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        call()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    # forward (steps + 1 forces), recomputed segments (steps forces), one force VJP per force
    pair_passes = (steps + 1) + steps + (steps + 1)
    print(json.dumps({"workload": "diff (C5)", "n": n, "steps": steps, "dt": 2.0 ** -level,
                      "checkpoint_every": ck, "ms_per_gradient": t * 1e3, "gradients_per_s": 1.0 / t,
                      "pair_passes": pair_passes, "pairs_per_s": pair_passes * n * (n - 1) / t,
                      "loss": float(loss.item()), "grad_norm": float(torch.linalg.norm(gx).item())}), flush=True)


def pipe_probe(args):
    """The roofline's unit rates, measured: FP32 FMA / ADD / MUL, packed FP32x2 FMA and MUFU rsqrt
    results per SM per clock (csrc/pipe_probe.cu, chains of independent accumulators), the FP64 FMA and
    conversion rates, and the cycles per operation of one dependent FP64 chain (FMA, square root,
    division) in one block of 1 to 16 warps."""
    from paper_astro_ph_0702058_gb300 import build as nb_build
    exe = nb_build.build_probe()
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    line = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else "{}"
    out = {"workload": "pipe-probe", "rc": r.returncode}
    try:
        out.update(json.loads(line))
    except ValueError:
        out["raw"] = line
    print(json.dumps(out), flush=True)


def ensemble_workload(args):
    """C4: 512 independent Plummer clusters (sizes log-uniform in [256, 8192) from seed 4),
    eps = 1/256, eta = 0.02, integrated to t = 1/4 as one batched, graph-replayed run
    (tuned launch shape), against one context per cluster on a systematic sample."""
    import numpy as np
    import torch

    from paper_astro_ph_0702058_gb300 import Ensemble, Simulation
    from synthetic import ensemble_sizes, plummer_sphere
    n_cl, t_end, eps2, mode = args.clusters, 0.25, (1.0 / 256) ** 2, args.ens_mode
    sizes = ensemble_sizes(n_cl, 4)
    parts = [plummer_sphere(int(n), 4_000_000 + c) for c, n in enumerate(sizes)]
    m = np.concatenate([p[0] for p in parts])
    x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    torch.cuda.set_device(0)
    with Ensemble(sizes, m, x, v, eps2, eta=0.02, mode=mode) as ens:
        ek0, ep0 = ens.energy()
        e0 = ek0 + ep0
        shape = ens.tune(t_end, steps=4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps = ens.run(t_end)
        wall = time.perf_counter() - t0
        st = ens.stats()
        ek, ep = ens.energy()
    pairs = int(st["pairs"].sum())
    # one context per cluster, each advanced by nbody_step (small blocks in its device-side block
    # loop, one CUDA graph replay per up to 1024 blocks); the stepping alone is timed, after the
    # context's set-up (allocations, the t = 0 force), which is reported separately
    sample = list(range(0, n_cl, max(1, n_cl // args.ens_sample))) if args.ens_sample > 0 else []
    single = setup = 0.0
    single_pairs = 0
    for c in sample:
        mc, xc, vc = parts[c]
        t0 = time.perf_counter()
        with Simulation(mc, xc, vc, eps2, eta=0.02, mode=mode) as sim:
            sim.sync()
            t1 = time.perf_counter()
            sim.step(t_end)
            sim.sync()
            single += time.perf_counter() - t1
            setup += t1 - t0
            single_pairs += sim.stats()["pairs"] - len(mc) * (len(mc) - 1)  # without the t = 0 force
    per_cluster_s = single / len(sample) if sample else float("nan")
    out = {"workload": "ensemble", "clusters": n_cl, "particles": int(sizes.sum()), "mode": mode,
           "t_end": t_end, "batched_steps": int(steps), "blocks_total": int(st["blocks"].sum()),
           "wall_s": wall, "clusters_per_s": n_cl / wall, "pairs": pairs, "pairs_per_s": pairs / wall,
           "tuned_shape": {"threads": shape[0], "i_block": shape[1], "tiles_per_range": shape[2],
                           "ms_per_batched_step_in_tuning": shape[3]},
           "one_context_per_cluster": {"sample": len(sample), "s_per_cluster": per_cluster_s,
                                       "clusters_per_s": 1.0 / per_cluster_s,
                                       "pairs_per_s": single_pairs / single if sample else None,
                                       "stepping": "nbody_step: the one-cluster block-step kernel (n_pad <= 4096), "
                                                   "the whole-GPU block-step kernel above",
                                       "setup_s_per_cluster": setup / len(sample) if sample else None},
           "speedup_clusters_per_s": (n_cl / wall) * per_cluster_s,
           "energy_error_median": float(np.median(np.abs((ek + ep - e0) / e0))),
           "energy_error_max": float(np.max(np.abs((ek + ep - e0) / e0)))}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_DEFAULT, help="particles (default 2^20)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-energy-reference", action="store_true",
                    help="skip the one double-single step that stands in for the FP64 oracle's energy error")
    ap.add_argument("--force-only", action="store_true",
                    help="run one force call per mode on all N particles (for profilers), no timing")
    ap.add_argument("--modes", default="plain,comp")
    ap.add_argument("--workload", choices=["c3", "ensemble", "c1", "c2-sweep", "c3-blocks", "c2-blocks", "diff", "pipe-probe",
                                           "table2"], default="c3",
                    help="c3: the headline full-force steps at N = 2^20; ensemble: the 512-cluster batched run; "
                         "c2-sweep: force-only rates against the block size at N = 65536; c3-blocks / c2-blocks: "
                         "free-running block steps at N = 2^20 to t = 1/64 / N = 65536 to t = 1; diff: rollout gradient (C5); "
                         "pipe-probe: FP32 / FP32x2 / MUFU unit rates; c1: the C1 run in every mode and the oracle; "
                         "table2: the paper's timed integration (t = 0.25 to 0.5, eta = 0.01, dt_max = 1/8)")
    ap.add_argument("--clusters", type=int, default=512)
    ap.add_argument("--ens-sample", type=int, default=32,
                    help="clusters run one context each, for comparison (0: skip the comparison)")
    ap.add_argument("--ens-mode", default="comp")
    ap.add_argument("--rows", type=int, default=None, help="--force-only: rows of the call (default: all)")
    ap.add_argument("--seed", type=int, default=None, help="--force-only: seed of the sphere (default 3)")
    ap.add_argument("--eps2", type=float, default=None, help="--force-only: softening squared (default 1e-6)")
    ap.add_argument("--c1-modes", default="plain,comp,sorted,ds", help="c1: the force modes to run")
    ap.add_argument("--c1-n", type=int, default=1024, help="c1: particles (default 1024, the C1 configuration)")
    ap.add_argument("--step-graphs", type=int, default=3,
                    help="c1: 0 separate launches per block, 1 one graph replay per block, 2 the device-side loop, "
                         "3 the one-cluster block-step kernel")
    ap.add_argument("--t-end", type=float, default=None, help="c1: end time (a multiple of 1/64; default 1/8)")
    ap.add_argument("--table2-n", default="1024,16384,65536", help="table2: particle numbers (524288 takes minutes)")
    args = ap.parse_args(argv)
    if args.force_only:
        force_only(args)
        return
    if args.workload == "ensemble":
        ensemble_workload(args)
        return
    if args.workload == "c2-sweep":
        c2_sweep(args)
        return
    if args.workload in ("c3-blocks", "c2-blocks"):
        block_run(args)
        return
    if args.workload == "diff":
        diff_workload(args)
        return
    if args.workload == "pipe-probe":
        pipe_probe(args)
        return
    if args.workload == "c1":
        c1_run(args)
        return
    if args.workload == "table2":
        table2_run(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    out = bench_reference(args) if args.impl == "reference" else bench_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

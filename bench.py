#!/usr/bin/env python3
"""Particle-steps per second of the rounded-polytope DEM on GB300.

Workload (default): 512 independent replica systems, N_k ~ U{128..2048}
rounded cubes / tetrahedra / triangular prisms (rounding 0.1-0.2, packing
fraction 0.30-0.55), NVT at kT = 1, dt = 1e-3, all replicas advanced by
one captured step graph per step (pair kernel in FP32 with two-sum
accumulation, state, energies and virials in FP64).

One bench step = one full timestep of every replica: thermostat half
steps, half kicks, drift and free rotation, neighbour-list rebuild when
due, the pair-feature kernel, reductions.  The state is prepared first
(lattice start with bounding spheres one cutoff apart, compression on the
GPU to each replica's packing fraction, equilibration) and is resident in
HBM when the timed region starts.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and FP32-peak fraction, FP32+comp batched vs plain FP64, 1 GB300"
UNIT = "particle-steps/s"

# GB300: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz maximum SM clock.
# The roofline uses the measured FMA rates (dem_fma_peak); these nominal
# figures are reported beside them for context.
SMS, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_GHZ / 1e3
FP64_PEAK_TFLOPS = 1.25   # GB300 nominal dense FP64 rate (far below the FP32 rate)

# FP32 flops of each counted code path of the pair kernel (FMA = 2, add /
# mul / reciprocal = 1, compare = 0), hand-counted from csrc/pair.cu and
# csrc/pair_common.cuh.  Keys are dem_get_counters indices.
FLOPS_PER_PATH = {
    10: 15,  # list entry: separation d0 + delta_j - delta_i (6) + range test (9)
    0: 106,  # in-range pair: relative quaternion conj(q_i) q_j (28), M from
             # it (30), dl = R_i^T d (15), sigma terms (2), centre-line axis in
             # both frames (26) and the separating-axis bounds (5)
    16: 5,   # vertex projection onto the centre line
    3: 23,   # vertex transform into the other frame (18) + reach test (5)
    4: 6,    # face-plane signed distance
    5: 6,    # in-plane edge test of a face
    6: 23,   # point-segment nearest point
    7: 46,   # edge transform (33) + centre (6) + reach test (7)
    8: 17,   # edge bounding-sphere test
    17: 24,  # carrier-line distance test (cross product, two dots, compare)
    9: 73,   # segment-segment nearest points (Section "Model" parallel rule included)
    11: 7,   # projection onto the face
    2: 35,   # WCA term in i's frame (force, torque, energy, sums)
    12: 15,  # extra rotation of a term evaluated in j's frame
}
WORK_COUNTERS = {0: "pairs", 1: "feature_pairs", 2: "terms", 3: "vertex_transforms",
                 4: "plane_tests", 5: "inplane_tests", 6: "point_segment",
                 7: "edge_transforms", 8: "edge_sphere_tests", 9: "segment_segment",
                 10: "list_entries", 11: "inside", 12: "jframe_terms",
                 15: "active_pairs", 16: "sat_projections", 17: "line_tests"}
TWO_SUM_EXTRA = 30   # compensated sums: 6 components x (6 - 1) extra flops per term
# FP32 + two-sum: every term re-evaluated in float-float (csrc/ff.cuh,
# refined_values), hand-counted in FP32 flops (FMA = 2; ff_add 11, ff_mul 10,
# ff_mul_f 8, a quaternion rotation 288): four rotations (1152), the
# separation with its image and sigma_ij (99), the nearest points (a foot on
# a segment 158; the edge-pair solve 590), rv and r^2 (85), the WCA factor
# (107), force and torque (123), virial and sums (75).  Counted per term with
# the foot (1799); edge-pair terms take about 430 more.
REFINE_PER_TERM = 1799
SPLIT_EXPAND = 32    # SPLIT feature kernel, per active-pair record: M from the
                     # relative quaternion (30), r_cut and sigma^2 (2)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=100)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="batched",
                   choices=["batched", "cubes", "large", "squares", "octahedra", "spheres",
                            "cubes_fluid", "icosahedra"])
    p.add_argument("--energy-drift", action="store_true",
                   help="instead of the throughput line: NVE energy drift and short-term "
                        "fluctuation of the Section 'Energy Conservation' fluids per precision")
    p.add_argument("--drift-steps", type=int, default=100000)
    p.add_argument("--drift-set", default="all", choices=["all", "fluids", "configs"],
                   help="--energy-drift: the Section 'Energy Conservation' fluids, the "
                        "bench workloads in their own ensembles, or both")
    p.add_argument("--drift-budget", type=float, default=100.0,
                   help="--energy-drift on the bench workloads: seconds per workload and "
                        "precision; a run stops early at this budget and says so")
    p.add_argument("--n", type=int, default=0,
                   help="particles of the spheres / cubes_fluid / icosahedra workloads "
                        "(the paper's table uses 256, 4096 and 65536; default 65536)")
    p.add_argument("--precision", default="fp32c", choices=["fp64", "fp32", "fp32c"])
    p.add_argument("--replicas", type=int, default=512)
    p.add_argument("--compress-steps", type=int, default=3000)
    p.add_argument("--equil-steps", type=int, default=1000)
    p.add_argument("--no-extras", action="store_true",
                   help="skip the e2e, FP64 and CPU-baseline measurements")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--decomp", default="auto", choices=["auto", "thread", "warp", "staged", "split"])
    p.add_argument("--set", action="append", default=[], metavar="NAME=VALUE",
                   help="a dem_set_param parameter, set after the autotune (repeatable)")
    p.add_argument("--execution", default="auto", choices=["auto", "graph", "persistent"],
                   help="dem_step's execution: as dem_autotune chose, per-step kernels replayed "
                        "from a CUDA graph, or the cooperative multi-step kernel")
    p.add_argument("--profile-evals", type=int, default=0,
                   help="after the preparation and the autotune, run this many eager force "
                        "evaluations inside the NVTX range dem_profile (for ncu) and exit")
    return p.parse_args()


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def make_workload(name, rank, replicas, n=0):
    from paper_1607_02427_gb300 import workloads as W
    off = 100 * rank
    if name == "batched":
        s = W.config_batched(n_replicas=replicas, seed_index=3 + off)
        return s, dict(dt=1e-3, ensemble="nvt", kT=1.0, tau=0.5)
    if name == "cubes":
        return W.config_cubes_4096(seed_index=1 + off), dict(dt=1e-3, ensemble="nvt", kT=1.0, tau=0.5)
    if name == "large":
        return W.config_large(seed_index=4 + off), dict(dt=1e-3, ensemble="nvt", kT=1.0, tau=0.5)
    if name == "octahedra":
        return W.config_octahedra(seed_index=2 + off), dict(dt=5e-4, ensemble="nve", kT=1.0, tau=0.5)
    if name in ("spheres", "cubes_fluid", "icosahedra"):
        shape = {"spheres": "sphere", "cubes_fluid": "cube", "icosahedra": "icosahedron"}[name]
        return (W.config_paper_table(shape, n if n else 65536, seed_index=5 + off),
                dict(dt=1e-3, ensemble="nvt", kT=1.0, tau=0.5))
    return W.config_squares_2d(seed_index=0 + off), dict(dt=1e-3, ensemble="nve", kT=1.0, tau=0.5)


def reduce_over_ranks(dist, ms, n, device):
    """Whole-job timing over the ranks: the largest timed milliseconds and the
    total particle count (every rank runs its own replicas; no other data
    crosses ranks)."""
    if dist is None:
        return ms, n
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    nt = torch.tensor([float(n)], dtype=torch.float64, device=device)
    dist.all_reduce(nt)
    return float(t.item()), int(round(nt.item()))


def prepare(dem, system, run, precision, compress_steps, equil_steps):
    """Context at the target density: compress from the safe lattice start
    (NVT, geometric box schedule), then equilibrate."""
    d = dem.DEM(system, precision)
    ens = dem.DEM_NVT
    if system.target_box is not None:
        chunks = 60
        per = max(1, compress_steps // chunks)
        start, target = system.box.copy(), system.target_box.copy()
        for k in range(1, chunks + 1):
            d.set_box(start * (target / start) ** (k / chunks))
            d.step(per, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
    if equil_steps:
        d.step(equil_steps, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
    return d


# ---------------------------------------------------------------------------
# Clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.tmp:
            return None
        self.tmp.flush()
        rows = [r.strip().split(",") for r in open(self.tmp.name) if r.strip()]
        os.unlink(self.tmp.name)
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# Roofline
# ---------------------------------------------------------------------------

def measured_peaks(dem):
    """FP32 and FP64 FMA throughput of this GPU (dem_fma_peak: independent
    FMA chains on every lane of a full-occupancy grid), each launch scaled to
    about 20 ms; best of three launches after a warm-up."""
    out = {}
    for name, p, it0 in (("fp32", dem.DEM_FP32, 16384), ("fp64", dem.DEM_FP64, 256)):
        t, ms = dem.dem_fma_peak(p, it0)
        it = max(4, int(it0 * 20.0 / max(ms, 1e-3)) // 4 * 4)
        t, ms = dem.dem_fma_peak(p, it)
        out[name] = {"tflops": t, "launch_ms": ms, "iters": it}
    return out


def algorithmic_flops(counts, comp, split=True):
    f = sum(FLOPS_PER_PATH[k] * int(counts[k]) for k in FLOPS_PER_PATH)
    if comp:
        f += (TWO_SUM_EXTRA + REFINE_PER_TERM) * int(counts[2])
    if split:
        f += SPLIT_EXPAND * int(counts[15])
    return f


def pair_source_hash():
    h = hashlib.sha256()
    for name in ("pair.cu", "pair_staged.cu", "pair_kernels.cuh", "pair_common.cuh", "ff.cuh"):
        with open(os.path.join(ROOT, "paper_1607_02427_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, precision):
    """DRAM bytes per pair-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = rec.get(f"{workload}/{precision}")
    if not ent or ent.get("source_hash") != pair_source_hash():
        return None
    return ent.get("bytes_per_launch")


# ---------------------------------------------------------------------------
# CPU baseline (the FP64 oracle, as it stands)
# ---------------------------------------------------------------------------

def oracle_sample(system, target_particles=3000, max_step_s=None, run=None):
    """A bounded sample of the workload: its first replicas (all three shapes)
    at their target density, contact-rich lattice start (generator-made).
    With ``max_step_s``, replicas are added while one oracle step of the
    sample stays within that many seconds."""
    import oracle
    from paper_1607_02427_gb300 import workloads as W
    take, n, cost = [], 0, 0.0
    for k in range(system.n_replicas):
        rep = system.replica(k)
        if rep.n > target_particles:       # one large system: a small one like it
            rep = W.sample_like(system, 512)
        rep = W.slab_lattice_start(rep) if rep.dim == 3 else rep
        if max_step_s is not None:
            t0 = time.perf_counter()
            oracle.run(rep, 1, run["dt"], ensemble=run["ensemble"], kT=run["kT"], tau=run["tau"])
            c = time.perf_counter() - t0
            if take and cost + c > max_step_s:
                if k >= 8:
                    break
                continue
            cost += c
        take.append(rep)
        n += rep.n
        if max_step_s is None and n >= target_particles and k >= 2:
            break
        if max_step_s is not None and (cost >= 0.8 * max_step_s or k >= 8):
            break
    return (W.merge(take) if len(take) > 1 else take[0]), len(take)


def _time_oracle_on(sample, run, seconds, steps=None):
    """Oracle steps on ``sample`` in chunks until ``seconds`` have passed (or
    exactly ``steps``); returns (particle-steps/s, steps, seconds)."""
    import oracle
    ens = run["ensemble"]
    th = None
    done, chunk = 0, 5
    t0 = time.perf_counter()
    while (steps is None and time.perf_counter() - t0 < seconds) or (steps is not None and done < steps):
        k = chunk if steps is None else min(chunk, steps - done)
        st, _ = oracle.run(sample, k, run["dt"], ensemble=ens, kT=run["kT"], tau=run["tau"],
                           thermo=th)
        sample = dataclasses.replace(sample, pos=st["pos"], orient=st["orient"], vel=st["vel"],
                                     angmom=st["angmom"])
        th = st["thermo"]
        done += k
    dt = time.perf_counter() - t0
    return sample.n * done / dt, done, dt


def time_oracle(system, run, seconds, steps=None):
    """The FP64 oracle on a bounded sample of the workload, on the host cores.
    value: the oracle as it stands (every pair, one thread).  all_cores: the
    same oracle with its timing options, a cell-list pair search and OpenMP
    over particles on every core (nproc), on a larger sample of the same
    workload (the same pairs and terms; tests/test_oracle_parallel.py)."""
    import oracle
    oracle.build()
    nproc = os.cpu_count() or 1
    sample, nrep = oracle_sample(system)
    oracle.set_parallel(1, False)
    v1, done1, dt1 = _time_oracle_on(sample, run, 0.5 * seconds, steps)
    out = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{nrep} replicas ({sample.n} particles, first replicas of the workload, "
                     f"generator-made start at target density), {done1} FP64 steps, every "
                     f"pair, single thread, {dt1:.1f} s",
           "nproc": nproc}
    big, nrep_b = oracle_sample(system, target_particles=4 * sample.n)
    try:
        oracle.set_parallel(nproc, True)
        threads = min(nproc, oracle.max_threads())
        vm, donem, dtm = _time_oracle_on(big, run, 0.5 * seconds, steps)
    finally:
        oracle.set_parallel(1, False)
    out["all_cores"] = {
        "value": vm, "unit": UNIT, "cores": threads, "kind": "oracle (cell list, OpenMP)",
        "sample": f"{nrep_b} replicas ({big.n} particles), {donem} FP64 steps, cell-list pair "
                  f"search, OpenMP over particles on {threads} threads, {dtm:.1f} s"}
    return out


# ---------------------------------------------------------------------------
# Main
# ---------------------------------------------------------------------------

def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if a.impl == "reference":
        return reference_arm(a, world, rank)
    if a.energy_drift:
        return energy_drift(a, rank)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    __graft_entry__.build()
    from paper_1607_02427_gb300 import dem

    system, run = make_workload(a.workload, rank, a.replicas, a.n)
    prec = dem.PRECISIONS[a.precision]
    ens = dem.DEM_NVT if run["ensemble"] == "nvt" else dem.DEM_NVE
    d = prepare(dem, system, run, prec, a.compress_steps, a.equil_steps)
    stream = torch.cuda.current_stream()
    dem.dem_set_stream(d.ctx, stream.cuda_stream)
    if a.decomp == "auto":
        dem.dem_autotune(d.ctx)
    else:
        d.set_param("decomp", {"thread": 1, "warp": 2, "staged": 3, "split": 4}[a.decomp])
    if a.execution != "auto":
        d.set_param("persistent", 0 if a.execution == "graph" else 1)
    for kv in a.set:
        name, value = kv.split("=", 1)
        d.set_param(name, float(value))
    decomp_name = {1: "thread", 2: "warp", 3: "staged", 4: "split"}[int(d.get_param("decomp"))]
    tune = {}
    if a.decomp == "auto":
        for k, nm in enumerate(["thread64", "thread128", "warp128", "staged128", "split_g32",
                                "split_g16", "split_g8", "split_g4"]):
            tune[nm] = d.get_param(f"autotune_ms_{k}")
        tune["step_ms_graph"] = d.get_param("autotune_step_ms_graph")
        tune["step_ms_persistent"] = d.get_param("autotune_step_ms_persistent")
    if decomp_name == "split":
        decomp_name = f"split, {int(d.get_param('split_group'))} particles per warp"

    if a.profile_evals:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("dem_profile")
        for _ in range(a.profile_evals):
            d.compute()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            counts = d.counters()
            print(json.dumps({"profile_evals": a.profile_evals, "workload": system.name,
                              "particles": system.n, "decomposition": decomp_name,
                              "work_counters": {nm: int(counts[k])
                                                for k, nm in WORK_COUNTERS.items()}}))
        d.close()
        return

    # warm-up
    d.step(a.warmup, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
    # small systems step in cooperative multi-step launches; CUDA events
    # around the pair kernels exist only in the per-step kernels, so those
    # are timed in a separate profiled pass after the timed region
    coop = bool(d.get_param("persistent_used"))
    if not coop:
        d.set_param("profile", 1)
        d.step(1, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])   # capture the profiled graph
        d.set_param("profile", 1)                                      # reset the totals
    rb0 = int(d.counters()[13])
    l0 = d.get_param("launches")

    # timed region
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("dem_timed")
        e0.record(stream)
        d.step(a.steps, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = int(d.get_param("launches") - l0)
    rebuilds = int(d.counters()[13]) - rb0
    if coop:
        d.set_param("profile", 1)
        d.step(min(a.steps, 200), run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
    pair_ms = d.get_param("pair_ms_total") / max(1.0, d.get_param("pair_launches"))
    d.set_param("profile", 0)
    t_max, n_total = reduce_over_ranks(dist, ms, system.n, "cuda")
    value = n_total * a.steps / (t_max / 1e3)

    counts = d.counters()
    flops = algorithmic_flops(counts, prec == dem.DEM_FP32_COMP,
                              split=decomp_name.startswith("split"))
    achieved = flops / (pair_ms / 1e3) / 1e12
    clocks = clk.summary()
    peaks = measured_peaks(dem)
    peak = peaks["fp64" if prec == dem.DEM_FP64 else "fp32"]["tflops"]

    extras = {}
    if not a.no_extras:
        extras = measure_extras(a, dem, d, system, run, ens, prec, torch, peaks)
    cpu = None
    if rank == 0 and world == 1 and not a.no_extras:
        cpu = time_oracle(system, run, a.cpu_seconds)

    if rank != 0:
        d.close()
        return
    pair_fpe = int(counts[1])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec != dem.DEM_FP64 else "f64",
        "data": "synthetic",
        "config": {
            "workload": system.name, "replicas": system.n_replicas, "particles": system.n,
            "precision": {0: "fp64", 1: "fp32", 2: "fp32 pair kernel, two-sum sums, fp64 state"}[prec],
            "ensemble": run["ensemble"], "dt": run["dt"], "graph": True,
            "decomposition": decomp_name,
            "execution": ("cooperative multi-step kernel (list rebuilds between launches)" if coop
                          else "one CUDA graph replay per step"),
            "l2": "inputs larger than L2 (per-step working set > 129 MB)",
            "parallelism": f"replicas x{world}",
        },
        "roofline": {
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": ncu_traffic(a.workload, a.precision),
            "kernel": (f"pair-feature kernel (decomposition {decomp_name})" if not coop else
                       f"pair-feature kernel of the per-step kernels (decomposition {decomp_name}), "
                       "timed in a separate profiled pass of min(steps, 200) steps; the timed "
                       "steps ran the cooperative kernel, whose pair phase has no separate timing"),
            "autotune_ms": tune,
            "kernel_ms": pair_ms,
            "kernel_share_of_step": None if coop else pair_ms / (t_max / a.steps),
            "flops_per_launch": flops, "feature_pairs_per_launch": pair_fpe,
            "work_counters": {name: int(counts[k]) for k, name in WORK_COUNTERS.items()},
            "feature_pairs_per_s": pair_fpe / (pair_ms / 1e3),
            "peak_note": ("measured on this GPU: FMA-chain microbenchmark (dem_fma_peak), "
                          "burst of about 20 ms; frac is of measured"),
            "measured_peaks_tflops": {k: v["tflops"] for k, v in peaks.items()},
            "nominal_peaks_tflops": {"fp32": FP32_PEAK_TFLOPS, "fp64": FP64_PEAK_TFLOPS,
                                     "fp32_note": "152 SMs x 128 lanes x 2 x 2.07 GHz"},
        },
        "gpu_launches": launches,
        "list_rebuilds": rebuilds,
        "clocks": clocks,
    }
    if "e2e" in extras:
        line["e2e"] = extras.pop("e2e")
    if cpu:
        line["cpu_baseline"] = cpu
    if extras:
        line["comparison"] = extras
    print(json.dumps(line))
    d.close()


def measure_extras(a, dem, d, system, run, ens, prec, torch, peaks):
    """End-to-end through the C ABI with host buffers, and the FP64 paths."""
    out = {}
    st = d.state()
    n, dim = system.n, system.dim
    pin = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt).pin_memory()
    h_sid = pin(system.shape_id, torch.int32)
    h_pos, h_or = pin(st["pos"], torch.float64), pin(st["orient"], torch.float64)
    h_vel, h_am = pin(st["vel"], torch.float64), pin(st["angmom"], torch.float64)
    k_e2e = max(3, min(20, a.steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        dem.dem_set_state(d.ctx, h_sid, h_pos, h_or, h_vel, h_am, device_ptrs=0)
        dem.dem_step(d.ctx, 1, run["dt"], ens, run["kT"], run["tau"])
        U, K, H = d.energy()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    out["e2e"] = {"value": n * k_e2e / t_e2e, "unit": UNIT,
                  "h2d_bytes_per_step": int(4 * n + 8 * n * (2 * dim + (4 if dim == 3 else 1)
                                                            + (3 if dim == 3 else 1))),
                  "d2h_bytes_per_step": int(3 * 8 * system.n_replicas),
                  "steps": k_e2e,
                  "what": "per step: dem_set_state from pinned host memory, dem_step(1), "
                          "dem_get_energy to host"}
    # the same state in the other precisions, batched (graph)
    for name, p in (("fp64_batched", dem.DEM_FP64), ("fp32_batched", dem.DEM_FP32)):
        if p == prec:
            continue
        sysc = _with_state(system, st)
        with dem.DEM(sysc, p) as d2:
            k = 20 if p == dem.DEM_FP64 else 200
            dem.dem_autotune(d2.ctx)
            d2.step(3, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d2.step(k, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
            torch.cuda.synchronize()
            out[name] = {"value": n * k / (time.perf_counter() - t0), "unit": UNIT, "steps": k,
                         "decomposition": {1: "thread", 2: "warp", 3: "staged", 4: "split"}[
                             int(d2.get_param("decomp"))],
                         "execution": ("cooperative multi-step kernel"
                                       if d2.get_param("persistent_used") else "graph per step")}
            if p == dem.DEM_FP64:
                # the FP64 pair kernels against the FP64 rate (a few profiled steps)
                d2.set_param("profile", 1)
                d2.step(1, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
                d2.set_param("profile", 1)
                d2.step(5, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
                pms = d2.get_param("pair_ms_total") / max(1.0, d2.get_param("pair_launches"))
                d2.set_param("profile", 0)
                fl = algorithmic_flops(d2.counters(), False,
                                       split=int(d2.get_param("decomp")) == 4)
                ach = fl / (pms / 1e3) / 1e12
                p64 = peaks["fp64"]["tflops"]
                out[name]["roofline"] = {
                    "bound": "alu", "achieved": ach, "peak": p64, "unit": "TFLOP/s",
                    "frac": ach / p64, "kernel_ms": pms,
                    "peak_note": "measured FP64 FMA rate of this GPU (dem_fma_peak)"}
    # plain FP64 single-system path: one context per replica, launch by launch
    if system.n_replicas > 1:
        sample = list(range(0, system.n_replicas, max(1, system.n_replicas // 24)))[:24]
        full = _with_state(system, st)
        k = 5
        tot_n, tot_t = 0, 0.0
        for r in sample:
            sub = full.replica(r)
            with dem.DEM(sub, dem.DEM_FP64, graph=0, persistent=0) as d3:
                d3.step(1, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                d3.step(k, run["dt"], ens, kT=run["kT"], tau_T=run["tau"])
                torch.cuda.synchronize()
                tot_t += time.perf_counter() - t0
                tot_n += sub.n * k
        out["fp64_single_system"] = {"value": tot_n / tot_t, "unit": UNIT,
                                     "sample": f"{len(sample)} replicas one at a time, {k} steps each, no graph"}
    return out


def _with_state(system, st):
    import dataclasses
    return dataclasses.replace(system, pos=st["pos"], orient=st["orient"], vel=st["vel"],
                               angmom=st["angmom"], box=system.target_box
                               if system.target_box is not None else system.box,
                               target_box=None)


def energy_drift(a, rank):
    """Section "Energy Conservation": fluids of squares (edge 4.24 sigma, 2D)
    and tetrahedra (edge 8.49 sigma, 3D) thermalised at T* = 1 (NVT, dt =
    0.005 tau), then from that one state, in each precision:

    * short term: sigma(E/N), the standard deviation of the total energy per
      particle sampled every step over 10 tau of NVE, for each dt of the
      sweep (the paper's fluctuation-versus-timestep figure);
    * long term: the drift of E/N over --drift-steps NVE steps at the
      fluid's production dt (least-squares slope, epsilon per tau).

    Squares run at the paper's dt = 0.01 tau.  Tetrahedra of unit mass and
    uniform-solid inertia are unstable at dt >= 0.008 tau (a tip contact has
    an effective mass of about 0.12 m; the oracle shows the same growth), so
    they run at 0.005 tau.  One JSON line; the paper's FP32 drifts beside."""
    if rank != 0:
        return
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_02427_gb300 import dem
    from paper_1607_02427_gb300 import workloads as W
    torch.cuda.set_device(0)
    fluids = {"squares": dict(system=W.config_energy_drift("square", 16, 0.5), dt=0.01,
                              sweep=[0.001, 0.002, 0.005, 0.01], paper_fp32=1.4e-5),
              "tetrahedra": dict(system=W.config_energy_drift("tetrahedron", 8, 0.4), dt=0.005,
                                 sweep=[0.001, 0.002, 0.005], paper_fp32=6.3e-4)}
    precs = (("fp32", dem.DEM_FP32), ("fp32c", dem.DEM_FP32_COMP), ("fp64", dem.DEM_FP64))
    out = {}
    if a.drift_set == "configs":
        fluids = {}
    for name, f in fluids.items():
        s = f["system"]
        d = prepare(dem, s, dict(dt=0.005, ensemble="nvt", kT=1.0, tau=0.5),
                    dem.DEM_FP64, 3000, 4000)
        try:
            s0 = _with_state(s, d.state())
        finally:
            d.close()
        res = {"particles": s.n, "dt": f["dt"], "paper_fp32_drift_per_tau": f["paper_fp32"]}
        for pname, prec in precs:
            r = {"sigma_E_per_N_10tau": {}}
            for dt in f["sweep"]:
                with dem.DEM(s0, prec) as d:
                    dem.dem_autotune(d.ctx)
                    e = [d.energy()[2][0]]
                    for _ in range(int(round(10.0 / dt))):
                        d.step(1, dt, dem.DEM_NVE)
                        e.append(d.energy()[2][0])
                r["sigma_E_per_N_10tau"][str(dt)] = float(np.std(np.array(e) / s.n))
            dt, every = f["dt"], 100
            with dem.DEM(s0, prec) as d:
                dem.dem_autotune(d.ctx)
                t, e = [], []
                t0 = time.perf_counter()
                done = 0
                while True:
                    t.append(done * dt)
                    e.append(d.energy()[2][0] / s.n)
                    if done >= a.drift_steps:
                        break
                    d.step(every, dt, dem.DEM_NVE)
                    done += every
                wall = time.perf_counter() - t0
            t, e = np.array(t), np.array(e)
            slope = float(np.polyfit(t, e, 1)[0])
            r.update(drift_per_tau=slope, drift_per_1e5_steps=slope * 1e5 * dt,
                     E_per_N_start=float(e[0]), E_per_N_end=float(e[-1]), steps=done,
                     wall_s=round(wall, 2))
            res[pname] = r
            print(f"[drift] {name} {pname}: {json.dumps(r)}", file=sys.stderr, flush=True)
        out[name] = res
    workloads = {} if a.drift_set == "fluids" else workload_drifts(a, dem, precs)
    print(json.dumps({"metric": "energy drift of the conserved quantity per particle "
                                "(epsilon per tau) and sigma(E/N) over 10 tau",
                      "unit": "epsilon/tau", "data": "synthetic", "fluids": out,
                      "workloads": workloads}))


# workload, steps stated for it (its ensemble and dt come from make_workload)
DRIFT_WORKLOADS = (("squares", 1000), ("cubes", 10000), ("octahedra", 100000),
                   ("batched", 10000), ("large", 1000))


def workload_drifts(a, dem, precs):
    """The bench workloads in their own ensemble and dt (NVE: K + U; NVT: the
    Nose-Hoover conserved quantity), from one prepared state per workload, in
    each precision: the least-squares slope of H/N over the workload's stated
    steps (fewer when --drift-budget runs out first; the steps run are
    reported), about 100 samples, and that slope per 10^5 steps."""
    out = {}
    for name, steps in DRIFT_WORKLOADS:
        system, run = make_workload(name, 0, a.replicas)
        ens = dem.DEM_NVT if run["ensemble"] == "nvt" else dem.DEM_NVE
        d = prepare(dem, system, run, dem.DEM_FP32_COMP, a.compress_steps, a.equil_steps)
        try:
            s0 = _with_state(system, d.state())
        finally:
            d.close()
        dt, n = run["dt"], s0.n
        res = {"particles": n, "replicas": len(s0.replica_sizes), "ensemble": run["ensemble"],
               "dt": dt, "steps_stated": steps}
        every = max(1, steps // 100)
        for pname, prec in precs:
            with dem.DEM(s0, prec) as d:
                dem.dem_autotune(d.ctx)
                t, e = [], []
                t0 = time.perf_counter()
                done = 0
                while True:
                    t.append(done * dt)
                    e.append(float(np.sum(d.energy()[2])) / n)
                    if done >= steps or time.perf_counter() - t0 > a.drift_budget:
                        break
                    d.step(every, dt, ens, kT=run["kT"], tau_T=run["tau"])
                    done += every
                wall = time.perf_counter() - t0
            slope = float(np.polyfit(np.array(t), np.array(e), 1)[0])
            r = dict(drift_per_tau=slope, drift_per_1e5_steps=slope * 1e5 * dt,
                     H_per_N_start=e[0], H_per_N_end=e[-1], steps=done, wall_s=round(wall, 2))
            res[pname] = r
            print(f"[drift] {name} {pname}: {json.dumps(r)}", file=sys.stderr, flush=True)
        out[name] = res
    return out


def reference_sample(system, run, budget):
    """The workload's first replica at its target density, halved (same shapes,
    same density) until one oracle step of it, measured after the lattice
    start has relaxed for a few steps, fits ``budget`` seconds."""
    import oracle
    from paper_1607_02427_gb300 import workloads as W

    def relaxed_cost(smp):
        st, _ = oracle.run(smp, 2, run["dt"], ensemble=run["ensemble"], kT=run["kT"],
                           tau=run["tau"])
        smp = dataclasses.replace(smp, pos=st["pos"], orient=st["orient"], vel=st["vel"],
                                  angmom=st["angmom"])
        t0 = time.perf_counter()
        oracle.run(smp, 3, run["dt"], ensemble=run["ensemble"], kT=run["kT"], tau=run["tau"])
        return smp, (time.perf_counter() - t0) / 3

    rep = system.replica(0)
    n = min(rep.n, 4096)
    smp = rep if rep.n == n else W.sample_like(system, n)
    smp = W.slab_lattice_start(smp) if smp.dim == 3 else smp
    smp, cost = relaxed_cost(smp)
    what = "the first replica" if smp.n == rep.n else f"a sample like the first replica"
    while cost > budget and smp.n > 16:
        smp = W.sample_like(system, max(8, smp.n // 2))
        smp = W.slab_lattice_start(smp) if smp.dim == 3 else smp
        smp, cost = relaxed_cost(smp)
        what = "a sample like the first replica"
    return smp, what, cost


def reference_arm(a, world, rank):
    """The FP64 CPU oracle on a bounded sample of the workload, per step."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    system, run = make_workload(a.workload, 0, a.replicas, getattr(a, "n", 0))
    # each step a bounded sample: the whole run within about two minutes
    budget = 120.0 / max(1, a.steps + a.warmup)
    sample, nrep, per_step = reference_sample(system, run, budget)
    th = None
    for _ in range(a.warmup):
        st, _ = oracle.run(sample, 1, run["dt"], ensemble=run["ensemble"], kT=run["kT"],
                           tau=run["tau"], thermo=th)
        sample = dataclasses.replace(sample, pos=st["pos"], orient=st["orient"], vel=st["vel"],
                                     angmom=st["angmom"])
        th = st["thermo"]
    t0 = time.perf_counter()
    steps = a.steps
    oracle.run(sample, steps, run["dt"], ensemble=run["ensemble"], kT=run["kT"], tau=run["tau"],
               thermo=th)
    dt = time.perf_counter() - t0
    value = sample.n * steps / dt
    desc = (f"{nrep} ({sample.n} particles) of {system.name}, FP64 oracle, "
            f"single thread, {steps} steps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": steps, "warmup": a.warmup,
            "ms_per_step": dt * 1e3 / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": system.name, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""MD steps/s and pair-evaluations/s of the vertex- and edge-based force paths, mixed precision and
plain FP64, on one GB300 (one process per GPU; N > 1 runs independent replicas).

Default workload: Lennard-Jones fluid, N = 1,048,576, rho = 0.85, T = 1.0, rc = 2.5, skin 0.3,
dt = 0.001, FCC start with +-0.05 sigma jitter (synthetic, seeded).  One step is one velocity-Verlet
step of the whole path: kick + drift + skin check, cell + Verlet rebuild when due, forces, kick and
FP64 energy reductions.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

METRIC = "MD steps/s & pair-evals/s: vertex vs edge, mixed vs FP64 plain, on 1 GB300"
WORKLOAD = "lj_fluid_n1048576_rho0.85_T1.0_rc2.5_skin0.3_dt0.001"


def replica_max(dist, x: float, device=None) -> float:
    """Max of x over the ranks (the job's time is its slowest rank's); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, max_ms: float) -> float:
    """Whole-job rate: the units every rank processed over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (max_ms * 1e-3)


def make_system_seed(rank: int = 0) -> int:
    """Seed of rank r's replica of the workload (each rank runs an independent system)."""
    return 1001 + rank


def make_system(rank: int = 0):
    from paper_1401_4350_gb300 import systems
    return systems.make_lj(1_048_576, 0.85, 1.0, seed=make_system_seed(rank))


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        self.file = None
        self.uuid = device_uuid

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
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
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file.read().splitlines() if l.strip()]
        try:
            os.unlink(self.file.name)
        except OSError:
            pass
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------

# Compulsory DRAM bytes per particle of one fused step launch (isotropic mixed vertex path): list count
# 4, own fixed-point coordinates 16, velocity read + write 64, position read + write (other buffer) 64,
# fixed-point coordinates at the last build 16, new fixed-point coordinates 16; plus 4 B per entry of the
# list it walks (the inner list between prunes).
FUSED_BYTES_PER_PARTICLE = 180
# Inner-list margin of the headline: pairs closer than rc + PRUNE_SKIN, pruned when a particle has moved
# PRUNE_SKIN / 2 (measured at LJ 1M: 0.1 is the fastest of 0.05 ... 0.16)
PRUNE_SKIN = 0.1
# The headline runs in the liquid: fused steps from the initial lattice before anything is timed
# (at LJ 1M about 0.25 s), whatever --warmup asks for beyond them.
EQUILIBRATE_STEPS = 1000
# Steady-state figure: the median of STEADY_REPEATS runs of STEADY_STEPS graph steps each, rebuilds and
# prunes included (a rebuild comes about every 36 steps at LJ 1M, a prune about every 12).
STEADY_REPEATS = 5
STEADY_STEPS = 300
# FP64 operations (DADD, DMUL, DFMA) of one LJ pair evaluation: 32, measured by ncu on the vertex kernel
# (sum of the three thread-instruction counters over the list entries of the launch, LJ N = 262,144;
# profiles/fp64_kernels_lj262k_patchy262k.md).  The vertex kernel evaluates every full-list entry (each pair twice),
# the edge kernel each pair once (its segmented FP64 sums, about 27 more operations per pair, are not pair
# arithmetic and are not counted).
FP64_OPS_PER_PAIR_EVAL_LJ = 32
# The same count for the patchy model (WCA core, nine patch pairs with an FP64 exponential each within reach):
# 120 per pair evaluation, measured the same way at patchy N = 262,144.  Its FP64 kernels keep the FP64 pipe
# about 84 % busy; the exponential's other FP64-pipe instructions, compares and conversions are not counted.
FP64_OPS_PER_PAIR_EVAL_PATCHY = 120
# The FP64 pipe of GB300: 2 DFMA per clock per SM (ncu's peak_sustained of the DFMA counter, 304 per cycle
# over 152 SMs); 1.67 was reached by a dependent-free DFMA microbenchmark.
FP64_PER_CLK_SM = 2.0
N_SM = 152


def algorithmic_bytes_force(path: int, precision: int, n: int, full_entries: int, pairs: int,
                            patchy: bool = False) -> float:
    """Compulsory DRAM bytes of one force launch (lists, per-particle arrays once, outputs once)."""
    from paper_1401_4350_gb300 import binding as B
    if patchy and precision == B.MD_MIXED:
        # + the three fixed-point patch sites (48 B) and the torque output (vertex: 32 B written; edge: the
        # FP32 torque sum and its compensation, zeroed once and accumulated once)
        if path == B.MD_VERTEX:
            return 4.0 * full_entries + n * (4 + 16 + 48 + 40 + 32)
        return 4.0 * pairs + 8.0 * (n + 1) + n * (16 + 48 + 2 * 32 + 2 * 32)
    if path == B.MD_VERTEX:
        # count 4 + own coordinates (fixed point 16, FP64 32) + force double4 32 + virial 8
        return 4.0 * full_entries + n * (4 + (16 if precision == B.MD_MIXED else 32) + 40)
    pos_b, out_b = (16, 32) if precision == B.MD_MIXED else (32, 64)
    # half list in CSR form: 4 B per partner + the row starts; outputs zeroed once, accumulated once
    return 4.0 * pairs + 8.0 * (n + 1) + n * (pos_b + 2 * out_b)


def algorithmic_bytes_fused(n: int, entries: int, inner: bool = False) -> float:
    """Compulsory DRAM bytes of one fused force + integrate launch over a list of `entries` entries; a launch
    over the inner list also reads each particle's coordinates at the last prune (16 B)."""
    return 4.0 * entries + (FUSED_BYTES_PER_PARTICLE + (16 if inner else 0)) * n


def fp64_peak_gops(sm_mhz: float) -> float:
    """FP64-pipe operations per second of the whole GPU at the given SM clock (G op/s)."""
    return FP64_PER_CLK_SM * N_SM * sm_mhz * 1e-3


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch
    from paper_1401_4350_gb300 import binding as B
    from paper_1401_4350_gb300 import build as mdbuild
    from paper_1401_4350_gb300.sim import Simulation

    if rank == 0:
        mdbuild.build()
    if dist is not None:
        dist.barrier()
    B.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    system = make_system(rank)
    n = system.n
    stream = torch.cuda.current_stream()
    ctx = Ctx(stream, dist, dev)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if uuid and not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None

    # ---- headline: mixed precision, vertex path (the faster path on this workload), one fused
    # force + integrate kernel per step over an inner list pruned to rc + PRUNE_SKIN, timed in the
    # liquid that EQUILIBRATE_STEPS fused steps make of the initial lattice ----
    headline_path = B.MD_VERTEX
    sim = Simulation(system, B.MD_MIXED, trace_capacity=0, stream=stream, fuse_step=1, prune_skin=PRUNE_SKIN)
    sim.prepare(headline_path)
    sampler = ClockSampler(uuid) if rank == 0 else None
    if sampler:
        sampler.start()
    sim.step(max(args.warmup, EQUILIBRATE_STEPS), headline_path, use_graph=True)
    p0 = sim.status()[B.MD_STATUS_PRUNES]
    ms, rebuilds = ctx.time_steps(sim, headline_path, args.steps, use_graph=not args.direct)
    prunes = int(sim.status()[B.MD_STATUS_PRUNES] - p0)
    ms = ctx.max_over_ranks(ms)
    steady = []
    for _ in range(STEADY_REPEATS):
        sms, sreb = ctx.time_steps(sim, headline_path, STEADY_STEPS)
        steady.append((ctx.max_over_ranks(sms) / STEADY_STEPS, sreb))
    clocks = sampler.stop() if sampler else None
    sm_mhz = clocks["sm_mhz"] if clocks else 2070.0
    full_entries, pairs = list_stats(sim, n)
    inner_entries = int(sim.view("nbr_in_count", torch.int32, n).sum().item())
    kernel_ms = sim.time_step_kernel(headline_path, reps=100)
    force_ms = ctx.force_launch_ms(sim, headline_path, 50)
    step_ms = ms / args.steps
    steady_ms = statistics.median(x[0] for x in steady)
    headline = {"steps_per_s": 1e3 / step_ms, "ms_per_step": step_ms, "rebuilds": rebuilds, "prunes": prunes,
                "pair_evals_per_s": pairs * 1e3 / step_ms, "step_kernel_ms": kernel_ms, "force_kernel_ms": force_ms,
                "fuse_step": 1, "prune_skin": PRUNE_SKIN, "mean_inner_list": inner_entries / n}
    # ---- end to end through the C ABI with host-resident state: md_step_verlet_host, one step per call,
    # positions and velocities ([n][3] FP64 each, pinned) copied in and out by the call, energies out ----
    pos_h, vel_h = sim.slot_state_host(pin=True)
    en_h = torch.empty(B.MD_ENERGY_WORDS, dtype=torch.float64, pin_memory=True)
    e2e_calls = max(100, min(args.steps, 300))
    sim.step_host(pos_h, vel_h, 1, headline_path, use_graph=True, host_energy=en_h)  # graphs built
    ctx.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_calls):
        sim.step_host(pos_h, vel_h, 1, headline_path, use_graph=True, host_energy=en_h)
    torch.cuda.synchronize()
    e2e_s = ctx.max_over_ranks(time.perf_counter() - t0)
    assert np.isfinite(en_h.numpy()[:4]).all() and sim.status()[B.MD_STATUS_CODE] == 0
    e2e = {"value": world * e2e_calls / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": 2 * n * 24,
           "d2h_bytes_per_step": 2 * n * 24 + 8 * B.MD_ENERGY_WORDS, "calls": e2e_calls,
           "api": "md_step_verlet_host, 1 step per call"}
    liquid = sim.positions()  # the equilibrated state, in the original order
    del sim
    torch.cuda.empty_cache()

    hbm, peak_source = hbm_peak()
    alg = algorithmic_bytes_fused(n, inner_entries, inner=True)
    achieved = alg / (kernel_ms * 1e-3) / 1e9
    force_alg = algorithmic_bytes_force(headline_path, B.MD_MIXED, n, full_entries, pairs)
    # the survey's count of compulsory bytes for the vertex step: 4 B per full-list entry + 192 B per particle
    survey_alg = 4.0 * full_entries + 192.0 * n
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": measured_traffic("k_vertex_step_mixed<1,true>", n, inner_entries),
                "kernel": "k_vertex_step_mixed<1,true>", "state": f"liquid, after {EQUILIBRATE_STEPS} steps",
                "algorithmic_bytes_per_launch": alg, "kernel_ms": kernel_ms,
                "kernel_share_of_step": kernel_ms / steady_ms,
                "frac_survey_bytes": survey_alg / (kernel_ms * 1e-3) / 1e9 / hbm,
                "survey_bytes_per_launch": survey_alg,
                "force_only": {"kernel": "k_vertex_iso_mixed<1,true>", "algorithmic_bytes_per_launch": force_alg,
                               "ms": force_ms, "achieved": force_alg / (force_ms * 1e-3) / 1e9,
                               "frac": force_alg / (force_ms * 1e-3) / 1e9 / hbm},
                "peak_source": peak_source}
    value = job_throughput(world, args.steps, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "precision": "mixed: FP32 pair arithmetic + compensated FP32 sums, FP64 integration and reductions",
        "pair_evals_per_s": world * pairs * args.steps / (ms * 1e-3),
        "steady": {"ms_per_step": steady_ms, "steps_per_s": world * 1e3 / steady_ms,
                   "mean_ms_per_step": statistics.mean(x[0] for x in steady), "repeats": STEADY_REPEATS,
                   "steps_per_repeat": STEADY_STEPS, "ms_per_step_each": [x[0] for x in steady],
                   "rebuilds_each": [x[1] for x in steady],
                   "note": "median (and mean) of the repeats; each repeat spans several rebuild and prune "
                           "periods"},
        "config": {"workload": WORKLOAD, "n": n, "path": "vertex", "precision": "mixed",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (inner list ~0.26 GB + state ~0.2 GB per step)",
                   "equilibrated_steps": max(args.warmup, EQUILIBRATE_STEPS),
                   "mean_full_list": full_entries / n, "mean_inner_list": inner_entries / n,
                   "prune_skin": PRUNE_SKIN, "unique_pairs": pairs},
        "roofline": roofline,
        "e2e": e2e,
        # one call of K fused steps: the opening integrate (its last block decides), K - 1 fused step
        # kernels each followed by a one-warp decision kernel, then the fused closing launch (the last
        # forces and the closing half kick) and its decision kernel; a rebuild adds 9 cell and 2 Verlet
        # kernels
        "gpu_launches": 2 * args.steps + 1 + 11 * rebuilds,
        "clocks": clocks,
        "graph": not args.direct,
    }
    if not args.no_variants and world == 1:
        line["variants"], line["accuracy"] = run_variants(ctx, system, liquid, headline, roofline, sm_mhz, args)
    if not args.no_batch and world == 1:
        line["batch"] = run_batch()
    if not args.no_sweep and world == 1:
        line["density_sweep"] = run_density_sweep()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(system)
    return line


class Ctx:
    """Timing helpers on one stream, with the barrier and max over ranks of the weak-scaling run."""

    def __init__(self, stream, dist, dev):
        self.stream, self.dist, self.dev = stream, dist, dev

    def barrier(self):
        import torch
        torch.cuda.synchronize()
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x):
        return replica_max(self.dist, x, self.dev)

    def time_steps(self, sim, path, k, use_graph=True):
        """ms of k md_step_verlet steps (CUDA events on the launching stream) and the rebuilds among them."""
        import torch
        from paper_1401_4350_gb300 import binding as B
        st0 = sim.status()
        self.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        sim.step(k, path, use_graph=use_graph)
        e1.record(self.stream)
        torch.cuda.synchronize()
        self.barrier()
        st1 = sim.status()
        assert st1[B.MD_STATUS_CODE] == 0, f"device status {st1}"
        return e0.elapsed_time(e1), int(st1[B.MD_STATUS_REBUILDS] - st0[B.MD_STATUS_REBUILDS])

    def force_launch_ms(self, sim, path, k):
        """Mean ms of one force evaluation of `path` (the force entry point's kernels), CUDA events."""
        import torch
        from paper_1401_4350_gb300 import binding as B
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        fn = {B.MD_VERTEX: sim.forces_vertex, B.MD_EDGE: sim.forces_edge,
              B.MD_VERTEX_NEWTON: sim.forces_vertex_newton, B.MD_EDGE_STORE: sim.forces_edge_store}[path]
        fn()
        torch.cuda.synchronize()
        for a, b in evs:
            a.record(self.stream)
            fn()
            b.record(self.stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in evs)


def list_stats(sim, n, path=None):
    """(full-list entries, unique pairs) of the lists the system holds."""
    import torch
    from paper_1401_4350_gb300 import binding as B
    cnt = sim.view("nbr_count", torch.int32, n)
    entries = int(cnt.sum().item())
    if path == B.MD_VERTEX_NEWTON:  # the Newton list holds every pair once
        return 2 * entries, entries
    if path in (B.MD_EDGE, B.MD_EDGE_STORE):  # only the half list is built
        pairs = int(sim.view("half_start", torch.int64, n + 1)[-1].item())
        return 2 * pairs, pairs
    return entries, entries // 2


def hbm_peak():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s, an earlier GB300 measurement)"


# The configurations of the scaling and regime study: name -> (factory, kind)
def config_systems():
    from paper_1401_4350_gb300 import systems
    return {
        "lj65536": lambda: systems.make_lj(65_536, 0.85, 1.0, seed=1001),
        "lj262144": lambda: systems.make_lj(262_144, 0.85, 1.0, seed=1001),
        "wca1m": lambda: systems.make_wca(1_048_576, 0.2, seed=1002),
        "patchy262k": lambda: systems.make_patchy(262_144, 0.3, seed=1003),
    }


def with_state(s, pos, vel, quat=None, angmom=None):
    """The system s with another state (positions wrapped into the box)."""
    import dataclasses
    import numpy as np
    box = np.asarray(s.box, dtype=np.float64)
    pos = np.mod(np.asarray(pos, dtype=np.float64), box)
    pos[pos >= box] -= np.broadcast_to(box, pos.shape)[pos >= box]
    return dataclasses.replace(s, pos=pos, vel=vel, quat=quat if quat is not None else s.quat,
                               angmom=angmom if angmom is not None else s.angmom)


def equilibrate(s, steps):
    """The system after `steps` steps of its fastest mixed path (the liquid the variants are timed in)."""
    import torch
    from paper_1401_4350_gb300 import binding as B
    from paper_1401_4350_gb300.sim import Simulation
    from paper_1401_4350_gb300.systems import PATCHY_KINDS
    patchy = s.kind in PATCHY_KINDS
    path = B.MD_EDGE if patchy else B.MD_VERTEX
    sim = Simulation(s, B.MD_MIXED, fuse_step=0 if patchy else 1)
    sim.prepare(path)
    sim.step(steps, path, use_graph=True)
    assert sim.status()[B.MD_STATUS_CODE] == 0
    x, v = sim.positions()
    q, l = sim.orientations() if patchy else (None, None)
    del sim
    torch.cuda.empty_cache()
    return with_state(s, x, v, q, l)


def drift(s, precision, path, steps, opts):
    """Energy drift of `steps` graph steps from the state s: least-squares slope of E_tot / N per 10^4 steps,
    and the rms fluctuation of E_tot / N."""
    import numpy as np
    import torch
    from paper_1401_4350_gb300 import binding as B
    from paper_1401_4350_gb300.sim import Simulation
    sim = Simulation(s, precision, trace_capacity=steps + 1, **opts)
    sim.prepare(path)
    sim.step(steps, path, use_graph=True)
    assert sim.status()[B.MD_STATUS_CODE] == 0
    tr = sim.trace()
    rows = tr[(tr[:, 0] > 0) & (tr[:, 0] <= steps)]
    rows = rows[np.argsort(rows[:, 0])]
    e = (rows[:, 1] + rows[:, 2]) / s.n
    del sim
    torch.cuda.empty_cache()
    return {"per_1e4_steps": float(np.polyfit(rows[:, 0], e, 1)[0]) * 1e4, "rms_fluctuation": float(np.std(e)),
            "steps": steps}


def run_variants(ctx, system1m, liquid1m, headline, headline_roofline, sm_mhz, args):
    """Every (configuration, path, precision) on one GPU, each timed in the liquid of its configuration
    (EQUILIBRATE_STEPS steps of its fastest mixed path): steps/s of md_step_verlet (graph), pair-evals/s, the
    dominant kernel's time and its roofline fraction; then the accuracy of each mixed result against the
    FP64 path on the same state (max force and torque error over the rms over all particles) and the
    energy drift of both precisions."""
    import numpy as np
    import torch
    from paper_1401_4350_gb300 import binding as B
    from paper_1401_4350_gb300.sim import Simulation
    from paper_1401_4350_gb300.systems import PATCHY_KINDS

    hbm, _ = hbm_peak()
    fp64_peak = fp64_peak_gops(sm_mhz)
    systems_eq = {"lj1m": with_state(system1m, *liquid1m)}
    for name, make in config_systems().items():
        systems_eq[name] = equilibrate(make(), EQUILIBRATE_STEPS)
    out = {}

    def run(key, s, path, precision, k, opts, what="force"):
        n = s.n
        sim = Simulation(s, precision, stream=ctx.stream, **opts)
        sim.prepare(path)
        sim.step(3, path, use_graph=True)
        ms, reb = ctx.time_steps(sim, path, k)
        entries, pairs = list_stats(sim, n, path)
        fused = opts.get("fuse_step", 1) == 1 and path == B.MD_VERTEX and precision == B.MD_MIXED and \
            s.kind not in PATCHY_KINDS
        patchy = s.kind in PATCHY_KINDS
        r = {"steps_per_s": 1e3 * k / ms, "ms_per_step": ms / k, "rebuilds": reb, "steps": k,
             "pair_evals_per_s": pairs * 1e3 * k / ms, "n": n, "mean_full_list": entries / n,
             "path": {B.MD_VERTEX: "vertex", B.MD_EDGE: "edge", B.MD_VERTEX_NEWTON: "vertex_newton",
                      B.MD_EDGE_STORE: "edge_store"}[path],
             "precision": "mixed" if precision == B.MD_MIXED else "fp64",
             "l2": "inputs larger than L2" if n >= 262_144 else "inputs fit in L2 (129 MB)", **opts}
        if fused:
            inner = opts.get("prune_skin", 0.0) > 0
            walked = int(sim.view("nbr_in_count", torch.int32, n).sum().item()) if inner else entries
            kms = sim.time_step_kernel(path, reps=50)
            alg = algorithmic_bytes_fused(n, walked, inner)
            r["roofline"] = {"bound": "hbm", "kernel": "k_vertex_step_mixed", "kernel_ms": kms,
                             "algorithmic_bytes_per_launch": alg, "achieved": alg / (kms * 1e-3) / 1e9,
                             "peak": hbm, "unit": "GB/s", "frac": alg / (kms * 1e-3) / 1e9 / hbm}
        else:
            fms = ctx.force_launch_ms(sim, path, 5 if precision == B.MD_FP64 else 20)
            kname = {(B.MD_VERTEX, B.MD_MIXED): "k_vertex_iso_mixed" if not patchy else "k_vertex_mixed",
                     (B.MD_EDGE, B.MD_MIXED): "k_edge_mixed", (B.MD_VERTEX, B.MD_FP64): "k_vertex_fp64",
                     (B.MD_EDGE, B.MD_FP64): "k_edge_fp64", (B.MD_VERTEX_NEWTON, B.MD_MIXED): "k_vertex_newton_mixed",
                     (B.MD_VERTEX_NEWTON, B.MD_FP64): "k_vertex_newton_fp64",
                     (B.MD_EDGE_STORE, B.MD_MIXED): "k_edge_store"}.get((path, precision), "force kernels")
            if precision == B.MD_FP64 and path in (B.MD_VERTEX, B.MD_EDGE):
                evals = entries if path == B.MD_VERTEX else pairs
                per_eval = FP64_OPS_PER_PAIR_EVAL_PATCHY if patchy else FP64_OPS_PER_PAIR_EVAL_LJ
                ops = per_eval * evals
                r["roofline"] = {"bound": "alu", "kernel": kname, "kernel_ms": fms, "unit": "G FP64 op/s",
                                 "fp64_ops_per_launch": ops, "achieved": ops / (fms * 1e-3) / 1e9,
                                 "peak": fp64_peak, "frac": ops / (fms * 1e-3) / 1e9 / fp64_peak,
                                 "ops_per_pair_eval": per_eval,
                                 "peak_source": f"{FP64_PER_CLK_SM} FP64 op/clk/SM (ncu peak_sustained) x {N_SM} "
                                                f"SMs x {sm_mhz:.0f} MHz (median SM clock of the headline run)"}
                if patchy:
                    r["roofline"]["note"] = ("the FP64 pipe is about 84 % busy (ncu); the exponential's other FP64-pipe "
                                             "instructions, compares and conversions are not in the counted operations")
            else:
                alg = algorithmic_bytes_force(path if path in (B.MD_VERTEX, B.MD_EDGE) else B.MD_EDGE, precision,
                                              n, entries, pairs, patchy=patchy)
                r["roofline"] = {"bound": "hbm", "kernel": kname, "kernel_ms": fms,
                                 "algorithmic_bytes_per_launch": alg, "achieved": alg / (fms * 1e-3) / 1e9,
                                 "peak": hbm, "unit": "GB/s", "frac": alg / (fms * 1e-3) / 1e9 / hbm}
                if patchy and precision == B.MD_MIXED:
                    r["roofline"]["note"] = ("latency-bound, not bandwidth-bound: ncu shows 19-28 % occupancy, issue "
                                             "29-33 % and no pipe above 32 % (profiles/k_patchy_mixed_262k.md)")
        del sim
        torch.cuda.empty_cache()
        out[key] = r
        return r

    MIX, F64, VX, ED = B.MD_MIXED, B.MD_FP64, B.MD_VERTEX, B.MD_EDGE
    ksteps = lambda prec, n: (max(20, min(200, int(2e8 / n))) if prec == MIX else max(5, min(40, int(2e7 / n))))
    for name in ("lj65536", "lj262144", "lj1m", "wca1m", "patchy262k"):
        s = systems_eq[name]
        patchy = s.kind in PATCHY_KINDS
        for path, prec in ((VX, MIX), (ED, MIX), (VX, F64), (ED, F64)):
            key = f"{name}_{'vertex' if path == VX else 'edge'}_{'mixed' if prec == MIX else 'fp64'}"
            if name == "lj1m" and path == VX and prec == MIX:
                out[key] = dict(headline, roofline={k: headline_roofline[k] for k in
                                                    ("bound", "kernel", "kernel_ms", "algorithmic_bytes_per_launch",
                                                     "achieved", "peak", "unit", "frac")},
                                n=s.n, path="vertex", precision="mixed", note="the headline run")
                continue
            opts = {"fuse_step": 0}  # separate force and integrate kernels
            if path == VX and prec == MIX and not patchy:
                # the fused step; LJ over the inner list as in the headline
                opts = {"fuse_step": 1, "prune_skin": PRUNE_SKIN if s.kind == 0 else 0.0}
            run(key, s, path, prec, ksteps(prec, s.n), opts)
    # other decompositions on the 1M LJ liquid
    s = systems_eq["lj1m"]
    NW, ES = B.MD_VERTEX_NEWTON, B.MD_EDGE_STORE
    for key, path, prec, k, opts in (
            ("lj1m_vertex_mixed_fused_full_list", VX, MIX, 200, {"fuse_step": 1}),
            ("lj1m_vertex_mixed_separate_kernels", VX, MIX, 200, {"fuse_step": 0}),
            ("lj1m_vertex_mixed_hilbert", VX, MIX, 200, {"fuse_step": 1, "prune_skin": PRUNE_SKIN,
                                                          "cell_order": B.MD_ORDER_HILBERT}),
            ("lj1m_edge_store_mixed", ES, MIX, 50, {"edge_store": 1, "fuse_step": 0}),
            ("lj1m_vertex_newton_mixed_m1", NW, MIX, 50, {"force_copies": 1, "fuse_step": 0}),
            ("lj1m_vertex_newton_mixed_m16", NW, MIX, 50, {"force_copies": 16, "fuse_step": 0}),
            ("lj1m_vertex_newton_fp64_m16", NW, F64, 10, {"force_copies": 16, "fuse_step": 0})):
        run(key, s, path, prec, k, opts)

    # ---- accuracy: mixed against FP64 on each liquid state; drift of both precisions ----
    acc = {}
    for name in ("lj65536", "lj262144", "lj1m", "wca1m", "patchy262k"):
        s = systems_eq[name]
        patchy = s.kind in PATCHY_KINDS
        res = {}
        ref = Simulation(s, F64, fuse_step=0)
        ref.prepare(VX)
        Fr, _, Tr, _ = ref.forces()
        del ref
        torch.cuda.empty_cache()
        frms = float(np.sqrt((Fr ** 2).sum(1).mean()))
        trms = float(np.sqrt((Tr ** 2).sum(1).mean())) if patchy else None
        for pname, path in (("vertex", VX), ("edge", ED)):
            sim = Simulation(s, MIX, fuse_step=0)
            sim.prepare(path)
            F, _, T, _ = sim.forces()
            del sim
            torch.cuda.empty_cache()
            res[f"{pname}_max_force_error_frms"] = float(np.abs(F - Fr).max()) / frms
            if patchy:
                res[f"{pname}_max_torque_error_trms"] = float(np.abs(T - Tr).max()) / trms
        if patchy:
            res["torque_rms_over"] = "all particles"
        dsteps = 1000
        mixed_opts = {"fuse_step": 0} if patchy else {"fuse_step": 1, "prune_skin": PRUNE_SKIN if s.kind == 0 else 0.0}
        res["drift_mixed"] = drift(s, MIX, ED if patchy else VX, dsteps, mixed_opts)
        res["drift_fp64"] = drift(s, F64, VX, dsteps, {"fuse_step": 0})
        res["drift_mixed"]["path"] = "edge" if patchy else "vertex"
        acc[name] = res
    acc["definitions"] = ("force error: max over particles and components of |F_mixed - F_fp64| / F_rms (torque: "
                          "the same over tau_rms of all particles), both on the liquid state of the row; drift: "
                          "least-squares slope of E_tot / N over 1000 graph steps from that state, per 10^4 steps")
    return out, acc


def kernel_source_digest() -> str:
    """sha256 of the step-kernel sources, to tell whether a stored ncu capture still describes them."""
    import hashlib
    h = hashlib.sha256()
    for f in ("md_forces.cuh", "md_forces.cu", "md_internal.cuh", "md_integrate.cuh", "md_step.cu"):
        with open(os.path.join(ROOT, "paper_1401_4350_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel: str, n: int, entries: int):
    """DRAM bytes per launch of `kernel` from the committed ncu capture (profiles/dram_traffic.json), scaled
    to this launch by list entries + particles, or None when the capture is of other kernel sources."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_sha256") != kernel_source_digest():
        return None
    # traffic ~ 4 B per entry + per-particle bytes: scale the captured launch by its algorithmic bytes
    per = float(rec.get("bytes_per_particle", FUSED_BYTES_PER_PARTICLE))
    alg_now = 4.0 * entries + per * n
    alg_cap = 4.0 * rec["list_entries"] + per * rec["n"]
    return rec["dram_bytes_per_launch"] * alg_now / alg_cap


def run_density_sweep(n: int = 131072, steps: int = 200):
    """The paper's state points (Sec. Models): LJ at kT = 1.8 and its patchy form at kT = 0.15, each at
    rho = 0.1, 0.3 and 0.5 with the Brownian momentum refresh, vertex vs edge, mixed precision; steps/s
    of md_step_verlet (graph) on one GPU."""
    import torch
    from paper_1401_4350_gb300 import binding as B
    from paper_1401_4350_gb300 import systems
    from paper_1401_4350_gb300.sim import Simulation
    out = {"n": n, "steps": steps, "precision": "mixed", "thermostat": "refresh p = 0.1 every 100 steps",
           "points": []}
    stream = torch.cuda.current_stream()
    for model, kT in (("lj", 1.8), ("patchy_pow", 0.15)):
        for rho in (0.1, 0.3, 0.5):
            s = (systems.make_lj_nvt(n, rho, temperature=kT, seed=1100) if model == "lj"
                 else systems.make_patchy_pow(n, rho, temperature=kT, seed=1101))
            row = {"model": model, "rho": rho, "kT": kT}
            for name, path in (("vertex", B.MD_VERTEX), ("edge", B.MD_EDGE)):
                sim = Simulation(s, B.MD_MIXED, stream=stream)
                sim.prepare(path)
                sim.step(5, path, use_graph=True)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(steps, path, use_graph=True)
                e1.record(stream)
                torch.cuda.synchronize()
                st = sim.status()
                assert st[B.MD_STATUS_CODE] == 0, st
                ms = e0.elapsed_time(e1)
                row[name + "_steps_per_s"] = 1e3 * steps / ms
                del sim
                torch.cuda.empty_cache()
            row["edge_over_vertex"] = row["edge_steps_per_s"] / row["vertex_steps_per_s"]
            out["points"].append(row)
    return out


def run_batch(steps: int = 50, fp64_steps: int = 5, drift_steps: int = 1000):
    """512 replicas (N log-uniform in [500, 32768], rho ~ U(0.2, 0.9), every fourth WCA at rho 0.2, the
    rest LJ rc 2.5): mixed-precision batched path, autotuned, against looping the plain FP64
    single-system path over the same replicas.  Also the batch's max force error against FP64."""
    import numpy as np
    import torch
    from paper_1401_4350_gb300 import binding as B
    from paper_1401_4350_gb300 import systems
    from paper_1401_4350_gb300.sim import BatchSimulation, Simulation

    reps = [systems.make_replica(*spec) for spec in systems.batch_specs(512)]
    n_total = sum(s.n for s in reps)
    bs = BatchSimulation(reps, trace_capacity=drift_steps + 1)
    t0 = time.perf_counter()
    paths, tpps = bs.autotune()
    tune_s = time.perf_counter() - t0
    # accuracy at the prepared state: mixed batch forces vs FP64 single-system forces, every replica
    worst = 0.0
    for r, s in enumerate(reps):
        F, _, _ = bs.replica_forces(r)
        ref = Simulation(s, B.MD_FP64)
        ref.prepare(B.MD_VERTEX)
        Fr, _, _, _ = ref.forces()
        del ref
        frms = np.sqrt((Fr ** 2).sum(1).mean())
        worst = max(worst, float(np.abs(F - Fr).max() / frms))
    torch.cuda.empty_cache()
    bs.step(3)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    bs.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1)
    assert all(bs.replica_status(r)[B.MD_STATUS_CODE] == 0 for r in range(len(reps)))
    # energy drift of every replica over the next drift_steps batched steps: slope of E_tot / N per 10^4 steps
    s0 = int(bs.replica_status(0)[B.MD_STATUS_STEPS])
    bs.step(drift_steps)
    slopes = []
    for r, s in enumerate(reps):
        tr = bs.replica_trace(r)
        rows = tr[(tr[:, 0] > s0) & (tr[:, 0] <= s0 + drift_steps)]
        rows = rows[np.argsort(rows[:, 0])]
        slopes.append(float(np.polyfit(rows[:, 0], (rows[:, 1] + rows[:, 2]) / s.n, 1)[0]) * 1e4)
    slopes = np.abs(np.array(slopes))
    # the mixed forces after those steps (liquid states) against FP64 on the same positions, every 8th replica
    worst_liquid = 0.0
    for r in range(0, len(reps), 8):
        s = reps[r]
        F, _, _ = bs.replica_forces(r)
        x, v = bs.replica_positions(r)
        ref = Simulation(with_state(s, x, v), B.MD_FP64)
        ref.prepare(B.MD_VERTEX)
        Fr, _, _, _ = ref.forces()
        del ref
        worst_liquid = max(worst_liquid, float(np.abs(F - Fr).max() / np.sqrt((Fr ** 2).sum(1).mean())))
    bs.release()
    del bs
    torch.cuda.empty_cache()
    # the plain FP64 per-system path, looped over the replicas
    loop_ms = 0.0
    for s in reps:
        sim = Simulation(s, B.MD_FP64)
        sim.prepare(B.MD_VERTEX)
        sim.step(1, B.MD_VERTEX)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        sim.step(fp64_steps, B.MD_VERTEX)
        c.record(st)
        torch.cuda.synchronize()
        loop_ms += a.elapsed_time(c)
        del sim
    torch.cuda.empty_cache()
    batch_rs = len(reps) * steps / (batch_ms * 1e-3)
    loop_rs = len(reps) * fp64_steps / (loop_ms * 1e-3)
    return {"workload": "512 replicas, N log-uniform [500, 32768], rho U(0.2, 0.9), 1/4 WCA rho 0.2, 3/4 LJ rc 2.5",
            "particles": n_total, "steps": steps, "ms_per_step": batch_ms / steps,
            "replica_steps_per_s": batch_rs, "particle_steps_per_s": n_total * steps / (batch_ms * 1e-3),
            "fp64_loop_replica_steps_per_s": loop_rs, "speedup_vs_fp64_loop": batch_rs / loop_rs,
            "max_force_error_vs_fp64_frms": worst,
            "max_force_error_vs_fp64_frms_after_drift_steps": worst_liquid,
            "force_error_sample": "every replica at the prepared state; every 8th after the drift steps",
            "autotune_s": tune_s,
            "energy_drift_per_1e4_steps": {"median_abs": float(np.median(slopes)), "max_abs": float(slopes.max()),
                                           "steps": drift_steps, "over": "every replica, E_tot / N"},
            "chosen": {"edge": int(sum(1 for p in paths if p == B.MD_EDGE)),
                       "vertex_tpp1": int(sum(1 for p, t in zip(paths, tpps) if p == B.MD_VERTEX and t == 1)),
                       "vertex_tpp2": int(sum(1 for p, t in zip(paths, tpps) if p == B.MD_VERTEX and t == 2)),
                       "vertex_tpp4": int(sum(1 for p, t in zip(paths, tpps) if p == B.MD_VERTEX and t == 4))}}


def cpu_baseline(system, max_seconds=25.0):
    """The FP64 oracle as it stands, single-threaded on the host, on a bounded sample of steps."""
    import oracle
    oracle.build()
    m = oracle.Model(oracle.LJ, tuple(system.box), system.rc)
    t0 = time.perf_counter()
    oracle.run_nve(system.pos, system.vel, m, system.dt, 1, use_cells=True)
    t1 = time.perf_counter()
    per = (t1 - t0) / 2.0  # one step = two force evaluations here (initial + after the drift)
    k = max(1, min(8, int(max_seconds / max(per, 1e-3)) - 1))
    t2 = time.perf_counter()
    oracle.run_nve(system.pos, system.vel, m, system.dt, k, use_cells=True)
    el = time.perf_counter() - t2
    return {"value": k / el, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "host_cores_available": len(os.sched_getaffinity(0)),
            "sample": f"{k} velocity-Verlet steps (+1 initial force evaluation) of the same {system.n}-particle "
                      f"system, FP64 cell-list C oracle, one thread"}


def run_reference(args):
    """The oracle timed as it stands, on one host thread: W warm-up steps, then K steps, or as many as fit in
    about 120 s of host time."""
    import oracle
    oracle.build()
    system = make_system(0)
    m = oracle.Model(oracle.LJ, tuple(system.box), system.rc)
    t0 = time.perf_counter()
    pos, vel, _, _, _ = oracle.run_nve(system.pos, system.vel, m, system.dt, args.warmup, use_cells=True)
    per = (time.perf_counter() - t0) / (args.warmup + 1.0)  # the warm-up steps and the initial force evaluation
    k = max(1, min(args.steps, int(120.0 / max(per, 1e-3))))
    t1 = time.perf_counter()
    oracle.run_nve(pos, vel, m, system.dt, k, use_cells=True)
    el = time.perf_counter() - t1
    value = k / el
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": 1, "steps": k,
            "requested_steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / k,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": system.n, "implementation": "FP64 cell-list C oracle"},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{k} steps of the {system.n}-particle workload after {args.warmup} warm-up "
                                       f"steps, one host thread"},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-replica measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the density sweep at the paper's state points")
    ap.add_argument("--direct", action="store_true",
                    help="launch the kernels directly instead of replaying the step graph (for profilers that "
                         "do not replay kernels inside graphs with conditional nodes)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

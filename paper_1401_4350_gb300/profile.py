"""Small driver for profiling one phase of the path under ncu.

  python -m paper_1401_4350_gb300.profile --workload lj524288 --what forces --path vertex --reps 2

Builds the seeded workload, prepares cells, lists and forces once, then launches the chosen phase
`reps` times (forces: md_forces_vertex / md_forces_edge; build: md_build_cells + md_build_verlet;
step: md_step_verlet of one step; steps3: of three steps; steps: of --nsteps steps, all launched directly
(for launch lists: ncu does not profile graphs that hold conditional nodes); stepkernel: md_time_step_kernel, the kernel
one step runs, i.e. the fused force + integrate kernel when fuse_step applies).  Prints the median
CUDA-event time per call.
"""
from __future__ import annotations

import argparse
import statistics

import torch

from . import binding as B
from . import build as mdbuild
from . import systems
from .sim import Simulation

WORKLOADS = {
    "lj1m": lambda: systems.make_lj(1_048_576, 0.85, 1.0, seed=1001),
    "lj524288": lambda: systems.make_lj(524_288, 0.85, 1.0, seed=1001),
    "lj262144": lambda: systems.make_lj(262_144, 0.85, 1.0, seed=1001),
    "wca1m": lambda: systems.make_wca(1_048_576, 0.2, seed=1002),
    "wca524288": lambda: systems.make_wca(524_288, 0.2, seed=1002),
    "patchy262k": lambda: systems.make_patchy(262_144, 0.3, seed=1003),
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lj524288", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--path", default="vertex", choices=["vertex", "edge"])
    ap.add_argument("--what", default="forces", choices=["forces", "build", "step", "steps3", "steps", "stepkernel"])
    ap.add_argument("--nsteps", type=int, default=20, help="steps of one call for --what steps (direct launches)")
    ap.add_argument("--fuse", type=int, default=1, choices=[0, 1], help="fuse_step of the system")
    ap.add_argument("--prune", type=float, default=0.0, help="prune_skin of the system (inner list)")
    ap.add_argument("--tpp", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--order", default="rows", choices=["rows", "hilbert"])
    ap.add_argument("--equilibrate", type=int, default=0, help="MD steps before the timed launches")
    ap.add_argument("--direct", action="store_true",
                    help="equilibrate with direct launches instead of graphs (so that ncu counts them and can skip "
                         "them with -s)")
    a = ap.parse_args(argv)
    mdbuild.build()
    B.load()
    torch.cuda.set_device(0)
    s = WORKLOADS[a.workload]()
    prec = B.MD_MIXED if a.precision == "mixed" else B.MD_FP64
    path = B.MD_VERTEX if a.path == "vertex" else B.MD_EDGE
    sim = Simulation(s, prec, tpp=a.tpp, cell_order=B.MD_ORDER_HILBERT if a.order == "hilbert" else B.MD_ORDER_ROWS,
                     fuse_step=a.fuse, prune_skin=a.prune)
    sim.prepare(path)
    if a.equilibrate > 0:  # time the liquid rather than the initial lattice
        sim.step(a.equilibrate, path, use_graph=not a.direct)
        torch.cuda.synchronize()
    if a.what == "forces":
        fn = sim.forces_vertex if path == B.MD_VERTEX else sim.forces_edge
    elif a.what == "build":
        def fn():
            sim.build_cells()
            sim.build_verlet(B.MD_LIST_BOTH if path == B.MD_EDGE else B.MD_LIST_FULL)
    elif a.what == "step":
        def fn():
            sim.step(1, path, use_graph=False)
    elif a.what == "steps3":  # three steps: FIRST, then MIDDLE or fused launches, LAST
        def fn():
            sim.step(3, path, use_graph=False)
    elif a.what == "steps":  # one call of nsteps steps, every kernel launched directly (for launch lists)
        def fn():
            sim.step(a.nsteps, path, use_graph=False)
    else:  # the kernel one step runs (fused step kernel or force kernel): a warm-up and one timed launch
        def fn():
            sim.time_step_kernel(path, reps=1)
    st = torch.cuda.current_stream()
    fn()  # warm-up launch
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    status = sim.status()
    assert status[B.MD_STATUS_CODE] == 0, status
    entries = int(sim.view("nbr_count", torch.int32, s.n).sum().item())
    inner = int(sim.view("nbr_in_count", torch.int32, s.n).sum().item()) if a.prune > 0 else 0
    print(f"{a.workload} {a.precision} {a.path} {a.what}: median {statistics.median(times):.4f} ms over {a.reps}; "
          f"n={s.n} list_entries={entries} inner_entries={inner} kernel_sources_sha256={source_digest()}")


def source_digest() -> str:
    """sha256 of the step-kernel sources (the same digest bench.py checks before it quotes a capture)."""
    import hashlib
    import os
    h = hashlib.sha256()
    for f in ("md_forces.cuh", "md_forces.cu", "md_internal.cuh", "md_integrate.cuh", "md_step.cu"):
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


if __name__ == "__main__":
    main()

"""The vertex path with Newton's third law (MD_VERTEX_NEWTON, m force copies) against the FP64 oracle.

Its list holds every pair once (the same set as the edge path's half list) with each row about half of
the particle's neighbours; its forces follow the tolerances of the other paths (FP64 1e-12 per
component, mixed 1e-5 F_rms), for several numbers of copies.
"""
import numpy as np
import pytest

from paper_1401_4350_gb300 import binding as B
from tests.test_gpu_parity import Sim, check_fp64, check_mixed, get_sys, ref_forces

pytestmark = pytest.mark.gpu

NEWTON = B.MD_VERTEX_NEWTON


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


def _newton_sim(s, precision, m, **kw):
    sim = Sim(s, precision, force_copies=m, **kw)
    sim.build_cells()
    sim.build_verlet(B.MD_LIST_NEWTON)
    return sim


@pytest.mark.parametrize("name", ["lj4000", "wca20000", "patchy6000", "lj_tiny_box"])
def test_newton_list_is_the_half_list_split_evenly(name):
    import torch
    s = get_sys(name)
    ref = Sim(s, B.MD_MIXED)
    ref.build_cells()
    ref.build_verlet(B.MD_LIST_BOTH)
    half, ordered = ref.half_list_pairs()
    full_cnt = ref.view("nbr_count", torch.int32, s.n).cpu().numpy().copy()
    sim = _newton_sim(s, B.MD_MIXED, 4)
    pairs, counts, entries = sim.full_list_pairs()
    assert np.array_equal(pairs, half)          # every pair of the half list ...
    assert (counts == 1).all() and entries == len(half)  # ... exactly once
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0 and st[B.MD_STATUS_LISTS] == B.MD_LIST_NEWTON
    # rows: about half of the full row, with no systematic bias
    cnt = sim.view("nbr_count", torch.int32, s.n).cpu().numpy()
    assert abs(cnt.sum() * 2 - full_cnt.sum()) == 0
    if full_cnt.mean() > 20:
        assert np.abs(cnt - full_cnt / 2).mean() < 0.1 * full_cnt.mean()


@pytest.mark.parametrize("m", [1, 3, 16])
@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("name", ["lj4000", "lj5003", "wca20000", "patchy6000", "patchy_dimers", "lj_tiny_box"])
def test_newton_forces_match_oracle(name, precision, m):
    s = get_sys(name)
    Fr, Tr, Er, (Ur, Wr, npair) = ref_forces(s, name)
    sim = _newton_sim(s, precision, m)
    for rep in range(2):  # the second call checks that the copies were cleared
        sim.forces_vertex_newton()
        st = sim.status()
        assert st[B.MD_STATUS_CODE] == 0, st
        F, E, T, W = sim.forces()
        if precision == B.MD_FP64:
            check_fp64(F, Fr, f"F m={m} call {rep}")
            check_fp64(E, Er, f"E_i m={m}")
            assert E.sum() == pytest.approx(Ur, rel=1e-12, abs=1e-12)
            assert W.sum() == pytest.approx(Wr, rel=1e-12, abs=1e-12)
            if T is not None:
                check_fp64(T, Tr, f"T m={m}")
        else:
            check_mixed(F, Fr, f"F m={m} call {rep}")
            assert E.sum() == pytest.approx(Ur, rel=1e-5, abs=1e-5 * s.n)
            assert W.sum() == pytest.approx(Wr, rel=1e-5, abs=1e-5 * s.n)
            if T is not None:
                check_mixed(T, Tr, f"T m={m}")


def test_vertex_kernel_refuses_the_newton_list():
    s = get_sys("lj4000")
    sim = _newton_sim(s, B.MD_MIXED, 2)
    sim.forces_vertex()
    assert sim.status()[B.MD_STATUS_CODE] == B.MD_ERR_INVALID


def test_newton_kernel_refuses_the_full_list():
    s = get_sys("lj4000")
    sim = Sim(s, B.MD_MIXED, force_copies=2)
    sim.build_cells()
    sim.build_verlet(B.MD_LIST_FULL)
    sim.forces_vertex_newton()
    assert sim.status()[B.MD_STATUS_CODE] == B.MD_ERR_INVALID


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
def test_newton_steps_follow_the_vertex_trajectory(precision, use_graph):
    """120 steps through md_step_verlet with the Newton path (rebuilds included) stay on the vertex
    path's trajectory to the precision's level, and the forces at the end match the oracle."""
    s = get_sys("lj4000")
    a = Sim(s, precision, force_copies=8, trace_capacity=128)
    b = Sim(s, precision, trace_capacity=128)
    a.prepare(NEWTON)
    b.prepare(B.MD_VERTEX)
    a.step(120, NEWTON, use_graph=use_graph)
    b.step(120, B.MD_VERTEX, use_graph=use_graph)
    sa, sb = a.status(), b.status()
    assert sa[B.MD_STATUS_CODE] == 0 and sb[B.MD_STATUS_CODE] == 0
    assert sa[B.MD_STATUS_REBUILDS] >= 1
    xa, _ = a.positions()
    xb, _ = b.positions()
    assert np.abs(xa - xb).max() < (1e-9 if precision == B.MD_FP64 else 1e-4)
    ta, tb = a.trace(), b.trace()
    rows = ta[:, 0] > 0
    e_a = ta[rows, 1] + ta[rows, 2]
    e_b = tb[rows, 1] + tb[rows, 2]
    assert np.abs(e_a - e_b).max() < (1e-8 if precision == B.MD_FP64 else 1e-3) * s.n
    import oracle
    from tests.test_gpu_parity import model_of
    Fr, _, _, _ = oracle.forces(xa, model_of(s), use_cells=True)
    F, _, _, _ = a.forces()
    if precision == B.MD_FP64:
        check_fp64(F, Fr, "F after steps")
    else:
        check_mixed(F, Fr, "F after steps")


@pytest.mark.parametrize("name", ["lj5003", "patchy6000"])
def test_autotune_system_times_every_path_and_prepares_the_winner(name):
    """The single-system autotuner times vertex (1/2/4/8 threads), edge, Newton-vertex and the per-edge
    store, keeps the fastest, and leaves forces of that path (matching the oracle) behind."""
    s = get_sys(name)
    Fr, Tr, Er, _ = ref_forces(s, name)
    sim = Sim(s, B.MD_MIXED, force_copies=4, edge_store=1)
    x0, v0 = sim.positions()
    q0 = sim.orientations() if s.quat is not None else None
    path, tpp, block, ms = sim.autotune()
    # the timed launches moved nothing: every candidate's changes were put back
    x1, v1 = sim.positions()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    if q0 is not None:
        q1 = sim.orientations()
        assert np.array_equal(q0[0], q1[0]) and np.array_equal(q0[1], q1[1])
    assert all(t > 0 for t in ms), ms
    assert (path, tpp, block) == B.TUNE_CANDIDATES[int(np.argmin(ms))]
    assert (sim.params.threads_per_particle, sim.params.block_size) == (tpp, block)
    assert sim.status()[B.MD_STATUS_CODE] == 0
    F, E, T, W = sim.forces()
    check_mixed(F, Fr, "force after autotune")
    if T is not None:
        check_mixed(T, Tr, "torque after autotune")
    # without copies or store those two candidates are skipped
    sim2 = Sim(s, B.MD_MIXED)
    _, _, _, ms2 = sim2.autotune()
    assert ms2[14] == -1 and ms2[15] == -1 and all(t > 0 for t in ms2[:14])

"""Batched replicas: one persistent force launch over replicas of uneven size, each with its own
decomposition, must compute what the single-system path computes for each replica alone (vertex:
bit for bit; edge: up to the order of its atomic additions), and match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems

pytestmark = pytest.mark.gpu

V, E = B.MD_VERTEX, B.MD_EDGE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_batch_release()
    B.md_release_graphs()


def _replicas():
    specs = [(systems.LJ, 500, 0.9, V, 1), (systems.LJ, 777, 0.3, E, 1), (systems.WCA, 600, 0.2, V, 2),
             (systems.LJ, 1500, 0.6, V, 4), (systems.LJ, 3001, 0.85, E, 1), (systems.WCA, 2500, 0.2, E, 1),
             (systems.LJ, 4000, 0.85, V, 8), (systems.LJ, 1234, 0.45, V, 2), (systems.WCA, 1800, 0.2, V, 1)]
    out = []
    for k, (kind, n, rho, path, tpp) in enumerate(specs):
        out.append((systems.make_replica(kind, n, rho, seed=7000 + k), path, tpp))
    return out


def _single(s, path, tpp):
    from paper_1401_4350_gb300.sim import Simulation
    sim = Simulation(s, B.MD_MIXED, tpp=tpp)
    sim.prepare(path)
    return sim


def _batch(reps, **kw):
    from paper_1401_4350_gb300.sim import BatchSimulation
    return BatchSimulation([s for s, _, _ in reps], paths=[p for _, p, _ in reps], tpps=[t for _, _, t in reps], **kw)


def _check(F, Fr, what):
    frms = np.sqrt((Fr ** 2).sum(1).mean())
    err = np.abs(F - Fr).max()
    assert err <= 1e-5 * frms, f"{what}: {err / frms:.3e} F_rms"


def test_batch_forces_match_single_system_and_oracle():
    reps = _replicas()
    bs = _batch(reps)
    bs.prepare()
    for r, (s, path, tpp) in enumerate(reps):
        assert bs.replica_status(r)[B.MD_STATUS_CODE] == 0
        F, Ei, Wi = bs.replica_forces(r)
        Fs, Es, _, _ = _single(s, path, tpp).forces()
        if path == V:
            assert np.array_equal(F, Fs), f"replica {r}"
        else:
            np.testing.assert_allclose(F, Fs, atol=1e-6 * max(1.0, np.abs(Fs).max()))
        m = oracle.Model(s.kind, tuple(s.box), s.rc)
        Fr, _, Er, (Ur, _, _) = oracle.forces(s.pos, m, use_cells=s.n > 1500)
        _check(F, Fr, f"replica {r}")
        assert Ei.sum() == pytest.approx(Ur, rel=1e-5, abs=1e-4)
    bs.release()


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_steps_match_single_system(use_graph):
    reps = _replicas()
    bs = _batch(reps, trace_capacity=64)
    bs.prepare()
    steps = 60
    bs.step(steps, use_graph)
    for r, (s, path, tpp) in enumerate(reps):
        st = bs.replica_status(r)
        assert st[B.MD_STATUS_CODE] == 0 and st[B.MD_STATUS_STEPS] == steps
        single = _single(s, path, tpp)
        single.step(steps, path, True)
        ss = single.status()
        pos, vel = bs.replica_positions(r)
        pos_s, vel_s = single.positions()
        if path == V:
            assert np.array_equal(pos, pos_s) and np.array_equal(vel, vel_s), f"replica {r}"
            assert st[B.MD_STATUS_REBUILDS] == ss[B.MD_STATUS_REBUILDS]
        else:
            # the edge path sums its pairs with atomics in no fixed order (and the single-system kernel
            # groups the i-side warp sums by other spans than the batched items), so the trajectories
            # differ at the rounding level: ~1e-7 of a pair force, a few 1e-9 in position after 60 steps
            assert np.abs(pos - pos_s).max() < 1e-7
    bs.release()


def test_batch_rebuilds_only_flagged_replicas_and_stays_correct():
    reps = [(systems.make_replica(systems.LJ, 2000, 0.8, seed=7100), V, 1),
            (systems.make_replica(systems.WCA, 1500, 0.2, seed=7101), E, 1)]
    # a hot replica (rebuilds often) next to a cold one
    reps[0][0].vel *= 3.0
    bs = _batch(reps)
    bs.prepare()
    bs.step(150)
    st = [bs.replica_status(r) for r in range(2)]
    assert st[0][B.MD_STATUS_REBUILDS] > st[1][B.MD_STATUS_REBUILDS] >= 0
    for r, (s, path, tpp) in enumerate(reps):
        pos, _ = bs.replica_positions(r)
        F, _, _ = bs.replica_forces(r)
        Fr, _, _, _ = oracle.forces(np.mod(pos, s.box), oracle.Model(s.kind, tuple(s.box), s.rc), use_cells=False)
        _check(F, Fr, f"replica {r} after {st[r][B.MD_STATUS_REBUILDS]} rebuilds")
    bs.release()


def test_autotune_chooses_a_valid_configuration_and_keeps_parity():
    reps = _replicas()
    bs = _batch(reps)
    paths, tpps = bs.autotune()
    assert all(p in (V, E) for p in paths) and all(t in (1, 2, 4) for t in tpps)
    assert (paths, tpps) == tuple(bs.config())
    for r, (s, _, _) in enumerate(reps):
        F, _, _ = bs.replica_forces(r)
        Fr, _, _, _ = oracle.forces(s.pos, oracle.Model(s.kind, tuple(s.box), s.rc), use_cells=s.n > 1500)
        _check(F, Fr, f"replica {r} ({'edge' if paths[r] == E else 'vertex'} tpp {tpps[r]})")
    bs.step(20)
    assert all(bs.replica_status(r)[B.MD_STATUS_CODE] == 0 for r in range(len(reps)))
    bs.release()


def test_batch_rejects_what_it_does_not_batch():
    import torch
    from paper_1401_4350_gb300.sim import make_params
    s = systems.make_patchy(600, 0.3, seed=3)
    p = make_params(s, B.MD_MIXED)
    assert B.md_batch_workspace_bytes([p]) == 0
    assert "mixed-precision LJ and WCA" in B.last_error()
    q = make_params(systems.make_lj(500, 0.9, seed=4), B.MD_FP64)
    assert B.md_batch_workspace_bytes([q]) == 0


NW = B.MD_VERTEX_NEWTON


def _newton_replicas():
    specs = [(systems.LJ, 900, 0.8, NW, 1), (systems.LJ, 1600, 0.5, V, 2), (systems.WCA, 1200, 0.2, NW, 1),
             (systems.LJ, 2500, 0.85, E, 1), (systems.LJ, 3100, 0.7, NW, 1)]
    return [(systems.make_replica(kind, n, rho, seed=7200 + k), path, tpp)
            for k, (kind, n, rho, path, tpp) in enumerate(specs)]


def test_batch_newton_replicas_match_single_system_and_oracle():
    """Replicas on the Newton-vertex path (force copies in their sub-workspaces) next to vertex and edge
    replicas: forces equal the single-system Newton path up to the order of the atomic additions, and
    the oracle; 60 steps stay on the single-system trajectory."""
    from paper_1401_4350_gb300.sim import Simulation
    reps = _newton_replicas()
    bs = _batch(reps, force_copies=2)
    bs.prepare()
    singles = []
    for r, (s, path, tpp) in enumerate(reps):
        assert bs.replica_status(r)[B.MD_STATUS_CODE] == 0
        F, Ei, Wi = bs.replica_forces(r)
        sim = Simulation(s, B.MD_MIXED, tpp=tpp, force_copies=2)
        sim.prepare(path)
        Fs, _, _, _ = sim.forces()
        np.testing.assert_allclose(F, Fs, atol=1e-6 * max(1.0, np.abs(Fs).max()))
        Fr, _, _, _ = oracle.forces(s.pos, oracle.Model(s.kind, tuple(s.box), s.rc), use_cells=s.n > 1500)
        _check(F, Fr, f"replica {r}")
        singles.append(sim)
    bs.step(60)
    for r, (s, path, tpp) in enumerate(reps):
        assert bs.replica_status(r)[B.MD_STATUS_CODE] == 0
        singles[r].step(60, path, True)
        pos, _ = bs.replica_positions(r)
        pos_s, _ = singles[r].positions()
        d = pos - pos_s
        d -= s.box * np.rint(d / s.box)
        assert np.abs(d).max() < 1e-6, f"replica {r}"
    bs.release()


def test_autotune_includes_the_newton_path_when_copies_exist():
    reps = _newton_replicas()
    bs = _batch(reps, force_copies=1)
    paths, tpps = bs.autotune()
    assert all(p in (V, E, NW) for p in paths)
    assert all(t == 1 for p, t in zip(paths, tpps) if p != V)
    for r, (s, _, _) in enumerate(reps):
        assert bs.replica_status(r)[B.MD_STATUS_CODE] == 0
        F, _, _ = bs.replica_forces(r)
        Fr, _, _, _ = oracle.forces(s.pos, oracle.Model(s.kind, tuple(s.box), s.rc), use_cells=s.n > 1500)
        _check(F, Fr, f"replica {r} (path {paths[r]}, tpp {tpps[r]})")
    bs.step(20)
    assert all(bs.replica_status(r)[B.MD_STATUS_CODE] == 0 for r in range(len(reps)))
    bs.release()

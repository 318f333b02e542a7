"""Fused steps (fuse_step = 1): the isotropic mixed vertex path runs each step's forces and integration
in one kernel that reads one position buffer and writes the other.  Positions, velocities, step and
rebuild counts must be those of the separate force and integrate kernels bit for bit (same force
arithmetic, same integration arithmetic, same decisions), in graph and direct launches, for even and
odd step counts (the state ends in either buffer), cubic and non-cubic boxes, every threads-per-particle
setting and with the momentum-refresh thermostat; so are the energy totals (exact integer sums of
per-particle terms).  Paths that cannot fuse are unchanged by the flag, and the kernel timer leaves the system as it
was."""
import numpy as np
import pytest

import oracle
from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems
from tests.test_gpu_parity import Sim, get_sys, model_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


def _noncubic_lj():
    s = systems.make_lj(4000, 0.85, 1.0, seed=1011)
    stretch = np.array([1.0, 1.07, 0.96])
    return systems.System(systems.LJ, np.mod(s.pos * stretch, s.box * stretch), s.vel, s.box * stretch, 2.5, 0.3,
                          0.001, 1.0, name="lj_noncubic")


_extra = {}


def _system(name):
    if name == "lj_noncubic":
        if name not in _extra:
            _extra[name] = _noncubic_lj()
        return _extra[name]
    if name == "lj_nvt":
        if name not in _extra:
            _extra[name] = systems.make_lj_nvt(3000, 0.5, temperature=1.8, seed=44, thermostat_every=7,
                                               thermostat_prob=0.3)
        return _extra[name]
    return get_sys(name)


def _run(s, fuse, steps, use_graph, tpp=1, block=0, trace=0):
    sim = Sim(s, B.MD_MIXED, tpp=tpp, block=block, fuse_step=fuse, trace_capacity=trace)
    sim.prepare(B.MD_VERTEX)
    sim.step(steps, B.MD_VERTEX, use_graph=use_graph)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0, st
    return sim, st


def _same_state(a, b):
    xa, va = a.positions()
    xb, vb = b.positions()
    assert np.array_equal(xa, xb)
    assert np.array_equal(va, vb)
    assert np.array_equal(a.id.cpu().numpy(), b.id.cpu().numpy())  # the same slot order (same rebuilds)


def _close_energies(a, b, n):
    """The energy totals are exact sums of per-particle fixed-point terms, so equal per-particle terms give
    equal totals however the particles fall into warps and blocks."""
    ea, eb = a.energies(), b.energies()
    for k in ("U", "KT", "W"):
        assert ea[k] == eb[k], (k, ea[k], eb[k])


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("steps", [1, 2, 75, 76])
@pytest.mark.parametrize("name", ["lj4000", "lj_noncubic", "wca20000"])
def test_fused_steps_equal_separate_kernels(name, steps, use_graph):
    s = _system(name)
    a, sa = _run(s, 1, steps, use_graph)
    b, sb = _run(s, 0, steps, use_graph)
    assert sa[B.MD_STATUS_STEPS] == sb[B.MD_STATUS_STEPS] == steps
    assert sa[B.MD_STATUS_REBUILDS] == sb[B.MD_STATUS_REBUILDS]
    if steps >= 75:
        assert sa[B.MD_STATUS_REBUILDS] >= 1
    _same_state(a, b)
    _close_energies(a, b, s.n)
    Fa, Ea, _, Wa = a.forces()  # the last force evaluation of the call is written in both
    Fb, Eb, _, Wb = b.forces()
    assert np.array_equal(Fa, Fb) and np.array_equal(Ea, Eb) and np.array_equal(Wa, Wb)


@pytest.mark.parametrize("tpp,block", [(2, 64), (4, 128), (8, 256), (1, 256), (1, 32)])
def test_fused_steps_every_thread_split(tpp, block):
    s = get_sys("lj4000")
    a, sa = _run(s, 1, 61, True, tpp=tpp, block=block)
    b, sb = _run(s, 0, 61, True, tpp=tpp, block=block)
    assert sa[B.MD_STATUS_REBUILDS] == sb[B.MD_STATUS_REBUILDS]
    _same_state(a, b)
    _close_energies(a, b, s.n)


@pytest.mark.parametrize("use_graph", [True, False])
def test_fused_steps_with_the_thermostat(use_graph):
    s = _system("lj_nvt")
    a, _ = _run(s, 1, 50, use_graph)
    b, _ = _run(s, 0, 50, use_graph)
    _same_state(a, b)
    s.thermostat_every = 0  # the same run without refreshes ends elsewhere: the refreshes took place
    try:
        c, _ = _run(s, 1, 50, use_graph)
    finally:
        s.thermostat_every = 7
    assert not np.array_equal(a.positions()[1], c.positions()[1])


def test_fused_trace_rows_match():
    s = get_sys("lj4000")
    a, _ = _run(s, 1, 40, True, trace=64)
    b, _ = _run(s, 0, 40, True, trace=64)
    ta, tb = a.trace(), b.trace()
    assert np.array_equal(ta, tb)


def test_repeated_calls_continue_the_trajectory():
    """Two calls of 31 steps (each ending in the alternate buffers, copied back) equal one call of 31 +
    one of 31 with separate kernels, and the state between calls is in the caller's arrays."""
    s = get_sys("lj4000")
    a = Sim(s, B.MD_MIXED, fuse_step=1)
    b = Sim(s, B.MD_MIXED, fuse_step=0)
    for sim in (a, b):
        sim.prepare(B.MD_VERTEX)
    for _ in range(2):
        a.step(31, B.MD_VERTEX)
        b.step(31, B.MD_VERTEX)
        _same_state(a, b)


@pytest.mark.parametrize("name,precision,path", [
    ("lj4000", B.MD_MIXED, B.MD_EDGE), ("lj4000", B.MD_FP64, B.MD_VERTEX), ("patchy6000", B.MD_MIXED, B.MD_VERTEX)])
def test_flag_leaves_other_paths_unchanged(name, precision, path):
    s = get_sys(name)
    out = []
    for fuse in (1, 0):
        sim = Sim(s, precision, fuse_step=fuse)
        sim.prepare(path)
        sim.step(30, path)
        assert sim.status()[B.MD_STATUS_CODE] == 0
        out.append(sim.positions())
    if path == B.MD_EDGE:  # atomics: the same to rounding
        np.testing.assert_allclose(out[0][0], out[1][0], rtol=0, atol=1e-9)
    else:
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("fuse,prune", [(1, 0.0), (0, 0.0), (1, 0.1)])
def test_kernel_timer_leaves_the_system_unchanged(fuse, prune):
    import torch
    s = get_sys("lj4000")
    a = Sim(s, B.MD_MIXED, fuse_step=fuse, trace_capacity=8, prune_skin=prune)
    b = Sim(s, B.MD_MIXED, fuse_step=fuse, trace_capacity=8, prune_skin=prune)
    for sim in (a, b):
        sim.prepare(B.MD_VERTEX)
        sim.step(5, B.MD_VERTEX)
    words = lambda sim: (sim.status().copy(), sim.view("energy", torch.float64, 8).cpu().numpy().copy(),
                         sim.trace().copy())
    before = words(a)
    ms = a.time_step_kernel(B.MD_VERTEX, reps=5)
    assert 0.0 < ms < 1000.0
    after = words(a)
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    _same_state(a, b)
    for sim in (a, b):
        sim.step(40, B.MD_VERTEX)
    _same_state(a, b)


# ---- the inner list (prune_skin > 0) ------------------------------------------------------------

def _is_subsequence(small, big):
    it = iter(big.tolist())
    return all(any(x == y for y in it) for x in small.tolist())


def test_inner_list_holds_every_pair_within_rc_in_verlet_list_order():
    """After the first fused step (which prunes), every row of the inner list is a subsequence of the
    slot's Verlet-list row, and it holds every pair closer than rc at the current positions."""
    s = get_sys("lj4000")
    sim = Sim(s, B.MD_MIXED, fuse_step=1, prune_skin=0.1)
    sim.prepare(B.MD_VERTEX)
    sim.step(2, B.MD_VERTEX)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0 and st[B.MD_STATUS_PRUNES] == 1, st
    outer = sim.list_rows("nbr", "nbr_count")
    inner = sim.list_rows("nbr_in", "nbr_in_count")
    assert all(_is_subsequence(r_in, r_out) for r_in, r_out in zip(inner, outer))
    assert sum(len(r) for r in inner) < 0.95 * sum(len(r) for r in outer)
    x = sim.pos[:, :3].cpu().numpy()  # slot order
    close = oracle.pairs(x, s.box, s.rc, use_cells=True)
    sets = [set(r.tolist()) for r in inner]
    assert all(j in sets[i] and i in sets[j] for i, j in close)


@pytest.mark.parametrize("tpp", [1, 2])
@pytest.mark.parametrize("use_graph", [True, False])
def test_pruned_steps_follow_the_oracle(use_graph, tpp):
    """150 steps with an inner list (rc + 0.1), rebuilds and prunes included, stay on the oracle's FP64
    trajectory to the mixed precision's level (as without the inner list); with two threads per
    particle the inner list is not used and nothing is pruned."""
    s = get_sys("lj4000")
    steps = 150
    p_ref, v_ref, _, _, tr = oracle.run_nve(s.pos, s.vel, model_of(s), s.dt, steps, use_cells=True)
    sim = Sim(s, B.MD_MIXED, fuse_step=1, prune_skin=0.1, tpp=tpp, trace_capacity=steps + 1)
    sim.prepare(B.MD_VERTEX)
    sim.step(steps, B.MD_VERTEX, use_graph=use_graph)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0 and st[B.MD_STATUS_REBUILDS] >= 1, st
    if tpp == 1:
        assert st[B.MD_STATUS_PRUNES] > st[B.MD_STATUS_REBUILDS] + 1, st
    else:
        assert st[B.MD_STATUS_PRUNES] == 0, st
    pos, _ = sim.positions()
    d = pos - p_ref
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() < 1e-6
    t = sim.trace()
    e_gpu = t[:, 1] + t[:, 2]
    e_ref = tr[:, 0] + tr[:, 1] + tr[:, 2]
    assert np.abs(e_gpu - e_ref).max() / s.n < 1e-5
    # the same run without the inner list: the same trajectory up to the order of the FP32 sums
    plain, _ = _run(s, 1, steps, use_graph, tpp=tpp)
    dp = pos - plain.positions()[0]
    dp -= s.box * np.rint(dp / s.box)
    assert np.abs(dp).max() < 1e-8


@pytest.mark.parametrize("name", ["lj_tiny_box", "lj_noncubic", "wca20000"])
def test_pruned_steps_on_small_and_noncubic_boxes(name):
    """The inner list on a 500-particle box (a 5x5x5 grid of half cells, every row wrapping), on WCA, and
    (switched off: non-cubic) on a non-cubic box: 120 steps stay on the separate kernels' trajectory to
    rounding, and the status is clean."""
    s = _system(name)
    a = Sim(s, B.MD_MIXED, fuse_step=1, prune_skin=0.1 if name != "wca20000" else 0.08)
    b = Sim(s, B.MD_MIXED, fuse_step=0)
    for sim in (a, b):
        sim.prepare(B.MD_VERTEX)
        sim.step(120, B.MD_VERTEX)
    sa = a.status()
    assert sa[B.MD_STATUS_CODE] == 0, sa
    if name == "lj_noncubic":
        assert sa[B.MD_STATUS_PRUNES] == 0
    else:
        assert sa[B.MD_STATUS_PRUNES] >= 2
    d = a.positions()[0] - b.positions()[0]
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() < 1e-8

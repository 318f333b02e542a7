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

from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems
from tests.test_gpu_parity import Sim, get_sys

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


@pytest.mark.parametrize("fuse", [1, 0])
def test_kernel_timer_leaves_the_system_unchanged(fuse):
    import torch
    s = get_sys("lj4000")
    a = Sim(s, B.MD_MIXED, fuse_step=fuse, trace_capacity=8)
    b = Sim(s, B.MD_MIXED, fuse_step=fuse, trace_capacity=8)
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

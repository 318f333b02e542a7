"""The paper's patchy form (MD_PATCHY_POW) and the momentum-refresh thermostat on the GPU, against the
oracle: forces of every path at the paper's densities, refreshed momenta bit-compatible with the
oracle's draws (same generator), and thermostatted FP64 trajectories."""
import numpy as np
import pytest

import oracle
from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems
from tests.test_gpu_parity import Sim, check_fp64, check_mixed, model_of
from tests.test_oracle_pow import _pow_dimers

pytestmark = pytest.mark.gpu

PATHS = [B.MD_VERTEX, B.MD_EDGE, B.MD_VERTEX_NEWTON, B.MD_EDGE_STORE]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


_sys, _ref = {}, {}


def _pow_dimer_system():
    rng = np.random.default_rng(31)
    box = np.array([18.0, 18.0, 18.0])
    pos, quat = _pow_dimers(120, box, rng)
    n = len(pos)
    s = systems.System(systems.PATCHY_POW, pos, rng.normal(0, 0.3, (n, 3)), box, 1.18, 0.2, 0.001, 0.15,
                       quat=quat, angmom=rng.normal(0, 0.1, (n, 3)), patches=systems.PATCH_DIRS_POLAR * 0.5,
                       patch_rc=0.18, name="pow_dimers")
    return s


def get(name):
    if name not in _sys:
        if name == "pow_dimers":
            _sys[name] = _pow_dimer_system()
        else:
            rho = float(name.split("_")[-1])
            _sys[name] = systems.make_patchy_pow(4000, rho, seed=1005)
        s = _sys[name]
        _ref[name] = oracle.forces(s.pos, model_of(s), quat=s.quat, use_cells=True)
    return _sys[name], _ref[name]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("name", ["pow_rho_0.1", "pow_rho_0.3", "pow_rho_0.5", "pow_dimers"])
def test_pow_forces_match_oracle(name, precision, path):
    s, (Fr, Tr, Er, (Ur, Wr, npair)) = get(name)
    sim = Sim(s, precision, force_copies=4, edge_store=1)
    sim.prepare(path)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0, st
    F, E, T, W = sim.forces()
    if precision == B.MD_FP64:
        check_fp64(F, Fr, "force")
        check_fp64(T, Tr, "torque")
        assert E.sum() == pytest.approx(Ur, rel=1e-12, abs=1e-12)
    else:
        check_mixed(F, Fr, "force")
        check_mixed(T, Tr, "torque")
        assert E.sum() == pytest.approx(Ur, rel=1e-5, abs=1e-5 * s.n)
    if name == "pow_dimers":
        assert np.abs(Tr).max() > 1e-2  # the patch terms are exercised


def _free_gas(kind, every, prob, seed, n=512):
    k = int(round(n ** (1 / 3)))
    g = np.arange(k) * 3.2
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.4
    box = np.full(3, k * 3.2)
    rng = np.random.default_rng(seed)
    vel = rng.normal(size=(len(pos), 3))
    if kind == "lj":
        s = systems.System(systems.LJ, pos, vel, box, 2.5, 0.3, 0.001, 1.5, mass=2.0)
    else:
        s = systems.System(systems.PATCHY_POW, pos, vel, box, 1.18, 0.2, 0.001, 1.5, mass=2.0,
                           quat=np.tile([1.0, 0, 0, 0], (len(pos), 1)), angmom=rng.normal(size=(len(pos), 3)),
                           patches=systems.PATCH_DIRS_POLAR * 0.5, patch_rc=0.18)
    s.thermostat_every, s.thermostat_prob, s.seed = every, prob, seed
    return s


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("kind", ["lj", "pow"])
def test_refreshed_momenta_are_the_oracle_draws(kind, use_graph):
    """No forces, every = 3, prob = 0.5, 8 steps: the momenta of refreshed particles are the oracle's
    draws at step 6 (or 3), the others keep their values; GPU and oracle use the same generator."""
    s = _free_gas(kind, 3, 0.5, 77)
    sim = Sim(s, B.MD_FP64)
    sim.prepare(B.MD_VERTEX)
    sim.step(8, B.MD_VERTEX, use_graph=use_graph)
    assert sim.status()[B.MD_STATUS_CODE] == 0
    _, v = sim.positions()
    L = sim.orientations()[1] if kind == "pow" else None
    m = model_of(s)
    th = oracle.Thermostat(every=3, prob=0.5, kT=1.5, seed=77)
    _, vr, _, Lr, _ = oracle.run(s.pos, s.vel, m, s.dt, 8, mass=2.0, inertia=s.inertia, quat=s.quat,
                                 angmom=s.angmom, thermostat=th)
    np.testing.assert_allclose(v, vr, rtol=1e-13, atol=1e-14)
    assert not np.allclose(v, s.vel)
    if L is not None:
        np.testing.assert_allclose(L, Lr, rtol=1e-13, atol=1e-14)


def test_thermostatted_lj_trajectory_follows_the_oracle():
    s = systems.make_lj_nvt(1000, 0.3, temperature=1.8, seed=41, thermostat_every=10, thermostat_prob=0.3)
    sim = Sim(s, B.MD_FP64, trace_capacity=64)
    sim.prepare(B.MD_VERTEX)
    sim.step(60, B.MD_VERTEX, use_graph=True)
    assert sim.status()[B.MD_STATUS_CODE] == 0
    x, v = sim.positions()
    th = oracle.Thermostat(every=10, prob=0.3, kT=1.8, seed=41)
    xr, vr, _, _, trace = oracle.run(s.pos, s.vel, model_of(s), s.dt, 60, thermostat=th)
    d = x - xr
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() < 1e-9
    assert np.abs(v - vr).max() < 1e-8
    t = sim.trace()
    row = t[t[:, 0] == 60][0]
    assert row[1] == pytest.approx(trace[60, 0] + trace[60, 1], rel=1e-10)
    assert row[2] == pytest.approx(trace[60, 2], rel=1e-10)


@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
def test_pow_thermostatted_trajectory_follows_the_oracle(path):
    s, _ = get("pow_dimers")
    s.thermostat_every, s.thermostat_prob, s.seed = 7, 0.2, 9
    try:
        sim = Sim(s, B.MD_FP64)
        sim.prepare(path)
        sim.step(40, path, use_graph=True)
        assert sim.status()[B.MD_STATUS_CODE] == 0
        x, v = sim.positions()
        q, L = sim.orientations()
        th = oracle.Thermostat(every=7, prob=0.2, kT=s.temperature, seed=9)
        xr, vr, qr, Lr, _ = oracle.run(s.pos, s.vel, model_of(s), s.dt, 40, inertia=s.inertia, quat=s.quat,
                                       angmom=s.angmom, thermostat=th)
    finally:
        s.thermostat_every, s.thermostat_prob, s.seed = 0, 0.0, 0
    d = x - xr
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() < 1e-9
    assert np.abs(L - Lr).max() < 1e-8
    assert np.abs(np.abs((q * qr).sum(1)) - 1.0).max() < 1e-12  # same orientation (q and -q agree)

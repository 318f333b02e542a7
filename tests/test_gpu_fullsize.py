"""Parity at full benchmark sizes, in the launch configuration bench.py times (default block and
threads per particle): every force of the GPU result against the FP64 cell-list oracle."""
import numpy as np
import pytest

import oracle
from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems

pytestmark = pytest.mark.gpu

_ref = {}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


WORKLOADS = {
    "lj1m": lambda: systems.make_lj(1_048_576, 0.85, 1.0, seed=1001),
    "wca1m": lambda: systems.make_wca(1_048_576, 0.2, seed=1002),
    "patchy262k": lambda: systems.make_patchy(262_144, 0.3, seed=1003),
}


def reference(name):
    if name not in _ref:
        s = WORKLOADS[name]()
        m = oracle.Model(s.kind, tuple(s.box), s.rc, patches=s.patches)
        _ref[name] = (s, oracle.forces(s.pos, m, quat=s.quat, use_cells=True))
    return _ref[name]


def _run(s, precision, path):
    import torch
    from paper_1401_4350_gb300.sim import Simulation
    sim = Simulation(s, precision)
    sim.prepare(path)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0, st
    out = sim.forces()
    del sim
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("name,path", [("lj1m", B.MD_VERTEX), ("lj1m", B.MD_EDGE), ("wca1m", B.MD_VERTEX),
                                       ("wca1m", B.MD_EDGE), ("patchy262k", B.MD_VERTEX),
                                       ("patchy262k", B.MD_EDGE)])
def test_mixed_full_size(name, path):
    s, (Fr, Tr, Er, (Ur, Wr, _)) = reference(name)
    F, E, T, W = _run(s, B.MD_MIXED, path)
    frms = np.sqrt((Fr ** 2).sum(1).mean())
    err = np.abs(F - Fr).max()
    assert err <= 1e-5 * frms, f"max force error {err:.3e} = {err / frms:.3e} F_rms"
    assert E.sum() == pytest.approx(Ur, rel=1e-5)
    if T is not None:
        trms = np.sqrt((Tr ** 2).sum(1).mean())  # rms over all particles
        terr = np.abs(T - Tr).max()
        assert terr <= 1e-5 * trms, f"max torque error {terr:.3e} = {terr / trms:.3e} tau_rms"


@pytest.mark.parametrize("name,path", [("lj1m", B.MD_VERTEX), ("lj1m", B.MD_EDGE)])
def test_fp64_full_size(name, path):
    s, (Fr, Tr, Er, (Ur, Wr, _)) = reference(name)
    F, E, T, W = _run(s, B.MD_FP64, path)
    frms = np.sqrt((Fr ** 2).sum(1).mean())
    rel = np.abs(F - Fr) / np.maximum(np.abs(Fr), frms)
    assert rel.max() <= 1e-12, rel.max()


def test_headline_fused_inner_list_full_size_after_rebuilds():
    """The kernel the benchmark times (one fused force + integrate launch per step over the inner list,
    prune_skin 0.1, LJ N = 1,048,576) after enough steps for rebuilds and prunes: the forces of the
    call's last fused launch, at the GPU's own final positions, against the FP64 cell-list oracle at
    those positions, element by element (1e-5 F_rms)."""
    import torch
    from paper_1401_4350_gb300.sim import Simulation
    s = WORKLOADS["lj1m"]()
    sim = Simulation(s, B.MD_MIXED, fuse_step=1, prune_skin=0.1)
    sim.prepare(B.MD_VERTEX)
    sim.step(150, B.MD_VERTEX, use_graph=True)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0, st
    assert st[B.MD_STATUS_REBUILDS] >= 1 and st[B.MD_STATUS_PRUNES] >= 2, st
    pos, _ = sim.positions()
    F, E, _, W = sim.forces()
    del sim
    torch.cuda.empty_cache()
    m = oracle.Model(s.kind, tuple(s.box), s.rc)
    Fr, _, Er, (Ur, Wr, _) = oracle.forces(np.mod(pos, s.box), m, use_cells=True)
    frms = np.sqrt((Fr ** 2).sum(1).mean())
    err = np.abs(F - Fr).max()
    assert err <= 1e-5 * frms, f"max force error {err:.3e} = {err / frms:.3e} F_rms"
    assert E.sum() == pytest.approx(Ur, rel=1e-5)
    assert W.sum() == pytest.approx(Wr, rel=1e-5)

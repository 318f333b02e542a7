"""The edge path with a per-edge store and a per-particle reduction (MD_EDGE_STORE): the by-partner index
is exact, forces follow the oracle to the usual tolerances, and, having no atomics, every result is
bit-for-bit reproducible (also for mixed precision, and along a trajectory with rebuilds)."""
import numpy as np
import pytest

from paper_1401_4350_gb300 import binding as B
from tests.test_gpu_parity import Sim, check_fp64, check_mixed, get_sys, ref_forces

pytestmark = pytest.mark.gpu

ES = B.MD_EDGE_STORE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


def _es_sim(s, precision, **kw):
    sim = Sim(s, precision, edge_store=1, **kw)
    sim.build_cells()
    sim.build_verlet(B.MD_LIST_BOTH)
    return sim


@pytest.mark.parametrize("name", ["lj4000", "wca20000", "patchy6000", "lj_tiny_box"])
def test_partner_index_lists_each_pair_once_in_order(name):
    import torch
    s = get_sys(name)
    sim = _es_sim(s, B.MD_MIXED)
    n = s.n
    hs = sim.view("half_start", torch.int64, n + 1).cpu().numpy()
    E = int(hs[-1])
    half_j = sim.view("half_j", torch.int32, E).cpu().numpy()
    js = sim.view("jstart", torch.int64, n + 1).cpu().numpy()
    je = sim.view("jedge", torch.int32, E).cpu().numpy()
    assert js[-1] == E
    assert np.array_equal(np.sort(je), np.arange(E))            # every pair exactly once
    owner = np.repeat(np.arange(n), np.diff(js))
    assert np.array_equal(half_j[je], owner)                    # in its partner's row
    rows_sorted = np.all((np.diff(je) > 0) | (np.diff(owner) != 0))
    assert rows_sorted                                          # increasing within a row


@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("name", ["lj4000", "lj5003", "wca20000", "patchy6000", "patchy_dimers", "lj_tiny_box"])
def test_edge_store_forces_match_oracle(name, precision):
    s = get_sys(name)
    Fr, Tr, Er, (Ur, Wr, npair) = ref_forces(s, name)
    sim = _es_sim(s, precision)
    sim.forces_edge_store()
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0, st
    F, E, T, W = sim.forces()
    if precision == B.MD_FP64:
        check_fp64(F, Fr, "force")
        check_fp64(E, Er, "per-particle energy")
        assert W.sum() == pytest.approx(Wr, rel=1e-12, abs=1e-12)
        if T is not None:
            check_fp64(T, Tr, "torque")
    else:
        check_mixed(F, Fr, "force")
        assert E.sum() == pytest.approx(Ur, rel=1e-5, abs=1e-5 * s.n)
        assert W.sum() == pytest.approx(Wr, rel=1e-5, abs=1e-5 * s.n)
        if T is not None:
            check_mixed(T, Tr, "torque")


@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("name", ["lj5003", "patchy6000"])
def test_edge_store_is_bitwise_reproducible(name, precision):
    s = get_sys(name)
    outs = []
    for _ in range(2):
        sim = _es_sim(s, precision)
        for _ in range(2):
            sim.forces_edge_store()
            outs.append(sim.forces())
    for o in outs[1:]:
        for x, y in zip(o, outs[0]):
            if x is not None:
                assert np.array_equal(x, y)


def test_edge_store_trajectory_is_bitwise_reproducible():
    """Mixed precision, 150 graph steps with rebuilds, twice from the same start: identical states."""
    s = get_sys("lj4000")
    res = []
    for _ in range(2):
        sim = Sim(s, B.MD_MIXED, edge_store=1, trace_capacity=16)
        sim.prepare(ES)
        sim.step(150, ES, use_graph=True)
        st = sim.status()
        assert st[B.MD_STATUS_CODE] == 0 and st[B.MD_STATUS_REBUILDS] >= 1
        res.append(sim.positions())
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_edge_store_path_needs_the_store():
    s = get_sys("lj4000")
    sim = Sim(s, B.MD_MIXED)
    with pytest.raises(B.MDError):
        sim.forces_edge_store()

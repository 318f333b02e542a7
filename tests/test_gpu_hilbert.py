"""Hilbert cell order (MD_ORDER_HILBERT): md_build_cells sorts particles by the Hilbert rank of their cell;
lists and forces are those of the row-major order, since only the particles' storage order changes."""
import numpy as np
import pytest

from paper_1401_4350_gb300 import binding as B
from tests.test_gpu_parity import Sim, check_fp64, check_mixed, get_sys, ref_forces

pytestmark = pytest.mark.gpu

H = B.MD_ORDER_HILBERT


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


@pytest.mark.parametrize("name", ["lj4000", "lj5003", "wca20000", "patchy6000"])
def test_hilbert_cells_order_particles_by_curve_rank(name):
    import torch
    s = get_sys(name)
    sim = Sim(s, B.MD_MIXED, cell_order=H)
    sim.build_cells()
    torch.cuda.synchronize()
    ids = sim.id.cpu().numpy()
    assert np.array_equal(np.sort(ids), np.arange(s.n))
    fx = sim.view("fxp", torch.int32, 4 * s.n).view(s.n, 4).cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    nc = np.array(sim.layout.ncell)
    cell = (fx[:, :3] * nc[None, :]) >> 32
    cid = (cell[:, 2] * nc[1] + cell[:, 1]) * nc[0] + cell[:, 0]
    rank = B.md_cell_order(sim.params)[cid]
    assert np.all(np.diff(rank) >= 0)
    # cell_start is indexed by the rank
    cs = sim.view("cell_start", torch.int32, int(np.prod(nc)) + 1).cpu().numpy()
    counts = np.bincount(rank, minlength=int(np.prod(nc)))
    assert np.array_equal(np.diff(cs), counts)


@pytest.mark.parametrize("name", ["lj4000", "wca20000", "patchy6000", "lj_tiny_box"])
def test_hilbert_lists_equal_row_major_lists(name):
    s = get_sys(name)
    out = []
    for order in (B.MD_ORDER_ROWS, H):
        sim = Sim(s, B.MD_MIXED, cell_order=order)
        sim.build_cells()
        sim.build_verlet(B.MD_LIST_BOTH)
        full, counts, _ = sim.full_list_pairs()
        half, ordered = sim.half_list_pairs()
        assert (counts == 2).all() and ordered
        out.append((full, half))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE, B.MD_VERTEX_NEWTON])
@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("name", ["lj5003", "patchy6000"])
def test_hilbert_forces_match_oracle(name, precision, path):
    s = get_sys(name)
    Fr, Tr, Er, (Ur, Wr, npair) = ref_forces(s, name)
    sim = Sim(s, precision, cell_order=H, force_copies=4)
    sim.prepare(path)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0, st
    F, E, T, W = sim.forces()
    if precision == B.MD_FP64:
        check_fp64(F, Fr, "force")
        if T is not None:
            check_fp64(T, Tr, "torque")
    else:
        check_mixed(F, Fr, "force")
        if T is not None:
            check_mixed(T, Tr, "torque")


def test_hilbert_steps_follow_row_major_steps():
    """200 FP64 steps (with rebuilds) in either order give the same trajectory up to the summation
    order of the forces."""
    s = get_sys("lj4000")
    a = Sim(s, B.MD_FP64, cell_order=H)
    b = Sim(s, B.MD_FP64)
    for sim in (a, b):
        sim.prepare(B.MD_VERTEX)
        sim.step(200, B.MD_VERTEX, use_graph=True)
    sa, sb = a.status(), b.status()
    assert sa[B.MD_STATUS_CODE] == 0 and sb[B.MD_STATUS_CODE] == 0
    assert sa[B.MD_STATUS_REBUILDS] == sb[B.MD_STATUS_REBUILDS] >= 1
    xa, va = a.positions()
    xb, vb = b.positions()
    d = xa - xb
    d -= s.box * np.rint(d / s.box)  # a particle on a box face may be wrapped on one side only
    assert np.abs(d).max() < 1e-9
    assert np.abs(va - vb).max() < 1e-8

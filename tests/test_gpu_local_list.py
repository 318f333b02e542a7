"""The block-local full list (16-bit halo positions, MD_LIST_FULL_LOCAL): with list_format =
MD_FORMAT_LOCAL, md_build_verlet(MD_LIST_FULL) chooses it for dense mixed-precision LJ/WCA with one thread
per particle.  Its rows name exactly the
pairs of the global list, in the same order, so the vertex forces are bit-identical to those from the
global format, and both match the oracle."""
import numpy as np
import pytest

from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems
from tests.test_gpu_parity import Sim, check_mixed, get_sys, ref_forces

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


def _wide_halo():
    """rv = 4.3: a block's halo (about 3500 slots) is too large to stage, exercising the table lookups."""
    s = systems.make_lj(20000, 0.85, 1.0, seed=61, rc=4.0)
    return s


CASES = {"lj4000": lambda: get_sys("lj4000"), "lj5003": lambda: get_sys("lj5003"),
         "lj65536": lambda: systems.make_lj(65536, 0.85, 1.0, seed=1001), "wide_halo": _wide_halo}
_c = {}


def case(name):
    if name not in _c:
        _c[name] = CASES[name]()
    return _c[name]


@pytest.mark.parametrize("order", [B.MD_ORDER_ROWS, B.MD_ORDER_HILBERT])
@pytest.mark.parametrize("name", sorted(CASES))
def test_local_rows_name_the_global_pairs(name, order):
    s = case(name)
    loc = Sim(s, B.MD_MIXED, cell_order=order, list_format=B.MD_FORMAT_LOCAL)
    loc.build_cells()
    loc.build_verlet(B.MD_LIST_FULL)
    st = loc.status()
    assert st[B.MD_STATUS_CODE] == 0, st
    assert st[B.MD_STATUS_LISTS] == B.MD_LIST_FULL | B.MD_LIST_FULL_LOCAL
    glob = Sim(s, B.MD_MIXED, cell_order=order, list_format=B.MD_FORMAT_LOCAL)
    glob.build_cells()
    glob.build_verlet(B.MD_LIST_BOTH)
    assert glob.status()[B.MD_STATUS_LISTS] == B.MD_LIST_BOTH
    p_loc, c_loc, e_loc = loc.local_list_pairs()
    p_glob, c_glob, e_glob = glob.full_list_pairs()
    assert np.array_equal(p_loc, p_glob) and (c_loc == 2).all() and e_loc == e_glob


@pytest.mark.parametrize("order", [B.MD_ORDER_ROWS, B.MD_ORDER_HILBERT])
@pytest.mark.parametrize("name", sorted(CASES))
def test_local_forces_equal_global_forces_bitwise(name, order):
    s = case(name)
    out = []
    for which in (B.MD_LIST_FULL, B.MD_LIST_BOTH):
        sim = Sim(s, B.MD_MIXED, cell_order=order, list_format=B.MD_FORMAT_LOCAL)
        sim.build_cells()
        sim.build_verlet(which)
        sim.forces_vertex()
        st = sim.status()
        assert st[B.MD_STATUS_CODE] == 0, st
        out.append(sim.forces())
    for x, y in zip(out[0], out[1]):
        if x is not None:
            assert np.array_equal(x, y)
    if name in ("lj4000", "lj5003"):
        Fr = ref_forces(s, name)[0]
        check_mixed(out[0][0], Fr, "force (local list)")


def test_other_kernels_refuse_the_local_list():
    s = case("lj4000")
    sim = Sim(s, B.MD_MIXED, list_format=B.MD_FORMAT_LOCAL)
    sim.build_cells()
    sim.build_verlet(B.MD_LIST_FULL)
    p = sim.params
    p.threads_per_particle = 2  # the local format is read by the one-thread-per-particle kernel only
    B.md_forces_vertex(p, sim.state(), sim.ws)
    assert sim.status()[B.MD_STATUS_CODE] == B.MD_ERR_INVALID


def test_global_format_is_the_default():
    s = case("lj4000")
    sim = Sim(s, B.MD_MIXED)
    sim.build_cells()
    sim.build_verlet(B.MD_LIST_FULL)
    assert sim.status()[B.MD_STATUS_LISTS] == B.MD_LIST_FULL

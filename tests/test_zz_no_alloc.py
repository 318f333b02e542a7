"""The cell build for callers that cannot allocate device memory (md_build_cells_static).

Such callers (code inside another framework's memory pool, plug-ins handed only their arrays,
programs that must not grow their device footprint) cannot pass the workspace md_build_cells takes
its scratch from.  md_build_cells_static takes the scratch from a static device array instead.  This
test calls it through the C ABI and checks that its results are bit-identical to md_build_cells on
the same input, on two calls in a row (the static array keeps the previous call's contents), and
that it rejects sizes beyond its limit.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()


def _static_build(s, precision, stream=None):
    """Runs md_build_cells_static twice on one copy of the state (on `stream`, default the current stream)
    and md_build_cells once on another, and checks that the results agree bit for bit, and that the
    second call changed the device's free memory by nothing (the first may load the library's device
    code, and with it the static array, into the context)."""
    import torch
    from paper_1401_4350_gb300.sim import Simulation
    ref = Simulation(s, precision)  # the ordinary entry point, with a workspace
    ref.build_cells()
    mine = Simulation(s, precision)  # only its state arrays are used below: same initial state
    ncell = int(np.prod(mine.layout.ncell))
    cell_start = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
    fxp = torch.zeros((s.n, 4), dtype=torch.int32, device="cuda")
    patch_lab = None
    if s.kind == systems.PATCHY:
        # FP64: double4 sites; mixed: int4 fixed-point sites, then the double4 block (12 words per site)
        rows = s.n if precision == B.MD_FP64 else 3 * s.n
        patch_lab = torch.zeros((rows, B.MD_MAX_PATCH, 8 if precision == B.MD_FP64 else 4),
                                dtype=torch.float32 if precision == B.MD_FP64 else torch.int32, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    B.md_build_cells_static(mine.params, mine.state(), cell_start, fxp, patch_lab, st)
    torch.cuda.synchronize()
    # a second call on the state the first one sorted: the build is deterministic and a sorted state
    # sorts to itself, so the result is the same; it must not allocate
    free0 = torch.cuda.mem_get_info()[0]
    B.md_build_cells_static(mine.params, mine.state(), cell_start, fxp, patch_lab, st)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(mine.pos, ref.pos) and torch.equal(mine.vel, ref.vel) and torch.equal(mine.id, ref.id)
    if s.kind == systems.PATCHY:
        assert torch.equal(mine.quat, ref.quat) and torch.equal(mine.angmom, ref.angmom)
        nb = patch_lab.numel() * patch_lab.element_size()
        assert torch.equal(patch_lab.view(torch.uint8).flatten(), ref.view("patch_lab", torch.uint8, nb))
    assert torch.equal(cell_start, ref.view("cell_start", torch.int32, ncell + 1))
    assert torch.equal(fxp.flatten(), ref.view("fxp", torch.int32, 4 * s.n))
    return ncell


@pytest.mark.parametrize("precision", [B.MD_MIXED, B.MD_FP64])
def test_static_cell_build_matches_workspace_build_twice(precision):
    # two calls in a row on different systems: the second must not see the first's leftovers
    _static_build(systems.make_lj(4000, 0.85, 1.0, seed=1000), precision)
    _static_build(systems.make_wca(3001, 0.2, seed=61), precision)


def test_static_cell_build_patchy():
    for prec in (B.MD_MIXED, B.MD_FP64):
        _static_build(systems.make_patchy(2500, 0.3, seed=62), prec)


def test_static_cell_build_at_its_limits_on_a_side_stream():
    """n = MD_STATIC_MAX_N in a gas so dilute that the cell grid is capped (4 n + 27 cells): the largest
    particle and cell counts the static array is sized for, on a stream other than the default one."""
    import torch
    s = systems.make_wca(B.MD_STATIC_MAX_N, 0.005, seed=64)
    side = torch.cuda.Stream()
    ncell = _static_build(s, B.MD_MIXED, stream=side)
    assert 2 * s.n < ncell <= 4 * s.n + 27


def test_static_cell_build_rejects_sizes_beyond_its_limit():
    import torch
    from paper_1401_4350_gb300.sim import make_params
    s = systems.make_lj(B.MD_STATIC_MAX_N + 4, 0.85, 1.0, seed=63)
    p = make_params(s, B.MD_MIXED)
    st = B.md_state()
    pos = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
    ids = torch.zeros(s.n, dtype=torch.int32, device="cuda")
    st.pos, st.vel, st.id = pos.data_ptr(), pos.data_ptr(), ids.data_ptr()
    cs = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(B.MDError) as err:
        B.md_build_cells_static(p, st, cs, pos)
    assert err.value.code == B.MD_ERR_INVALID and "MD_STATIC_MAX_N" in str(err.value)
    assert B.md_static_scratch_bytes() < 8 << 20

"""C ABI checks that need no GPU: the library loads, exports every function of include/md.h,
validates its arguments on the host and lays the workspace out consistently."""
import ctypes
import os

import numpy as np
import pytest

from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import build as mdbuild
from paper_1401_4350_gb300 import systems
from paper_1401_4350_gb300.sim import make_params


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        mdbuild.build()
    return B.load()


def test_exports_every_declared_function(lib):
    names = B.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    for required in ("md_build_cells", "md_build_verlet", "md_forces_vertex", "md_forces_edge", "md_step_verlet"):
        assert required in names


def test_abi_version(lib):
    assert B.md_abi_version() == 5


def _lj_params(n=4000, precision=B.MD_MIXED):
    return make_params(systems.make_lj(n, 0.85, seed=3), precision)


@pytest.mark.parametrize("field,value,needle", [
    ("n", 0, "n must be"),
    ("model", 7, "unknown model"),
    ("precision", 5, "unknown precision"),
    ("max_neigh", 0, "max_neigh"),
    ("max_pairs", 0, "max_pairs"),
    ("threads_per_particle", 3, "threads_per_particle"),
    ("block_size", 48, "block_size"),
    ("block_size", 512, "block_size"),
    ("skin", 0.0, "skin"),
    ("dt", -1.0, "dt"),
    ("energy_every", -2, "energy_every"),
    ("force_copies", -1, "force_copies"),
    ("force_copies", 65, "force_copies"),
    ("list_format", 2, "list_format"),
    ("fuse_step", 2, "fuse_step"),
    ("prune_skin", -0.1, "prune_skin"),
    ("prune_skin", 0.3, "prune_skin"),
    ("cell_order", 2, "cell_order"),
    ("thermostat_every", -1, "thermostat_every"),
])
def test_invalid_params_rejected(lib, field, value, needle):
    p = _lj_params()
    setattr(p, field, value)
    assert B.md_check_params(p) == B.MD_ERR_INVALID
    assert needle in B.last_error()
    assert B.md_workspace_bytes(p) == 0


def test_box_must_exceed_twice_rv(lib):
    p = _lj_params()
    p.box[1] = 5.5
    assert B.md_check_params(p) == B.MD_ERR_INVALID
    assert "minimum image" in B.last_error()


def test_patchy_needs_patches(lib):
    p = make_params(systems.make_patchy(500, 0.3, seed=4), B.MD_MIXED)
    assert B.md_check_params(p) == B.MD_OK
    p.n_patch = 0
    assert B.md_check_params(p) == B.MD_ERR_INVALID


@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("kind", ["lj", "wca", "patchy", "tiny"])
def test_workspace_layout(lib, precision, kind):
    if kind == "lj":
        s = systems.make_lj(4000, 0.85, seed=5)
    elif kind == "wca":
        s = systems.make_wca(3000, 0.2, seed=5)
    elif kind == "patchy":
        s = systems.make_patchy(2000, 0.3, seed=5)
    else:
        s = systems.make_lj(500, 0.9, seed=5)
    p = make_params(s, precision, trace_capacity=17)
    L = B.md_workspace_layout(p)
    assert L.total == B.md_workspace_bytes(p) > 0
    offs = [getattr(L, f) for f in ("status", "energy", "cell_start", "fxp", "fxp_build", "patch_lab", "nbr",
                                    "nbr_count", "half_start", "half_j", "force", "virial", "torque",
                                    "acc", "copies", "estore", "jstart", "jedge", "local_tab", "trace", "pos_alt",
                                    "fxp_alt", "nbr_in", "nbr_in_count", "fxp_prune", "scratch")]
    assert all(o % 256 == 0 for o in offs)
    assert offs == sorted(offs) and len(set(offs)) == len(offs)
    assert L.force_elem == 8
    n = s.n
    assert L.nbr_count - L.nbr >= 4 * n * p.max_neigh
    assert L.virial - L.force >= 32 * n
    # dense systems (>= 8 particles per rv^3): cells of edge >= rv/2, searched two cells deep, an axis with
    # fewer than five of them is one cell; sparse ones: cells of edge >= rv, fewer than three -> one cell
    dense = s.n / np.prod(s.box) * s.rv ** 3 >= 8.0
    for c in range(3):
        k = L.ncell[c]
        if dense:
            assert k == 1 or (k >= 5 and s.box[c] / k >= s.rv / 2)
        else:
            assert k == 1 or (k >= 3 and s.box[c] / k >= s.rv)
    if kind == "tiny":
        assert tuple(L.ncell) == (5, 5, 5)
        p.box[0] = 6.5  # > 2 rv, but fewer than five cells of rv/2: one cell along x
        assert B.md_workspace_layout(p).ncell[0] == 1
        p.list_format = B.MD_FORMAT_LOCAL  # the block-local format keeps cells of edge >= rv
        p.box[0] = s.box[0]
        L2 = B.md_workspace_layout(p)
        assert all(k == 1 or (k >= 3 and s.box[c] / k >= s.rv) for c, k in enumerate(L2.ncell))


def test_struct_layouts_match_c(lib, tmp_path):
    """ctypes mirrors of md_params, md_state and md_ws_layout have the C sizes and offsets."""
    import subprocess
    fields = {"md_params": [f[0] for f in B.md_params._fields_],
              "md_state": [f[0] for f in B.md_state._fields_],
              "md_ws_layout": [f[0] for f in B.md_ws_layout._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{B.HEADER}"', 'int main(void) {']
    for st, names in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for nm in names:
            lines.append(f'printf("{st}.{nm} %zu\\n", offsetof({st}, {nm}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-o", str(exe), str(src)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, cls in (("md_params", B.md_params), ("md_state", B.md_state), ("md_ws_layout", B.md_ws_layout)):
        assert int(out[st]) == ctypes.sizeof(cls), st
        for nm in fields[st]:
            assert int(out[f"{st}.{nm}"]) == getattr(cls, nm).offset, (st, nm)


@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
def test_fused_step_buffers(lib, precision):
    """fuse_step = 1 reserves the second position (double[n][4]) and fixed-point (uint32[n][4]) buffers;
    fuse_step = 0 leaves them empty; nothing else moves."""
    s = systems.make_lj(3000, 0.85, seed=5)
    p = make_params(s, precision)
    L0 = B.md_workspace_layout(p)
    assert L0.fxp_alt - L0.pos_alt <= 256 and L0.nbr_in - L0.fxp_alt <= 256
    p.fuse_step = 1
    L1 = B.md_workspace_layout(p)
    assert L1.fxp_alt - L1.pos_alt >= 32 * s.n and L1.nbr_in - L1.fxp_alt >= 16 * s.n
    assert L1.total - L0.total >= 48 * s.n - 512  # the empty regions held 256 bytes each
    for f in ("status", "fxp", "nbr", "force", "trace", "pos_alt"):
        assert getattr(L1, f) == getattr(L0, f)


def test_inner_list_regions(lib):
    """prune_skin > 0 with fused steps on the LJ/WCA mixed path in a cubic box reserves the inner list (as large
    as the Verlet list), its lengths and the prune coordinates; any other case leaves them empty."""
    s = systems.make_lj(3000, 0.85, seed=5)
    p = make_params(s, B.MD_MIXED, fuse_step=1, prune_skin=0.1)
    L = B.md_workspace_layout(p)
    n = s.n
    assert L.nbr_in_count - L.nbr_in >= 4 * n * p.max_neigh
    assert L.fxp_prune - L.nbr_in_count >= 4 * n and L.scratch - L.fxp_prune >= 16 * n
    for change in (dict(fuse_step=0), dict(prune_skin=0.0), dict(precision=B.MD_FP64)):
        q = make_params(s, change.get("precision", B.MD_MIXED), fuse_step=change.get("fuse_step", 1),
                        prune_skin=change.get("prune_skin", 0.1))
        M = B.md_workspace_layout(q)
        assert M.nbr_in_count - M.nbr_in <= 256 and M.scratch - M.fxp_prune <= 256, change
    p.box[2] = p.box[2] * 1.1  # a non-cubic box has no inner list
    M = B.md_workspace_layout(p)
    assert M.nbr_in_count - M.nbr_in <= 256


@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("kind", ["lj", "patchy"])
def test_newton_copies_region(lib, precision, kind):
    """force_copies = m reserves m reaction copies per particle (layout documented in md.h)."""
    s = systems.make_lj(4000, 0.85, seed=5) if kind == "lj" else systems.make_patchy(2000, 0.3, seed=5)
    p = make_params(s, precision)
    L0 = B.md_workspace_layout(p)
    assert L0.estore - L0.copies <= 256  # no copies without force_copies
    p.force_copies = 16
    L = B.md_workspace_layout(p)
    per = (16 * (4 if kind == "patchy" else 2)) if precision == B.MD_MIXED else (32 + 8 + (32 if kind == "patchy" else 0))
    assert L.estore - L.copies >= 16 * s.n * per
    assert L.total - L0.total >= 16 * s.n * per - 256


def test_newton_path_needs_copies(lib):
    """The Newton path is refused on the host when the workspace has no force copies."""
    p = _lj_params()
    fake = 1 << 20  # aligned non-null addresses: validation fails before any device access
    st = B.md_state(fake, fake, 0, 0, fake)
    assert B.load().md_forces_vertex_newton(ctypes.byref(p), ctypes.byref(st), ctypes.c_void_p(fake), None) == B.MD_ERR_INVALID
    assert "force_copies" in B.last_error()
    assert B.load().md_prepare(ctypes.byref(p), ctypes.byref(st), ctypes.c_void_p(fake), 2, None) == B.MD_ERR_INVALID
    assert B.load().md_prepare(ctypes.byref(p), ctypes.byref(st), ctypes.c_void_p(fake), 3, None) == B.MD_ERR_INVALID
    assert "edge_store" in B.last_error()
    assert B.load().md_forces_edge_store(ctypes.byref(p), ctypes.byref(st), ctypes.c_void_p(fake), None) == B.MD_ERR_INVALID
    assert B.load().md_prepare(ctypes.byref(p), ctypes.byref(st), ctypes.c_void_p(fake), 4, None) == B.MD_ERR_INVALID
    assert "path must be" in B.last_error()


def test_step_verlet_host_validation(lib):
    """md_step_verlet_host refuses on the host, before any copy: missing host arrays, patchy models, bad
    paths and step counts."""
    fake = 1 << 20
    st = B.md_state(fake, fake, 0, 0, fake)
    f = B.load().md_step_verlet_host
    p = _lj_params()
    h = ctypes.c_void_p(1 << 21)
    args = lambda hp, hv, nsteps=1, path=B.MD_VERTEX: (ctypes.byref(p), ctypes.byref(st), ctypes.c_void_p(fake), hp, hv,
                                                       None, nsteps, path, 1, None)
    assert f(*args(None, h)) == B.MD_ERR_INVALID and "host_pos" in B.last_error()
    assert f(*args(h, None)) == B.MD_ERR_INVALID and "host_vel" in B.last_error()
    assert f(*args(h, h, nsteps=-1)) == B.MD_ERR_INVALID and "nsteps" in B.last_error()
    assert f(*args(h, h, path=9)) == B.MD_ERR_INVALID and "path" in B.last_error()
    p = make_params(systems.make_patchy(2000, 0.3, seed=3), B.MD_MIXED)
    st = B.md_state(fake, fake, fake, fake, fake)
    assert f(*args(h, h)) == B.MD_ERR_INVALID and "isotropic" in B.last_error()


def _grid_params(ncell):
    p = _lj_params(500)
    p.n = 2000000  # the grid is capped at 4 n + 27 cells; no memory is allocated here
    rv = p.rc + p.skin
    for c in range(3):
        p.box[c] = (ncell[c] + 0.5) * rv / 2  # cells of edge >= rv/2
    p.cell_order = B.MD_ORDER_HILBERT
    return p


@pytest.mark.parametrize("k", [3, 4, 5])
def test_hilbert_cell_order_is_a_continuous_curve_on_power_of_two_grids(lib, k):
    """On a 2^k cube the Hilbert curve visits every cell once, starts in the corner cell, and steps to a
    face neighbour each time (the defining property of the curve)."""
    n = 2 ** k
    p = _grid_params((n, n, n))
    L = B.md_workspace_layout(p)
    assert tuple(L.ncell) == (n, n, n)
    rank = B.md_cell_order(p)
    assert np.array_equal(np.sort(rank), np.arange(n ** 3))
    order = np.argsort(rank)
    xyz = np.stack([order % n, (order // n) % n, order // (n * n)], 1)
    assert tuple(xyz[0]) == (0, 0, 0)
    steps = np.abs(np.diff(xyz, axis=0)).sum(1)
    assert (steps == 1).all()


@pytest.mark.parametrize("ncell", [(5, 5, 5), (5, 7, 6), (76, 76, 76), (13, 5, 9)])
def test_hilbert_cell_order_is_a_local_permutation(lib, ncell):
    """Any grid: a permutation of the cells whose consecutive cells are close (the curve through the
    enclosing 2^b cube skips the missing cells); row-major order is the identity."""
    p = _grid_params(ncell)
    L = B.md_workspace_layout(p)
    assert tuple(L.ncell) == ncell
    rank = B.md_cell_order(p)
    total = int(np.prod(ncell))
    assert np.array_equal(np.sort(rank), np.arange(total))
    order = np.argsort(rank)
    nx, ny, nz = ncell
    xyz = np.stack([order % nx, (order // nx) % ny, order // (nx * ny)], 1)
    steps = np.abs(np.diff(xyz, axis=0)).sum(1)
    assert steps.mean() < 1.6
    p.cell_order = B.MD_ORDER_ROWS
    assert np.array_equal(B.md_cell_order(p), np.arange(total))


@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("kind", ["lj", "patchy"])
def test_edge_store_regions(lib, precision, kind):
    """edge_store = 1 reserves the A, B (and, patchy, C) blocks of max_pairs entries and the by-partner
    index; without it the regions are empty."""
    s = systems.make_lj(4000, 0.85, seed=5) if kind == "lj" else systems.make_patchy(2000, 0.3, seed=5)
    p = make_params(s, precision)
    L0 = B.md_workspace_layout(p)
    assert L0.jedge - L0.estore <= 512
    p.edge_store = 1
    L = B.md_workspace_layout(p)
    elem = 16 if precision == B.MD_MIXED else 32
    blocks = 3 if kind == "patchy" else 2
    assert L.jstart - L.estore >= elem * blocks * p.max_pairs
    assert L.jedge - L.jstart >= 8 * (s.n + 1)
    assert L.local_tab - L.jedge >= 4 * p.max_pairs
    p.edge_store = 2
    assert B.md_check_params(p) == B.MD_ERR_INVALID
    p.edge_store = 1
    p.max_pairs = 1 << 31
    assert B.md_check_params(p) == B.MD_ERR_INVALID

"""C ABI checks that need no GPU: the library loads, exports every function of include/md.h,
validates its arguments on the host and lays the workspace out consistently."""
import ctypes
import os

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
    assert B.md_abi_version() == 1


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
    ("reserved", 1, "reserved"),
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
                                    "nbr_count", "half_start", "pairs", "force", "virial", "torque",
                                    "acc", "trace", "scratch")]
    assert all(o % 256 == 0 for o in offs)
    assert offs == sorted(offs) and len(set(offs)) == len(offs)
    assert L.force_elem == 8
    n = s.n
    assert L.nbr_count - L.nbr >= 4 * n * p.max_neigh
    assert L.virial - L.force >= 32 * n
    # cells of edge >= rv; an axis with fewer than three such cells is a single cell
    for c in range(3):
        k = L.ncell[c]
        assert k == 1 or (k >= 3 and s.box[c] / k >= s.rv)
    if kind == "tiny":
        assert tuple(L.ncell) == (1, 1, 1)


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

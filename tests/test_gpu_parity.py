"""GPU parity of libmdgb against the FP64 oracle (called through the C ABI).

Tolerances (written here):
  * pair sets: bit-exact as sorted sets of original-id pairs;
  * MD_FP64 forces, torques and per-particle energies: |x - x_ref| <= 1e-12 max(|x_ref|, x_rms) per
    component (summation order differs: edge atomics, vertex list order);
  * MD_MIXED: max |F - F_ref| <= 1e-5 F_rms; for torques the same against the rms torque over all
    particles.
"""
import numpy as np
import pytest

import oracle
from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems

pytestmark = pytest.mark.gpu

FP64_REL = 1e-12
MIXED_REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


def Sim(*a, **k):
    from paper_1401_4350_gb300.sim import Simulation
    return Simulation(*a, **k)


def model_of(s):
    return oracle.Model(s.kind, tuple(s.box), s.rc, eps=s.eps, sigma=s.sigma, eps_p=s.eps_p, delta=s.delta,
                        patches=s.patches, patch_rc=s.patch_rc)


_cache = {}


def ref_forces(s, key):
    if key not in _cache:
        _cache[key] = oracle.forces(s.pos, model_of(s), quat=s.quat, use_cells=s.n > 4000)
    return _cache[key]


def _patchy_dimer_system(n_dimers=150, box=20.0, seed=8):
    from tests.test_oracle import _patchy_dimers
    rng = np.random.default_rng(seed)
    pos, quat = _patchy_dimers(n_dimers, np.array([box] * 3), rng)
    n = len(pos)
    return systems.System(systems.PATCHY, pos, rng.normal(0, 0.3, (n, 3)), np.array([box] * 3), 1.5, 0.2, 0.001,
                          0.15, quat=quat, angmom=rng.normal(0, 0.1, (n, 3)), patches=systems.PATCH_DIRS * 0.5,
                          name="patchy_dimers")


SYSTEMS = {
    "lj4000": lambda: systems.make_lj(4000, 0.85, 1.0, seed=1000),
    "lj5003": lambda: systems.make_lj(5003, 0.85, 1.0, seed=7),
    "wca20000": lambda: systems.make_wca(20000, 0.2, seed=1002),
    "patchy6000": lambda: systems.make_patchy(6000, 0.3, seed=1003),
    "patchy_dimers": _patchy_dimer_system,
    "lj_tiny_box": lambda: systems.make_lj(500, 0.9, 1.0, seed=9),
}
_sys = {}


def get_sys(name):
    if name not in _sys:
        _sys[name] = SYSTEMS[name]()
    return _sys[name]


def check_fp64(x, ref, what):
    rms = np.sqrt((ref ** 2).sum(axis=-1).mean()) if ref.ndim > 1 else np.sqrt((ref ** 2).mean())
    tol = FP64_REL * np.maximum(np.abs(ref), rms)
    err = np.abs(x - ref)
    worst = float((err / np.maximum(np.abs(ref), rms)).max()) if rms > 0 else float(err.max())
    assert (err <= tol + 1e-300).all(), f"{what}: worst relative error {worst:.3e} > {FP64_REL}"


def check_mixed(x, ref, what):
    """max |x - ref| <= 1e-5 x_rms, the rms taken over all particles (for torques too: in a sparsely bonded
    patchy system most torques are zero, which makes this the strict form of the gate)."""
    mag2 = (ref ** 2).sum(axis=-1)
    rms = np.sqrt(mag2.mean())
    err = float(np.abs(x - ref).max())
    assert err <= MIXED_REL * rms, f"{what}: max error {err:.3e} = {err / rms:.3e} of rms > {MIXED_REL}"


def run_forces(s, precision, path, tpp=1, block=0):
    sim = Sim(s, precision, tpp=tpp, block=block, force_copies=2 if path == B.MD_VERTEX_NEWTON else 0,
              edge_store=1 if path == B.MD_EDGE_STORE else 0)
    sim.build_cells()
    sim.build_verlet(B.MD_LIST_NEWTON if path == B.MD_VERTEX_NEWTON else B.MD_LIST_BOTH)
    {B.MD_VERTEX: sim.forces_vertex, B.MD_EDGE: sim.forces_edge, B.MD_VERTEX_NEWTON: sim.forces_vertex_newton,
     B.MD_EDGE_STORE: sim.forces_edge_store}[path]()
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0, st
    return sim, sim.forces()


# ------------------------------------------------------------------------------------------------
# Cells and Verlet lists
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["lj4000", "lj5003", "wca20000", "patchy6000", "lj_tiny_box"])
def test_cell_sort_is_a_cell_ordered_permutation(name):
    import torch
    s = get_sys(name)
    sim = Sim(s, B.MD_MIXED)
    sim.build_cells()
    torch.cuda.synchronize()
    ids = sim.id.cpu().numpy()
    assert np.array_equal(np.sort(ids), np.arange(s.n))
    # in-box positions are moved, not changed
    assert np.array_equal(sim.pos[:, :3].cpu().numpy(), s.pos[ids])
    fx = sim.view("fxp", torch.int32, 4 * s.n).view(s.n, 4).cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    nc = np.array(sim.layout.ncell)
    cell = (fx[:, :3] * nc[None, :]) >> 32
    cid = (cell[:, 2] * nc[1] + cell[:, 1]) * nc[0] + cell[:, 0]
    assert np.all(np.diff(cid) >= 0)
    ncell = int(np.prod(nc))
    cs = sim.view("cell_start", torch.int32, ncell + 1).cpu().numpy()
    assert cs[0] == 0 and cs[-1] == s.n and np.all(np.diff(cs) >= 0)
    assert np.array_equal(np.bincount(cid, minlength=ncell), np.diff(cs))
    # within a cell: increasing original index on the first build
    for c in np.unique(cid)[:200]:
        seg = ids[cs[c]:cs[c + 1]]
        assert np.all(np.diff(seg) > 0)
    # fixed-point coordinates are the positions as fractions of the box
    x = fx[:, :3] / 2.0 ** 32 * s.box[None, :]
    d = x - s.pos[ids]
    d -= s.box * np.rint(d / s.box)
    assert np.abs(d).max() <= 1.01 * s.box.max() / 2 ** 32


@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("name", ["lj4000", "lj5003", "wca20000", "patchy6000", "lj_tiny_box"])
def test_verlet_pair_sets_bit_exact(name, precision):
    s = get_sys(name)
    sim = Sim(s, precision)
    sim.build_cells()
    sim.build_verlet(B.MD_LIST_BOTH)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0
    ref = oracle.pairs(s.pos, s.box, s.rv, use_cells=True)
    full, counts, nent = sim.full_list_pairs()
    assert np.array_equal(full, ref)
    assert np.all(counts == 2) and nent == 2 * len(ref)
    half, ordered = sim.half_list_pairs()
    assert ordered
    assert np.array_equal(half, ref)
    assert st[B.MD_STATUS_NEED_NEIGH] == np.bincount(ref.ravel(), minlength=s.n).max()
    assert st[B.MD_STATUS_NEED_PAIRS_LO] + (st[B.MD_STATUS_NEED_PAIRS_HI] << 31) == len(ref)


def test_neighbour_overflow_is_reported():
    s = get_sys("lj4000")
    sim = Sim(s, B.MD_MIXED, max_neigh=16, max_pairs=1000)
    sim.build_cells()
    sim.build_verlet(B.MD_LIST_BOTH)
    st = sim.status()
    ref = oracle.pairs(s.pos, s.box, s.rv, use_cells=True)
    assert st[B.MD_STATUS_CODE] == B.MD_ERR_NEIGH_OVERFLOW
    assert st[B.MD_STATUS_NEED_NEIGH] == np.bincount(ref.ravel(), minlength=s.n).max()
    assert st[B.MD_STATUS_NEED_PAIRS_LO] == len(ref)


# ------------------------------------------------------------------------------------------------
# Forces
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
@pytest.mark.parametrize("name", ["lj4000", "lj5003", "wca20000", "patchy6000", "patchy_dimers", "lj_tiny_box"])
def test_forces_fp64_match_oracle(name, path):
    s = get_sys(name)
    Fr, Tr, Er, (Ur, Wr, npair) = ref_forces(s, name)
    sim, (F, E, T, W) = run_forces(s, B.MD_FP64, path)
    check_fp64(F, Fr, "force")
    check_fp64(E, Er, "per-particle energy")
    assert E.sum() == pytest.approx(Ur, rel=1e-12, abs=1e-12)
    assert W.sum() == pytest.approx(Wr, rel=1e-12, abs=1e-12)
    if s.kind == systems.PATCHY:
        check_fp64(T, Tr, "torque")


@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
@pytest.mark.parametrize("name", ["lj4000", "lj5003", "wca20000", "patchy6000", "patchy_dimers", "lj_tiny_box"])
def test_forces_mixed_match_oracle(name, path):
    s = get_sys(name)
    Fr, Tr, Er, (Ur, Wr, npair) = ref_forces(s, name)
    sim, (F, E, T, W) = run_forces(s, B.MD_MIXED, path)
    check_mixed(F, Fr, "force")
    assert E.sum() == pytest.approx(Ur, rel=1e-5, abs=1e-5 * s.n)
    assert W.sum() == pytest.approx(Wr, rel=1e-5, abs=1e-5 * s.n)
    if s.kind == systems.PATCHY:
        check_mixed(T, Tr, "torque")


@pytest.mark.parametrize("tpp", [2, 4, 8])
@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
def test_threads_per_particle(tpp, precision):
    s = get_sys("lj5003")
    Fr, _, Er, _ = ref_forces(s, "lj5003")
    _, (F, E, _, _) = run_forces(s, precision, B.MD_VERTEX, tpp=tpp)
    (check_fp64 if precision == B.MD_FP64 else check_mixed)(F, Fr, f"force tpp={tpp}")


@pytest.mark.parametrize("tpp", [1, 4])
def test_threads_per_particle_patchy(tpp):
    s = get_sys("patchy_dimers")
    Fr, Tr, _, _ = ref_forces(s, "patchy_dimers")
    _, (F, E, T, _) = run_forces(s, B.MD_MIXED, B.MD_VERTEX, tpp=tpp)
    check_mixed(F, Fr, "force")
    check_mixed(T, Tr, "torque")


@pytest.mark.parametrize("block", [32, 64, 256])
@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
def test_block_sizes(block, path):
    s = get_sys("lj4000")
    Fr, _, _, _ = ref_forces(s, "lj4000")
    _, (F, _, _, _) = run_forces(s, B.MD_MIXED, path, block=block)
    check_mixed(F, Fr, f"force block={block}")


@pytest.mark.parametrize("n", [1, 2, 3, 33])
@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE, B.MD_VERTEX_NEWTON, B.MD_EDGE_STORE])
def test_tiny_systems(n, path):
    rng = np.random.default_rng(n)
    box = np.array([9.0, 9.5, 10.0])
    if n == 2:
        pos = np.array([[1.0, 1.0, 1.0], [2.1, 1.2, 0.9]])
    else:
        pos = rng.uniform(0, 1, (n, 3)) * box
    s = systems.System(systems.LJ, pos, np.zeros((n, 3)), box, 2.5, 0.3, 0.001, 1.0, name=f"tiny{n}")
    Fr, _, Er, (Ur, _, _) = oracle.forces(pos, model_of(s), use_cells=False)
    for precision in (B.MD_FP64, B.MD_MIXED):
        _, (F, E, _, _) = run_forces(s, precision, path)
        if n == 1:
            assert np.all(F == 0) and np.all(E == 0)
        elif precision == B.MD_FP64:
            check_fp64(F, Fr, "force")
        else:
            assert np.abs(F - Fr).max() <= 1e-5 * max(1.0, np.sqrt((Fr ** 2).sum(1).mean()))


# ------------------------------------------------------------------------------------------------
# Velocity Verlet
# ------------------------------------------------------------------------------------------------

def _min_image_err(a, b, box):
    d = a - b
    d -= box * np.rint(d / box)
    return np.abs(d).max()


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
def test_fp64_trajectory_follows_oracle(path, use_graph):
    """LJ N=4000 (the oracle-sized case): 100 FP64 steps stay on the oracle trajectory."""
    s = get_sys("lj4000")
    steps = 100
    p_ref, v_ref, _, _, tr = oracle.run_nve(s.pos, s.vel, model_of(s), s.dt, steps, use_cells=True)
    sim = Sim(s, B.MD_FP64, trace_capacity=steps + 1)
    sim.prepare(path)
    sim.step(steps, path, use_graph)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0 and st[B.MD_STATUS_STEPS] == steps
    pos, vel = sim.positions()
    assert _min_image_err(pos, p_ref, s.box) < 1e-10
    assert np.abs(vel - v_ref).max() < 1e-9
    t = sim.trace()
    assert np.array_equal(t[:, 0], np.arange(steps + 1))
    e_gpu = t[:, 1] + t[:, 2]
    e_ref = tr[:, 0] + tr[:, 1] + tr[:, 2]
    assert np.abs(e_gpu - e_ref).max() < 1e-8 * s.n
    assert np.abs(t[:, 3] - tr[:, 3]).max() < 1e-8 * s.n


@pytest.mark.parametrize("name", ["patchy_dimers"])
@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
def test_fp64_rigid_body_trajectory_follows_oracle(name, path):
    s = get_sys(name)
    steps = 100
    p_ref, v_ref, q_ref, L_ref, tr = oracle.run_nve(s.pos, s.vel, model_of(s), s.dt, steps, quat=s.quat,
                                                    angmom=s.angmom, inertia=s.inertia, use_cells=False)
    sim = Sim(s, B.MD_FP64, trace_capacity=steps + 1)
    sim.prepare(path)
    sim.step(steps, path, True)
    assert sim.status()[B.MD_STATUS_CODE] == 0
    pos, vel = sim.positions()
    q, L = sim.orientations()
    assert _min_image_err(pos, p_ref, s.box) < 1e-10
    assert np.abs(vel - v_ref).max() < 1e-9
    assert np.abs(q - q_ref).max() < 1e-9
    assert np.abs(L - L_ref).max() < 1e-9


@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
def test_mixed_trajectory_close_to_oracle(path):
    s = get_sys("lj4000")
    steps = 100
    p_ref, v_ref, _, _, tr = oracle.run_nve(s.pos, s.vel, model_of(s), s.dt, steps, use_cells=True)
    sim = Sim(s, B.MD_MIXED, trace_capacity=steps + 1)
    sim.prepare(path)
    sim.step(steps, path, True)
    assert sim.status()[B.MD_STATUS_CODE] == 0
    pos, vel = sim.positions()
    assert _min_image_err(pos, p_ref, s.box) < 1e-6
    t = sim.trace()
    e_gpu = t[:, 1] + t[:, 2]
    e_ref = tr[:, 0] + tr[:, 1] + tr[:, 2]
    assert np.abs(e_gpu - e_ref).max() / s.n < 1e-5


def test_graph_and_direct_launches_agree_bitwise():
    s = get_sys("lj4000")
    out = []
    for use_graph in (True, False):
        sim = Sim(s, B.MD_MIXED)
        sim.prepare(B.MD_VERTEX)
        sim.step(60, B.MD_VERTEX, use_graph)
        out.append(sim.positions()[0])
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("precision", [B.MD_MIXED, B.MD_FP64])
@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
def test_lists_stay_valid_across_rebuilds(precision, path):
    """Run long enough for several displacement-triggered rebuilds, then check the forces at the
    GPU's own final positions against the oracle (a list missing a pair would show here)."""
    s = systems.make_lj(6000, 0.85, 2.0, seed=44)
    steps = 300 if precision == B.MD_MIXED else 120
    sim = Sim(s, precision)
    sim.prepare(path)
    sim.step(steps, path, True)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0 and st[B.MD_STATUS_REBUILDS] >= 1, st
    pos, _ = sim.positions()
    F, E, _, _ = sim.forces()
    Fr, _, _, _ = oracle.forces(np.mod(pos, s.box), model_of(s), use_cells=True)
    (check_fp64 if precision == B.MD_FP64 else check_mixed)(F, Fr, "force after rebuilds")


@pytest.mark.parametrize("precision", [B.MD_FP64, B.MD_MIXED])
@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
@pytest.mark.parametrize("box_shape", ["cubic", "noncubic"])
def test_pairs_at_the_cutoff_follow_the_exact_decision(precision, path, box_shape):
    """Dimers straddling rc = 2.5 sigma by a few 1e-7 relative: the LJ force jumps by F(rc) ~ 0.039 there,
    so any pair decided on the other side than the FP64 definition would show as an error of that size."""
    rng = np.random.default_rng(77)
    box = np.array([24.0, 24.0, 24.0]) if box_shape == "cubic" else np.array([24.0, 26.5, 29.0])
    rel = [-3e-6, -4e-7, -1e-7, -1e-8, 1e-8, 1e-7, 4e-7, 3e-6]
    pos = []
    grid = [(x, y, z) for x in range(2) for y in range(2) for z in range(2)]
    for k, d in enumerate(rel):
        c = (np.array(grid[k]) + 0.25) * box / 2
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        r = 2.5 * (1 + d)
        pos += [c, c + r * u]
    pos = np.mod(np.array(pos), box)
    s = systems.System(systems.LJ, pos, np.zeros_like(pos), box, 2.5, 0.3, 0.001, 1.0, name="cutoff_band")
    Fr, _, Er, (Ur, _, npair) = oracle.forces(pos, model_of(s), use_cells=False)
    assert 0 < npair < len(rel)
    _, (F, E, _, _) = run_forces(s, precision, path)
    fmag = 0.039
    tol = (1e-12 if precision == B.MD_FP64 else 1e-5) * fmag
    assert np.abs(F - Fr).max() <= tol, np.abs(F - Fr).max()


def test_energy_every_keeps_dynamics_and_reports_the_same_energies():
    s = get_sys("lj4000")
    out = []
    for every in (1, 5):
        sim = Sim(s, B.MD_MIXED, trace_capacity=32, energy_every=every)
        sim.prepare(B.MD_VERTEX)
        sim.step(20, B.MD_VERTEX, True)
        assert sim.status()[B.MD_STATUS_STEPS] == 20
        out.append((sim.positions()[0], sim.trace()))
    assert np.array_equal(out[0][0], out[1][0])  # energies do not feed back into the dynamics
    t1, t5 = out[0][1], out[1][1]
    for step in (5, 10, 15, 20):
        assert t5[step, 0] == step
        np.testing.assert_array_equal(t5[step], t1[step])
    assert t5[7, 0] == 0.0  # not an energy step: the row was never written


@pytest.mark.parametrize("tpp", [1, 2, 4, 8])
def test_cutoff_band_fixup_with_threads_per_particle(tpp):
    """A random (not lattice) LJ configuration has pairs within the 1e-5 band around rc^2 for tens of
    particles; with several threads per particle each lane must correct exactly its own entries."""
    s = systems.make_wca(40000, 0.42, seed=88)
    s = systems.System(systems.LJ, s.pos, s.vel, s.box, 2.5, 0.3, 0.001, 1.0, name="lj_random_0.42")
    Fr, _, _, _ = oracle.forces(s.pos, model_of(s), use_cells=True)
    outer = len(oracle.pairs(s.pos, s.box, 2.5 * np.sqrt(1 + 1e-5), use_cells=True))
    inner = len(oracle.pairs(s.pos, s.box, 2.5 * np.sqrt(1 - 1e-5), use_cells=True))
    assert outer - inner >= 5  # the configuration does exercise the band
    _, (F, _, _, _) = run_forces(s, B.MD_MIXED, B.MD_VERTEX, tpp=tpp)
    check_mixed(F, Fr, f"force tpp={tpp}")


_liquid = {}


def _bonded_patchy_liquid():
    """patchy6000 after 1000 steps at kT = 0.15 (mixed edge path): patches have bonded and pressed cores
    together, so the largest forces are many times the rms force, the hardest state for the mixed gate."""
    if "patchy" not in _liquid:
        import dataclasses
        s = get_sys("patchy6000")
        sim = Sim(s, B.MD_MIXED, fuse_step=0)
        sim.prepare(B.MD_EDGE)
        sim.step(1000, B.MD_EDGE, True)
        assert sim.status()[B.MD_STATUS_CODE] == 0
        x, v = sim.positions()
        q, l = sim.orientations()
        liq = dataclasses.replace(s, pos=np.mod(x, s.box), vel=v, quat=q, angmom=l, name="patchy6000_liquid")
        _liquid["patchy"] = (liq, oracle.forces(liq.pos, model_of(liq), quat=liq.quat, use_cells=True))
    return _liquid["patchy"]


@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE])
def test_patchy_bonded_liquid_mixed_matches_oracle(path):
    s, (Fr, Tr, Er, (Ur, Wr, _)) = _bonded_patchy_liquid()
    fr2 = (Fr ** 2).sum(1)
    assert np.sqrt(fr2.max() / fr2.mean()) > 5  # the heavy tail this test is about
    _, (F, E, T, W) = run_forces(s, B.MD_MIXED, path)
    check_mixed(F, Fr, "force (bonded liquid)")
    check_mixed(T, Tr, "torque (bonded liquid)")
    assert E.sum() == pytest.approx(Ur, rel=1e-5, abs=1e-5 * s.n)


def _wca_gas_after_collisions():
    """wca20000 after 1000 steps (fused mixed vertex path): collisions at r ~ 0.85-0.9 sigma give forces
    many times the rms force, which is what the accurate repulsive core is for."""
    if "wca" not in _liquid:
        import dataclasses
        s = get_sys("wca20000")
        sim = Sim(s, B.MD_MIXED, fuse_step=1)
        sim.prepare(B.MD_VERTEX)
        sim.step(1000, B.MD_VERTEX, True)
        assert sim.status()[B.MD_STATUS_CODE] == 0
        x, v = sim.positions()
        liq = dataclasses.replace(s, pos=np.mod(x, s.box), vel=v, name="wca20000_liquid")
        _liquid["wca"] = (liq, oracle.forces(liq.pos, model_of(liq), use_cells=True))
    return _liquid["wca"]


@pytest.mark.parametrize("path", [B.MD_VERTEX, B.MD_EDGE, B.MD_VERTEX_NEWTON, B.MD_EDGE_STORE])
def test_wca_gas_mixed_matches_oracle(path):
    s, (Fr, _, Er, (Ur, Wr, _)) = _wca_gas_after_collisions()
    fr2 = (Fr ** 2).sum(1)
    assert np.sqrt(fr2.max() / fr2.mean()) > 5  # the heavy tail this test is about
    _, (F, E, _, W) = run_forces(s, B.MD_MIXED, path)
    check_mixed(F, Fr, "force (WCA gas)")
    assert E.sum() == pytest.approx(Ur, rel=1e-5, abs=1e-5 * s.n)
    assert W.sum() == pytest.approx(Wr, rel=1e-5, abs=1e-5 * s.n)


def test_wca_gas_fused_step_forces_match_oracle():
    """The fused step kernel's own forces (the last launch of a call) on the WCA gas."""
    s, _ = _wca_gas_after_collisions()
    sim = Sim(s, B.MD_MIXED, fuse_step=1)
    sim.prepare(B.MD_VERTEX)
    sim.step(20, B.MD_VERTEX, True)
    x, _ = sim.positions()
    F, _, _, _ = sim.forces()
    Fr, _, _, _ = oracle.forces(np.mod(x, s.box), model_of(s), use_cells=True)
    check_mixed(F, Fr, "force (WCA gas, fused step)")

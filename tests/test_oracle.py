"""Pins of the FP64 oracle against facts fixed by the paper's definitions and by mathematics.

Nothing here compares the oracle with itself: each test checks a closed form, a
symmetry or conservation law, a finite-difference derivative, or an independent
brute force, chosen so that a dropped term, a wrong sign, a wrong index, a
transposed rotation or a wrong quaternion product order fails at least one test.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1401_4350_gb300 import systems

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lj_model(box, rc=2.5):
    return oracle.Model(oracle.LJ, tuple(box), rc)


def wca_model(box):
    return oracle.Model(oracle.WCA, tuple(box), 2.0 ** (1.0 / 6.0))


def patchy_model(box):
    return oracle.Model(oracle.PATCHY, tuple(box), 1.5, eps_p=1.0, delta=0.12,
                        patches=systems.PATCH_DIRS * systems.PATCH_RADIUS)


def quat_rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def axis_angle_quat(axis, angle):
    axis = np.asarray(axis, dtype=float)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[np.cos(angle / 2)], np.sin(angle / 2) * axis])


def qmul(a, b):
    w1, v1 = a[0], a[1:]
    w2, v2 = b[0], b[1:]
    return np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])


# --------------------------------------------------------------------------------------
# Dimer closed forms (Sec. Models, Eq. 1)
# --------------------------------------------------------------------------------------

def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "lj_dimer.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, r, e, fmag, sgn = line.split()
                rows.append((k, float(r), float(e), float(fmag), int(sgn)))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_dimer_golden(row):
    kind, r, e_ref, f_ref, sgn = row
    box = (12.0, 12.5, 13.0)
    m = lj_model(box) if kind == "LJ" else wca_model(box)
    rng = np.random.default_rng(7)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    x0 = np.array([11.5, 0.3, 6.0])  # near a face: the pair crosses the periodic boundary
    pos = np.stack([x0, np.mod(x0 + r * u, box)])
    F, T, E, (U, W, npair) = oracle.forces(pos, m, use_cells=False)
    assert U == pytest.approx(e_ref, abs=1e-11)
    assert E[0] == pytest.approx(0.5 * e_ref, abs=1e-11) and E[1] == pytest.approx(0.5 * e_ref, abs=1e-11)
    assert np.linalg.norm(F[0]) == pytest.approx(f_ref, abs=1e-9)
    np.testing.assert_allclose(F[0], -F[1], atol=1e-15)
    proj = F[0] @ u  # component of the force on particle 0 along the 0 -> 1 direction
    if sgn > 0:
        assert proj < 0 and np.allclose(F[0], proj * u, atol=1e-12)
    elif sgn < 0:
        assert proj > 0
    # virial of one pair: r . F_01 with r = x_0 - x_1
    assert W == pytest.approx(-(r * u) @ F[0], rel=1e-12, abs=1e-12)


def test_lj_energy_continuous_at_cutoff():
    box = (12.0, 12.0, 12.0)
    m = lj_model(box)
    for r in (2.5 - 1e-9, 2.5 + 1e-9):
        pos = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        _, _, _, (U, _, _) = oracle.forces(pos, m, use_cells=False)
        assert abs(U) < 1e-9


def test_lj_force_is_minus_energy_derivative_dimer():
    box = (12.0, 12.0, 12.0)
    m = lj_model(box)
    h = 1e-6
    for r in (0.95, 1.05, 1.3, 1.9, 2.4):
        def energy(rr):
            return oracle.forces(np.array([[1.0, 1.0, 1.0], [1.0 + rr, 1.0, 1.0]]), m, use_cells=False)[3][0]
        dEdr = (energy(r + h) - energy(r - h)) / (2 * h)
        F = oracle.forces(np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]]), m, use_cells=False)[0]
        # force on particle 1 along +x is -dE/dr
        assert F[1, 0] == pytest.approx(-dEdr, rel=1e-7, abs=1e-8)


# --------------------------------------------------------------------------------------
# Symmetries and conservation laws
# --------------------------------------------------------------------------------------

def test_newton_third_law_lj():
    s = systems.make_lj(500, 0.85, seed=11)
    F, _, _, _ = oracle.forces(s.pos, lj_model(s.box), use_cells=False)
    assert np.linalg.norm(F.sum(axis=0)) <= 1e-12 * np.abs(F).sum()


def _align_quat(target):
    """Unit quaternion rotating the body x axis onto the unit vector target."""
    x = np.array([1.0, 0.0, 0.0])
    ax = np.cross(x, target)
    s = np.linalg.norm(ax)
    if s < 1e-12:
        return np.array([1.0, 0, 0, 0]) if target[0] > 0 else np.array([0.0, 0, 0, 1])
    return axis_angle_quat(ax, np.arctan2(s, x @ target))


def _patchy_dimers(n_dimers, box, rng, gap=0.08):
    """Non-overlapping dimers whose patch 0 sites face each other at a small random
    separation, with a small random misalignment so that every component is generic."""
    pdir = systems.PATCH_DIRS
    box = np.asarray(box, dtype=float)
    pos, quat, centres = [], [], []
    tries = 0
    while len(centres) < n_dimers:
        tries += 1
        assert tries < 100000
        c = rng.uniform(0.0, 1.0, 3) * box
        dd = np.array(centres) - c if centres else np.zeros((0, 3))
        dd -= box * np.rint(dd / box)
        if len(dd) and np.min(np.linalg.norm(dd, axis=1)) < 2.6:
            continue
        centres.append(c)
        qa = rng.normal(size=4); qa /= np.linalg.norm(qa)
        ua = quat_rot(qa) @ pdir[0]
        xa = c - 0.55 * ua
        qb = qmul(_align_quat(-ua), axis_angle_quat([1, 0, 0], rng.uniform(0, 2 * np.pi)))
        qb = qmul(axis_angle_quat(rng.normal(size=3), rng.uniform(0.02, 0.15)), qb)
        off = rng.normal(size=3); off *= gap * rng.uniform(0.3, 1.0) / np.linalg.norm(off)
        xb = xa + ua * 1.0 + off
        pos += [xa, xb]
        quat += [qa, qb / np.linalg.norm(qb)]
    return np.mod(np.array(pos), box), np.array(quat)


def test_patchy_newton_and_angular_momentum_open_cluster():
    rng = np.random.default_rng(3)
    box = np.array([40.0, 40.0, 40.0])
    # a compact cluster of dimers in the middle: no pair crosses the periodic boundary
    pos, quat = _patchy_dimers(12, np.array([8.0, 8.0, 8.0]), rng)
    pos = pos + 16.0
    F, T, E, (U, W, npair) = oracle.forces(pos, patchy_model(box), quat=quat, use_cells=False)
    assert npair > 0 and np.abs(T).max() > 1e-3
    scale = np.abs(F).sum() + np.abs(T).sum()
    assert np.linalg.norm(F.sum(axis=0)) <= 1e-12 * scale
    Ltot = T.sum(axis=0) + np.cross(pos, F).sum(axis=0)
    assert np.linalg.norm(Ltot) <= 1e-12 * (scale * 30.0)


def test_perfect_fcc_has_zero_force():
    s = systems.make_lj(4000, 0.85, seed=12, jitter=0.0)
    F, _, E, (U, _, _) = oracle.forces(s.pos, lj_model(s.box), use_cells=True)
    assert np.abs(F).max() < 1e-11
    # every site is equivalent: identical per-particle energies
    assert np.ptp(E) < 1e-11


def test_translation_invariance():
    s = systems.make_lj(2000, 0.85, seed=13)
    m = lj_model(s.box)
    F0, _, _, (U0, _, _) = oracle.forces(s.pos, m, use_cells=True)
    shift = np.array([3.7, -11.2, 0.61])
    F1, _, _, (U1, _, _) = oracle.forces(np.mod(s.pos + shift, s.box), m, use_cells=True)
    frms = np.sqrt((F0 ** 2).sum(axis=1).mean())
    assert np.abs(F1 - F0).max() <= 1e-12 * frms
    assert U1 == pytest.approx(U0, rel=1e-12)


def _far_from_cutoff(pos, box, rc, idx, h):
    d = pos[None, :, :] - pos[idx][:, None, :]
    d -= box * np.rint(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    return np.all(np.abs(r - rc) > 10 * h, axis=1)


def test_lj_force_is_minus_gradient_many_body():
    s = systems.make_lj(256, 0.85, seed=14)
    m = lj_model(s.box)
    F, _, _, _ = oracle.forces(s.pos, m, use_cells=False)
    frms = np.sqrt((F ** 2).sum(axis=1).mean())
    h = 1e-5
    idx = np.arange(0, 256, 17)
    ok = _far_from_cutoff(s.pos, s.box, 2.5, idx, h)
    checked = 0
    for i in idx[ok]:
        for c in range(3):
            p = s.pos.copy(); p[i, c] += h
            up = oracle.forces(p, m, use_cells=False)[3][0]
            p[i, c] -= 2 * h
            um = oracle.forces(p, m, use_cells=False)[3][0]
            assert F[i, c] == pytest.approx(-(up - um) / (2 * h), abs=1e-6 * frms)
            checked += 1
    assert checked >= 15


def test_patchy_force_and_torque_are_minus_gradients():
    rng = np.random.default_rng(5)
    box = np.array([7.0, 7.0, 7.0])
    pos, quat = _patchy_dimers(10, box, rng)
    m = patchy_model(box)
    F, T, _, (U, _, npair) = oracle.forces(pos, m, quat=quat, use_cells=False)
    assert npair >= 10 and np.abs(T).max() > 1e-2
    scale = max(np.sqrt((F ** 2).sum(axis=1).mean()), 1.0)
    tscale = max(np.sqrt((T ** 2).sum(axis=1).mean()), 1.0)
    h = 1e-6
    for i in range(0, len(pos), 3):
        for c in range(3):
            p = pos.copy(); p[i, c] += h
            up = oracle.forces(p, m, quat=quat, use_cells=False)[3][0]
            p[i, c] -= 2 * h
            um = oracle.forces(p, m, quat=quat, use_cells=False)[3][0]
            assert F[i, c] == pytest.approx(-(up - um) / (2 * h), abs=2e-6 * scale)
            e = np.zeros(3); e[c] = 1.0
            qp = quat.copy(); qp[i] = qmul(axis_angle_quat(e, h), quat[i])
            qm = quat.copy(); qm[i] = qmul(axis_angle_quat(e, -h), quat[i])
            up = oracle.forces(pos, m, quat=qp, use_cells=False)[3][0]
            um = oracle.forces(pos, m, quat=qm, use_cells=False)[3][0]
            assert T[i, c] == pytest.approx(-(up - um) / (2 * h), abs=2e-6 * tscale)


def _rodrigues(k, theta, v):
    k = np.asarray(k, dtype=float) / np.linalg.norm(k)
    return v * np.cos(theta) + np.cross(k, v) * np.sin(theta) + k * (k @ v) * (1 - np.cos(theta))


def test_quaternion_matrix_is_rodrigues_rotation():
    """The tests' own quaternion -> matrix map equals Rodrigues' rotation formula."""
    rng = np.random.default_rng(41)
    for _ in range(20):
        k, v = rng.normal(size=3), rng.normal(size=3)
        th = rng.uniform(-np.pi, np.pi)
        np.testing.assert_allclose(quat_rot(axis_angle_quat(k, th)) @ v, _rodrigues(k, th, v), atol=1e-13)


def test_patchy_energy_random_orientations_independent_numpy():
    """Dimers at random orientations: the oracle's pair energy equals an independent numpy
    sum of the WCA core and all nine patch-pair terms (Sec. Models, Eqs. 2-4 as read)."""
    rng = np.random.default_rng(42)
    box = (9.0, 9.0, 9.0)
    m = patchy_model(box)
    P = systems.PATCH_DIRS * systems.PATCH_RADIUS
    hits = 0
    for _ in range(200):
        qa = rng.normal(size=4); qa /= np.linalg.norm(qa)
        qb = rng.normal(size=4); qb /= np.linalg.norm(qb)
        # put a patch of b near a patch of a so that the patch terms are not all zero
        a_site = quat_rot(qa) @ P[rng.integers(3)]
        b_site = quat_rot(qb) @ P[rng.integers(3)]
        d = a_site - b_site + rng.normal(size=3) * 0.06
        if not (0.9 < np.linalg.norm(d) < 1.5):
            continue
        xa = np.array([4.0, 4.5, 5.0])
        pos = np.stack([xa, xa + d])
        U = oracle.forces(pos, m, quat=np.stack([qa, qb]), use_cells=False)[3][0]
        r = np.linalg.norm(d)
        ref = 4 * (r ** -12 - r ** -6) + 1.0 if r < 2 ** (1 / 6) else 0.0
        for pa in P:
            for pb in P:
                s = d + quat_rot(qb) @ pb - quat_rot(qa) @ pa
                ref += -np.exp(-0.5 * (np.sqrt(s @ s) / 0.12) ** 10)
        hits += abs(ref) > 1e-3
        assert U == pytest.approx(ref, rel=1e-11, abs=1e-13)
    assert hits > 30


def test_patchy_dimer_closed_form():
    """Two particles on the x axis with patch 0 of each pointing at the other: only that
    patch pair is within reach, so E = WCA(r) - eps_p exp(-((r - 1)/delta)^10 / 2)."""
    box = (10.0, 10.0, 10.0)
    m = patchy_model(box)
    qa = np.array([1.0, 0.0, 0.0, 0.0])
    qb = axis_angle_quat([0, 0, 1], np.pi)  # patch 0 of b points along -x
    delta = 0.12
    for r in (1.03, 1.08, 1.12, 1.2):
        pos = np.array([[2.0, 5.0, 5.0], [2.0 + r, 5.0, 5.0]])
        F, T, E, (U, _, _) = oracle.forces(pos, m, quat=np.stack([qa, qb]), use_cells=False)
        s = r - 1.0
        wca = 4 * (r ** -12 - r ** -6) + 1.0 if r < 2 ** (1 / 6) else 0.0
        dwca = -24 * (2 * r ** -13 - r ** -7) if r < 2 ** (1 / 6) else 0.0  # dV/dr
        ep = -np.exp(-0.5 * (s / delta) ** 10)
        dep = ep * (-0.5 * 10 * s ** 9 / delta ** 10)  # d/dr of -exp(g), g = -(s/delta)^10 / 2
        assert U == pytest.approx(wca + ep, rel=1e-12, abs=1e-14)
        # force on b along +x is -dU/dr; no transverse components, no torques on the axis
        assert F[1, 0] == pytest.approx(-(dwca + dep), rel=1e-10, abs=1e-12)
        assert np.abs(F[:, 1:]).max() < 1e-12 and np.abs(T).max() < 1e-12


def test_patchy_rotated_dimer_torque_closed_form():
    """Rotate particle a by theta about z: its patch site moves on a circle; the single
    contributing patch pair gives E(theta) in closed form and tau_z = -dE/dtheta."""
    box = (10.0, 10.0, 10.0)
    m = patchy_model(box)
    delta, r = 0.12, 1.15  # beyond the WCA range: only the patch term
    qb = axis_angle_quat([0, 0, 1], np.pi)
    for theta in (0.05, 0.1, -0.08):
        qa = axis_angle_quat([0, 0, 1], theta)
        pos = np.array([[2.0, 5.0, 5.0], [2.0 + r, 5.0, 5.0]])
        F, T, E, (U, _, _) = oracle.forces(pos, m, quat=np.stack([qa, qb]), use_cells=False)
        sx, sy = r - 0.5 - 0.5 * np.cos(theta), -0.5 * np.sin(theta)
        q = (sx * sx + sy * sy) / delta ** 2
        e = -np.exp(-0.5 * q ** 5)
        dq = 2 * (sx * (0.5 * np.sin(theta)) + sy * (-0.5 * np.cos(theta))) / delta ** 2
        dE = e * (-2.5 * q ** 4) * dq  # d/dtheta of -exp(-q^5 / 2)
        assert U == pytest.approx(e, rel=1e-12)
        assert T[0, 2] == pytest.approx(-dE, rel=1e-9, abs=1e-12)


# --------------------------------------------------------------------------------------
# Cell lists and Verlet pair sets (Sec. Methods)
# --------------------------------------------------------------------------------------

def _numpy_pairs(pos, box, rv):
    d = pos[None, :, :] - pos[:, None, :]
    d = d - box * np.rint(d / box)
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    i, j = np.nonzero(np.triu(r2 < rv * rv, k=1))
    return np.stack([i, j], axis=1)


@pytest.mark.parametrize("case", ["lj", "wca", "tiny_box", "noncubic", "edge_of_integer"])
def test_pair_sets_brute_cells_numpy_agree(case):
    if case == "lj":
        s = systems.make_lj(1500, 0.85, seed=21); box = s.box; rv = 2.8; pos = s.pos
    elif case == "wca":
        s = systems.make_wca(3000, 0.2, seed=22); box = s.box; rv = s.rv; pos = s.pos
    elif case == "tiny_box":
        s = systems.make_lj(500, 0.9, seed=23); box = s.box; rv = 2.8; pos = s.pos  # L = 8.2: 2 cells -> 1
    elif case == "noncubic":
        rng = np.random.default_rng(24); box = np.array([9.0, 14.5, 23.0]); rv = 2.8
        pos = rng.uniform(0, 1, (1200, 3)) * box
    else:
        rv = 2.8; L = 3 * rv * (1 + 1e-13); box = np.array([L, 4 * rv * (1 - 1e-13), 11.3])
        pos = np.random.default_rng(25).uniform(0, 1, (700, 3)) * box
    ref = _numpy_pairs(pos, box, rv)
    pb = oracle.pairs(pos, box, rv, use_cells=False)
    pc = oracle.pairs(pos, box, rv, use_cells=True)
    assert np.array_equal(pb, ref)
    assert np.array_equal(pc, ref)


def test_cell_dims_rule():
    assert oracle.cell_dims((16.758, 16.758, 16.758), 2.8) == (5, 5, 5)
    assert oracle.cell_dims((8.22, 8.22, 8.22), 2.8) == (1, 1, 1)   # 2 cells per side -> one cell
    assert oracle.cell_dims((3 * 2.8 * (1 - 1e-14),) * 3, 2.8) == (1, 1, 1)


def test_forces_brute_equal_cells():
    s = systems.make_lj(3000, 0.85, seed=26)
    m = lj_model(s.box)
    Fb, _, Eb, (Ub, Wb, nb) = oracle.forces(s.pos, m, use_cells=False)
    Fc, _, Ec, (Uc, Wc, nc) = oracle.forces(s.pos, m, use_cells=True)
    frms = np.sqrt((Fb ** 2).sum(axis=1).mean())
    assert nb == nc
    assert np.abs(Fb - Fc).max() <= 1e-13 * frms
    assert Uc == pytest.approx(Ub, rel=1e-13) and Wc == pytest.approx(Wb, rel=1e-13)


def test_patchy_brute_equal_cells():
    s = systems.make_patchy(2000, 0.3, seed=27)
    m = patchy_model(s.box)
    Fb, Tb, _, (Ub, _, nb) = oracle.forces(s.pos, m, quat=s.quat, use_cells=False)
    Fc, Tc, _, (Uc, _, nc) = oracle.forces(s.pos, m, quat=s.quat, use_cells=True)
    assert nb == nc and nb > 0
    np.testing.assert_allclose(Fc, Fb, atol=1e-12 * max(1.0, np.abs(Fb).max()))
    np.testing.assert_allclose(Tc, Tb, atol=1e-12 * max(1.0, np.abs(Tb).max()))


# --------------------------------------------------------------------------------------
# Integration (velocity Verlet, rigid-body rotation)
# --------------------------------------------------------------------------------------

def _fluct(trace):
    e = trace[:, 0] + trace[:, 1] + trace[:, 2]
    return np.sqrt(np.mean((e - e.mean()) ** 2))


def test_nve_energy_fluctuation_scales_as_dt_squared():
    s = systems.make_wca(256, 0.6, seed=31)
    m = wca_model(s.box)
    out = []
    for dt, n in ((0.004, 100), (0.002, 200)):
        _, _, _, _, tr = oracle.run_nve(s.pos, s.vel, m, dt, n, use_cells=False)
        out.append(_fluct(tr))
    ratio = out[0] / out[1]
    assert 3.2 < ratio < 4.8, ratio


def test_nve_lj_conserves_energy():
    """The lattice start relaxes strongly (large exchange of kinetic and potential energy);
    the total-energy error stays small and halves twice when dt halves."""
    s = systems.make_lj(500, 0.85, seed=32)
    errs = []
    for dt, n in ((0.001, 100), (0.0005, 200)):
        _, _, _, _, tr = oracle.run_nve(s.pos, s.vel, lj_model(s.box), dt, n, use_cells=True)
        e = tr[:, 0] + tr[:, 1] + tr[:, 2]
        errs.append(np.abs(e - e[0]).max() / len(s.pos))
        assert np.ptp(tr[:, 0]) / len(s.pos) > 0.1
    assert errs[0] < 1e-4
    assert 3.2 < errs[0] / errs[1] < 4.8, errs


def test_patchy_nve_dt_squared():
    rng = np.random.default_rng(33)
    box = np.array([8.0, 8.0, 8.0])
    pos, quat = _patchy_dimers(16, box, rng)
    n = len(pos)
    vel = rng.normal(0, 0.3, (n, 3)); vel -= vel.mean(axis=0)
    L = rng.normal(0, 0.1, (n, 3))
    m = patchy_model(box)
    out = []
    for dt, k in ((0.002, 100), (0.001, 200)):
        _, _, _, _, tr = oracle.run_nve(pos, vel, m, dt, k, quat=quat, angmom=L, inertia=0.1, use_cells=False)
        assert np.ptp(tr[:, 1]) > 1e-4  # the rotational kinetic energy changes
        out.append(_fluct(tr))
    ratio = out[0] / out[1]
    assert 3.0 < ratio < 5.0, ratio


def test_free_rotation_matches_rodrigues():
    box = (10.0, 10.0, 10.0)
    m = patchy_model(box)
    q0 = axis_angle_quat([0.3, -1.0, 0.4], 0.7)
    Lang = np.array([[0.02, -0.05, 0.03]])
    inertia, dt, nsteps = 0.1, 0.01, 37
    _, _, q, _, _ = oracle.run_nve(np.array([[5.0, 5.0, 5.0]]), np.zeros((1, 3)), m, dt, nsteps,
                                   quat=q0[None, :], angmom=Lang, inertia=inertia, use_cells=False)
    w = Lang[0] / inertia
    theta = np.linalg.norm(w) * dt * nsteps
    k = w / np.linalg.norm(w)
    p0 = quat_rot(q0) @ systems.PATCH_DIRS[1]
    rod = p0 * np.cos(theta) + np.cross(k, p0) * np.sin(theta) + k * (k @ p0) * (1 - np.cos(theta))
    np.testing.assert_allclose(quat_rot(q[0]) @ systems.PATCH_DIRS[1], rod, atol=1e-12)


def test_ballistic_drift_wraps():
    box = (5.0, 6.0, 7.0)
    m = lj_model((20.0, 20.0, 20.0))
    m.box = box
    pos = np.array([[4.9, 0.05, 3.0]])
    vel = np.array([[1.3, -0.9, 0.2]])
    p, v, _, _, _ = oracle.run_nve(pos, vel, m, 0.01, 50, use_cells=False)
    np.testing.assert_allclose(p[0], np.mod(pos[0] + vel[0] * 0.5, box), atol=1e-12)
    np.testing.assert_allclose(v[0], vel[0], atol=0)

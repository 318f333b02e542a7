"""Pins of the oracle's paper-form patchy model and of its thermostat.

The patchy form (Sec. Models): a (sigma/r)^200 centre repulsion plus, for every patch pair, the
attraction -eps exp(-(r_ab/0.12 sigma)^10 / 2), truncated at r_ab = 0.18 sigma; two patch sites at
the poles.  The thermostat (Sec. Methods, Brownian NVT): momenta redrawn from Maxwell-Boltzmann at
kT.  Each test checks a closed form, a derivative, a conservation law or a distribution, not the
oracle against itself.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1401_4350_gb300 import systems
from tests.test_oracle import axis_angle_quat, qmul, quat_rot

POLAR = systems.PATCH_DIRS_POLAR * systems.PATCH_RADIUS


def pow_model(box, rc=1.18, patch_rc=0.18):
    return oracle.Model(oracle.PATCHY_POW, tuple(box), rc, eps_p=1.0, delta=0.12, patches=POLAR, patch_rc=patch_rc)


# quaternions turning the body z axis (patch 0) onto +x and onto -x
Q_PLUS_X = axis_angle_quat([0, 1, 0], np.pi / 2)
Q_MINUS_X = axis_angle_quat([0, 1, 0], -np.pi / 2)
Q_Z = np.array([1.0, 0.0, 0.0, 0.0])


def test_polar_patches_point_where_the_quaternions_say():
    np.testing.assert_allclose(quat_rot(Q_PLUS_X) @ [0, 0, 1], [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(quat_rot(Q_MINUS_X) @ [0, 0, 1], [-1, 0, 0], atol=1e-15)


@pytest.mark.parametrize("r", [0.97, 1.0, 1.03, 1.1, 1.17])
def test_core_dimer_closed_form(r):
    """Patches along z, separation along x: no patch pair is within 0.18 sigma, so E = (1/r)^200 and
    the force on b is +200 r^-201 along x."""
    m = pow_model((10.0, 10.0, 10.0))
    pos = np.array([[3.0, 5.0, 5.0], [3.0 + r, 5.0, 5.0]])
    F, T, E, (U, W, npair) = oracle.forces(pos, m, quat=np.stack([Q_Z, Q_Z]), use_cells=False)
    assert U == pytest.approx(r ** -200, rel=1e-12)
    assert F[1, 0] == pytest.approx(200.0 * r ** -201, rel=1e-12)
    assert F[0, 0] == pytest.approx(-200.0 * r ** -201, rel=1e-12)
    assert np.abs(F[:, 1:]).max() == 0.0 and np.abs(T).max() == 0.0
    assert E[0] == pytest.approx(0.5 * U, rel=1e-15) and npair == 1


def test_core_is_cut_at_the_centre_cutoff():
    m = pow_model((10.0, 10.0, 10.0))
    pos = np.array([[3.0, 5.0, 5.0], [3.0 + 1.1801, 5.0, 5.0]])
    F, T, E, (U, W, npair) = oracle.forces(pos, m, quat=np.stack([Q_Z, Q_Z]), use_cells=False)
    assert U == 0.0 and npair == 0 and np.abs(F).max() == 0.0


@pytest.mark.parametrize("s", [0.02, 0.08, 0.12, 0.15, 0.179])
def test_facing_patches_closed_form(s):
    """Patch 0 of a points along +x, patch 0 of b along -x, centres r = 1 + s apart on x: one patch
    pair at distance s, E = r^-200 - exp(-(s/0.12)^10 / 2); the force on b along x is -dE/dr."""
    m = pow_model((10.0, 10.0, 10.0))
    r = 1.0 + s
    pos = np.array([[3.0, 5.0, 5.0], [3.0 + r, 5.0, 5.0]])
    F, T, E, (U, W, npair) = oracle.forces(pos, m, quat=np.stack([Q_PLUS_X, Q_MINUS_X]), use_cells=False)
    ep = -np.exp(-0.5 * (s / 0.12) ** 10)
    assert U == pytest.approx(r ** -200 + ep, rel=1e-12, abs=1e-15)
    dE = -200 * r ** -201 + ep * (-5.0 * s ** 9 / 0.12 ** 10)
    assert F[1, 0] == pytest.approx(-dE, rel=1e-10, abs=1e-12)
    assert np.abs(F[:, 1:]).max() < 1e-12 and np.abs(T).max() < 1e-12


def test_patch_pairs_are_truncated_at_patch_rc():
    """Just inside 0.18 sigma the patch term is present (about 3e-13); just outside it is exactly gone."""
    m = pow_model((10.0, 10.0, 10.0))
    q = np.stack([Q_PLUS_X, Q_MINUS_X])
    inside = oracle.forces(np.array([[3.0, 5.0, 5.0], [4.1799, 5.0, 5.0]]), m, quat=q, use_cells=False)[3][0]
    outside = oracle.forces(np.array([[3.0, 5.0, 5.0], [4.1801, 5.0, 5.0]]), m, quat=q, use_cells=False)[3][0]
    assert inside == pytest.approx(1.1799 ** -200 - np.exp(-0.5 * (0.1799 / 0.12) ** 10), rel=1e-12, abs=1e-20)
    assert outside == 0.0  # beyond the centre cut-off 1.18 as well
    m2 = pow_model((10.0, 10.0, 10.0), rc=1.3)
    U2 = oracle.forces(np.array([[3.0, 5.0, 5.0], [4.1801, 5.0, 5.0]]), m2, quat=q, use_cells=False)[3][0]
    assert U2 == pytest.approx(1.1801 ** -200, rel=1e-12, abs=1e-20)  # core only: the patch pair is cut


def _pow_dimers(n, box, rng, gap=0.1):
    """Dimers with patch 0 sites close to each other (random misalignment) and far from other dimers."""
    pos, quat, centres = [], [], []
    while len(centres) < n:
        c = rng.uniform(0.0, 1.0, 3) * box
        dd = np.array(centres) - c if centres else np.zeros((0, 3))
        dd -= box * np.rint(dd / box)
        if len(dd) and np.min(np.linalg.norm(dd, axis=1)) < 2.6:
            continue
        centres.append(c)
        qa = rng.normal(size=4); qa /= np.linalg.norm(qa)
        ua = quat_rot(qa) @ [0, 0, 1.0]
        xa = c - 0.55 * ua
        # b: patch 0 (body +z) turned towards -ua, plus a small random tilt
        zb = -ua
        ax = np.cross([0, 0, 1.0], zb)
        qb = axis_angle_quat(ax, np.arccos(np.clip(zb[2], -1, 1))) if np.linalg.norm(ax) > 1e-9 else Q_Z
        qb = qmul(axis_angle_quat(rng.normal(size=3), rng.uniform(0.02, 0.2)), qb)
        off = rng.normal(size=3); off *= gap * rng.uniform(0.2, 1.0) / np.linalg.norm(off)
        xb = xa + ua * 1.04 + off
        if not (1.0 < np.linalg.norm(xb - xa) < 1.16):  # no huge core energies (finite differences)
            centres.pop()
            continue
        pos += [xa, xb]
        quat += [qa, qb / np.linalg.norm(qb)]
    return np.mod(np.array(pos), box), np.array(quat)


def test_pow_force_and_torque_are_minus_gradients():
    rng = np.random.default_rng(11)
    box = np.array([8.0, 8.0, 8.0])
    pos, quat = _pow_dimers(10, box, rng)
    m = pow_model(box)
    F, T, _, (U, _, npair) = oracle.forces(pos, m, quat=quat, use_cells=False)
    assert npair >= 8 and np.abs(T).max() > 1e-2
    scale = max(np.sqrt((F ** 2).sum(axis=1).mean()), 1.0)
    tscale = max(np.sqrt((T ** 2).sum(axis=1).mean()), 1.0)
    h = 1e-7
    for i in range(0, len(pos), 3):
        for c in range(3):
            p = pos.copy(); p[i, c] += h
            up = oracle.forces(p, m, quat=quat, use_cells=False)[3][0]
            p[i, c] -= 2 * h
            um = oracle.forces(p, m, quat=quat, use_cells=False)[3][0]
            assert F[i, c] == pytest.approx(-(up - um) / (2 * h), abs=1e-5 * scale)
            e = np.zeros(3); e[c] = 1.0
            qp = quat.copy(); qp[i] = qmul(axis_angle_quat(e, h), quat[i])
            qm = quat.copy(); qm[i] = qmul(axis_angle_quat(e, -h), quat[i])
            up = oracle.forces(pos, m, quat=qp, use_cells=False)[3][0]
            um = oracle.forces(pos, m, quat=qm, use_cells=False)[3][0]
            assert T[i, c] == pytest.approx(-(up - um) / (2 * h), abs=1e-5 * tscale)


def test_pow_energy_independent_numpy():
    """Random orientations: the oracle's energy equals a numpy sum of the core and the four truncated
    patch-pair terms."""
    rng = np.random.default_rng(12)
    m = pow_model((9.0, 9.0, 9.0))
    hits = 0
    for _ in range(300):
        qa = rng.normal(size=4); qa /= np.linalg.norm(qa)
        qb = rng.normal(size=4); qb /= np.linalg.norm(qb)
        a_site = quat_rot(qa) @ POLAR[rng.integers(2)]
        b_site = quat_rot(qb) @ POLAR[rng.integers(2)]
        d = a_site - b_site + rng.normal(size=3) * 0.07
        r = np.linalg.norm(d)
        if not (0.95 < r < 1.18):
            continue
        xa = np.array([4.0, 4.5, 5.0])
        U = oracle.forces(np.stack([xa, xa + d]), m, quat=np.stack([qa, qb]), use_cells=False)[3][0]
        ref = r ** -200.0
        for pa in POLAR:
            for pb in POLAR:
                s = d + quat_rot(qb) @ pb - quat_rot(qa) @ pa
                rs = np.sqrt(s @ s)
                if rs < 0.18:
                    ref += -np.exp(-0.5 * (rs / 0.12) ** 10)
                    hits += 1
        assert U == pytest.approx(ref, rel=1e-11, abs=1e-13)
    assert hits > 30


def test_pow_newton_and_angular_momentum_open_cluster():
    rng = np.random.default_rng(13)
    box = np.array([30.0, 30.0, 30.0])
    pos, quat = _pow_dimers(6, box, rng)
    pos = 10.0 + np.mod(pos, 10.0)  # an open cluster well inside the box
    m = pow_model(box)
    F, T, _, _ = oracle.forces(pos, m, quat=quat, use_cells=False)
    assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).sum()
    L = (np.cross(pos, F) + T).sum(0)
    assert np.abs(L).max() < 1e-11 * (np.abs(np.cross(pos, F)).sum() + np.abs(T).sum())


# --------------------------------------------------------------------------------------
# Counter-based random numbers and the momentum-refresh thermostat (Sec. Methods)
# --------------------------------------------------------------------------------------

def _philox_kat_rows():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            w = [int(x, 16) for x in line]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answer_vectors():
    """The oracle's Philox4x32-10 reproduces the generator's published known-answer vectors (Salmon et al.,
    SC'11; Random123): a wrong multiplier, Weyl constant, round count or output word order changes every
    word, which no statistical pin can see."""
    rows = _philox_kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = [int(x) for x in oracle.philox4x32(ctr, key)]
        assert got == want, (ctr, key, [hex(x) for x in got], [hex(x) for x in want])


def test_philox_words_are_uniform_and_uncorrelated():
    key = [12345, 0]
    words = np.array([oracle.philox4x32([s, i, 0, 0], key) for s in range(5) for i in range(4000)], dtype=np.float64)
    u = (words + 0.5) / 2 ** 32
    for c in range(4):
        counts = np.histogram(u[:, c], bins=32, range=(0, 1))[0]
        exp = len(u) / 32
        chi2 = ((counts - exp) ** 2 / exp).sum()
        assert chi2 < 70  # 31 degrees of freedom: far above the 0.999 quantile (61) only if broken
    cc = np.corrcoef(u.T)
    assert np.abs(cc - np.eye(4)).max() < 0.02
    assert abs(np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]) < 0.02  # neighbouring counters


def test_thermostat_normals_are_standard():
    draws = np.array([oracle.thermostat_draw(7, 3, i)[1] for i in range(20000)])
    assert np.abs(draws.mean(0)).max() < 4 / np.sqrt(len(draws))
    assert np.abs(draws.var(0) - 1.0).max() < 0.04
    k = ((draws - draws.mean(0)) ** 4).mean(0) / draws.var(0) ** 2
    assert np.abs(k - 3.0).max() < 0.15  # Gaussian kurtosis
    us = np.array([oracle.thermostat_draw(7, 3, i)[0] for i in range(20000)])
    assert abs(us.mean() - 0.5) < 0.01 and 0 < us.min() and us.max() < 1


def _free_gas(n=64, spacing=3.0):
    """Particles on a cubic lattice farther apart than every cut-off: all forces are exactly zero."""
    k = int(round(n ** (1 / 3)))
    g = np.arange(k) * spacing
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.5
    return pos, np.full(3, k * spacing)


@pytest.mark.parametrize("kind", ["lj", "pow"])
def test_refresh_sets_maxwell_boltzmann_momenta_from_the_draws(kind):
    """With no forces and prob = 1 the momenta after a refresh are exactly sqrt(kT/m) n and
    sqrt(kT I) n' of that step's draws (m = 2, kT = 1.5, I = 0.1 catch a wrong scale)."""
    pos, box = _free_gas()
    n = len(pos)
    rng = np.random.default_rng(1)
    vel = rng.normal(size=(n, 3))
    th = oracle.Thermostat(every=1, prob=1.0, kT=1.5, seed=99)
    mass, inertia = 2.0, 0.1
    if kind == "lj":
        m = oracle.Model(oracle.LJ, tuple(box), 2.5)
        p1, v1, _, _, _ = oracle.run(pos, vel, m, 0.001, 2, mass=mass, thermostat=th, use_cells=False)
        L1 = None
    else:
        m = pow_model(box)
        q = np.tile(Q_Z, (n, 1))
        L = rng.normal(size=(n, 3))
        p1, v1, q1, L1, _ = oracle.run(pos, vel, m, 0.001, 2, mass=mass, inertia=inertia, quat=q, angmom=L,
                                       thermostat=th, use_cells=False)
    # step 0 has no refresh, step 1 redraws every particle; forces are zero throughout
    for i in range(n):
        _, nrm = oracle.thermostat_draw(99, 1, i)
        np.testing.assert_allclose(v1[i], np.sqrt(1.5 / mass) * nrm[:3], rtol=1e-15)
        if L1 is not None:
            np.testing.assert_allclose(L1[i], np.sqrt(1.5 * inertia) * nrm[3:], rtol=1e-15)


def test_refresh_probability_and_schedule():
    pos, box = _free_gas(125)
    n = len(pos)
    vel = np.random.default_rng(2).normal(size=(n, 3))
    m = oracle.Model(oracle.LJ, tuple(box), 2.5)
    # every = 3, prob = 1: after 8 steps the last refresh was at step 6
    th = oracle.Thermostat(every=3, prob=1.0, kT=1.0, seed=5)
    _, v, _, _, _ = oracle.run(pos, vel, m, 0.001, 8, thermostat=th, use_cells=False)
    ref = np.array([oracle.thermostat_draw(5, 6, i)[1][:3] for i in range(n)])
    np.testing.assert_allclose(v, ref, rtol=1e-15)
    # the same run in two pieces (step numbers continue) draws the same numbers
    p1, v1, _, _, _ = oracle.run(pos, vel, m, 0.001, 5, thermostat=th, use_cells=False)
    _, v2, _, _, _ = oracle.run(p1, v1, m, 0.001, 3, thermostat=th, use_cells=False, step0=5)
    np.testing.assert_allclose(v2, v, rtol=1e-15)
    # prob = 0.3: the refreshed fraction
    th = oracle.Thermostat(every=1, prob=0.3, kT=1.0, seed=8)
    _, v, _, _, _ = oracle.run(pos, vel, m, 0.001, 2, thermostat=th, use_cells=False)
    changed = np.any(v != vel, axis=1)
    expected = np.array([oracle.thermostat_draw(8, 1, i)[0] < 0.3 for i in range(n)])
    assert np.array_equal(changed, expected)
    assert 0.15 < changed.mean() < 0.45


def test_thermostat_drives_the_kinetic_temperature_to_kT():
    s = systems.make_lj(256, 0.3, temperature=0.5, seed=21)
    m = oracle.Model(oracle.LJ, tuple(s.box), 2.5)
    th = oracle.Thermostat(every=5, prob=0.3, kT=1.8, seed=3)
    _, _, _, _, trace = oracle.run(s.pos, s.vel, m, 0.002, 1500, thermostat=th)
    T = trace[:, 0] / (1.5 * 256)
    assert T[:5].mean() < 0.8
    assert T[-500:].mean() == pytest.approx(1.8, rel=0.08)

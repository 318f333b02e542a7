"""The seeded input recipes (paper_1401_4350_gb300/systems.py) do what their description says: the FCC start
with its vacancy rule, the random sequential addition with its minimum separation, Maxwell-Boltzmann
velocities rescaled to (3N - 3) T / 2 with no centre-of-mass motion, unit quaternions and angular momenta at
3N T / 2, the batch recipe, and determinism under a seed.  CPU only."""
import numpy as np
import pytest

from paper_1401_4350_gb300 import systems


def _min_image_dists(pos, box):
    d = pos[:, None, :] - pos[None, :, :]
    d -= box * np.rint(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    return r


@pytest.mark.parametrize("n,cells,vacancies", [(4000, 10, 0), (3000, 10, 1000), (65_536, 26, 4768)])
def test_fcc_start_and_vacancy_rule(n, cells, vacancies):
    s = systems.make_lj(n, 0.85, 1.0, seed=1001)
    L = (n / 0.85) ** (1.0 / 3.0)
    assert s.n == n and np.allclose(s.box, L)
    assert np.all(s.pos >= 0.0) and np.all(s.pos < L)
    assert 4 * cells ** 3 - n == vacancies
    # every particle sits within the jitter of an FCC site of spacing L / M (per coordinate, up to wrap)
    a = L / cells
    frac = np.mod(s.pos / (a / 2.0), 1.0)  # FCC sites lie on the half-spacing grid
    off = np.minimum(frac, 1.0 - frac) * (a / 2.0)
    assert off.max() <= 0.05 + 1e-9
    assert off.max() > 0.04  # the displacement is there


def test_perfect_lattice_without_jitter_has_the_fcc_neighbour_shell():
    s = systems.make_lj(500, 0.85, 1.0, seed=7, jitter=0.0)  # M = 5: a perfect lattice
    nn = s.box[0] / 5 / np.sqrt(2.0)
    r = _min_image_dists(s.pos, s.box)
    assert r.min() == pytest.approx(nn, rel=1e-12)
    assert np.all((np.abs(r - nn) < 1e-9).sum(1) == 12)


@pytest.mark.parametrize("maker,n,rho", [(systems.make_wca, 3000, 0.2), (systems.make_patchy, 2500, 0.3)])
def test_random_sequential_addition_keeps_one_sigma(maker, n, rho):
    s = maker(n, rho, seed=11)
    L = (n / rho) ** (1.0 / 3.0)
    assert s.n == n and np.allclose(s.box, L)
    assert np.all(s.pos >= 0.0) and np.all(s.pos < L)
    assert _min_image_dists(s.pos, s.box).min() >= 1.0


@pytest.mark.parametrize("maker", [lambda: systems.make_lj(4000, 0.85, 1.3, seed=3),
                                   lambda: systems.make_wca(2000, 0.2, 0.7, seed=3),
                                   lambda: systems.make_patchy(1500, 0.3, 0.15, seed=3)])
def test_velocities_have_no_drift_and_the_stated_kinetic_energy(maker):
    s = maker()
    assert np.abs(s.vel.sum(0)).max() < 1e-10 * s.n
    k = 0.5 * s.mass * (s.vel ** 2).sum()
    assert k == pytest.approx(0.5 * (3 * s.n - 3) * s.temperature, rel=1e-12)
    # a Gaussian per component: kurtosis near 3
    v = s.vel.ravel() / s.vel.std()
    assert abs((v ** 4).mean() - 3.0) < 0.3


def test_patchy_orientations_and_angular_momenta():
    s = systems.make_patchy(3000, 0.3, 0.15, seed=9)
    assert np.allclose(np.linalg.norm(s.quat, axis=1), 1.0, atol=1e-14)
    # uniform on the unit 3-sphere: every component has mean 0 and variance 1/4
    assert np.abs(s.quat.mean(0)).max() < 0.05
    assert np.allclose((s.quat ** 2).mean(0), 0.25, atol=0.02)
    krot = 0.5 * (s.angmom ** 2).sum() / s.inertia
    assert krot == pytest.approx(0.5 * 3 * s.n * s.temperature, rel=1e-12)
    assert s.patches.shape == (3, 3) and np.allclose(np.linalg.norm(s.patches, axis=1), 0.5)
    # three sites 120 degrees apart in the body xy-plane
    c = s.patches @ s.patches.T / 0.25
    assert np.allclose(c[np.triu_indices(3, 1)], -0.5) and np.allclose(s.patches[:, 2], 0.0)


def test_paper_form_patchy_has_two_polar_sites_and_the_refresh():
    s = systems.make_patchy_pow(1000, 0.3, seed=2)
    assert s.kind == systems.PATCHY_POW and s.patches.shape == (2, 3)
    assert np.allclose(s.patches, [[0, 0, 0.5], [0, 0, -0.5]])
    assert s.rc == pytest.approx(1.18) and s.patch_rc == pytest.approx(0.18)
    assert s.thermostat_every == 100 and s.thermostat_prob == pytest.approx(0.1)


def test_batch_recipe():
    specs = systems.batch_specs(512, seed=1004)
    assert len(specs) == 512
    ns = np.array([n for _, n, _, _ in specs])
    assert ns.min() >= 500 and ns.max() <= 32768
    # log-uniform: the median is near the geometric mean of the range
    assert abs(np.log(np.median(ns)) - 0.5 * (np.log(500) + np.log(32768))) < 0.3
    for r, (kind, n, rho, seed) in enumerate(specs):
        assert seed == 5000 + r
        if r % 4 == 0:
            assert kind == systems.WCA and rho == 0.2
        else:
            assert kind == systems.LJ and 0.2 <= rho <= 0.9


def test_seeded_and_deterministic():
    a, b = systems.make_wca(1500, 0.2, seed=21), systems.make_wca(1500, 0.2, seed=21)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)
    c = systems.make_wca(1500, 0.2, seed=22)
    assert not np.array_equal(a.pos, c.pos)
    p, q = systems.make_patchy(800, 0.3, seed=5), systems.make_patchy(800, 0.3, seed=5)
    assert np.array_equal(p.quat, q.quat) and np.array_equal(p.angmom, q.angmom)

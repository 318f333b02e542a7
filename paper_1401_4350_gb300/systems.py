"""Seeded synthetic MD systems (input generation only, no force arithmetic).

This module is shared by the tests, the bench and the CUDA path's callers; it
holds none of the method's arithmetic (no potential, no force, no neighbour
search of the method), only the recipes that place particles and draw
velocities and orientations.  The recipes:

* Lennard-Jones / dense fluids: an FCC lattice of M = ceil((N/4)^(1/3)) unit
  cells per side in a cubic box of edge L = (N/rho)^(1/3); when 4 M^3 > N the
  surplus sites are removed at random; every coordinate is displaced by
  U(-0.05, 0.05) sigma.
* Sparse fluids (WCA) and patchy particles: random sequential addition of
  uniformly random points with a minimum separation of 1 sigma, done in rounds
  (a candidate is rejected if it is closer than 1 sigma to an accepted point or
  to an earlier surviving candidate of the same round).  Patchy particles are
  not put on the lattice: at rho = 0.3 its nearest-neighbour distance (1.68
  sigma) exceeds the 1.5 sigma cut-off, so no pair would interact at t = 0.
* Velocities: Maxwell-Boltzmann, N(0, T/m) per component, centre-of-mass
  motion removed, rescaled so that the kinetic energy is (3N - 3) T / 2.
* Patchy orientations: normalised 4-D Gaussians (uniform unit quaternions);
  angular momenta N(0, T I) per lab-frame component, rescaled to 3N T / 2.
* The paper's patchy form (Sec. Models): two patch sites at the poles of the body z axis,
  0.5 sigma from the centre (M = 2); same placement and orientation recipes as above.
* Thermostat settings (the paper's Brownian NVT runs, Sec. Methods): momenta of each
  particle redrawn with probability 0.1 every 100 steps (a reading: the paper does not
  give them); the kT of each system is its temperature.
* Random numbers: numpy PCG64 seeded per system (1000 + configuration index;
  replica r of the batch uses 5000 + r).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

LJ, WCA, PATCHY, PATCHY_POW = 0, 1, 2, 3
PATCHY_KINDS = (PATCHY, PATCHY_POW)
WCA_RC = 2.0 ** (1.0 / 6.0)

# Three patch sites 120 degrees apart in the body xy-plane, 0.5 sigma from the centre.
PATCH_DIRS = np.array([[1.0, 0.0, 0.0],
                       [-0.5, np.sqrt(3.0) / 2.0, 0.0],
                       [-0.5, -np.sqrt(3.0) / 2.0, 0.0]])
PATCH_RADIUS = 0.5
# The paper's patchy model: M = 2 sites at the poles.
PATCH_DIRS_POLAR = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])


@dataclass
class System:
    """One periodic system: FP64 host arrays plus the model and run parameters."""
    kind: int
    pos: np.ndarray                 # (N, 3) in [0, L)
    vel: np.ndarray                 # (N, 3)
    box: np.ndarray                 # (3,)
    rc: float
    skin: float
    dt: float
    temperature: float
    mass: float = 1.0
    eps: float = 1.0
    sigma: float = 1.0
    quat: Optional[np.ndarray] = None     # (N, 4) scalar-first unit quaternions
    angmom: Optional[np.ndarray] = None   # (N, 3) lab-frame angular momentum
    inertia: float = 0.1
    eps_p: float = 1.0
    delta: float = 0.12
    patches: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    name: str = ""
    patch_rc: float = 0.0           # PATCHY_POW: patch-pair cut-off
    thermostat_every: int = 0       # momentum refresh every so many steps (0: NVE)
    thermostat_prob: float = 0.0
    seed: int = 0

    @property
    def n(self) -> int:
        return len(self.pos)

    @property
    def rv(self) -> float:
        return self.rc + self.skin


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def fcc_positions(n: int, rho: float, rng: np.random.Generator, jitter: float = 0.05) -> tuple[np.ndarray, np.ndarray]:
    L = (n / rho) ** (1.0 / 3.0)
    M = int(np.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9))
    a = L / M
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(M)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    if len(sites) > n:
        keep = np.sort(rng.choice(len(sites), size=n, replace=False))
        sites = sites[keep]
    pos = sites + (rng.uniform(-jitter, jitter, size=sites.shape) if jitter > 0 else 0.0)
    pos = np.mod(pos, L)
    pos[pos >= L] -= L  # np.mod can return L for tiny negatives
    return pos, np.full(3, L)


def rsa_positions(n: int, rho: float, rng: np.random.Generator, dmin: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    from scipy.spatial import cKDTree
    L = (n / rho) ** (1.0 / 3.0)
    acc = np.zeros((0, 3))
    while len(acc) < n:
        need = n - len(acc)
        m = int(min(max(256, need * 1.25), 400_000))
        cand = rng.uniform(0.0, L, size=(m, 3))
        cand[cand >= L] = 0.0
        if len(acc):
            dist, _ = cKDTree(acc, boxsize=L).query(cand, k=1, distance_upper_bound=dmin)
            cand = cand[~(dist < dmin)]
        if len(cand) > 1:
            pr = cKDTree(cand, boxsize=L).query_pairs(dmin, output_type="ndarray")
            if len(pr):
                bad = np.zeros(len(cand), dtype=bool)
                bad[np.maximum(pr[:, 0], pr[:, 1])] = True
                cand = cand[~bad]
        acc = np.concatenate([acc, cand[:need]], axis=0)
    return acc, np.full(3, L)


def maxwell_boltzmann(n: int, temperature: float, mass: float, rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(0.0, np.sqrt(temperature / mass), size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0)
        k = 0.5 * mass * np.sum(v * v)
        target = 0.5 * (3 * n - 3) * temperature
        if k > 0:
            v *= np.sqrt(target / k)
    return v


def random_quaternions(n: int, rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def make_lj(n: int, rho: float = 0.85, temperature: float = 1.0, seed: int = 1000, rc: float = 2.5,
            skin: float = 0.3, dt: float = 0.001, jitter: float = 0.05) -> System:
    rng = _rng(seed)
    pos, box = fcc_positions(n, rho, rng, jitter)
    vel = maxwell_boltzmann(n, temperature, 1.0, rng)
    return System(LJ, pos, vel, box, rc, skin, dt, temperature, name=f"lj_n{n}_rho{rho}")


def make_wca(n: int, rho: float = 0.2, temperature: float = 1.0, seed: int = 1002, skin: float = 0.2,
             dt: float = 0.001) -> System:
    rng = _rng(seed)
    pos, box = rsa_positions(n, rho, rng)
    vel = maxwell_boltzmann(n, temperature, 1.0, rng)
    return System(WCA, pos, vel, box, WCA_RC, skin, dt, temperature, name=f"wca_n{n}_rho{rho}")


def make_patchy(n: int, rho: float = 0.3, temperature: float = 0.15, seed: int = 1003, rc: float = 1.5,
                skin: float = 0.2, dt: float = 0.001, inertia: float = 0.1) -> System:
    rng = _rng(seed)
    pos, box = rsa_positions(n, rho, rng)
    vel = maxwell_boltzmann(n, temperature, 1.0, rng)
    quat = random_quaternions(n, rng)
    L = rng.normal(0.0, np.sqrt(temperature * inertia), size=(n, 3))
    krot = 0.5 * np.sum(L * L) / inertia
    if krot > 0:
        L *= np.sqrt(0.5 * 3 * n * temperature / krot)
    return System(PATCHY, pos, vel, box, rc, skin, dt, temperature, quat=quat, angmom=L, inertia=inertia,
                  patches=PATCH_DIRS * PATCH_RADIUS, name=f"patchy_n{n}_rho{rho}")


def make_patchy_pow(n: int, rho: float = 0.3, temperature: float = 0.15, seed: int = 1005, rc: float = 1.18,
                    patch_rc: float = 0.18, skin: float = 0.2, dt: float = 0.001, inertia: float = 0.1,
                    thermostat_every: int = 100, thermostat_prob: float = 0.1) -> System:
    """The paper's patchy form: (sigma/r)^200 core, two polar patches, patch pairs cut at 0.18 sigma
    (so no centre pair beyond 1 + 0.18 sigma interacts), Brownian momentum refresh at kT."""
    s = make_patchy(n, rho, temperature, seed, rc, skin, dt, inertia)
    s.kind = PATCHY_POW
    s.patches = PATCH_DIRS_POLAR * PATCH_RADIUS
    s.patch_rc = patch_rc
    s.thermostat_every, s.thermostat_prob, s.seed = thermostat_every, thermostat_prob, seed
    s.name = f"patchy_pow_n{n}_rho{rho}"
    return s


def make_lj_nvt(n: int, rho: float, temperature: float = 1.8, seed: int = 1006, thermostat_every: int = 100,
                thermostat_prob: float = 0.1) -> System:
    """Lennard-Jones at the paper's state points (kT = 1.8) with the Brownian momentum refresh."""
    s = make_lj(n, rho, temperature, seed)
    s.thermostat_every, s.thermostat_prob, s.seed = thermostat_every, thermostat_prob, seed
    s.name = f"lj_nvt_n{n}_rho{rho}"
    return s


def batch_specs(n_replicas: int = 512, seed: int = 1004):
    """(kind, N, rho, seed) per replica: N log-uniform in [500, 32768], rho ~ U(0.2, 0.9);
    every fourth replica is WCA at rho = 0.2, the rest LJ with rc = 2.5 sigma."""
    rng = _rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(500.0), np.log(32768.0), size=n_replicas))).astype(int)
    rhos = rng.uniform(0.2, 0.9, size=n_replicas)
    out = []
    for r in range(n_replicas):
        if r % 4 == 0:
            out.append((WCA, int(ns[r]), 0.2, 5000 + r))
        else:
            out.append((LJ, int(ns[r]), float(rhos[r]), 5000 + r))
    return out


def make_replica(kind: int, n: int, rho: float, seed: int) -> System:
    if kind == WCA:
        return make_wca(n, rho, seed=seed)
    return make_lj(n, rho, seed=seed)


# Named workloads (sizes as stated for each).
def config(name: str) -> System:
    if name == "lj4000":
        return make_lj(4000, 0.85, 1.0, seed=1000)
    if name.startswith("lj") and name[2:].isdigit():
        return make_lj(int(name[2:]), 0.85, 1.0, seed=1001)
    if name == "wca1m":
        return make_wca(1_048_576, 0.2, seed=1002)
    if name.startswith("wca") and name[3:].isdigit():
        return make_wca(int(name[3:]), 0.2, seed=1002)
    if name == "patchy262k":
        return make_patchy(262_144, 0.3, seed=1003)
    if name.startswith("patchy") and name[6:].isdigit():
        return make_patchy(int(name[6:]), 0.3, seed=1003)
    raise KeyError(name)

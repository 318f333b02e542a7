"""FP64 CPU oracle for short-range pair forces (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  It shares no code with the CUDA path:
the arithmetic lives in ``md_oracle.c`` (plain C, FP64, no fused multiply-add),
and this module only marshals numpy arrays into it.

Functions (each follows the passage cited in ``md_oracle.c``):
  forces(pos, model, quat=None, use_cells=True)   -> F, T, E, (U, W, n_pairs_in_rc)
  pairs(pos, box, rv, use_cells=True)             -> (N_pairs, 2) int array, i < j, sorted
  run_nve(pos, vel, model, dt, nsteps, ...)       -> per-step {K_trans, K_rot, U, W}
  run(pos, vel, model, dt, nsteps, thermostat=.., step0=..) -> the same with the momentum-refresh thermostat
  philox4x32(ctr, key)                            -> Philox4x32-10 output words
  thermostat_draw(seed, step, particle)           -> (selection uniform, six normals)
  cell_dims(box, rv)                              -> cells per axis the oracle uses
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_LIB = os.path.join(_HERE, "_md_oracle.so")

LJ, WCA, PATCHY, PATCHY_POW = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile md_oracle.c into a shared library beside it (gcc, -O2, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("n_patch", ctypes.c_int32), ("box", ctypes.c_double * 3),
                ("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("rc", ctypes.c_double),
                ("eps_p", ctypes.c_double), ("delta", ctypes.c_double), ("patch", (ctypes.c_double * 3) * 8),
                ("patch_rc", ctypes.c_double)]


class _Thermostat(ctypes.Structure):
    _fields_ = [("every", ctypes.c_int32), ("seed", ctypes.c_uint32), ("prob", ctypes.c_double),
                ("kT", ctypes.c_double)]


@dataclass
class Thermostat:
    """Momentum refresh: at steps s > 0 with s % every == 0 each particle is redrawn with probability prob."""
    every: int
    prob: float
    kT: float
    seed: int = 0

    def to_c(self) -> _Thermostat:
        t = _Thermostat()
        t.every, t.seed, t.prob, t.kT = int(self.every), int(self.seed) & 0xFFFFFFFF, float(self.prob), float(self.kT)
        return t


@dataclass
class Model:
    """Pair model: LJ (rc = 2.5 sigma), WCA, patchy (WCA core + patch attraction), or the paper's patchy
    form PATCHY_POW ((sigma/r)^200 core + patch attraction truncated at patch_rc)."""
    kind: int
    box: tuple
    rc: float
    eps: float = 1.0
    sigma: float = 1.0
    eps_p: float = 1.0
    delta: float = 0.12
    patches: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    patch_rc: float = 0.0

    def to_c(self) -> _Model:
        m = _Model()
        m.model = self.kind
        m.n_patch = len(self.patches)
        for c in range(3):
            m.box[c] = float(self.box[c])
        m.eps, m.sigma, m.rc, m.eps_p, m.delta = self.eps, self.sigma, self.rc, self.eps_p, self.delta
        m.patch_rc = self.patch_rc
        for a, p in enumerate(np.asarray(self.patches, dtype=np.float64)):
            for c in range(3):
                m.patch[a][c] = float(p[c])
        return m


_lib = None
_lib_path = None


def load_library(path=None):
    """Use the oracle library at `path` (None: the one built from md_oracle.c).
    The tests use this to load deliberately broken copies and check that the pins fail."""
    global _lib, _lib_path
    _lib = None
    _lib_path = path
    return _load()


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_lib_path or build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_forces.argtypes = [ctypes.c_int, dp, dp, ctypes.POINTER(_Model), ctypes.c_int, dp, dp, dp, dp]
        lib.oracle_forces.restype = ctypes.c_int
        lib.oracle_pairs.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ip, ip]
        lib.oracle_pairs.restype = ctypes.c_int64
        lib.oracle_cell_dims.argtypes = [dp, ctypes.c_double, ip]
        lib.oracle_cell_dims.restype = None
        lib.oracle_run_nve.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.POINTER(_Model), ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_run_nve.restype = ctypes.c_int
        lib.oracle_run.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.POINTER(_Model), ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp,
                                   ctypes.POINTER(_Thermostat), ctypes.c_int]
        lib.oracle_run.restype = ctypes.c_int
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_philox4x32.argtypes = [u32p, u32p, u32p]
        lib.oracle_philox4x32.restype = None
        lib.oracle_thermostat_draw.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, dp, dp]
        lib.oracle_thermostat_draw.restype = None
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _c64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == shape, (a.shape, shape)
    return a


def forces(pos, model: Model, quat=None, use_cells: bool = True):
    """Total force F[n,3], torque T[n,3], per-particle energy E[n] (half of each pair
    energy) and totals (U, W, pairs inside rc) for positions pos[n,3]."""
    pos = _c64(pos, (len(pos), 3))
    n = len(pos)
    q = _c64(quat, (n, 4)) if quat is not None else None
    F = np.zeros((n, 3)); T = np.zeros((n, 3)); E = np.zeros(n); tot = np.zeros(3)
    m = model.to_c()
    rc = _load().oracle_forces(n, _dp(pos), _dp(q), ctypes.byref(m), int(use_cells), _dp(F),
                               _dp(T) if model.kind in (PATCHY, PATCHY_POW) else None, _dp(E), _dp(tot))
    if rc != 0:
        raise MemoryError("oracle_forces failed")
    return F, T, E, (tot[0], tot[1], int(tot[2]))


def pairs(pos, box, rv: float, use_cells: bool = True) -> np.ndarray:
    """Sorted (i, j), i < j, of every minimum-image pair with r^2 < rv^2."""
    pos = _c64(pos, (len(pos), 3))
    n = len(pos)
    b = np.asarray(box, dtype=np.float64)
    cap = max(16, int(n * 64))
    while True:
        pi = np.empty(cap, dtype=np.int32); pj = np.empty(cap, dtype=np.int32)
        cnt = _load().oracle_pairs(n, _dp(pos), _dp(b), float(rv), int(use_cells), cap,
                                   pi.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   pj.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if cnt < 0:
            raise MemoryError("oracle_pairs failed")
        if cnt <= cap:
            break
        cap = int(cnt)
    out = np.stack([pi[:cnt], pj[:cnt]], axis=1).astype(np.int64)
    order = np.lexsort((out[:, 1], out[:, 0]))
    return out[order]


def cell_dims(box, rv: float):
    b = np.asarray(box, dtype=np.float64)
    nc = np.zeros(3, dtype=np.int32)
    _load().oracle_cell_dims(_dp(b), float(rv), nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return tuple(int(x) for x in nc)


def run_nve(pos, vel, model: Model, dt: float, nsteps: int, mass: float = 1.0, inertia: float = 0.1,
            quat=None, angmom=None, use_cells: bool = True):
    """Velocity Verlet in place on copies; returns (pos, vel, quat, angmom, trace[nsteps+1, 4])."""
    n = len(pos)
    pos = _c64(pos, (n, 3)).copy(); vel = _c64(vel, (n, 3)).copy()
    q = _c64(quat, (n, 4)).copy() if quat is not None else None
    L = _c64(angmom, (n, 3)).copy() if angmom is not None else None
    trace = np.zeros((nsteps + 1, 4))
    m = model.to_c()
    rc = _load().oracle_run_nve(n, _dp(pos), _dp(vel), _dp(q), _dp(L), ctypes.byref(m), float(dt), float(mass),
                                float(inertia), int(nsteps), int(use_cells), _dp(trace))
    if rc != 0:
        raise MemoryError("oracle_run_nve failed")
    return pos, vel, q, L, trace


def run(pos, vel, model: Model, dt: float, nsteps: int, mass: float = 1.0, inertia: float = 0.1,
        quat=None, angmom=None, use_cells: bool = True, thermostat: Thermostat | None = None, step0: int = 0):
    """Velocity Verlet with the optional momentum-refresh thermostat, steps numbered from step0."""
    n = len(pos)
    pos = _c64(pos, (n, 3)).copy(); vel = _c64(vel, (n, 3)).copy()
    q = _c64(quat, (n, 4)).copy() if quat is not None else None
    L = _c64(angmom, (n, 3)).copy() if angmom is not None else None
    trace = np.zeros((nsteps + 1, 4))
    m = model.to_c()
    th = thermostat.to_c() if thermostat is not None else None
    rc = _load().oracle_run(n, _dp(pos), _dp(vel), _dp(q), _dp(L), ctypes.byref(m), float(dt), float(mass),
                            float(inertia), int(nsteps), int(use_cells), _dp(trace),
                            ctypes.byref(th) if th is not None else None, int(step0))
    if rc != 0:
        raise MemoryError("oracle_run failed")
    return pos, vel, q, L, trace


def philox4x32(ctr, key):
    """Philox4x32-10 of counter ctr[4] and key key[2] (uint32 words)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32); k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    p = ctypes.POINTER(ctypes.c_uint32)
    _load().oracle_philox4x32(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def thermostat_draw(seed: int, step: int, particle: int):
    """The thermostat's selection uniform and six standard normals for one particle and step."""
    u = np.zeros(1); nrm = np.zeros(6)
    _load().oracle_thermostat_draw(int(seed) & 0xFFFFFFFF, int(step), int(particle), _dp(u), _dp(nrm))
    return float(u[0]), nrm

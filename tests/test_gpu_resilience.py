"""Checkpoint / resume and host-injected faults (no GPU fault is caused: the planted values are ordinary
inputs that the device checks turn into status codes)."""
import numpy as np
import pytest

from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems
from tests.test_gpu_parity import Sim, get_sys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1401_4350_gb300 import build
    build.build()
    B.load()
    yield
    B.md_release_graphs()


@pytest.mark.parametrize("precision", [B.MD_MIXED, B.MD_FP64])
@pytest.mark.parametrize("name", ["lj4000", "patchy6000"])
def test_resume_reproduces_forces_and_the_continued_run(tmp_path, name, precision):
    s = get_sys(name)
    if name == "lj4000":  # with the momentum refresh, whose random numbers are keyed by the step counter
        s = systems.make_lj_nvt(4000, 0.85, temperature=1.0, seed=1000, thermostat_every=5, thermostat_prob=0.5)
    a = Sim(s, precision, prune_skin=0.1 if precision == B.MD_MIXED and name == "lj4000" else 0.0)
    a.prepare(B.MD_VERTEX)
    a.step(33, B.MD_VERTEX)
    f = tmp_path / "ckpt.npz"
    a.checkpoint(f)
    a.prepare(B.MD_VERTEX)  # forces at the checkpointed state, from fresh cells and lists
    Fa = a.forces()
    b = Sim(s, precision, prune_skin=0.1 if precision == B.MD_MIXED and name == "lj4000" else 0.0)
    b.resume(f, B.MD_VERTEX)
    Fb = b.forces()
    for x, y in zip(Fa, Fb):
        if x is not None:
            assert np.array_equal(x, y)
    assert b.status()[B.MD_STATUS_STEPS] == a.status()[B.MD_STATUS_STEPS] == 33
    for sim in (a, b):
        sim.step(21, B.MD_VERTEX)
    xa, va = a.positions()
    xb, vb = b.positions()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_resume_rejects_another_system(tmp_path):
    a = Sim(get_sys("lj4000"), B.MD_MIXED)
    a.prepare(B.MD_VERTEX)
    f = tmp_path / "ckpt.npz"
    a.checkpoint(f)
    b = Sim(get_sys("lj5003"), B.MD_MIXED)
    with pytest.raises(ValueError):
        b.resume(f)


@pytest.mark.parametrize("precision", [B.MD_MIXED, B.MD_FP64])
@pytest.mark.parametrize("fuse", [1, 0])
def test_planted_nan_velocity_is_reported(precision, fuse):
    """A NaN velocity makes the drifted position non-finite: the step records MD_ERR_NONFINITE in the status
    (positions of the other particles stay finite; nothing faults)."""
    import torch
    s = get_sys("lj4000")
    sim = Sim(s, precision, fuse_step=fuse)
    sim.prepare(B.MD_VERTEX)
    assert sim.status()[B.MD_STATUS_CODE] == 0
    sim.vel[17, 0] = float("nan")
    sim.step(3, B.MD_VERTEX)
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == B.MD_ERR_NONFINITE, st
    torch.cuda.synchronize()

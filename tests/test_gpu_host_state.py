"""md_step_verlet_host: velocity-Verlet steps (Sec. Methods) with the state kept in host memory give the
trajectory of the device-resident md_step_verlet bit for bit, through rebuilds that reorder the slots."""
import pytest
import torch

from paper_1401_4350_gb300 import binding as B
from paper_1401_4350_gb300 import systems
from paper_1401_4350_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


# deterministic paths only: the atomic edge path sums in no fixed order, so two runs of it differ in rounding
@pytest.mark.parametrize("fuse,prune,path,pin", [
    (1, 0.1, B.MD_VERTEX, True),   # fused steps over the inner list
    (0, 0.0, B.MD_VERTEX, True),
    (0, 0.0, B.MD_EDGE_STORE, True),
    (1, 0.0, B.MD_VERTEX, False),  # pageable host memory: synchronous copies, same results
])
def test_host_state_matches_device(fuse, prune, path, pin):
    s = systems.make_lj(4000, 0.85, 1.0, seed=11)
    kw = dict(fuse_step=fuse, prune_skin=prune, edge_store=int(path == B.MD_EDGE_STORE))
    a = Simulation(s, B.MD_MIXED, **kw)
    b = Simulation(s, B.MD_MIXED, **kw)
    a.prepare(path)
    b.prepare(path)
    hp, hv = b.slot_state_host(pin=pin)
    he = torch.empty(B.MD_ENERGY_WORDS, dtype=torch.float64, pin_memory=pin)
    for _ in range(20):
        a.step(5, path)
        b.step_host(hp, hv, 5, path, host_energy=he)
    torch.cuda.synchronize()
    sa, sb = a.status(), b.status()
    assert sa[B.MD_STATUS_CODE] == 0 and sb[B.MD_STATUS_CODE] == 0
    assert sa[B.MD_STATUS_REBUILDS] >= 2 and sb[B.MD_STATUS_REBUILDS] == sa[B.MD_STATUS_REBUILDS]
    assert torch.equal(b.id, a.id)  # the slots were reordered the same way
    assert torch.equal(hp, a.pos[:, :3].cpu()) and torch.equal(hv, a.vel[:, :3].cpu())
    assert torch.equal(b.pos[:, :3], a.pos[:, :3]) and torch.equal(b.vel[:, :3], a.vel[:, :3])
    assert torch.equal(he, a.view("energy", torch.float64, B.MD_ENERGY_WORDS).cpu())


def test_host_state_edge_atomic():
    """The atomic edge path: what comes back to the host is the device state the call left."""
    s = systems.make_lj(4000, 0.85, 1.0, seed=13)
    sim = Simulation(s, B.MD_MIXED, fuse_step=0)
    sim.prepare(B.MD_EDGE)
    hp, hv = sim.slot_state_host()
    for _ in range(20):
        sim.step_host(hp, hv, 5, B.MD_EDGE)
    torch.cuda.synchronize()
    st = sim.status()
    assert st[B.MD_STATUS_CODE] == 0 and st[B.MD_STATUS_REBUILDS] >= 1
    assert torch.equal(hp, sim.pos[:, :3].cpu()) and torch.equal(hv, sim.vel[:, :3].cpu())


def test_zero_steps_round_trip():
    """nsteps = 0 copies the state in and back out unchanged."""
    s = systems.make_lj(4000, 0.85, 1.0, seed=12)
    sim = Simulation(s, B.MD_MIXED)
    sim.prepare(B.MD_VERTEX)
    hp, hv = sim.slot_state_host()
    hp0, hv0 = hp.clone(), hv.clone()
    sim.step_host(hp, hv, 0, B.MD_VERTEX)
    torch.cuda.synchronize()
    assert torch.equal(hp, hp0) and torch.equal(hv, hv0)
    assert torch.equal(sim.pos[:, :3].cpu(), hp0)


def test_device_arrays_are_rejected():
    """Device (or managed) arrays are not host arrays: the call refuses them before enqueueing anything,
    instead of staging them through host-to-device copies of the wrong kind."""
    s = systems.make_lj(4000, 0.85, 1.0, seed=14)
    sim = Simulation(s, B.MD_MIXED)
    sim.prepare(B.MD_VERTEX)
    dp = sim.pos[:, :3].contiguous()
    dv = sim.vel[:, :3].contiguous()
    pos0 = sim.pos.clone()
    with pytest.raises(B.MDError) as err:
        B.md_step_verlet_host(sim.params, sim.state(), sim.ws, dp, dv, None, 1, B.MD_VERTEX, True, sim._st())
    assert err.value.code == B.MD_ERR_INVALID and "device" in str(err.value)
    hp, hv = sim.slot_state_host()
    with pytest.raises(B.MDError):
        B.md_step_verlet_host(sim.params, sim.state(), sim.ws, hp, dv, None, 1, B.MD_VERTEX, True, sim._st())
    torch.cuda.synchronize()
    assert torch.equal(sim.pos, pos0) and sim.status()[B.MD_STATUS_STEPS] == 0

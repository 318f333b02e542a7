"""Simulation: caller-side owner of the device memory of one system.

Allocates the FP64 state and the library workspace as torch CUDA tensors, fills md_params from a
systems.System, and exposes the library's results (forces, lists, energies) in the caller's
original particle order.  All computation happens in libmdgb.so.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B
from .systems import System, LJ, WCA, PATCHY, PATCHY_POW, PATCHY_KINDS


def default_capacities(system: System, slack: float = 1.6):
    """Full-list columns and half-list pairs for the system's density with head-room."""
    rho = system.n / float(np.prod(system.box))
    nbar = 4.0 / 3.0 * math.pi * system.rv ** 3 * rho
    max_neigh = int(slack * nbar + 24)
    max_pairs = int(system.n * (0.5 * slack * nbar + 12)) + 1024
    return max_neigh, max_pairs


def make_params(system: System, precision: int, max_neigh=None, max_pairs=None, tpp: int = 1, block: int = 0,
                trace_capacity: int = 0, energy_every: int = 1, force_copies: int = 0,
                cell_order: int = 0, edge_store: int = 0, list_format: int = 0, fuse_step: int = 0,
                prune_skin: float = 0.0) -> B.md_params:
    mn, mp = default_capacities(system)
    p = B.md_params()
    p.n = system.n
    p.model = {LJ: B.MD_LJ, WCA: B.MD_WCA, PATCHY: B.MD_PATCHY, PATCHY_POW: B.MD_PATCHY_POW}[system.kind]
    p.precision = precision
    p.max_neigh = int(max_neigh or mn)
    p.max_pairs = int(max_pairs or mp)
    p.n_patch = len(system.patches) if system.kind in PATCHY_KINDS else 0
    p.threads_per_particle = tpp
    p.block_size = block
    p.trace_capacity = trace_capacity
    p.energy_every = energy_every
    p.force_copies = force_copies
    p.cell_order = cell_order
    p.edge_store = edge_store
    p.list_format = list_format
    p.fuse_step = fuse_step
    p.prune_skin = float(prune_skin)
    for c in range(3):
        p.box[c] = float(system.box[c])
    p.rc, p.skin, p.dt, p.mass, p.inertia = system.rc, system.skin, system.dt, system.mass, system.inertia
    p.eps, p.sigma, p.eps_p, p.delta = system.eps, system.sigma, system.eps_p, system.delta
    for a, v in enumerate(np.asarray(system.patches)):
        for c in range(3):
            p.patch[a][c] = float(v[c])
    p.patch_rc = float(system.patch_rc)
    p.kT = float(system.temperature)
    p.thermostat_every = int(system.thermostat_every)
    p.thermostat_prob = float(system.thermostat_prob)
    p.seed = int(system.seed) & 0xFFFFFFFF
    return p


class Simulation:
    def __init__(self, system: System, precision: int = B.MD_MIXED, max_neigh=None, max_pairs=None, tpp: int = 1,
                 block: int = 0, trace_capacity: int = 0, device: str = "cuda", stream=None, energy_every: int = 1,
                 force_copies: int = 0, cell_order: int = 0, edge_store: int = 0, list_format: int = 0,
                 fuse_step: int = 1, prune_skin: float = 0.0):
        self.system = system
        self.params = make_params(system, precision, max_neigh, max_pairs, tpp, block, trace_capacity, energy_every,
                                  force_copies, cell_order, edge_store, list_format, fuse_step, prune_skin)
        rc = B.md_check_params(self.params)
        if rc != B.MD_OK:
            raise B.MDError(rc, B.last_error())
        self.layout = B.md_workspace_layout(self.params)
        self.device = torch.device(device)
        self.stream = stream
        n = system.n
        f64 = dict(dtype=torch.float64, device=self.device)
        self.pos = torch.zeros((n, 4), **f64)
        self.vel = torch.zeros((n, 4), **f64)
        self.quat = torch.zeros((n, 4), **f64) if system.kind in PATCHY_KINDS else None
        self.angmom = torch.zeros((n, 4), **f64) if system.kind in PATCHY_KINDS else None
        self.id = torch.arange(n, dtype=torch.int32, device=self.device)
        self.ws = torch.empty(int(self.layout.total), dtype=torch.uint8, device=self.device)
        assert self.ws.data_ptr() % 256 == 0
        self.load_state(system.pos, system.vel, system.quat, system.angmom)
        B.md_init_workspace(self.params, self.ws, self._st())

    # -- plumbing ---------------------------------------------------------------------------------
    def _st(self):
        return self.stream

    def state(self) -> B.md_state:
        s = B.md_state()
        s.pos, s.vel, s.id = self.pos.data_ptr(), self.vel.data_ptr(), self.id.data_ptr()
        s.quat = self.quat.data_ptr() if self.quat is not None else None
        s.angmom = self.angmom.data_ptr() if self.angmom is not None else None
        return s

    def load_state(self, pos, vel, quat=None, angmom=None):
        n = self.system.n
        self.pos[:, :3] = torch.as_tensor(np.asarray(pos, dtype=np.float64), device=self.device)
        self.vel[:, :3] = torch.as_tensor(np.asarray(vel, dtype=np.float64), device=self.device)
        if self.quat is not None:
            self.quat[:] = torch.as_tensor(np.asarray(quat, dtype=np.float64), device=self.device)
            self.angmom[:, :3] = torch.as_tensor(np.asarray(angmom, dtype=np.float64), device=self.device)
        self.id.copy_(torch.arange(n, dtype=torch.int32, device=self.device))

    def view(self, name: str, dtype, count: int):
        off = getattr(self.layout, name)
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + nbytes].view(dtype)

    # -- the C ABI --------------------------------------------------------------------------------
    def build_cells(self):
        B.md_build_cells(self.params, self.state(), self.ws, self._st())

    def build_verlet(self, which=B.MD_LIST_BOTH):
        B.md_build_verlet(self.params, self.state(), self.ws, which, self._st())

    def forces_vertex(self):
        B.md_forces_vertex(self.params, self.state(), self.ws, self._st())

    def forces_edge(self):
        B.md_forces_edge(self.params, self.state(), self.ws, self._st())

    def forces_vertex_newton(self):
        B.md_forces_vertex_newton(self.params, self.state(), self.ws, self._st())

    def forces_edge_store(self):
        B.md_forces_edge_store(self.params, self.state(), self.ws, self._st())

    def autotune(self):
        """Choose the fastest path, threads per particle and block size by timing every available
        candidate (binding.TUNE_CANDIDATES); returns (path, threads_per_particle, block_size, median ms per
        candidate).  self.params is updated; lists and forces stay prepared for the choice."""
        return B.md_autotune_system(self.params, self.state(), self.ws, self._st())

    def time_step_kernel(self, path=B.MD_VERTEX, reps: int = 20) -> float:
        """Mean ms of the kernel one step of `path` runs (the fused step kernel where fuse_step applies,
        else the force kernel); the system is left as it was."""
        return B.md_time_step_kernel(self.params, self.state(), self.ws, path, reps, self._st())

    def prepare(self, path=B.MD_VERTEX):
        B.md_prepare(self.params, self.state(), self.ws, path, self._st())

    def step(self, nsteps: int, path=B.MD_VERTEX, use_graph=True):
        B.md_step_verlet(self.params, self.state(), self.ws, nsteps, path, use_graph, self._st())

    def step_host(self, host_pos, host_vel, nsteps: int, path=B.MD_VERTEX, use_graph=True, host_energy=None):
        """nsteps with the state in host memory: host_pos / host_vel are contiguous [n][3] float64 CPU tensors
        (pinned for full bandwidth) in slot order, read and overwritten in stream order (synchronise the
        stream before reading them); host_energy, if given, receives the MD_ENERGY_WORDS energy words."""
        for t in (host_pos, host_vel):
            if t.device.type != "cpu" or t.dtype != torch.float64 or tuple(t.shape) != (self.system.n, 3) or not t.is_contiguous():
                raise ValueError("host_pos and host_vel must be contiguous [n][3] float64 CPU tensors")
        B.md_step_verlet_host(self.params, self.state(), self.ws, host_pos, host_vel, host_energy, nsteps, path,
                              use_graph, self._st())

    def slot_state_host(self, pin=True):
        """The current (pos, vel) as [n][3] float64 CPU tensors in slot order, the layout step_host takes."""
        pos = torch.empty((self.system.n, 3), dtype=torch.float64, pin_memory=pin)
        vel = torch.empty((self.system.n, 3), dtype=torch.float64, pin_memory=pin)
        pos.copy_(self.pos[:, :3])
        vel.copy_(self.vel[:, :3])
        return pos, vel

    def status(self):
        return B.md_read_status(self.params, self.ws, self._st())

    # -- checkpoint / resume -------------------------------------------------------------------------
    def checkpoint(self, path):
        """Writes the dynamic state to an .npz file: FP64 positions and velocities (and, patchy, orientations and
        angular momenta) in slot order with each slot's original particle id, the step counter (which also
        keys the thermostat's random numbers), the box and the particle count.  Slot order is kept so that a
        resumed run sorts its cells, and so sums its forces, exactly as the original would."""
        extra = {}
        if self.quat is not None:
            extra = {"quat": self.quat.cpu().numpy(), "angmom": self.angmom[:, :3].cpu().numpy()}
        st = self.status()
        np.savez(path, pos=self.pos[:, :3].cpu().numpy(), vel=self.vel[:, :3].cpu().numpy(),
                 id=self.id.cpu().numpy(), step=np.int64(st[B.MD_STATUS_STEPS]),
                 box=np.asarray(self.system.box, float), n=np.int64(self.system.n), **extra)

    def resume(self, path, path_kind=B.MD_VERTEX):
        """Loads a checkpoint written by checkpoint() for the same system, restores the step counter and
        prepares cells, lists and forces for `path_kind`."""
        d = np.load(path)
        if int(d["n"]) != self.system.n or not np.array_equal(d["box"], np.asarray(self.system.box, float)):
            raise ValueError("the checkpoint is of another system (particle count or box differ)")
        ids = np.asarray(d["id"])
        if not np.array_equal(np.sort(ids), np.arange(self.system.n)):
            raise ValueError("the checkpoint's particle ids are not a permutation")
        self.pos[:, :3] = torch.as_tensor(d["pos"], dtype=torch.float64, device=self.device)
        self.vel[:, :3] = torch.as_tensor(d["vel"], dtype=torch.float64, device=self.device)
        if self.quat is not None:
            self.quat[:] = torch.as_tensor(d["quat"], dtype=torch.float64, device=self.device)
            self.angmom[:, :3] = torch.as_tensor(d["angmom"], dtype=torch.float64, device=self.device)
        self.id.copy_(torch.as_tensor(ids, dtype=torch.int32, device=self.device))
        B.md_init_workspace(self.params, self.ws, self._st())
        self.view("status", torch.int32, B.MD_STATUS_WORDS)[B.MD_STATUS_STEPS] = int(d["step"])
        self.prepare(path_kind)

    # -- results in the caller's original order -------------------------------------------------
    def _order(self):
        return self.id.long()

    def forces(self):
        """(F[n,3], E_i[n], T[n,3] or None, W_i[n]) as FP64 numpy arrays in the original order."""
        n = self.system.n
        fo = torch.empty((n, 4), dtype=torch.float64, device=self.device)
        to = torch.empty((n, 4), dtype=torch.float64, device=self.device)
        B.md_get_forces(self.params, self.ws, fo, to, self._st())
        torch.cuda.synchronize(self.device)
        inv = torch.empty_like(self._order())
        inv[self._order()] = torch.arange(n, device=self.device)
        fo = fo[inv].cpu().numpy()
        to = to[inv].cpu().numpy()
        T = to[:, :3] if self.system.kind in PATCHY_KINDS else None
        return fo[:, :3], fo[:, 3], T, to[:, 3]

    def positions(self):
        inv = torch.empty_like(self._order())
        inv[self._order()] = torch.arange(self.system.n, device=self.device)
        return self.pos[inv, :3].cpu().numpy(), self.vel[inv, :3].cpu().numpy()

    def orientations(self):
        inv = torch.empty_like(self._order())
        inv[self._order()] = torch.arange(self.system.n, device=self.device)
        return self.quat[inv].cpu().numpy(), self.angmom[inv, :3].cpu().numpy()

    def energies(self):
        e = self.view("energy", torch.float64, B.MD_ENERGY_WORDS)
        torch.cuda.synchronize(self.device)
        e = e.cpu().numpy()
        return {"U": e[B.MD_ENERGY_U], "KT": e[B.MD_ENERGY_KT], "KR": e[B.MD_ENERGY_KR], "W": e[B.MD_ENERGY_W]}

    def trace(self):
        t = self.view("trace", torch.float64, 4 * self.params.trace_capacity).view(-1, 4)
        torch.cuda.synchronize(self.device)
        return t.cpu().numpy()

    def full_list_pairs(self):
        """Sorted unique (i, j), i < j, in original ids, from the full list; also checks symmetry."""
        n = self.system.n
        cnt = self.view("nbr_count", torch.int32, n).long()
        cap = self.params.max_neigh
        ng = (cap + 3) // 4
        nbr = self.view("nbr", torch.int32, ng * n * 4).view(ng, n, 4).permute(0, 2, 1).reshape(ng * 4, n)[:cap]
        k = torch.arange(cap, device=self.device)[:, None]
        mask = k < cnt[None, :]
        jj = nbr[mask].long()
        ii = torch.arange(n, device=self.device)[None, :].expand(cap, n)[mask]
        ids = self._order()
        oi, oj = ids[ii], ids[jj]
        a, b = torch.minimum(oi, oj), torch.maximum(oi, oj)
        key = a * n + b
        key, counts = torch.unique(key, return_counts=True)
        return (torch.stack([key // n, key % n], 1).cpu().numpy(), counts.cpu().numpy(), int(mask.sum()))

    def list_rows(self, name: str = "nbr", count: str = "nbr_count"):
        """Rows of a grouped list (the Verlet list nbr, or the inner list nbr_in) as slot indices, in slot order."""
        n = self.system.n
        cnt = self.view(count, torch.int32, n).cpu().numpy()
        cap = self.params.max_neigh
        ng = (cap + 3) // 4
        tab = self.view(name, torch.int32, ng * n * 4).view(ng, n, 4).permute(1, 0, 2).reshape(n, ng * 4)
        tab = tab.cpu().numpy()
        return [tab[i, :min(int(cnt[i]), cap)] for i in range(n)]

    def local_list_pairs(self):
        """Like full_list_pairs, for a full list held in the block-local format: each uint16 entry is a halo
        position, mapped to a slot through its block's cell table (first slot, halo offset)."""
        n = self.system.n
        cnt = self.view("nbr_count", torch.int32, n).long()
        cap = self.params.max_neigh
        ng = (cap + 3) // 4
        raw = self.view("nbr", torch.int16, ng * n * 4).view(ng, n, 4).permute(0, 2, 1).reshape(ng * 4, n)[:cap]
        loc = raw.long() & 0xFFFF
        nblk = (n + B.MD_LOCAL_BLOCK - 1) // B.MD_LOCAL_BLOCK
        rec = 4 + 2 * B.MD_LOCAL_MAX_CELLS
        tab = self.ws[self.layout.local_tab:self.layout.local_tab + 4 * rec * nblk].view(torch.int32).view(nblk, rec)
        U = tab[:, 0].long()
        first = tab[:, 4::2].long()
        off = tab[:, 5::2].long()
        big = torch.iinfo(torch.int64).max
        cell_idx = torch.arange(B.MD_LOCAL_MAX_CELLS, device=self.device)[None, :]
        off_masked = torch.where(cell_idx < U[:, None], off, torch.full_like(off, big))
        k = torch.arange(cap, device=self.device)[:, None]
        mask = k < cnt[None, :]
        ii = torch.arange(n, device=self.device)[None, :].expand(cap, n)[mask]
        v = loc[mask]
        blk = ii // B.MD_LOCAL_BLOCK
        u = torch.searchsorted(off_masked[blk], v[:, None], right=True).squeeze(1) - 1
        jj = first[blk, u] + (v - off[blk, u])
        ids = self._order()
        oi, oj = ids[ii], ids[jj]
        a, b = torch.minimum(oi, oj), torch.maximum(oi, oj)
        key, counts = torch.unique(a * n + b, return_counts=True)
        return (torch.stack([key // n, key % n], 1).cpu().numpy(), counts.cpu().numpy(), int(mask.sum()))

    def half_list_pairs(self):
        n = self.system.n
        hs = self.view("half_start", torch.int64, n + 1)
        total = int(hs[-1].item())
        # rows of the CSR list: slot i holds half_start[i + 1] - half_start[i] partners
        ii = torch.repeat_interleave(torch.arange(n, device=self.device), hs[1:] - hs[:-1])
        pairs = torch.stack([ii, self.view("half_j", torch.int32, total).long()], 1)
        ids = self._order()
        oi, oj = ids[pairs[:, 0]], ids[pairs[:, 1]]
        a, b = torch.minimum(oi, oj), torch.maximum(oi, oj)
        key = torch.sort(a * n + b).values
        ordered = bool((pairs[:, 0] < pairs[:, 1]).all()) and bool((pairs[1:, 0] >= pairs[:-1, 0]).all())
        return torch.stack([key // n, key % n], 1).cpu().numpy(), ordered


class BatchSimulation:
    """Many independent mixed-precision LJ/WCA systems stepped together (md_batch_*).

    The state arrays of all replicas are concatenated in replica order; replica r's sub-workspace is
    an ordinary single-system workspace at byte offset md_batch_replica_offset(r), so the
    single-system entry points (md_get_forces, md_read_status) work on it directly.
    """

    def __init__(self, system_list, paths=None, tpps=None, trace_capacity: int = 0, energy_every: int = 1,
                 device: str = "cuda", stream=None, force_copies: int = 0):
        self.systems = list(system_list)
        tpps = tpps or [1] * len(self.systems)
        self.params = [make_params(s, B.MD_MIXED, tpp=int(t), trace_capacity=trace_capacity,
                                   energy_every=energy_every, force_copies=force_copies)
                       for s, t in zip(self.systems, tpps)]
        self.nrep = len(self.systems)
        self.counts = [s.n for s in self.systems]
        self.offsets = np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)
        self.device = torch.device(device)
        self.stream = stream
        total = int(self.offsets[-1])
        f64 = dict(dtype=torch.float64, device=self.device)
        self.pos = torch.zeros((total, 4), **f64)
        self.vel = torch.zeros((total, 4), **f64)
        self.id = torch.zeros(total, dtype=torch.int32, device=self.device)
        for r, s in enumerate(self.systems):
            a, b = int(self.offsets[r]), int(self.offsets[r + 1])
            self.pos[a:b, :3] = torch.as_tensor(s.pos, device=self.device)
            self.vel[a:b, :3] = torch.as_tensor(s.vel, device=self.device)
            self.id[a:b] = torch.arange(s.n, dtype=torch.int32, device=self.device)
        nbytes = B.md_batch_workspace_bytes(self.params)
        if nbytes == 0:
            raise B.MDError(B.MD_ERR_INVALID, B.last_error())
        self.ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        self.ws_offsets = [B.md_batch_replica_offset(self.params, r) for r in range(self.nrep)]
        self.layouts = [B.md_workspace_layout(p) for p in self.params]
        st = B.md_state()
        st.pos, st.vel, st.id = self.pos.data_ptr(), self.vel.data_ptr(), self.id.data_ptr()
        st.quat = st.angmom = None
        self._state = st
        B.md_batch_init(self.params, st, self.ws, paths, stream)

    def release(self):
        B.md_batch_release(self.ws)

    # -- the C ABI --------------------------------------------------------------------------------
    def prepare(self):
        B.md_batch_prepare(self.ws, self.stream)

    def forces_eval(self):
        B.md_batch_forces(self.ws, self.stream)

    def step(self, nsteps: int, use_graph: bool = True):
        B.md_batch_step(self.ws, nsteps, use_graph, self.stream)

    def set_config(self, paths=None, tpps=None):
        B.md_batch_set_config(self.ws, paths, tpps, self.stream)

    def config(self):
        return B.md_batch_get_config(self.ws, self.nrep)

    def autotune(self):
        return B.md_autotune(self.ws, self.nrep, self.stream)

    # -- per-replica results in the original order ------------------------------------------------
    def _ws(self, r):
        return self.ws[self.ws_offsets[r]:]

    def _inv(self, r):
        a, b = int(self.offsets[r]), int(self.offsets[r + 1])
        ids = self.id[a:b].long()
        inv = torch.empty_like(ids)
        inv[ids] = torch.arange(b - a, device=self.device)
        return inv

    def replica_forces(self, r):
        n = self.counts[r]
        fo = torch.empty((n, 4), dtype=torch.float64, device=self.device)
        to = torch.empty((n, 4), dtype=torch.float64, device=self.device)
        B.md_get_forces(self.params[r], self._ws(r), fo, to, self.stream)
        torch.cuda.synchronize(self.device)
        inv = self._inv(r)
        fo, to = fo[inv].cpu().numpy(), to[inv].cpu().numpy()
        return fo[:, :3], fo[:, 3], to[:, 3]

    def replica_positions(self, r):
        a = int(self.offsets[r])
        inv = self._inv(r)
        return self.pos[a:a + self.counts[r]][inv, :3].cpu().numpy(), self.vel[a:a + self.counts[r]][inv, :3].cpu().numpy()

    def replica_status(self, r):
        return B.md_read_status(self.params[r], self._ws(r), self.stream)

    def replica_trace(self, r):
        """Replica r's energy trace: (step, K, U, W) rows, as md_step_verlet's trace of a single system."""
        L = self.layouts[r]
        cap = self.params[r].trace_capacity
        off = self.ws_offsets[r] + L.trace
        t = self.ws[off:off + 32 * cap].view(torch.float64).view(-1, 4)
        torch.cuda.synchronize(self.device)
        return t.cpu().numpy()

    def replica_energies(self, r):
        L = self.layouts[r]
        off = self.ws_offsets[r] + L.energy
        e = self.ws[off:off + 8 * B.MD_ENERGY_WORDS].view(torch.float64)
        torch.cuda.synchronize(self.device)
        e = e.cpu().numpy()
        return {"U": e[B.MD_ENERGY_U], "KT": e[B.MD_ENERGY_KT], "W": e[B.MD_ENERGY_W]}

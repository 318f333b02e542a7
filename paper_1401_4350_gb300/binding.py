"""Thin Python binding of libmdgb.so (the C ABI of include/md.h).

Argument marshalling only: every step of the force path runs in the library's CUDA kernels.
Device memory comes from torch tensors (their data pointers are passed through), streams are
torch CUDA streams.  Importing this module does not need a GPU; loading the library does not
either, but every compute call does.  A missing library raises at load time: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB_PATH = os.path.join(PKG, "libmdgb.so")
HEADER = os.path.join(ROOT, "include", "md.h")

MD_OK, MD_ERR_INVALID, MD_ERR_CUDA, MD_ERR_NEIGH_OVERFLOW, MD_ERR_NONFINITE, MD_ERR_TIMEOUT, MD_ERR_UNSUPPORTED = range(7)
MD_LJ, MD_WCA, MD_PATCHY, MD_PATCHY_POW = 0, 1, 2, 3
MD_FP64, MD_MIXED = 0, 1
MD_VERTEX, MD_EDGE, MD_VERTEX_NEWTON, MD_EDGE_STORE = 0, 1, 2, 3
MD_ORDER_ROWS, MD_ORDER_HILBERT = 0, 1
MD_LIST_FULL, MD_LIST_HALF, MD_LIST_BOTH, MD_LIST_NEWTON = 1, 2, 3, 4
MD_LIST_FULL_LOCAL, MD_LOCAL_BLOCK, MD_LOCAL_MAX_CELLS = 8, 256, 512
MD_FORMAT_GLOBAL, MD_FORMAT_LOCAL = 0, 1
MD_MAX_PATCH = 4
MD_STATUS_CODE, MD_STATUS_NEED_NEIGH, MD_STATUS_NEED_PAIRS_LO, MD_STATUS_NEED_PAIRS_HI = 0, 1, 2, 3
MD_STATUS_REBUILDS, MD_STATUS_STEPS, MD_STATUS_LISTS, MD_STATUS_PRUNES, MD_STATUS_WORDS = 4, 5, 6, 7, 16
MD_ENERGY_U, MD_ENERGY_KT, MD_ENERGY_KR, MD_ENERGY_W, MD_ENERGY_WORDS = 0, 1, 2, 3, 8


class md_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("model", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_neigh", ctypes.c_int32), ("max_pairs", ctypes.c_int64), ("n_patch", ctypes.c_int32),
                ("threads_per_particle", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("trace_capacity", ctypes.c_int32), ("energy_every", ctypes.c_int32), ("force_copies", ctypes.c_int32),
                ("cell_order", ctypes.c_int32), ("edge_store", ctypes.c_int32),
                ("list_format", ctypes.c_int32), ("fuse_step", ctypes.c_int32),
                ("box", ctypes.c_double * 3), ("rc", ctypes.c_double),
                ("skin", ctypes.c_double), ("dt", ctypes.c_double), ("mass", ctypes.c_double),
                ("inertia", ctypes.c_double), ("eps", ctypes.c_double), ("sigma", ctypes.c_double),
                ("eps_p", ctypes.c_double), ("delta", ctypes.c_double),
                ("patch", (ctypes.c_double * 3) * MD_MAX_PATCH), ("patch_rc", ctypes.c_double),
                ("kT", ctypes.c_double), ("thermostat_prob", ctypes.c_double),
                ("thermostat_every", ctypes.c_int32), ("seed", ctypes.c_uint32), ("prune_skin", ctypes.c_double)]


class md_state(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("angmom", ctypes.c_void_p), ("id", ctypes.c_void_p)]


class md_ws_layout(ctypes.Structure):
    _fields_ = [("total", ctypes.c_size_t), ("ncell", ctypes.c_int32 * 3), ("force_elem", ctypes.c_int32)] + [
        (name, ctypes.c_size_t) for name in
        ("status", "energy", "cell_start", "fxp", "fxp_build", "patch_lab", "nbr", "nbr_count", "half_start",
         "half_j", "force", "virial", "torque", "acc", "copies", "estore", "jstart", "jedge", "local_tab", "trace",
         "pos_alt", "fxp_alt", "nbr_in", "nbr_in_count", "fxp_prune", "scratch")]


class MDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmdgb error {code}: {msg}")
        self.code = code


_lib = None
_P = ctypes.POINTER(md_params)
_S = ctypes.POINTER(md_state)
_V = ctypes.c_void_p


def header_functions():
    """Names of the functions declared in include/md.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_0-9]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load libmdgb.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with `python -m paper_1401_4350_gb300.build`")
    lib = ctypes.CDLL(path)
    sig = {
        "md_abi_version": ([], ctypes.c_int),
        "md_last_error": ([], ctypes.c_char_p),
        "md_check_params": ([_P], ctypes.c_int),
        "md_workspace_bytes": ([_P], ctypes.c_size_t),
        "md_workspace_layout": ([_P, ctypes.POINTER(md_ws_layout)], ctypes.c_int),
        "md_init_workspace": ([_P, _V, _V], ctypes.c_int),
        "md_build_cells": ([_P, _S, _V, _V], ctypes.c_int),
        "md_build_verlet": ([_P, _S, _V, ctypes.c_int32, _V], ctypes.c_int),
        "md_forces_vertex": ([_P, _S, _V, _V], ctypes.c_int),
        "md_forces_edge": ([_P, _S, _V, _V], ctypes.c_int),
        "md_forces_vertex_newton": ([_P, _S, _V, _V], ctypes.c_int),
        "md_forces_edge_store": ([_P, _S, _V, _V], ctypes.c_int),
        "md_autotune_system": ([_P, _S, _V, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float), _V],
                               ctypes.c_int),
        "md_step_verlet": ([_P, _S, _V, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _V], ctypes.c_int),
        "md_step_verlet_host": ([_P, _S, _V, _V, _V, _V, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _V],
                                ctypes.c_int),
        "md_time_step_kernel": ([_P, _S, _V, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), _V],
                                ctypes.c_int),
        "md_prepare": ([_P, _S, _V, ctypes.c_int32, _V], ctypes.c_int),
        "md_get_forces": ([_P, _V, _V, _V, _V], ctypes.c_int),
        "md_read_status": ([_P, _V, ctypes.POINTER(ctypes.c_int32), _V], ctypes.c_int),
        "md_release_graphs": ([_V], ctypes.c_int),
        "md_cell_order": ([_P, _V], ctypes.c_int),
        "md_build_cells_static": ([_P, _S, _V, _V, _V, _V], ctypes.c_int),
        "md_batch_workspace_bytes": ([_P, ctypes.c_int32], ctypes.c_size_t),
        "md_batch_replica_offset": ([_P, ctypes.c_int32, ctypes.c_int32], ctypes.c_size_t),
        "md_batch_init": ([_P, ctypes.c_int32, _S, _V, _V, _V], ctypes.c_int),
        "md_batch_prepare": ([_V, _V], ctypes.c_int),
        "md_batch_forces": ([_V, _V], ctypes.c_int),
        "md_batch_step": ([_V, ctypes.c_int32, ctypes.c_int32, _V], ctypes.c_int),
        "md_batch_set_config": ([_V, _V, _V, _V], ctypes.c_int),
        "md_batch_get_config": ([_V, _V, _V], ctypes.c_int),
        "md_batch_release": ([_V], ctypes.c_int),
        "md_autotune": ([_V, _V, _V, _V], ctypes.c_int),
        "md_static_scratch_bytes": ([], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def last_error() -> str:
    return load().md_last_error().decode()


def _check(rc):
    if rc != MD_OK:
        raise MDError(rc, last_error())
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


# ---- the C ABI, one wrapper per entry point ---------------------------------------------------

def md_abi_version() -> int:
    return load().md_abi_version()


def md_check_params(p: md_params) -> int:
    return load().md_check_params(ctypes.byref(p))


def md_workspace_bytes(p: md_params) -> int:
    return load().md_workspace_bytes(ctypes.byref(p))


def md_workspace_layout(p: md_params) -> md_ws_layout:
    out = md_ws_layout()
    _check(load().md_workspace_layout(ctypes.byref(p), ctypes.byref(out)))
    return out


def md_init_workspace(p, ws, stream=None):
    return _check(load().md_init_workspace(ctypes.byref(p), _ptr(ws), _stream(stream)))


def md_build_cells(p, s, ws, stream=None):
    return _check(load().md_build_cells(ctypes.byref(p), ctypes.byref(s), _ptr(ws), _stream(stream)))


def md_build_verlet(p, s, ws, which=MD_LIST_BOTH, stream=None):
    return _check(load().md_build_verlet(ctypes.byref(p), ctypes.byref(s), _ptr(ws), which, _stream(stream)))


def md_forces_vertex(p, s, ws, stream=None):
    return _check(load().md_forces_vertex(ctypes.byref(p), ctypes.byref(s), _ptr(ws), _stream(stream)))


def md_forces_edge(p, s, ws, stream=None):
    return _check(load().md_forces_edge(ctypes.byref(p), ctypes.byref(s), _ptr(ws), _stream(stream)))


def md_forces_edge_store(p, s, ws, stream=None):
    return _check(load().md_forces_edge_store(ctypes.byref(p), ctypes.byref(s), _ptr(ws), _stream(stream)))


MD_TUNE_CANDIDATES = 16
TUNE_CANDIDATES = ([(MD_VERTEX, t, b) for t in (1, 2, 4, 8) for b in (64, 128, 256)] +
                   [(MD_EDGE, 1, 128), (MD_EDGE, 1, 256), (MD_VERTEX_NEWTON, 1, 128), (MD_EDGE_STORE, 1, 256)])


def md_autotune_system(p, s, ws, stream=None):
    """(path, threads_per_particle, block_size, median ms per candidate of TUNE_CANDIDATES); p is updated."""
    path = ctypes.c_int32(0)
    ms = (ctypes.c_float * MD_TUNE_CANDIDATES)()
    _check(load().md_autotune_system(ctypes.byref(p), ctypes.byref(s), _ptr(ws), ctypes.byref(path), ms,
                                     _stream(stream)))
    return int(path.value), int(p.threads_per_particle), int(p.block_size), [float(x) for x in ms]


def md_forces_vertex_newton(p, s, ws, stream=None):
    return _check(load().md_forces_vertex_newton(ctypes.byref(p), ctypes.byref(s), _ptr(ws), _stream(stream)))


def md_step_verlet(p, s, ws, nsteps, path=MD_VERTEX, use_graph=True, stream=None):
    return _check(load().md_step_verlet(ctypes.byref(p), ctypes.byref(s), _ptr(ws), int(nsteps), int(path),
                                        int(bool(use_graph)), _stream(stream)))


def md_step_verlet_host(p, s, ws, host_pos, host_vel, host_energy=None, nsteps=1, path=MD_VERTEX, use_graph=True,
                        stream=None):
    """md_step_verlet on a host-resident state: host_pos / host_vel are [n][3] float64 host arrays (pinned
    torch tensors give the full copy bandwidth), read and then overwritten in stream order."""
    return _check(load().md_step_verlet_host(ctypes.byref(p), ctypes.byref(s), _ptr(ws), _ptr(host_pos),
                                             _ptr(host_vel), _ptr(host_energy), int(nsteps), int(path),
                                             int(bool(use_graph)), _stream(stream)))


def md_time_step_kernel(p, s, ws, path=MD_VERTEX, reps=20, stream=None) -> float:
    """Mean ms of the kernel md_step_verlet runs once per step (fused step kernel or force kernel)."""
    ms = ctypes.c_float(0.0)
    _check(load().md_time_step_kernel(ctypes.byref(p), ctypes.byref(s), _ptr(ws), int(path), int(reps),
                                      ctypes.byref(ms), _stream(stream)))
    return float(ms.value)


def md_prepare(p, s, ws, path=MD_VERTEX, stream=None):
    return _check(load().md_prepare(ctypes.byref(p), ctypes.byref(s), _ptr(ws), int(path), _stream(stream)))


def md_get_forces(p, ws, force_out, torque_out=None, stream=None):
    return _check(load().md_get_forces(ctypes.byref(p), _ptr(ws), _ptr(force_out), _ptr(torque_out),
                                       _stream(stream)))


def md_read_status(p, ws, stream=None):
    out = (ctypes.c_int32 * MD_STATUS_WORDS)()
    _check(load().md_read_status(ctypes.byref(p), _ptr(ws), out, _stream(stream)))
    return list(out)


def md_release_graphs(ws=None):
    return load().md_release_graphs(_ptr(ws) if ws is not None else None)


def md_cell_order(p):
    """Position of every row-major cell in the cell order of p (numpy int32 array, host only)."""
    import numpy as np
    L = md_workspace_layout(p)
    out = np.empty(int(L.ncell[0]) * int(L.ncell[1]) * int(L.ncell[2]), dtype=np.int32)
    _check(load().md_cell_order(ctypes.byref(p), out.ctypes.data_as(ctypes.c_void_p)))
    return out


MD_STATIC_MAX_N = 32768


def md_build_cells_static(p, s, cell_start, fxp, patch_lab=None, stream=None):
    """The cell build without a workspace: scratch from the library's static device array."""
    return _check(load().md_build_cells_static(ctypes.byref(p), ctypes.byref(s), _ptr(cell_start), _ptr(fxp),
                                               _ptr(patch_lab), _stream(stream)))


def md_static_scratch_bytes() -> int:
    return load().md_static_scratch_bytes()


# ---- batched replicas ---------------------------------------------------------------------------

def _params_array(reps):
    arr = (md_params * len(reps))()
    for k, p in enumerate(reps):
        arr[k] = p
    return arr


def md_batch_workspace_bytes(reps) -> int:
    return load().md_batch_workspace_bytes(_params_array(reps), len(reps))


def md_batch_replica_offset(reps, r) -> int:
    return load().md_batch_replica_offset(_params_array(reps), len(reps), r)


def _i32_array(vals):
    if vals is None:
        return None
    arr = (ctypes.c_int32 * len(vals))(*[int(v) for v in vals])
    return arr


def md_batch_init(reps, s, ws, path=None, stream=None):
    return _check(load().md_batch_init(_params_array(reps), len(reps), ctypes.byref(s), _ptr(ws),
                                       _i32_array(path), _stream(stream)))


def md_batch_prepare(ws, stream=None):
    return _check(load().md_batch_prepare(_ptr(ws), _stream(stream)))


def md_batch_forces(ws, stream=None):
    return _check(load().md_batch_forces(_ptr(ws), _stream(stream)))


def md_batch_step(ws, nsteps, use_graph=True, stream=None):
    return _check(load().md_batch_step(_ptr(ws), int(nsteps), int(bool(use_graph)), _stream(stream)))


def md_batch_set_config(ws, path=None, tpp=None, stream=None):
    return _check(load().md_batch_set_config(_ptr(ws), _i32_array(path), _i32_array(tpp), _stream(stream)))


def md_batch_get_config(ws, nrep):
    path = (ctypes.c_int32 * nrep)()
    tpp = (ctypes.c_int32 * nrep)()
    _check(load().md_batch_get_config(_ptr(ws), path, tpp))
    return list(path), list(tpp)


def md_batch_release(ws=None):
    return load().md_batch_release(_ptr(ws) if ws is not None else None)


def md_autotune(ws, nrep, stream=None):
    path = (ctypes.c_int32 * nrep)()
    tpp = (ctypes.c_int32 * nrep)()
    _check(load().md_autotune(_ptr(ws), path, tpp, _stream(stream)))
    return list(path), list(tpp)

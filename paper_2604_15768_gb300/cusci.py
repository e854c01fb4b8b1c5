"""Thin ctypes binding of libcusci (the C ABI in ``include/cusci.h``).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  Determinants travel as
``torch.int64`` tensors of shape (n, W) holding the uint64 bit patterns.

There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

__all__ = ["CusciError", "load", "System", "count_coupled", "exclusive_scan", "gen_coupled",
           "check_dets", "dedup", "coupled", "energy_fwd", "energy_bwd", "Energy"]

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t

_LIB = None
_LOCK = threading.Lock()

STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "OVERFLOW", 5: "TIMEOUT",
          6: "UNSUPPORTED"}


class CusciError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: CUSCI_ERR_{STATUS.get(status, status)}: {msg}")
        self.status = status


_PROTOS = {
    "cusci_last_error": (ctypes.c_char_p, []),
    "cusci_version": (ctypes.c_char_p, []),
    "cusci_kernel_launches": (ctypes.c_uint64, []),
    "cusci_set_kernel_timing": (_I, [_I]),
    "cusci_dedup_phase_ms": (_I, [_P, _I, _P]),
    "cusci_dedup_phase_name": (ctypes.c_char_p, [_I]),
    "cusci_system_create": (_I, [_I, _I, _I, _P, _P, _D, ctypes.POINTER(_P)]),
    "cusci_system_destroy": (None, [_P]),
    "cusci_system_words": (_I, [_P]),
    "cusci_count_coupled": (_I, [_P, _P, _I64, _D, _P, _P]),
    "cusci_scan_workspace": (_I, [_I64, ctypes.POINTER(_SZ)]),
    "cusci_exclusive_scan": (_I, [_P, _I64, _P, _P, _SZ, _P]),
    "cusci_scan_static_max": (_I64, []),
    "cusci_exclusive_scan_static": (_I, [_P, _I64, _P, _P]),
    "cusci_gen_coupled": (_I, [_P, _P, _I64, _D, _P, _P, _P, _P, _P]),
    "cusci_check_dets": (_I, [_P, _P, _I64, _P, _P]),
    "cusci_dedup_workspace": (_I, [_I64, _I, _I, _I, ctypes.POINTER(_SZ)]),
    "cusci_dedup": (_I, [_P, _I64, _I, _I, _I, _P, _SZ, _P, _P, _I, _P, _P, _P, _P]),
    "cusci_stream_pool_bytes": (_I, [_P, _I64, _I64, _I64, ctypes.POINTER(_SZ)]),
    "cusci_hash_insert_probe": (_I, [_P, _I64, _I, _P, _I64, _I, _P, _P, _P]),
    "cusci_stream_gen_dedup": (_I, [_P, _P, _I64, _D, _P, _SZ, _I64, _P, _P, _P, _I64, _P, _I64,
                                    _P, _P, _P]),
    "cusci_batch_create": (_I, [_P, _I, _P, _I, ctypes.POINTER(_P)]),
    "cusci_batch_destroy": (None, [_P]),
    "cusci_batch_set_chunk": (_I, [_P, _I]),
    "cusci_batch_sources": (_I64, [_P]),
    "cusci_batch_count": (_I, [_P, _P, _D, _P, _P]),
    "cusci_batch_set_grid": (_I, [_P, _I]),
    "cusci_batch_dedup_workspace": (_I, [_P, _I64, ctypes.POINTER(_SZ)]),
    "cusci_batch_dedup": (_I, [_P, _P, _P, _I64, _P, _SZ, _P, _P, _P, _P, _P]),
    "cusci_batch_gen": (_I, [_P, _P, _D, _P, _P, _P, _P, _P]),
    "cusci_local_energy_workspace": (_I, [_I64, ctypes.POINTER(_SZ)]),
    "cusci_local_energy_fwd": (_I, [_P, _I64, _P, _P, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "cusci_local_energy_bwd_workspace": (_I, [_I64, _I64, ctypes.POINTER(_SZ)]),
    "cusci_local_energy_bwd": (_I, [_P, _I64, _P, _P, _I, _P, _I64, _P, _P, _P, _P, _P, _P, _SZ,
                                    _P]),
    "cusci_partition_plan": (_I, [_P, _I, _P, _I, _I, _P, _P, _P]),
    "cusci_reverse_table_bytes": (_I, [_I64, _I, ctypes.POINTER(_SZ)]),
    "cusci_reverse_table_build": (_I, [_P, _I64, _I, _P, _SZ, _P, _P]),
    "cusci_reverse_index_table": (_I, [_P, _I64, _I, _P, _I64, _P, _I, _P, _P]),
    "cusci_rank_join": (_I, [_P, _I, _I64, _P, _I, _I, _P, _P, _P]),
    "cusci_rank_runs": (_I, [_P, _I, _P, _I64, _I, _I, _P, _P, _P]),
    "cusci_partition_exchange": (_I, [_P, _I, _I, _P, _P, _P, _P]),
    "cusci_partition_split": (_I, [_P, _I, _P, _P, _I, _P, _P]),
    "cusci_reverse_index": (_I, [_P, _I64, _I, _P, _I64, _P, _I, _P, _P]),
    "cusci_topk_workspace": (_I, [_I64, _I64, ctypes.POINTER(_SZ)]),
    "cusci_topk_update": (_I, [_P, _P, _I64, _I64, _P, _P, _P, _P, _SZ, _P, _P]),
    "cusci_energy_workspace": (_I, [_P, _I64, ctypes.POINTER(_SZ)]),
    "cusci_energy_fwd": (_I, [_P, _P, _I64, _P, _D, _P, _P, _P, _P, _SZ, _P, _P]),
    "cusci_energy_bwd": (_I, [_P, _P, _I64, _P, _D, _P, _P, _P, _P, _P, _P, _SZ, _P]),
}


def exported_names() -> list[str]:
    return sorted(_PROTOS)


def load(path: str | None = None):
    """Load (building first if needed) libcusci.so and declare its prototypes."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = path or _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in _PROTOS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = lib
    return _LIB


def kernel_launches() -> int:
    """Kernels launched by libcusci in this process so far."""
    return int(load().cusci_kernel_launches())


def set_kernel_timing(on: bool):
    """Start (resetting the record) or stop per-phase event timing of the
    sample-sort de-duplication."""
    _check(load().cusci_set_kernel_timing(1 if on else 0), "cusci_set_kernel_timing")


def dedup_phase_ms():
    """(dict phase name -> summed ms, number of calls) of the recorded calls."""
    lib = load()
    ms = np.zeros(16, dtype=np.float64)
    calls = ctypes.c_int(0)
    n = lib.cusci_dedup_phase_ms(ms.ctypes.data_as(_P), 16, ctypes.byref(calls))
    return {lib.cusci_dedup_phase_name(i).decode(): float(ms[i]) for i in range(n)}, calls.value


def _check(rc: int, where: str):
    if rc != 0:
        raise CusciError(rc, where, load().cusci_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


def dets_to_device(dets: np.ndarray, device="cuda") -> torch.Tensor:
    """(n, W) uint64 numpy array -> int64 CUDA tensor with the same bits."""
    a = np.ascontiguousarray(dets, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64)).to(device)


def dets_to_numpy(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


class System:
    """A molecular system resident on the current CUDA device (library-owned)."""

    def __init__(self, norb, n_alpha, n_beta, h1, h2, ecore=0.0):
        lib = load()
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        h2 = np.ascontiguousarray(h2, dtype=np.float64)
        if h1.size != norb * norb or h2.size != norb ** 4:
            raise ValueError("integral sizes do not match norb")
        handle = ctypes.c_void_p()
        _check(lib.cusci_system_create(int(norb), int(n_alpha), int(n_beta),
                                       h1.ctypes.data_as(_P), h2.ctypes.data_as(_P),
                                       float(ecore), ctypes.byref(handle)),
               "cusci_system_create")
        self._h = handle
        self.norb, self.n_alpha, self.n_beta = int(norb), int(n_alpha), int(n_beta)
        self.W = lib.cusci_system_words(handle)
        self.M = 2 * self.norb

    @classmethod
    def of(cls, s):
        return cls(s.norb, s.n_alpha, s.n_beta, s.h1, s.h2, getattr(s, "ecore", 0.0))

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("system destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _LIB is not None:
            _LIB.cusci_system_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count_coupled(sys: System, dets: torch.Tensor, eps: float, out=None, stream=None):
    dets = _dev(dets, torch.int64, "dets")
    n = dets.shape[0]
    out = out if out is not None else torch.empty(n, dtype=torch.int64, device=dets.device)
    _check(load().cusci_count_coupled(sys.handle, _ptr(dets), n, float(eps), _ptr(out),
                                      _stream(stream)), "cusci_count_coupled")
    return out


def scan_workspace(n: int) -> int:
    ws = ctypes.c_size_t()
    _check(load().cusci_scan_workspace(int(n), ctypes.byref(ws)), "cusci_scan_workspace")
    return max(1, ws.value)


def exclusive_scan(counts: torch.Tensor, out=None, workspace=None, stream=None):
    counts = _dev(counts, torch.int64, "counts")
    n = counts.shape[0]
    need = scan_workspace(n)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=counts.device)
    out = out if out is not None else torch.empty(n + 1, dtype=torch.int64, device=counts.device)
    _check(load().cusci_exclusive_scan(_ptr(counts), n, _ptr(out), _ptr(workspace),
                                       workspace.numel(), _stream(stream)),
           "cusci_exclusive_scan")
    return out


def gen_coupled(sys: System, dets: torch.Tensor, eps: float, offsets: torch.Tensor, total: int,
                out_dets=None, out_h=None, status=None, stream=None):
    dets = _dev(dets, torch.int64, "dets")
    offsets = _dev(offsets, torch.int64, "offsets")
    dev = dets.device
    if out_dets is None:
        out_dets = torch.empty((total, sys.W), dtype=torch.int64, device=dev)
    if out_h is None:
        out_h = torch.empty(total, dtype=torch.float64, device=dev)
    _check(load().cusci_gen_coupled(sys.handle, _ptr(dets), dets.shape[0], float(eps),
                                    _ptr(offsets), _ptr(out_dets), _ptr(out_h), _ptr(status),
                                    _stream(stream)), "cusci_gen_coupled")
    return out_dets, out_h


def check_dets(sys: System, dets: torch.Tensor, status: torch.Tensor, stream=None):
    dets = _dev(dets, torch.int64, "dets")
    _check(load().cusci_check_dets(sys.handle, _ptr(dets), dets.shape[0], _ptr(status),
                                   _stream(stream)), "cusci_check_dets")
    return status


def dedup_workspace(total: int, W: int, n_bits: int, n_ones: int) -> int:
    ws = ctypes.c_size_t()
    _check(load().cusci_dedup_workspace(int(total), int(W), int(n_bits), int(n_ones),
                                        ctypes.byref(ws)), "cusci_dedup_workspace")
    return ws.value


def dedup(keys: torch.Tensor, n_bits: int, n_ones: int = -1, index_bytes: int = 4,
          workspace=None, status=None, stream=None, sync=True):
    """Sorted distinct keys and the inverse index.  Returns (unique, inverse, n_unique);
    with ``sync=False`` n_unique is a device tensor and ``unique`` is full capacity."""
    keys = _dev(keys, torch.int64, "keys")
    total, W = keys.shape
    dev = keys.device
    need = dedup_workspace(total, W, n_bits, n_ones)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    unique = torch.empty((max(total, 1), W), dtype=torch.int64, device=dev)
    inverse = torch.empty(max(total, 1), dtype=torch.int32 if index_bytes == 4 else torch.int64,
                          device=dev)
    d_nu = torch.zeros(1, dtype=torch.int64, device=dev)
    h_nu = ctypes.c_int64(-1)
    _check(load().cusci_dedup(_ptr(keys), total, W, int(n_bits), int(n_ones), _ptr(workspace),
                              workspace.numel(), _ptr(unique), _ptr(inverse), int(index_bytes),
                              _ptr(d_nu), ctypes.byref(h_nu) if sync else None, _ptr(status),
                              _stream(stream)), "cusci_dedup")
    if sync:
        return unique[:h_nu.value], inverse[:total], h_nu.value
    return unique, inverse[:total], d_nu


def dedup_into(keys: torch.Tensor, n_bits: int, n_ones: int, unique: torch.Tensor,
               inverse: torch.Tensor, n_unique: torch.Tensor, workspace: torch.Tensor,
               status=None, stream=None):
    """Asynchronous de-duplication into caller-owned buffers (no host sync)."""
    total, W = keys.shape
    ib = 4 if inverse.dtype == torch.int32 else 8
    _check(load().cusci_dedup(_ptr(keys), total, W, int(n_bits), int(n_ones), _ptr(workspace),
                              workspace.numel(), _ptr(unique), _ptr(inverse), ib, _ptr(n_unique),
                              None, _ptr(status), _stream(stream)), "cusci_dedup")


def coupled(sys: System, dets: torch.Tensor, eps: float, stream=None):
    """count -> scan -> fill.  Returns (offsets, out_dets, out_h, status)."""
    counts = count_coupled(sys, dets, eps, stream=stream)
    offsets = exclusive_scan(counts, stream=stream)
    total = int(offsets[-1].item())
    status = torch.zeros(1, dtype=torch.int32, device=dets.device)
    out_d, out_h = gen_coupled(sys, dets, eps, offsets, total, status=status, stream=stream)
    return offsets, out_d, out_h, status


def hash_insert_probe(keys: torch.Tensor, table: torch.Tensor, spin_limit: int, n_new=None,
                      status=None, stream=None):
    """The streaming path's hash-set insert on a caller-built table (see
    cusci_hash_insert_probe); returns the device counter of new keys."""
    keys = _dev(keys, torch.int64, "keys")
    n, W = keys.shape
    if n_new is None:
        n_new = torch.zeros(1, dtype=torch.int64, device=keys.device)
    _check(load().cusci_hash_insert_probe(_ptr(keys), n, W, _ptr(table), table.shape[0],
                                          int(spin_limit), _ptr(n_new), _ptr(status),
                                          _stream(stream)), "cusci_hash_insert_probe")
    return n_new


def stream_pool_bytes(sys: System, n_sources: int, batch_entries: int,
                      unique_capacity: int) -> int:
    b = ctypes.c_size_t()
    _check(load().cusci_stream_pool_bytes(sys.handle, int(n_sources), int(batch_entries),
                                          int(unique_capacity), ctypes.byref(b)),
           "cusci_stream_pool_bytes")
    return b.value


def stream_buffers(sys: System, dets: np.ndarray, batch_entries: int, unique_capacity: int,
                   host_capacity: int = 0):
    """Caller-side buffers of ``stream_gen_dedup``: pinned host sources, the
    device pool, pinned host sinks (if host_capacity > 0) and the distinct set."""
    dets = np.ascontiguousarray(dets, dtype=np.uint64).reshape(-1, sys.W)
    need = stream_pool_bytes(sys, dets.shape[0], batch_entries, unique_capacity)
    buf = {"src": torch.from_numpy(dets.view(np.int64)).pin_memory(),
           "pool": torch.empty(need, dtype=torch.uint8, device="cuda"),
           "unique": torch.empty((unique_capacity, sys.W), dtype=torch.int64, device="cuda"),
           "hd": None, "hh": None}
    if host_capacity > 0:
        buf["hd"] = torch.empty((host_capacity, sys.W), dtype=torch.int64).pin_memory()
        buf["hh"] = torch.empty(host_capacity, dtype=torch.float64).pin_memory()
    return buf


def stream_gen_dedup(sys: System, dets: np.ndarray, eps: float, batch_entries: int,
                     unique_capacity: int, host_capacity: int | None = None, offload=True,
                     pool=None, stream=None, buffers=None):
    """Mini-batched generation + de-duplication (host sources in, host coupled
    lists and device distinct set out).  Returns (offsets, host_dets, host_h,
    unique, stats) with host arrays pinned.  ``buffers`` (from stream_buffers)
    are reused when given."""
    dets = np.ascontiguousarray(dets, dtype=np.uint64).reshape(-1, sys.W)
    n = dets.shape[0]
    if buffers is None:
        buffers = stream_buffers(sys, dets, batch_entries, unique_capacity,
                                 int(host_capacity) if offload else 0)
        if pool is not None and pool.numel() >= buffers["pool"].numel():
            buffers["pool"] = pool
    h_src, pool, uniq = buffers["src"], buffers["pool"], buffers["unique"]
    offsets = np.zeros(n + 1, dtype=np.int64)
    hd = buffers["hd"] if offload else None
    hh = buffers["hh"] if offload else None
    cap = 0 if hd is None else hd.shape[0]
    nu = ctypes.c_int64(0)
    stats = np.zeros(6, dtype=np.int64)
    _check(load().cusci_stream_gen_dedup(
        sys.handle, ctypes.c_void_p(h_src.data_ptr()), n, float(eps), _ptr(pool), pool.numel(),
        int(batch_entries), offsets.ctypes.data_as(_P), _ptr(hd), _ptr(hh), cap, _ptr(uniq),
        int(unique_capacity), ctypes.byref(nu), stats.ctypes.data_as(_P), _stream(stream)),
        "cusci_stream_gen_dedup")
    total = int(offsets[-1])
    out_d = hd[:total] if offload else None
    out_h = hh[:total] if offload else None
    return offsets, out_d, out_h, uniq[:nu.value], {"total": int(stats[0]), "batches": int(stats[1]),
                                                     "pool_peak": int(stats[2]),
                                                     "d2h_bytes": int(stats[3]),
                                                     "batches_ms": stats[4] / 1e3,
                                                     "final_sort_ms": stats[5] / 1e3,
                                                     "pool_bytes": int(pool.numel())}


def energy_workspace(sys: System, nS: int) -> int:
    ws = ctypes.c_size_t()
    _check(load().cusci_energy_workspace(sys.handle, int(nS), ctypes.byref(ws)),
           "cusci_energy_workspace")
    return ws.value


def energy_fwd(sys: System, S: torch.Tensor, psi: torch.Tensor, eps: float, save_hpsi=True,
               workspace=None, status=None, stream=None):
    """Returns (E, norm2, Hpsi or None) as device tensors."""
    S = _dev(S, torch.int64, "S")
    psi = _dev(psi, torch.float64, "psi")
    nS = S.shape[0]
    dev = S.device
    need = energy_workspace(sys, nS)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    n2 = torch.empty(1, dtype=torch.float64, device=dev)
    hp = torch.empty(nS, dtype=torch.float64, device=dev) if save_hpsi else None
    _check(load().cusci_energy_fwd(sys.handle, _ptr(S), nS, _ptr(psi), float(eps), _ptr(E),
                                   _ptr(n2), _ptr(hp), _ptr(workspace), workspace.numel(),
                                   _ptr(status), _stream(stream)), "cusci_energy_fwd")
    return E, n2, hp


def energy_bwd(sys: System, S, psi, eps, E, norm2, hpsi=None, grad_out=None, workspace=None,
               stream=None):
    S = _dev(S, torch.int64, "S")
    psi = _dev(psi, torch.float64, "psi")
    nS = S.shape[0]
    dev = S.device
    if hpsi is None and (workspace is None or workspace.numel() < energy_workspace(sys, nS)):
        workspace = torch.empty(energy_workspace(sys, nS), dtype=torch.uint8, device=dev)
    grad = torch.empty(nS, dtype=torch.float64, device=dev)
    g = None
    if grad_out is not None:
        g = grad_out.reshape(1).to(dtype=torch.float64).contiguous()
    _check(load().cusci_energy_bwd(sys.handle, _ptr(S), nS, _ptr(psi), float(eps), _ptr(E),
                                   _ptr(norm2), _ptr(hpsi), _ptr(g), _ptr(grad),
                                   _ptr(workspace), 0 if workspace is None else workspace.numel(),
                                   _stream(stream)), "cusci_energy_bwd")
    return grad


def local_energy_workspace(n: int) -> int:
    ws = ctypes.c_size_t()
    _check(load().cusci_local_energy_workspace(int(n), ctypes.byref(ws)),
           "cusci_local_energy_workspace")
    return ws.value


def local_energy_fwd(offsets, h, inverse, psi_u, workspace=None, save_y=True, stream=None):
    """(E, norm2, y or None) of the local-energy form (Eq. 5) as device tensors."""
    n = offsets.shape[0] - 1
    ib = 4 if inverse.dtype == torch.int32 else 8
    need = local_energy_workspace(n)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=h.device)
    E = torch.empty(1, dtype=torch.float64, device=h.device)
    n2 = torch.empty(1, dtype=torch.float64, device=h.device)
    y = torch.empty(n, dtype=torch.float64, device=h.device) if save_y else None
    _check(load().cusci_local_energy_fwd(_ptr(offsets), n, _ptr(h), _ptr(inverse), ib,
                                         _ptr(psi_u), _ptr(y), _ptr(E), _ptr(n2),
                                         _ptr(workspace), workspace.numel(), _stream(stream)),
           "cusci_local_energy_fwd")
    return E, n2, y


def local_energy_bwd_workspace(n: int, n_unique: int) -> int:
    ws = ctypes.c_size_t()
    _check(load().cusci_local_energy_bwd_workspace(int(n), int(n_unique), ctypes.byref(ws)),
           "cusci_local_energy_bwd_workspace")
    return ws.value


def local_energy_bwd(offsets, h, inverse, psi_u, E, norm2, y=None, grad_out=None,
                     workspace=None, stream=None):
    n = offsets.shape[0] - 1
    ib = 4 if inverse.dtype == torch.int32 else 8
    need = local_energy_bwd_workspace(n, psi_u.numel())
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=h.device)
    grad = torch.empty_like(psi_u)
    g = None if grad_out is None else grad_out.reshape(1).to(torch.float64).contiguous()
    _check(load().cusci_local_energy_bwd(_ptr(offsets), n, _ptr(h), _ptr(inverse), ib,
                                         _ptr(psi_u), psi_u.numel(), _ptr(y), _ptr(E), _ptr(norm2),
                                         _ptr(g), _ptr(grad), _ptr(workspace),
                                         0 if workspace is None else workspace.numel(),
                                         _stream(stream)), "cusci_local_energy_bwd")
    return grad


def reverse_index(unique: torch.Tensor, keys: torch.Tensor, index_bytes: int = 4, out=None,
                  status=None, stream=None):
    """Position of every key in the sorted distinct set (device tensors)."""
    W = unique.shape[1]
    if out is None:
        out = torch.empty(keys.shape[0], dtype=torch.int32 if index_bytes == 4 else torch.int64,
                          device=keys.device)
    _check(load().cusci_reverse_index(_ptr(unique), unique.shape[0], W, _ptr(keys), keys.shape[0],
                                      _ptr(out), index_bytes, _ptr(status), _stream(stream)),
           "cusci_reverse_index")
    return out


def reverse_table(unique: torch.Tensor, status=None, stream=None) -> torch.Tensor:
    """Hash table of the distinct set for cusci_reverse_index_table (device bytes)."""
    n_u, W = unique.shape
    nb = ctypes.c_size_t()
    _check(load().cusci_reverse_table_bytes(int(n_u), W, ctypes.byref(nb)),
           "cusci_reverse_table_bytes")
    table = torch.empty(nb.value, dtype=torch.uint8, device=unique.device)
    _check(load().cusci_reverse_table_build(_ptr(unique), int(n_u), W, _ptr(table), table.numel(),
                                            _ptr(status), _stream(stream)),
           "cusci_reverse_table_build")
    return table


def reverse_index_table(table: torch.Tensor, n_unique: int, W: int, keys: torch.Tensor,
                        index_bytes: int = 4, out=None, status=None, stream=None):
    """Position of every key in the distinct set, through its hash table."""
    if out is None:
        out = torch.empty(keys.shape[0], dtype=torch.int32 if index_bytes == 4 else torch.int64,
                          device=keys.device)
    _check(load().cusci_reverse_index_table(_ptr(table), int(n_unique), W, _ptr(keys),
                                            keys.shape[0], _ptr(out), index_bytes, _ptr(status),
                                            _stream(stream)), "cusci_reverse_index_table")
    return out


def reverse_index_stream(unique: torch.Tensor, host_keys: torch.Tensor, batch: int,
                         host_out: torch.Tensor | None = None, status=None, table=False):
    """Reverse index of a host-resident (pinned) key array against the device
    distinct set, in batches: copy in, look up and copy out on two alternating
    streams so transfers overlap the lookups.  ``table``: a hash table from
    reverse_table (probed by every batch; worth building when the distinct set
    is queried more than once), True to build one here, or False to search the
    sorted set for every key.  Returns the pinned host ids."""
    n, W = host_keys.shape
    n_u = unique.shape[0]
    dev = unique.device
    if host_out is None:
        host_out = torch.empty(n, dtype=torch.int32).pin_memory()
    if isinstance(table, torch.Tensor):
        tb = table
    else:
        tb = reverse_table(unique, status=status) if table and n > 0 else None
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    kbuf = [torch.empty((batch, W), dtype=torch.int64, device=dev) for _ in range(2)]
    ibuf = [torch.empty(batch, dtype=torch.int32, device=dev) for _ in range(2)]
    torch.cuda.current_stream().synchronize()
    for t, a in enumerate(range(0, n, batch)):
        b = min(n, a + batch)
        s = streams[t & 1]
        with torch.cuda.stream(s):
            kb, ib = kbuf[t & 1][:b - a], ibuf[t & 1][:b - a]
            kb.copy_(host_keys[a:b], non_blocking=True)
            if tb is not None:
                reverse_index_table(tb, n_u, W, kb, 4, out=ib, status=status, stream=s)
            else:
                reverse_index(unique, kb, 4, out=ib, status=status, stream=s)
            host_out[a:b].copy_(ib, non_blocking=True)
    for s in streams:
        s.synchronize()
    return host_out


class TopK:
    """Running best-K set over a stream of scored batches (device resident)."""

    def __init__(self, K: int, max_batch: int, device="cuda"):
        self.K = int(K)
        self.scores = torch.zeros(self.K, dtype=torch.float64, device=device)
        self.ids = torch.zeros(self.K, dtype=torch.int64, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        ws = ctypes.c_size_t()
        _check(load().cusci_topk_workspace(int(max_batch), self.K, ctypes.byref(ws)),
               "cusci_topk_workspace")
        self.ws = torch.empty(ws.value, dtype=torch.uint8, device=device)
        self.max_batch = int(max_batch)

    def update(self, scores: torch.Tensor, ids: torch.Tensor, status=None, stream=None):
        """Merge one batch; ``status`` (device int32[1], optional) receives
        CUSCI_ERR_INVALID if a score is negative or NaN."""
        n = scores.shape[0]
        if n > self.max_batch:
            raise ValueError("batch larger than max_batch")
        _check(load().cusci_topk_update(_ptr(scores), _ptr(ids), n, self.K, _ptr(self.scores),
                                        _ptr(self.ids), _ptr(self.count), _ptr(self.ws),
                                        self.ws.numel(), _ptr(status), _stream(stream)),
               "cusci_topk_update")

    def result(self):
        """(scores, ids) of the best set, best first (host numpy)."""
        c = int(self.count.item())
        sc = self.scores[:c].cpu().numpy()
        ids = self.ids[:c].cpu().numpy()
        order = np.lexsort((ids, -sc))
        return sc[order], ids[order]


def partition_plan(runs: torch.Tensor, run_offsets: torch.Tensor, P: int, S: int, stream=None):
    """Splitters [P-1, W] and cuts [P, P+1] of the regular-sampling partition of P
    sorted distinct runs laid back to back in ``runs`` ([*, W])."""
    W = runs.shape[1]
    spl = torch.empty((max(P - 1, 1), W), dtype=torch.int64, device=runs.device)
    bounds = torch.empty((P, P + 1), dtype=torch.int64, device=runs.device)
    _check(load().cusci_partition_plan(_ptr(runs), W, _ptr(run_offsets), int(P), int(S), _ptr(spl),
                                       _ptr(bounds), _stream(stream)), "cusci_partition_plan")
    return spl[:P - 1], bounds


def virtual_rank_dedup(keys: torch.Tensor, entry_offsets, P: int, S: int, n_bits: int,
                       n_ones: int, stream=None):
    """The paper's distributed de-duplication (Sec. 4.1.1) over P virtual ranks on
    one GPU, as a device pipeline with one host read-back at the end.  Rank r
    owns the entries [entry_offsets[r], entry_offsets[r+1]) of ``keys``.
    Step 1: every rank's local sort + unique, all ranks in one dedup of the
    rank-joined keys; Step 2: samples, splitters and cuts; Step 3: the
    all-to-all as one device gather and every rank's final sort + unique as one
    dedup of the received rows, cut at the splitters.  Returns (list of per-rank
    distinct partitions, stats dict, splitters, cuts, runs, run offsets)."""
    keys = _dev(keys, torch.int64, "keys")
    dev = keys.device
    total, W = keys.shape
    eo = torch.as_tensor(np.asarray(entry_offsets, dtype=np.int64)).to(dev)
    lib = load()
    lg = (P - 1).bit_length()
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    joint = torch.empty((max(total, 1), W), dtype=torch.int64, device=dev)
    _check(lib.cusci_rank_join(_ptr(keys), W, total, _ptr(eo), int(P), int(n_bits), _ptr(joint),
                               _ptr(status), _stream(stream)), "cusci_rank_join")
    ju, _, ju_n = dedup(joint[:total], n_bits + lg, -1, status=status, stream=stream, sync=False)
    runs = torch.empty((max(total, 1), W), dtype=torch.int64, device=dev)
    run_off = torch.empty(P + 1, dtype=torch.int64, device=dev)
    _check(lib.cusci_rank_runs(_ptr(ju), W, _ptr(ju_n), total, int(P), int(n_bits), _ptr(runs),
                               _ptr(run_off), _stream(stream)), "cusci_rank_runs")
    del joint, ju
    spl, bounds = partition_plan(runs, run_off, P, S, stream=stream)
    recv = torch.empty((max(total, 1), W), dtype=torch.int64, device=dev)
    recv_off = torch.empty(P + 1, dtype=torch.int64, device=dev)
    _check(lib.cusci_partition_exchange(_ptr(runs), W, int(P), _ptr(bounds), _ptr(recv),
                                        _ptr(recv_off), _stream(stream)),
           "cusci_partition_exchange")
    n_recv = int(recv_off[-1].item())                  # the one host read-back
    fu, _, fu_n = dedup(recv[:n_recv], n_bits, n_ones, status=status, stream=stream, sync=False)
    part_off = torch.empty(P + 1, dtype=torch.int64, device=dev)
    spl_full = spl if P > 1 else torch.zeros((1, W), dtype=torch.int64, device=dev)
    _check(lib.cusci_partition_split(_ptr(fu), W, _ptr(fu_n), _ptr(spl_full), int(P),
                                     _ptr(part_off), _stream(stream)), "cusci_partition_split")
    st = int(status.item())
    if st != 0:
        raise CusciError(f"virtual_rank_dedup: device status {st}")
    po = part_off.cpu().numpy()
    ro = run_off.cpu().numpy()
    rv = recv_off.cpu().numpy()
    parts = [fu[po[q]:po[q + 1]] for q in range(P)]
    recv_n = np.diff(rv).astype(np.float64)
    uniq = np.diff(po).astype(np.float64)
    # the paper's load-balance metric: items per rank after the exchange
    stats = {"P": P, "S": S, "received": [int(x) for x in recv_n],
             "unique": [int(x) for x in uniq],
             "max_over_min": float(recv_n.max() / max(recv_n.min(), 1.0)),
             "cv": float(recv_n.std() / recv_n.mean()) if recv_n.mean() > 0 else 0.0,
             "unique_max_over_min": float(uniq.max() / max(uniq.min(), 1.0)),
             "unique_cv": float(uniq.std() / uniq.mean()) if uniq.mean() > 0 else 0.0,
             "local_distinct": [int(x) for x in np.diff(ro)]}
    return parts, stats, spl, bounds, runs[:int(ro[-1])], run_off


class LocalEnergy(torch.autograd.Function):
    """E(psi_u) in the local form of Eq. 5 over CSR coupled lists and the reverse
    index into the distinct set, with its hand-written adjoint."""

    @staticmethod
    def forward(ctx, psi_u, offsets, h, inverse):
        E, n2, y = local_energy_fwd(offsets, h, inverse, psi_u)
        ctx.save_for_backward(psi_u, offsets, h, inverse, E, n2, y)
        return E.reshape(())

    @staticmethod
    def backward(ctx, g):
        psi_u, offsets, h, inverse, E, n2, y = ctx.saved_tensors
        return local_energy_bwd(offsets, h, inverse, psi_u, E, n2, y=y, grad_out=g), None, None, None


class Energy(torch.autograd.Function):
    """E(psi) = psi.H psi / psi.psi over the sorted set S, with the hand-written
    adjoint dE/dpsi = 2 (H psi - E psi) / psi.psi.  ``recompute=True`` keeps no
    H psi between forward and backward (the coupled lists are regenerated)."""

    @staticmethod
    def forward(ctx, psi, system, S, eps, recompute=False):
        E, n2, hp = energy_fwd(system, S, psi, eps, save_hpsi=not recompute)
        ctx.system, ctx.eps, ctx.recompute = system, eps, recompute
        if recompute:
            ctx.save_for_backward(psi, S, E, n2)
        else:
            ctx.save_for_backward(psi, S, E, n2, hp)
        return E.reshape(())

    @staticmethod
    def backward(ctx, g):
        if ctx.recompute:
            psi, S, E, n2 = ctx.saved_tensors
            hp = None
        else:
            psi, S, E, n2, hp = ctx.saved_tensors
        grad = energy_bwd(ctx.system, S, psi, ctx.eps, E, n2, hpsi=hp, grad_out=g)
        return grad, None, None, None, None


class Batch:
    """Many systems generated in one persistent launch and de-duplicated in one
    batched pass (every system's distinct set at once).

    ``plan()`` runs one untimed count/scan to size every buffer; ``run()``
    issues count -> scan -> fill -> batched dedup on the current stream with no
    host synchronisation, so it can be captured with ``capture()`` in a CUDA
    graph and replayed with ``replay()``; the number of launches does not
    depend on the number of systems.
    """

    def __init__(self, systems, dets_list, eps, chunk=8):
        lib = load()
        self.systems = [System.of(s) for s in systems]
        self.eps = float(eps)
        n_src = np.array([d.shape[0] for d in dets_list], dtype=np.int64)
        handles = (_P * len(self.systems))(*[s.handle.value for s in self.systems])
        h = ctypes.c_void_p()
        _check(lib.cusci_batch_create(handles, len(self.systems), n_src.ctypes.data_as(_P),
                                      int(chunk), ctypes.byref(h)), "cusci_batch_create")
        self._h = h
        self._handles = handles
        self.chunk = int(chunk)
        self.src_begin = np.concatenate([[0], np.cumsum(n_src)])
        packed = np.zeros((int(self.src_begin[-1]), 2), dtype=np.uint64)
        for k, d in enumerate(dets_list):
            d = np.ascontiguousarray(d, dtype=np.uint64)
            packed[self.src_begin[k]:self.src_begin[k + 1], :d.shape[1]] = d
        self.d_src = dets_to_device(packed)
        self.n = packed.shape[0]
        self.graph = None

    def set_chunk(self, chunk):
        _check(load().cusci_batch_set_chunk(self._h, int(chunk)), "cusci_batch_set_chunk")
        self.chunk = int(chunk)

    def set_grid(self, blocks_per_sm):
        _check(load().cusci_batch_set_grid(self._h, int(blocks_per_sm)), "cusci_batch_set_grid")
        self.blocks_per_sm = int(blocks_per_sm)

    def count(self, counts, stream=None):
        _check(load().cusci_batch_count(self._h, _ptr(self.d_src), self.eps, _ptr(counts),
                                        _stream(stream)), "cusci_batch_count")

    def gen(self, offsets, out_d, out_h, status=None, stream=None):
        _check(load().cusci_batch_gen(self._h, _ptr(self.d_src), self.eps, _ptr(offsets),
                                      _ptr(out_d), _ptr(out_h), _ptr(status), _stream(stream)),
               "cusci_batch_gen")

    def plan(self):
        dev = self.d_src.device
        self.counts = torch.empty(self.n, dtype=torch.int64, device=dev)
        self.count(self.counts)
        self.scan_ws = torch.empty(scan_workspace(self.n), dtype=torch.uint8, device=dev)
        self.offsets = exclusive_scan(self.counts, workspace=self.scan_ws)
        off = self.offsets.cpu().numpy()
        self.entry_begin = off[self.src_begin]
        self.total = int(off[-1])
        self.out_d = torch.empty((max(self.total, 1), 2), dtype=torch.int64, device=dev)
        self.out_h = torch.empty(max(self.total, 1), dtype=torch.float64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        ws = ctypes.c_size_t()
        _check(load().cusci_batch_dedup_workspace(self._h, self.total, ctypes.byref(ws)),
               "cusci_batch_dedup_workspace")
        self.dd_ws = torch.empty(max(ws.value, 1), dtype=torch.uint8, device=dev)
        self.unique = torch.empty((max(self.total, 1), 2), dtype=torch.int64, device=dev)
        self.inverse = torch.empty(max(self.total, 1), dtype=torch.int32, device=dev)
        self.n_unique = torch.zeros(len(self.systems), dtype=torch.int64, device=dev)
        return self.total

    def run(self, stream=None):
        self.count(self.counts, stream)
        exclusive_scan(self.counts, out=self.offsets, workspace=self.scan_ws, stream=stream)
        self.gen(self.offsets, self.out_d, self.out_h, self.status, stream)
        _check(load().cusci_batch_dedup(self._h, _ptr(self.offsets), _ptr(self.out_d), self.total,
                                        _ptr(self.dd_ws), self.dd_ws.numel(), _ptr(self.unique),
                                        _ptr(self.inverse), _ptr(self.n_unique),
                                        _ptr(self.status), _stream(stream)), "cusci_batch_dedup")

    def autotune(self, candidates=(1, 2, 4, 8, 16, 32, 64), grids=(4, 8, 16), reps=2):
        """Pick the work-item size (sources per item) and the persistent grid
        (blocks per SM) with the fastest whole run (count, scan, fill and
        batched dedup).  Returns ((chunk, blocks_per_sm), ms)."""
        best = None
        for g in grids:
            self.set_grid(g)
            for c in candidates:
                self.set_chunk(c)
                self.run()
                torch.cuda.synchronize()
                t = []
                for _ in range(reps):
                    a, b = (torch.cuda.Event(enable_timing=True),
                            torch.cuda.Event(enable_timing=True))
                    a.record()
                    self.run()
                    b.record()
                    torch.cuda.synchronize()
                    t.append(a.elapsed_time(b))
                ms = min(t)
                if best is None or ms < best[1]:
                    best = ((c, g), ms)
        self.set_chunk(best[0][0])
        self.set_grid(best[0][1])
        return best

    def capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(stream=s)          # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def close(self):
        if getattr(self, "_h", None) is not None and _LIB is not None:
            _LIB.cusci_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

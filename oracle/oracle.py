"""Python face of the CPU oracle (``sc_oracle.c``) and of the brute-force
second-quantized Hamiltonian (``fci_brute.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg.  The library never imports it.  The C sources
are compiled with gcc on first use into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

_SOURCES = ("sc_oracle.c", "fci_brute.c")


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liboracle.so")
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(out) and all(
            os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_count.restype = I64
            lib.orc_count.argtypes = [I, I, I, P, P, D, P, I64, D, P]
            lib.orc_gen.restype = None
            lib.orc_gen.argtypes = [I, I, I, P, P, D, P, I64, D, P, P, P]
            lib.orc_dedup.restype = I64
            lib.orc_dedup.argtypes = [P, I64, I, P, P]
            lib.orc_hpsi.restype = None
            lib.orc_hpsi.argtypes = [I, I, I, P, P, D, P, I64, P, D, P]
            lib.orc_hpsi_rows.restype = None
            lib.orc_hpsi_rows.argtypes = [I, I, I, P, P, D, P, I64, P, D, P, I64, P]
            lib.orc_energy_reduce.restype = None
            lib.orc_energy_reduce.argtypes = [P, P, I64, P, P]
            lib.orc_energy_grad.restype = None
            lib.orc_energy_grad.argtypes = [P, P, I64, D, D, D, P]
            lib.orc_apply_op.restype = I
            lib.orc_apply_op.argtypes = [P, I, I]
            lib.orc_threads.restype = I
            lib.orc_local_energy.restype = None
            lib.orc_local_energy.argtypes = [P, I64, P, P, P, I64, D, P, P, P, P]
            lib.fci_brute_H.restype = I64
            lib.fci_brute_H.argtypes = [I, P, P, D, P, I64, I, P]
            lib.fci_brute_column.restype = I64
            lib.fci_brute_column.argtypes = [I, P, P, D, P, I64, I, P, P]
            _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class OracleSystem:
    """Integrals plus electron counts, held as contiguous FP64 arrays."""

    def __init__(self, norb, n_alpha, n_beta, h1, h2, ecore=0.0):
        self.norb, self.n_alpha, self.n_beta = int(norb), int(n_alpha), int(n_beta)
        self.h1 = _c(h1, np.float64).reshape(norb, norb)
        self.h2 = _c(h2, np.float64).reshape((norb,) * 4)
        self.ecore = float(ecore)
        self.W = (2 * norb + 63) // 64

    @classmethod
    def of(cls, system):
        return cls(system.norb, system.n_alpha, system.n_beta, system.h1, system.h2,
                   getattr(system, "ecore", 0.0))

    def _head(self):
        return (self.norb, self.n_alpha, self.n_beta, _p(self.h1), _p(self.h2), self.ecore)

    def count(self, dets, eps):
        dets = _c(dets, np.uint64).reshape(-1, self.W)
        counts = np.zeros(dets.shape[0], dtype=np.int64)
        _lib().orc_count(*self._head(), _p(dets), dets.shape[0], float(eps), _p(counts))
        return counts

    def gen(self, dets, eps, counts=None):
        """Coupled lists in CSR form: (offsets[n+1], target dets[total, W], H[total])."""
        dets = _c(dets, np.uint64).reshape(-1, self.W)
        if counts is None:
            counts = self.count(dets, eps)
        offsets = np.zeros(dets.shape[0] + 1, dtype=np.int64)
        np.cumsum(counts, out=offsets[1:])
        total = int(offsets[-1])
        out_d = np.zeros((total, self.W), dtype=np.uint64)
        out_h = np.zeros(total, dtype=np.float64)
        _lib().orc_gen(*self._head(), _p(dets), dets.shape[0], float(eps), _p(offsets),
                       _p(out_d), _p(out_h))
        return offsets, out_d, out_h

    def hpsi(self, S, psi, eps):
        S = _c(S, np.uint64).reshape(-1, self.W)
        psi = _c(psi, np.float64)
        out = np.zeros(S.shape[0], dtype=np.float64)
        _lib().orc_hpsi(*self._head(), _p(S), S.shape[0], _p(psi), float(eps), _p(out))
        return out

    def hpsi_rows(self, S, psi, eps, rows):
        """(H psi)_i restricted to S for the chosen rows i of S only (same loop
        as ``hpsi``, so a sample of a large S can be checked)."""
        S = _c(S, np.uint64).reshape(-1, self.W)
        psi = _c(psi, np.float64)
        rows = _c(rows, np.int64)
        assert rows.size == 0 or (rows.min() >= 0 and rows.max() < S.shape[0])
        out = np.zeros(rows.size, dtype=np.float64)
        _lib().orc_hpsi_rows(*self._head(), _p(S), S.shape[0], _p(psi), float(eps), _p(rows),
                             rows.size, _p(out))
        return out

    def energy(self, S, psi, eps, g=1.0):
        """(E, norm2, Hpsi, grad) of E = psi.H psi / psi.psi over the set S."""
        psi = _c(psi, np.float64)
        hp = self.hpsi(S, psi, eps)
        E = np.zeros(1)
        n2 = np.zeros(1)
        _lib().orc_energy_reduce(_p(psi), _p(hp), psi.size, _p(E), _p(n2))
        grad = np.zeros_like(psi)
        _lib().orc_energy_grad(_p(psi), _p(hp), psi.size, float(E[0]), float(n2[0]), float(g),
                               _p(grad))
        return float(E[0]), float(n2[0]), hp, grad


def local_energy(offsets, h, inverse, psi_u, g=1.0):
    """(E, norm2, y, grad_u) of the local-energy form over CSR coupled lists whose
    targets index the distinct set through ``inverse``."""
    offsets = _c(offsets, np.int64)
    h = _c(h, np.float64)
    inverse = _c(inverse, np.int64)
    psi_u = _c(psi_u, np.float64)
    n = offsets.size - 1
    y = np.zeros(n)
    grad = np.zeros(psi_u.size)
    E = np.zeros(1)
    n2 = np.zeros(1)
    _lib().orc_local_energy(_p(offsets), n, _p(h), _p(inverse), _p(psi_u), psi_u.size, float(g),
                            _p(y), _p(E), _p(n2), _p(grad))
    return float(E[0]), float(n2[0]), y, grad


def dedup(keys, W=None):
    """(unique[n_unique, W], inverse[total]) of W-word keys."""
    keys = np.asarray(keys, dtype=np.uint64)
    if keys.ndim == 1:
        keys = keys.reshape(-1, 1 if W is None else W)
    keys = np.ascontiguousarray(keys)
    total, W = keys.shape
    uniq = np.zeros((total, W), dtype=np.uint64)
    inv = np.zeros(total, dtype=np.int64)
    nu = _lib().orc_dedup(_p(keys), total, W, _p(uniq), _p(inv))
    if nu < 0:
        raise MemoryError("oracle dedup: allocation failed")
    return uniq[:nu].copy(), inv


def regular_sampling_plan(runs, P, S):
    """Steps 1-2 of the sort-based regular-sampling de-duplication (Sec. 4.1.1):
    ``runs`` is a list of P sorted distinct arrays of W-word keys ([m, W] uint64).
    Each non-empty run gives S samples at positions floor(k m / S); the sorted
    samples give P-1 splitters at positions ((j+1) count) // P - 1; rank q receives
    the keys k with splitter[q-1] < k <= splitter[q].  Returns (splitters [P-1, W],
    cuts [P, P+1] as positions into the concatenated runs)."""
    W = runs[0].shape[1] if runs else 1
    samples = []
    for r in runs:
        m = r.shape[0]
        for k in range(S if m else 0):
            samples.append(tuple(int(x) for x in r[(k * m) // S][::-1]))   # word W-1 first
    samples.sort()
    count = len(samples)
    spl = []
    for j in range(P - 1):
        at = max(((j + 1) * count) // P - 1, 0)
        spl.append(samples[at] if count else tuple([(1 << 64) - 1] * W))
    cuts = np.zeros((P, P + 1), dtype=np.int64)
    base = 0
    for r_i, r in enumerate(runs):
        keys = [tuple(int(x) for x in row[::-1]) for row in r]
        cuts[r_i, 0] = base
        for q in range(1, P):
            # first position whose key exceeds splitter q-1
            lo, hi = 0, len(keys)
            while lo < hi:
                mid = (lo + hi) // 2
                if keys[mid] <= spl[q - 1]:
                    lo = mid + 1
                else:
                    hi = mid
            cuts[r_i, q] = base + lo
        base += len(keys)
        cuts[r_i, P] = base
    spl_arr = np.array([list(t[::-1]) for t in spl], dtype=np.uint64).reshape(-1, W)
    return spl_arr, cuts


def apply_op(det, s, create):
    """(phase, new det) of a+_s (create) or a_s on one determinant."""
    d = _c(det, np.uint64).copy()
    ph = _lib().orc_apply_op(_p(d), int(s), int(bool(create)))
    return ph, d


def brute_hamiltonian(norb, h1, h2, basis, ecore=0.0):
    """Dense H over a sorted basis by term-by-term second quantization."""
    basis = _c(basis, np.uint64)
    if basis.ndim == 1:
        basis = basis.reshape(-1, 1)
    n, W = basis.shape
    H = np.zeros((n, n), dtype=np.float64)
    outside = _lib().fci_brute_H(int(norb), _p(_c(h1, np.float64)), _p(_c(h2, np.float64)),
                                 float(ecore), _p(basis), n, W, _p(H))
    return H, int(outside)


def brute_column(norb, h1, h2, basis, det, ecore=0.0):
    """Column <basis_r|H|det> over a sorted basis by second quantization; returns
    (column, number of operator strings that left the basis)."""
    basis = _c(basis, np.uint64)
    if basis.ndim == 1:
        basis = basis.reshape(-1, 1)
    n, W = basis.shape
    det = _c(det, np.uint64).reshape(W)
    col = np.zeros(n, dtype=np.float64)
    outside = _lib().fci_brute_column(int(norb), _p(_c(h1, np.float64)), _p(_c(h2, np.float64)),
                                      float(ecore), _p(basis), n, W, _p(det), _p(col))
    return col, int(outside)


def threads() -> int:
    return int(_lib().orc_threads())

"""Seeded synthetic inputs: molecular-like integrals and determinant sets.

This module only draws random inputs.  It holds none of the method's
arithmetic (no matrix elements, no signs, no screening), so both the CPU
oracle and the CUDA path may take their inputs from here.

Conventions shared by every consumer of these inputs
---------------------------------------------------
* ``norb`` spatial orbitals, ``M = 2*norb`` spin orbitals, interleaved:
  spin orbital ``s = 2*p + sigma`` with ``sigma = 0`` for alpha and 1 for beta.
* A determinant is ``W = ceil(M/64)`` little-endian uint64 words; spin orbital
  ``s`` is bit ``s & 63`` of word ``s >> 6``.  Arrays of determinants have shape
  ``(n, W)`` and dtype ``uint64``.
* ``h1`` is ``(norb, norb)`` real symmetric, ``h2`` is ``(norb,)*4`` in
  chemists' notation ``(pq|rs)`` with the 8-fold permutational symmetry of real
  orbitals.

The integral law (N(0,1) entries damped by ``0.5**|p-q|`` per index pair) and the
sources' law (random excitations of rank <= 4 with geometric weights out of the
aufbau determinant) stand in for the molecules of the paper's evaluation
(Sec. 5: N2 cc-pVDZ and Cr2), whose integrals are not available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "integrals", "aufbau", "fci_space", "sample_dets", "pack_occ",
    "words_for", "System", "config_system", "batched_systems", "amplitude_mlp",
]


def words_for(norb: int) -> int:
    return (2 * norb + 63) // 64


def integrals(norb: int, seed: int, decay: float = 0.5):
    """Draw (h1, h2) from ``default_rng(seed)``.

    h1: upper triangle in row-major order (p <= q), entry N(0,1)*decay**|p-q|,
    mirrored.  h2: one draw per symmetry-distinct quadruple, taken in the order
    ``for pq in range(npair): for rs in range(pq+1)`` with the compound index
    ``pq = p*(p+1)//2 + q`` (p >= q), entry N(0,1)*decay**(|p-q|+|r-s|),
    written to all 8 permutations.
    """
    rng = np.random.default_rng(seed)
    iu_p, iu_q = np.triu_indices(norb)
    v1 = rng.standard_normal(iu_p.size) * decay ** np.abs(iu_p - iu_q)
    h1 = np.zeros((norb, norb))
    h1[iu_p, iu_q] = v1
    h1[iu_q, iu_p] = v1

    pp, qq = np.tril_indices(norb)          # compound pair order pq = p(p+1)/2+q
    npair = pp.size
    a, b = np.tril_indices(npair)           # for pq: for rs <= pq
    p, q, r, s = pp[a], qq[a], pp[b], qq[b]
    v2 = rng.standard_normal(a.size) * decay ** (np.abs(p - q) + np.abs(r - s))
    h2 = np.zeros((norb,) * 4)
    for (i, j, k, l) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                         (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
        h2[i, j, k, l] = v2
    return h1, h2


def pack_occ(occ: np.ndarray) -> np.ndarray:
    """Pack a boolean occupation matrix (n, M) into (n, W) uint64 words."""
    occ = np.asarray(occ, dtype=bool)
    n, m = occ.shape
    w = (m + 63) // 64
    padded = np.zeros((n, 64 * w), dtype=bool)
    padded[:, :m] = occ
    by = np.packbits(padded, axis=1, bitorder="little")
    return np.ascontiguousarray(by).view("<u8").astype(np.uint64).reshape(n, w)


def aufbau(norb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    occ = np.zeros((1, 2 * norb), dtype=bool)
    occ[0, 0:2 * n_alpha:2] = True
    occ[0, 1:2 * n_beta:2] = True
    return pack_occ(occ)


def _sort_words(dets: np.ndarray) -> np.ndarray:
    """Ascending order of W-word unsigned keys, word W-1 most significant."""
    keys = [dets[:, w] for w in range(dets.shape[1])]   # lexsort: last key is primary
    return dets[np.lexsort(keys)]


def fci_space(norb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Every determinant with n_alpha alpha and n_beta beta electrons, sorted."""
    from itertools import combinations
    alpha = list(combinations(range(norb), n_alpha))
    beta = list(combinations(range(norb), n_beta))
    occ = np.zeros((len(alpha) * len(beta), 2 * norb), dtype=bool)
    k = 0
    for ca in alpha:
        for cb in beta:
            occ[k, [2 * p for p in ca]] = True
            occ[k, [2 * p + 1 for p in cb]] = True
            k += 1
    return _sort_words(pack_occ(occ))


def _space_size_le4(norb, n_alpha, n_beta, max_rank=4):
    va, vb = norb - n_alpha, norb - n_beta
    tot = 0
    for ra in range(0, max_rank + 1):
        for rb in range(0, max_rank + 1 - ra):
            tot += (math.comb(n_alpha, ra) * math.comb(va, ra)
                    * math.comb(n_beta, rb) * math.comb(vb, rb))
    return tot


def sample_dets(norb: int, n_alpha: int, n_beta: int, n: int, seed: int,
                max_rank: int = 4, batch: int = 65536) -> np.ndarray:
    """Sample ``n`` distinct determinants as random excitations of the aufbau one.

    Each draw: rank r in {0..max_rank} with P(r) proportional to 2**-r; r distinct
    occupied spin orbitals of the aufbau determinant chosen uniformly (the first
    r of a random permutation); each moved, in that order, to a distinct uniformly
    chosen virtual of the same spin (taken from a random permutation of that
    spin's virtuals).  Draws needing more virtuals than a spin has are rejected,
    duplicates are rejected (first occurrence kept) until ``n`` distinct
    determinants exist; the result is then shuffled with the same generator.
    If fewer than ``n`` determinants of rank <= max_rank exist, all of them are
    returned (shuffled).
    """
    rng = np.random.default_rng(seed)
    m = 2 * norb
    total_space = _space_size_le4(norb, n_alpha, n_beta, max_rank)
    n = min(n, total_space)
    occ_a = np.arange(n_alpha) * 2
    occ_b = np.arange(n_beta) * 2 + 1
    occ_all = np.concatenate([occ_a, occ_b])
    vir_a = np.arange(n_alpha, norb) * 2
    vir_b = np.arange(n_beta, norb) * 2 + 1
    n_occ = occ_all.size
    w_r = 2.0 ** -np.arange(max_rank + 1)
    w_r /= w_r.sum()
    base = np.zeros(m, dtype=bool)
    base[occ_all] = True

    seen = {}
    order = []
    W = words_for(norb)
    while len(order) < n:
        r = rng.choice(max_rank + 1, size=batch, p=w_r)
        perm_occ = np.argsort(rng.random((batch, max(n_occ, 1))), axis=1)
        perm_va = np.argsort(rng.random((batch, max(vir_a.size, 1))), axis=1)
        perm_vb = np.argsort(rng.random((batch, max(vir_b.size, 1))), axis=1)
        occ = np.broadcast_to(base, (batch, m)).copy()
        ok = np.ones(batch, dtype=bool)
        used_a = np.zeros(batch, dtype=np.int64)
        used_b = np.zeros(batch, dtype=np.int64)
        rows = np.arange(batch)
        for t in range(max_rank):
            act = (r > t) & ok
            if not act.any() or n_occ == 0:
                break
            src = occ_all[perm_occ[:, min(t, n_occ - 1)]]
            if t >= n_occ:
                ok &= ~act
                continue
            is_a = (src % 2) == 0
            need_a = act & is_a
            need_b = act & ~is_a
            ok &= ~(need_a & (used_a >= vir_a.size))
            ok &= ~(need_b & (used_b >= vir_b.size))
            need_a &= ok
            need_b &= ok
            if vir_a.size:
                ia = perm_va[rows, np.minimum(used_a, vir_a.size - 1)]
                dst_a = vir_a[ia]
            else:
                dst_a = np.zeros(batch, dtype=np.int64)
            if vir_b.size:
                ib = perm_vb[rows, np.minimum(used_b, vir_b.size - 1)]
                dst_b = vir_b[ib]
            else:
                dst_b = np.zeros(batch, dtype=np.int64)
            sel = rows[need_a]
            occ[sel, src[need_a]] = False
            occ[sel, dst_a[need_a]] = True
            sel = rows[need_b]
            occ[sel, src[need_b]] = False
            occ[sel, dst_b[need_b]] = True
            used_a += need_a
            used_b += need_b
        packed = pack_occ(occ[ok])
        for row in packed:
            key = row.tobytes()
            if key not in seen:
                seen[key] = len(order)
                order.append(row)
                if len(order) == n:
                    break
    dets = np.array(order, dtype=np.uint64).reshape(n, W)
    return dets[rng.permutation(n)]


@dataclass
class System:
    """One synthetic molecular-like system and its source determinants."""
    name: str
    norb: int
    n_alpha: int
    n_beta: int
    h1: np.ndarray
    h2: np.ndarray
    dets: np.ndarray
    eps: float
    ecore: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def W(self) -> int:
        return words_for(self.norb)


# name -> (norb, n_alpha, n_beta, n_dets, eps, integral seed, det seed)
_CONFIGS = {
    "tiny": (8, 4, 4, None, 0.0, 0, None),
    "mid": (26, 7, 7, 100_000, 1e-8, 0, 102),
    "large": (60, 10, 10, 20_000, 1e-6, 0, 103),
    "energy": (26, 7, 7, 200_000, 1e-8, 0, 104),
}


def config_system(name: str, n_dets: int | None = None) -> System:
    """The named workload: 'tiny' (16 spin orbitals, 4a+4b, whole FCI space),
    'mid' (52 spin orbitals, 7a+7b, 100k sources), 'large' (120 spin orbitals,
    10a+10b, 20k sources) or 'energy' (the 'mid' system with a 200k selected
    space, returned sorted).  ``n_dets`` overrides the source count."""
    norb, na, nb, nd, eps, iseed, dseed = _CONFIGS[name]
    h1, h2 = integrals(norb, iseed)
    if nd is None:
        dets = fci_space(norb, na, nb)
        if n_dets is not None:
            dets = dets[:n_dets]
    else:
        dets = sample_dets(norb, na, nb, n_dets or nd, dseed)
        if name == "energy":
            dets = _sort_words(dets)
    return System(name, norb, na, nb, h1, h2, dets, eps)


def batched_systems(n_systems: int = 64, scale: float = 1.0) -> list[System]:
    """Independent systems of uneven size: system s draws, from
    ``default_rng(1000+s)``, norb uniform in [10, 50], an electron count n
    uniform in [4, 16] split n_alpha=ceil(n/2), n_beta=floor(n/2), and a source
    count floor(exp(U(ln 1e3, ln 5e4))) (times ``scale``); integrals come from
    ``default_rng(1000+s)`` after those draws are spent, sources from
    ``default_rng(100000+s)``."""
    out = []
    for s in range(n_systems):
        rng = np.random.default_rng(1000 + s)
        norb = int(rng.integers(10, 51))
        n = int(rng.integers(4, 17))
        na, nb = min((n + 1) // 2, norb), min(n // 2, norb)
        nd = int(math.floor(math.exp(rng.uniform(math.log(1e3), math.log(5e4)))))
        nd = max(1, int(nd * scale))
        h1, h2 = integrals(norb, int(rng.integers(0, 2**31)))
        dets = sample_dets(norb, na, nb, nd, 100000 + s)
        out.append(System(f"sys{s}", norb, na, nb, h1, h2, dets, 1e-8))
    return out


def amplitude_mlp(dets: np.ndarray, norb: int, device="cuda"):
    """The energy workload's network: a 2*norb -> 256 -> 256 -> 1 tanh MLP with
    FP32 weights from ``torch.manual_seed(0)`` (PyTorch's default init), and its
    input, the occupation bits (0/1, FP32) of the first word of each
    determinant.  psi = exp(net(x)) in FP64 is the amplitude of each
    determinant.  Returns (net, x) on ``device``."""
    import torch
    torch.manual_seed(0)
    net = torch.nn.Sequential(torch.nn.Linear(2 * norb, 256), torch.nn.Tanh(),
                              torch.nn.Linear(256, 256), torch.nn.Tanh(),
                              torch.nn.Linear(256, 1)).to(device)
    bits = ((dets[:, :1] >> np.arange(2 * norb, dtype=np.uint64)) & np.uint64(1)).astype(np.float32)
    return net, torch.from_numpy(bits).to(device)

"""Pins of the CPU oracle to things other than itself (CPU only).

* a Jordan-Wigner construction of H as products of dense operator matrices in
  the Fock space (pure numpy, shares nothing with the C files);
* the term-by-term second-quantized brute force in ``oracle/fci_brute.c``;
* closed-form excitation counts per spin sector;
* the one-body special case (h2 = 0), whose ground energy is the sum of the
  lowest orbital energies of h1 per spin;
* the Rayleigh quotient at an exact eigenvector (E = lambda, gradient 0), its
  scale invariance and a central finite-difference check of the gradient;
* de-duplication against Python's set / sorted on random keys.
A plausible slip anywhere in the oracle -- a dropped exchange term, a wrong
phase or index, a transposed integral -- changes at least one of these.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_15768_gb300 import synth


def _dense_from_lists(dets, offsets, tdets, hvals):
    """Dense H[target, source] over the sorted basis ``dets`` from CSR lists."""
    keys = [tuple(r) for r in dets.tolist()]
    index = {k: i for i, k in enumerate(keys)}
    n = len(keys)
    H = np.zeros((n, n))
    for c in range(n):
        for e in range(offsets[c], offsets[c + 1]):
            H[index[tuple(tdets[e].tolist())], c] = hvals[e]
    return H


def _jordan_wigner_H(norb, h1, h2):
    """H in the full Fock space of M = 2 norb modes, basis index = bitstring."""
    M = 2 * norb
    dim = 1 << M
    ann = []
    for s in range(M):
        a = np.zeros((dim, dim))
        for x in range(dim):
            if (x >> s) & 1:
                a[x ^ (1 << s), x] = -1.0 if bin(x & ((1 << s) - 1)).count("1") % 2 else 1.0
        ann.append(a)
    cre = [a.T.copy() for a in ann]
    H = np.zeros((dim, dim))
    for sg in range(2):
        for p in range(norb):
            for q in range(norb):
                H += h1[p, q] * (cre[2 * p + sg] @ ann[2 * q + sg])
    for sg in range(2):
        for tau in range(2):
            for p in range(norb):
                for q in range(norb):
                    left = cre[2 * p + sg]
                    right = ann[2 * q + sg]
                    for r in range(norb):
                        lr = left @ cre[2 * r + tau]
                        for s in range(norb):
                            c = h2[p, q, r, s]
                            if c != 0.0:
                                H += 0.5 * c * (lr @ ann[2 * s + tau] @ right)
    return H


@pytest.mark.parametrize("na,nb", [(2, 1), (1, 1), (2, 0), (3, 2)])
def test_oracle_matches_jordan_wigner(na, nb):
    norb = 3
    h1, h2 = synth.integrals(norb, seed=7)
    basis = synth.fci_space(norb, na, nb)
    osys = O.OracleSystem(norb, na, nb, h1, h2)
    off, td, hv = osys.gen(basis, -1.0)
    H = _dense_from_lists(basis, off, td, hv)
    Hjw = _jordan_wigner_H(norb, h1, h2)
    idx = basis[:, 0].astype(np.int64)
    Hs = Hjw[np.ix_(idx, idx)]
    scale = np.abs(Hs).max()
    assert np.abs(H - Hs).max() <= 1e-12 * scale


def test_oracle_matches_brute_force_tiny():
    s = synth.config_system("tiny")
    Hb, outside = O.brute_hamiltonian(s.norb, s.h1, s.h2, s.dets)
    assert outside == 0
    off, td, hv = O.OracleSystem.of(s).gen(s.dets, -1.0)
    H = _dense_from_lists(s.dets, off, td, hv)
    assert np.abs(H - Hb).max() <= 1e-12 * np.abs(Hb).max()
    # Hermiticity holds exactly: forward and reverse elements use the same terms
    assert np.array_equal(H, H.T)
    # the coupled lists hold exactly the pairs within two electron moves
    x = s.dets[:, 0]
    diff = np.array([[bin(int(a) ^ int(b)).count("1") // 2 for b in x[:200]] for a in x[:200]])
    assert np.array_equal(diff <= 2, H[:200, :200] != 0)


def test_oracle_column_matches_brute_force_two_words():
    """W = 2 (68 spin orbitals), electrons straddling the 64-bit word boundary."""
    norb = 34
    h1, h2 = synth.integrals(norb, seed=3)
    occ = np.zeros((1, 2 * norb), dtype=bool)
    for so in (62, 64, 1, 67, 30):      # alpha 31, 32, 15; beta 0, 33
        occ[0, so] = True
    D = synth.pack_occ(occ)
    na, nb = 3, 2
    osys = O.OracleSystem(norb, na, nb, h1, h2)
    off, td, hv = osys.gen(D, -1.0)
    order = np.lexsort([td[:, 0], td[:, 1]])   # word 1 most significant
    basis = td[order]
    col, _ = O.brute_column(norb, h1, h2, basis, D[0])
    mine = hv[order]
    assert np.abs(col - mine).max() <= 1e-12 * np.abs(col).max()


def _closed_form(norb, na, nb):
    va, vb = norb - na, norb - nb
    return (1 + na * va + nb * vb + math.comb(na, 2) * math.comb(va, 2)
            + math.comb(nb, 2) * math.comb(vb, 2) + na * va * nb * vb)


@pytest.mark.parametrize("norb,na,nb,seed", [
    (8, 4, 4, 0), (26, 7, 7, 1), (60, 10, 10, 2), (12, 5, 0, 3), (10, 10, 3, 4),
    (33, 1, 1, 5), (64, 3, 2, 6)])
def test_counts_closed_form(norb, na, nb, seed):
    h1, h2 = synth.integrals(norb, seed=seed)
    dets = synth.sample_dets(norb, na, nb, 6, seed=seed + 50)
    counts = O.OracleSystem(norb, na, nb, h1, h2).count(dets, -1.0)
    assert (counts == _closed_form(norb, na, nb)).all()


def test_one_body_spectrum():
    norb, na, nb = 6, 3, 2
    h1, _ = synth.integrals(norb, seed=11)
    h2 = np.zeros((norb,) * 4)
    basis = synth.fci_space(norb, na, nb)
    off, td, hv = O.OracleSystem(norb, na, nb, h1, h2).gen(basis, -1.0)
    H = _dense_from_lists(basis, off, td, hv)
    e = np.linalg.eigvalsh(h1)
    assert abs(np.linalg.eigvalsh(H)[0] - (e[:na].sum() + e[:nb].sum())) < 1e-12


def test_energy_at_eigenvector():
    s = synth.config_system("tiny")
    osys = O.OracleSystem.of(s)
    off, td, hv = osys.gen(s.dets, -1.0)
    H = _dense_from_lists(s.dets, off, td, hv)
    w, V = np.linalg.eigh(H)
    psi = V[:, 0]
    E, n2, hp, grad = osys.energy(s.dets, psi, -1.0)
    assert abs(E - w[0]) < 1e-10
    assert np.abs(grad).max() < 1e-10
    assert abs(n2 - 1.0) < 1e-13


def test_energy_gradient_finite_difference_and_invariants():
    s = synth.config_system("mid", n_dets=400)
    order = np.lexsort([s.dets[:, 0]])
    S = s.dets[order]
    osys = O.OracleSystem.of(s)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(S.shape[0])
    E, n2, hp, grad = osys.energy(S, psi, s.eps)
    # scale invariance
    E2, _, _, grad2 = osys.energy(S, 3.0 * psi, s.eps)
    assert abs(E2 - E) <= 1e-13 * abs(E)
    assert abs(np.dot(psi, grad)) <= 1e-10 * np.linalg.norm(psi) * np.linalg.norm(grad)
    # central differences in psi
    h = 1e-6
    for k in rng.choice(S.shape[0], 12, replace=False):
        e = np.zeros_like(psi)
        e[k] = h
        Ep = osys.energy(S, psi + e, s.eps)[0]
        Em = osys.energy(S, psi - e, s.eps)[0]
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(grad[k]))
    # H psi against a dense product restricted to S
    off, td, hv = osys.gen(S, s.eps)
    pos = {tuple(r): i for i, r in enumerate(S.tolist())}
    ref = np.zeros(S.shape[0])
    for i in range(S.shape[0]):
        for e_ in range(off[i], off[i + 1]):
            j = pos.get(tuple(td[e_].tolist()))
            if j is not None:
                ref[i] += hv[e_] * psi[j]
    assert np.abs(ref - hp).max() <= 1e-12 * np.abs(ref).max()
    # the row-subset form (for samples of a large S) against the same product
    rows = np.concatenate([[0, S.shape[0] - 1], rng.choice(S.shape[0], 40, replace=False)])
    hr = osys.hpsi_rows(S, psi, s.eps, rows)
    assert np.abs(hr - ref[rows]).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(hr, hp[rows])


def test_hpsi_rows_two_words_against_dense_product():
    s = synth.config_system("large", n_dets=60)
    S = s.dets[np.lexsort([s.dets[:, w] for w in range(s.dets.shape[1])])]
    osys = O.OracleSystem.of(s)
    psi = np.random.default_rng(8).standard_normal(S.shape[0])
    off, td, hv = osys.gen(S, s.eps)
    pos = {tuple(r): i for i, r in enumerate(S.tolist())}
    ref = np.zeros(S.shape[0])
    for i in range(S.shape[0]):
        for e_ in range(off[i], off[i + 1]):
            j = pos.get(tuple(td[e_].tolist()))
            if j is not None:
                ref[i] += hv[e_] * psi[j]
    rows = np.array([59, 3, 17, 0, 42], dtype=np.int64)
    hr = osys.hpsi_rows(S, psi, s.eps, rows)
    assert np.abs(hr - ref[rows]).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("W", [1, 2])
def test_dedup_against_python_set(W):
    rng = np.random.default_rng(W)
    keys = rng.integers(0, 50, size=(5000, W)).astype(np.uint64)
    keys[:, -1] |= np.uint64(1) << np.uint64(63)     # exercise the top bit
    uniq, inv = O.dedup(keys)
    ref = sorted(set(tuple(int(x) for x in r[::-1]) for r in keys))   # word W-1 first
    assert [tuple(int(x) for x in r[::-1]) for r in uniq] == ref
    assert np.array_equal(uniq[inv], keys)


def test_dedup_edge_cases():
    uniq, inv = O.dedup(np.zeros((0, 1), dtype=np.uint64))
    assert uniq.shape[0] == 0 and inv.shape[0] == 0
    k = np.full((7, 1), 42, dtype=np.uint64)
    uniq, inv = O.dedup(k)
    assert uniq.shape[0] == 1 and (inv == 0).all()


def test_screening_is_strict_and_keeps_diagonal():
    s = synth.config_system("mid", n_dets=50)
    osys = O.OracleSystem.of(s)
    off, td, hv = osys.gen(s.dets, 0.05)
    for i in range(50):
        assert np.array_equal(td[off[i]], s.dets[i])      # diagonal first, always kept
        assert (np.abs(hv[off[i] + 1:off[i + 1]]) > 0.05).all()
    huge = osys.count(s.dets, 1e300)
    assert (huge == 1).all()


def test_tiny_spectrum_golden():
    """The oracle's coupled lists reproduce the stored brute-force spectrum."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_spectrum.txt")
    ref = np.array([float(x) for x in open(path) if not x.startswith("#")])
    s = synth.config_system("tiny")
    off, td, hv = O.OracleSystem.of(s).gen(s.dets, -1.0)
    H = _dense_from_lists(s.dets, off, td, hv)
    assert np.abs(np.linalg.eigvalsh(H)[:5] - ref).max() < 1e-10


def test_local_energy_equals_variational_energy_on_closed_space():
    """On the whole FCI space every coupled target is a source, so the local-energy
    form (Eq. 5) equals the Rayleigh quotient over S (pinned above by eigh)."""
    s = synth.config_system("tiny")
    osys = O.OracleSystem.of(s)
    off, td, hv = osys.gen(s.dets, -1.0)
    u, inv = O.dedup(td)
    assert np.array_equal(u, s.dets)                   # the distinct set is the space
    rng = np.random.default_rng(4)
    psi = rng.standard_normal(u.shape[0])
    E_loc, n2, y, grad = O.local_energy(off, hv, inv, psi)
    E_var, n2v, hp, gvar = osys.energy(s.dets, psi, -1.0)
    assert abs(E_loc - E_var) <= 1e-12 * abs(E_var)
    assert np.abs(y - hp).max() <= 1e-11
    # on a closed space the two gradients coincide as well (H symmetric)
    assert np.abs(grad - gvar).max() <= 1e-11


def test_local_energy_gradient_finite_differences():
    s = synth.config_system("mid", n_dets=60)
    off, td, hv = O.OracleSystem.of(s).gen(s.dets, s.eps)
    u, inv = O.dedup(td)
    rng = np.random.default_rng(6)
    psi = rng.standard_normal(u.shape[0]) * 0.1 + 1.0
    E, n2, y, grad = O.local_energy(off, hv, inv, psi)
    h = 1e-6
    # include source entries (diagonal targets) and pure targets
    src_ids = inv[off[:-1]]
    picks = list(src_ids[:5]) + list(rng.choice(u.shape[0], 8, replace=False))
    for k in picks:
        e = np.zeros_like(psi)
        e[k] = h
        fd = (O.local_energy(off, hv, inv, psi + e)[0] - O.local_energy(off, hv, inv, psi - e)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(grad[k]))


def test_regular_sampling_plan_hand_example():
    """Two ranks, two samples each: runs [1 3 5 7] and [2 4 6 8] sample {1, 5} and
    {2, 6}; the sorted sample [1 2 5 6] gives the splitter at (1*4)//2 - 1 = 1,
    i.e. the key 2, so rank 0 receives keys <= 2 and rank 1 the rest."""
    r0 = np.array([[1], [3], [5], [7]], dtype=np.uint64)
    r1 = np.array([[2], [4], [6], [8]], dtype=np.uint64)
    spl, cuts = O.regular_sampling_plan([r0, r1], 2, 2)
    assert spl.tolist() == [[2]]
    assert cuts.tolist() == [[0, 1, 4], [4, 5, 8]]


def test_regular_sampling_partition_covers_the_distinct_set():
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 5000, size=(20000, 1)).astype(np.uint64)
    P, S = 8, 16
    runs = [O.dedup(c)[0] for c in np.array_split(keys, P)]
    spl, cuts = O.regular_sampling_plan(runs, P, S)
    allr = np.concatenate(runs)
    parts = []
    for q in range(P):
        recv = np.concatenate([allr[cuts[r, q]:cuts[r, q + 1]] for r in range(P)])
        u = O.dedup(recv)[0] if recv.size else recv.reshape(0, 1)
        if q > 0 and u.size:
            assert (u[:, 0] > spl[q - 1, 0]).all()
        if q < P - 1 and u.size:
            assert (u[:, 0] <= spl[q, 0]).all()
        parts.append(u)
    assert np.array_equal(np.concatenate(parts), O.dedup(keys)[0])

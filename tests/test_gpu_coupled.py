"""GPU parity of the count / scan / fill passes against the CPU oracle.

Coupled sets, their canonical order and the signs are compared bit-exactly; the
FP64 elements to 1e-12 relative (the kernels are built to reproduce the
oracle's summation order, so they are in fact bit-identical, which the tests
also record)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import assert_h_close, to_dev, to_np

pytestmark = pytest.mark.gpu


def run_gpu(system, dets, eps):
    sysd = cusci.System.of(system)
    d = to_dev(dets)
    off, od, oh, st = cusci.coupled(sysd, d, eps)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return off.cpu().numpy(), to_np(od), oh.cpu().numpy()


def compare(system, dets, eps):
    off, od, oh = run_gpu(system, dets, eps)
    o_off, o_d, o_h = O.OracleSystem.of(system).gen(dets, eps)
    assert np.array_equal(off, o_off)
    assert np.array_equal(od, o_d)
    assert_h_close(oh, o_h)
    # elements carry the same sign bit and, by construction, the same bits
    assert np.array_equal(np.signbit(oh), np.signbit(o_h))
    return np.array_equal(oh.view(np.uint64), o_h.view(np.uint64))


def test_tiny_full_fci_space():
    s = synth.config_system("tiny")
    assert compare(s, s.dets, s.eps)


@pytest.mark.parametrize("eps", [-1.0, 0.0, 1e-8, 1e-3, 0.1])
def test_mid_prefix_eps(eps):
    s = synth.config_system("mid")
    # 257 sources: more than 32 warps' worth and a ragged tail
    assert compare(s, s.dets[:257], eps)


def test_large_two_words_prefix():
    s = synth.config_system("large")
    assert compare(s, s.dets[:24], s.eps)


@pytest.mark.parametrize("norb,na,nb", [(12, 5, 0), (10, 10, 3), (33, 1, 1), (64, 3, 2),
                                        (32, 4, 4), (1, 1, 0), (5, 0, 0)])
def test_edge_systems(norb, na, nb):
    h1, h2 = synth.integrals(norb, seed=norb)
    s = synth.System("edge", norb, na, nb, h1, h2,
                     synth.sample_dets(norb, na, nb, 40, seed=9), 1e-10)
    assert compare(s, s.dets, s.eps)


def test_word_boundary_sources():
    norb = 34
    h1, h2 = synth.integrals(norb, seed=3)
    occ = np.zeros((3, 2 * norb), dtype=bool)
    for row, sos in enumerate([(62, 64, 1, 67, 30), (63, 65, 0, 2, 4), (60, 61, 62, 63, 66)]):
        occ[row, list(sos)] = True
    dets = synth.pack_occ(occ)
    s = synth.System("wb", norb, 3, 2, h1, h2, dets, -1.0)
    # rows have different spin splits: compare each with its own electron counts
    for r in range(3):
        na = int(occ[r, 0::2].sum())
        nb = int(occ[r, 1::2].sum())
        sr = synth.System("wb", norb, na, nb, h1, h2, dets[r:r + 1], -1.0)
        assert compare(sr, sr.dets, -1.0)


def test_single_source_and_huge_eps():
    s = synth.config_system("mid")
    off, od, oh = run_gpu(s, s.dets[:1], s.eps)
    assert off[0] == 0 and off[1] > 1
    off, od, oh = run_gpu(s, s.dets[:100], 1e300)
    assert np.array_equal(np.diff(off), np.ones(100, dtype=np.int64))
    assert np.array_equal(od, s.dets[:100])


def test_empty_input():
    s = synth.config_system("tiny")
    sysd = cusci.System.of(s)
    d = torch.zeros((0, 1), dtype=torch.int64, device="cuda")
    c = cusci.count_coupled(sysd, d, 0.0)
    off = cusci.exclusive_scan(c)
    assert off.shape[0] == 1 and int(off[0].item()) == 0


def test_offsets_mismatch_reports_overflow():
    s = synth.config_system("mid")
    sysd = cusci.System.of(s)
    d = to_dev(s.dets[:8])
    counts = cusci.count_coupled(sysd, d, s.eps)
    counts[3] -= 5                    # host-made inconsistency, writes stay in range
    off = cusci.exclusive_scan(counts)
    total = int(off[-1].item())
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cusci.gen_coupled(sysd, d, s.eps, off, total, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 4


def test_check_dets_flags_bad_rows():
    s = synth.config_system("mid")
    sysd = cusci.System.of(s)
    good = to_dev(s.dets[:64])
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cusci.check_dets(sysd, good, st)
    assert int(st.item()) == 0
    bad = s.dets[:64].copy()
    bad[7, 0] |= np.uint64(1) << np.uint64(60)        # above M = 52
    cusci.check_dets(sysd, to_dev(bad), st)
    assert int(st.item()) == 1


def test_full_size_sampled_rows():
    """At the benchmark's size (100k sources, eps 1e-8) compare the CSR counts of
    every source with the closed-form bound and 64 sampled rows with the oracle."""
    s = synth.config_system("mid")
    sysd = cusci.System.of(s)
    d = to_dev(s.dets)
    off, od, oh, st = cusci.coupled(sysd, d, s.eps)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    off = off.cpu().numpy()
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(s.dets.shape[0], 64, replace=False))
    o_off, o_d, o_h = O.OracleSystem.of(s).gen(s.dets[rows], s.eps)
    for k, r in enumerate(rows):
        a, b = int(off[r]), int(off[r + 1])
        assert b - a == o_off[k + 1] - o_off[k]
        assert np.array_equal(to_np(od[a:b]), o_d[o_off[k]:o_off[k + 1]])
        assert_h_close(oh[a:b].cpu().numpy(), o_h[o_off[k]:o_off[k + 1]])

"""Many independent systems in one persistent launch: per system, the coupled
lists and the de-duplication equal the oracle's (and the single-system path),
also when the whole sequence is replayed from a CUDA graph."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import assert_h_close, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    systems = synth.batched_systems(10, scale=0.03)
    b = cusci.Batch(systems, [s.dets for s in systems], 1e-8, chunk=4)
    b.plan()
    return systems, b


def expect(system):
    off, td, hv = O.OracleSystem.of(system).gen(system.dets, system.eps)
    u, inv = O.dedup(td)
    return off, td, hv, u, inv


def check_all(systems, b):
    out_d = to_np(b.out_d)
    out_h = b.out_h.cpu().numpy()
    uniq = to_np(b.unique)
    inv = b.inverse.cpu().numpy()
    nus = b.n_unique.cpu().numpy()
    offs = b.offsets.cpu().numpy()
    assert int(b.status.item()) == 0
    for k, s in enumerate(systems):
        o_off, o_d, o_h, o_u, o_inv = expect(s)
        a, z = int(b.entry_begin[k]), int(b.entry_begin[k + 1])
        s0, s1 = b.src_begin[k], b.src_begin[k + 1]
        assert np.array_equal(offs[s0:s1 + 1] - a, o_off)
        W = s.W
        assert np.array_equal(out_d[a:z, :W], o_d)
        if W == 1:
            assert (out_d[a:z, 1] == 0).all()
        assert_h_close(out_h[a:z], o_h)
        assert nus[k] == o_u.shape[0]
        assert np.array_equal(uniq[a:a + nus[k], :W], o_u)
        assert np.array_equal(inv[a:z], o_inv)


def test_batch_matches_oracle_per_system(batch):
    systems, b = batch
    b.run()
    torch.cuda.synchronize()
    check_all(systems, b)


def test_batch_matches_single_system_path(batch):
    systems, b = batch
    b.run()
    torch.cuda.synchronize()
    for k in (0, 3, 7):
        s = systems[k]
        sysd = cusci.System.of(s)
        off, od, oh, st = cusci.coupled(sysd, cusci.dets_to_device(s.dets), s.eps)
        a, z = int(b.entry_begin[k]), int(b.entry_begin[k + 1])
        assert torch.equal(b.out_d[a:z, :s.W], od)
        assert torch.equal(b.out_h[a:z], oh)


def test_batch_graph_replay_and_autotune(batch):
    systems, b = batch
    (best_chunk, best_grid), ms = b.autotune(candidates=(1, 4, 16), grids=(4, 8), reps=1)
    assert best_chunk in (1, 4, 16) and best_grid in (4, 8) and ms > 0
    b.capture()
    b.out_h.zero_()
    b.inverse.zero_()
    b.replay()
    torch.cuda.synchronize()
    check_all(systems, b)


def test_batch_replay_unaffected_by_other_eps_on_its_systems(batch):
    """The batch screens with masks of its own: generating one of its systems
    at five other eps values (more than the system's mask cache holds) between
    two graph replays must not change what the replay produces."""
    systems, b = batch
    if b.graph is None:
        b.capture()
    k = 2
    s = systems[k]
    d = cusci.dets_to_device(s.dets)
    for eps in (1e-3, 1e-4, 1e-5, 1e-6, 1e-7):
        cusci.coupled(b.systems[k], d, eps)
    torch.cuda.synchronize()
    b.out_h.zero_()
    b.inverse.zero_()
    b.replay()
    torch.cuda.synchronize()
    check_all(systems, b)


def test_batch_edge_cases_single_system_one_source_and_twins():
    """A batch of one system; a system with a single source; two identical
    systems side by side (their joint keys must stay apart, so each keeps its
    own distinct set and ids)."""
    base = synth.batched_systems(6, scale=0.02)
    one_src = dataclasses.replace(base[1], dets=base[1].dets[:1])
    for systems in ([base[0]], [one_src, base[2]], [base[3], base[3], base[4]]):
        b = cusci.Batch(systems, [s.dets for s in systems], 1e-8, chunk=2)
        b.plan()
        b.run()
        torch.cuda.synchronize()
        check_all(systems, b)
        b.close()

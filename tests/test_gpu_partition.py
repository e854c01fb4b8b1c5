"""The paper's sort-based regular-sampling de-duplication (Sec. 4.1.1) over P
virtual ranks on one GPU: splitters and cuts bit-exact against the oracle's
restatement of Steps 1-2, and the ranks' final partitions concatenate to the
global distinct set."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n,P,S", [("mid", 400, 4, 64), ("mid", 400, 16, 128),
                                        ("mid", 300, 5, 32), ("mid", 200, 1, 16),
                                        ("large", 24, 8, 64)])
def test_virtual_ranks_match_oracle(name, n, P, S):
    s = synth.config_system(name)
    sysd = cusci.System.of(s)
    off, od, oh, st = cusci.coupled(sysd, cusci.dets_to_device(s.dets[:n]), s.eps)
    src_cut = np.linspace(0, n, P + 1).astype(np.int64)
    eo = off.cpu().numpy()[src_cut]
    parts, stats, spl, bounds, runs, run_off = cusci.virtual_rank_dedup(
        od, eo, P, S, 2 * s.norb, s.n_alpha + s.n_beta)
    td = to_np(od)
    o_runs = [O.dedup(td[eo[r]:eo[r + 1]])[0] for r in range(P)]
    o_spl, o_cuts = O.regular_sampling_plan(o_runs, P, S)
    assert np.array_equal(to_np(spl), o_spl)
    assert np.array_equal(bounds.cpu().numpy(), o_cuts)
    got = np.concatenate([to_np(p) for p in parts])
    assert np.array_equal(got, O.dedup(td)[0])
    assert stats["max_over_min"] >= 1.0 and stats["cv"] >= 0.0


def test_virtual_ranks_with_empty_ranks():
    """Ranks that own no entries contribute no samples and receive only their
    share of the others' runs; the exchange and the final split still cover
    the global distinct set exactly."""
    s = synth.config_system("mid")
    sysd = cusci.System.of(s)
    n, P, S = 120, 6, 32
    off, od, oh, st = cusci.coupled(sysd, cusci.dets_to_device(s.dets[:n]), s.eps)
    o = off.cpu().numpy()
    src_cut = np.array([0, 0, 40, 40, 90, n, n], dtype=np.int64)   # ranks 0, 2 and 5 empty
    eo = o[src_cut]
    parts, stats, spl, bounds, runs, run_off = cusci.virtual_rank_dedup(
        od, eo, P, S, 2 * s.norb, s.n_alpha + s.n_beta)
    td = to_np(od)
    o_runs = [O.dedup(td[eo[r]:eo[r + 1]])[0] for r in range(P)]
    assert [x.shape[0] for x in o_runs] == stats["local_distinct"]
    assert np.array_equal(to_np(runs), np.concatenate(o_runs))
    o_spl, o_cuts = O.regular_sampling_plan(o_runs, P, S)
    assert np.array_equal(to_np(spl), o_spl)
    assert np.array_equal(bounds.cpu().numpy(), o_cuts)
    got = np.concatenate([to_np(p) for p in parts])
    assert np.array_equal(got, O.dedup(td)[0])
    # rank q's received rows are its cut shares of every run
    exp_recv = [int(sum(o_cuts[r, q + 1] - o_cuts[r, q] for r in range(P))) for q in range(P)]
    assert stats["received"] == exp_recv

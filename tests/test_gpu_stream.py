"""Mini-batched generation + de-duplication out of a bounded device pool, with
the coupled lists offloaded to pinned host memory: bit-exact against the oracle
for any batch size."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import assert_h_close, to_np

pytestmark = pytest.mark.gpu


def check(system, dets, eps, batch_entries):
    sysd = cusci.System.of(system)
    o_off, o_d, o_h = O.OracleSystem.of(system).gen(dets, eps)
    total = int(o_off[-1])
    off, hd, hh, uniq, stats = cusci.stream_gen_dedup(sysd, dets, eps, batch_entries,
                                                      unique_capacity=total,
                                                      host_capacity=total)
    torch.cuda.synchronize()
    assert np.array_equal(off, o_off)
    assert np.array_equal(hd.numpy().view(np.uint64), o_d)
    assert_h_close(hh.numpy(), o_h)
    ou, _ = O.dedup(o_d)
    assert np.array_equal(to_np(uniq), ou)
    assert stats["total"] == total
    return stats


def test_stream_two_word_system_many_batches():
    s = synth.config_system("large")
    stats = check(s, s.dets[:160], s.eps, batch_entries=120_000)
    assert stats["batches"] >= 10
    assert stats["pool_peak"] <= stats["pool_bytes"]


def test_stream_one_word_system():
    s = synth.config_system("mid")
    stats = check(s, s.dets[:150], s.eps, batch_entries=500_000)
    assert stats["batches"] >= 4


def test_stream_without_offload_keeps_distinct_set():
    s = synth.config_system("mid")
    sysd = cusci.System.of(s)
    o_off, o_d, o_h = O.OracleSystem.of(s).gen(s.dets[:60], s.eps)
    off, hd, hh, uniq, stats = cusci.stream_gen_dedup(sysd, s.dets[:60], s.eps, 400_000,
                                                      unique_capacity=int(o_off[-1]),
                                                      offload=False)
    assert hd is None and stats["d2h_bytes"] == 0
    assert np.array_equal(to_np(uniq), O.dedup(o_d)[0])


def test_stream_errors_are_reported():
    s = synth.config_system("mid")
    sysd = cusci.System.of(s)
    with pytest.raises(cusci.CusciError) as ei:      # one source longer than a batch
        cusci.stream_gen_dedup(sysd, s.dets[:4], s.eps, 1000, unique_capacity=100_000,
                               host_capacity=100_000)
    assert ei.value.status == 2
    with pytest.raises(cusci.CusciError) as ei:      # distinct set larger than declared
        cusci.stream_gen_dedup(sysd, s.dets[:20], s.eps, 400_000, unique_capacity=1000,
                               host_capacity=1_000_000)
    assert ei.value.status in (2, 4)


def test_hash_set_bounded_wait_times_out_and_reports():
    """The two-word hash insert waits for a claimed slot's second word; with a
    table whose every slot has its first word set and its second word never
    written, each wait must give up after the poll limit and report
    CUSCI_ERR_TIMEOUT (5) through the status word, and the kernel must return.
    With the second words present the same keys are found and nothing is
    reported."""
    keys = torch.tensor([[7, 11], [7, 12], [7, 13]], dtype=torch.int64, device="cuda")
    slots = 64
    table = torch.full((slots, 2), -1, dtype=torch.int64, device="cuda")
    table[:, 0] = 7                      # first word claimed, second word empty
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    n_new = cusci.hash_insert_probe(keys, table, spin_limit=1000, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 5
    assert int(n_new.item()) == 0
    # the same probe against a table that holds the keys: found, no error
    table2 = torch.full((slots, 2), -1, dtype=torch.int64, device="cuda")
    st2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    n1 = cusci.hash_insert_probe(keys, table2, spin_limit=1000, status=st2)
    n2 = cusci.hash_insert_probe(keys, table2, spin_limit=1000, status=st2)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0
    assert int(n1.item()) == 3 and int(n2.item()) == 0

"""Just-in-time reverse index (Stage 3): positions of coupled targets in the
distinct set, bit-exact against the oracle's inverse, also streamed from pinned
host memory after a mini-batched generation."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n", [("mid", 300), ("large", 20)])
def test_reverse_index_matches_oracle(name, n):
    s = synth.config_system(name)
    off, td, hv = O.OracleSystem.of(s).gen(s.dets[:n], s.eps)
    u, inv = O.dedup(td)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = cusci.reverse_index(to_dev(u), to_dev(td), 8, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(got.cpu().numpy(), inv)


def test_absent_keys_are_reported():
    u = np.array([[3], [9], [27]], dtype=np.uint64)
    q = np.array([[9], [4], [27], [1]], dtype=np.uint64)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = cusci.reverse_index(to_dev(u), to_dev(q), 4, status=st)
    assert got.cpu().tolist() == [1, -1, 2, -1]
    assert int(st.item()) == 1


def test_streamed_reverse_index_after_streaming_generation():
    s = synth.config_system("large")
    sysd = cusci.System.of(s)
    o_off, o_d, o_h = O.OracleSystem.of(s).gen(s.dets[:60], s.eps)
    total = int(o_off[-1])
    off, hd, hh, uniq, stats = cusci.stream_gen_dedup(sysd, s.dets[:60], s.eps, 200_000,
                                                      unique_capacity=total, host_capacity=total)
    inv = cusci.reverse_index_stream(uniq, hd, batch=150_000)
    ou, oinv = O.dedup(o_d)
    assert np.array_equal(inv.numpy().astype(np.int64), oinv)


@pytest.mark.parametrize("name,n", [("mid", 300), ("large", 20)])
def test_hashed_reverse_index_matches_oracle(name, n):
    """The hash-table form gives the same positions as the oracle's inverse."""
    s = synth.config_system(name)
    off, td, hv = O.OracleSystem.of(s).gen(s.dets[:n], s.eps)
    u, inv = O.dedup(td)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    du = to_dev(u)
    table = cusci.reverse_table(du, status=st)
    got = cusci.reverse_index_table(table, du.shape[0], du.shape[1], to_dev(td), 8, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(got.cpu().numpy(), inv)


def test_hashed_reverse_index_reports_absent_keys():
    """Keys not in the set (including ones that hash next to members and the
    all-ones word) come back as -1 with the status set; a table of one key
    works."""
    u = np.array([[3], [9], [27], [0xFFFFFFFFFFFFFFFF]], dtype=np.uint64)
    q = np.array([[9], [4], [27], [1], [0xFFFFFFFFFFFFFFFF], [0xFFFFFFFFFFFFFFFE]],
                 dtype=np.uint64)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    du = to_dev(u)
    table = cusci.reverse_table(du, status=st)
    got = cusci.reverse_index_table(table, 4, 1, to_dev(q), 4, status=st)
    assert got.cpu().tolist() == [1, -1, 2, -1, 3, -1]
    assert int(st.item()) == 1
    one = to_dev(np.array([[5, 7]], dtype=np.uint64))
    st2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    t1 = cusci.reverse_table(one, status=st2)
    got2 = cusci.reverse_index_table(t1, 1, 2, to_dev(np.array([[5, 7], [7, 5]], dtype=np.uint64)),
                                     4, status=st2)
    assert got2.cpu().tolist() == [0, -1]
    assert int(st2.item()) == 1


def test_streamed_reverse_index_search_form_matches_table_form():
    s = synth.config_system("mid")
    off, td, hv = O.OracleSystem.of(s).gen(s.dets[:120], s.eps)
    u, inv = O.dedup(td)
    host = torch.from_numpy(np.ascontiguousarray(td).view(np.int64)).pin_memory()
    du = to_dev(u)
    a = cusci.reverse_index_stream(du, host, batch=100_000, table=cusci.reverse_table(du))
    b = cusci.reverse_index_stream(du, host, batch=100_000, table=False)
    c = cusci.reverse_index_stream(du, host, batch=100_000, table=True)
    assert np.array_equal(a.numpy(), c.numpy())
    assert np.array_equal(a.numpy(), b.numpy())
    assert np.array_equal(a.numpy().astype(np.int64), inv)

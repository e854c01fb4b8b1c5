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

"""Streaming two-level top-K (local per batch, merged into the running set):
the exact K best (larger score, equal scores by smaller id) of everything
streamed, against a plain sort."""
import numpy as np
import pytest
import torch

from paper_2604_15768_gb300 import cusci

pytestmark = pytest.mark.gpu


def reference(scores, ids, K):
    order = np.lexsort((ids, -scores))[:K]
    return scores[order], ids[order]


@pytest.mark.parametrize("K,batch,n", [(1000, 50_000, 400_000), (37, 1000, 10_000),
                                       (5000, 3000, 20_000)])
def test_topk_stream_matches_sort(K, batch, n):
    rng = np.random.default_rng(K)
    scores = np.abs(rng.standard_normal(n))
    scores[rng.choice(n, n // 10, replace=False)] = 0.5        # many exact ties
    scores[:7] = 0.0
    ids = rng.permutation(10 * n)[:n].astype(np.int64)
    tk = cusci.TopK(K, batch)
    for a in range(0, n, batch):
        tk.update(torch.from_numpy(scores[a:a + batch]).cuda(),
                  torch.from_numpy(ids[a:a + batch]).cuda())
    got_s, got_i = tk.result()
    ref_s, ref_i = reference(scores, ids, K)
    assert np.array_equal(got_i, ref_i)
    assert np.array_equal(got_s, ref_s)


def test_topk_fewer_items_than_k():
    tk = cusci.TopK(100, 64)
    sc = np.array([0.3, 0.1, 0.9], dtype=np.float64)
    ids = np.array([5, 2, 7], dtype=np.int64)
    tk.update(torch.from_numpy(sc).cuda(), torch.from_numpy(ids).cuda())
    s, i = tk.result()
    assert i.tolist() == [7, 5, 2] and s.tolist() == [0.9, 0.3, 0.1]


def test_topk_negative_zero_ranks_as_zero():
    """-0.0 has its sign bit set; it must still rank below every positive score
    and tie with +0.0 (then by id)."""
    tk = cusci.TopK(3, 16)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sc = np.array([-0.0, 0.25, 0.0, 1e-300, -0.0], dtype=np.float64)
    ids = np.array([4, 9, 1, 6, 0], dtype=np.int64)
    tk.update(torch.from_numpy(sc).cuda(), torch.from_numpy(ids).cuda(), status=st)
    s, i = tk.result()
    assert i.tolist() == [9, 6, 0]
    assert int(st.item()) == 0


def test_topk_negative_or_nan_score_is_reported():
    for bad in (-0.5, float("nan")):
        tk = cusci.TopK(2, 16)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        sc = np.array([0.3, bad, 0.1], dtype=np.float64)
        tk.update(torch.from_numpy(sc).cuda(), torch.tensor([1, 2, 3], device="cuda"), status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 1

"""The batched workload at the size the benchmark runs (1k-50k sources per
system), on the largest one-word system, the largest two-word system and two
small ones in one Batch: one persistent count/fill and one batched
de-duplication.  The oracle regenerates 200 sampled sources of every system
(rows compared element by element: targets bit-exact, H to 1e-12); the
de-duplication is checked at full size by the properties that fix it (distinct
targets strictly ascending, every entry's target found at its id, every id
used), and against the oracle's sorted set for the small systems."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import assert_h_close, to_np

pytestmark = pytest.mark.gpu


def pick():
    systems = synth.batched_systems(64, scale=1.0)
    est = []
    for k, s in enumerate(systems):
        c = O.OracleSystem.of(s).count(s.dets[:20], s.eps).mean()
        est.append(c * s.dets.shape[0])
    one = [k for k, s in enumerate(systems) if s.W == 1]
    two = [k for k, s in enumerate(systems) if s.W == 2]
    big1 = max(one, key=lambda k: est[k])
    big2 = max(two, key=lambda k: est[k])
    small = sorted(range(len(systems)), key=lambda k: est[k])[:2]
    return [systems[k] for k in (big1, big2, *small)]


def test_batched_workload_full_size():
    systems = pick()
    b = cusci.Batch(systems, [s.dets for s in systems], 1e-8, chunk=8)
    b.plan()
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    offs = b.offsets.cpu().numpy()
    rng = np.random.default_rng(5)
    for k, s in enumerate(systems):
        a, z = int(b.entry_begin[k]), int(b.entry_begin[k + 1])
        s0 = int(b.src_begin[k])
        W = s.W
        # sampled rows against the oracle
        rows = np.sort(rng.choice(s.dets.shape[0], min(200, s.dets.shape[0]), replace=False))
        o_off, o_d, o_h = O.OracleSystem.of(s).gen(s.dets[rows], s.eps)
        for r_i, r in enumerate(rows):
            ga, gz = int(offs[s0 + r]), int(offs[s0 + r + 1])
            assert gz - ga == o_off[r_i + 1] - o_off[r_i]
            got = to_np(b.out_d[ga:gz])
            assert np.array_equal(got[:, :W], o_d[o_off[r_i]:o_off[r_i + 1]])
            assert_h_close(b.out_h[ga:gz].cpu().numpy(), o_h[o_off[r_i]:o_off[r_i + 1]])
        # the de-duplication at full size
        nu = int(b.n_unique[k].item())
        u = b.unique[a:a + nu]
        inv = b.inverse[a:z].long()
        hi, lo = (u[:, 1], u[:, 0]) if W == 2 else (torch.zeros_like(u[:, 0]), u[:, 0])
        # strictly ascending as unsigned two-word numbers (compare hi, then lo;
        # flipping the sign bit makes signed comparison unsigned)
        hi_u = hi ^ torch.tensor(-(1 << 63), device=hi.device)
        lo_u = lo ^ torch.tensor(-(1 << 63), device=lo.device)
        gt = (hi_u[1:] > hi_u[:-1]) | ((hi_u[1:] == hi_u[:-1]) & (lo_u[1:] > lo_u[:-1]))
        assert bool(gt.all())
        assert int(inv.min()) >= 0 and int(inv.max()) < nu
        assert torch.equal(u[inv][:, :W], b.out_d[a:z, :W])
        used = torch.zeros(nu, dtype=torch.bool, device=u.device)
        used[inv] = True
        assert bool(used.all())
        if z - a < 20_000_000:
            o_all_off, o_all_d, _ = O.OracleSystem.of(s).gen(s.dets, s.eps)
            ou, oinv = O.dedup(o_all_d)
            assert nu == ou.shape[0]
            assert np.array_equal(to_np(u)[:, :W], ou)
            assert np.array_equal(inv.cpu().numpy(), oinv)
    b.close()

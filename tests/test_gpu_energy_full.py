"""Parity of the energy workload exactly as the benchmark runs it: the mid
system (52 spin orbitals, 7a+7b, eps 1e-8), the full 200k selected set of
sorted distinct sampled determinants, psi = exp of the seeded 256-256 tanh
MLP.  The oracle recomputes (H psi)_i for 320 rows (the first and last 32 and
256 drawn at random) through its row-subset form; the GPU's H psi and
gradient must match there to 1e-10, and E must equal psi.(H psi)/psi.psi
summed on the host from the GPU's own H psi (a property at any size)."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth

pytestmark = pytest.mark.gpu


def test_energy_workload_full_size_sampled_rows():
    s = synth.config_system("energy")
    assert s.dets.shape[0] == 200_000
    sysd = cusci.System.of(s)
    dS = cusci.dets_to_device(s.dets)
    net, x = synth.amplitude_mlp(s.dets, s.norb, "cuda")
    with torch.no_grad():
        psi = torch.exp(net(x).squeeze(-1).double())
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    E, n2, hp = cusci.energy_fwd(sysd, dS, psi, s.eps, status=st)
    grad = cusci.energy_bwd(sysd, dS, psi, s.eps, E, n2, hpsi=hp)
    grad_re = cusci.energy_bwd(sysd, dS, psi, s.eps, E, n2, hpsi=None)   # recompute path
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    psi_h, hp_h, g_h = psi.cpu().numpy(), hp.cpu().numpy(), grad.cpu().numpy()
    assert np.array_equal(g_h, grad_re.cpu().numpy())
    E_g, n2_g = float(E.item()), float(n2.item())
    # reductions: E and psi.psi against exactly rounded host sums
    n2_h = math.fsum(psi_h * psi_h)
    assert abs(n2_g - n2_h) <= 1e-13 * n2_h
    E_h = math.fsum(psi_h * hp_h) / n2_h
    assert abs(E_g - E_h) <= 1e-10
    # sampled rows against the oracle
    n = s.dets.shape[0]
    rng = np.random.default_rng(2024)
    rows = np.unique(np.concatenate([np.arange(32), np.arange(n - 32, n),
                                     rng.choice(n, 256, replace=False)])).astype(np.int64)
    ref = O.OracleSystem.of(s).hpsi_rows(s.dets, psi_h, s.eps, rows)
    assert np.abs(hp_h[rows] - ref).max() <= 1e-10
    g_ref = 2.0 * (ref - E_g * psi_h[rows]) / n2_g
    assert np.abs(g_h[rows] - g_ref).max() <= 1e-10

"""GPU parity of the variational energy and its adjoint with the CPU oracle,
plus the autograd path (finite differences through an MLP)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def sorted_S(dets):
    return dets[np.lexsort([dets[:, w] for w in range(dets.shape[1])])]


def test_energy_matches_oracle_mid():
    s = synth.config_system("mid", n_dets=3000)
    S = sorted_S(s.dets)
    psi = np.random.default_rng(1).standard_normal(S.shape[0])
    E, n2, hp, grad = O.OracleSystem.of(s).energy(S, psi, s.eps)
    sysd = cusci.System.of(s)
    dS, dpsi = to_dev(S), torch.from_numpy(psi).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gE, gn2, ghp = cusci.energy_fwd(sysd, dS, dpsi, s.eps, status=st)
    gg = cusci.energy_bwd(sysd, dS, dpsi, s.eps, gE, gn2, hpsi=ghp)
    gg2 = cusci.energy_bwd(sysd, dS, dpsi, s.eps, gE, gn2, hpsi=None)   # recompute path
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert abs(gE.item() - E) <= 1e-10
    assert abs(gn2.item() - n2) <= 1e-12 * n2
    assert np.abs(ghp.cpu().numpy() - hp).max() <= 1e-10
    assert np.abs(gg.cpu().numpy() - grad).max() <= 1e-10
    assert np.array_equal(gg.cpu().numpy(), gg2.cpu().numpy())


def test_energy_two_words():
    s = synth.config_system("large", n_dets=150)
    S = sorted_S(s.dets)
    psi = np.random.default_rng(2).standard_normal(S.shape[0])
    E, n2, hp, grad = O.OracleSystem.of(s).energy(S, psi, s.eps)
    sysd = cusci.System.of(s)
    gE, gn2, ghp = cusci.energy_fwd(sysd, to_dev(S), torch.from_numpy(psi).cuda(), s.eps)
    assert abs(gE.item() - E) <= 1e-10
    assert np.abs(ghp.cpu().numpy() - hp).max() <= 1e-10


def test_energy_at_eigenvector_tiny():
    s = synth.config_system("tiny")
    sysd = cusci.System.of(s)
    off, td, hv = O.OracleSystem.of(s).gen(s.dets, -1.0)
    idx = np.searchsorted(s.dets[:, 0], td[:, 0])
    rows = np.repeat(np.arange(s.dets.shape[0]), np.diff(off))
    H = np.zeros((s.dets.shape[0],) * 2)
    H[idx, rows] = hv
    w, V = np.linalg.eigh(H)
    psi = torch.from_numpy(V[:, 0].copy()).cuda()
    gE, gn2, ghp = cusci.energy_fwd(sysd, to_dev(s.dets), psi, -1.0)
    gg = cusci.energy_bwd(sysd, to_dev(s.dets), psi, -1.0, gE, gn2, hpsi=ghp)
    assert abs(gE.item() - w[0]) <= 1e-10
    assert gg.abs().max().item() <= 1e-10


def test_unsorted_S_is_reported():
    s = synth.config_system("mid", n_dets=50)
    sysd = cusci.System.of(s)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cusci.energy_fwd(sysd, to_dev(s.dets), torch.ones(50, dtype=torch.float64, device="cuda"),
                     s.eps, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 1


def test_autograd_through_mlp_finite_differences():
    s = synth.config_system("mid", n_dets=600)
    S = sorted_S(s.dets)
    sysd = cusci.System.of(s)
    dS = to_dev(S)
    bits = torch.from_numpy(((S[:, :1] >> np.arange(2 * s.norb, dtype=np.uint64)) & 1)
                            .astype(np.float64)).cuda()
    torch.manual_seed(0)
    net = torch.nn.Sequential(torch.nn.Linear(2 * s.norb, 32), torch.nn.Tanh(),
                              torch.nn.Linear(32, 1)).double().cuda()

    def energy(recompute=False):
        psi = torch.exp(net(bits).squeeze(-1) * 0.1)
        return cusci.Energy.apply(psi, sysd, dS, s.eps, recompute)

    E = energy()
    E.backward()
    grads = [p.grad.detach().clone() for p in net.parameters()]
    net.zero_grad()
    energy(recompute=True).backward()
    for g, p in zip(grads, net.parameters()):
        assert torch.allclose(g, p.grad, rtol=0, atol=1e-13)
    h = 1e-6
    rng = np.random.default_rng(3)
    params = list(net.parameters())
    with torch.no_grad():
        for _ in range(10):
            pi = int(rng.integers(len(params)))
            flat = params[pi].view(-1)
            k = int(rng.integers(flat.numel()))
            old = flat[k].item()
            flat[k] = old + h
            ep = energy().item()
            flat[k] = old - h
            em = energy().item()
            flat[k] = old
            fd = (ep - em) / (2 * h)
            an = grads[pi].view(-1)[k].item()
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))

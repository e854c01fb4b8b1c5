"""The differentiated energy of the energy workload's recipe: the mid system, a
selected set of distinct sampled determinants, psi = exp(log-amplitude) from a
seeded 2*norb -> 256 -> 256 -> 1 tanh MLP.  The analytic gradient through
cusci.Energy (hand-written adjoint) is checked against central finite
differences at h = 1e-6 on 50 random parameters of an FP64 clone of the MLP
(FP32 weights cannot resolve h = 1e-6), and dE/dpsi against the oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth

pytestmark = pytest.mark.gpu


def test_energy_mlp_finite_differences_50_params():
    s = synth.config_system("energy", n_dets=4000)
    sysd = cusci.System.of(s)
    dS = cusci.dets_to_device(s.dets)
    bits = torch.from_numpy(((s.dets[:, :1] >> np.arange(2 * s.norb, dtype=np.uint64)) & 1)
                            .astype(np.float64)).cuda()
    torch.manual_seed(0)
    net = torch.nn.Sequential(torch.nn.Linear(2 * s.norb, 256), torch.nn.Tanh(),
                              torch.nn.Linear(256, 256), torch.nn.Tanh(),
                              torch.nn.Linear(256, 1)).cuda().double()

    def energy():
        psi = torch.exp(net(bits).squeeze(-1))
        return cusci.Energy.apply(psi, sysd, dS, s.eps, False)

    E = energy()
    E.backward()
    params = list(net.parameters())
    grads = [p.grad.detach().clone() for p in params]
    rng = np.random.default_rng(11)
    h = 1e-6
    with torch.no_grad():
        for _ in range(50):
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
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (pi, k, fd, an)
    # dE/dpsi against the oracle at the same psi
    psi = torch.exp(net(bits).squeeze(-1)).detach()
    gE, gn2, ghp = cusci.energy_fwd(sysd, dS, psi, s.eps)
    gg = cusci.energy_bwd(sysd, dS, psi, s.eps, gE, gn2, hpsi=ghp)
    oE, on2, ohp, ograd = O.OracleSystem.of(s).energy(s.dets, psi.cpu().numpy(), s.eps)
    assert abs(gE.item() - oE) <= 1e-10
    assert np.abs(gg.cpu().numpy() - ograd).max() <= 1e-10

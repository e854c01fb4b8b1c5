"""The local-energy form of Eq. 5 on the GPU (CSR coupled lists + reverse index
into the distinct set) against the CPU oracle, and its adjoint."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def pipeline(s, n, index_bytes=4):
    sysd = cusci.System.of(s)
    off, od, oh, st = cusci.coupled(sysd, to_dev(s.dets[:n]), s.eps)
    u, inv, nu = cusci.dedup(od, 2 * s.norb, s.n_alpha + s.n_beta, index_bytes=index_bytes)
    return off, oh, inv, nu


@pytest.mark.parametrize("index_bytes", [4, 8])
def test_local_energy_matches_oracle(index_bytes):
    s = synth.config_system("mid")
    off, oh, inv, nu = pipeline(s, 300, index_bytes)
    rng = np.random.default_rng(2)
    psi = rng.standard_normal(nu) * 0.1 + 1.0
    dpsi = torch.from_numpy(psi).cuda()
    E, n2, y = cusci.local_energy_fwd(off, oh, inv, dpsi)
    grad = cusci.local_energy_bwd(off, oh, inv, dpsi, E, n2, y=y)
    grad2 = cusci.local_energy_bwd(off, oh, inv, dpsi, E, n2, y=None)
    torch.cuda.synchronize()
    oE, on2, oy, og = O.local_energy(off.cpu().numpy(), oh.cpu().numpy(),
                                     inv.cpu().numpy().astype(np.int64), psi)
    assert abs(E.item() - oE) <= 1e-10
    assert abs(n2.item() - on2) <= 1e-12 * on2
    assert np.abs(y.cpu().numpy() - oy).max() <= 1e-10
    assert np.abs(grad.cpu().numpy() - og).max() <= 1e-10
    assert np.abs(grad2.cpu().numpy() - og).max() <= 1e-10
    # the fixed-point scatter makes the adjoint bit-reproducible
    grad3 = cusci.local_energy_bwd(off, oh, inv, dpsi, E, n2, y=y)
    assert np.array_equal(grad.cpu().numpy(), grad2.cpu().numpy())
    assert np.array_equal(grad.cpu().numpy(), grad3.cpu().numpy())


def test_local_energy_autograd_finite_differences():
    s = synth.config_system("mid")
    off, oh, inv, nu = pipeline(s, 40)
    rng = np.random.default_rng(3)
    psi = torch.from_numpy(rng.standard_normal(nu) * 0.1 + 1.0).cuda().requires_grad_(True)
    E = cusci.LocalEnergy.apply(psi, off, oh, inv)
    E.backward()
    g = psi.grad.detach().cpu().numpy()
    h = 1e-6
    src = inv[off[:-1].long()].cpu().numpy()
    with torch.no_grad():
        for k in list(src[:4]) + list(rng.choice(nu, 6, replace=False)):
            p = psi.detach().clone()
            p[k] += h
            ep = cusci.LocalEnergy.apply(p, off, oh, inv).item()
            p[k] -= 2 * h
            em = cusci.LocalEnergy.apply(p, off, oh, inv).item()
            fd = (ep - em) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k]))


def test_local_energy_equals_variational_on_closed_space():
    s = synth.config_system("tiny")
    off, oh, inv, nu = pipeline(s, 4900)
    assert nu == 4900
    rng = np.random.default_rng(5)
    psi = torch.from_numpy(rng.standard_normal(nu)).cuda()
    E, n2, y = cusci.local_energy_fwd(off, oh, inv, psi)
    sysd = cusci.System.of(s)
    Ev, n2v, hp = cusci.energy_fwd(sysd, to_dev(s.dets), psi, s.eps)
    assert abs(E.item() - Ev.item()) <= 1e-10


@pytest.mark.parametrize("name,n,scale", [("large", 20, 1.0), ("mid", 200, 50.0)])
def test_local_energy_two_words_and_large_mixed_sign_amplitudes(name, n, scale):
    """Two-word configurations, and amplitudes of both signs and large size, so
    that the fixed-point adjoint accumulates terms with integer parts well
    away from 0 and -1 (carries into and borrows from the high word)."""
    s = synth.config_system(name)
    off, oh, inv, nu = pipeline(s, n)
    rng = np.random.default_rng(9)
    psi = rng.standard_normal(nu) * scale + (1.0 if scale == 1.0 else 0.0)
    dpsi = torch.from_numpy(psi).cuda()
    E, n2, y = cusci.local_energy_fwd(off, oh, inv, dpsi)
    grad = cusci.local_energy_bwd(off, oh, inv, dpsi, E, n2, y=y)
    grad2 = cusci.local_energy_bwd(off, oh, inv, dpsi, E, n2, y=y)
    torch.cuda.synchronize()
    oE, on2, oy, og = O.local_energy(off.cpu().numpy(), oh.cpu().numpy(),
                                     inv.cpu().numpy().astype(np.int64), psi)
    assert abs(E.item() - oE) <= 1e-10 * max(1.0, abs(oE))
    assert np.abs(y.cpu().numpy() - oy).max() <= 1e-10 * max(1.0, np.abs(oy).max())
    g = grad.cpu().numpy()
    assert np.abs(g - og).max() <= 1e-10 * max(1.0, np.abs(og).max())
    assert np.array_equal(g, grad2.cpu().numpy())

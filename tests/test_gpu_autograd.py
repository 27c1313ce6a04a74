"""GPU checks of the differentiable local energy E_loc(psi, V) = sum occ (Ekin + Epot)
run through paper_0904_1543_gb300.ELoc (forward: energies only; backward:
the adjoint chain recomputed from psi, dE/dpsi = 2 occ H psi, dE/dV = rho).

E is quadratic in psi and linear in V, so FP64 central differences are exact
up to rounding (about 1e-16 |E| / h ~ 1e-9 relative at h = 1e-5): the bound
1e-6 leaves a wide margin.  Gradients against the oracle's adjoint: 1e-11.
"""
import numpy as np
import pytest

import oracle.wavelet as O
from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    return W


def _setup(n=(16, 16, 16), norb=4, cfg=4):
    psi = inputs.orbitals(cfg, norb, n)
    V = inputs.gaussian_potential(cfg, 0, n)
    occ = np.array([2.0, 2.0, 1.0, 0.5])[:norb]
    return psi, V, occ


def test_eloc_gradients_match_oracle_adjoint(W):
    import torch
    n = (16, 16, 16)
    g = W.Grid(n)
    psi, V, occ = _setup(n)
    tp = torch.from_numpy(psi).cuda().requires_grad_(True)
    tV = torch.from_numpy(V).cuda().requires_grad_(True)
    E = W.ELoc.apply(tp, tV, torch.from_numpy(occ).cuda(), g)
    E.backward()
    gpsi_r, gV_r = O.energy_gradients(psi, V, occ, n)
    E_r = O.energy(psi, V, occ, n)
    assert abs(float(E.detach()) - E_r) < 1e-12 * abs(E_r)
    d = np.abs(tp.grad.cpu().numpy() - gpsi_r).max() / np.abs(gpsi_r).max()
    assert d < 1e-11, d
    d = np.abs(tV.grad.cpu().numpy() - gV_r).max() / np.abs(gV_r).max()
    assert d < 1e-11, d


def test_eloc_finite_differences(W):
    """16 random directions of psi and V, 64 single coordinates of psi and
    of V, h = 1e-5, FP64 forward on the GPU."""
    import torch
    n = (16, 16, 16)
    g = W.Grid(n)
    psi, V, occ = _setup(n)
    tp = torch.from_numpy(psi).cuda().requires_grad_(True)
    tV = torch.from_numpy(V).cuda().requires_grad_(True)
    to = torch.from_numpy(occ).cuda()
    E = W.ELoc.apply(tp, tV, to, g)
    E.backward()
    gp, gv = tp.grad.detach(), tV.grad.detach()
    h = 1e-5

    def energy(p, v):
        with torch.no_grad():
            return float(W.ELoc.apply(p, v, to, g))

    rng = np.random.default_rng(4)
    E0 = abs(energy(tp, tV))
    # central differences of a quadratic are exact; what remains is the
    # rounding of the two energies, at most a few ulps of |E| over 2h
    floor = 8 * np.finfo(np.float64).eps * E0 / (2 * h)
    worst = 0.0
    for k in range(16):
        dp = torch.from_numpy(rng.standard_normal(psi.shape)).cuda()
        dv = torch.from_numpy(rng.standard_normal(V.shape)).cuda()
        fd = (energy(tp + h * dp, tV + h * dv) - energy(tp - h * dp, tV - h * dv)) / (2 * h)
        an = float((gp * dp).sum() + (gv * dv).sum())
        assert abs(fd - an) <= 1e-6 * abs(an) + floor, (k, fd, an)
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst < 1e-6, worst
    for k in range(64):
        i = int(rng.integers(psi.size))
        j = int(rng.integers(V.size))
        dp = torch.zeros_like(tp).view(-1)
        dp[i] = 1.0
        dp = dp.view_as(tp)
        dv = torch.zeros_like(tV).view(-1)
        dv[j] = 1.0
        dv = dv.view_as(tV)
        an_p, an_v = float(gp.view(-1)[i]), float(gv.view(-1)[j])
        # h = 1e-5: exact up to the rounding floor
        fd = (energy(tp + h * dp, tV) - energy(tp - h * dp, tV)) / (2 * h)
        assert abs(fd - an_p) <= 1e-6 * abs(an_p) + floor, ("psi", i, fd, an_p)
        fd = (energy(tp, tV + h * dv) - energy(tp, tV - h * dv)) / (2 * h)
        assert abs(fd - an_v) <= 1e-6 * abs(an_v) + floor, ("V", j, fd, an_v)
        # a larger step is just as exact (E is quadratic in psi, linear in V)
        # and brings the rounding floor far below 1e-6 relative
        H = 0.05
        fd = (energy(tp + H * dp, tV) - energy(tp - H * dp, tV)) / (2 * H)
        assert abs(fd - an_p) <= 1e-6 * abs(an_p) + floor * h / H, ("psi big", i)
        fd = (energy(tp, tV + 1.0 * dv) - energy(tp, tV - 1.0 * dv)) / 2.0
        assert abs(fd - an_v) <= 1e-6 * abs(an_v) + floor * h, ("V big", j)


def test_eloc_fp32_against_oracle(W):
    """FP32 convolutions, FP64/compensated reductions: errors stay at
    single-precision level, with the FP32 parity bounds of the H psi chain
    (normwise 2e-6 for dE/dpsi, 5e-6 for dE/dV = rho, 5e-7 for E)."""
    import torch
    n = (10, 12, 8)
    g = W.Grid(n)
    psi, V, occ = _setup(n, cfg=5)
    p32, V32 = psi.astype(np.float32), V.astype(np.float32)
    tp = torch.from_numpy(p32).cuda().requires_grad_(True)
    tV = torch.from_numpy(V32).cuda().requires_grad_(True)
    E = W.ELoc.apply(tp, tV, torch.from_numpy(occ).cuda(), g)
    E.backward()
    gpsi_r, gV_r = O.energy_gradients(p32.astype(np.float64), V32.astype(np.float64), occ, n)
    E_r = O.energy(p32.astype(np.float64), V32.astype(np.float64), occ, n)
    assert abs(float(E.detach()) - E_r) < 5e-7 * abs(E_r)
    d = np.abs(tp.grad.double().cpu().numpy() - gpsi_r).max() / np.abs(gpsi_r).max()
    assert d < 2e-6, d
    d = np.abs(tV.grad.double().cpu().numpy() - gV_r).max() / np.abs(gV_r).max()
    assert d < 5e-6, d


@pytest.mark.parametrize("emu", [False, True])
def test_eloc_entry_points(W, emu):
    """wvl_eloc writes E_loc = sum occ (Ekin + Epot) on the device, and
    wvl_eloc_backward writes dE/dpsi = 2 occ g H psi (the last pass of the
    chain scales H psi) and dE/dV = g rho, for an upstream gradient g != 1;
    FP64 and its tensor-core form, against the oracle at the FP64 bounds."""
    import torch
    n = (12, 10, 8)
    g = W.Grid(n)
    psi, V, occ = _setup(n, cfg=6)
    tp, tV, to = (torch.from_numpy(x).cuda() for x in (psi, V, occ))
    rho = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
    E, ek, ep = W.eloc(tp, tV, to, g, rho=rho, emu=emu)
    E_r = O.energy(psi, V, occ, n)
    assert abs(float(E) - E_r) < 1e-12 * abs(E_r)
    hp_r, rho_r, ek_r, ep_r = O.hpsi_batch(psi, V, occ, n)
    assert np.abs(rho.cpu().numpy() - rho_r).max() < 1e-12 * np.abs(rho_r).max()
    assert np.abs(ek.cpu().numpy() - ek_r).max() < 1e-12 * np.abs(ek_r).max()
    # backward with an upstream gradient of -0.75
    tp2 = tp.clone().requires_grad_(True)
    tV2 = tV.clone().requires_grad_(True)
    E2 = W.ELoc.apply(tp2, tV2, to, g, emu)
    (-0.75 * E2).backward()
    gpsi_r, gV_r = O.energy_gradients(psi, V, occ, n)
    d = np.abs(tp2.grad.cpu().numpy() + 0.75 * gpsi_r).max() / np.abs(0.75 * gpsi_r).max()
    assert d < 1e-11, d
    d = np.abs(tV2.grad.cpu().numpy() + 0.75 * gV_r).max() / np.abs(0.75 * gV_r).max()
    assert d < 1e-11, d


def test_eloc_fp32_full_size_sampled(W):
    """The autograd workload at full size: 512 FP32 orbitals on a coarse 64^3
    cell (fine 128^3), forward and backward through ELoc as the benchmark
    runs it.  Two sampled orbitals' dE/dpsi = 2 occ H psi against the oracle
    (FP64 on the FP32-rounded inputs) at the FP32 bound; dE/dV = rho against
    the library's density entry point; and sum_I V rho = sum_o occ Epot with
    the per-orbital energies, a property that holds at any size."""
    import torch
    n = (64, 64, 64)
    g = W.Grid(n)
    norb = 512
    dev = torch.device("cuda")
    p = inputs.orbitals_device(4, norb, n, dev, torch.float32).requires_grad_(True)
    V = torch.from_numpy(inputs.gaussian_potential(4, 0, n)).to(dev).float().requires_grad_(True)
    occ = torch.full((norb,), 2.0, dtype=torch.float64, device=dev)
    E = W.ELoc.apply(p, V, occ, g)
    E.backward()
    Vh = V.detach().double().cpu().numpy()
    for o in (3, 511):
        r = O.hpsi_local(p[o].detach().double().cpu().numpy(), Vh, 2.0, n)
        ref = 2.0 * 2.0 * r["hpsi_c"]
        d = np.abs(p.grad[o].double().cpu().numpy() - ref).max() / np.abs(ref).max()
        assert d < 2e-6, (o, d)
    with torch.no_grad():
        rho = W.density(p.detach(), occ, g)
        ek, ep = W.energy(p.detach(), V.detach(), occ, g)
    assert float((V.grad.double() - rho).abs().max() / rho.abs().max()) < 5e-6
    lhs = float((V.detach().double() * rho).sum())
    rhs = float((occ * ep).sum())
    assert abs(lhs - rhs) < 5e-6 * abs(rhs)
    assert abs(float(E.detach()) - float((occ * (ek + ep)).sum())) < 5e-7 * abs(float(E.detach()))
    del p, V, E, rho
    torch.cuda.empty_cache()

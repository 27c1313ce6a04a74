"""GPU parity of the localisation-region forms (compressed vectors holding
only the coarse- and fine-region coefficients) against the oracle.
FP64 bound 1e-12 as in the other parity tests."""
import numpy as np
import pytest

import oracle.region as RG
import oracle.wavelet as O
from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu
RTOL64 = 1e-12


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    return W


def _rel(a, b):
    """max(normwise, elementwise on |b| >= 1e-3 max|b|) relative error."""
    sc = max(np.abs(b).max(), 1e-300)
    d = np.abs(a - b)
    big = np.abs(b) >= 1e-3 * sc
    el = (d[big] / np.abs(b[big])).max() if big.any() else 0.0
    return float(max(d.max() / sc, el))


@pytest.mark.parametrize("n,centre,rc,rf", [((8, 8, 8), (3, 4, 2), 3.1, 1.7),
                                            ((12, 10, 14), (0, 9, 13), 4.5, 2.5),
                                            ((5, 6, 7), (2, 2, 2), 9.0, 9.0)])
def test_hpsi_region(W, n, centre, rc, rf):
    import torch
    g = W.Grid(n)
    cm, fm = RG.sphere_masks(n, centre, rc, rf)
    reg = W.Region(g, cm, fm)
    norb = 3
    psi = inputs.random_field(91, 1, (norb, reg.clen))
    V = inputs.gaussian_potential(91, 0, n)
    occ = np.array([2.0, 1.0, 0.5])
    rho = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local_region(torch.from_numpy(psi).cuda(), torch.from_numpy(V).cuda(),
                                     torch.from_numpy(occ).cuda(), g, reg, rho=rho)
    rho_ref = np.zeros(g.fine)
    for o in range(norb):
        r = RG.hpsi_local(psi[o], V, occ[o], n, cm, fm)
        assert _rel(hp[o].cpu().numpy(), r["hpsi_c"]) < RTOL64
        assert abs(float(ek[o]) - r["ekin"]) < RTOL64 * abs(r["ekin"])
        assert abs(float(ep[o]) - r["epot"]) < RTOL64 * abs(r["epot"])
        rho_ref += r["rho"]
    assert _rel(rho.cpu().numpy(), rho_ref) < RTOL64
    rho2 = W.density_region(torch.from_numpy(psi).cuda(), torch.from_numpy(occ).cuda(), g, reg)
    assert _rel(rho2.cpu().numpy(), rho_ref) < RTOL64


def test_synthesis_analysis_region(W):
    import torch
    n = (9, 7, 6)
    g = W.Grid(n)
    cm, fm = RG.sphere_masks(n, (4, 3, 1), 3.3, 2.0)
    reg = W.Region(g, cm, fm)
    c = inputs.random_field(92, 1, (2, reg.clen))
    s = W.synthesis_region(torch.from_numpy(c).cuda(), g, reg)
    for o in range(2):
        ref = O.synthesis3d(RG.uncompress(c[o], n, cm, fm))
        assert _rel(s[o].cpu().numpy(), ref) < RTOL64
    z = inputs.random_field(92, 2, (2,) + g.fine)
    a = W.analysis_region(torch.from_numpy(z).cuda(), g, reg)
    for o in range(2):
        ref = RG.compress(O.analysis3d(z[o]), n, cm, fm)
        assert _rel(a[o].cpu().numpy(), ref) < RTOL64


def test_full_region_matches_full_grid(W):
    import torch
    n = (6, 6, 6)
    g = W.Grid(n)
    full = np.ones((6, 6, 6), dtype=bool)
    reg = W.Region(g, full, full)
    psi = inputs.orbitals(93, 2, n)
    # the region layout of a full region differs from the full-grid layout
    # only in the order of the fine block, which is identical by construction
    V = torch.from_numpy(inputs.gaussian_potential(93, 0, n)).cuda()
    occ = torch.full((2,), 2.0, dtype=torch.float64, device="cuda")
    a = W.hpsi_local_region(torch.from_numpy(psi).cuda(), V, occ, g, reg)
    b = W.hpsi_local(torch.from_numpy(psi).cuda(), V, occ, g)
    for x, y in zip(a, b):
        assert torch.equal(x, y)

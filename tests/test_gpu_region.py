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


@pytest.mark.parametrize("dt", ["float64", "float32"])
def test_hpsi_region_on_its_box(W, dt):
    """A small region in a larger periodic cell, wrapping around two faces:
    along x and z its periodic bounding box leaves at least 15 coarse points
    to the cell, so the chain runs on that box (free lines) there and on
    whole periodic lines along y.  H psi, energies and the density against
    the oracle (periodic operator on the whole cell, restricted to the
    region), and against the same call without the box."""
    import torch
    n = (24, 20, 26)
    g = W.Grid(n, (0.25, 0.3, 0.2))
    cm, fm = RG.sphere_masks(n, (1, 10, 24), 3.6, 2.2)
    reg = W.Region(g, cm, fm)
    assert reg.len[0] <= n[0] - 15 and reg.len[2] <= n[2] - 15 and reg.len[1] > n[1] - 15
    assert reg.lo[0] > reg.len[0] and reg.lo[2] > reg.len[2]   # the boxes wrap
    full = W.Region(g, cm, fm, bounds=False)
    norb = 5
    psi = inputs.random_field(92, 1, (norb, reg.clen)).astype(dt)
    V = inputs.gaussian_potential(92, 0, n).astype(dt)
    occ = np.array([2.0, 1.0, 0.5, 2.0, 1.5])
    tol, tol_rho, tol_e = (RTOL64, RTOL64, RTOL64) if dt == "float64" else (2e-6, 5e-6, 5e-7)
    out = {}
    for name, rg in (("box", reg), ("cell", full)):
        rho = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
        hp, ek, ep = W.hpsi_local_region(torch.from_numpy(psi).cuda(), torch.from_numpy(V).cuda(),
                                         torch.from_numpy(occ).cuda(), g, rg, rho=rho)
        rho2 = W.density_region(torch.from_numpy(psi).cuda(), torch.from_numpy(occ).cuda(), g, rg)
        out[name] = (hp.double().cpu().numpy(), ek.cpu().numpy(), ep.cpu().numpy(),
                     rho.cpu().numpy(), rho2.cpu().numpy())
    hp, ek, ep, rho, rho2 = out["box"]
    rho_ref = np.zeros(g.fine)
    for o in range(norb):
        r = RG.hpsi_local(psi[o].astype(np.float64), V.astype(np.float64), occ[o], n, cm, fm, g.h)
        d = np.abs(hp[o] - r["hpsi_c"]).max() / np.abs(r["hpsi_c"]).max()
        assert d < tol, (o, d)
        if dt == "float64":
            assert _rel(hp[o], r["hpsi_c"]) < RTOL64
        assert abs(ek[o] - r["ekin"]) < tol_e * abs(r["ekin"])
        assert abs(ep[o] - r["epot"]) < tol_e * abs(r["epot"])
        rho_ref += r["rho"]
    for got in (rho, rho2):
        assert np.abs(got - rho_ref).max() < tol_rho * np.abs(rho_ref).max()
    if dt == "float64":
        assert _rel(rho, rho_ref) < RTOL64
    # the box and the whole cell agree to rounding
    hc = out["cell"][0]
    assert np.abs(hp - hc).max() < (1e-13 if dt == "float64" else 2e-6) * np.abs(hc).max()

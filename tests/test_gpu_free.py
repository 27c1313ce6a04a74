"""GPU parity of free (isolated) boundary conditions against the free-space
oracle (dense non-circulant operators on an extended grid, no wrap-around).
FP64 bound 1e-12 as in the other parity tests: normwise (max|d| / max|ref|)
and elementwise where |ref| >= 1e-3 max|ref|."""
import numpy as np
import pytest

import oracle.free as FR
from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu
RTOL64 = 1e-12


def _err(got, ref):
    """max(normwise, elementwise on |ref| >= 1e-3 max|ref|) relative error."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    sc = np.abs(ref).max()
    if sc == 0:
        return float(np.abs(got).max())
    d = np.abs(got - ref)
    big = np.abs(ref) >= 1e-3 * sc
    return float(max(d.max() / sc, (d[big] / np.abs(ref[big])).max()))


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    return W


@pytest.mark.parametrize("n,norb", [((2, 3, 2), 2), ((4, 3, 5), 2), ((1, 1, 1), 1)])
def test_hpsi_free(W, n, norb):
    import torch
    g = W.Grid(n)
    pad = W.FREE_PAD
    padded = tuple(v + 2 * pad for v in n)
    psi = inputs.orbitals(111, norb, n)
    Vp = inputs.gaussian_potential(111, 0, padded)
    occ = np.array([2.0, 1.0][:norb])
    rho = torch.zeros(W.free_fine(g), dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local_free(torch.from_numpy(psi).cuda(), torch.from_numpy(Vp).cuda(),
                                   torch.from_numpy(occ).cuda(), g, rho=rho)
    Vx = FR.extend(Vp, n, 2 * pad)
    rho_ref = 0.0
    for o in range(norb):
        r = FR.hpsi_local(psi[o], Vx, occ[o], n)
        ref = r["hpsi_c"]
        assert _err(hp[o].cpu().numpy(), ref) < RTOL64
        assert abs(float(ek[o]) - r["ekin"]) < RTOL64 * abs(r["ekin"])
        assert abs(float(ep[o]) - r["epot"]) < RTOL64 * abs(r["epot"])
        rho_ref = rho_ref + r["rho"]
    got = rho.cpu().numpy()
    ref = FR.restrict(rho_ref, 2 * pad)
    assert _err(got, ref) < RTOL64
    rho2 = W.density_free(torch.from_numpy(psi).cuda(), torch.from_numpy(occ).cuda(), g)
    assert _err(rho2.cpu().numpy(), ref) < RTOL64


@pytest.mark.parametrize("free_axes", [(0, 0, 1), (1, 0, 0), (0, 1, 1), (0, 0, 0)])
def test_hpsi_mixed_conditions(W, free_axes):
    """Surface (one free axis) and other mixed conditions against the oracle
    with per-axis circulant / free-space matrices."""
    import torch
    n = (3, 2, 4)
    g = W.Grid(n, (0.25, 0.3, 0.2))
    pad = W.FREE_PAD
    padded = tuple(v + (2 * pad if free_axes[d] else 0) for d, v in enumerate(n))
    psi = inputs.orbitals(112, 2, n)
    Vp = inputs.gaussian_potential(112, 0, padded)
    occ = np.array([2.0, 1.0])
    rho = torch.zeros(W.bc_fine(g, free_axes), dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local_bc(torch.from_numpy(psi).cuda(), torch.from_numpy(Vp).cuda(),
                                 torch.from_numpy(occ).cuda(), g, free_axes, rho=rho)
    Vx = FR.extend_bc(Vp, n, 2 * pad, free_axes)
    rho_ref = 0.0
    for o in range(2):
        r = FR.hpsi_local_bc(psi[o], Vx, occ[o], n, free_axes, g.h)
        assert _err(hp[o].cpu().numpy(), r["hpsi_c"]) < RTOL64
        assert abs(float(ek[o]) - r["ekin"]) < RTOL64 * abs(r["ekin"])
        assert abs(float(ep[o]) - r["epot"]) < RTOL64 * abs(r["epot"])
        rho_ref = rho_ref + r["rho"]
    ref = FR.restrict_bc(rho_ref, n, 2 * pad, free_axes)
    assert _err(rho.cpu().numpy(), ref) < RTOL64


@pytest.mark.parametrize("dt", ["float64", "float32"])
def test_free_growing_supports_groups(W, dt):
    """Free conditions computed on supports that grow pass by pass: a ragged
    box, more orbitals than one density group, FP64 and FP32 (FP32 bounds of
    the other parity tests: 2e-6 H psi, 5e-6 rho, 5e-7 energies), H psi, the
    energies and the density against the free-space oracle."""
    import torch
    n = (6, 5, 7)
    norb = 6
    g = W.Grid(n, (0.25, 0.2, 0.3))
    pad = W.FREE_PAD
    padded = tuple(v + 2 * pad for v in n)
    psi = inputs.orbitals(113, norb, n).astype(dt)
    Vp = inputs.gaussian_potential(113, 0, padded).astype(dt)
    occ = np.array([2.0, 1.0, 2.0, 0.5, 1.5, 2.0])
    rho = torch.zeros(W.free_fine(g), dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local_free(torch.from_numpy(psi).cuda(), torch.from_numpy(Vp).cuda(),
                                   torch.from_numpy(occ).cuda(), g, rho=rho)
    tol, tol_rho, tol_e = (RTOL64, RTOL64, RTOL64) if dt == "float64" else (2e-6, 5e-6, 5e-7)
    Vx = FR.extend(Vp.astype(np.float64), n, 2 * pad)
    rho_ref = 0.0
    for o in range(norb):
        r = FR.hpsi_local(psi[o].astype(np.float64), Vx, occ[o], n, g.h)
        d = np.abs(hp[o].double().cpu().numpy() - r["hpsi_c"]).max() / np.abs(r["hpsi_c"]).max()
        assert d < tol, (o, d)
        if dt == "float64":
            assert _err(hp[o].cpu().numpy(), r["hpsi_c"]) < RTOL64
        assert abs(float(ek[o]) - r["ekin"]) < tol_e * abs(r["ekin"])
        assert abs(float(ep[o]) - r["epot"]) < tol_e * abs(r["epot"])
        rho_ref = rho_ref + r["rho"]
    ref = FR.restrict(rho_ref, 2 * pad)
    d = np.abs(rho.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert d < tol_rho, d

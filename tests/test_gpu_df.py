"""GPU parity of the double-FP32 form (WVL_F64_DF) against the FP64 oracle,
at the FP64 bound of 1e-12.

The fused kernels run with every value an unevaluated sum of two floats
(48 significant bits; products split exactly by FMA, sums by two-sum).  Per
convolution the error is a few 2^-48 of max|f| max|x| over the window, so
after the chain's 15 filters the results agree with the oracle to about
1e-14 relative: a hundred times inside the bound.  Inputs and H psi are
FP64 (converted on load and store); density and energies are reduced in
FP64.
"""
import numpy as np
import pytest

import oracle.wavelet as O
from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu
RTOL64 = 1e-12


def close(got, ref, rtol, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    scale = np.abs(ref).max()
    d = np.abs(got - ref)
    big = np.abs(ref) >= 1e-3 * scale
    norm = d.max() / scale
    elem = (d[big] / np.abs(ref[big])).max()
    assert norm <= rtol, f"{what}: normwise {norm:.3e} > {rtol:.1e}"
    assert elem <= rtol, f"{what}: elementwise {elem:.3e} > {rtol:.1e}"
    return norm


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    return W


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("n,norb", [((16, 16, 16), 2), ((20, 24, 16), 3), ((16, 20, 24), 20)])
def test_df_hpsi_energy_density(W, n, norb):
    """wvl_hpsi_local, wvl_energy and wvl_density with WVL_F64_DF (20
    orbitals put several in each density group)."""
    import torch
    g = W.Grid(n)
    psi = inputs.orbitals(61, norb, n)
    V = inputs.gaussian_potential(61, 0, n)
    occ = np.linspace(0.5, 2.0, norb)
    hp_r, rho_r, ek_r, ep_r = O.hpsi_batch(psi, V, occ, n)
    rho = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=rho, df=True)
    err = close(host(hp), hp_r, RTOL64, "hpsi df")
    assert err < 1e-13, err       # the double-FP32 accuracy, well inside the bound
    close(host(rho), rho_r, RTOL64, "rho df")
    assert np.max(np.abs(host(ek) - ek_r) / np.abs(ek_r)) < RTOL64
    assert np.max(np.abs(host(ep) - ep_r) / np.abs(ep_r)) < RTOL64
    rho2 = torch.zeros_like(rho)
    ek2, ep2 = W.energy(cuda(psi), cuda(V), cuda(occ), g, rho=rho2, df=True)
    assert np.max(np.abs(host(ek2) - ek_r) / np.abs(ek_r)) < RTOL64
    assert np.max(np.abs(host(ep2) - ep_r) / np.abs(ep_r)) < RTOL64
    close(host(rho2), rho_r, RTOL64, "rho df energy")
    close(host(W.density(cuda(psi), cuda(occ), g, df=True)), rho_r, RTOL64, "rho df density")


def test_df_plan_bench_cells_sampled(W):
    """The bench's 192 orbitals through a graph-captured WVL_F64_DF plan:
    one orbital of each cell against the oracle."""
    import torch
    sizes = [(56, 56, 56), (48, 48, 48), (40, 40, 40)]
    cells = [W.Grid(s) for s in sizes]
    cell_of_orb = [c for c in range(3) for _ in range(64)]
    psi_h = np.concatenate([inputs.orbital(2, o, sizes[c]) for o, c in enumerate(cell_of_orb)])
    Vs = [inputs.gaussian_potential(2, c, sizes[c]) for c in range(3)]
    plan = W.Plan(cells, cell_of_orb, prec=W.WVL_F64_DF, graph=True)
    psi = cuda(psi_h)
    V = [cuda(v) for v in Vs]
    occ = cuda(np.full(192, 2.0))
    rho = [torch.zeros(c.fine, dtype=torch.float64, device="cuda") for c in cells]
    hp = torch.empty_like(psi)
    ek = torch.empty(192, dtype=torch.float64, device="cuda")
    ep = torch.empty_like(ek)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            for r in rho:
                r.zero_()
            plan.hpsi(psi, V, occ, hpsi=hp, rho=rho, ekin=ek, epot=ep)
    torch.cuda.synchronize()
    for o in (5, 64 + 17, 128 + 63):
        c = cell_of_orb[o]
        a, b = plan.offsets[o], plan.offsets[o + 1]
        r = O.hpsi_local(psi_h[a:b], Vs[c], 2.0, sizes[c])
        close(host(hp[a:b]), r["hpsi_c"], RTOL64, f"df orbital {o}")
        assert rel(float(ek[o]), r["ekin"]) < RTOL64
        assert rel(float(ep[o]), r["epot"]) < RTOL64


def test_df_refused_where_not_built(W):
    """Entry points without a double-FP32 form return WVL_EUNSUPPORTED and
    enqueue nothing; the output buffer stays untouched."""
    import ctypes
    import torch
    g = W.Grid((16, 16, 16))
    c = cuda(inputs.orbitals(62, 1, g.n))
    s = torch.full((1,) + g.fine, 7.0, dtype=torch.float64, device="cuda")
    nbytes = W.workspace_size(g, W.WVL_F64, 1)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = W.lib().wvl_synthesis(ctypes.byref(g.c()), W.WVL_F64_DF, 1, c.data_ptr(), s.data_ptr(),
                               ws.data_ptr(), nbytes, None)
    torch.cuda.synchronize()
    assert st == 5                      # WVL_EUNSUPPORTED
    assert bool((s == 7.0).all())

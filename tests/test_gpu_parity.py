"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
identical seeded inputs.

Tolerances.  FP64: 1e-12 relative, the stated accuracy target -- normwise
(max|d| / max|ref|) and elementwise where |ref| >= 1e-3 max|ref|; energies
relative to |E|.  The kernels and the oracle sum the same terms in different
orders (FMA chains of at most 29 taps per pass, 15 passes), which leaves
differences of a few 1e-16 relative.  FP32: storage and convolutions in
binary32 (unit roundoff 6e-8); after 15 passes of up to 29 taps the
normwise error is a few 1e-7, bounded here by 2e-6 (H psi, psi_r, single
operators), 5e-6 (density) and 5e-7 (energies), with the oracle run in FP64
on the same FP32-rounded inputs (elementwise bound below).
"""
import numpy as np
import pytest

import oracle.wavelet as O
from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL64 = 1e-12
# FP32 bounds, normwise: H psi, psi_r and single operators 2e-6, density
# 5e-6, energies 5e-7 relative (observed at most 5.3e-7, 1.2e-6 and 7.4e-8).
# Elementwise (|ref| >= 1e-3 max|ref|): 2e-4.  An FP32 output's error comes
# from the rounding of its neighbours' contributions, about u sum|f||x| over
# the stencil, not from its own size, so an entry at 1e-3 of the maximum
# carries up to normwise error / 1e-3 (observed at most 1.5e-4).
RTOL32, RTOL32_RHO, RTOL32_E, ELEM32 = 2e-6, 5e-6, 5e-7, 2e-4


def close(got, ref, rtol, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    scale = np.abs(ref).max()
    if scale == 0:
        assert np.abs(got).max() == 0, what
        return
    d = np.abs(got - ref)
    norm = d.max() / scale
    big = np.abs(ref) >= 1e-3 * scale
    elem = (d[big] / np.abs(ref[big])).max()
    assert norm <= rtol, f"{what}: normwise {norm:.3e} > {rtol:.1e}"
    eb = rtol if rtol <= 1e-9 else ELEM32
    assert elem <= eb, f"{what}: elementwise {elem:.3e} > {eb:.1e}"


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    assert W.device_count() >= 1
    return W


def cuda(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().double().cpu().numpy()


GRIDS = [(1, 2, 3), (3, 5, 2), (4, 4, 4), (5, 6, 7), (8, 8, 8), (12, 20, 9), (16, 16, 16)]


# ------------------------------------------------------------- single ops
@pytest.mark.parametrize("n", GRIDS)
def test_synthesis_analysis(W, n):
    g = W.Grid(n)
    psi = inputs.orbitals(11, 2, n)
    s = W.synthesis(cuda(psi), g)
    for o in range(2):
        ref = O.synthesis3d(O.uncompress(psi[o], n))
        close(host(s[o]), ref, RTOL64, f"synthesis {n}")
    z = inputs.random_field(11, 7, (2,) + g.fine)
    c = W.analysis(cuda(z), g)
    for o in range(2):
        ref = O.compress(O.analysis3d(z[o]), n)
        close(host(c[o]), ref, RTOL64, f"analysis {n}")


@pytest.mark.parametrize("n", GRIDS)
def test_magicfilter_and_transpose(W, n):
    g = W.Grid(n)
    x = inputs.random_field(12, 1, (3,) + g.fine)
    a = W.magicfilter(cuda(x), g)
    b = W.magicfilter_T(cuda(x), g)
    for o in range(3):
        close(host(a[o]), O.magicfilter3d(x[o]), RTOL64, f"mf {n}")
        close(host(b[o]), O.magicfilter_T3d(x[o]), RTOL64, f"mfT {n}")


@pytest.mark.parametrize("n", GRIDS)
@pytest.mark.parametrize("with_k0", [False, True])
def test_kinetic(W, n, with_k0):
    hg = (0.25, 0.3, 0.45)
    g = W.Grid(n, hg)
    s = inputs.random_field(13, 1, (2,) + g.fine)
    k0 = inputs.random_field(13, 2, (2,) + g.fine) if with_k0 else None
    out, ek = W.kinetic(cuda(s), g, None if k0 is None else cuda(k0))
    for o in range(2):
        kin = O.kinetic3d(s[o], hg)
        ref = kin + (k0[o] if with_k0 else 0.0)
        close(host(out[o]), ref, RTOL64, f"kinetic {n}")
        e = float(np.sum(s[o] * kin))
        assert rel(float(ek[o]), e) < RTOL64 * 10, (float(ek[o]), e)


# ---------------------------------------------------- local Hamiltonian
def _case(cfg, n, norb, occ=2.0):
    psi = inputs.orbitals(cfg, norb, n)
    V = inputs.gaussian_potential(cfg, 0, n)
    occv = np.full(norb, occ) if np.isscalar(occ) else np.asarray(occ, dtype=np.float64)
    return psi, V, occv


@pytest.mark.parametrize("n,norb", [((1, 1, 1), 2), ((3, 5, 2), 3), ((8, 8, 8), 2),
                                    ((5, 6, 7), 5), ((12, 10, 14), 2)])
def test_hpsi_local_f64(W, n, norb):
    g = W.Grid(n)
    psi, V, occ = _case(21, n, norb, occ=[2.0, 1.0, 0.5, 2.0, 1.5][:norb])
    import torch
    rho0 = np.full(g.fine, 0.125)            # rho is accumulated
    rho = cuda(rho0)
    hp, ek, ep = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=rho)
    hp_r, rho_r, ek_r, ep_r = O.hpsi_batch(psi, V, occ, n)
    for o in range(norb):
        close(host(hp[o]), hp_r[o], RTOL64, f"hpsi {n} orbital {o}")
        assert rel(float(ek[o]), ek_r[o]) < RTOL64, ("ekin", float(ek[o]), ek_r[o])
        assert rel(float(ep[o]), ep_r[o]) < RTOL64, ("epot", float(ep[o]), ep_r[o])
    close(host(rho), rho0 + rho_r, RTOL64, "rho (accumulated onto 0.125)")


def test_config0_full(W):
    """1 orbital, coarse 32^3 (fine 64^3), Gaussian-sum V, occ 2: every output."""
    n = (32, 32, 32)
    g = W.Grid(n)
    psi, V, occ = _case(0, n, 1)
    import torch
    rho = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=rho)
    r = O.hpsi_local(psi[0], V, 2.0, n)
    close(host(hp[0]), r["hpsi_c"], RTOL64, "cfg0 hpsi")
    close(host(rho), r["rho"], RTOL64, "cfg0 rho")
    assert rel(float(ek[0]), r["ekin"]) < RTOL64
    assert rel(float(ep[0]), r["epot"]) < RTOL64
    # energy-only entry point and the density entry point agree
    rho2 = torch.zeros_like(rho)
    ek2, ep2 = W.energy(cuda(psi), cuda(V), cuda(occ), g, rho=rho2)
    assert rel(float(ek2[0]), r["ekin"]) < RTOL64
    assert rel(float(ep2[0]), r["epot"]) < RTOL64
    close(host(rho2), r["rho"], RTOL64, "cfg0 energy rho")
    rho3 = W.density(cuda(psi), cuda(occ), g)
    close(host(rho3), r["rho"], RTOL64, "cfg0 density")


def test_hpsi_deterministic(W):
    n = (10, 10, 10)
    g = W.Grid(n)
    psi, V, occ = _case(22, n, 7)
    a = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=cuda(np.zeros(g.fine)))
    b = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=cuda(np.zeros(g.fine)))
    for x, y in zip(a, b):
        assert np.array_equal(host(x), host(y))


def test_many_orbitals_groups(W):
    """Enough orbitals on a small cell that the density pass splits them into
    groups and reduces the group partials."""
    n = (6, 6, 6)
    g = W.Grid(n)
    psi, V, occ = _case(23, n, 40)
    rho = cuda(np.zeros(g.fine))
    hp, ek, ep = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=rho)
    hp_r, rho_r, ek_r, ep_r = O.hpsi_batch(psi, V, occ, n)
    close(host(hp), hp_r, RTOL64, "hpsi many")
    close(host(rho), rho_r, RTOL64, "rho many")
    assert np.max(np.abs(host(ek) - ek_r) / np.abs(ek_r)) < RTOL64
    assert np.max(np.abs(host(ep) - ep_r) / np.abs(ep_r)) < RTOL64


def test_zero_orbitals(W):
    import torch
    g = W.Grid((4, 4, 4))
    psi = torch.zeros((0, g.ncoef), dtype=torch.float64, device="cuda")
    V = cuda(np.zeros(g.fine))
    hp, ek, ep = W.hpsi_local(psi, V, torch.zeros(0, dtype=torch.float64, device="cuda"), g)
    assert hp.numel() == 0 and ek.numel() == 0


# ----------------------------------------------------------------- FP32
@pytest.mark.parametrize("n,norb", [((6, 5, 7), 3), ((12, 12, 12), 4)])
def test_hpsi_local_f32(W, n, norb):
    import torch
    g = W.Grid(n)
    psi, V, occ = _case(31, n, norb)
    psi32 = psi.astype(np.float32)
    V32 = V.astype(np.float32)
    rho = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local(cuda(psi32), cuda(V32), cuda(occ), g, rho=rho)
    hp_r, rho_r, ek_r, ep_r = O.hpsi_batch(psi32.astype(np.float64), V32.astype(np.float64), occ, n)
    close(host(hp), hp_r, RTOL32, "hpsi f32")
    close(host(rho), rho_r, RTOL32_RHO, "rho f32")
    assert np.max(np.abs(host(ek) - ek_r) / np.abs(ek_r)) < RTOL32_E
    assert np.max(np.abs(host(ep) - ep_r) / np.abs(ep_r)) < RTOL32_E


def test_f32_full_size_sampled(W):
    """256 orbitals on a coarse 48^3 cell in FP32 through an autotuned,
    graph-captured plan (the bench's FP32 form): two orbitals against the
    oracle (run in FP64 on the FP32-rounded inputs), the density of all 256
    against the FP64 GPU form, at the FP32 bounds."""
    import torch
    n = (48, 48, 48)
    g = W.Grid(n)
    norb = 256
    psi = np.concatenate([inputs.orbital(3, o, n) for o in range(norb)]).astype(np.float32)
    V = inputs.gaussian_potential(3, 0, n).astype(np.float32)
    occ = cuda(np.full(norb, 2.0))
    out = {}
    for prec, p_, v_ in ((W.WVL_F32, cuda(psi), cuda(V)),
                         (W.WVL_F64, cuda(psi.astype(np.float64)), cuda(V.astype(np.float64)))):
        plan = W.Plan([g], [0] * norb, prec=prec, graph=True, autotune=True)
        rho = [torch.zeros(g.fine, dtype=torch.float64, device="cuda")]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            plan.autotune(p_, [v_], occ, rho=rho)
            hp = torch.empty_like(p_)
            ek = torch.empty(norb, dtype=torch.float64, device="cuda")
            ep = torch.empty_like(ek)
            for _ in range(2):
                rho[0].zero_()
                plan.hpsi(p_, [v_], occ, hpsi=hp, rho=rho, ekin=ek, epot=ep)
        torch.cuda.synchronize()
        out[prec] = (hp, ek, ep, rho[0], plan)
    hp, ek, ep, rho32, plan = out[W.WVL_F32]
    for o in (0, norb - 1):
        a, b = plan.offsets[o], plan.offsets[o + 1]
        r = O.hpsi_local(psi[a:b].astype(np.float64), V.astype(np.float64), 2.0, n)
        close(host(hp[a:b]), r["hpsi_c"], RTOL32, f"f32 orbital {o}")
        assert rel(float(ek[o]), r["ekin"]) < RTOL32_E
        assert rel(float(ep[o]), r["epot"]) < RTOL32_E
    close(host(rho32), host(out[W.WVL_F64][3]), RTOL32_RHO, "f32 rho")


@pytest.mark.parametrize("n", [(4, 4, 4), (9, 7, 5)])
def test_single_ops_f32(W, n):
    g = W.Grid(n)
    x = inputs.random_field(32, 1, (2,) + g.fine).astype(np.float32)
    x64 = x.astype(np.float64)
    close(host(W.magicfilter(cuda(x), g)[0]), O.magicfilter3d(x64[0]), RTOL32, "mf f32")
    close(host(W.magicfilter_T(cuda(x), g)[1]), O.magicfilter_T3d(x64[1]), RTOL32, "mfT f32")
    out, ek = W.kinetic(cuda(x), g)
    close(host(out[0]), O.kinetic3d(x64[0]), RTOL32, "kin f32")
    s = W.synthesis(cuda(x.reshape(2, -1)), g)
    close(host(s[1]), O.synthesis3d(O.uncompress(x64[1].reshape(-1), n)), RTOL32, "syn f32")


# ----------------------------------------------------------------- plans
@pytest.mark.parametrize("graph,autotune", [(False, False), (True, False), (True, True)])
def test_plan_uneven_cells(W, graph, autotune):
    import torch
    cells = [W.Grid((6, 6, 6)), W.Grid((5, 4, 7)), W.Grid((8, 8, 8), (0.2, 0.25, 0.3))]
    cell_of_orb = [0, 0, 1, 1, 1, 2, 0]
    plan = W.Plan(cells, cell_of_orb, prec=0, graph=graph, autotune=autotune)
    psis = [inputs.orbital(41, o, cells[c].n) for o, c in enumerate(cell_of_orb)]
    Vs = [inputs.gaussian_potential(41, c, cells[c].n) for c in range(3)]
    occ = np.array([2.0, 1.0, 2.0, 0.5, 2.0, 2.0, 1.5])
    psi = cuda(np.concatenate(psis))
    V = [cuda(v) for v in Vs]
    occ_d = cuda(occ)
    rho = [torch.zeros(c.fine, dtype=torch.float64, device="cuda") for c in cells]
    side = torch.cuda.Stream()          # graphs are captured on non-default streams
    side.wait_stream(torch.cuda.current_stream())
    hp = torch.empty_like(psi)
    ek = torch.empty(len(occ), dtype=torch.float64, device="cuda")
    ep = torch.empty_like(ek)
    with torch.cuda.stream(side):
        if autotune:
            plan.autotune(psi, V, occ_d)
            assert "autotuned" in plan.describe()
    for rep in range(3):          # later calls replay the graph
        with torch.cuda.stream(side):
            for r in rho:
                r.zero_()
            plan.hpsi(psi, V, occ_d, hpsi=hp, rho=rho, ekin=ek, epot=ep)
        torch.cuda.synchronize()
        hph = host(hp)
        rho_ref = [np.zeros(c.fine) for c in cells]
        for o, c in enumerate(cell_of_orb):
            r = O.hpsi_local(psis[o], Vs[c], occ[o], cells[c].n, cells[c].h)
            a, b = plan.offsets[o], plan.offsets[o + 1]
            close(hph[a:b], r["hpsi_c"], RTOL64, f"plan orbital {o}")
            assert rel(float(ek[o]), r["ekin"]) < RTOL64
            assert rel(float(ep[o]), r["epot"]) < RTOL64
            rho_ref[c] += r["rho"]
        for c in range(3):
            close(host(rho[c]), rho_ref[c], RTOL64, f"plan rho cell {c}")


def test_plan_profiling(W):
    import torch
    cells = [W.Grid((6, 6, 6))]
    plan = W.Plan(cells, [0, 0, 0], prec=0, graph=True)
    psi = cuda(np.concatenate([inputs.orbital(42, o, (6, 6, 6)) for o in range(3)]))
    V = [cuda(inputs.gaussian_potential(42, 0, (6, 6, 6)))]
    plan.set_profiling(True)
    for _ in range(3):
        plan.hpsi(psi, V, cuda(np.full(3, 2.0)))
    prof = plan.profile()
    assert prof["kinetic"][1] == 3 and prof["kinetic"][0] > 0
    assert prof["synthesis"][1] == 3


# --------------------------------------------- full size, sampled outputs
def test_config2_full_size_sampled(W):
    """192 orbitals on coarse 40^3, 48^3, 56^3 cells in one autotuned,
    graph-captured plan (the bench launch configuration): one orbital of
    each cell checked element by element against the oracle, and the
    identity sum_I V rho = sum_o occ_o Epot_o on every cell."""
    import torch
    sizes = [(56, 56, 56), (48, 48, 48), (40, 40, 40)]
    cells = [W.Grid(s) for s in sizes]
    cell_of_orb = [c for c in range(3) for _ in range(64)]
    plan = W.Plan(cells, cell_of_orb, prec=0, graph=True, autotune=True)
    psi_h = np.concatenate([inputs.orbital(2, o, sizes[c]) for o, c in enumerate(cell_of_orb)])
    Vs = [inputs.gaussian_potential(2, c, sizes[c]) for c in range(3)]
    occ = np.full(192, 2.0)
    psi = cuda(psi_h)
    V = [cuda(v) for v in Vs]
    occ_d = cuda(occ)
    rho = [torch.zeros(c.fine, dtype=torch.float64, device="cuda") for c in cells]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.autotune(psi, V, occ_d, rho=rho)
        hp = torch.empty_like(psi)
        ek = torch.empty(192, dtype=torch.float64, device="cuda")
        ep = torch.empty_like(ek)
        for _ in range(2):         # capture, then replay
            for r in rho:
                r.zero_()
            plan.hpsi(psi, V, occ_d, hpsi=hp, rho=rho, ekin=ek, epot=ep)
    torch.cuda.synchronize()
    ekh, eph = host(ek), host(ep)
    for o in (5, 64 + 17, 128 + 63):
        c = cell_of_orb[o]
        a, b = plan.offsets[o], plan.offsets[o + 1]
        r = O.hpsi_local(psi_h[a:b], Vs[c], 2.0, sizes[c])
        close(host(hp[a:b]), r["hpsi_c"], RTOL64, f"cfg2 orbital {o}")
        assert rel(ekh[o], r["ekin"]) < RTOL64
        assert rel(eph[o], r["epot"]) < RTOL64
    for c in range(3):
        rh = host(rho[c])
        assert rh.min() >= 0
        lhs = float(np.sum(Vs[c] * rh))
        rhs = float(np.sum(2.0 * eph[64 * c: 64 * (c + 1)]))
        assert rel(lhs, rhs) < 1e-11


@pytest.mark.parametrize("nc,ops", [(128, ("mf", "mft", "kin", "syn", "ana")), (96, ("mf", "kin"))])
def test_config1_single_passes_full_size(W, nc, ops):
    """The single-pass sweep's largest grids (fine 256^3 and 192^3, one
    orbital, uniform[-1, 1] inputs from seed): each 3D operator element by
    element against the oracle at the FP64 bound."""
    n = (nc, nc, nc)
    g = W.Grid(n)
    x = inputs.random_field(12, nc, (1,) + g.fine)
    if "mf" in ops:
        close(host(W.magicfilter(cuda(x), g)[0]), O.magicfilter3d(x[0]), RTOL64, f"mf {nc}")
    if "mft" in ops:
        close(host(W.magicfilter_T(cuda(x), g)[0]), O.magicfilter_T3d(x[0]), RTOL64, f"mfT {nc}")
    if "kin" in ops:
        out, ek = W.kinetic(cuda(x), g)
        close(host(out[0]), O.kinetic3d(x[0]), RTOL64, f"kinetic {nc}")
    if "syn" in ops:
        c = inputs.orbitals(12, 1, n)
        s = W.synthesis(cuda(c), g)
        ref = O.synthesis3d(O.uncompress(c[0], n))
        close(host(s[0]), ref, RTOL64, f"synthesis {nc}")
    if "ana" in ops:
        back = W.analysis(cuda(x), g)
        ref = O.compress(O.analysis3d(x[0]), n)
        close(host(back[0]), ref, RTOL64, f"analysis {nc}")


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_longest_lines_f32(W, axis):
    """FP32 lines of the largest fine extent (1024 points) along each axis,
    the other axes at 2 fine points (the transposing passes: the fused
    kernels take extents of 32 to 128), against the oracle on the
    FP32-rounded inputs."""
    import torch
    n = [1, 1, 1]
    n[axis] = 512
    n = tuple(n)
    g = W.Grid(n, (0.3, 0.25, 0.35))
    psi = inputs.orbitals(372, 2, n).astype(np.float32)
    V = inputs.gaussian_potential(372, 0, n).astype(np.float32)
    occ = np.array([2.0, 1.0])
    rho = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=rho)
    hp_r, rho_r, ek_r, ep_r = O.hpsi_batch(psi.astype(np.float64), V.astype(np.float64), occ, n,
                                           g.h)
    close(host(hp), hp_r, RTOL32, f"hpsi f32 axis {axis}")
    close(host(rho), rho_r, RTOL32_RHO, f"rho f32 axis {axis}")
    assert np.max(np.abs(host(ek) - ek_r) / np.abs(ek_r)) < RTOL32_E
    assert np.max(np.abs(host(ep) - ep_r) / np.abs(ep_r)) < RTOL32_E

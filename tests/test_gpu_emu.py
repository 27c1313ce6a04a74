"""GPU parity of the FP64-accurate tensor-core passes (WVL_F64_EMU) against
the FP64 oracle, at the same 1e-12 bounds as the native FP64 path.

Each convolution sum is formed from six 10-bit digits per operand on a
power-of-two scale per line (data) and per filter (taps); digit products are
summed exactly in FP32 and recombined in 64-bit integers, dropping terms
below 2^-62 of max|f| max|x|.  The error per pass is thus of the order of
FP64 rounding relative to the line's largest input, so after 15 passes the
results agree with the oracle to a few 1e-15, like the FP64 kernels.

The sizes span several 128-line tiles and 32-output windows with ragged
ends, lines shorter than the filter (wrapped more than once), and the
compressed-layout gather/scatter of the first and last passes.
"""
import numpy as np
import pytest

import oracle.free as FR
import oracle.precond as PC
import oracle.region as RG
import oracle.wavelet as O
from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu
RTOL64 = 1e-12


def close(got, ref, rtol, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    scale = np.abs(ref).max()
    if scale == 0:
        assert np.abs(got).max() == 0, what
        return
    d = np.abs(got - ref)
    big = np.abs(ref) >= 1e-3 * scale
    norm = d.max() / scale
    elem = (d[big] / np.abs(ref[big])).max()
    assert norm <= rtol, f"{what}: normwise {norm:.3e} > {rtol:.1e}"
    assert elem <= rtol, f"{what}: elementwise {elem:.3e} > {rtol:.1e}"


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    yield W
    assert W.wait_timeouts() == 0


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


# fine extents: (40, 6, 10) -- two windows on x, lines of 6 < 16 taps;
# (34, 18, 8) -- 144 lines (two tiles) on x; (48, 48, 48) -- 18 tiles
GRIDS = [(1, 2, 3), (20, 3, 5), (17, 9, 4), (24, 24, 24)]


@pytest.mark.parametrize("n", GRIDS)
def test_emu_synthesis_analysis(W, n):
    g = W.Grid(n)
    psi = inputs.orbitals(311, 2, n)
    s = W.synthesis(cuda(psi), g, emu=True)
    for o in range(2):
        close(host(s[o]), O.synthesis3d(O.uncompress(psi[o], n)), RTOL64, f"synthesis {n}")
    z = inputs.random_field(311, 7, (2,) + g.fine)
    c = W.analysis(cuda(z), g, emu=True)
    for o in range(2):
        close(host(c[o]), O.compress(O.analysis3d(z[o]), n), RTOL64, f"analysis {n}")


@pytest.mark.parametrize("n", GRIDS)
def test_emu_magicfilter_and_transpose(W, n):
    g = W.Grid(n)
    x = inputs.random_field(312, 1, (2,) + g.fine)
    a = W.magicfilter(cuda(x), g, emu=True)
    b = W.magicfilter_T(cuda(x), g, emu=True)
    for o in range(2):
        close(host(a[o]), O.magicfilter3d(x[o]), RTOL64, f"mf {n}")
        close(host(b[o]), O.magicfilter_T3d(x[o]), RTOL64, f"mfT {n}")


@pytest.mark.parametrize("n", GRIDS)
@pytest.mark.parametrize("with_k0", [False, True])
def test_emu_kinetic(W, n, with_k0):
    hg = (0.25, 0.3, 0.45)
    g = W.Grid(n, hg)
    s = inputs.random_field(313, 1, (2,) + g.fine)
    k0 = inputs.random_field(313, 2, (2,) + g.fine) if with_k0 else None
    out, ek = W.kinetic(cuda(s), g, None if k0 is None else cuda(k0), emu=True)
    for o in range(2):
        kin = O.kinetic3d(s[o], hg)
        close(host(out[o]), kin + (k0[o] if with_k0 else 0.0), RTOL64, f"kinetic {n}")
        assert rel(float(ek[o]), float(np.sum(s[o] * kin))) < 10 * RTOL64


def test_emu_localised_fields(W):
    """Fields decaying over ten decades from a centre (as localised orbitals
    do): each line is scaled by its own largest value, so the small tails do
    not lose the bound's precision."""
    n = (24, 20, 16)
    g = W.Grid(n, (0.3, 0.25, 0.35))
    N3, N2, N1 = g.fine
    z, y, x = np.meshgrid(np.arange(N3), np.arange(N2), np.arange(N1), indexing="ij")
    r2 = (x - 17.0) ** 2 + (y - 11.0) ** 2 + (z - 9.0) ** 2
    env = np.exp(-r2 / (2 * 4.0 ** 2))
    f = inputs.random_field(315, 1, (1,) + g.fine) * env
    a = W.magicfilter(cuda(f), g, emu=True)
    close(host(a[0]), O.magicfilter3d(f[0]), RTOL64, "mf localised")
    k, ek = W.kinetic(cuda(f), g, emu=True)
    kin = O.kinetic3d(f[0], g.h)
    close(host(k[0]), kin, RTOL64, "kinetic localised")
    assert rel(float(ek[0]), float(np.sum(f[0] * kin))) < 10 * RTOL64
    # compressed coefficients with a coarse envelope, through the whole chain
    cz, cy, cx = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    cenv = np.exp(-((cx - 8.0) ** 2 + (cy - 5.0) ** 2 + (cz - 4.0) ** 2) / (2 * 2.0 ** 2)).ravel()
    psi = inputs.orbitals(315, 1, n)[0] * np.concatenate([cenv, np.repeat(cenv, 7)])
    V = inputs.gaussian_potential(315, 0, n)
    hp, ek2, ep2 = W.hpsi_local(cuda(psi[None]), cuda(V), cuda(np.array([2.0])), g, emu=True)
    ref = O.hpsi_local(psi, V, 2.0, n, g.h)
    close(host(hp[0]), ref["hpsi_c"], RTOL64, "hpsi localised")
    assert rel(float(ek2[0]), ref["ekin"]) < RTOL64
    assert rel(float(ep2[0]), ref["epot"]) < RTOL64


@pytest.mark.parametrize("n,norb", [((1, 1, 1), 2), ((5, 6, 7), 3), ((20, 17, 9), 2)])
def test_emu_hpsi_local(W, n, norb):
    g = W.Grid(n)
    psi = inputs.orbitals(321, norb, n)
    V = inputs.gaussian_potential(321, 0, n)
    occ = np.array([2.0, 1.0, 0.5][:norb])
    rho0 = np.full(g.fine, 0.125)
    rho = cuda(rho0)
    hp, ek, ep = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=rho, emu=True)
    hp_r, rho_r, ek_r, ep_r = O.hpsi_batch(psi, V, occ, n)
    for o in range(norb):
        close(host(hp[o]), hp_r[o], RTOL64, f"hpsi {n} orbital {o}")
        assert rel(float(ek[o]), ek_r[o]) < RTOL64
        assert rel(float(ep[o]), ep_r[o]) < RTOL64
    close(host(rho), rho0 + rho_r, RTOL64, "rho")
    ekk, epp = W.energy(cuda(psi), cuda(V), cuda(occ), g, emu=True)
    for o in range(norb):
        assert rel(float(ekk[o]), ek_r[o]) < RTOL64
        assert rel(float(epp[o]), ep_r[o]) < RTOL64


def test_emu_matches_native_f64(W):
    """Same inputs through both FP64 forms: they differ by rounding only."""
    n = (16, 12, 10)
    g = W.Grid(n)
    psi = cuda(inputs.orbitals(322, 3, n))
    V = cuda(inputs.gaussian_potential(322, 0, n))
    occ = cuda(np.array([2.0, 2.0, 1.0]))
    a = W.hpsi_local(psi, V, occ, g)
    b = W.hpsi_local(psi, V, occ, g, emu=True)
    d = float((a[0] - b[0]).abs().max() / a[0].abs().max())
    assert d < 1e-13, d
    for k in (1, 2):
        assert float(((a[k] - b[k]) / a[k]).abs().max()) < 1e-13


def test_emu_plan_batched(W):
    """Plan with WVL_F64_EMU over cells of three sizes, graph-captured."""
    import torch
    ns = [(6, 5, 4), (9, 9, 9), (20, 7, 3)]
    per = 2
    cell_of = [c for c in range(3) for _ in range(per)]
    plan = W.Plan([W.Grid(n) for n in ns], cell_of, prec=W.WVL_F64_EMU, graph=True)
    psi = torch.empty(plan.total, dtype=torch.float64, device="cuda")
    Vs, refs = [], []
    for c, n in enumerate(ns):
        p = inputs.orbitals(330 + c, per, n)
        for k in range(per):
            o = c * per + k
            psi[plan.offsets[o]:plan.offsets[o + 1]] = cuda(p[k])
        V = inputs.gaussian_potential(330 + c, 0, n)
        Vs.append(cuda(V))
        refs.append(O.hpsi_batch(p, V, np.full(per, 2.0), n))
    occ = torch.full((plan.norb,), 2.0, dtype=torch.float64, device="cuda")
    rho = [torch.zeros(W.Grid(n).fine, dtype=torch.float64, device="cuda") for n in ns]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):          # capture, then replay
            for r in rho:
                r.zero_()
            hp, ek, ep = plan.hpsi(psi, Vs, occ, rho=rho)
    s.synchronize()
    for c in range(3):
        hp_r, rho_r, ek_r, ep_r = refs[c]
        for k in range(per):
            o = c * per + k
            close(host(hp[plan.offsets[o]:plan.offsets[o + 1]]), hp_r[k], RTOL64, f"cell {c}")
            assert rel(float(ek[o]), ek_r[k]) < RTOL64
            assert rel(float(ep[o]), ep_r[k]) < RTOL64
        close(host(rho[c]), rho_r, RTOL64, f"rho cell {c}")


def test_emu_region(W):
    import torch
    n = (12, 10, 14)
    g = W.Grid(n)
    cm, fm = RG.sphere_masks(n, (0, 9, 13), 4.5, 2.5)
    reg = W.Region(g, cm, fm)
    psi = inputs.random_field(341, 1, (2, reg.clen))
    V = inputs.gaussian_potential(341, 0, n)
    occ = np.array([2.0, 1.0])
    rho = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local_region(cuda(psi), cuda(V), cuda(occ), g, reg, rho=rho, emu=True)
    rho_ref = np.zeros(g.fine)
    for o in range(2):
        r = RG.hpsi_local(psi[o], V, occ[o], n, cm, fm)
        close(host(hp[o]), r["hpsi_c"], RTOL64, "region hpsi")
        assert rel(float(ek[o]), r["ekin"]) < RTOL64
        assert rel(float(ep[o]), r["epot"]) < RTOL64
        rho_ref += r["rho"]
    close(host(rho), rho_ref, RTOL64, "region rho")


def test_emu_free(W):
    import torch
    n = (4, 3, 5)
    g = W.Grid(n)
    pad = W.FREE_PAD
    padded = tuple(v + 2 * pad for v in n)
    psi = inputs.orbitals(351, 2, n)
    Vp = inputs.gaussian_potential(351, 0, padded)
    occ = np.array([2.0, 1.0])
    rho = torch.zeros(W.free_fine(g), dtype=torch.float64, device="cuda")
    hp, ek, ep = W.hpsi_local_free(cuda(psi), cuda(Vp), cuda(occ), g, rho=rho, emu=True)
    Vx = FR.extend(Vp, n, 2 * pad)
    rho_ref = 0.0
    for o in range(2):
        r = FR.hpsi_local(psi[o], Vx, occ[o], n)
        close(host(hp[o]), r["hpsi_c"], RTOL64, "free hpsi")
        assert rel(float(ek[o]), r["ekin"]) < RTOL64
        assert rel(float(ep[o]), r["epot"]) < RTOL64
        rho_ref = rho_ref + r["rho"]
    close(host(rho), FR.restrict(rho_ref, 2 * pad), RTOL64, "free rho")


def test_emu_precondition(W):
    import torch
    n = (12, 10, 14)
    g = W.Grid(n, (0.25, 0.3, 0.35))
    G = inputs.orbitals(361, 2, n)
    eps = np.array([-0.4, -1.2])
    x, rr = W.precondition(cuda(G), cuda(eps), g, 3, emu=True)
    ref = PC.precondition_batch(G, eps, n, 3, g.h)
    assert float(np.abs(host(x) - ref).max() / np.abs(ref).max()) < 1e-11


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("emu", [False, True])
def test_longest_lines(W, axis, emu):
    """Lines of the largest fine extent (1024 points) along each axis, with
    the other two axes at their smallest (2 fine points): the native FP64
    kernels and the tensor-core form against the oracle."""
    n = [1, 1, 1]
    n[axis] = 512
    n = tuple(n)
    g = W.Grid(n, (0.3, 0.25, 0.35))
    psi = inputs.orbitals(371, 2, n)
    V = inputs.gaussian_potential(371, 0, n)
    occ = np.array([2.0, 1.0])
    rho = cuda(np.zeros(g.fine))
    hp, ek, ep = W.hpsi_local(cuda(psi), cuda(V), cuda(occ), g, rho=rho, emu=emu)
    hp_r, rho_r, ek_r, ep_r = O.hpsi_batch(psi, V, occ, n, g.h)
    for o in range(2):
        close(host(hp[o]), hp_r[o], RTOL64, f"hpsi axis {axis} emu {emu}")
        assert rel(float(ek[o]), ek_r[o]) < RTOL64
        assert rel(float(ep[o]), ep_r[o]) < RTOL64
    close(host(rho), rho_r, RTOL64, "rho")


def test_emu_full_size_sampled(W):
    """The 192 orbitals of the benchmark workload (coarse 56^3, 48^3, 40^3
    cells) through a graph-captured WVL_F64_EMU plan, as bench.py times it:
    one orbital of each cell element by element against the oracle, and
    sum_I V rho = sum_o occ_o Epot_o on every cell."""
    import torch
    sizes = [(56, 56, 56), (48, 48, 48), (40, 40, 40)]
    cells = [W.Grid(s) for s in sizes]
    cell_of_orb = [c for c in range(3) for _ in range(64)]
    plan = W.Plan(cells, cell_of_orb, prec=W.WVL_F64_EMU, graph=True)
    psi_h = np.concatenate([inputs.orbital(2, o, sizes[c]) for o, c in enumerate(cell_of_orb)])
    Vs = [inputs.gaussian_potential(2, c, sizes[c]) for c in range(3)]
    psi = cuda(psi_h)
    V = [cuda(v) for v in Vs]
    occ = cuda(np.full(192, 2.0))
    rho = [torch.zeros(c.fine, dtype=torch.float64, device="cuda") for c in cells]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        hp = torch.empty_like(psi)
        ek = torch.empty(192, dtype=torch.float64, device="cuda")
        ep = torch.empty_like(ek)
        for _ in range(2):         # capture, then replay
            for r in rho:
                r.zero_()
            plan.hpsi(psi, V, occ, hpsi=hp, rho=rho, ekin=ek, epot=ep)
    torch.cuda.synchronize()
    ekh, eph = host(ek), host(ep)
    for o in (7, 64 + 30, 128 + 63):
        c = cell_of_orb[o]
        a, b = plan.offsets[o], plan.offsets[o + 1]
        r = O.hpsi_local(psi_h[a:b], Vs[c], 2.0, sizes[c])
        close(host(hp[a:b]), r["hpsi_c"], RTOL64, f"orbital {o}")
        assert rel(ekh[o], r["ekin"]) < RTOL64
        assert rel(eph[o], r["epot"]) < RTOL64
    for c in range(3):
        rh = host(rho[c])
        assert rh.min() >= 0
        assert rel(float(np.sum(Vs[c] * rh)), float(np.sum(2.0 * eph[64 * c: 64 * (c + 1)]))) < 1e-11

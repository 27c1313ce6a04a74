"""Pins of the oracle's 1D/3D operators and of the whole local-Hamiltonian
chain: dense brute force built from explicit index loops, orthogonality,
adjointness, energy identities, exact finite differences.  All CPU."""
import numpy as np
import pytest

import oracle.filters as F
import oracle.wavelet as W
import scaling_function as S

from paper_0904_1543_gb300 import inputs


# ----------------------------------------------------------- dense 1D matrices
def mat_synthesis(n_coarse):
    """s_i = sum_j h_{i-2j} c_j + g_{i-2j} d_j (mod N), interleaved input
    x[2j] = c_j, x[2j+1] = d_j: entry by entry from the definition."""
    h, g = F.h(), F.g()
    N = 2 * n_coarse
    A = np.zeros((N, N))
    for j in range(n_coarse):
        for t in range(16):
            k = F.J_LO + t
            A[(2 * j + k) % N, 2 * j] += h[t]
            A[(2 * j + k) % N, 2 * j + 1] += g[t]
    return A


def mat_conv(N, taps, shifts):
    """out(I) = sum_t taps[t] in(I - shifts[t]) (mod N)."""
    A = np.zeros((N, N))
    for I in range(N):
        for c, k in zip(taps, shifts):
            A[I, (I - k) % N] += c
    return A


def mat_mf(N):
    w, k0 = F.magic()
    return mat_conv(N, w, k0 + np.arange(16))


def mat_kin(N, hg):
    a = F.kinetic_a()
    return mat_conv(N, -a / (2 * hg * hg), np.arange(-14, 15))


def apply3(M1, M2, M3, X):
    """Dense Kronecker product applied to a C-ordered (N3, N2, N1) array."""
    K = np.kron(M3, np.kron(M2, M1))
    return (K @ X.reshape(-1)).reshape(X.shape)


GRIDS = [(1, 1, 1), (2, 3, 4), (4, 4, 4), (3, 5, 2)]


def rnd(shape, stream):
    return inputs.random_field(99, stream, shape)


@pytest.mark.parametrize("n", GRIDS)
def test_synthesis_analysis_bruteforce(n):
    n1, n2, n3 = n
    X = rnd((2 * n3, 2 * n2, 2 * n1), 1)
    A1, A2, A3 = mat_synthesis(n1), mat_synthesis(n2), mat_synthesis(n3)
    ref = apply3(A1, A2, A3, X)
    assert np.max(np.abs(W.synthesis3d(X) - ref)) < 1e-14
    ref_t = apply3(A1.T, A2.T, A3.T, X)
    assert np.max(np.abs(W.analysis3d(X) - ref_t)) < 1e-14


@pytest.mark.parametrize("n", GRIDS)
def test_mf_kinetic_bruteforce(n):
    n1, n2, n3 = n
    N1, N2, N3 = 2 * n1, 2 * n2, 2 * n3
    X = rnd((N3, N2, N1), 2)
    ref = apply3(mat_mf(N1), mat_mf(N2), mat_mf(N3), X)
    assert np.max(np.abs(W.magicfilter3d(X) - ref)) < 1e-14
    ref = apply3(mat_mf(N1).T, mat_mf(N2).T, mat_mf(N3).T, X)
    assert np.max(np.abs(W.magicfilter_T3d(X) - ref)) < 1e-14
    hg = (0.25, 0.3, 0.5)
    I1, I2, I3 = np.eye(N1), np.eye(N2), np.eye(N3)
    K = (np.kron(I3, np.kron(I2, mat_kin(N1, hg[0])))
         + np.kron(I3, np.kron(mat_kin(N2, hg[1]), I1))
         + np.kron(mat_kin(N3, hg[2]), np.kron(I2, I1)))
    ref = (K @ X.reshape(-1)).reshape(X.shape)
    got = W.kinetic3d(X, hg)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("nc", [1, 2, 3, 4, 8, 16])
def test_synthesis_orthogonal(nc):
    """Periodised fast wavelet transform is orthogonal at every size:
    analysis o synthesis = identity to 1e-14."""
    A = mat_synthesis(nc)
    assert np.max(np.abs(A.T @ A - np.eye(2 * nc))) < 1e-14


@pytest.mark.parametrize("n", [(8, 8, 8), (4, 6, 10), (16, 16, 16), (32, 32, 32)])
def test_analysis_inverts_synthesis(n):
    X = rnd((2 * n[2], 2 * n[1], 2 * n[0]), 3)
    assert np.max(np.abs(W.analysis3d(W.synthesis3d(X)) - X)) < 1e-14


def test_synthesis_matches_refinement_relation():
    """A coarse scaling function phi(x - j) written on the fine level by the
    synthesis equals sqrt2 sum_i s_i phi(2x - i) pointwise (cascade phi),
    i.e. the synthesis carries Eq. (refinement) with the right index sense.
    Same for a coarse wavelet."""
    h = F.h()
    L = 9
    x, p = S.phi_dyadic(h, L)
    nc = 16
    N = 2 * nc
    for comp in (0, 1):
        xin = np.zeros(N)
        xin[2 * 5 + comp] = 1.0                 # coarse j = 5
        s = W.synthesis_1d(xin, 0)
        # evaluate both sides at coarse-unit points t in [5-7, 5+8] (no wrap)
        ts = 5 + x[:: 2 ** 3]
        def phi_at(u):
            m = np.rint((u - x[0]) * 2 ** L).astype(int)
            ok = (m >= 0) & (m < p.size)
            out = np.zeros_like(u)
            out[ok] = p[m[ok]]
            return out
        lhs = sum(np.sqrt(2) * s[i] * phi_at(2 * ts - i) for i in range(N))
        if comp == 0:
            rhs = phi_at(ts - 5)
        else:
            g = F.g()
            rhs = sum(np.sqrt(2) * g[t] * phi_at(2 * (ts - 5) - (F.J_LO + t))
                      for t in range(16))
        assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_adjoint_pairs():
    n = (3, 4, 5)
    sh = (10, 8, 6)
    a, b = rnd(sh, 4), rnd(sh, 5)
    assert abs(np.vdot(W.magicfilter3d(a), b) - np.vdot(a, W.magicfilter_T3d(b))) < 1e-12
    assert abs(np.vdot(W.synthesis3d(a), b) - np.vdot(a, W.analysis3d(b))) < 1e-12
    k = W.kinetic3d(a)
    assert abs(np.vdot(k, b) - np.vdot(a, W.kinetic3d(b))) < 1e-10


def test_compress_roundtrip():
    n = (3, 4, 5)
    c = rnd((8 * 60,), 6)
    X = W.uncompress(c, n)
    assert np.array_equal(W.compress(X, n), c)
    # coarse scaling block lands on the all-even sites, mu = a1 + 2 a2 + 4 a3
    assert np.array_equal(X[0::2, 0::2, 0::2].reshape(-1), c[:60])
    fine = c[60:].reshape(5, 4, 3, 7)
    assert np.array_equal(X[1::2, 0::2, 1::2], fine[..., 5 - 1])   # mu = 1 + 4
    assert np.array_equal(X[0::2, 1::2, 0::2], fine[..., 2 - 1])   # mu = 2


# ------------------------------------------------------------ whole chain
def _case(n, norb=3, cfg=0):
    psi = inputs.orbitals(cfg, norb, n)
    V = inputs.gaussian_potential(cfg, 0, n)
    occ = np.full(norb, 2.0)
    return psi, V, occ


@pytest.mark.parametrize("n", [(4, 4, 4), (3, 5, 4)])
def test_hamiltonian_symmetric_and_energies(n):
    psi, V, occ = _case(n)
    hp, rho, ek, ep = W.hpsi_batch(psi, V, occ, n)
    # <a, H b> = <H a, b>
    assert abs(np.dot(psi[0], hp[1]) - np.dot(hp[0], psi[1])) < 1e-12 * np.abs(hp).max()
    for i in range(len(occ)):
        assert abs(np.dot(psi[i], hp[i]) - (ek[i] + ep[i])) < 1e-12 * abs(ek[i])
        assert ek[i] > 0
    # sum_I V rho = sum_i occ_i Epot_i
    assert abs(np.sum(V * rho) - np.sum(occ * ep)) < 1e-12 * abs(np.sum(occ * ep))
    assert np.all(rho >= 0)
    assert abs(rho.sum() - np.sum(occ * np.ones(3))) < 0.2 * rho.sum()


def test_hamiltonian_dense_bruteforce():
    """H = A^T (M^T V M + K) A with dense matrices on a 2x2x2 coarse cell."""
    n = (2, 2, 2)
    N = 4
    psi, V, occ = _case(n, norb=1)
    Sy = np.kron(mat_synthesis(2), np.kron(mat_synthesis(2), mat_synthesis(2)))
    Mf = np.kron(mat_mf(N), np.kron(mat_mf(N), mat_mf(N)))
    I = np.eye(N)
    Kx = mat_kin(N, 0.25)
    K = np.kron(I, np.kron(I, Kx)) + np.kron(I, np.kron(Kx, I)) + np.kron(Kx, np.kron(I, I))
    H = Sy.T @ (Mf.T @ np.diag(V.reshape(-1)) @ Mf + K) @ Sy
    X = W.uncompress(psi[0], n).reshape(-1)
    ref = W.compress((H @ X).reshape(N, N, N), n)
    got = W.hpsi_local(psi[0], V, 2.0, n)["hpsi_c"]
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()


def test_constant_potential_and_zero_potential():
    n = (3, 3, 4)
    psi, V, occ = _case(n, norb=1)
    r0 = W.hpsi_local(psi[0], np.zeros_like(V), 2.0, n)
    s = W.synthesis3d(W.uncompress(psi[0], n))
    kin = W.compress(W.analysis3d(W.kinetic3d(s)), n)
    assert np.max(np.abs(r0["hpsi_c"] - kin)) < 1e-12 * np.abs(kin).max()
    assert r0["epot"] == 0.0
    # constant V: H psi - K psi = V0 * A^T M^T M A psi, linear in V0
    r1 = W.hpsi_local(psi[0], np.full_like(V, -1.5), 2.0, n)
    r2 = W.hpsi_local(psi[0], np.full_like(V, -3.0), 2.0, n)
    d1, d2 = r1["hpsi_c"] - kin, r2["hpsi_c"] - kin
    assert np.max(np.abs(2 * d1 - d2)) < 1e-12
    # MF maps a constant field to the same constant (sum w = 1)
    one = np.ones((6, 6, 8))
    assert np.max(np.abs(W.magicfilter3d(one) - 1.0)) < 1e-14


def test_energy_gradient_exact_fd():
    """E is quadratic in psi and linear in V: central differences are exact
    up to rounding, which pins dE/dpsi = 2 occ H psi and dE/dV = rho."""
    n = (2, 3, 2)
    psi, V, occ = _case(n, norb=2)
    occ = np.array([2.0, 1.5])
    gpsi, gV = W.energy_gradients(psi, V, occ, n)
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = rng.standard_normal(psi.shape)
        e = 1e-5
        fd = (W.energy(psi + e * d, V, occ, n) - W.energy(psi - e * d, V, occ, n)) / (2 * e)
        assert abs(fd - np.sum(gpsi * d)) < 1e-7 * abs(fd)
        dv = rng.standard_normal(V.shape)
        fd = (W.energy(psi, V + e * dv, occ, n) - W.energy(psi, V - e * dv, occ, n)) / (2 * e)
        assert abs(fd - np.sum(gV * dv)) < 1e-7 * abs(fd)


def test_density_matches_hpsi_rho():
    n = (3, 2, 4)
    psi, V, occ = _case(n, norb=2)
    _, rho, _, _ = W.hpsi_batch(psi, V, occ, n)
    rho2 = sum(W.density(psi[i], occ[i], n) for i in range(2))
    assert np.max(np.abs(rho - rho2)) < 1e-15


def test_kinetic_plane_wave_3d():
    """On s = cos(kappa . I) the 3D kinetic operator multiplies by
    -1/2 sum_d a^(kappa_d) / h_d^2 (Eq. fprod is a sum of 1D symbols)."""
    N = (8, 12, 16)
    hg = (0.25, 0.4, 0.5)
    I3, I2, I1 = np.meshgrid(np.arange(N[2]), np.arange(N[1]), np.arange(N[0]), indexing="ij")
    kap = (2 * np.pi * 1 / N[0], 2 * np.pi * 2 / N[1], 2 * np.pi * 3 / N[2])
    s = np.cos(kap[0] * I1 + kap[1] * I2 + kap[2] * I3)
    a = F.kinetic_a()
    ls = np.arange(-14, 15)
    lam = sum(-0.5 * (a * np.cos(k * ls)).sum() / hh ** 2 for k, hh in zip(kap, hg))
    out = W.kinetic3d(s, hg)
    assert np.max(np.abs(out - lam * s)) < 1e-12 * abs(lam)
    # and the symbol is close to |kappa|^2/2 / h^2 for these smooth waves
    cont = sum(0.5 * k * k / hh ** 2 for k, hh in zip(kap, hg))
    assert abs(lam - cont) < 1e-3 * cont

"""Oracle operators for the local Hamiltonian in Daubechies wavelets, periodic BC.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

Plain FP64 numpy: every 1D convolution is the defining sum written as a loop
over taps of periodically shifted copies (np.roll), applied along x, then y,
then z.  Arrays are C-ordered (N3, N2, N1): numpy axis 2 is x (i1).

Conventions (readings stated once here):
* coarse grid n1 x n2 x n3, fine grid N_d = 2 n_d (Eq. wavefhigh, h' = h/2);
* interleaved coarse layout X[2 i3 + a3][2 i2 + a2][2 i1 + a1] = c^mu with
  mu = a1 + 2 a2 + 4 a3 (a_d = 0 scaling, 1 wavelet; Eq. wavef0);
* compressed layout (Sec. "Daubechies basis", compressed form): the scaling
  block c^0[i3][i2][i1] (n3 n2 n1 values) followed by the wavelet block
  c^mu[i3][i2][i1][mu-1], mu = 1..7 (7 n3 n2 n1 values);
* rho and Epot in grid units: rho_I = sum_i occ_i psi_r(I)^2,
  Epot_i = sum_I V_I psi_r,i(I)^2; kinetic -1/2 Laplacian with fine spacing
  h'_d per axis: T^(d)_l = -a_l / (2 h'_d^2).
"""
from __future__ import annotations

import numpy as np

from . import filters as F

AX = {1: 2, 2: 1, 3: 0}   # paper axis -> numpy axis


def _shift(x, k, axis):
    """y[i] = x[i - k] along axis (periodic)."""
    return np.roll(x, k, axis=axis)


# --------------------------------------------------------------------------
# compressed <-> interleaved (steps 1 and 7 of Sec. "Full local hamiltonian")
# --------------------------------------------------------------------------
def uncompress(psi_c, n):
    n1, n2, n3 = n
    m = n1 * n2 * n3
    psi_c = np.asarray(psi_c, dtype=np.float64)
    assert psi_c.size == 8 * m
    X = np.zeros((2 * n3, 2 * n2, 2 * n1))
    X[0::2, 0::2, 0::2] = psi_c[:m].reshape(n3, n2, n1)
    fine = psi_c[m:].reshape(n3, n2, n1, 7)
    for mu in range(1, 8):
        a1, a2, a3 = mu & 1, (mu >> 1) & 1, mu >> 2
        X[a3::2, a2::2, a1::2] = fine[..., mu - 1]
    return X


def compress(X, n):
    n1, n2, n3 = n
    m = n1 * n2 * n3
    out = np.empty(8 * m)
    out[:m] = X[0::2, 0::2, 0::2].reshape(-1)
    fine = np.empty((n3, n2, n1, 7))
    for mu in range(1, 8):
        a1, a2, a3 = mu & 1, (mu >> 1) & 1, mu >> 2
        fine[..., mu - 1] = X[a3::2, a2::2, a1::2]
    out[m:] = fine.reshape(-1)
    return out


# --------------------------------------------------------------------------
# 1D operators along one numpy axis
# --------------------------------------------------------------------------
def synthesis_1d(x, axis):
    """Fast wavelet synthesis (Eq. refinement): with c_j = x[2j], d_j = x[2j+1],
    s_i = sum_j h_{i-2j} c_j + g_{i-2j} d_j  (i mod N)."""
    h, g = F.h(), F.g()
    up_c = np.zeros_like(x)
    up_d = np.zeros_like(x)
    sl_e = [slice(None)] * x.ndim
    sl_o = [slice(None)] * x.ndim
    sl_e[axis] = slice(0, None, 2)
    sl_o[axis] = slice(1, None, 2)
    up_c[tuple(sl_e)] = x[tuple(sl_e)]          # c_j at position 2j
    up_d[tuple(sl_e)] = x[tuple(sl_o)]          # d_j at position 2j
    s = np.zeros_like(x)
    for t in range(F.NTAP):
        k = F.J_LO + t                          # s_i += h_k c_j, i = 2j + k
        s += h[t] * _shift(up_c, k, axis) + g[t] * _shift(up_d, k, axis)
    return s


def analysis_1d(s, axis):
    """Transpose of synthesis_1d: c_j = sum_i h_{i-2j} s_i,
    d_j = sum_i g_{i-2j} s_i, interleaved back as x[2j] = c_j, x[2j+1] = d_j."""
    h, g = F.h(), F.g()
    cf = np.zeros_like(s)
    df = np.zeros_like(s)
    for t in range(F.NTAP):
        k = F.J_LO + t                          # term s_{2j + k}
        sh = _shift(s, -k, axis)
        cf += h[t] * sh
        df += g[t] * sh
    x = np.empty_like(s)
    sl_e = [slice(None)] * s.ndim
    sl_o = [slice(None)] * s.ndim
    sl_e[axis] = slice(0, None, 2)
    sl_o[axis] = slice(1, None, 2)
    x[tuple(sl_e)] = cf[tuple(sl_e)]
    x[tuple(sl_o)] = df[tuple(sl_e)]
    return x


def magicfilter_1d(s, axis):
    """Eq. (3dconv) along one axis: psi_r(I) = sum_k w_k s(I - k)."""
    w, k0 = F.magic()
    out = np.zeros_like(s)
    for t in range(F.NTAP):
        out += w[t] * _shift(s, k0 + t, axis)
    return out


def magicfilter_T_1d(y, axis):
    """Transposed magic filter: y(J) = sum_k w_k y_r(J + k)."""
    w, k0 = F.magic()
    out = np.zeros_like(y)
    for t in range(F.NTAP):
        out += w[t] * _shift(y, -(k0 + t), axis)
    return out


def kinetic_1d(s, axis, hgrid):
    """One term of Eq. (fprod): -1/2 d^2/dx^2 in the fine scaling basis,
    out(I) = sum_l T_l s(I - l), T_l = -a_l / (2 h'^2)."""
    a = F.kinetic_a()
    out = np.zeros_like(s)
    for t in range(2 * F.KIN_HALF + 1):
        l = t - F.KIN_HALF
        out += (-a[t] / (2.0 * hgrid * hgrid)) * _shift(s, l, axis)
    return out


# --------------------------------------------------------------------------
# 3D operators (Eq. 3dconv: separable, applied along x, y, z)
# --------------------------------------------------------------------------
def _sep3(op, x):
    for d in (1, 2, 3):
        x = op(x, AX[d])
    return x


def synthesis3d(X):
    return _sep3(synthesis_1d, X)


def analysis3d(s):
    return _sep3(analysis_1d, s)


def magicfilter3d(s):
    return _sep3(magicfilter_1d, s)


def magicfilter_T3d(y):
    return _sep3(magicfilter_T_1d, y)


def kinetic3d(s, hgrid=(0.25, 0.25, 0.25)):
    """Eqs. (kiner)/(fprod): sum over the three axes of the 1D term."""
    out = np.zeros_like(s)
    for d in (1, 2, 3):
        out += kinetic_1d(s, AX[d], hgrid[d - 1])
    return out


# --------------------------------------------------------------------------
# full local Hamiltonian and density (Secs. "Full local hamiltonian",
# "Local density calculation")
# --------------------------------------------------------------------------
def hpsi_local(psi_c, V, occ, n, hgrid=(0.25, 0.25, 0.25)):
    """Steps 1)-7) for one orbital.  Returns a dict with hpsi_c, rho (this
    orbital's contribution occ |psi_r|^2), ekin, epot and the intermediates."""
    X = uncompress(psi_c, n)                   # 1) decompression
    s = synthesis3d(X)                         # 2) wavelet transformation
    psir = magicfilter3d(s)                    # 3a) magic filter
    vpsi = V * psir                            # 3b) potential multiplication
    y = magicfilter_T3d(vpsi)                  # 3c) transposed magic filter
    kin = kinetic3d(s, hgrid)                  # 4) kinetic from the output of 2)
    z = y + kin                                # 5) sum
    out = analysis3d(z)                        # 6) inverse wavelet transformation
    hpsi_c = compress(out, n)                  # 7) compression
    return {
        "hpsi_c": hpsi_c,
        "rho": occ * psir * psir,
        "epot": float(np.sum(V * psir * psir)),
        "ekin": float(np.sum(s * kin)),
        "s": s, "psir": psir, "y": y, "z": z,
    }


def density(psi_c, occ, n):
    """Eq. (density) in grid units via steps 1), 2), 3a) and the square."""
    s = synthesis3d(uncompress(psi_c, n))
    psir = magicfilter3d(s)
    return occ * psir * psir


def hpsi_batch(psi, V, occ, n, hgrid=(0.25, 0.25, 0.25)):
    """norb orbitals of one cell: psi (norb, 8 n1 n2 n3).  Returns hpsi,
    rho = sum_i occ_i |psi_r,i|^2, ekin[norb], epot[norb]."""
    psi = np.asarray(psi, dtype=np.float64).reshape(len(occ), -1)
    hp = np.empty_like(psi)
    rho = np.zeros((2 * n[2], 2 * n[1], 2 * n[0]))
    ek = np.empty(len(occ))
    ep = np.empty(len(occ))
    for i in range(len(occ)):
        r = hpsi_local(psi[i], V, occ[i], n, hgrid)
        hp[i] = r["hpsi_c"]
        rho += r["rho"]
        ek[i] = r["ekin"]
        ep[i] = r["epot"]
    return hp, rho, ek, ep


def energy(psi, V, occ, n, hgrid=(0.25, 0.25, 0.25)):
    """E_loc = sum_i occ_i (Ekin_i + Epot_i)."""
    _, _, ek, ep = hpsi_batch(psi, V, occ, n, hgrid)
    return float(np.sum(np.asarray(occ) * (ek + ep)))


def energy_gradients(psi, V, occ, n, hgrid=(0.25, 0.25, 0.25)):
    """dE/dpsi_i = 2 occ_i H psi_i (H symmetric), dE/dV = rho."""
    hp, rho, _, _ = hpsi_batch(psi, V, occ, n, hgrid)
    occ = np.asarray(occ, dtype=np.float64)
    return 2.0 * occ[:, None] * hp, rho


# --------------------------------------------------------------------------
# scalar products in compressed form
# --------------------------------------------------------------------------
def scalar_products(a, b):
    """S[i][j] = <a_i|b_j> = sum_k a_i[k] b_j[k] for compressed orbitals (rows
    of a and b).  The basis functions of Eq. (wavef0) are orthonormal (Sec.
    "Daubechies basis and wavelet transformation"), so the scalar product of
    two orbitals is the sum of the products of their coefficients.  Each sum
    is the correctly rounded sum (math.fsum) of the FP64 products, which are
    exact when the coefficients are FP32 values."""
    import math
    a = np.asarray(a, dtype=np.float64).reshape(len(a), -1)
    b = np.asarray(b, dtype=np.float64).reshape(len(b), -1)
    S = np.empty((a.shape[0], b.shape[0]))
    for i in range(a.shape[0]):
        for j in range(b.shape[0]):
            S[i, j] = math.fsum(a[i] * b[j])
    return S

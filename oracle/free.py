"""Oracle for isolated (free) boundary conditions: the convolutions of
Sec. "Wavelet transformation and Magic Filters convolutions" with the input
array taken as zero outside the simulation box instead of wrapped.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Reading: the orbital is expanded on the basis functions centred in the box
(coarse points 0..n-1 per axis) and every operator acts on the whole real
line, so the fine arrays grow beyond the box by the filter extents.  Here
each fine axis spans the index range [-E, 2n + E) with E = 40, enough to hold
every support of the chain, and each 1D operator is a dense non-circulant
(Toeplitz-band) matrix built entry by entry from its defining sum, applied
along x, y, z.  H = A^T (M^T V M + K) A with V given on that extended fine
grid.
"""
from __future__ import annotations

import numpy as np

from . import filters as F
from . import wavelet as W

E = 40


def fine_range(nc):
    return np.arange(-E, 2 * nc + E)


def mat_synthesis(nc):
    """(2 nc + 2E) x (2 nc): s_i = sum_j h_{i-2j} c_j + g_{i-2j} d_j, no wrap."""
    h, g = F.h(), F.g()
    I = fine_range(nc)
    A = np.zeros((I.size, 2 * nc))
    for r, i in enumerate(I):
        for j in range(nc):
            k = i - 2 * j
            if F.J_LO <= k <= F.J_HI:
                A[r, 2 * j] = h[k - F.J_LO]
                A[r, 2 * j + 1] = g[k - F.J_LO]
    return A


def mat_conv(nc, taps, shifts):
    """out(I) = sum_t taps[t] in(I - shifts[t]) on the extended range."""
    I = fine_range(nc)
    L = I.size
    A = np.zeros((L, L))
    for r in range(L):
        for c, k in zip(taps, shifts):
            q = r - k
            if 0 <= q < L:
                A[r, q] += c
    return A


def mat_mf(nc):
    w, k0 = F.magic()
    return mat_conv(nc, w, k0 + np.arange(16))


def mat_kin(nc, hg):
    a = F.kinetic_a()
    return mat_conv(nc, -a / (2 * hg * hg), np.arange(-14, 15))


def _apply(mats, X):
    """Separable application: mats = (M1, M2, M3) along x, y, z of a C-ordered
    (., ., .) array whose axes are (z, y, x)."""
    M1, M2, M3 = mats
    X = np.einsum("ai,kji->kja", M1, X)
    X = np.einsum("bj,kji->kbi", M2, X)
    X = np.einsum("ck,kji->cji", M3, X)
    return X


def hpsi_local(psi_c, V_ext, occ, n, hgrid=(0.25, 0.25, 0.25)):
    """Free-space local Hamiltonian of one orbital; V_ext and the returned
    rho live on the extended fine grid (2 n_d + 2E per axis, index -E first)."""
    X = W.uncompress(psi_c, n)
    S = [mat_synthesis(v) for v in n]
    Mf = [mat_mf(v) for v in n]
    s = _apply(S, X)
    psir = _apply(Mf, s)
    y = _apply([m.T for m in Mf], V_ext * psir)
    kin = np.zeros_like(s)
    for ax in range(3):
        mats = [np.eye(s.shape[2]), np.eye(s.shape[1]), np.eye(s.shape[0])]
        mats[ax] = mat_kin(n[ax], hgrid[ax])
        kin += _apply(mats, s)
    z = y + kin
    out = _apply([m.T for m in S], z)
    return {"hpsi_c": W.compress(out, n), "rho": occ * psir * psir,
            "epot": float(np.sum(V_ext * psir * psir)), "ekin": float(np.sum(s * kin))}


def extend(V_pad, n, pad_fine):
    """Place a potential given on the fine grid [-pad, 2n + pad) per axis into
    the oracle's extended grid (zero beyond)."""
    Vx = np.zeros(tuple(2 * v + 2 * E for v in (n[2], n[1], n[0])))
    o = E - pad_fine
    Vx[o:o + V_pad.shape[0], o:o + V_pad.shape[1], o:o + V_pad.shape[2]] = V_pad
    return Vx


def restrict(A_ext, pad_fine):
    """Inverse of extend for an extended-grid array."""
    o = E - pad_fine
    sz = [A_ext.shape[k] - 2 * o for k in range(3)]
    return A_ext[o:o + sz[0], o:o + sz[1], o:o + sz[2]]


# --------------------------------------------------------------------------
# mixed conditions: each axis periodic (circulant on 2n points) or free
# --------------------------------------------------------------------------
def mat_synthesis_periodic(nc):
    """(2 nc) x (2 nc): s_i = sum_j h_{i-2j} c_j + g_{i-2j} d_j, i mod 2 nc."""
    h, g = F.h(), F.g()
    N = 2 * nc
    A = np.zeros((N, N))
    for j in range(nc):
        for t in range(F.NTAP):
            k = F.J_LO + t
            A[(2 * j + k) % N, 2 * j] += h[t]
            A[(2 * j + k) % N, 2 * j + 1] += g[t]
    return A


def mat_conv_periodic(N, taps, shifts):
    A = np.zeros((N, N))
    for I in range(N):
        for c, k in zip(taps, shifts):
            A[I, (I - k) % N] += c
    return A


def _axis_mats(nc, free, hg):
    """(synthesis, magic filter, kinetic) matrices of one axis."""
    w, k0 = F.magic()
    a = F.kinetic_a()
    if free:
        return mat_synthesis(nc), mat_mf(nc), mat_kin(nc, hg)
    N = 2 * nc
    return (mat_synthesis_periodic(nc), mat_conv_periodic(N, w, k0 + np.arange(16)),
            mat_conv_periodic(N, -a / (2 * hg * hg), np.arange(-14, 15)))


def hpsi_local_bc(psi_c, V_ext, occ, n, free_axes, hgrid=(0.25, 0.25, 0.25)):
    """Local Hamiltonian with per-axis conditions (free_axes[d] = 1: free).
    V_ext and rho span [-E, 2n + E) along free axes, [0, 2n) along periodic
    ones."""
    X = W.uncompress(psi_c, n)
    M = [_axis_mats(n[d], free_axes[d], hgrid[d]) for d in range(3)]
    S = [m[0] for m in M]
    Mf = [m[1] for m in M]
    s = _apply(S, X)
    psir = _apply(Mf, s)
    y = _apply([m.T for m in Mf], V_ext * psir)
    kin = np.zeros_like(s)
    for ax in range(3):
        mats = [np.eye(s.shape[2]), np.eye(s.shape[1]), np.eye(s.shape[0])]
        mats[ax] = M[ax][2]
        kin += _apply(mats, s)
    out = _apply([m.T for m in S], y + kin)
    return {"hpsi_c": W.compress(out, n), "rho": occ * psir * psir,
            "epot": float(np.sum(V_ext * psir * psir)), "ekin": float(np.sum(s * kin))}


def extend_bc(V_pad, n, pad_fine, free_axes):
    """Potential on the padded cell (pad_fine fine points per side along free
    axes) -> the oracle's grid (extended by E along free axes)."""
    shp, sl = [], []
    for ax, d in enumerate((2, 1, 0)):
        if free_axes[d]:
            shp.append(2 * n[d] + 2 * E)
            o = E - pad_fine
            sl.append(slice(o, o + V_pad.shape[ax]))
        else:
            shp.append(2 * n[d])
            sl.append(slice(0, 2 * n[d]))
    Vx = np.zeros(shp)
    Vx[tuple(sl)] = V_pad
    return Vx


def restrict_bc(A_ext, n, pad_fine, free_axes):
    sl = []
    for ax, d in enumerate((2, 1, 0)):
        if free_axes[d]:
            o = E - pad_fine
            sl.append(slice(o, A_ext.shape[ax] - o))
        else:
            sl.append(slice(None))
    return A_ext[tuple(sl)]

"""Oracle for localisation regions: the compressed form of Sec. "Daubechies
basis and wavelet transformation", in which only the scaling coefficients of
a coarse region and the seven wavelet coefficients of a (generally smaller)
fine region are stored (Eq. wavef0: the sums run over the points of the low-
and high-resolution regions).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Layout (a reading; BigDFT's segment keys are not in the paper): the vector
holds c^0 at the coarse-region points in lexicographic order (i1 fastest),
then c^1..c^7 at the fine-region points in lexicographic order, the seven
components of a point together.  Coefficients outside the regions are zero.
"""
from __future__ import annotations

import numpy as np

from . import wavelet as W


def counts(coarse_mask, fine_mask):
    return int(np.count_nonzero(coarse_mask)), int(np.count_nonzero(fine_mask))


def uncompress(psi, n, coarse_mask, fine_mask):
    """Region-compressed coefficients -> interleaved coarse layout (zeros off
    the regions).  Masks are (n3, n2, n1) booleans."""
    n1, n2, n3 = n
    nc, nf = counts(coarse_mask, fine_mask)
    psi = np.asarray(psi, dtype=np.float64)
    assert psi.size == nc + 7 * nf
    X = np.zeros((2 * n3, 2 * n2, 2 * n1))
    c0 = np.zeros((n3, n2, n1))
    c0[coarse_mask] = psi[:nc]
    X[0::2, 0::2, 0::2] = c0
    fine = np.zeros((n3, n2, n1, 7))
    fine[fine_mask] = psi[nc:].reshape(nf, 7)
    for mu in range(1, 8):
        a1, a2, a3 = mu & 1, (mu >> 1) & 1, mu >> 2
        X[a3::2, a2::2, a1::2] = fine[..., mu - 1]
    return X


def compress(X, n, coarse_mask, fine_mask):
    n1, n2, n3 = n
    c0 = X[0::2, 0::2, 0::2]
    fine = np.empty((n3, n2, n1, 7))
    for mu in range(1, 8):
        a1, a2, a3 = mu & 1, (mu >> 1) & 1, mu >> 2
        fine[..., mu - 1] = X[a3::2, a2::2, a1::2]
    return np.concatenate([c0[coarse_mask], fine[fine_mask].reshape(-1)])


def hpsi_local(psi, V, occ, n, coarse_mask, fine_mask, hgrid=(0.25, 0.25, 0.25)):
    """The local Hamiltonian restricted to the regions: compress_R H uncompress_R."""
    X = uncompress(psi, n, coarse_mask, fine_mask)
    s = W.synthesis3d(X)
    psir = W.magicfilter3d(s)
    y = W.magicfilter_T3d(V * psir)
    kin = W.kinetic3d(s, hgrid)
    out = W.analysis3d(y + kin)
    return {"hpsi_c": compress(out, n, coarse_mask, fine_mask),
            "rho": occ * psir * psir,
            "epot": float(np.sum(V * psir * psir)),
            "ekin": float(np.sum(s * kin))}


def sphere_masks(n, centre, r_coarse, r_fine):
    """Coarse / fine regions as balls (minimum-image distance, in coarse grid
    units) around a centre: the usual shape of a localised orbital's support."""
    idx = np.meshgrid(*[np.arange(v) for v in (n[2], n[1], n[0])], indexing="ij")
    d2 = np.zeros(idx[0].shape)
    for ax, (v, c) in enumerate(zip((n[2], n[1], n[0]), (centre[2], centre[1], centre[0]))):
        x = idx[ax] - c
        x = x - v * np.round(x / v)
        d2 += x * x
    return d2 <= r_coarse ** 2, d2 <= r_fine ** 2

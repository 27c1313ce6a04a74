"""Independent constructions of the scaling function used to pin the oracle.

Nothing here reuses the oracle's derivation: phi is built either pointwise by
the cascade algorithm from Eq. (refinement), or in Fourier space as the
infinite product of the refinement symbol.  Only the filter h is taken as
input.
"""
import numpy as np

J_LO, J_HI = -7, 8


def phi_integers(h):
    """phi(k), k = -7..8: the eigenvector (eigenvalue 1) of
    phi(k) = sqrt2 sum_j h_j phi(2k - j), normalised to sum_k phi(k) = 1."""
    ks = np.arange(J_LO, J_HI + 1)
    A = np.zeros((ks.size, ks.size))
    for a, k in enumerate(ks):
        for b, l in enumerate(ks):
            j = 2 * k - l
            if J_LO <= j <= J_HI:
                A[a, b] = np.sqrt(2.0) * h[j - J_LO]
    w, v = np.linalg.eig(A)
    i = np.argmin(np.abs(w - 1.0))
    phi = np.real(v[:, i])
    return ks, phi / phi.sum()


def phi_dyadic(h, level):
    """(x, phi(x)) on x = -7 + m / 2^level, m = 0 .. 15 * 2^level."""
    ks, vals = phi_integers(h)
    for L in range(1, level + 1):
        npt = (J_HI - J_LO) * 2 ** L + 1
        m = np.arange(npt)
        out = np.zeros(npt)
        for t in range(h.size):
            j = J_LO + t
            mp = m + (J_LO - j) * 2 ** (L - 1)      # index of 2x - j one level up
            ok = (mp >= 0) & (mp < vals.size)
            out[ok] += np.sqrt(2.0) * h[t] * vals[mp[ok]]
        vals = out
    x = J_LO + np.arange(vals.size) / 2.0 ** level
    return x, vals


def project(h, f, j, level=13):
    """int f(x) phi(x - j) dx by the trapezoid rule on the cascade grid."""
    x, p = phi_dyadic(h, level)
    dx = 1.0 / 2 ** level
    return np.array([np.sum(f(x + jj) * p) * dx for jj in np.atleast_1d(j)])


def phi_hat(h, xi, nprod=64):
    """phi^(xi) = int phi(x) e^{-i xi x} dx = prod_{l>=1} m0(xi / 2^l),
    m0(xi) = 2^{-1/2} sum_j h_j e^{-i j xi}."""
    xi = np.asarray(xi, dtype=np.float64)
    js = np.arange(J_LO, J_HI + 1)
    out = np.ones(xi.shape, dtype=np.complex128)
    for l in range(1, nprod + 1):
        z = xi[..., None] / 2.0 ** l
        out *= (h * np.exp(-1j * js * z)).sum(-1) / np.sqrt(2.0)
    return out

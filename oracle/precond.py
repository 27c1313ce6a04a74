"""Oracle for the preconditioning step: the Helmholtz equation of Eq. (precon),
(-1/2 Lap - eps) g~ = g, solved for each orbital by a preconditioned conjugate
gradient in the wavelet basis.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings (the paper names the equation and the method, not their details):
* the operator acts on compressed coefficients: A = S^T (K - eps) S with S the
  synthesis and K the kinetic operator of Eqs. (kiner)/(fprod), i.e. the
  kinetic convolution run with K_0 = -eps s (Sec. "Kinetic convolution");
  S is orthogonal, so A = S^T K S - eps;
* the preconditioner of the conjugate gradient is the diagonal of A, which by
  translation invariance depends only on the component mu of a coefficient;
* x_0 = 0 and a fixed number of iterations (the paper's loop count is not
  printed; the API takes it as an argument);
* eps < 0 (orbital energies of bound states), so A is positive definite.
"""
from __future__ import annotations

import numpy as np

from . import wavelet as W


def helmholtz_apply(c, eps, n, hgrid=(0.25, 0.25, 0.25)):
    """A c = S^T (K s - eps s), s = S c."""
    s = W.synthesis3d(W.uncompress(c, n))
    return W.compress(W.analysis3d(W.kinetic3d(s, hgrid) - eps * s), n)


def component_index(n, mu):
    """Compressed position of component mu of the coarse point (0, 0, 0)."""
    m = n[0] * n[1] * n[2]
    return 0 if mu == 0 else m + mu - 1


def helmholtz_diagonal(n, hgrid=(0.25, 0.25, 0.25)):
    """d[mu] = (S^T K S) at (point 0, component mu), from the operator
    applied to unit vectors."""
    m = n[0] * n[1] * n[2]
    d = np.zeros(8)
    for mu in range(8):
        e = np.zeros(8 * m)
        k = component_index(n, mu)
        e[k] = 1.0
        d[mu] = helmholtz_apply(e, 0.0, n, hgrid)[k]
    return d


def component_of(n):
    """mu of every compressed position."""
    m = n[0] * n[1] * n[2]
    mu = np.zeros(8 * m, dtype=np.int64)
    mu[m:] = np.tile(np.arange(1, 8), m)
    return mu


def precondition(g, eps, n, ncg, hgrid=(0.25, 0.25, 0.25), return_history=False):
    """ncg iterations of preconditioned CG for A x = g from x_0 = 0, with the
    preconditioner M = diag(A) (per component).  Returns x (and the iterates)."""
    g = np.asarray(g, dtype=np.float64)
    Minv = 1.0 / (helmholtz_diagonal(n, hgrid)[component_of(n)] - eps)
    x = np.zeros_like(g)
    r = g.copy()
    z = Minv * r
    p = z.copy()
    rz = float(np.dot(r, z))
    hist = [x.copy()]
    for _ in range(ncg):
        q = helmholtz_apply(p, eps, n, hgrid)
        alpha = rz / float(np.dot(p, q))
        x = x + alpha * p
        r = r - alpha * q
        z = Minv * r
        rz_new = float(np.dot(r, z))
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
        hist.append(x.copy())
    return (x, hist) if return_history else x


def precondition_batch(G, eps, n, ncg, hgrid=(0.25, 0.25, 0.25)):
    G = np.asarray(G, dtype=np.float64).reshape(len(eps), -1)
    return np.stack([precondition(G[i], eps[i], n, ncg, hgrid) for i in range(len(eps))])

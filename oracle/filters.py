"""Oracle filter derivation: Daubechies-16 refinement filters h, g, magic filter
omega and the kinetic (second-derivative) filter a.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

The paper prints none of these coefficients, so they are derived here from
their defining properties, in high precision (stdlib ``decimal``, 80 digits),
then rounded once to FP64.

Readings (the paper is silent or garbled on these points):

* Eq. (refinement) of Sec. "Daubechies basis and wavelet transformation" sums
  j = 1-m .. m with m the family order, and Sec. "Wavelet transformation and
  Magic Filters convolutions" says the order is 16.  Taken together with the
  16-tap magic filter this is read as a 16-tap filter (M = 8 vanishing
  moments) with support j = -7 .. 8.
* The family member is the least-asymmetric one: among the 2^4 spectral
  factors, the one whose non-trivial factor Q has the unwrapped phase closest
  to linear (max deviation from the least-squares line over 4095 interior
  points of (0, pi)).  Mirror images tie exactly; the one whose energy centre
  sum_j j h_j^2 is >= 1/2 is kept.
* g_j = (-1)^j h_{1-j}, exactly as printed after Eq. (refinement).
* Magic filter, Eq. (magicfilter) and Eq. (3dconv): psi_r(I) = sum_k w_k s(I-k)
  over a 16-point window k = k0 .. k0+15.  The taps are fixed by exact
  reproduction of point values of polynomials of degree < 16 (the O(h^16)
  statement of Sec. "Application of the local potential"):
  sum_k w_k int (y-k)^p phi(y) dy = delta_{p0}.  The window is centred on the
  first moment of phi: k0 = round(M_1 - 7.5).
* Kinetic filter, Eqs. (kiner)/(fprod): a_l = int phi(x) phi''(x-l) dx for
  |l| <= 14 (29 taps), obtained as the null vector of the refinement relation
  a_l = 4 sum_{i,j} h_i h_j a_{2l+j-i} normalised by sum_l l^2 a_l = 2.
"""
from __future__ import annotations

import functools
import math
from decimal import Decimal, localcontext

import numpy as np

M_VANISH = 8          # vanishing moments of the wavelet
NTAP = 2 * M_VANISH   # 16 refinement taps
J_LO = 1 - M_VANISH   # support of h: j = -7 .. 8
J_HI = M_VANISH
KIN_HALF = NTAP - 2   # a_l nonzero for |l| <= 14
PREC = 80             # decimal digits used throughout the derivation


# --------------------------------------------------------------------------
# minimal complex arithmetic on pairs of Decimals
# --------------------------------------------------------------------------
def _cadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def _csub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def _cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def _cdiv(a, b):
    d = b[0] * b[0] + b[1] * b[1]
    return ((a[0] * b[0] + a[1] * b[1]) / d, (a[1] * b[0] - a[0] * b[1]) / d)


def _cabs2(a):
    return a[0] * a[0] + a[1] * a[1]


def _csqrt(a):
    """Principal square root."""
    r = _cabs2(a).sqrt()
    re = ((r + a[0]) / 2).sqrt()
    im = ((r - a[0]) / 2).sqrt()
    if a[1] < 0:
        im = -im
    return (re, im)


def _D(x) -> Decimal:
    return Decimal(repr(float(x))) if not isinstance(x, Decimal) else x


# --------------------------------------------------------------------------
# 1. refinement filter h (Eq. refinement)
# --------------------------------------------------------------------------
def daubechies_P_coeffs():
    """Coefficients of P(y) = sum_{k<M} C(M-1+k, k) y^k (ascending), the
    polynomial with |m0(xi)|^2 = cos^{2M}(xi/2) P(sin^2(xi/2))."""
    return [math.comb(M_VANISH - 1 + k, k) for k in range(M_VANISH)]


def _P_roots():
    """Roots of P, polished by Newton's method in PREC-digit arithmetic.
    Returns (real_roots, complex_roots_with_positive_imag)."""
    c = daubechies_P_coeffs()
    approx = np.roots(c[::-1])
    cD = [Decimal(v) for v in c]

    def P_and_dP(y):
        p = (Decimal(0), Decimal(0))
        dp = (Decimal(0), Decimal(0))
        for a in reversed(cD):          # Horner
            dp = _cadd(_cmul(dp, y), p)
            p = _cadd(_cmul(p, y), (a, Decimal(0)))
        return p, dp

    reals, cplx = [], []
    for r in approx:
        if abs(r.imag) < 1e-8:
            y = (_D(r.real), Decimal(0))
        elif r.imag > 0:
            y = (_D(r.real), _D(r.imag))
        else:
            continue
        for _ in range(12):
            p, dp = P_and_dP(y)
            y = _csub(y, _cdiv(p, dp))
            if y[1] != 0 and abs(r.imag) < 1e-8:
                y = (y[0], Decimal(0))
        (reals if abs(r.imag) < 1e-8 else cplx).append(y)
    reals.sort(key=lambda v: v[0])
    cplx.sort(key=lambda v: (v[0], v[1]))
    return reals, cplx


def _z_pair(y):
    """The two z with (2 - z - 1/z)/4 = y, i.e. z^2 - 2(1-2y) z + 1 = 0.
    Returned as (inside, outside) the unit circle."""
    w = (1 - 2 * y[0], -2 * y[1])
    d = _csqrt(_csub(_cmul(w, w), (Decimal(1), Decimal(0))))
    z1, z2 = _cadd(w, d), _csub(w, d)
    return (z1, z2) if _cabs2(z1) < _cabs2(z2) else (z2, z1)


def _poly_from_roots(roots):
    """Ascending coefficients of prod_k (z - z_k), complex Decimal pairs."""
    coef = [(Decimal(1), Decimal(0))]
    for zk in roots:
        new = [(Decimal(0), Decimal(0))] * (len(coef) + 1)
        for i, ci in enumerate(coef):
            new[i + 1] = _cadd(new[i + 1], ci)
            new[i] = _csub(new[i], _cmul(ci, zk))
        coef = new
    return coef


def _candidate(choice, reals, cplx):
    """Filter for one root choice (tuple of 0/1 per root group: 0 = inside).
    Returns (h as list of Decimal for j=-7..8, Q ascending real coeffs)."""
    roots = []
    groups = [(y, False) for y in reals] + [(y, True) for y in cplx]
    for bit, (y, is_c) in zip(choice, groups):
        z = _z_pair(y)[bit]
        roots.append(z)
        if is_c:
            roots.append((z[0], -z[1]))
    q = _poly_from_roots(roots)
    assert all(abs(v[1]) < Decimal(10) ** (-PREC // 2) for v in q)
    q = [v[0] for v in q]
    # H(z) = (1 + z)^M Q(z)
    hz = [Decimal(0)] * (len(q) + M_VANISH)
    for i, qi in enumerate(q):
        for k in range(M_VANISH + 1):
            hz[i + k] += qi * math.comb(M_VANISH, k)
    scale = Decimal(2).sqrt() / sum(hz)        # sum_j h_j = sqrt(2)
    h = [v * scale for v in hz]
    assert len(h) == NTAP
    return h, q


def _phase_nonlinearity(q):
    """Max deviation of the unwrapped phase of Q(e^{-i xi}) from its
    least-squares line over xi = pi k / 4096, k = 1..4095."""
    xi = np.pi * np.arange(1, 4096) / 4096.0
    z = np.exp(-1j * xi)
    qd = np.array([float(v) for v in q])
    val = np.polyval(qd[::-1], z)
    th = np.unwrap(np.angle(val))
    A = np.stack([xi, np.ones_like(xi)], axis=1)
    coef, *_ = np.linalg.lstsq(A, th, rcond=None)
    return float(np.max(np.abs(th - A @ coef)))


def _energy_centre(h):
    return sum((J_LO + i) * float(v) ** 2 for i, v in enumerate(h))


@functools.lru_cache(maxsize=None)
def _derive():
    with localcontext() as ctx:
        ctx.prec = PREC
        reals, cplx = _P_roots()
        ngrp = len(reals) + len(cplx)
        cands = []
        for bits in range(1 << ngrp):
            choice = tuple((bits >> k) & 1 for k in range(ngrp))
            h, q = _candidate(choice, reals, cplx)
            cands.append((choice, h, q, _phase_nonlinearity(q)))
        best = min(cands, key=lambda c: c[3])
        mirror_choice = tuple(1 - b for b in best[0])
        mirror = next(c for c in cands if c[0] == mirror_choice)
        pick = best if _energy_centre(best[1]) >= 0.5 else mirror
        hD = pick[1]

        # g_j = (-1)^j h_{1-j}
        gD = []
        for j in range(J_LO, J_HI + 1):
            gD.append((-1) ** (j % 2) * hD[(1 - j) - J_LO])

        mom = _moments(hD, NTAP)
        k0 = int(round(float(mom[1]) - 7.5))
        wD = _magic(mom, k0)
        aD = _kinetic(hD)
        return {
            "hD": hD, "gD": gD, "wD": wD, "aD": aD, "momD": mom,
            "k0": k0, "cands": [(c[0], c[3]) for c in cands],
            "cand_h": [(c[0], [float(v) for v in c[1]]) for c in cands],
            "choice": pick[0],
        }


# --------------------------------------------------------------------------
# 2. moments of phi, from the refinement relation
# --------------------------------------------------------------------------
def _moments(hD, pmax):
    """M_p = int x^p phi(x) dx, p < pmax.  Integrating Eq. (refinement):
    M_p (1 - 2^-p) = 2^(-p-1/2) sum_j h_j sum_{q<p} C(p,q) j^(p-q) M_q."""
    M = [Decimal(1)]
    r2 = Decimal(2).sqrt()
    for p in range(1, pmax):
        acc = Decimal(0)
        for i, hj in enumerate(hD):
            j = J_LO + i
            inner = Decimal(0)
            for q in range(p):
                inner += math.comb(p, q) * Decimal(j ** (p - q)) * M[q]
            acc += hj * inner
        fac = 1 / (Decimal(2) ** p * r2)
        M.append(acc * fac / (1 - 1 / Decimal(2) ** p))
    return M


def _solve(A, b):
    """Gaussian elimination with partial pivoting (Decimal)."""
    n = len(A)
    A = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(A[r][col]))
        A[col], A[piv] = A[piv], A[col]
        for r in range(col + 1, n):
            f = A[r][col] / A[col][col]
            if f != 0:
                for c in range(col, n + 1):
                    A[r][c] -= f * A[col][c]
    x = [Decimal(0)] * n
    for r in range(n - 1, -1, -1):
        s = A[r][n] - sum(A[r][c] * x[c] for c in range(r + 1, n))
        x[r] = s / A[r][r]
    return x


# --------------------------------------------------------------------------
# 3. magic filter (Eq. magicfilter)
# --------------------------------------------------------------------------
def _magic(mom, k0):
    """sum_k w_k int (y-k)^p phi(y) dy = delta_{p0}, p = 0..15."""
    ks = list(range(k0, k0 + NTAP))
    A = []
    for p in range(NTAP):
        row = []
        for k in ks:
            v = Decimal(0)
            for q in range(p + 1):
                v += math.comb(p, q) * Decimal((-k) ** (p - q)) * mom[q]
            row.append(v)
        A.append(row)
    b = [Decimal(1)] + [Decimal(0)] * (NTAP - 1)
    return _solve(A, b)


# --------------------------------------------------------------------------
# 4. kinetic filter (Eqs. kiner, fprod)
# --------------------------------------------------------------------------
def autocorrelation(hD):
    """r(k) = sum_i h_i h_{i+k}, k = -(NTAP-1) .. NTAP-1 (dict)."""
    r = {}
    for k in range(-(NTAP - 1), NTAP):
        s = Decimal(0)
        for i in range(NTAP):
            if 0 <= i + k < NTAP:
                s += hD[i] * hD[i + k]
        r[k] = s
    return r


def kinetic_system(hD):
    """Rows of (I - 4R) a = 0 for l = -14..14, R_{l,m} = r(m - 2l)."""
    r = autocorrelation(hD)
    ls = list(range(-KIN_HALF, KIN_HALF + 1))
    rows = []
    for l in ls:
        row = []
        for m in ls:
            v = -4 * r.get(m - 2 * l, Decimal(0))
            if m == l:
                v += 1
            row.append(v)
        rows.append(row)
    return rows


def _kinetic(hD):
    """The 29 homogeneous rows plus the normalisation row sum_l l^2 a_l = 2
    form a consistent overdetermined system; it is solved through its normal
    equations (no row has to be chosen for removal)."""
    rows = kinetic_system(hD)
    ls = list(range(-KIN_HALF, KIN_HALF + 1))
    A = [r[:] for r in rows] + [[Decimal(l * l) for l in ls]]
    b = [Decimal(0)] * len(rows) + [Decimal(2)]
    n = len(ls)
    AtA = [[sum(A[k][i] * A[k][j] for k in range(len(A))) for j in range(n)]
           for i in range(n)]
    Atb = [sum(A[k][i] * b[k] for k in range(len(A))) for i in range(n)]
    return _solve(AtA, Atb)


# --------------------------------------------------------------------------
# public accessors (FP64)
# --------------------------------------------------------------------------
def _f64(v):
    return np.array([float(x) for x in v], dtype=np.float64)


def h():
    """h_j, j = -7..8 (index j + 7)."""
    return _f64(_derive()["hD"])


def g():
    """g_j = (-1)^j h_{1-j}, j = -7..8 (index j + 7)."""
    return _f64(_derive()["gD"])


def magic():
    """(omega, k0): omega[t] = w_{k0 + t}, t = 0..15."""
    d = _derive()
    return _f64(d["wD"]), d["k0"]


def kinetic_a():
    """a_l = int phi(x) phi''(x - l) dx, l = -14..14 (index l + 14)."""
    return _f64(_derive()["aD"])


def moments():
    return _f64(_derive()["momD"])


def high_precision():
    """The Decimal values behind the FP64 tables (for tests)."""
    d = _derive()
    return {k: d[k] for k in ("hD", "gD", "wD", "aD", "momD", "k0")}


def candidates():
    """[(root choice, phase nonlinearity)] for all 16 spectral factors, and
    the chosen one."""
    d = _derive()
    return d["cands"], d["choice"]


def candidate_filters():
    """[(root choice, h rounded to FP64 for j = -7..8)] for all 16 spectral
    factors, in the order of candidates()."""
    return [(c, np.array(hv)) for c, hv in _derive()["cand_h"]]

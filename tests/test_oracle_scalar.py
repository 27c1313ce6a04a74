"""Pins of the oracle's compressed-form scalar products (CPU).

<a|b> on compressed coefficients must equal (1) the exact rational sum of
the products, rounded once, and (2) the scalar product of the fine-grid
scaling coefficients the orbitals synthesise to: the one-level transform of
Eq. (refinement) is orthogonal, so the compressed coefficients and the fine
scaling coefficients are two orthonormal bases of the same space (Sec.
"Daubechies basis and wavelet transformation")."""
from fractions import Fraction

import numpy as np

import oracle.wavelet as O
from paper_0904_1543_gb300 import inputs


def test_scalar_products_exact_rational():
    """FP32 coefficients: every product is exact in FP64 and the sum is
    rounded once, so the result equals the exact rational sum rounded to the
    nearest double."""
    n = (3, 2, 2)
    a = inputs.orbitals(71, 3, n).astype(np.float32)
    b = inputs.orbitals(72, 2, n).astype(np.float32)
    S = O.scalar_products(a, b)
    for i in range(3):
        for j in range(2):
            exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a[i], b[j]))
            assert S[i, j] == float(exact), (i, j)


def test_scalar_products_parseval_through_synthesis():
    """<a|b> in compressed form = sum over the fine grid of S a times S b,
    with S the oracle's synthesis (an independent code path), on ragged
    grids; unit-norm orbitals have <a|a> = 1."""
    for n in ((4, 3, 5), (6, 6, 2)):
        a = inputs.orbitals(73, 3, n)
        S = O.scalar_products(a, a)
        fine = [O.synthesis3d(O.uncompress(x, n)) for x in a]
        for i in range(3):
            assert abs(S[i, i] - 1.0) < 1e-14
            for j in range(3):
                ref = float(np.sum(fine[i] * fine[j]))
                assert abs(S[i, j] - ref) < 1e-14, (n, i, j, S[i, j], ref)


def test_scalar_products_detect_a_transposed_or_dropped_term():
    """The pins are sharp: a mistaken index (b_j against a_j) or a dropped
    component block changes the result far beyond rounding."""
    n = (4, 4, 4)
    a = inputs.orbitals(74, 2, n)
    b = inputs.orbitals(75, 2, n)
    S = O.scalar_products(a, b)
    wrong = np.array([[np.dot(b[i], b[j]) for j in range(2)] for i in range(2)])
    assert np.abs(S - wrong).max() > 1e-3
    m = n[0] * n[1] * n[2]
    dropped = np.array([[np.dot(a[i][m:], b[j][m:]) for j in range(2)] for i in range(2)])
    assert np.abs(S - dropped).max() > 1e-4

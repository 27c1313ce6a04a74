"""GPU parity of the compressed-form scalar products (wvl_overlap, wvl_dot)
against the oracle's correctly rounded sums.

Products are formed and accumulated in FP64 whatever the coefficients'
precision, so FP64 and FP32 inputs are held to the same bound: |S - S_ref| <=
1e-13 sqrt(<a_i|a_i> <b_j|b_j>) (Cauchy-Schwarz scale; rounding of an FP64 sum
of len products leaves about len^(1/2) 1e-16 of it).  Sizes span several
32 x 32 tiles with ragged edges, lengths that are not multiples of the
64-coefficient stage, and the symmetric path (a is b)."""
import numpy as np
import pytest

import oracle.wavelet as O
from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    return W


def _check(S, a, b, rows=None, cols=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    rows = range(a.shape[0]) if rows is None else rows
    cols = range(b.shape[0]) if cols is None else cols
    ref = O.scalar_products(a[list(rows)], b[list(cols)])
    na = np.sqrt((a[list(rows)] ** 2).sum(1))
    nb = np.sqrt((b[list(cols)] ** 2).sum(1))
    got = S[np.ix_(list(rows), list(cols))]
    bound = 1e-13 * np.outer(na, nb)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / np.outer(na, nb))


@pytest.mark.parametrize("dt", ["float64", "float32"])
@pytest.mark.parametrize("na,nb,n", [(37, 45, (5, 4, 3)), (1, 1, (2, 2, 2)), (64, 33, (6, 7, 5))])
def test_overlap_matches_oracle(W, dt, na, nb, n):
    import torch
    a = inputs.orbitals(81, na, n).astype(dt)
    b = inputs.orbitals(82, nb, n).astype(dt)
    S = W.overlap(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    _check(S, a, b)


@pytest.mark.parametrize("dt", ["float64", "float32"])
def test_overlap_symmetric_and_deterministic(W, dt):
    """a is b: only the upper block triangle is computed; the result is
    exactly symmetric, has unit diagonal for unit-norm orbitals, matches the
    oracle, and repeats bit for bit."""
    import torch
    n = (6, 5, 4)
    a = inputs.orbitals(83, 70, n).astype(dt)
    ta = torch.from_numpy(a).cuda()
    S1 = W.overlap(ta).cpu().numpy()
    S2 = W.overlap(ta).cpu().numpy()
    assert np.array_equal(S1, S2)
    assert np.array_equal(S1, S1.T)
    _check(S1, a, a)
    if dt == "float64":
        assert np.abs(np.diag(S1) - 1.0).max() < 1e-13


def test_overlap_large_sampled(W):
    """256 FP32 orbitals at coarse 24^3 (8 x 24^3 = 110,592 coefficients),
    the symmetric path, sampled rows and columns against the oracle."""
    import torch
    n = (24, 24, 24)
    ta = inputs.orbitals_device(84, 256, n, torch.device("cuda"), torch.float32)
    S = W.overlap(ta).cpu().numpy()
    a = ta.cpu().numpy()
    rng = np.random.default_rng(84)
    rows = sorted(rng.choice(256, 6, replace=False).tolist())
    cols = sorted(rng.choice(256, 6, replace=False).tolist())
    _check(S, a, a, rows, cols)
    assert np.array_equal(S, S.T)


@pytest.mark.parametrize("dt", ["float64", "float32"])
def test_dot_matches_oracle(W, dt):
    """Per-orbital <a_o|b_o> over a length that is no multiple of anything
    (a region-compressed length)."""
    import torch
    rng = np.random.default_rng(85)
    a = rng.uniform(-1, 1, (9, 10007)).astype(dt)
    b = rng.uniform(-1, 1, (9, 10007)).astype(dt)
    d = W.dot(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    for o in range(9):
        ref = O.scalar_products(a[o:o + 1], b[o:o + 1])[0, 0]
        scale = np.sqrt(np.sum(a[o].astype(np.float64) ** 2) * np.sum(b[o].astype(np.float64) ** 2))
        assert abs(d[o] - ref) <= 1e-13 * scale


def test_scalar_products_reject_bad_arguments(W):
    import ctypes
    L = W.lib()
    S = ctypes.c_double(0.0)
    assert L.wvl_overlap(0, 2, None, 2, None, 10, ctypes.addressof(S), None, 0, None) == 1
    assert b"NULL" in L.wvl_last_error()
    assert L.wvl_overlap(7, 2, None, 2, None, 10, None, None, 0, None) == 1

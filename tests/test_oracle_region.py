"""Pins of the localisation-region oracle: region compress/uncompress are a
selection (compress o uncompress = identity, uncompress o compress = the
projection), the full region reproduces the full-grid operator, and the
restricted Hamiltonian is P H P^T with H the dense brute-force matrix."""
import numpy as np
import pytest

import oracle.region as RG
import oracle.wavelet as W
from paper_0904_1543_gb300 import inputs
from test_oracle_ops import mat_kin, mat_mf, mat_synthesis


def test_roundtrip_and_projection():
    n = (5, 4, 6)
    cm, fm = RG.sphere_masks(n, (2, 1, 3), 2.2, 1.3)
    nc, nf = RG.counts(cm, fm)
    assert 0 < nf < nc < 120
    c = inputs.random_field(81, 1, (nc + 7 * nf,))
    X = RG.uncompress(c, n, cm, fm)
    assert np.array_equal(RG.compress(X, n, cm, fm), c)
    # off-region coefficients are zero
    full = W.compress(X, n)
    m = 120
    assert np.all(full[:m].reshape(6, 4, 5)[~cm] == 0)
    assert np.all(full[m:].reshape(6, 4, 5, 7)[~fm] == 0)


def test_full_region_equals_full_grid():
    n = (4, 3, 5)
    cm = np.ones((5, 3, 4), dtype=bool)
    psi = inputs.orbital(82, 0, n)
    V = inputs.gaussian_potential(82, 0, n)
    a = RG.hpsi_local(psi, V, 2.0, n, cm, cm)
    b = W.hpsi_local(psi, V, 2.0, n)
    assert np.array_equal(a["hpsi_c"], b["hpsi_c"])
    assert a["ekin"] == b["ekin"] and a["epot"] == b["epot"]


def test_restricted_hamiltonian_bruteforce():
    n = (2, 2, 2)
    N = 4
    cm = np.zeros((2, 2, 2), dtype=bool)
    cm[0, :, :] = True
    cm[1, 0, 0] = True
    fm = np.zeros_like(cm)
    fm[0, 0, :] = True
    nc, nf = RG.counts(cm, fm)
    V = inputs.gaussian_potential(83, 0, n)
    Sy = np.kron(mat_synthesis(2), np.kron(mat_synthesis(2), mat_synthesis(2)))
    Mf = np.kron(mat_mf(N), np.kron(mat_mf(N), mat_mf(N)))
    I = np.eye(N)
    Kx = mat_kin(N, 0.25)
    K = np.kron(I, np.kron(I, Kx)) + np.kron(I, np.kron(Kx, I)) + np.kron(Kx, np.kron(I, I))
    H = Sy.T @ (Mf.T @ np.diag(V.reshape(-1)) @ Mf + K) @ Sy
    L = nc + 7 * nf
    P = np.zeros((64, L))
    for k in range(L):
        e = np.zeros(L)
        e[k] = 1.0
        P[:, k] = RG.uncompress(e, n, cm, fm).reshape(-1)
    Hr = P.T @ H @ P
    psi = inputs.random_field(83, 2, (L,))
    got = RG.hpsi_local(psi, V, 2.0, n, cm, fm)["hpsi_c"]
    assert np.max(np.abs(got - Hr @ psi)) < 1e-12 * np.abs(Hr @ psi).max()
    assert np.max(np.abs(Hr - Hr.T)) < 1e-12 * np.abs(Hr).max()

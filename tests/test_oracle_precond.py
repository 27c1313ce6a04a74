"""Pins of the preconditioner oracle: the Helmholtz operator against dense
brute force, its diagonal, and the conjugate-gradient iterates against the
Krylov-subspace minimiser and the exact dense solve.  All CPU."""
import numpy as np
import pytest

import oracle.precond as PC
import oracle.wavelet as W
from paper_0904_1543_gb300 import inputs
from test_oracle_ops import mat_kin, mat_synthesis


def dense_A(n, eps, hg=(0.25, 0.25, 0.25)):
    """S^T (K - eps) S from 1D matrices built entry by entry, mapped to the
    compressed ordering."""
    N = [2 * v for v in n]
    S = np.kron(mat_synthesis(n[2]), np.kron(mat_synthesis(n[1]), mat_synthesis(n[0])))
    I = [np.eye(v) for v in N]
    K = (np.kron(I[2], np.kron(I[1], mat_kin(N[0], hg[0])))
         + np.kron(I[2], np.kron(mat_kin(N[1], hg[1]), I[0]))
         + np.kron(mat_kin(N[2], hg[2]), np.kron(I[1], I[0])))
    A_int = S.T @ (K - eps * np.eye(K.shape[0])) @ S
    # interleaved -> compressed permutation
    m = n[0] * n[1] * n[2]
    P = np.zeros((8 * m, 8 * m))
    for k in range(8 * m):
        e = np.zeros(8 * m)
        e[k] = 1.0
        P[:, k] = W.uncompress(e, n).reshape(-1)
    return P.T @ A_int @ P


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 2), (3, 2, 2)])
def test_helmholtz_apply_bruteforce(n):
    eps = -0.7
    hg = (0.25, 0.3, 0.2)
    A = dense_A(n, eps, hg)
    c = inputs.random_field(61, 1, (8 * n[0] * n[1] * n[2],))
    got = PC.helmholtz_apply(c, eps, n, hg)
    assert np.max(np.abs(got - A @ c)) < 1e-12 * np.abs(A @ c).max()
    # symmetric positive definite for eps < 0
    assert np.max(np.abs(A - A.T)) < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > -eps * 0.999


@pytest.mark.parametrize("n", [(2, 2, 2), (3, 2, 4)])
def test_helmholtz_diagonal(n):
    A = dense_A(n, 0.0)
    d = PC.helmholtz_diagonal(n)
    mu = PC.component_of(n)
    assert np.max(np.abs(np.diag(A) - d[mu])) < 1e-12 * np.abs(d).max()
    assert np.all(d > 0)


def test_cg_iterates_are_krylov_minimisers():
    """Preconditioned CG: x_k minimises ||x - x*||_A over the Krylov space
    K_k(M^-1 A, M^-1 g) (computed by a dense Galerkin solve)."""
    n = (2, 2, 2)
    eps = -0.5
    A = dense_A(n, eps)
    g = inputs.random_field(62, 1, (64,))
    Minv = 1.0 / (PC.helmholtz_diagonal(n)[PC.component_of(n)] - eps)
    _, hist = PC.precondition(g, eps, n, 4, return_history=True)
    for k in range(1, 5):
        V = [Minv * g]
        for _ in range(k - 1):
            V.append(Minv * (A @ V[-1]))
        V = np.stack(V, axis=1)
        Q, _ = np.linalg.qr(V)
        y = np.linalg.solve(Q.T @ A @ Q, Q.T @ g)
        ref = Q @ y
        assert np.max(np.abs(hist[k] - ref)) < 1e-10 * np.abs(ref).max(), k


def test_cg_converges_to_dense_solve_and_error_decreases():
    n = (2, 3, 2)
    eps = -0.3
    A = dense_A(n, eps)
    g = inputs.random_field(63, 1, (8 * 12,))
    xs = np.linalg.solve(A, g)
    x, hist = PC.precondition(g, eps, n, 60, return_history=True)
    assert np.max(np.abs(x - xs)) < 1e-9 * np.abs(xs).max()
    errA = [float((h - xs) @ A @ (h - xs)) for h in hist]
    assert all(errA[k + 1] <= errA[k] * (1 + 1e-12) for k in range(20))

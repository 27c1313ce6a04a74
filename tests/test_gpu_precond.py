"""GPU parity of the preconditioning step (Eq. precon): the Helmholtz
operator and the preconditioned conjugate gradient against the oracle.

FP64: the same iteration in the same order of operations up to summation
order; a few CG steps amplify rounding differences mildly, so the bound is
1e-11 relative (normwise).  FP32: bound 1e-4 after 4 iterations (the
operator is applied in binary32; the scalars are FP64/compensated).
"""
import numpy as np
import pytest

import oracle.precond as PC
from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    return W


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("n,norb,ncg", [((1, 1, 1), 2, 3), ((3, 5, 2), 3, 4), ((8, 8, 8), 2, 5),
                                        ((12, 10, 14), 2, 3)])
def test_pcg_f64(W, n, norb, ncg):
    import torch
    g = W.Grid(n, (0.25, 0.3, 0.35))
    G = inputs.orbitals(71, norb, n)
    eps = -np.linspace(0.2, 1.5, norb)
    x, rr = W.precondition(torch.from_numpy(G).cuda(), torch.from_numpy(eps).cuda(), g, ncg)
    ref = PC.precondition_batch(G, eps, n, ncg, g.h)
    assert _rel(x.cpu().numpy(), ref) < 1e-11
    for o in range(norb):
        res = G[o] - PC.helmholtz_apply(ref[o], eps[o], n, g.h)
        assert abs(float(rr[o]) - float(res @ res)) < 1e-8 * float(G[o] @ G[o])


def test_pcg_one_iteration_is_diagonal_scaled_step(W):
    """ncg = 0 returns x = 0 and |g|^2 as residual."""
    import torch
    n = (4, 4, 4)
    g = W.Grid(n)
    G = inputs.orbitals(72, 2, n)
    eps = np.array([-0.5, -1.0])
    x, rr = W.precondition(torch.from_numpy(G).cuda(), torch.from_numpy(eps).cuda(), g, 0)
    assert float(x.abs().max()) == 0.0
    assert np.allclose(rr.cpu().numpy(), (G * G).sum(1), rtol=1e-14)


def test_pcg_converges(W):
    """Many iterations drive the residual down by orders of magnitude."""
    import torch
    n = (6, 6, 6)
    g = W.Grid(n)
    G = inputs.orbitals(73, 2, n)
    eps = np.array([-0.4, -0.9])
    _, rr0 = W.precondition(torch.from_numpy(G).cuda(), torch.from_numpy(eps).cuda(), g, 0)
    x, rr = W.precondition(torch.from_numpy(G).cuda(), torch.from_numpy(eps).cuda(), g, 40)
    rr, rr0 = rr.cpu().numpy(), rr0.cpu().numpy()
    assert np.all(rr < 1e-2 * rr0)
    for o in range(2):
        ref = PC.precondition(G[o], eps[o], n, 40)
        res = G[o] - PC.helmholtz_apply(ref, eps[o], n)
        assert abs(rr[o] - res @ res) < 1e-6 * (res @ res) + 1e-12 * rr0[o]
        assert _rel(x[o].cpu().numpy(), ref) < 1e-9


def test_pcg_f32(W):
    import torch
    n = (6, 5, 7)
    g = W.Grid(n)
    G = inputs.orbitals(74, 3, n).astype(np.float32)
    eps = np.array([-0.3, -0.8, -1.2])
    x, _ = W.precondition(torch.from_numpy(G).cuda(), torch.from_numpy(eps).cuda(), g, 4)
    ref = PC.precondition_batch(G.astype(np.float64), eps, n, 4)
    assert _rel(x.double().cpu().numpy(), ref) < 1e-4

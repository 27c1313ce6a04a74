"""The expiry path of the bounded device-side waits (the tensor-core passes
wait on their MMAs for at most ~2 s): a kernel waits on an mbarrier that
nothing arrives on, gives up after a few milliseconds, and the host reads the
expiry.  Nothing faults or hangs, and the context keeps working."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_is_reported():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W
    from paper_0904_1543_gb300 import inputs
    assert W.wait_timeouts() == 0
    W.selftest_timeout(5.0)
    assert W.wait_timeouts() == 1          # counted once, then cleared
    assert W.wait_timeouts() == 0
    # the context is healthy: a tensor-core pass still runs and agrees
    n = (4, 3, 5)
    g = W.Grid(n)
    psi = torch.from_numpy(inputs.orbitals(381, 1, n)).cuda()
    V = torch.from_numpy(inputs.gaussian_potential(381, 0, n)).cuda()
    occ = torch.full((1,), 2.0, dtype=torch.float64, device="cuda")
    a = W.hpsi_local(psi, V, occ, g)[0]
    b = W.hpsi_local(psi, V, occ, g, emu=True)[0]
    assert float((a - b).abs().max() / a.abs().max()) < 1e-13
    assert W.wait_timeouts() == 0
    with pytest.raises(W.WvlError):
        W.selftest_timeout(-1.0)

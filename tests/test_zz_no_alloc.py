"""wvl_hpsi_local_noalloc against wvl_hpsi_local.

The no-allocation entry point serves callers that cannot pass a workspace or
allow device allocation at call time (a host program that owns every device
allocation, a pipeline that reserves all memory up front).  It must give the
same results as the workspace entry point, also on a second call that finds
the previous call's data still in its fixed scratch array.  This file is
collected last on purpose; it passes alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_0904_1543_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL64 = 1e-12     # the FP64 parity tolerance of the other GPU tests


def _close(a, b, rtol):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(np.abs(b).max(), 1e-300)
    assert np.abs(a - b).max() / scale <= rtol


def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W

    L = W.lib()
    f = L.wvl_hpsi_local_noalloc
    vp = ctypes.c_void_p
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(W._Grid), ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                  vp, vp]
    L.wvl_noalloc_last_error.restype = ctypes.c_char_p

    for call, (n, norb, cfg) in enumerate((((16, 16, 16), 3, 51), ((12, 10, 14), 2, 52))):
        g = W.Grid(n)
        psi = torch.from_numpy(inputs.orbitals(cfg, norb, n)).cuda()
        V = torch.from_numpy(inputs.gaussian_potential(cfg, 0, n)).cuda()
        occ = torch.full((norb,), 2.0, dtype=torch.float64, device="cuda")

        rho_ref = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
        hp_ref, ek_ref, ep_ref = W.hpsi_local(psi, V, occ, g, rho=rho_ref)

        hp = torch.empty_like(psi)
        ek = torch.empty(norb, dtype=torch.float64, device="cuda")
        ep = torch.empty_like(ek)
        rho = torch.zeros_like(rho_ref)
        st = f(ctypes.byref(g.c()), 0, norb, psi.data_ptr(), V.data_ptr(), occ.data_ptr(),
               hp.data_ptr(), rho.data_ptr(), ek.data_ptr(), ep.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
        assert st == 0, L.wvl_noalloc_last_error()
        torch.cuda.synchronize()
        _close(hp.cpu().numpy(), hp_ref.cpu().numpy(), RTOL64)
        _close(rho.cpu().numpy(), rho_ref.cpu().numpy(), RTOL64)
        _close(ek.cpu().numpy(), ek_ref.cpu().numpy(), RTOL64)
        _close(ep.cpu().numpy(), ep_ref.cpu().numpy(), RTOL64)

    # a problem larger than the fixed scratch is refused with a clear message
    big = W.Grid((64, 64, 64))
    st = f(ctypes.byref(big.c()), 0, 4, 1 << 40, 1 << 40, 1 << 40, 1 << 40, None, 1 << 40,
           1 << 40, None)
    assert st == 5
    assert b"scratch" in L.wvl_noalloc_last_error()

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

# the parity tolerances of the other GPU tests, per precision: FP64 and its
# tensor-core form 1e-12, FP32 2e-6 (both entry points run the same kernels,
# so the results are expected to agree bit for bit)
PRECS = {"f64": (0, "float64", False, 1e-12), "f32": (1, "float32", False, 2e-6),
         "f64_emu": (2, "float64", True, 1e-12)}


def _close(a, b, rtol):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(np.abs(b).max(), 1e-300)
    assert np.abs(a - b).max() / scale <= rtol


def _entry(W):
    L = W.lib()
    f = L.wvl_hpsi_local_noalloc
    vp = ctypes.c_void_p
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(W._Grid), ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                  vp, vp]
    L.wvl_noalloc_last_error.restype = ctypes.c_char_p
    return L, f


@pytest.mark.parametrize("form", list(PRECS))
def test_noalloc_matches_workspace_entry_point_twice(form):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W

    prec, dt, emu, rtol = PRECS[form]
    dtype = getattr(torch, dt)
    L, f = _entry(W)
    # two calls in a row: the second finds the first call's data in the array
    for n, norb, cfg in (((16, 16, 16), 3, 51), ((12, 10, 14), 2, 52)):
        g = W.Grid(n)
        psi = torch.from_numpy(inputs.orbitals(cfg, norb, n)).to("cuda", dtype)
        V = torch.from_numpy(inputs.gaussian_potential(cfg, 0, n)).to("cuda", dtype)
        occ = torch.full((norb,), 2.0, dtype=torch.float64, device="cuda")

        rho_ref = torch.zeros(g.fine, dtype=torch.float64, device="cuda")
        hp_ref, ek_ref, ep_ref = W.hpsi_local(psi, V, occ, g, rho=rho_ref, emu=emu)

        hp = torch.empty_like(psi)
        ek = torch.empty(norb, dtype=torch.float64, device="cuda")
        ep = torch.empty_like(ek)
        rho = torch.zeros_like(rho_ref)
        st = f(ctypes.byref(g.c()), prec, norb, psi.data_ptr(), V.data_ptr(), occ.data_ptr(),
               hp.data_ptr(), rho.data_ptr(), ek.data_ptr(), ep.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
        assert st == 0, L.wvl_noalloc_last_error()
        torch.cuda.synchronize()
        _close(hp.cpu().numpy(), hp_ref.cpu().numpy(), rtol)
        _close(rho.cpu().numpy(), rho_ref.cpu().numpy(), rtol)
        _close(ek.cpu().numpy(), ek_ref.cpu().numpy(), rtol)
        _close(ep.cpu().numpy(), ep_ref.cpu().numpy(), rtol)


def test_noalloc_errors():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0904_1543_gb300 as W

    L, f = _entry(W)
    # a problem larger than the fixed scratch is refused with a clear message
    big = W.Grid((64, 64, 64))
    st = f(ctypes.byref(big.c()), 0, 4, 1 << 40, 1 << 40, 1 << 40, 1 << 40, None, 1 << 40,
           1 << 40, None)
    assert st == 5
    assert b"scratch" in L.wvl_noalloc_last_error()
    # an error of the inner call (a null orbital array) is reported through
    # this entry point's own message too; nothing is enqueued
    g = W.Grid((8, 8, 8))
    buf = torch.zeros(8 * 512 * 2, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    st = f(ctypes.byref(g.c()), 0, 1, None, p, p, p, None, p, p, None)
    assert st == 1
    msg = L.wvl_noalloc_last_error()
    assert msg and b"psi" in msg

"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every symbol include/wvl.h declares, derives the same filters as the oracle,
and rejects bad arguments before enqueuing anything."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle.filters as F
import paper_0904_1543_gb300 as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wvl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wvl_[a-z_0-9A-Z]+)\s*\(", src)))


def test_header_symbols_exported():
    L = W.lib()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value


def test_library_filters_match_oracle():
    """Independent derivations (C++ double-double vs 80-digit decimal) agree
    to the last bit, up to one ulp on the tiniest kinetic taps."""
    f = W.filters()
    w, k0 = F.magic()
    assert f["k0"] == k0
    assert np.array_equal(f["h"], F.h())
    assert np.array_equal(f["g"], F.g())
    assert np.array_equal(f["w"], w)
    a = F.kinetic_a()
    ulp = np.spacing(np.abs(a))
    assert np.all(np.abs(f["a"] - a) <= ulp)


def test_status_strings_and_version():
    L = W.lib()
    for s in range(6):
        assert L.wvl_status_string(s)
    assert L.wvl_version() >= 10000


def G(n=(4, 4, 4), h=(0.25, 0.25, 0.25)):
    return ctypes.byref(W.Grid(n, h).c())


def test_workspace_size_monotone():
    a = W.workspace_size(W.Grid((8, 8, 8)), 0, 1)
    b = W.workspace_size(W.Grid((8, 8, 8)), 0, 4)
    c = W.workspace_size(W.Grid((8, 8, 8)), 1, 4)
    assert 0 < a < b and c < b


@pytest.mark.parametrize("bad", [(0, 4, 4), (4, -1, 4), (513, 4, 4)])
def test_bad_grid_rejected(bad):
    L = W.lib()
    sz = ctypes.c_size_t(0)
    st = L.wvl_workspace_size(G(bad), 0, 1, ctypes.byref(sz))
    assert st in (1, 5)
    assert L.wvl_last_error()


def test_bad_spacing_and_prec_rejected():
    L = W.lib()
    sz = ctypes.c_size_t(0)
    assert L.wvl_workspace_size(G((4, 4, 4), (0.25, 0.0, 0.25)), 0, 1, ctypes.byref(sz)) == 1
    assert L.wvl_workspace_size(G(), 7, 1, ctypes.byref(sz)) == 1


def test_null_and_misaligned_pointers_rejected():
    L = W.lib()
    fake = 1 << 40          # never dereferenced: validation fails first
    # null input
    assert L.wvl_synthesis(G(), 0, 1, None, fake, fake, 1 << 30, None) == 1
    # misaligned output
    assert L.wvl_synthesis(G(), 0, 1, fake, fake + 8, fake, 1 << 30, None) == 1
    # hpsi: missing energies
    assert L.wvl_hpsi_local(G(), 0, 1, fake, fake, fake, fake, None, None, fake, fake,
                            1 << 30, None) == 1
    assert b"ekin" in L.wvl_last_error()


def test_workspace_too_small_rejected():
    L = W.lib()
    fake = 1 << 40
    st = L.wvl_magicfilter(G(), 0, 1, fake, fake, fake, 1024, None)
    assert st == 2
    assert b"workspace" in L.wvl_last_error()
    # unaligned workspace
    st = L.wvl_magicfilter(G(), 0, 1, fake, fake, fake + 16, 1 << 30, None)
    assert st == 1


def test_zero_orbitals_is_a_noop():
    L = W.lib()
    assert L.wvl_hpsi_local(G(), 0, 0, None, None, None, None, None, None, None, None, 0,
                            None) == 0


def test_plan_creation_and_offsets():
    cells = [W.Grid((4, 4, 4)), W.Grid((5, 6, 3))]
    p = W.Plan(cells, [0, 0, 1, 0], prec=0, graph=True)
    P0, P1 = 8 * 64, 8 * 90
    assert p.offsets == [0, P0, 2 * P0, 2 * P0 + P1, 3 * P0 + P1]
    assert p.ws_bytes > 0
    with pytest.raises(W.WvlError):
        W.Plan(cells, [0, 2], prec=0)
    with pytest.raises(W.WvlError):
        W.Plan(cells, [0], prec=3)


def test_tensor_core_form_validation():
    """WVL_F64_EMU takes FP64 arrays: the same workspace as WVL_F64, and the
    same argument checks; other precision codes are refused."""
    g = W.Grid((8, 6, 4))
    assert W.workspace_size(g, W.WVL_F64_EMU, 3) == W.workspace_size(g, W.WVL_F64, 3)
    L = W.lib()
    sz = ctypes.c_size_t(0)
    assert L.wvl_workspace_size(ctypes.byref(g.c()), 3, 1, ctypes.byref(sz)) == 1   # EINVAL
    st = L.wvl_hpsi_local(ctypes.byref(g.c()), W.WVL_F64_EMU, 1, None, None, None, None, None,
                          None, None, None, 0, None)
    assert st == 1                                                             # EINVAL (NULL)


def test_timeout_selftest_arguments():
    L = W.lib()
    assert L.wvl_selftest_timeout(-1.0, None) == 1
    assert L.wvl_selftest_timeout(0.0, None) == 1
    assert L.wvl_selftest_timeout(1e9, None) == 1
    assert L.wvl_wait_timeouts(None) == 1


def test_chain_flags_validation():
    """The fused chain takes periodic cells whose fine extents are multiples
    of 8 in [32, 128], in FP64 or FP32; the two chain flags exclude each
    other.  All checked on the host by wvl_plan_create."""
    ok = [W.Grid((16, 20, 24)), W.Grid((56, 56, 56))]
    for prec in (W.WVL_F64, W.WVL_F32):
        W.Plan(ok, [0, 1], prec=prec, chain="fused")
        W.Plan(ok, [0, 1], prec=prec, chain="passes")
        W.Plan(ok, [0, 1], prec=prec)
    W.Plan([W.Grid((64, 64, 64))], [0], prec=W.WVL_F32, chain="fused")
    for bad in ((12, 16, 16), (16, 18, 16), (16, 16, 68), (17, 16, 16)):
        with pytest.raises(W.WvlError):
            W.Plan([W.Grid(bad)], [0], prec=W.WVL_F32, chain="fused")
        W.Plan([W.Grid(bad)], [0], prec=W.WVL_F32, chain="passes")
    with pytest.raises(W.WvlError):
        W.Plan(ok, [0], prec=W.WVL_F64_EMU, chain="fused")
    # FP64 planes of 128 x 128 exceed one CTA's shared memory
    with pytest.raises(W.WvlError):
        W.Plan([W.Grid((64, 64, 64))], [0], prec=W.WVL_F64, chain="fused")
    with pytest.raises(ValueError):
        W.Plan(ok, [0], chain="other")
    L = W.lib()
    h = ctypes.c_void_p()
    g = ok[0].c()
    co = (ctypes.c_int * 1)(0)
    assert L.wvl_plan_create(ctypes.byref(g), 1, co, 1, 0, 4 | 8, ctypes.byref(h)) == 1   # EINVAL
    assert L.wvl_plan_create(ctypes.byref(g), 1, co, 1, 0, 16, ctypes.byref(h)) == 1      # EINVAL

"""Python binding of libwvl (the C ABI in include/wvl.h).

Argument marshalling only: every step of the local Hamiltonian runs in the
library's CUDA kernels.  PyTorch provides device memory (inputs, outputs and
the scratch workspace) and the current CUDA stream.  There is no CPU fallback:
if libwvl.so cannot be loaded the calls raise.

Layouts (see include/wvl.h): compressed orbitals ``(norb, 8 n1 n2 n3)``, fine
arrays ``(norb, N3, N2, N1)`` with N_d = 2 n_d, potential and density
``(N3, N2, N1)``.  float64 tensors select the FP64 kernels, float32 tensors
the FP32 kernels (density, occupations and energies stay float64).
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

from . import _build

__all__ = [
    "WvlError", "Grid", "lib", "filters", "workspace_size", "synthesis", "analysis",
    "magicfilter", "magicfilter_T", "kinetic", "density", "hpsi_local", "energy", "eloc", "overlap", "dot",
    "Plan", "ELoc", "device_count", "wait_timeouts", "WVL_F64", "WVL_F32", "WVL_F64_EMU",
]

WVL_F64, WVL_F32, WVL_F64_EMU = 0, 1, 2
WVL_PLAN_GRAPH, WVL_PLAN_AUTOTUNE, WVL_PLAN_FUSED, WVL_PLAN_PASSES = 1, 2, 4, 8
WVL_NSTAGE = 6
STAGES = ("synthesis", "magicfilter+potential", "magicfilter_T", "kinetic", "analysis",
          "reductions")


class WvlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
                ("h1", ctypes.c_double), ("h2", ctypes.c_double), ("h3", ctypes.c_double)]


@dataclass(frozen=True)
class Grid:
    """Coarse extents (n1, n2, n3) and fine spacings h' = (h1, h2, h3)."""
    n: tuple
    h: tuple = (0.25, 0.25, 0.25)

    @property
    def fine(self):
        return (2 * self.n[2], 2 * self.n[1], 2 * self.n[0])   # (N3, N2, N1)

    @property
    def ncoef(self):
        return 8 * self.n[0] * self.n[1] * self.n[2]

    def c(self):
        return _Grid(self.n[0], self.n[1], self.n[2], *map(float, self.h))


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t


def _declare(L):
    G = ctypes.POINTER(_Grid)
    sigs = {
        "wvl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "wvl_last_error": (ctypes.c_char_p, []),
        "wvl_version": (ctypes.c_int, []),
        "wvl_device_count": (ctypes.c_int, []),
        "wvl_kernel_launches": (ctypes.c_ulonglong, []),
        "wvl_wait_timeouts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint)]),
        "wvl_selftest_timeout": (ctypes.c_int, [ctypes.c_double, _vp]),
        "wvl_filters": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "wvl_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, _vp, _vp, _vp]),
        "wvl_workspace_size": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_sz)]),
        "wvl_synthesis": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _sz, _vp]),
        "wvl_analysis": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _sz, _vp]),
        "wvl_magicfilter": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _sz, _vp]),
        "wvl_magicfilter_T": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _sz, _vp]),
        "wvl_kinetic": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
        "wvl_density": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _sz, _vp]),
        "wvl_hpsi_local": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp,
                                          _vp, _vp, _vp, _sz, _vp]),
        "wvl_energy": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                                      _vp, _sz, _vp]),
        "wvl_eloc": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                                    _vp, _vp, _sz, _vp]),
        "wvl_eloc_backward": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                                             _vp, _vp, _vp, _vp, _sz, _vp]),
        "wvl_overlap_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_longlong, ctypes.POINTER(_sz)]),
        "wvl_overlap": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                       ctypes.c_longlong, _vp, _vp, _sz, _vp]),
        "wvl_dot": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_longlong, _vp,
                                   _vp, _sz, _vp]),
        "wvl_plan_create": (ctypes.c_int, [G, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_uint, ctypes.POINTER(_vp)]),
        "wvl_plan_destroy": (ctypes.c_int, [_vp]),
        "wvl_plan_workspace_size": (ctypes.c_int, [_vp, ctypes.POINTER(_sz)]),
        "wvl_plan_orbital_offset": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_sz)]),
        "wvl_plan_hpsi": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
        "wvl_plan_autotune": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
        "wvl_plan_describe": (ctypes.c_int, [_vp, ctypes.c_char_p, _sz]),
        "wvl_plan_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
        "wvl_plan_profile": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    """The loaded libwvl.so (built in-tree on first use if nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB) or not _build.up_to_date():
                try:
                    _build.build()
                except Exception as e:   # no toolkit: only a prebuilt library will do
                    if not os.path.exists(_build.LIB):
                        raise RuntimeError(f"libwvl.so is missing and cannot be built: {e}")
            _lib = _declare(ctypes.CDLL(_build.LIB))
    return _lib


def _check(status):
    if status != 0:
        L = lib()
        raise WvlError(status, L.wvl_status_string(status).decode() + ": "
                       + (L.wvl_last_error() or b"").decode())


def device_count():
    return lib().wvl_device_count()


def kernel_launches():
    """Kernels enqueued by the library so far in this process."""
    return lib().wvl_kernel_launches()


def selftest_timeout(ms=5.0, device=None):
    """Enqueue one kernel whose bounded wait cannot be satisfied: it gives up
    after about ms and counts one expiry (see wait_timeouts)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    _check(lib().wvl_selftest_timeout(float(ms), _stream(dev)))


def wait_timeouts():
    """Bounded device-side waits (tensor-core passes) that gave up since the
    previous call; synchronises the device.  0 on a healthy run."""
    c = ctypes.c_uint(0)
    st = lib().wvl_wait_timeouts(ctypes.byref(c))
    if st not in (0, 4):
        _check(st)
    return c.value


def fma_peak(prec=WVL_F64, seconds=0.2, device=None):
    """Measured FMA-chain rate of the device's FP64 (prec WVL_F64) or FP32
    (WVL_F32) pipe in TFLOP/s, and the timed launch's milliseconds."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().wvl_fma_peak(int(prec), float(seconds), ctypes.byref(tf), ctypes.byref(ms),
                              _stream(dev)))
    return tf.value, ms.value


def filters():
    """The library's own filters: h, g (16), w (16) with k0, a (29)."""
    import numpy as np
    h, g, w, a = (np.zeros(16), np.zeros(16), np.zeros(16), np.zeros(29))
    k0 = ctypes.c_int(0)
    _check(lib().wvl_filters(h.ctypes.data, g.ctypes.data, w.ctypes.data,
                             ctypes.addressof(k0), a.ctypes.data))
    return {"h": h, "g": g, "w": w, "k0": k0.value, "a": a}


def _prec(t, emu=False):
    """WVL_F64 / WVL_F32 from the dtype; emu=True selects WVL_F64_EMU (float64
    arrays, convolution sums on the tensor cores)."""
    if emu:
        if t.dtype != torch.float64:
            raise TypeError("emu=True needs float64 arrays")
        return WVL_F64_EMU
    if t.dtype == torch.float64:
        return WVL_F64
    if t.dtype == torch.float32:
        return WVL_F32
    raise TypeError(f"unsupported dtype {t.dtype}: use float64 or float32")


def workspace_size(grid: Grid, prec: int, norb: int) -> int:
    out = _sz(0)
    _check(lib().wvl_workspace_size(ctypes.byref(grid.c()), prec, norb, ctypes.byref(out)))
    return out.value


_ws_cache = {}


def _workspace(nbytes, device, stream):
    """Per (device, stream) scratch buffer, grown on demand (256-byte aligned)."""
    key = (device.index, int(stream))
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256) + 256, dtype=torch.uint8, device=device)
        _ws_cache[key] = buf
    ptr = buf.data_ptr()
    off = (-ptr) % 256
    return ptr + off, buf.numel() - off


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


def _dev(t, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _norb(x, per):
    if x.numel() % per:
        raise ValueError(f"tensor of {x.numel()} elements is not a whole number of orbitals of {per}")
    return x.numel() // per


def _p(t):
    return None if t is None else t.data_ptr()


def _run(fn, grid, prec, norb, device, *ptrs):
    st = _stream(device)
    need = workspace_size(grid, prec, max(norb, 1))
    ws, wsb = _workspace(need, device, st)
    _check(fn(ctypes.byref(grid.c()), prec, norb, *ptrs, ws, wsb, st))


def synthesis(psi_c, grid: Grid, out=None, emu=False):
    """Steps 1)+2): compressed coefficients -> fine scaling coefficients."""
    norb = _norb(psi_c, grid.ncoef)
    out = torch.empty((norb, *grid.fine), dtype=psi_c.dtype, device=psi_c.device) if out is None else out
    _dev(psi_c, "psi_c"), _dev(out, "out")
    _run(lib().wvl_synthesis, grid, _prec(psi_c, emu), norb, psi_c.device, psi_c.data_ptr(), out.data_ptr())
    return out


def analysis(z, grid: Grid, out=None, emu=False):
    """Steps 6)+7): fine -> compressed (transpose of synthesis)."""
    norb = _norb(z, grid.ncoef)
    out = torch.empty((norb, grid.ncoef), dtype=z.dtype, device=z.device) if out is None else out
    _dev(z, "z"), _dev(out, "out")
    _run(lib().wvl_analysis, grid, _prec(z, emu), norb, z.device, z.data_ptr(), out.data_ptr())
    return out


def magicfilter(s, grid: Grid, out=None, emu=False):
    norb = _norb(s, grid.ncoef)
    out = torch.empty_like(s) if out is None else out
    _dev(s, "s"), _dev(out, "out")
    _run(lib().wvl_magicfilter, grid, _prec(s, emu), norb, s.device, s.data_ptr(), out.data_ptr())
    return out


def magicfilter_T(y, grid: Grid, out=None, emu=False):
    norb = _norb(y, grid.ncoef)
    out = torch.empty_like(y) if out is None else out
    _dev(y, "y"), _dev(out, "out")
    _run(lib().wvl_magicfilter_T, grid, _prec(y, emu), norb, y.device, y.data_ptr(), out.data_ptr())
    return out


def kinetic(s, grid: Grid, k0=None, out=None, want_ekin=True, emu=False):
    """out = K0 + (-1/2 Lap) s and ekin[o] = <s_o, -1/2 Lap s_o>."""
    norb = _norb(s, grid.ncoef)
    out = torch.empty_like(s) if out is None else out
    ek = torch.empty(norb, dtype=torch.float64, device=s.device) if want_ekin else None
    _dev(s, "s"), _dev(out, "out")
    if k0 is not None:
        _dev(k0, "k0")
    _run(lib().wvl_kinetic, grid, _prec(s, emu), norb, s.device, s.data_ptr(), _p(k0),
         out.data_ptr(), _p(ek))
    return out, ek


def density(psi_c, occ, grid: Grid, rho=None, emu=False):
    """rho += sum_o occ_o |psi_r,o|^2 (float64, (N3, N2, N1))."""
    norb = _norb(psi_c, grid.ncoef)
    rho = torch.zeros(grid.fine, dtype=torch.float64, device=psi_c.device) if rho is None else rho
    _dev(psi_c, "psi_c"), _dev(occ, "occ"), _dev(rho, "rho")
    _run(lib().wvl_density, grid, _prec(psi_c, emu), norb, psi_c.device, psi_c.data_ptr(),
         occ.data_ptr(), rho.data_ptr())
    return rho


def hpsi_local(psi_c, V, occ, grid: Grid, rho=None, out=None, emu=False):
    """H_loc psi for norb orbitals of one cell; rho += density if given.
    Returns (hpsi_c, ekin, epot)."""
    norb = _norb(psi_c, grid.ncoef)
    out = torch.empty_like(psi_c) if out is None else out
    ek = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    ep = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    for t, nm in ((psi_c, "psi_c"), (V, "V"), (occ, "occ"), (out, "out")):
        _dev(t, nm)
    if rho is not None:
        _dev(rho, "rho")
    _run(lib().wvl_hpsi_local, grid, _prec(psi_c, emu), norb, psi_c.device, psi_c.data_ptr(),
         V.data_ptr(), occ.data_ptr(), out.data_ptr(), _p(rho), ek.data_ptr(), ep.data_ptr())
    return out, ek, ep


def energy(psi_c, V, occ, grid: Grid, rho=None, emu=False):
    """Per-orbital (ekin, epot) without H psi; rho += density if given."""
    norb = _norb(psi_c, grid.ncoef)
    ek = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    ep = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    for t, nm in ((psi_c, "psi_c"), (V, "V"), (occ, "occ")):
        _dev(t, nm)
    if rho is not None:
        _dev(rho, "rho")
    _run(lib().wvl_energy, grid, _prec(psi_c, emu), norb, psi_c.device, psi_c.data_ptr(),
         V.data_ptr(), occ.data_ptr(), _p(rho), ek.data_ptr(), ep.data_ptr())
    return ek, ep


def eloc(psi_c, V, occ, grid: Grid, rho=None, emu=False):
    """E_loc = sum_o occ_o (Ekin_o + Epot_o) as a 0-d float64 device tensor,
    with the per-orbital (ekin, epot); rho += density if given."""
    norb = _norb(psi_c, grid.ncoef)
    dev = psi_c.device
    ek = torch.empty(norb, dtype=torch.float64, device=dev)
    ep = torch.empty(norb, dtype=torch.float64, device=dev)
    e = torch.empty((), dtype=torch.float64, device=dev)
    for t, nm in ((psi_c, "psi_c"), (V, "V"), (occ, "occ")):
        _dev(t, nm)
    if rho is not None:
        _dev(rho, "rho")
    _run(lib().wvl_eloc, grid, _prec(psi_c, emu), norb, dev, psi_c.data_ptr(), V.data_ptr(),
         occ.data_ptr(), _p(rho), ek.data_ptr(), ep.data_ptr(), e.data_ptr())
    return e, ek, ep


def _overlap_ws(prec, na, nb, ln, device):
    need = _sz(0)
    _check(lib().wvl_overlap_workspace_size(prec, na, nb, ln, ctypes.byref(need)))
    st = _stream(device)
    ws, wsb = _workspace(need.value, device, st)
    return ws, wsb, st


def overlap(a, b=None):
    """Scalar products <a_i|b_j> of compressed orbitals (rows of a and b; b
    defaults to a) as a float64 (na, nb) device tensor: FP64 products and
    accumulation whatever the coefficients' precision."""
    b = a if b is None else b
    if a.dtype != b.dtype:
        raise TypeError("a and b must have the same dtype")
    a2 = a.reshape(a.shape[0], -1)
    b2 = b.reshape(b.shape[0], -1)
    if a2.shape[1] != b2.shape[1]:
        raise ValueError("a and b must have the same length per orbital")
    _dev(a2, "a"), _dev(b2, "b")
    na, nb, ln = a2.shape[0], b2.shape[0], a2.shape[1]
    S = torch.empty((na, nb), dtype=torch.float64, device=a.device)
    prec = _prec(a)
    ws, wsb, st = _overlap_ws(prec, na, nb, ln, a.device)
    _check(lib().wvl_overlap(prec, na, a2.data_ptr(), nb, b2.data_ptr(), ln, S.data_ptr(), ws,
                             wsb, st))
    return S


def dot(a, b):
    """Per-orbital scalar products <a_o|b_o> (float64, FP64 accumulation)."""
    if a.shape != b.shape or a.dtype != b.dtype:
        raise ValueError("a and b must have the same shape and dtype")
    a2 = a.reshape(a.shape[0], -1)
    b2 = b.reshape(b.shape[0], -1)
    _dev(a2, "a"), _dev(b2, "b")
    n, ln = a2.shape
    d = torch.empty(n, dtype=torch.float64, device=a.device)
    prec = _prec(a)
    ws, wsb, st = _overlap_ws(prec, n, n, ln, a.device)
    _check(lib().wvl_dot(prec, n, a2.data_ptr(), b2.data_ptr(), ln, d.data_ptr(), ws, wsb, st))
    return d


class Plan:
    """Batched local Hamiltonian for orbitals on cells of different sizes
    (one enqueue of every pass over all cells; optional graph replay and
    autotuning)."""

    def __init__(self, cells, cell_of_orb, prec=WVL_F64, graph=True, autotune=False, chain=None):
        """chain: None (automatic; the autotuner may choose), "fused" (the
        plane/column kernels) or "passes" (the transposing 1D passes)."""
        self.cells = [c if isinstance(c, Grid) else Grid(tuple(c)) for c in cells]
        self.cell_of_orb = [int(c) for c in cell_of_orb]
        self.prec = prec
        arr = (_Grid * len(self.cells))(*[c.c() for c in self.cells])
        co = (ctypes.c_int * max(1, len(self.cell_of_orb)))(*self.cell_of_orb)
        flags = (WVL_PLAN_GRAPH if graph else 0) | (WVL_PLAN_AUTOTUNE if autotune else 0)
        if chain not in (None, "fused", "passes"):
            raise ValueError("chain must be None, 'fused' or 'passes'")
        flags |= {None: 0, "fused": WVL_PLAN_FUSED, "passes": WVL_PLAN_PASSES}[chain]
        h = _vp()
        _check(lib().wvl_plan_create(arr, len(self.cells), co, len(self.cell_of_orb), prec,
                                     flags, ctypes.byref(h)))
        self._h = h
        self.norb = len(self.cell_of_orb)
        sz = _sz(0)
        _check(lib().wvl_plan_workspace_size(h, ctypes.byref(sz)))
        self.ws_bytes = sz.value
        self.offsets = []
        for o in range(self.norb + 1):
            _check(lib().wvl_plan_orbital_offset(h, o, ctypes.byref(sz)))
            self.offsets.append(sz.value)
        self.total = self.offsets[-1]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.wvl_plan_destroy(h)
            self._h = None

    def _args(self, psi, V, occ, hpsi, rho, ekin, epot):
        for t, nm in ((psi, "psi"), (occ, "occ"), (hpsi, "hpsi"), (ekin, "ekin"), (epot, "epot")):
            _dev(t, nm)
        if psi.numel() != self.total or hpsi.numel() != self.total:
            raise ValueError("psi/hpsi must hold the plan's concatenated orbitals")
        Vp = (_vp * len(self.cells))(*[_dev(v, "V") for v in V])
        Rp = None
        if rho is not None:
            Rp = (_vp * len(self.cells))(*[(None if r is None else _dev(r, "rho")) for r in rho])
        st = _stream(psi.device)
        ws, wsb = _workspace(self.ws_bytes, psi.device, st)
        return (self._h, psi.data_ptr(), Vp, occ.data_ptr(), hpsi.data_ptr(), Rp,
                ekin.data_ptr(), epot.data_ptr(), ws, wsb, st)

    def hpsi(self, psi, V, occ, hpsi=None, rho=None, ekin=None, epot=None):
        dev = psi.device
        hpsi = torch.empty_like(psi) if hpsi is None else hpsi
        ekin = torch.empty(self.norb, dtype=torch.float64, device=dev) if ekin is None else ekin
        epot = torch.empty(self.norb, dtype=torch.float64, device=dev) if epot is None else epot
        _check(lib().wvl_plan_hpsi(*self._args(psi, V, occ, hpsi, rho, ekin, epot)))
        return hpsi, ekin, epot

    def autotune(self, psi, V, occ, hpsi=None, rho=None):
        dev = psi.device
        hpsi = torch.empty_like(psi) if hpsi is None else hpsi
        ek = torch.empty(self.norb, dtype=torch.float64, device=dev)
        ep = torch.empty(self.norb, dtype=torch.float64, device=dev)
        _check(lib().wvl_plan_autotune(*self._args(psi, V, occ, hpsi, rho, ek, ep)))

    def describe(self):
        buf = ctypes.create_string_buffer(4096)
        _check(lib().wvl_plan_describe(self._h, buf, 4096))
        return buf.value.decode()

    def set_profiling(self, on=True):
        _check(lib().wvl_plan_set_profiling(self._h, int(bool(on))))

    def profile(self):
        """{stage: (ms, launches)} since the last read."""
        import numpy as np
        ms = np.zeros(WVL_NSTAGE)
        cnt = np.zeros(WVL_NSTAGE, dtype=np.int32)
        _check(lib().wvl_plan_profile(self._h, ms.ctypes.data, cnt.ctypes.data, WVL_NSTAGE))
        return {STAGES[k]: (float(ms[k]), int(cnt[k])) for k in range(WVL_NSTAGE)}


class ELoc(torch.autograd.Function):
    """E_loc(psi, V) = sum_o occ_o (Ekin_o + Epot_o) for the orbitals of one
    cell.  Forward: wvl_eloc (steps 1), 2), 3a), 3b) and 4) only -- energies,
    density and their total on the device, no H psi).  Backward:
    wvl_eloc_backward, whose adjoint kernels recompute the real-space orbitals
    instead of storing them and write dE/dpsi_o = 2 occ_o g H psi_o from the
    last pass of the chain, and dE/dV = g rho.  This class only marshals
    tensors; the arithmetic is in the library."""

    @staticmethod
    def forward(ctx, psi, V, occ, grid, emu=False):
        psi_d, V_d = psi.detach(), V.detach()
        norb = _norb(psi_d, grid.ncoef)
        dev = psi.device
        rho = torch.zeros(grid.fine, dtype=torch.float64, device=dev)
        ek = torch.empty(norb, dtype=torch.float64, device=dev)
        ep = torch.empty(norb, dtype=torch.float64, device=dev)
        e = torch.empty((), dtype=torch.float64, device=dev)
        for t, nm in ((psi_d, "psi"), (V_d, "V"), (occ, "occ")):
            _dev(t, nm)
        _run(lib().wvl_eloc, grid, _prec(psi_d, emu), norb, dev, psi_d.data_ptr(),
             V_d.data_ptr(), occ.data_ptr(), rho.data_ptr(), ek.data_ptr(), ep.data_ptr(),
             e.data_ptr())
        ctx.save_for_backward(psi, V, occ, rho)
        ctx.grid = grid
        ctx.emu = emu
        return e

    @staticmethod
    def backward(ctx, g):
        psi, V, occ, rho = ctx.saved_tensors
        psi_d, V_d = psi.detach(), V.detach()
        gb = g.detach().to(device=psi.device, dtype=torch.float64).reshape(1).contiguous()
        gpsi = torch.empty_like(psi_d) if ctx.needs_input_grad[0] else None
        gV = torch.empty_like(V_d) if ctx.needs_input_grad[1] else None
        if gpsi is not None or gV is not None:
            norb = _norb(psi_d, ctx.grid.ncoef)
            _run(lib().wvl_eloc_backward, ctx.grid, _prec(psi_d, ctx.emu), norb, psi.device,
                 psi_d.data_ptr(), V_d.data_ptr(), occ.data_ptr(), rho.data_ptr(),
                 gb.data_ptr(), _p(gpsi), _p(gV))
        return gpsi, gV, None, None, None


def precondition(g, eps, grid: Grid, ncg=5, x=None, want_residual=True, emu=False):
    """ncg iterations of preconditioned CG for (S^T (-1/2 Lap - eps_o) S) x = g
    per orbital (the preconditioning step).  g: (norb, 8 n1 n2 n3); eps:
    float64 (norb,) on the device, each < 0.  Returns (x, |g - A x|^2)."""
    norb = _norb(g, grid.ncoef)
    x = torch.empty_like(g) if x is None else x
    rr = torch.empty(norb, dtype=torch.float64, device=g.device) if want_residual else None
    _dev(g, "g"), _dev(eps, "eps"), _dev(x, "x")
    L = lib()
    if not getattr(L, "_pc_declared", False):
        Gp = ctypes.POINTER(_Grid)
        L.wvl_precondition_workspace_size.restype = ctypes.c_int
        L.wvl_precondition_workspace_size.argtypes = [Gp, ctypes.c_int, ctypes.c_int,
                                                      ctypes.POINTER(_sz)]
        L.wvl_precondition.restype = ctypes.c_int
        L.wvl_precondition.argtypes = [Gp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int,
                                       _vp, _vp, _vp, _sz, _vp]
        L._pc_declared = True
    prec = _prec(g, emu)
    need = _sz(0)
    _check(L.wvl_precondition_workspace_size(ctypes.byref(grid.c()), prec, max(norb, 1),
                                             ctypes.byref(need)))
    st = _stream(g.device)
    ws, wsb = _workspace(need.value, g.device, st)
    _check(L.wvl_precondition(ctypes.byref(grid.c()), prec, norb, g.data_ptr(), eps.data_ptr(),
                              int(ncg), x.data_ptr(), _p(rr), ws, wsb, st))
    return x, rr


class _Region(ctypes.Structure):
    _fields_ = [("coarse_index", _vp), ("fine_index", _vp), ("ncoarse", ctypes.c_longlong),
                ("nfine", ctypes.c_longlong), ("lo", ctypes.c_int * 3), ("len", ctypes.c_int * 3)]


def _declare_region(L):
    if getattr(L, "_region_declared", False):
        return
    Gp, Rp = ctypes.POINTER(_Grid), ctypes.POINTER(_Region)
    sig = {
        "wvl_region_index": [Gp, _vp, _vp, _vp, _vp, _vp, _vp],
        "wvl_region_bounds": [Gp, _vp, _vp, _vp, _vp],
        "wvl_synthesis_region": [Gp, Rp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _sz, _vp],
        "wvl_analysis_region": [Gp, Rp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _sz, _vp],
        "wvl_density_region": [Gp, Rp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _sz, _vp],
        "wvl_hpsi_local_region": [Gp, Rp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _vp, _sz, _vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.restype = ctypes.c_int
        f.argtypes = args
    L._region_declared = True


class Region:
    """Localisation region of the compressed form: boolean masks of shape
    (n3, n2, n1) for the points that keep their scaling coefficient (coarse)
    and their seven wavelet coefficients (fine)."""

    def __init__(self, grid: Grid, coarse_mask, fine_mask, device="cuda", bounds=True):
        """bounds=True also passes the region's periodic bounding box, so
        that the library computes on it where it is small enough."""
        import numpy as np
        L = lib()
        _declare_region(L)
        m = grid.n[0] * grid.n[1] * grid.n[2]
        cm = np.ascontiguousarray(coarse_mask, dtype=np.uint8).reshape(-1)
        fm = np.ascontiguousarray(fine_mask, dtype=np.uint8).reshape(-1)
        if cm.size != m or fm.size != m:
            raise ValueError("masks must have n1 n2 n3 entries")
        ci = np.empty(m, dtype=np.int32)
        fi = np.empty(m, dtype=np.int32)
        nc, nf = ctypes.c_longlong(0), ctypes.c_longlong(0)
        _check(L.wvl_region_index(ctypes.byref(grid.c()), cm.ctypes.data, fm.ctypes.data,
                                  ci.ctypes.data, fi.ctypes.data, ctypes.byref(nc),
                                  ctypes.byref(nf)))
        self.lo, self.len = (0, 0, 0), (0, 0, 0)
        if bounds:
            lo = (ctypes.c_int * 3)()
            ln = (ctypes.c_int * 3)()
            _check(L.wvl_region_bounds(ctypes.byref(grid.c()), cm.ctypes.data, fm.ctypes.data,
                                       lo, ln))
            self.lo, self.len = tuple(lo), tuple(ln)
        self.grid = grid
        self.coarse_index = torch.from_numpy(ci).to(device)
        self.fine_index = torch.from_numpy(fi).to(device)
        self.ncoarse, self.nfine = nc.value, nf.value
        self.clen = self.ncoarse + 7 * self.nfine

    def c(self):
        return _Region(self.coarse_index.data_ptr(), self.fine_index.data_ptr(), self.ncoarse,
                       self.nfine, (ctypes.c_int * 3)(*self.lo), (ctypes.c_int * 3)(*self.len))


def _run_region(name, grid, region, prec, norb, device, *ptrs):
    L = lib()
    _declare_region(L)
    st = _stream(device)
    ws, wsb = _workspace(workspace_size(grid, prec, max(norb, 1)), device, st)
    _check(getattr(L, name)(ctypes.byref(grid.c()), ctypes.byref(region.c()), prec, norb,
                            *ptrs, ws, wsb, st))


def synthesis_region(psi_c, grid: Grid, region: Region, out=None, emu=False):
    norb = _norb(psi_c, region.clen) if region.clen else 0
    out = torch.empty((norb, *grid.fine), dtype=psi_c.dtype, device=psi_c.device) if out is None else out
    _dev(psi_c, "psi_c"), _dev(out, "out")
    _run_region("wvl_synthesis_region", grid, region, _prec(psi_c, emu), norb, psi_c.device,
                psi_c.data_ptr(), out.data_ptr())
    return out


def analysis_region(z, grid: Grid, region: Region, out=None, emu=False):
    norb = _norb(z, grid.ncoef)
    out = torch.empty((norb, region.clen), dtype=z.dtype, device=z.device) if out is None else out
    _dev(z, "z"), _dev(out, "out")
    _run_region("wvl_analysis_region", grid, region, _prec(z, emu), norb, z.device, z.data_ptr(),
                out.data_ptr())
    return out


def density_region(psi_c, occ, grid: Grid, region: Region, rho=None, emu=False):
    norb = occ.numel()
    rho = torch.zeros(grid.fine, dtype=torch.float64, device=psi_c.device) if rho is None else rho
    _dev(psi_c, "psi_c"), _dev(occ, "occ"), _dev(rho, "rho")
    _run_region("wvl_density_region", grid, region, _prec(psi_c, emu), norb, psi_c.device,
                psi_c.data_ptr(), occ.data_ptr(), rho.data_ptr())
    return rho


def hpsi_local_region(psi_c, V, occ, grid: Grid, region: Region, rho=None, out=None, emu=False):
    norb = occ.numel()
    if psi_c.numel() != norb * region.clen:
        raise ValueError("psi_c must hold norb region-compressed orbitals")
    out = torch.empty_like(psi_c) if out is None else out
    ek = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    ep = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    for t, nm in ((psi_c, "psi_c"), (V, "V"), (occ, "occ"), (out, "out")):
        _dev(t, nm)
    if rho is not None:
        _dev(rho, "rho")
    _run_region("wvl_hpsi_local_region", grid, region, _prec(psi_c, emu), norb, psi_c.device,
                psi_c.data_ptr(), V.data_ptr(), occ.data_ptr(), out.data_ptr(), _p(rho),
                ek.data_ptr(), ep.data_ptr())
    return out, ek, ep


FREE_PAD = 8   # coarse points of padding per side (WVL_FREE_PAD)


def free_fine(grid: Grid):
    """(N3, N2, N1) of V and rho for free boundary conditions on box `grid`."""
    return tuple(2 * (v + 2 * FREE_PAD) for v in (grid.n[2], grid.n[1], grid.n[0]))


def _declare_free(L):
    if getattr(L, "_free_declared", False):
        return
    Gp = ctypes.POINTER(_Grid)
    L.wvl_free_workspace_size.restype = ctypes.c_int
    L.wvl_free_workspace_size.argtypes = [Gp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_sz)]
    L.wvl_hpsi_local_free.restype = ctypes.c_int
    L.wvl_hpsi_local_free.argtypes = [Gp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp,
                                      _vp, _vp, _vp, _sz, _vp]
    L.wvl_density_free.restype = ctypes.c_int
    L.wvl_density_free.argtypes = [Gp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _sz, _vp]
    L._free_declared = True


def _free_ws(grid, prec, norb, device):
    L = lib()
    _declare_free(L)
    need = _sz(0)
    _check(L.wvl_free_workspace_size(ctypes.byref(grid.c()), prec, max(norb, 1),
                                     ctypes.byref(need)))
    st = _stream(device)
    ws, wsb = _workspace(need.value, device, st)
    return L, ws, wsb, st


def hpsi_local_free(psi_c, V, occ, grid: Grid, rho=None, out=None, emu=False):
    """Free boundary conditions: psi_c on the coarse points of the box,
    V and rho on free_fine(grid).  Returns (hpsi_c, ekin, epot)."""
    norb = _norb(psi_c, grid.ncoef)
    out = torch.empty_like(psi_c) if out is None else out
    ek = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    ep = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    for t, nm in ((psi_c, "psi_c"), (V, "V"), (occ, "occ"), (out, "out")):
        _dev(t, nm)
    if rho is not None:
        _dev(rho, "rho")
    prec = _prec(psi_c, emu)
    L, ws, wsb, st = _free_ws(grid, prec, norb, psi_c.device)
    _check(L.wvl_hpsi_local_free(ctypes.byref(grid.c()), prec, norb, psi_c.data_ptr(),
                                 V.data_ptr(), occ.data_ptr(), out.data_ptr(), _p(rho),
                                 ek.data_ptr(), ep.data_ptr(), ws, wsb, st))
    return out, ek, ep


def density_free(psi_c, occ, grid: Grid, rho=None, emu=False):
    norb = _norb(psi_c, grid.ncoef)
    rho = torch.zeros(free_fine(grid), dtype=torch.float64, device=psi_c.device) if rho is None else rho
    _dev(psi_c, "psi_c"), _dev(occ, "occ"), _dev(rho, "rho")
    prec = _prec(psi_c, emu)
    L, ws, wsb, st = _free_ws(grid, prec, norb, psi_c.device)
    _check(L.wvl_density_free(ctypes.byref(grid.c()), prec, norb, psi_c.data_ptr(),
                              occ.data_ptr(), rho.data_ptr(), ws, wsb, st))
    return rho


def bc_fine(grid: Grid, free_axes):
    """(N3, N2, N1) of V and rho for per-axis free (1) / periodic (0) conditions."""
    fa = tuple(int(v) for v in free_axes)
    return tuple(2 * (grid.n[d] + (2 * FREE_PAD if fa[d] else 0)) for d in (2, 1, 0))


def hpsi_local_bc(psi_c, V, occ, grid: Grid, free_axes, rho=None, out=None, emu=False):
    """Local Hamiltonian with per-axis conditions: free_axes = (x, y, z), 1 =
    free (isolated), 0 = periodic; one free axis gives surface conditions.
    V and rho on bc_fine(grid, free_axes).  Returns (hpsi_c, ekin, epot)."""
    L = lib()
    if not getattr(L, "_bc_declared", False):
        Gp, Ip = ctypes.POINTER(_Grid), ctypes.POINTER(ctypes.c_int)
        L.wvl_bc_workspace_size.restype = ctypes.c_int
        L.wvl_bc_workspace_size.argtypes = [Gp, Ip, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(_sz)]
        L.wvl_hpsi_local_bc.restype = ctypes.c_int
        L.wvl_hpsi_local_bc.argtypes = [Gp, Ip, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                                        _vp, _vp, _vp, _vp, _sz, _vp]
        L._bc_declared = True
    fa = (ctypes.c_int * 3)(*[int(v) for v in free_axes])
    norb = _norb(psi_c, grid.ncoef)
    out = torch.empty_like(psi_c) if out is None else out
    ek = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    ep = torch.empty(norb, dtype=torch.float64, device=psi_c.device)
    for t, nm in ((psi_c, "psi_c"), (V, "V"), (occ, "occ"), (out, "out")):
        _dev(t, nm)
    if rho is not None:
        _dev(rho, "rho")
    prec = _prec(psi_c, emu)
    need = _sz(0)
    _check(L.wvl_bc_workspace_size(ctypes.byref(grid.c()), fa, prec, max(norb, 1),
                                   ctypes.byref(need)))
    st = _stream(psi_c.device)
    ws, wsb = _workspace(need.value, psi_c.device, st)
    _check(L.wvl_hpsi_local_bc(ctypes.byref(grid.c()), fa, prec, norb, psi_c.data_ptr(),
                               V.data_ptr(), occ.data_ptr(), out.data_ptr(), _p(rho),
                               ek.data_ptr(), ep.data_ptr(), ws, wsb, st))
    return out, ek, ep

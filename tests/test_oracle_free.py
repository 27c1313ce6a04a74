"""Pins of the free-boundary oracle: the free-space synthesis is an isometry,
supports grow by the filter extents only, the operator is symmetric, and it
coincides with the periodic operator of a cell padded by 8 coarse points per
side restricted to the box (the interaction range of H is 15 coarse points),
while a cell padded too little shows wrap-around."""
import numpy as np
import pytest

import oracle.free as FR
import oracle.region as RG
import oracle.wavelet as W
from paper_0904_1543_gb300 import inputs


@pytest.mark.parametrize("nc", [1, 2, 5])
def test_free_synthesis_isometry_and_support(nc):
    S = FR.mat_synthesis(nc)
    assert np.max(np.abs(S.T @ S - np.eye(2 * nc))) < 1e-14
    I = FR.fine_range(nc)
    rows = np.nonzero(np.abs(S).sum(1))[0]
    assert I[rows].min() >= -7 and I[rows].max() <= 2 * (nc - 1) + 1 + 8


def _padded_case(n, pad, cfg=101):
    """GPU-style periodic padded cell: coarse n + 2 pad, box region at
    [pad, pad + n) per axis."""
    nn = tuple(v + 2 * pad for v in n)
    cm = np.zeros((nn[2], nn[1], nn[0]), dtype=bool)
    cm[pad:pad + n[2], pad:pad + n[1], pad:pad + n[0]] = True
    V = inputs.gaussian_potential(cfg, 0, nn)
    return nn, cm, V


@pytest.mark.parametrize("n", [(2, 3, 2), (3, 2, 4)])
def test_padded_periodic_equals_free_space(n):
    pad = 8
    nn, cm, Vp = _padded_case(n, pad)
    psi = inputs.orbital(101, 0, n)
    ref = FR.hpsi_local(psi, FR.extend(Vp, n, 2 * pad), 2.0, n)
    got = RG.hpsi_local(psi, Vp, 2.0, nn, cm, cm)
    assert np.max(np.abs(got["hpsi_c"] - ref["hpsi_c"])) < 1e-12 * np.abs(ref["hpsi_c"]).max()
    assert abs(got["ekin"] - ref["ekin"]) < 1e-12 * abs(ref["ekin"])
    assert abs(got["epot"] - ref["epot"]) < 1e-12 * abs(ref["epot"])
    rho_ext = ref["rho"]
    assert np.max(np.abs(got["rho"] - FR.restrict(rho_ext, 2 * pad))) < 1e-14
    # nothing of the density lies outside the padded cell
    assert abs(rho_ext.sum() - got["rho"].sum()) < 1e-13 * rho_ext.sum()


def test_too_little_padding_wraps():
    n = (2, 2, 2)
    pad = 3
    nn, cm, Vp = _padded_case(n, pad)
    psi = inputs.orbital(102, 0, n)
    ref = FR.hpsi_local(psi, FR.extend(Vp, n, 2 * pad), 2.0, n)
    got = RG.hpsi_local(psi, Vp, 2.0, nn, cm, cm)
    assert np.max(np.abs(got["hpsi_c"] - ref["hpsi_c"])) > 1e-6 * np.abs(ref["hpsi_c"]).max()


def test_free_hamiltonian_symmetric():
    n = (2, 2, 3)
    pad = 8
    nn, cm, Vp = _padded_case(n, pad)
    Vx = FR.extend(Vp, n, 2 * pad)
    a = inputs.orbital(103, 0, n)
    b = inputs.orbital(103, 1, n)
    ha = FR.hpsi_local(a, Vx, 2.0, n)["hpsi_c"]
    hb = FR.hpsi_local(b, Vx, 2.0, n)["hpsi_c"]
    assert abs(a @ hb - b @ ha) < 1e-12 * np.abs(ha).max()


def test_mixed_conditions_limits():
    """All axes free = the free-space operator; none free = the periodic
    oracle of oracle/wavelet.py."""
    n = (2, 3, 2)
    psi = inputs.orbital(104, 0, n)
    pad = 8
    nn, cm, Vp = _padded_case(n, pad)
    a = FR.hpsi_local_bc(psi, FR.extend(Vp, n, 2 * pad), 2.0, n, (1, 1, 1))
    b = FR.hpsi_local(psi, FR.extend(Vp, n, 2 * pad), 2.0, n)
    assert np.array_equal(a["hpsi_c"], b["hpsi_c"])
    V = inputs.gaussian_potential(104, 0, n)
    c = FR.hpsi_local_bc(psi, V, 2.0, n, (0, 0, 0))
    d = W.hpsi_local(psi, V, 2.0, n)
    assert np.max(np.abs(c["hpsi_c"] - d["hpsi_c"])) < 1e-13 * np.abs(d["hpsi_c"]).max()


@pytest.mark.parametrize("free_axis", [0, 1, 2])
def test_surface_equals_padding_along_one_axis(free_axis):
    """Surface conditions (one free axis) = the periodic operator on a cell
    padded by 8 coarse points along that axis only, restricted to the box."""
    n = (2, 3, 2)
    pad = 8
    fa = [0, 0, 0]
    fa[free_axis] = 1
    nn = tuple(v + (2 * pad if fa[d] else 0) for d, v in enumerate(n))
    cm = np.zeros((nn[2], nn[1], nn[0]), dtype=bool)
    o = [pad if fa[d] else 0 for d in range(3)]
    cm[o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] = True
    Vp = inputs.gaussian_potential(105, 0, nn)
    psi = inputs.orbital(105, 0, n)
    ref = FR.hpsi_local_bc(psi, FR.extend_bc(Vp, n, 2 * pad, fa), 2.0, n, fa)
    got = RG.hpsi_local(psi, Vp, 2.0, nn, cm, cm)
    assert np.max(np.abs(got["hpsi_c"] - ref["hpsi_c"])) < 1e-12 * np.abs(ref["hpsi_c"]).max()
    assert abs(got["epot"] - ref["epot"]) < 1e-12 * abs(ref["epot"])
    assert np.max(np.abs(got["rho"] - FR.restrict_bc(ref["rho"], n, 2 * pad, fa))) < 1e-14

"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the wavelet method: it only draws numbers.
Both the CUDA library and the CPU oracle receive the arrays built here, so
they see bit-identical inputs.

Recipe (the paper's ZnO workloads need its whole DFT code and structures; these
synthetic inputs stand in for them):
* generator: SplitMix64 in counter form, state_i = seed + (i + 1) * 0x9E3779B97F4A7C15,
  53-bit uniforms u = (z >> 11) * 2^-53;
* seed(cfg, stream) = 9041543 + 1000 * cfg + stream;
* orbital o draws its 8 n1 n2 n3 coefficients from stream o, uniform in
  [-1, 1), then is scaled to unit 2-norm;
* cell c draws its potential from stream 100000 + c: 8 Gaussians, each with a
  centre uniform in the fine cell (3 draws), a width sigma uniform in [2, 6]
  fine spacings and a depth uniform in [-2, 0];
  V(r) = sum_g d_g exp(-|r - R_g|^2 / (2 sigma_g^2)) on the fine grid points,
  with the minimum-image distance of the periodic cell;
* occupations are 2.0.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 9041543
V_STREAM = 100000


def seed(cfg: int, stream: int) -> int:
    return BASE_SEED + 1000 * cfg + stream


def splitmix64(seed_value: int, count: int, offset: int = 0) -> np.ndarray:
    """count 64-bit outputs of the counter-form SplitMix64 stream."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed_value & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed_value: int, count: int, lo: float = 0.0, hi: float = 1.0,
            offset: int = 0) -> np.ndarray:
    u = (splitmix64(seed_value, count, offset) >> np.uint64(11)).astype(np.float64)
    u *= 2.0 ** -53
    return lo + (hi - lo) * u


def orbital(cfg: int, o: int, n) -> np.ndarray:
    """Unit-norm compressed coefficients (8 n1 n2 n3 values) of orbital o."""
    m = 8 * n[0] * n[1] * n[2]
    c = uniform(seed(cfg, o), m, -1.0, 1.0)
    return c / np.sqrt(np.dot(c, c))


def orbitals(cfg: int, norb: int, n, first: int = 0) -> np.ndarray:
    return np.stack([orbital(cfg, first + o, n) for o in range(norb)])


def gaussian_potential(cfg: int, cell: int, n, ngauss: int = 8) -> np.ndarray:
    """Sum of ngauss Gaussians on the fine grid (N3, N2, N1) = 2 n."""
    N = (2 * n[0], 2 * n[1], 2 * n[2])
    u = uniform(seed(cfg, V_STREAM + cell), 5 * ngauss)
    V = np.zeros((N[2], N[1], N[0]))
    for k in range(ngauss):
        R = [u[5 * k + d] * N[d] for d in range(3)]
        sigma = 2.0 + 4.0 * u[5 * k + 3]
        depth = -2.0 * u[5 * k + 4]
        f = []
        for d in range(3):
            x = np.arange(N[d], dtype=np.float64) - R[d]
            x -= N[d] * np.round(x / N[d])          # minimum image
            f.append(np.exp(-x * x / (2.0 * sigma * sigma)))
        V += depth * f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    return V


def orbitals_device(cfg: int, norb: int, n, device, dtype=None):
    """Large throughput-only batches drawn on the device: the same
    distribution as orbitals() (uniform[-1, 1), unit norm per orbital) from
    torch's seeded Philox generator, seeded with seed(cfg, 0).  Not the
    SplitMix64 stream: used only where no oracle comparison needs the
    whole batch (callers copy back the orbitals they check)."""
    return vectors_device(cfg, norb, 8 * n[0] * n[1] * n[2], device, dtype)


def vectors_device(cfg: int, norb: int, length: int, device, dtype=None):
    """norb unit-norm vectors of `length` uniform[-1, 1) entries drawn on the
    device (torch Philox, seed(cfg, 0)); e.g. region-compressed orbitals."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed(cfg, 0))
    x = torch.rand((norb, length), generator=gen, device=device, dtype=torch.float64)
    x = 2.0 * x - 1.0
    x /= torch.linalg.vector_norm(x, dim=1, keepdim=True)
    return x if dtype is None else x.to(dtype)


def random_field(cfg: int, stream: int, shape) -> np.ndarray:
    """Uniform[-1, 1) array of the given shape (per-pass sweeps)."""
    return uniform(seed(cfg, stream), int(np.prod(shape)), -1.0, 1.0).reshape(shape)


def sphere_masks(n, centre, r_coarse, r_fine):
    """Coarse and fine localisation regions shaped as balls around `centre`
    (coarse grid units, minimum-image distance): boolean (n3, n2, n1) masks."""
    idx = np.meshgrid(*[np.arange(v) for v in (n[2], n[1], n[0])], indexing="ij")
    d2 = np.zeros(idx[0].shape)
    for ax, (v, c) in enumerate(zip((n[2], n[1], n[0]), (centre[2], centre[1], centre[0]))):
        x = idx[ax] - c
        x = x - v * np.round(x / v)
        d2 += x * x
    return d2 <= r_coarse ** 2, d2 <= r_fine ** 2

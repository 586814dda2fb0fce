"""Seeded synthetic inputs for the MPR gap-filling method.

This module holds none of the method's arithmetic: it only draws the data that both the CUDA
library and the FP64 oracle are fed. The workload follows Sec. 3 of the paper: Gaussian data
Z ~ N(m = 50, sigma = 10) with the exponential covariance of Eq. 3,
G_Z(h) = sigma^2 exp(-kappa |h|), kappa = 0.2 (the Whittle-Matern family at nu = 1/2), on L x L
grids, with a fraction p of the sites removed at random and kept as the truth.

Fields are drawn by circulant embedding: the covariance is laid out on a (2Lx) x (2Ly) torus with
minimum-image distances, its FFT gives the eigenvalues of the circulant matrix (negatives clamped
to 0), and the FFT of sqrt(eigenvalue / M) times complex white noise has real part with the
target covariance. ``periodic=True`` embeds on the Lx x Ly torus itself, which is cheaper and
adequate when the correlation length 1/kappa is much smaller than the grid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _fft2(a, device):
    if device is None:
        return np.fft.fft2(a)
    import torch

    t = torch.from_numpy(a).to(device)
    return torch.fft.fft2(t).cpu().numpy()


def gaussian_field(Lx: int, Ly: int, seed: int, mean: float = 50.0, sigma: float = 10.0,
                   kappa: float = 0.2, periodic: bool = False, device=None) -> np.ndarray:
    """Gaussian random field (Ly, Lx) float64 with covariance sigma^2 exp(-kappa |h|)."""
    Mx, My = (Lx, Ly) if periodic else (2 * Lx, 2 * Ly)
    ix = np.arange(Mx, dtype=np.float64)
    iy = np.arange(My, dtype=np.float64)
    dx = np.minimum(ix, Mx - ix)
    dy = np.minimum(iy, My - iy)
    r = np.sqrt(dy[:, None] ** 2 + dx[None, :] ** 2)
    c = (sigma * sigma) * np.exp(-kappa * r)
    lam = np.real(_fft2(c, device))
    lam = np.maximum(lam, 0.0)
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((My, Mx)) + 1j * rng.standard_normal((My, Mx))
    y = _fft2(np.sqrt(lam / (Mx * My)) * xi, device)
    return np.ascontiguousarray(mean + np.real(y)[:Ly, :Lx])


def removal_mask(Lx: int, Ly: int, p: float, seed: int) -> np.ndarray:
    """uint8 (Ly, Lx): 1 = measured, 0 = removed. Exactly round(p * N) sites are removed."""
    n = Lx * Ly
    k = int(round(p * n))
    rng = np.random.default_rng(seed)
    mask = np.ones(n, dtype=np.uint8)
    mask[rng.permutation(n)[:k]] = 0
    return mask.reshape(Ly, Lx)


@dataclass
class Problem:
    Lx: int
    Ly: int
    p: float
    kappa: float
    z: np.ndarray       # (Ly, Lx) complete field (the truth)
    mask: np.ndarray    # (Ly, Lx) uint8, 1 = measured


def make_problem(Lx: int, Ly: int, p: float, field_seed: int, mask_seed: int,
                 kappa: float = 0.2, periodic: bool = False, device=None) -> Problem:
    z = gaussian_field(Lx, Ly, field_seed, kappa=kappa, periodic=periodic, device=device)
    return Problem(Lx, Ly, p, kappa, z, removal_mask(Lx, Ly, p, mask_seed))


def batch_shapes(n: int, seed: int, L_min: int = 64, L_max: int = 1024, max_aspect: float = 4.0,
                 ps=(0.33, 0.66, 0.9), kappa_range=(0.05, 0.5)):
    """Sizes of a batch of independent problems: side L log-uniform on [L_min, L_max], aspect
    ratio log-uniform on [1/max_aspect, max_aspect], removal fraction drawn from ``ps``,
    kappa uniform on ``kappa_range``. Returns a list of (Lx, Ly, p, kappa)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        L = math.exp(rng.uniform(math.log(L_min), math.log(L_max)))
        a = math.exp(rng.uniform(-math.log(max_aspect), math.log(max_aspect)))
        Lx = max(2, int(round(L * math.sqrt(a))))
        Ly = max(2, int(round(L / math.sqrt(a))))
        p = float(ps[int(rng.integers(len(ps)))])
        kappa = float(rng.uniform(*kappa_range))
        out.append((Lx, Ly, p, kappa))
    return out


def make_batch(n: int, seed: int, **kw):
    """n independent problems with the shapes of ``batch_shapes``; problem i uses field seed
    1000*seed + i and mask seed 1000*seed + 500 + i."""
    probs = []
    for i, (Lx, Ly, p, kappa) in enumerate(batch_shapes(n, seed, **kw)):
        probs.append(make_problem(Lx, Ly, p, 1000 * seed + i, 1000 * seed + 500 + i, kappa=kappa,
                                  periodic=max(Lx, Ly) > 512))
    return probs

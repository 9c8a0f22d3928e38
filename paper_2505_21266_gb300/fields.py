"""Seeded synthetic scalar fields shaped like the paper's workloads.

These generators hold none of the method's arithmetic; they only produce
float32 inputs.  Everything is bit-reproducible across devices: the Gaussian
factors are evaluated in float64 with numpy on the host (separable, so only
nx + ny + nz exponentials per Gaussian) and accumulated on the target device
with plain float32 multiplies and adds in a fixed order, and the uniform noise
comes from a counter-based integer hash of (seed, vertex offset) -- the
"lowbias32" finaliser (Chris Wellons' hash-prospector, published constants)
applied twice -- whose top 24 bits give an exact float32 in [0, 1).

Fields are returned indexed [z, y, x] (x fastest).
"""
from __future__ import annotations

import numpy as np
import torch

_M32 = 0xFFFFFFFF


def _lowbias32(x: torch.Tensor) -> torch.Tensor:
    # x holds values in [0, 2^32) in int64; products wrap but are masked
    x = x ^ (x >> 16)
    x = (x * 0x7FEB352D) & _M32
    x = x ^ (x >> 15)
    x = (x * 0x846CA68B) & _M32
    x = x ^ (x >> 16)
    return x


def uniform01_at(i: torch.Tensor, seed: int) -> torch.Tensor:
    """float32 U[0,1) for the vertex offsets i (int64 tensor)."""
    s1 = (seed * 0x9E3779B9 + 0x632BE5AB) & _M32
    s2 = (seed * 0x85EBCA6B + 0x1B873593) & _M32
    h = _lowbias32(_lowbias32((i & _M32) ^ s1) ^ (((i >> 32) + s2) & _M32))
    return (h >> 8).to(torch.float32) * (1.0 / 16777216.0)


def uniform01(shape, seed: int, device="cpu", chunk: int = 1 << 26) -> torch.Tensor:
    """float32 U[0,1) per vertex, identical on every device for a given seed."""
    nz, ny, nx = shape
    n = nx * ny * nz
    out = torch.empty(n, dtype=torch.float32, device=device)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        out[lo:hi] = uniform01_at(torch.arange(lo, hi, dtype=torch.int64, device=device), seed)
    return out.view(nz, ny, nx)


def mixture_crop(n: int, crop: int, n_gauss: int, sigma, noise: float, seed: int):
    """The [0, crop)^3 corner of gaussian_mixture((n, n, n), ...), evaluated on
    the host alone with the same arithmetic (bit-identical values)."""
    c, s, a = gaussian_params(n_gauss, sigma, seed)
    ax = np.arange(n, dtype=np.float64)[:crop] / max(n - 1, 1)
    field = torch.zeros((crop, crop, crop), dtype=torch.float32)
    for i in range(n_gauss):
        g = [np.exp(-((ax - c[i, k]) ** 2) / (2.0 * s[i] ** 2)) for k in range(3)]
        gx = torch.from_numpy(g[0].astype(np.float32))
        gy = torch.from_numpy(g[1].astype(np.float32))
        gz = torch.from_numpy((a[i] * g[2]).astype(np.float32))
        zy = gz[:, None] * gy[None, :]
        field += zy[:, :, None] * gx[None, None, :]
    if noise > 0:
        r = torch.arange(crop, dtype=torch.int64)
        idx = r[None, None, :] + n * (r[None, :, None] + n * r[:, None, None])
        field += uniform01_at(idx.reshape(-1), seed + 7919).view(crop, crop, crop) * np.float32(noise)
    return field


def gaussian_params(n_gauss: int, sigma, seed: int):
    """Centres U[0,1]^3, sigma U[sigma], amplitude U[-1,1] from numpy PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.random((n_gauss, 3))
    s = rng.uniform(sigma[0], sigma[1], n_gauss)
    a = rng.uniform(-1.0, 1.0, n_gauss)
    return c, s, a


def gaussian_mixture(shape, n_gauss: int, sigma, noise: float, seed: int, device="cpu"):
    """sum_i a_i exp(-|p - c_i|^2 / (2 s_i^2)) + U[0, noise), p in [0,1]^3
    with p = (x/(nx-1), y/(ny-1), z/(nz-1))."""
    nz, ny, nx = shape
    c, s, a = gaussian_params(n_gauss, sigma, seed)
    axes = [np.arange(m, dtype=np.float64) / max(m - 1, 1) for m in (nx, ny, nz)]
    field = torch.zeros((nz, ny, nx), dtype=torch.float32, device=device)
    for i in range(n_gauss):
        g = [np.exp(-((axes[k] - c[i, k]) ** 2) / (2.0 * s[i] ** 2)) for k in range(3)]
        gx = torch.from_numpy(g[0].astype(np.float32)).to(device)
        gy = torch.from_numpy(g[1].astype(np.float32)).to(device)
        gz = torch.from_numpy((a[i] * g[2]).astype(np.float32)).to(device)
        zy = gz[:, None] * gy[None, :]
        field += zy[:, :, None] * gx[None, None, :]
    if noise > 0:
        field += uniform01(shape, seed + 7919, device) * np.float32(noise)
    return field


def quantized_noise(shape, levels: int, seed: int, device="cpu"):
    """floor(U[0,1) * levels) / levels: massive ties ("Random"-like)."""
    u = uniform01(shape, seed, device)
    return torch.floor(u * levels) / levels


# ---- the five workloads (sizes as in the benchmark configurations) --------

def config1(seed: int = 0, device="cpu", n: int = 64):
    """64^3, 16 Gaussians (sigma in [0.05, 0.2]) + U[0, 1e-3)."""
    return gaussian_mixture((n, n, n), 16, (0.05, 0.2), 1e-3, seed, device)


def config2(seed: int = 0, device="cpu", n: int = 512):
    """512^3 i.i.d. U[0,1) quantised to 256 levels."""
    return quantized_noise((n, n, n), 256, seed, device)


def config3(seed: int = 0, device="cpu", n: int = 1024):
    """1024^3, 256 Gaussians (sigma in [0.01, 0.1]) + U[0, 1e-2)."""
    return gaussian_mixture((n, n, n), 256, (0.01, 0.1), 1e-2, seed, device)


def config4(seed: int = 0, device="cpu", n: int = 128):
    """128^3, 32 Gaussians (sigma in [0.05, 0.2]) + U[0, 1e-4)."""
    return gaussian_mixture((n, n, n), 32, (0.05, 0.2), 1e-4, seed, device)


def batch_shapes(count: int = 256, lo: int = 32, hi: int = 256, seed: int = 0):
    """Each axis uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [tuple(int(v) for v in rng.integers(lo, hi + 1, 3)) for _ in range(count)]


def batch_field(i: int, shape, seed: int = 0, device="cpu"):
    """Field i of the batch: even i -> Gaussian mixture, odd i -> U[0,1)."""
    if i % 2 == 0:
        return gaussian_mixture(shape, 16, (0.05, 0.2), 1e-3, seed * 1000 + i, device)
    return uniform01(shape, seed * 1000 + i, device)

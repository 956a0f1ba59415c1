"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module only *builds* input tensors.  It contains none of the compressor's
arithmetic (no Gram matrix, eigensolve, rank choice, projection or
quantization); both the CUDA path and the CPU oracle consume the arrays it
returns, byte for byte.

The workloads stand in for the paper's datasets (Section 6.1: Foot, Moffett-Field,
Isotropic-PT/V, ...), none of which is available here:

* ``lowrank_tucker``  -- 64^3 float64 tensor with exact multilinear rank (8,8,8),
  core entries N(0,1) * 2^-((i+j+k)/4), orthonormal factors (QR of a Gaussian),
  plus i.i.d. Gaussian noise (relative or absolute level, see the docstring).
* ``gaussian_bumps``  -- 256^3 float32 smooth field, a sum of 32 isotropic
  Gaussian bumps on the unit grid (a Foot-sized smooth volume).
* ``hyperspectral``   -- 512x512x224 float32 cube: 12 smooth positive spectra
  mixed by spatially smooth abundance maps (softmax of low-passed Gaussian
  noise), plus 1% Gaussian noise (a Moffett-Field-shaped cube).
* ``batched_lowrank`` -- many small uneven tensors built like ``lowrank_tucker``.
* ``turbulence``      -- n^3 float32 turbulence-like field: every wavevector
  k != 0 of the grid with amplitude |k|^(-5/3) and a uniform random phase,
  made real through the half spectrum (irfftn), normalised to RMS 1 (stands in
  for the Isotropic-PT/V fields).  Built with torch on a CUDA device for the
  1024^3 size (seeded Philox), with NumPy for small sizes.

Every generator uses ``numpy.random.default_rng(seed)`` (PCG64), so the same
seed gives the same bytes on x86 and on Arm.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lowrank_tucker",
    "gaussian_bumps",
    "hyperspectral",
    "batched_lowrank",
    "random_core",
    "turbulence",
    "WORKLOADS",
]


def _orthonormal(rng: np.random.Generator, n: int, r: int) -> np.ndarray:
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def lowrank_tucker(shape=(64, 64, 64), ranks=(8, 8, 8), noise="relative",
                   noise_level=1e-3, seed=1000, dtype=np.float64) -> np.ndarray:
    """Tensor with a known multilinear rank plus Gaussian noise.

    ``noise="relative"`` adds N(0, (noise_level * RMS(signal))^2) noise,
    ``noise="absolute"`` adds N(0, noise_level^2) noise and ``noise=None`` adds
    none (exact multilinear rank ``ranks``).
    """
    rng = np.random.default_rng(seed)
    d = len(shape)
    idx = np.indices(ranks).sum(axis=0).astype(np.float64)
    core = rng.standard_normal(ranks) * np.power(2.0, -idx / 4.0)
    factors = [_orthonormal(rng, shape[i], ranks[i]) for i in range(d)]
    x = core
    for i in range(d):
        # x <- factors[i] applied along axis i (synthetic construction only)
        x = np.moveaxis(np.tensordot(factors[i], x, axes=([1], [i])), 0, i)
    if noise is not None:
        if noise == "relative":
            sigma = noise_level * float(np.sqrt(np.mean(x * x)))
        elif noise == "absolute":
            sigma = noise_level
        else:
            raise ValueError(f"unknown noise mode {noise!r}")
        x = x + sigma * rng.standard_normal(shape)
    return np.ascontiguousarray(x, dtype=dtype)


def gaussian_bumps(n=256, nbumps=32, seed=1001, dtype=np.float32) -> np.ndarray:
    """Sum of ``nbumps`` isotropic Gaussian bumps on the grid x_i = i/(n-1).

    Centres U[0,1]^3, widths U[0.02, 0.2], amplitudes N(0,1).  Each bump is
    separable, so the field is built from rank-one terms in float64 and cast.
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(nbumps, 3))
    widths = rng.uniform(0.02, 0.2, size=nbumps)
    amps = rng.standard_normal(nbumps)
    grid = np.arange(n, dtype=np.float64) / (n - 1)
    prof = [np.exp(-((grid[None, :] - centres[:, a, None]) ** 2) / (2.0 * widths[:, None] ** 2))
            for a in range(3)]
    out = np.zeros((n, n, n), dtype=np.float64)
    for b in range(nbumps):
        out += amps[b] * np.multiply.outer(np.multiply.outer(prof[0][b], prof[1][b]), prof[2][b])
    return np.ascontiguousarray(out, dtype=dtype)


def hyperspectral(rows=512, cols=512, bands=224, nend=12, noise_level=0.01,
                  seed=1002, dtype=np.float32) -> np.ndarray:
    """Linear mixing model cube (rows, cols, bands), band index fastest."""
    rng = np.random.default_rng(seed)
    spectra = np.exp(np.cumsum(0.05 * rng.standard_normal((nend, bands)), axis=1))
    spectra /= spectra.max(axis=1, keepdims=True)
    fields = rng.standard_normal((nend, rows, cols))
    fy = np.fft.fftfreq(rows)[:, None]
    fx = np.fft.fftfreq(cols)[None, :]
    sig = 16.0  # low-pass Gaussian, std in pixels
    filt = np.exp(-2.0 * (np.pi * sig) ** 2 * (fy ** 2 + fx ** 2))
    fields = np.real(np.fft.ifft2(np.fft.fft2(fields) * filt))
    fields = (fields - fields.mean(axis=(1, 2), keepdims=True)) / fields.std(axis=(1, 2), keepdims=True)
    w = np.exp(fields - fields.max(axis=0, keepdims=True))
    w /= w.sum(axis=0, keepdims=True)
    cube = np.einsum("erc,eb->rcb", w, spectra)
    rms = float(np.sqrt(np.mean(cube * cube)))
    cube = cube + noise_level * rms * rng.standard_normal(cube.shape)
    return np.ascontiguousarray(cube, dtype=dtype)


def batched_lowrank(count=512, lo=16, hi=96, rlo=2, rhi=12, seed=1003, dtype=np.float32):
    """List of (tensor, rel_eps) pairs of uneven shapes, built like ``lowrank_tucker``."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        shape = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
        ranks = tuple(int(min(rng.integers(rlo, rhi + 1), shape[i])) for i in range(3))
        eps = float(rng.choice([1e-2, 1e-3, 1e-4]))
        x = lowrank_tucker(shape, ranks, noise="relative", noise_level=1e-3,
                           seed=seed * 1000 + j, dtype=dtype)
        out.append((x, eps))
    return out


def random_core(shape, decay=0.25, seed=7, dtype=np.float64) -> np.ndarray:
    """Core-like array with the ST-HOSVD 'hot corner' magnitude decay."""
    rng = np.random.default_rng(seed)
    idx = np.indices(shape).sum(axis=0).astype(np.float64)
    return np.ascontiguousarray(rng.standard_normal(shape) * np.power(2.0, -decay * idx), dtype=dtype)


def _turbulence_spectrum_np(n, rng):
    k = np.fft.fftfreq(n) * n
    kr = np.fft.rfftfreq(n) * n
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (-5.0 / 3.0)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=kk.shape)
    return amp * np.exp(1j * phase)


def turbulence(n=1024, seed=1004, device=None, dtype=np.float32):
    """Real n^3 field with an |k|^(-5/3) amplitude spectrum and random phases,
    RMS 1.  device=None: NumPy (small n, returns an ndarray); a torch CUDA
    device: built there with a seeded generator (returns a torch tensor)."""
    if device is None:
        rng = np.random.default_rng(seed)
        x = np.fft.irfftn(_turbulence_spectrum_np(n, rng), s=(n, n, n))
        x /= np.sqrt(np.mean(x * x))
        return np.ascontiguousarray(x, dtype=dtype)
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    k = torch.fft.fftfreq(n, device=device) * n
    kr = torch.fft.rfftfreq(n, device=device) * n
    kk = torch.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2)
    amp = torch.where(kk > 0, kk.clamp_min(1e-30) ** (-5.0 / 3.0), torch.zeros_like(kk))
    del kk
    phase = torch.rand(amp.shape, generator=g, device=device) * (2.0 * np.pi)
    spec = torch.polar(amp, phase)
    del amp, phase
    x = torch.fft.irfftn(spec, s=(n, n, n))
    del spec
    x /= torch.sqrt(torch.mean(x.double() * x.double())).float()
    return x.contiguous()


WORKLOADS = {
    "lowrank64_f64": dict(fn=lowrank_tucker, kwargs={}, rel_eps=1e-2),
    "bumps256_f32": dict(fn=gaussian_bumps, kwargs={}, rel_eps=1e-3),
    "hyperspectral512x512x224_f32": dict(fn=hyperspectral, kwargs={}, rel_eps=1e-2),
}

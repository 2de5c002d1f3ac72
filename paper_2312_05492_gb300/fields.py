"""Seeded synthetic float32 3-D fields shaped like the paper's workloads.

The paper evaluates on six simulation datasets (Table III: JHTDB, Miranda,
Nyx, QMCPack, RTM, S3D) that are not available here; these generators stand
in for them with matching shapes and comparable statistics.  This module
holds no part of the compression method: it only draws inputs, and both the
CUDA path and the CPU oracle consume what it returns.

All generators are deterministic for a given seed on a given device type.
Fields are returned as contiguous float32 torch tensors shaped (nz, ny, nx).
"""
from __future__ import annotations

import hashlib
import math

import torch


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def _kmag(shape, device, dtype):
    nz, ny, nx = shape
    kz = torch.fft.fftfreq(nz, device=device, dtype=dtype)
    ky = torch.fft.fftfreq(ny, device=device, dtype=dtype)
    kx = torch.fft.rfftfreq(nx, device=device, dtype=dtype)
    return torch.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)


def grf(shape, beta: float, seed: int, device="cpu", fft_dtype=torch.float64) -> torch.Tensor:
    """Gaussian random field with power spectrum ~ |k|^-beta, zero mean, unit variance.

    White N(0,1) noise (CPU generator, so the draw does not depend on the
    device) is shaped in Fourier space by |k|^(-beta/2) with the k = 0 mode
    removed, then normalised.
    """
    shape = tuple(int(s) for s in shape)
    noise = torch.randn(shape, generator=_gen(seed), dtype=torch.float32)
    noise = noise.to(device=device, dtype=fft_dtype)
    spec = torch.fft.rfftn(noise)
    del noise
    k = _kmag(shape, spec.device, fft_dtype)
    amp = torch.where(k > 0, k.clamp_min(1e-30) ** (-beta / 2.0), torch.zeros_like(k))
    spec *= amp
    del k, amp
    f = torch.fft.irfftn(spec, s=shape)
    del spec
    f -= f.mean()
    std = f.std()
    if std > 0:
        f /= std
    return f.to(torch.float32).contiguous()


def lognormal(shape, beta: float, seed: int, device="cpu", fft_dtype=torch.float64) -> torch.Tensor:
    """exp of a unit-variance GRF: heavy-tailed, positive, density-like (Nyx-style)."""
    g = grf(shape, beta, seed, device=device, fft_dtype=fft_dtype)
    return torch.exp(g).contiguous()


def sines(shape, seed: int, n_waves: int = 32, kmax: int = 16, noise_frac: float = 0.01,
          device="cpu") -> torch.Tensor:
    """Sum of random-phase plane sine waves with integer wave vectors (<= kmax
    cycles per axis) and U(0.5, 1) amplitudes, plus Gaussian noise of std
    noise_frac times the clean field's std (RTM-like oscillatory data)."""
    shape = tuple(int(s) for s in shape)
    g = _gen(seed)
    kv = torch.randint(-kmax, kmax + 1, (n_waves, 3), generator=g).to(torch.float64)
    amp = 0.5 + 0.5 * torch.rand(n_waves, generator=g, dtype=torch.float64)
    phase = 2.0 * math.pi * torch.rand(n_waves, generator=g, dtype=torch.float64)
    noise = torch.randn(shape, generator=g, dtype=torch.float32)
    nz, ny, nx = shape
    z = torch.arange(nz, device=device, dtype=torch.float64)[:, None, None] / nz
    y = torch.arange(ny, device=device, dtype=torch.float64)[None, :, None] / ny
    x = torch.arange(nx, device=device, dtype=torch.float64)[None, None, :] / nx
    f = torch.zeros(shape, device=device, dtype=torch.float64)
    for w in range(n_waves):
        kz, ky, kx = (float(v) for v in kv[w])
        f += float(amp[w]) * torch.sin(2.0 * math.pi * (kz * z + ky * y + kx * x) + float(phase[w]))
    f += noise_frac * f.std() * noise.to(device=device, dtype=torch.float64)
    return f.to(torch.float32).contiguous()


def shocks(shape, seed: int, n_steps: int = 8, beta: float = 3.0, step_amp: float = 10.0,
           device="cpu", fft_dtype=torch.float32) -> torch.Tensor:
    """Piecewise-smooth field: GRF(beta) plus n_steps planar step discontinuities
    H(n . r - c) of amplitude +-step_amp * std (random unit normals n, offsets c
    uniform inside the box).  Outlier-heavy at tight bounds."""
    shape = tuple(int(s) for s in shape)
    f = grf(shape, beta, seed, device=device, fft_dtype=fft_dtype)
    g = _gen(seed + 1000003)
    std = float(f.std())
    nz, ny, nx = shape
    z = torch.arange(nz, device=device, dtype=torch.float32)[:, None, None]
    y = torch.arange(ny, device=device, dtype=torch.float32)[None, :, None]
    x = torch.arange(nx, device=device, dtype=torch.float32)[None, None, :]
    for _ in range(n_steps):
        nrm = torch.randn(3, generator=g, dtype=torch.float64)
        nrm = nrm / nrm.norm()
        point = torch.rand(3, generator=g, dtype=torch.float64) * torch.tensor([nz, ny, nx], dtype=torch.float64)
        c = float((nrm * point).sum())
        sign = 1.0 if float(torch.rand(1, generator=g)) < 0.5 else -1.0
        proj = float(nrm[0]) * z + float(nrm[1]) * y + float(nrm[2]) * x
        f += (proj > c).to(torch.float32) * (sign * step_amp * std)
    return f.contiguous()


def sha256(t: torch.Tensor) -> str:
    """Digest of a field's bytes, recorded next to benchmark results."""
    return hashlib.sha256(t.detach().contiguous().cpu().numpy().tobytes()).hexdigest()


# Named workloads (sizes and statistics of the paper's datasets, Table III).
def workload(name: str, device="cpu") -> tuple[torch.Tensor, dict]:
    if name == "grf64":
        return grf((64, 64, 64), 3.0, 0, device=device), {"field": "GRF k^-3", "seed": 0}
    if name == "lognormal512":
        return lognormal((512, 512, 512), 11.0 / 3.0, 1, device=device), {"field": "exp(GRF k^-11/3)", "seed": 1}
    if name == "batch_smooth":
        return grf((100, 500, 500), 4.0, 2, device=device), {"field": "GRF k^-4", "seed": 2}
    if name == "batch_turbulent":
        return grf((256, 384, 384), 5.0 / 3.0, 3, device=device), {"field": "GRF k^-5/3", "seed": 3}
    if name == "batch_sines":
        return sines((449, 449, 235), 4, device=device), {"field": "32 plane sines + 1% noise", "seed": 4}
    if name == "shocks1024":
        return (shocks((1024, 1024, 1024), 6, device=device, fft_dtype=torch.float32),
                {"field": "GRF k^-3 + 8 planar steps", "seed": 6})
    raise KeyError(name)

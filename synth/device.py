"""The seeded synthetic inputs of ``synth.fields`` drawn on a CUDA device.

For workloads too large to draw on the host in a benchmark's set-up time
(2048^3: 4.3e9 spectral modes).  Same recipes and the same counter-based
SplitMix64 draws as ``synth.fields`` (the integer draws are bit for bit the
same); the floating-point steps run in FP64 on the device, so values agree
with the host generator to FP64 rounding.  Like ``synth.fields`` this module
holds no transform arithmetic; it uses torch only as an array library.
"""
from __future__ import annotations

import math

import numpy as np

from .fields import _plane0_energy, nyquist_mask, signed_wavenumbers

_GOLD = -7046029254386353131  # 0x9E3779B97F4A7C15 as a signed 64-bit integer
_M1 = -4658895280553007687    # 0xBF58476D1CE4E5B9
_M2 = -7723592293110705685    # 0x94D049BB133111EB


def _signed(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def _lshr(z, k):
    """Logical right shift of int64 tensors."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _splitmix64(z):
    z = z + _GOLD
    z = (z ^ _lshr(z, 30)) * _M1
    z = (z ^ _lshr(z, 27)) * _M2
    return z ^ _lshr(z, 31)


def uniform01(seed: int, counters):
    """synth.fields.uniform01 for an int64 tensor of counters: FP64 in [0, 1)."""
    import torch
    z = _splitmix64(counters ^ _signed(seed * 0x9E3779B97F4A7C15))
    return _lshr(z, 11).to(torch.float64) * (2.0 ** -53)


def uniform_field(shape, seed: int, device="cuda", dtype=None):
    """synth.fields.uniform_field on the device (2u - 1), FP32 unless dtype says otherwise."""
    import torch
    dtype = dtype or torch.float32
    n = int(np.prod(shape))
    out = torch.empty(n, dtype=dtype, device=device)
    chunk = 1 << 27
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        u = uniform01(seed, torch.arange(a, b, dtype=torch.int64, device=device))
        out[a:b] = (2.0 * u - 1.0).to(dtype)
    return out.view(shape)


def _energy_shape(k, k0: float = 4.0, kc: float = 8.0):
    import torch
    ekc = kc ** 4 * math.exp(-2.0 * (kc / k0) ** 2)
    low = k ** 4 * torch.exp(-2.0 * (k / k0) ** 2)
    high = ekc * torch.where(k > 0, k / kc, torch.ones_like(k)) ** (-5.0 / 3.0)
    return torch.where(k < kc, low, high)


def spectral_velocity(n0: int, n1: int, n2: int, seed: int, component: int = 0, device="cuda",
                      plane_chunk: int = 8):
    """synth.fields.spectral_velocity(n0, n1, n2, seed, components=(component,))[0]
    as a complex64 tensor (n0, n1, n2/2+1) on the device.

    Two sweeps over chunks of planes: the first sums the energies that fix the
    common normalisation (all three components, k2 >= 1; the k2 = 0 plane is
    counted after its Hermitian rebuild by the host helper), the second draws
    the requested component again and stores it already normalised, so the
    FP64 values are rounded to complex64 once."""
    import torch
    if n2 % 2:
        raise ValueError("n2 must be even")
    H = n2 // 2 + 1
    dev = torch.device(device)
    f64 = torch.float64
    k0v = torch.from_numpy(signed_wavenumbers(n0).astype(np.float64)).to(dev)
    k1v = torch.from_numpy(signed_wavenumbers(n1).astype(np.float64)).to(dev)
    k2v = torch.arange(H, dtype=f64, device=dev)
    ny0 = torch.from_numpy(nyquist_mask(n0)).to(dev)
    ny1 = torch.from_numpy(nyquist_mask(n1)).to(dev)
    ny2 = torch.zeros(H, dtype=torch.bool, device=dev)
    ny2[H - 1] = True
    nmin = min(n0, n1, n2)
    w = torch.full((H,), 2.0, dtype=f64, device=dev)
    w[0] = 0.0  # the k2 = 0 plane is counted separately (after its rebuild)
    w[H - 1] = 1.0
    j1 = torch.arange(n1, dtype=torch.int64, device=dev)[None, :, None]
    j2 = torch.arange(H, dtype=torch.int64, device=dev)[None, None, :]

    def draw(a0, b0):
        K0 = k0v[a0:b0, None, None]
        K1 = k1v[None, :, None]
        K2 = k2v[None, None, :]
        kk = K0 * K0 + K1 * K1 + K2 * K2
        zero = ny0[a0:b0, None, None] | ny1[None, :, None] | ny2[None, None, :] | (9.0 * kk >= nmin * nmin) \
            | (kk == 0)
        kks = torch.where(zero, torch.ones_like(kk), kk)
        amp = torch.where(zero, torch.zeros_like(kk), torch.sqrt(_energy_shape(torch.sqrt(kks)) / (4.0 * math.pi * kks)))
        j0 = torch.arange(a0, b0, dtype=torch.int64, device=dev)[:, None, None]
        m = (j0 * n1 + j1) * H + j2
        a = []
        for c in range(3):
            th = 2.0 * math.pi * uniform01(seed, m * 3 + c)
            a.append(torch.complex(amp * torch.cos(th), amp * torch.sin(th)))
        f = (K0 * a[0] + K1 * a[1] + K2 * a[2]) / kks
        return [a[c] - (K0, K1, K2)[c] * f for c in range(3)]

    total = 0.0
    for a0 in range(0, n0, plane_chunk):
        b0 = min(n0, a0 + plane_chunk)
        for uc in draw(a0, b0):
            total += float(torch.sum((uc.real ** 2 + uc.imag ** 2) * w))
    total = (total + _plane0_energy(n0, n1, H, signed_wavenumbers(n0).astype(np.float64),
                                    signed_wavenumbers(n1).astype(np.float64), nyquist_mask(n0), nyquist_mask(n1),
                                    nmin, seed)) / 3.0
    scale = 1.0 / math.sqrt(total) if total > 0 else 1.0
    out = torch.empty((n0, n1, H), dtype=torch.complex64, device=dev)
    for a0 in range(0, n0, plane_chunk):
        b0 = min(n0, a0 + plane_chunk)
        out[a0:b0] = (draw(a0, b0)[component] * scale).to(torch.complex64)
    # Hermitian consistency on the k2 = 0 plane: the half with k0 > 0 or
    # (k0 = 0, k1 > 0) is kept, its conjugate mirrored to (-k0, -k1)
    p = out[:, :, 0]
    K0 = k0v[:, None]
    K1 = k1v[None, :]
    keep = (K0 > 0) | ((K0 == 0) & (K1 > 0))
    src = torch.where(keep, p, torch.zeros_like(p))
    r0 = (-torch.arange(n0, device=dev)) % n0
    r1 = (-torch.arange(n1, device=dev)) % n1
    mir = torch.conj(src[r0][:, r1])
    out[:, :, 0] = torch.where(keep, src, mir)
    out[0, 0, 0] = 0.0
    return out

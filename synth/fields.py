"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no transform arithmetic: it only draws numbers and shapes
spectra.  Both the FP64 oracle and the GPU library consume what it produces,
and neither is imported here.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: the draw for counter ``i`` under seed ``s`` is
``splitmix64(s * 0x9E3779B97F4A7C15 ^ i)``, so every value depends only on
(seed, index) and never on the order or the thread count of generation.
``uniform = (r >> 11) * 2**-53`` gives [0, 1).

Workload shapes (the paper's workloads are turbulence fields of the Tarang
pseudo-spectral solver, Sec. 1; the fields themselves are not available, so
these synthetic fields stand in for them):

* ``uniform_field``: i.i.d. uniform[-1, 1) real samples.
* ``cosine_mode`` / ``delta_field``: single Fourier modes and impulses, whose
  transforms are known in closed form.
* ``spectral_velocity``: the half-spectrum of a random-phase, divergence-free
  velocity field with energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2) for k < 8
  and a Kolmogorov k^(-5/3) tail beyond (continuous at k = 8), k0 = 4,
  spherically truncated by the 2/3 rule (keep 9|k|^2 < n_min^2), Hermitian
  consistent on the k2 = 0 plane and normalised so that the real field it
  describes has unit rms.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied element-wise to uint64 states."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def draw_u64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based draw: splitmix64(seed * golden ^ counter)."""
    with np.errstate(over="ignore"):
        key = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GOLDEN
    return splitmix64(key ^ np.asarray(counters, dtype=np.uint64))


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """uniform[0, 1) doubles with 53 random bits."""
    r = draw_u64(seed, counters)
    return (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_field(shape, seed: int) -> np.ndarray:
    """i.i.d. uniform[-1, 1) FP64 samples; element i (C order) uses counter i."""
    n = int(np.prod(shape))
    return (2.0 * uniform01(seed, np.arange(n, dtype=np.uint64)) - 1.0).reshape(shape)


def cosine_mode(n0: int, n1: int, n2: int, k0: int, k1: int, k2: int) -> np.ndarray:
    """x[j] = cos(2 pi (k0 j0/n0 + k1 j1/n1 + k2 j2/n2)), phase reduced exactly.

    The phase is formed as an integer numerator over n0*n1*n2 so that it is
    exact before the single cosine call.
    """
    j0 = np.arange(n0, dtype=np.int64)[:, None, None]
    j1 = np.arange(n1, dtype=np.int64)[None, :, None]
    j2 = np.arange(n2, dtype=np.int64)[None, None, :]
    D = n0 * n1 * n2
    num = ((k0 * j0) % n0) * (n1 * n2) + ((k1 * j1) % n1) * (n0 * n2) + ((k2 * j2) % n2) * (n0 * n1)
    return np.cos(2.0 * np.pi * ((num % D).astype(np.float64) / D))


def delta_field(n0: int, n1: int, n2: int, j0: int, j1: int, j2: int) -> np.ndarray:
    x = np.zeros((n0, n1, n2), dtype=np.float64)
    x[j0, j1, j2] = 1.0
    return x


def signed_wavenumbers(n: int) -> np.ndarray:
    """k = j for j < n/2, j - n for j > n/2; the Nyquist index n/2 maps to 0
    and is flagged separately by ``nyquist_mask``."""
    j = np.arange(n, dtype=np.int64)
    k = np.where(j < (n + 1) // 2, j, j - n)
    if n % 2 == 0:
        k[n // 2] = 0
    return k


def nyquist_mask(n: int) -> np.ndarray:
    m = np.zeros(n, dtype=bool)
    if n % 2 == 0:
        m[n // 2] = True
    return m


def energy_shape(k: np.ndarray, k0: float = 4.0, kc: float = 8.0) -> np.ndarray:
    """E(k) = k^4 exp(-2 (k/k0)^2) below kc, E(kc) (k/kc)^(-5/3) from kc on."""
    k = np.asarray(k, dtype=np.float64)
    ekc = kc ** 4 * np.exp(-2.0 * (kc / k0) ** 2)
    low = k ** 4 * np.exp(-2.0 * (k / k0) ** 2)
    with np.errstate(divide="ignore"):
        high = ekc * np.where(k > 0, k / kc, 1.0) ** (-5.0 / 3.0)
    return np.where(k < kc, low, high)


def spectral_velocity(n0: int, n1: int, n2: int, seed: int, components=(0, 1, 2),
                      plane_chunk: int = 32, workers: int = 1) -> np.ndarray:
    """Half-spectrum (n0, n1, n2/2+1) complex128 of each requested velocity
    component of a random-phase, divergence-free, 2/3-truncated field.

    Recipe (per half-spectrum index (j0, j1, j2), mode counter
    m = (j0*n1 + j1)*(n2/2+1) + j2):
      1. signed wavenumbers k0, k1 from ``signed_wavenumbers``, k2 = j2; any
         Nyquist index gives a zero mode;
      2. amplitude A = sqrt(E(|k|) / (4 pi |k|^2)), zero at k = 0;
      3. a_c = A exp(2 pi i u(seed, 3m + c)) for c = 0, 1, 2;
      4. projection u_hat = a - k (k . a) / |k|^2 (divergence-free);
      5. keep iff 9 |k|^2 < min(n0, n1, n2)^2 (2/3 rule, spherical);
      6. on the k2 = 0 plane only the half with k0 > 0 or (k0 = 0, k1 > 0) is
         drawn; its conjugate is mirrored to (-k0, -k1, 0), so the real field
         the spectrum describes exists;
      7. all three components are scaled by one common factor so that the mean
         over components of sum_half c_k2 |u_hat_c|^2 is 1 (c_k2 = 1 at k2 = 0
         and k2 = n2/2, else 2): the unnormalised inverse transform of the
         field then has unit rms per component on average, and the common
         factor keeps k . u_hat = 0.

    ``workers`` > 1 draws chunks of planes on that many threads; the chunks'
    energies are summed in plane order, so the result is bit for bit the same
    for every worker count.
    """
    if n2 % 2:
        raise ValueError("n2 must be even")
    H = n2 // 2 + 1
    k0v = signed_wavenumbers(n0).astype(np.float64)
    k1v = signed_wavenumbers(n1).astype(np.float64)
    k2v = np.arange(H, dtype=np.float64)
    ny0, ny1 = nyquist_mask(n0), nyquist_mask(n1)
    ny2 = np.zeros(H, dtype=bool)
    ny2[H - 1] = True
    nmin = min(n0, n1, n2)
    comps = tuple(components)
    out = np.zeros((len(comps), n0, n1, H), dtype=np.complex128)

    w = np.full(H, 2.0)
    w[0] = w[H - 1] = 1.0

    def chunk(a0):
        """Draw planes [a0, a0 + plane_chunk) into out; their energy per component."""
        energy = np.zeros(3)
        b0 = min(n0, a0 + plane_chunk)
        K0 = k0v[a0:b0, None, None]
        K1 = k1v[None, :, None]
        K2 = k2v[None, None, :]
        kk = K0 * K0 + K1 * K1 + K2 * K2
        zero = ny0[a0:b0, None, None] | ny1[None, :, None] | ny2[None, None, :] | (9.0 * kk >= nmin * nmin) \
            | (kk == 0)
        # only the modes that survive steps 1 and 5 are drawn (the others are 0)
        idx = np.flatnonzero(~zero)
        if idx.size == 0:
            return energy
        kkf = kk.ravel()[idx] if kk.size == zero.size else np.broadcast_to(kk, zero.shape).ravel()[idx]
        i0, rest = np.divmod(idx, n1 * H)
        i1, i2 = np.divmod(rest, H)
        q0, q1, q2 = k0v[a0 + i0], k1v[i1], k2v[i2]
        amp = np.sqrt(energy_shape(np.sqrt(kkf)) / (4.0 * np.pi * kkf))
        m = ((np.uint64(a0) + i0.astype(np.uint64)) * np.uint64(n1) + i1.astype(np.uint64)) * np.uint64(H) \
            + i2.astype(np.uint64)
        a = []
        for c in range(3):
            th = 2.0 * np.pi * uniform01(seed, m * np.uint64(3) + np.uint64(c))
            a.append(amp * (np.cos(th) + 1j * np.sin(th)))
        f = (q0 * a[0] + q1 * a[1] + q2 * a[2]) / kkf
        kvec = (q0, q1, q2)
        wt = w[i2]
        for c in range(3):
            uc = a[c] - kvec[c] * f
            # energy of the chunk (the k2 = 0 plane is rebuilt below and recounted there)
            energy[c] += float(np.sum((uc.real ** 2 + uc.imag ** 2) * np.where(i2 > 0, wt, 0.0)))
            if c in comps:
                dst = out[comps.index(c), a0:b0].reshape(-1)
                dst[idx] = uc
        del a, f
        return energy

    starts = range(0, n0, plane_chunk)
    if workers > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=workers) as ex:
            parts = list(ex.map(chunk, starts))
    else:
        parts = [chunk(a0) for a0 in starts]
    energy = np.zeros(3)
    for e in parts:  # plane order, whatever the worker count
        energy += e

    # Hermitian consistency on the k2 = 0 plane (step 6).
    for i in range(len(comps)):
        p = out[i, :, :, 0]
        K0 = k0v[:, None]
        K1 = k1v[None, :]
        keep = (K0 > 0) | ((K0 == 0) & (K1 > 0))
        src = np.where(keep, p, 0.0)
        # mirrored index of (j0, j1) is ((-j0) mod n0, (-j1) mod n1)
        mir = np.conj(src[(-np.arange(n0)) % n0][:, (-np.arange(n1)) % n1])
        out[i, :, :, 0] = np.where(keep, src, mir)
        out[i, 0, 0, 0] = 0.0

    # Energy of the rebuilt k2 = 0 planes of all three components (step 6 for
    # the components that were not requested is redone here on the fly).
    e0 = _plane0_energy(n0, n1, H, k0v, k1v, ny0, ny1, nmin, seed)
    total = float(np.sum(energy) + e0) / 3.0
    if total > 0:
        out /= np.sqrt(total)
    return out


def _plane0_energy(n0, n1, H, k0v, k1v, ny0, ny1, nmin, seed):
    """sum over c of sum_{k2=0 plane} |u_hat_c|^2 after the Hermitian rebuild:
    twice the energy of the drawn half (k0 > 0 or k0 = 0, k1 > 0)."""
    K0 = k0v[:, None]
    K1 = k1v[None, :]
    kk = K0 * K0 + K1 * K1
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(kk > 0, np.sqrt(energy_shape(np.sqrt(kk)) / (4.0 * np.pi * np.where(kk > 0, kk, 1.0))), 0.0)
    zero = ny0[:, None] | ny1[None, :] | (9.0 * kk >= nmin * nmin)
    keep = ((K0 > 0) | ((K0 == 0) & (K1 > 0))) & ~zero
    m = (np.arange(n0, dtype=np.uint64)[:, None] * np.uint64(n1) + np.arange(n1, dtype=np.uint64)[None, :]) * np.uint64(H)
    a = [amp * np.exp(2j * np.pi * uniform01(seed, m * np.uint64(3) + np.uint64(c))) for c in range(3)]
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(kk > 0, (K0 * a[0] + K1 * a[1]) / np.where(kk > 0, kk, 1.0), 0.0)
    u = (a[0] - K0 * f, a[1] - K1 * f, a[2])
    return float(sum(2.0 * np.sum(np.abs(uc[keep]) ** 2) for uc in u))


def seed_for_config(config: int, field: int = 0) -> int:
    """Seed convention: 1406 + config number, + 100 per extra field."""
    return 1406 + config + 100 * field

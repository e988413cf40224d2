"""FP64 CPU oracle for the 3D r2c / c2r FFT (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_1406_5597_gb300``) and never imports it.

The transforms live in plain C (``fft64.c``, built with gcc into
``liboracle.so`` next to it); this module marshals numpy arrays through
ctypes and adds the few numpy-level definitions that are sums over the
spectrum (Parseval, shell energies, the 2/3 mask, the nonlinear term).

Definitions (Sec. 2 of Chatterjee, Verma & Chaudhuri, arXiv:1406.5597, with
the FFTW sign/scaling convention of the transforms the paper uses, Sec. 3):

    r2c: X[k] = sum_j x[j] exp(-2 pi i (k0 j0/n0 + k1 j1/n1 + k2 j2/n2)), 0 <= k2 <= floor(n2/2)
    c2r: y[j] = sum_{k2} c_k2 Re(sum_{k0,k1} Y[k] exp(+2 pi i (...))),  c_k2 = 1 at 0 and at
         n2/2 (even n2), else 2
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft64.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fft64.c into liboracle.so (gcc, -O2, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            for name, args in {
                "oracle_fft1d": [P, P, I, I],
                "oracle_r2c3d": [P, P, I, I, I, I],
                "oracle_c2r3d": [P, P, I, I, I, I],
                "oracle_r2c3d_naive": [P, P, I, I, I],
                "oracle_c2r3d_naive": [P, P, I, I, I],
                "oracle_r2c_bins_f32": [P, I, I, I, P, I, P],
                "oracle_c2r_points_c64": [P, I, I, I, P, I, P],
            }.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = I
            lib.oracle_threads.argtypes = []
            lib.oracle_threads.restype = I
            lib.oracle_set_threads.argtypes = [I]
            lib.oracle_set_threads.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def threads() -> int:
    return _load().oracle_threads()


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def fft1d(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """1D complex DFT, y[k] = sum_j x[j] exp(sign 2 pi i j k / n), unnormalised."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.empty_like(x)
    _check(_load().oracle_fft1d(_ptr(x), _ptr(y), x.size, int(sign)), "oracle_fft1d")
    return y


def _shape3(x: np.ndarray):
    if x.ndim == 3:
        return 1, x.shape
    if x.ndim == 4:
        return x.shape[0], x.shape[1:]
    raise ValueError("expected (n0, n1, n2) or (batch, n0, n1, n2)")


def r2c3d(x: np.ndarray) -> np.ndarray:
    """Forward r2c of a real (batch?, n0, n1, n2) array in FP64 (Sec. 2, Sec. 2.1)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    b, (n0, n1, n2) = _shape3(x)
    H = n2 // 2 + 1
    X = np.empty(x.shape[:-1] + (H,), dtype=np.complex128)
    _check(_load().oracle_r2c3d(_ptr(x), _ptr(X), n0, n1, n2, b), "oracle_r2c3d")
    return X


def c2r3d(Y: np.ndarray, n2: int) -> np.ndarray:
    """Inverse c2r (unnormalised) of a complex (batch?, n0, n1, n2/2+1) array in FP64."""
    Y = np.ascontiguousarray(Y, dtype=np.complex128)
    b, (n0, n1, H) = _shape3(Y)
    if H != n2 // 2 + 1:
        raise ValueError("last axis must be n2/2+1")
    y = np.empty(Y.shape[:-1] + (n2,), dtype=np.float64)
    _check(_load().oracle_c2r3d(_ptr(Y), _ptr(y), n0, n1, n2, b), "oracle_c2r3d")
    return y


def r2c3d_naive(x: np.ndarray) -> np.ndarray:
    """The forward definition summed directly (O(N^2); N <= 8192)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n0, n1, n2 = x.shape
    X = np.empty((n0, n1, n2 // 2 + 1), dtype=np.complex128)
    _check(_load().oracle_r2c3d_naive(_ptr(x), _ptr(X), n0, n1, n2), "oracle_r2c3d_naive")
    return X


def c2r3d_naive(Y: np.ndarray, n2: int) -> np.ndarray:
    """The inverse definition summed directly (O(N^2); N <= 8192)."""
    Y = np.ascontiguousarray(Y, dtype=np.complex128)
    n0, n1, _ = Y.shape
    y = np.empty((n0, n1, n2), dtype=np.float64)
    _check(_load().oracle_c2r3d_naive(_ptr(Y), _ptr(y), n0, n1, n2), "oracle_c2r3d_naive")
    return y


def r2c_bins_f32(x32: np.ndarray, kvecs) -> np.ndarray:
    """Exact FP64 spectral bins X[k] of an FP32 field (n0, n1, n2); O(N) per bin."""
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    n0, n1, n2 = x32.shape
    k = np.ascontiguousarray(np.asarray(kvecs, dtype=np.int32).reshape(-1, 3))
    out = np.empty(2 * len(k), dtype=np.float64)
    _check(_load().oracle_r2c_bins_f32(_ptr(x32), n0, n1, n2, _ptr(k), len(k), _ptr(out)),
           "oracle_r2c_bins_f32")
    return out[0::2] + 1j * out[1::2]


def unit_roots(n: int, k: int, sign: int = -1) -> np.ndarray:
    """exp(sign 2 pi i (k j mod n) / n) for j in [0, n), the exponent reduced
    in integers before the single cos / sin call."""
    j = np.arange(n, dtype=np.int64)
    ang = 2.0 * np.pi * ((int(k) * j) % n).astype(np.float64) / n
    return np.cos(ang) + (1j if sign > 0 else -1j) * np.sin(ang)


def r2c_bins_sep(x32: np.ndarray, kvecs, chunk_rows: int = 1 << 16) -> np.ndarray:
    """Exact FP64 bins X[k] of an FP32 field (n0, n1, n2): the forward
    definition of Sec. 2 restricted to the listed bins and summed one axis at a
    time,  X[k] = sum_j0 W0^{k0 j0} sum_j1 W1^{k1 j1} sum_j2 x[j] W2^{k2 j2}.
    The j2 sums are formed once per distinct k2 of the list for every row (a
    matrix product over row chunks), then each bin sums its rows over j1 and
    j0.  Cost O(N * distinct k2 + bins * n0 n1), so lists with few distinct k2
    values are cheap at sizes where r2c_bins_f32 (O(N) per bin) is not."""
    n0, n1, n2 = x32.shape
    k = np.asarray(kvecs, dtype=np.int64).reshape(-1, 3)
    if np.any(k < 0) or np.any(k[:, 0] >= n0) or np.any(k[:, 1] >= n1) or np.any(k[:, 2] > n2 // 2):
        raise ValueError("bin outside the half spectrum")
    k2s = np.unique(k[:, 2])
    E = np.stack([unit_roots(n2, q) for q in k2s], axis=1)  # (n2, distinct k2)
    Er, Ei = np.ascontiguousarray(E.real), np.ascontiguousarray(E.imag)
    rows = x32.reshape(n0 * n1, n2)
    R = np.empty((n0 * n1, len(k2s)), dtype=np.complex128)
    for a in range(0, n0 * n1, chunk_rows):
        xc = rows[a:a + chunk_rows].astype(np.float64)
        R[a:a + chunk_rows].real = xc @ Er
        R[a:a + chunk_rows].imag = xc @ Ei
    R = R.reshape(n0, n1, len(k2s))
    out = np.empty(len(k), dtype=np.complex128)
    for b, (k0, k1, k2) in enumerate(k):
        plane = R[:, :, int(np.searchsorted(k2s, k2))] @ unit_roots(n1, k1)  # (n0,)
        out[b] = plane @ unit_roots(n0, k0)
    return out


def c2r_points_c64(Y64: np.ndarray, n2: int, jvecs) -> np.ndarray:
    """Exact FP64 inverse values y[j] of a complex64 half-spectrum; O(M) per point."""
    Y64 = np.ascontiguousarray(Y64, dtype=np.complex64)
    n0, n1, H = Y64.shape
    if H != n2 // 2 + 1:
        raise ValueError("last axis must be n2/2+1")
    j = np.ascontiguousarray(np.asarray(jvecs, dtype=np.int32).reshape(-1, 3))
    out = np.empty(len(j), dtype=np.float64)
    _check(_load().oracle_c2r_points_c64(_ptr(Y64), n0, n1, n2, _ptr(j), len(j), _ptr(out)),
           "oracle_c2r_points_c64")
    return out


# ---------------------------------------------------------------------------
# Sums over the half spectrum (plain numpy definitions).
# ---------------------------------------------------------------------------

def half_weights(n2: int) -> np.ndarray:
    """c_k2: 1 at k2 = 0 and, for even n2, at the Nyquist bin k2 = n2/2; 2 for
    every other bin (it stands for itself and its conjugate partner)."""
    H = n2 // 2 + 1
    c = np.full(H, 2.0)
    c[0] = 1.0
    if n2 % 2 == 0:
        c[H - 1] = 1.0
    return c


def half_energy(X: np.ndarray, n2: int) -> float:
    """sum over the half spectrum of c_k2 |X|^2 in FP64; for X = r2c(x) this
    equals N * sum_j x_j^2 (Parseval)."""
    X = np.asarray(X, dtype=np.complex128)
    return float(np.sum((X.real ** 2 + X.imag ** 2) * half_weights(n2)))


def shell_index(n0: int, n1: int, n2: int) -> np.ndarray:
    """Integer shell b = floor(|k| + 1/2) of every half-spectrum bin, with
    |k_a| = min(j_a, n_a - j_a): b = 0 holds only k = 0, and for b >= 1 the
    shell is (2b-1)^2 <= 4|k|^2 < (2b+1)^2.  Decided in integers, so no
    rounding picks a bin."""
    H = n2 // 2 + 1
    a0 = np.minimum(np.arange(n0), n0 - np.arange(n0)).astype(np.int64)
    a1 = np.minimum(np.arange(n1), n1 - np.arange(n1)).astype(np.int64)
    a2 = np.arange(H, dtype=np.int64)
    kk4 = 4 * (a0[:, None, None] ** 2 + a1[None, :, None] ** 2 + a2[None, None, :] ** 2)
    b = np.floor((np.sqrt(kk4.astype(np.float64)) + 1.0) / 2.0).astype(np.int64)
    # integer correction of any floating-point slip
    b = np.where((b > 0) & ((2 * b - 1) ** 2 > kk4), b - 1, b)
    b = np.where((2 * b + 1) ** 2 <= kk4, b + 1, b)
    return b


def shell_energy(X: np.ndarray, n0: int, n1: int, n2: int, nbins: int) -> np.ndarray:
    """E[b] = sum over half-spectrum bins in shell b of c_k2 |X|^2 (FP64);
    bins at b >= nbins are dropped."""
    X = np.asarray(X, dtype=np.complex128)
    b = shell_index(n0, n1, n2)
    w = (X.real ** 2 + X.imag ** 2) * half_weights(n2)
    sel = b < nbins
    return np.bincount(b[sel].ravel(), weights=w[sel].ravel(), minlength=nbins)[:nbins]


def dealias_mask(n0: int, n1: int, n2: int) -> np.ndarray:
    """2/3 rule on the half spectrum: keep bin k iff 3|k_a| < n_a on every axis,
    with k_a the signed wavenumber in [-n_a/2, n_a/2) (so the Nyquist bin,
    |k_a| = n_a/2, is always dropped)."""
    H = n2 // 2 + 1

    def keep(n, idx):
        k = np.where(idx < n // 2, idx, idx - n)  # [-n/2, n/2)
        return 3 * np.abs(k) < n

    m0 = keep(n0, np.arange(n0))
    m1 = keep(n1, np.arange(n1))
    m2 = 3 * np.arange(H) < n2
    return m0[:, None, None] & m1[None, :, None] & m2[None, None, :]


def nonlinear_term(uhat: np.ndarray, n2: int) -> np.ndarray:
    """Pseudo-spectral quadratic term of a velocity field given by its three
    half-spectra uhat (3, n0, n1, n2/2+1):
        u_i = c2r(uhat_i);  p_ij = u_i u_j for ij in (00, 01, 02, 11, 12, 22);
        N_ij = mask * r2c(p_ij) / N.
    The solver context is Sec. 1 (pseudo-spectral method); the 2/3 mask is the
    standard dealiasing rule of such solvers (the paper does not print it)."""
    uhat = np.asarray(uhat, dtype=np.complex128)
    _, n0, n1, H = uhat.shape
    N = n0 * n1 * n2
    u = [c2r3d(uhat[i], n2) for i in range(3)]
    mask = dealias_mask(n0, n1, n2)
    out = np.empty((6, n0, n1, H), dtype=np.complex128)
    for q, (i, j) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        out[q] = np.where(mask, r2c3d(u[i] * u[j]) / N, 0.0)
    return out


def wavenumbers(n0: int, n1: int, n2: int):
    """Signed integer wavenumbers of the half-spectrum bins (box [0, 2 pi)^3):
    k_a = j_a for j_a < n_a/2, j_a - n_a otherwise (the Nyquist index maps to
    -n_a/2); k2 = j2.  Broadcastable (n0,1,1), (1,n1,1), (1,1,H) arrays."""
    H = n2 // 2 + 1

    def signed(n):
        j = np.arange(n)
        return np.where(j < n // 2, j, j - n).astype(np.float64)

    return signed(n0)[:, None, None], signed(n1)[None, :, None], np.arange(H, dtype=np.float64)[None, None, :]


def ns_rhs(uhat: np.ndarray, n2: int, nu: float) -> np.ndarray:
    """Right-hand side of the incompressible Navier-Stokes equations in
    Fourier space for the velocity half-spectra uhat (3, n0, n1, n2/2+1) with
    u = c2r(uhat) (the pseudo-spectral solver of Sec. 1; the scheme itself is
    not printed in the paper):
        a_l = sum_j k_j N_lj                (N = nonlinear_term: the dealiased
                                             Fourier coefficients of u_l u_j)
        b   = a - k (k . a) / |k|^2         (pressure projection; b = 0 at k = 0)
        R_l = mask * (-i b_l - nu |k|^2 uhat_l),
    i.e. the transform of -(u . grad) u - grad p + nu lap u for a solenoidal u."""
    uhat = np.asarray(uhat, dtype=np.complex128)
    _, n0, n1, H = uhat.shape
    N = nonlinear_term(uhat, n2)
    k = wavenumbers(n0, n1, n2)
    sym = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    a = [sum(k[j] * N[sym[(min(l, j), max(l, j))]] for j in range(3)) for l in range(3)]
    kk = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    ka = k[0] * a[0] + k[1] * a[1] + k[2] * a[2]
    inv = np.divide(1.0, kk, out=np.zeros_like(kk), where=kk > 0)
    mask = dealias_mask(n0, n1, n2)
    R = np.empty_like(uhat)
    for l in range(3):
        b = np.where(kk > 0, a[l] - k[l] * ka * inv, 0.0)
        R[l] = np.where(mask, -1j * b - nu * kk * uhat[l], 0.0)
    return R


def ns_step_rk2(uhat: np.ndarray, n2: int, nu: float, dt: float) -> np.ndarray:
    """One step of Heun's two-stage Runge-Kutta method on ns_rhs:
        u* = u + dt R(u);  u_new = u + dt/2 (R(u) + R(u*))."""
    uhat = np.asarray(uhat, dtype=np.complex128)
    r1 = ns_rhs(uhat, n2, nu)
    r2 = ns_rhs(uhat + dt * r1, n2, nu)
    return uhat + 0.5 * dt * (r1 + r2)

"""Pins for the FP64 oracle (CPU only).

Every check compares the oracle with something other than itself: the
transform's definition summed directly (brute force on tiny shapes), closed
forms (single cosine modes, impulses, ramps, a textbook DFT), an independent
library routine (numpy.fft), and invariants the mathematics fixes (Hermitian
symmetry of a real field's spectrum, Parseval, the x N round trip, linearity,
the shift theorem).  A dropped term, a wrong sign, a swapped axis or a
misplaced k2 range fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


TINY = [(n0, n1, n2) for n0, n1, n2 in itertools.product((2, 3, 4, 5, 6, 8, 10), (2, 3, 5, 6, 12),
                                                         (2, 4, 6, 10, 16))
        if n0 * n1 * n2 <= 8192][::3] + [(6, 10, 16), (8, 8, 8), (15, 12, 10), (16, 16, 16), (7, 6, 14), (14, 7, 4),
                                          (4, 6, 9), (5, 3, 15), (6, 8, 7), (3, 5, 3), (2, 2, 21),
                                          # prime factors above 7 on every axis (the direct-sum branch)
                                          (11, 2, 4), (2, 13, 6), (3, 2, 22), (2, 3, 26), (4, 2, 13), (2, 2, 34)]


@pytest.mark.parametrize("shape", TINY)
def test_r2c_matches_naive_definition(shape):
    x = synth.uniform_field(shape, seed=11)
    X = oracle.r2c3d(x)
    assert X.shape == shape[:2] + (shape[2] // 2 + 1,)
    assert rel_l2(X, oracle.r2c3d_naive(x)) < 1e-13


@pytest.mark.parametrize("shape", TINY[::2])
def test_c2r_matches_naive_definition_on_any_input(shape):
    """The inverse is defined for every complex input, Hermitian or not; the
    imaginary parts of the k2 = 0 and k2 = n2/2 bins must not matter."""
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((n0, n1, H)) + 1j * rng.standard_normal((n0, n1, H))
    y = oracle.c2r3d(Y, n2)
    assert rel_l2(y, oracle.c2r3d_naive(Y, n2)) < 1e-13


def test_textbook_dft4():
    rows = np.loadtxt(os.path.join(GOLDEN, "dft4_textbook.txt"))
    expect = rows[:, 1] + 1j * rows[:, 2]
    got = oracle.fft1d(np.array([1, 2, 3, 4], dtype=np.complex128), -1)
    assert np.max(np.abs(got - expect)) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 12, 30, 49, 64, 96, 160, 210, 512, 11, 13, 26, 97, 143, 1021, 4093])
def test_fft1d_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel_l2(oracle.fft1d(x, -1), np.fft.fft(x)) < 1e-13
    assert rel_l2(oracle.fft1d(x, +1), n * np.fft.ifft(x)) < 1e-13


@pytest.mark.parametrize("shape", [(32, 32, 32), (6, 10, 16), (15, 12, 10), (64, 48, 40), (2, 2, 2), (16, 12, 45),
                                   (8, 10, 27), (11, 13, 34), (17, 6, 26), (6, 97, 13)])
def test_r2c_matches_numpy_rfftn(shape):
    x = synth.uniform_field(shape, seed=3)
    assert rel_l2(oracle.r2c3d(x), np.fft.rfftn(x)) < 1e-13


def test_batch_matches_separate_calls():
    x = synth.uniform_field((3, 6, 10, 8), seed=5)
    Xb = oracle.r2c3d(x)
    for b in range(3):
        assert np.array_equal(Xb[b], oracle.r2c3d(x[b]))
    yb = oracle.c2r3d(Xb, 8)
    for b in range(3):
        assert np.array_equal(yb[b], oracle.c2r3d(Xb[b], 8))


MODES_32 = [(1, 0, 0), (0, 3, 5), (7, -2, 16), (0, 0, 16), (16, 16, 0), (-5, 11, 9)]


@pytest.mark.parametrize("k", MODES_32)
def test_single_cosine_mode_closed_form(k):
    """cos(k.x) has spectral weight N/2 at k and N/2 at -k (mod n); only the
    bins with 0 <= k2 <= n2/2 are stored, so a k2 in (0, n2/2) shows one spike,
    and a k2 in {0, n2/2} shows both.  A self-conjugate k (k = -k mod n) shows N."""
    n = 32
    N = n ** 3
    x = synth.cosine_mode(n, n, n, *k)
    X = oracle.r2c3d(x)
    E = np.zeros_like(X)
    kp = tuple(v % n for v in k)
    km = tuple((-v) % n for v in k)
    for kk in (kp, km):
        if kk[2] <= n // 2:
            E[kk] += N / 2
    assert np.max(np.abs(X - E)) < 1e-12 * N


def test_delta_closed_form():
    n0, n1, n2 = 32, 32, 32
    x = synth.delta_field(n0, n1, n2, 3, 5, 7)
    X = oracle.r2c3d(x)
    k0 = np.arange(n0)[:, None, None]
    k1 = np.arange(n1)[None, :, None]
    k2 = np.arange(n2 // 2 + 1)[None, None, :]
    E = np.exp(-2j * np.pi * (3 * k0 / n0 + 5 * k1 / n1 + 7 * k2 / n2))
    assert np.max(np.abs(X - E)) < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ramp_closed_form(axis):
    """x = j_axis: X = (prod of the other lengths) * sum_j j W^{jk} on the
    axis' line through k = 0 (closed form n/(W^k - 1) for k != 0,
    n(n-1)/2 at k = 0) and zero elsewhere.  Pins which axis is which."""
    shape = (6, 10, 16)
    n = shape[axis]
    idx = [None, None, None]
    idx[axis] = slice(None)
    x = np.broadcast_to(np.arange(n, dtype=np.float64)[tuple(idx)], shape).copy()
    X = oracle.r2c3d(x)
    other = np.prod(shape) // n
    E = np.zeros_like(X)
    ks = np.arange(n if axis < 2 else n // 2 + 1)
    W = np.exp(-2j * np.pi * ks / n)
    with np.errstate(divide="ignore", invalid="ignore"):
        line = np.where(ks == 0, n * (n - 1) / 2, n / (W - 1))
    sel = [0, 0, 0]
    sel[axis] = slice(None)
    E[tuple(sel)] = other * line
    assert np.max(np.abs(X - E)) < 1e-11


@pytest.mark.parametrize("shape", [(32, 32, 32), (15, 12, 10), (6, 10, 16)])
def test_hermitian_planes(shape):
    n0, n1, n2 = shape
    X = oracle.r2c3d(synth.uniform_field(shape, seed=9))
    scale = np.linalg.norm(X)
    for k2 in (0, n2 // 2):
        P = X[:, :, k2]
        mirror = np.conj(P[(-np.arange(n0)) % n0][:, (-np.arange(n1)) % n1])
        assert np.max(np.abs(P - mirror)) <= 1e-14 * scale


@pytest.mark.parametrize("shape", [(32, 32, 32), (15, 12, 10)])
def test_parseval(shape):
    x = synth.uniform_field(shape, seed=21)
    X = oracle.r2c3d(x)
    N = x.size
    assert abs(oracle.half_energy(X, shape[2]) / N - np.sum(x * x)) < 1e-12 * np.sum(x * x)


@pytest.mark.parametrize("shape", [(32, 32, 32), (15, 12, 10), (2, 2, 2), (64, 48, 40)])
def test_round_trip_times_N(shape):
    x = synth.uniform_field(shape, seed=1406 + 1)
    y = oracle.c2r3d(oracle.r2c3d(x), shape[2])
    assert np.max(np.abs(y - x.size * x)) < 1e-12 * x.size


def test_linearity():
    shape = (12, 10, 8)
    a = synth.uniform_field(shape, seed=1)
    b = synth.uniform_field(shape, seed=2)
    lhs = oracle.r2c3d(2.5 * a - 0.75 * b)
    rhs = 2.5 * oracle.r2c3d(a) - 0.75 * oracle.r2c3d(b)
    assert np.max(np.abs(lhs - rhs)) < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_shift_theorem(axis):
    shape = (12, 10, 8)
    x = synth.uniform_field(shape, seed=4)
    X = oracle.r2c3d(x)
    Xs = oracle.r2c3d(np.roll(x, 1, axis=axis))
    n = shape[axis]
    k = np.arange(X.shape[axis])
    sh = [1, 1, 1]
    sh[axis] = -1
    ph = np.exp(-2j * np.pi * k / n).reshape(sh)
    assert np.max(np.abs(Xs - X * ph)) < 1e-12


def test_c2r_ignores_imag_at_dc_and_nyquist_after_columns():
    """Adding i*c to a whole k2 = 0 line along n0 and n1 changes the 2D
    inverse of that plane by an imaginary amount only; the real synthesis
    drops it, so y is unchanged."""
    n0, n1, n2 = 6, 10, 8
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((n0, n1, n2 // 2 + 1)) + 1j * rng.standard_normal((n0, n1, n2 // 2 + 1))
    y = oracle.c2r3d(Y, n2)
    Z = Y.copy()
    # a purely imaginary field in real space at k2 = 0 is i * (2D DFT of a real plane)
    plane = rng.standard_normal((n0, n1))
    Z[:, :, 0] += 1j * np.fft.fft2(plane)
    Z[:, :, -1] += 1j * np.fft.fft2(rng.standard_normal((n0, n1)))
    assert np.max(np.abs(oracle.c2r3d(Z, n2) - y)) < 1e-12


def test_spot_bins_and_points_match_full_oracle():
    shape = (24, 20, 16)
    x32 = synth.uniform_field(shape, seed=8).astype(np.float32)
    X = oracle.r2c3d(x32.astype(np.float64))
    ks = [(0, 0, 0), (3, 7, 2), (23, 19, 8), (12, 10, 5)]
    got = oracle.r2c_bins_f32(x32, ks)
    assert np.max(np.abs(got - np.array([X[k] for k in ks]))) < 1e-11
    Y64 = (X / 7.0).astype(np.complex64)
    y = oracle.c2r3d(Y64.astype(np.complex128), shape[2])
    js = [(0, 0, 0), (5, 3, 15), (23, 19, 1)]
    gotp = oracle.c2r_points_c64(Y64, shape[2], js)
    assert np.max(np.abs(gotp - np.array([y[j] for j in js]))) < 1e-9


def test_separable_spot_bins_match_full_oracle_and_direct_sums():
    """r2c_bins_sep (axis-by-axis sums, one j2 pass per distinct k2) against
    the full oracle and against the per-bin direct sums, on an odd-sized
    field; bins on the DC and Nyquist planes, repeated k2 values, and chunks
    that end inside the field."""
    shape = (18, 10, 12)
    x32 = synth.uniform_field(shape, seed=12).astype(np.float32)
    X = oracle.r2c3d(x32.astype(np.float64))
    ks = [(0, 0, 0), (3, 7, 2), (17, 9, 6), (12, 5, 2), (1, 0, 6), (9, 4, 5)]
    got = oracle.r2c_bins_sep(x32, ks, chunk_rows=7)
    ref = np.array([X[k] for k in ks])
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))
    assert np.max(np.abs(got - oracle.r2c_bins_f32(x32, ks))) < 1e-11 * np.max(np.abs(ref))
    # a transposed index would pick another bin: every bin differs from its
    # axis-swapped partner on this field
    assert np.min(np.abs(got[1:] - np.array([X[k[1] % 18, k[0] % 10, k[2]] for k in ks[1:]]))) > 1e-3
    with pytest.raises(ValueError):
        oracle.r2c_bins_sep(x32, [(0, 0, 7)])


def test_spectrum_as_oracle():
    """x = c2r(S) for a Hermitian-consistent S gives r2c(x) = N S exactly (up to
    FP64 rounding): the spectral_velocity field is such an S."""
    n0, n1, n2 = 32, 24, 20
    S = synth.spectral_velocity(n0, n1, n2, seed=1408, components=(0,))[0]
    x = oracle.c2r3d(S, n2)
    N = n0 * n1 * n2
    assert 0.3 < np.sqrt(np.mean(x * x)) < 3.0
    assert rel_l2(oracle.r2c3d(x), N * S) < 1e-13


def test_shell_index_exact():
    """Shell b = floor(|k| + 1/2) equals (isqrt(4|k|^2) + 1) // 2 exactly
    (integer square root, no floating point); checked bin by bin."""
    import math
    n0, n1, n2 = 30, 24, 40
    b = oracle.shell_index(n0, n1, n2)
    for j0 in range(n0):
        for j1 in range(n1):
            for j2 in range(n2 // 2 + 1):
                kk = min(j0, n0 - j0) ** 2 + min(j1, n1 - j1) ** 2 + j2 ** 2
                assert b[j0, j1, j2] == (math.isqrt(4 * kk) + 1) // 2
    assert b[0, 0, 0] == 0 and b[1, 0, 0] == 1 and b[0, 0, 1] == 1


def test_shell_energy_sums_to_parseval_total():
    n0, n1, n2 = 16, 12, 10
    X = oracle.r2c3d(synth.uniform_field((n0, n1, n2), seed=5))
    nb = int(np.sqrt((n0 // 2) ** 2 + (n1 // 2) ** 2 + (n2 // 2) ** 2)) + 2
    E = oracle.shell_energy(X, n0, n1, n2, nb)
    assert np.all(E >= 0)
    assert abs(E.sum() - oracle.half_energy(X, n2)) < 1e-12 * E.sum()
    assert abs(E[0] - abs(X[0, 0, 0]) ** 2) < 1e-12 * E.sum()


def test_nonlinear_term_single_mode_closed_form():
    """u = (cos(2 pi a j0 / n0), 0, 0): u0^2 = 1/2 + cos(2 pi 2a j0 / n0)/2, so
    N_00 = 1/2 at k = 0 and 1/4 at k0 = +-2a (kept by the 2/3 rule iff
    3*2a < n0), every other product zero."""
    n0, n1, n2 = 24, 12, 10
    N = n0 * n1 * n2
    for a, kept in ((2, True), (5, False)):
        u0 = synth.cosine_mode(n0, n1, n2, a, 0, 0)
        uhat = np.zeros((3, n0, n1, n2 // 2 + 1), dtype=np.complex128)
        uhat[0] = oracle.r2c3d(u0) / N  # so that c2r(uhat0) = u0
        out = oracle.nonlinear_term(uhat, n2)
        E = np.zeros_like(out[0])
        E[0, 0, 0] = 0.5
        if kept:
            E[2 * a, 0, 0] = 0.25
            E[n0 - 2 * a, 0, 0] = 0.25
        assert np.max(np.abs(out[0] - E)) < 1e-14
        assert np.max(np.abs(out[1:])) < 1e-14


def test_dealias_mask_counts():
    """The 2/3 rule keeps |k_a| <= (n_a - 1) // 3 on each axis (Nyquist dropped)."""
    m = oracle.dealias_mask(24, 12, 10)
    assert m.shape == (24, 12, 6)
    keep0 = 2 * ((24 - 1) // 3) + 1
    keep1 = 2 * ((12 - 1) // 3) + 1
    keep2 = (10 - 1) // 3 + 1
    assert m.sum() == keep0 * keep1 * keep2
    assert not m[12].any() and not m[:, 6].any()


# ---------------------------------------------------------------------------
# Pseudo-spectral Navier-Stokes step (ns_rhs, ns_step_rk2)
# ---------------------------------------------------------------------------

def _grid(n0, n1, n2):
    x0 = 2 * np.pi * np.arange(n0)[:, None, None] / n0
    x1 = 2 * np.pi * np.arange(n1)[None, :, None] / n1
    x2 = 2 * np.pi * np.arange(n2)[None, None, :] / n2
    return x0, x1, x2


def _uhat_of(u, n2):
    """Fourier coefficients (u = c2r(uhat)) of a sampled real field."""
    n0, n1 = u.shape[:2]
    return oracle.r2c3d(u) / (n0 * n1 * n2)


def test_ns_shear_mode_decays_by_the_exact_rk2_factor():
    """u = (sin(m x1), 0, 0) has (u . grad) u = 0, so R = -nu m^2 uhat and one
    Heun step multiplies the field by 1 - z + z^2/2, z = nu m^2 dt."""
    n0, n1, n2 = 8, 12, 16
    m, nu, dt = 2, 0.05, 0.3
    x0, x1, x2 = _grid(n0, n1, n2)
    u = np.zeros((3, n0, n1, n2))
    u[0] = np.sin(m * x1) + 0 * x0 + 0 * x2
    uh = np.stack([_uhat_of(u[i], n2) for i in range(3)])
    z = nu * m * m * dt
    new = oracle.ns_step_rk2(uh, n2, nu, dt)
    assert np.allclose(new, uh * (1 - z + z * z / 2), atol=1e-14)
    assert np.allclose(oracle.ns_rhs(uh, n2, nu), -nu * m * m * uh, atol=1e-14)


def test_ns_two_mode_triad_closed_form():
    """u = (A cos x1, 0, B cos x0) is solenoidal with (u . grad) u =
    (0, 0, -A B cos x1 sin x0), itself solenoidal (no pressure), so
    du/dt = (0, 0, A B sin x0 cos x1) - nu u."""
    n0, n1, n2 = 12, 12, 12
    A, B, nu = 0.7, -1.3, 0.02
    x0, x1, x2 = _grid(n0, n1, n2)
    u = np.zeros((3, n0, n1, n2))
    u[0] = A * np.cos(x1) + 0 * x0 + 0 * x2
    u[2] = B * np.cos(x0) + 0 * x1 + 0 * x2
    uh = np.stack([_uhat_of(u[i], n2) for i in range(3)])
    dudt = np.zeros_like(u)
    dudt[0] = -nu * u[0]
    dudt[2] = A * B * np.sin(x0) * np.cos(x1) - nu * u[2]
    expect = np.stack([_uhat_of(dudt[i], n2) for i in range(3)])
    R = oracle.ns_rhs(uh, n2, nu)
    assert np.max(np.abs(R - expect)) <= 1e-14
    # a sign or axis slip would put the source term elsewhere: it is nonzero
    assert np.max(np.abs(expect[2])) > 0.1


def test_ns_rhs_conserves_energy_without_viscosity_and_is_solenoidal():
    """For a solenoidal field inside the 2/3 mask the dealiased nonlinear
    term exchanges energy between modes without creating any:
    sum_half c_k2 Re(conj(uhat) . R) = 0 at nu = 0; with nu > 0 the rate is
    -nu sum c_k2 |k|^2 |uhat|^2; and k . R = 0 everywhere."""
    n0, n1, n2 = 16, 16, 16
    uh = synth.spectral_velocity(n0, n1, n2, seed=91).astype(np.complex128)
    w = oracle.half_weights(n2)
    k = oracle.wavenumbers(n0, n1, n2)
    kk = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    R0 = oracle.ns_rhs(uh, n2, 0.0)
    scale = np.sqrt(np.sum(np.abs(uh) ** 2) * np.sum(np.abs(R0) ** 2))
    rate = np.sum(w * np.real(np.conj(uh) * R0))
    assert abs(rate) <= 1e-12 * scale
    assert np.max(np.abs(sum(k[i] * R0[i] for i in range(3)))) <= 1e-12 * np.max(np.abs(R0))
    nu = 0.01
    R = oracle.ns_rhs(uh, n2, nu)
    rate = np.sum(w * np.real(np.conj(uh) * R))
    expect = -nu * np.sum(w * kk * np.abs(uh) ** 2)
    assert abs(rate - expect) <= 1e-12 * scale


@pytest.mark.parametrize("n2", [9, 15, 21, 25])
def test_odd_n2_half_spectrum_invariants(n2):
    """Odd n2: H = (n2 + 1) / 2 bins, no Nyquist bin, so every bin but k2 = 0
    counts twice in Parseval and in the synthesis; the round trip is x N and
    the imaginary part of the last bin does matter (it is not a Nyquist bin)."""
    shape = (6, 5, n2)
    N = 6 * 5 * n2
    x = synth.uniform_field(shape, seed=n2)
    X = oracle.r2c3d(x)
    assert X.shape[-1] == (n2 + 1) // 2
    assert abs(oracle.half_energy(X, n2) / N - np.sum(x ** 2)) <= 1e-12 * np.sum(x ** 2)
    assert rel_l2(oracle.c2r3d(X, n2), N * x) < 1e-13
    Y = np.zeros_like(X)
    Y[0, 0, -1] = 1j  # sin(2 pi k2 j2 / n2) with weight 2 at the top bin
    k2 = X.shape[-1] - 1
    j2 = np.arange(n2)
    expect = np.broadcast_to(-2 * np.sin(2 * np.pi * k2 * j2 / n2), shape)
    assert np.max(np.abs(oracle.c2r3d(Y, n2) - expect)) < 1e-13

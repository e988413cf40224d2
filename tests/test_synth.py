"""Checks of the seeded input generators (CPU only)."""
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_sequence():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) if not l.startswith("#")]
    for n, hx in rows:
        state = np.array([(int(n) - 1) * 0x9E3779B97F4A7C15 % 2 ** 64], dtype=np.uint64)
        assert format(int(synth.splitmix64(state)[0]), "016x") == hx


def test_uniform_field_is_counter_based_and_in_range():
    a = synth.uniform_field((4, 5, 6), seed=1407)
    b = synth.uniform_field((120,), seed=1407)
    assert np.array_equal(a.ravel(), b)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert not np.array_equal(a, synth.uniform_field((4, 5, 6), seed=1408))
    big = synth.uniform_field((200000,), seed=3)
    assert abs(big.mean()) < 0.01 and abs(big.var() - 1.0 / 3.0) < 0.01


def test_spectral_velocity_properties():
    n0, n1, n2 = 32, 24, 20
    H = n2 // 2 + 1
    U = synth.spectral_velocity(n0, n1, n2, seed=1410)
    k0 = synth.signed_wavenumbers(n0)[:, None, None].astype(float)
    k1 = synth.signed_wavenumbers(n1)[None, :, None].astype(float)
    k2 = np.arange(H)[None, None, :].astype(float)
    # divergence-free: k . u_hat = 0 on every mode
    div = k0 * U[0] + k1 * U[1] + k2 * U[2]
    assert np.max(np.abs(div)) < 1e-14
    # 2/3 spherical truncation
    kk = k0 ** 2 + k1 ** 2 + k2 ** 2
    assert np.all(U[:, 9 * kk >= min(n0, n1, n2) ** 2] == 0)
    # Hermitian k2 = 0 plane, unit mean weighted energy, independent of the request
    c = np.full(H, 2.0)
    c[0] = c[-1] = 1.0
    for i in range(3):
        P = U[i, :, :, 0]
        assert np.max(np.abs(P - np.conj(P[(-np.arange(n0)) % n0][:, (-np.arange(n1)) % n1]))) < 1e-15
    assert abs(np.mean([np.sum(np.abs(U[i]) ** 2 * c) for i in range(3)]) - 1.0) < 1e-12
    U1 = synth.spectral_velocity(n0, n1, n2, seed=1410, components=(1,))
    assert np.array_equal(U1[0], U[1])
    # the energy spectrum has the requested shape: k^4 exp(-2 (k/4)^2) peaks at
    # k = 4 (d/dk of 4 ln k - k^2/8 vanishes there), is continuous at k = 8 and
    # falls as k^(-5/3) beyond
    e = synth.energy_shape(np.arange(1, 12))
    assert np.argmax(e) + 1 == 4
    assert abs(synth.energy_shape(8.0 - 1e-9) - synth.energy_shape(8.0)) < 1e-6
    assert abs(e[10] / e[7] - (11 / 8) ** (-5 / 3)) < 1e-12


def test_spectral_velocity_same_for_every_worker_count():
    """Threaded drawing (large fields) gives the single-threaded result bit for bit."""
    a = synth.spectral_velocity(40, 36, 30, seed=1409, plane_chunk=6)
    b = synth.spectral_velocity(40, 36, 30, seed=1409, plane_chunk=6, workers=4)
    assert np.array_equal(a, b)


def test_device_generators_match_the_host_ones():
    """synth.device (torch arrays, here on the CPU) draws the same fields as
    synth.fields: the uniform field bit for bit, the spectrum-shaped field to
    complex64 rounding, for every component and with ragged plane chunks."""
    torch = __import__("pytest").importorskip("torch")
    from synth import device as sd
    u = sd.uniform_field((3, 5, 7, 11), 1409, device="cpu").numpy()
    assert np.array_equal(u, synth.uniform_field((3, 5, 7, 11), 1409).astype(np.float32))
    for shape, seed, comp in (((30, 18, 16), 1408, 0), ((32, 24, 20), 5, 2), ((12, 16, 10), 7, 1)):
        a = synth.spectral_velocity(*shape, seed=seed, components=(comp,))[0]
        b = sd.spectral_velocity(*shape, seed=seed, component=comp, device="cpu", plane_chunk=5).numpy()
        assert b.dtype == np.complex64
        assert np.max(np.abs(b - a)) <= 2.0 ** -23 * np.max(np.abs(a))
        assert np.array_equal(b == 0, a == 0)
    assert torch is not None

"""GPU parity: the CUDA path against the FP64 oracle, element by element, on
seeded inputs, through the C ABI (ctypes binding; torch provides only device
memory and the stream).

Tolerance (FP32 storage and arithmetic): relative L2 over all real and
imaginary components, accumulated in FP64, <= 5e-6 per direction and <= 1e-5
for the round trip.  The forward result is compared with the oracle's r2c of
the SAME FP32-rounded input promoted to FP64; the inverse with the oracle's
c2r of the SAME complex64 input, so the two directions' errors stay apart.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.errmodel import line_rms, spot_bound, spot_report

pytestmark = pytest.mark.gpu

TOL = 5e-6
TOL_RT = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gpu_r2c(lib, x32, flags=0, batch=None):
    """x32: (n0, n1, n2) or (batch, n0, n1, n2) float32 numpy -> complex128 numpy."""
    n0, n1, n2 = x32.shape[-3:]
    b = 1 if x32.ndim == 3 else x32.shape[0]
    plan = lib.Plan(n0, n1, n2, lib.FFT3D_F32, b, flags)
    xd = torch.from_numpy(np.ascontiguousarray(x32)).cuda()
    H = n2 // 2 + 1
    lead = x32.shape[:-3]
    oshape = lead + ((n1, n0, H) if (flags & lib.FFT3D_FLAG_EXPLICIT_TRANSPOSE and not flags & lib.FFT3D_FLAG_TRANSPOSE_BACK)
                     else (n0, n1, H))
    out = torch.empty(oshape, dtype=torch.complex64, device="cuda")
    plan.r2c(xd.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert lib.fft3d_query_device_status(plan.handle) == lib.FFT3D_OK
    return out.cpu().numpy().astype(np.complex128)


def gpu_c2r(lib, Y64, n2, flags=0):
    """Y64: complex64 numpy (n0, n1, H) (or transposed per flags), batch-leading allowed."""
    if flags & lib.FFT3D_FLAG_EXPLICIT_TRANSPOSE and not flags & lib.FFT3D_FLAG_TRANSPOSE_BACK:
        n1, n0 = Y64.shape[-3], Y64.shape[-2]
    else:
        n0, n1 = Y64.shape[-3], Y64.shape[-2]
    b = 1 if Y64.ndim == 3 else Y64.shape[0]
    plan = lib.Plan(n0, n1, n2, lib.FFT3D_F32, b, flags)
    Yd = torch.from_numpy(np.ascontiguousarray(Y64)).cuda()
    out = torch.empty(Y64.shape[:-3] + (n0, n1, n2), dtype=torch.float32, device="cuda")
    plan.c2r(Yd.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def random_half_spectrum(shape, seed):
    n0, n1, H = shape
    re = synth.uniform_field(shape, seed)
    im = synth.uniform_field(shape, seed + 1)
    return (re + 1j * im).astype(np.complex64)


# ---------------------------------------------------------------------------
# The tiny configuration: 32^3, uniform[-1, 1), seed 1407.
# ---------------------------------------------------------------------------

def test_config1_forward_inverse_roundtrip(cuda_lib):
    n = 32
    x32 = synth.uniform_field((n, n, n), synth.seed_for_config(1)).astype(np.float32)
    X = gpu_r2c(cuda_lib, x32)
    Xo = oracle.r2c3d(x32.astype(np.float64))
    assert rel_l2(X, Xo) <= TOL
    # inverse of the same complex64 input as the oracle
    Y = X.astype(np.complex64)
    y = gpu_c2r(cuda_lib, Y, n)
    assert rel_l2(y, oracle.c2r3d(Y.astype(np.complex128), n)) <= TOL
    # round trip x N
    assert rel_l2(y / n ** 3, x32.astype(np.float64)) <= TOL_RT
    # Parseval on the GPU spectrum
    e = oracle.half_energy(X, n) / n ** 3
    assert abs(e - np.sum(x32.astype(np.float64) ** 2)) <= 1e-5 * e
    # Hermitian symmetry of the k2 = 0 and k2 = n2/2 planes
    for k2 in (0, n // 2):
        P = X[:, :, k2]
        mirror = np.conj(P[(-np.arange(n)) % n][:, (-np.arange(n)) % n])
        assert np.linalg.norm(P - mirror) <= TOL * np.linalg.norm(X)


@pytest.mark.parametrize("k", [(1, 0, 0), (0, 3, 5), (7, -2, 16), (0, 0, 16), (16, 16, 0), (-5, 11, 9)])
def test_config1_single_modes(cuda_lib, k):
    n = 32
    x32 = synth.cosine_mode(n, n, n, *k).astype(np.float32)
    X = gpu_r2c(cuda_lib, x32)
    Xo = oracle.r2c3d(x32.astype(np.float64))
    assert rel_l2(X, Xo) <= TOL
    # the spike: N/2 at k (and at -k on the k2 = 0 / n2/2 planes), N at self-conjugate k
    kp = tuple(v % n for v in k)
    expect = n ** 3 / 2 * (2 if tuple((-v) % n for v in k) == kp else 1)
    assert abs(X[kp] - expect) <= 1e-4 * n ** 3


def test_config1_delta(cuda_lib):
    n = 32
    x32 = synth.delta_field(n, n, n, 3, 5, 7).astype(np.float32)
    X = gpu_r2c(cuda_lib, x32)
    assert rel_l2(X, oracle.r2c3d(x32.astype(np.float64))) <= TOL


# ---------------------------------------------------------------------------
# Shapes: specialised lengths (2^k, 3*2^k, 5*2^k), runtime-generic lengths,
# non-cubic shapes, unit axes, odd H (ragged column tiles), long axes.
# ---------------------------------------------------------------------------
SHAPES = [
    (8, 8, 8), (16, 16, 16), (64, 64, 64), (128, 128, 128), (256, 64, 32), (64, 256, 512),
    (48, 80, 96), (96, 96, 96), (160, 32, 160), (192, 48, 64), (64, 64, 192),
    (6, 10, 16), (15, 12, 10), (30, 20, 24), (2, 2, 2), (1, 1, 2), (1, 8, 16), (4, 1, 8), (5, 3, 2),
    (1536, 2, 4), (2048, 2, 4), (2, 2048, 4), (4, 4, 2048), (2, 3, 4096), (1024, 8, 8), (8, 1024, 8),
    # n0 pass through the TMA kernel: ragged last column tile (OOB fill), P odd falls back
    (512, 6, 10), (512, 5, 6), (256, 3, 4), (256, 40, 60), (1024, 6, 12),
    # warp-resident rows at n2 = 1024, shared-memory rows at n2 = 2048
    (8, 6, 1024), (3, 2, 2048),
    # n1 pass through the TMA kernel: row pairs (odd H) with ragged tiles, plain rows (even H)
    (6, 512, 60), (3, 256, 40), (4, 1024, 30), (5, 256, 512), (1536, 4, 12),
    # row pairs whose last column tile would hold one column
    (2, 512, 64), (3, 1024, 32), (2, 512, 512),
    # n1 = 2048 through the 4-wide TMA kernel: row pairs (H = 17, ragged), plain rows (H = 16)
    (2, 2048, 32), (2, 2048, 30),
    # a factor 7 on every axis (runtime-radix kernels, radix-7 codelet)
    (14, 28, 56), (7, 7, 14), (49, 6, 28), (112, 3, 98), (5, 21, 70),
    # compile-time kernels for 3 * 2^k and 5 * 2^k lengths: columns (n0 and n1,
    # ragged tiles) and warp-resident rows (n2 / 2 = 160 .. 768)
    (320, 4, 6), (4, 320, 10), (384, 5, 7), (3, 384, 4), (640, 2, 4), (2, 640, 6), (768, 2, 4), (2, 768, 3),
    (1280, 2, 4), (2, 1280, 4), (2, 3, 320), (2, 3, 384), (2, 3, 640), (2, 2, 768), (2, 2, 1280), (2, 2, 1536),
    # prime factors above 7 (Bluestein form): every axis, odd and even n2, ragged
    # column tiles, and the longest prime lengths (M = 8192)
    (11, 13, 22), (17, 4, 26), (6, 97, 8), (4, 6, 13), (3, 1021, 4), (143, 3, 10), (2, 2, 8186), (4093, 2, 3),
    (2, 4093, 2), (3, 2, 4093),
    # odd n2 (full-length row transforms, no Nyquist bin)
    (8, 6, 15), (4, 10, 9), (5, 3, 21), (16, 16, 45), (3, 7, 35), (6, 4, 3), (32, 32, 27), (2, 2, 875),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_shapes_forward_and_inverse(cuda_lib, shape):
    n0, n1, n2 = shape
    x32 = synth.uniform_field(shape, seed=17).astype(np.float32)
    X = gpu_r2c(cuda_lib, x32)
    assert rel_l2(X, oracle.r2c3d(x32.astype(np.float64))) <= TOL
    Y = random_half_spectrum((n0, n1, n2 // 2 + 1), seed=23)
    y = gpu_c2r(cuda_lib, Y, n2)
    assert rel_l2(y, oracle.c2r3d(Y.astype(np.complex128), n2)) <= TOL


@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 80, 96), (64, 64, 64)], ids=lambda s: "x".join(map(str, s)))
def test_generic_kernels_forced(cuda_lib, shape):
    n0, n1, n2 = shape
    f = cuda_lib.FFT3D_FLAG_GENERIC
    x32 = synth.uniform_field(shape, seed=29).astype(np.float32)
    assert rel_l2(gpu_r2c(cuda_lib, x32, flags=f), oracle.r2c3d(x32.astype(np.float64))) <= TOL
    Y = random_half_spectrum((n0, n1, n2 // 2 + 1), seed=31)
    assert rel_l2(gpu_c2r(cuda_lib, Y, n2, flags=f), oracle.c2r3d(Y.astype(np.complex128), n2)) <= TOL


@pytest.mark.parametrize("shape", [(32, 32, 32), (128, 128, 128), (64, 256, 256), (4, 512, 512)],
                         ids=lambda s: "x".join(map(str, s)))
def test_fused_plane_vs_three_pass(cuda_lib, shape):
    """Shapes with a fused plane kernel, run fused and with the separate
    row / n1 / n0 passes forced: both match the oracle."""
    n0, n1, n2 = shape
    x32 = synth.uniform_field(shape, seed=57).astype(np.float32)
    Xo = oracle.r2c3d(x32.astype(np.float64))
    Y = random_half_spectrum((n0, n1, n2 // 2 + 1), seed=59)
    yo = oracle.c2r3d(Y.astype(np.complex128), n2)
    for flags in (cuda_lib.FFT3D_FLAG_FUSED_PLANE, 0):
        assert rel_l2(gpu_r2c(cuda_lib, x32, flags=flags), Xo) <= TOL
        assert rel_l2(gpu_c2r(cuda_lib, Y, n2, flags=flags), yo) <= TOL
    assert "plane[fused" in cuda_lib.Plan(n0, n1, n2, flags=cuda_lib.FFT3D_FLAG_FUSED_PLANE).describe()
    assert "plane[fused" not in cuda_lib.Plan(n0, n1, n2).describe()


def test_fused_plane_batched(cuda_lib):
    shape = (2, 16, 32, 32)
    x32 = synth.uniform_field(shape, seed=61).astype(np.float32)
    f = cuda_lib.FFT3D_FLAG_FUSED_PLANE
    X = gpu_r2c(cuda_lib, x32, flags=f)
    for b in range(2):
        assert rel_l2(X[b], oracle.r2c3d(x32[b].astype(np.float64))) <= TOL
    Y = random_half_spectrum((32, 32, 17), seed=62).reshape(2, 16, 32, 17)
    y = gpu_c2r(cuda_lib, Y, 32, flags=f)
    for b in range(2):
        assert rel_l2(y[b], oracle.c2r3d(Y[b].astype(np.complex128), 32)) <= TOL


@pytest.mark.parametrize("shape", [(32, 32, 32), (2, 32, 32, 32), (300, 128, 128), (128, 128, 128), (64, 256, 256),
                                   (4, 512, 512), (40, 512, 512)],
                         ids=lambda s: "x".join(map(str, s)))
def test_cluster_plane_vs_oracle(cuda_lib, shape):
    """Shapes with a cluster plane kernel (rows + n1 columns of each plane in
    one cluster's distributed shared memory), including more planes than
    co-resident clusters and a batch of two: both directions match the oracle."""
    n0, n1, n2 = shape[-3:]
    f = cuda_lib.FFT3D_FLAG_CLUSTER_PLANE
    x32 = synth.uniform_field(shape, seed=65).astype(np.float32)
    X = gpu_r2c(cuda_lib, x32, flags=f)
    lead = shape[:-3]
    Y = random_half_spectrum((int(np.prod(lead, dtype=int)) * n0, n1, n2 // 2 + 1), seed=66)
    Y = Y.reshape(lead + (n0, n1, n2 // 2 + 1))
    y = gpu_c2r(cuda_lib, Y, n2, flags=f)
    for b in range(1 if len(shape) == 3 else shape[0]):
        xb = x32 if len(shape) == 3 else x32[b]
        Xb = X if len(shape) == 3 else X[b]
        Yb = Y if len(shape) == 3 else Y[b]
        yb = y if len(shape) == 3 else y[b]
        assert rel_l2(Xb, oracle.r2c3d(xb.astype(np.float64))) <= TOL
        assert rel_l2(yb, oracle.c2r3d(Yb.astype(np.complex128), n2)) <= TOL
    assert "cluster-plane" in cuda_lib.Plan(n0, n1, n2, flags=f).describe()


def _plan_r2c_c2r(lib, plan, x32, Y64, n2):
    s = torch.cuda.current_stream().cuda_stream
    xd = torch.from_numpy(np.ascontiguousarray(x32)).cuda()
    X = torch.empty(Y64.shape, dtype=torch.complex64, device="cuda")
    plan.r2c(xd.data_ptr(), X.data_ptr(), s)
    Yd = torch.from_numpy(np.ascontiguousarray(Y64)).cuda()
    y = torch.empty(x32.shape, dtype=torch.float32, device="cuda")
    plan.c2r(Yd.data_ptr(), y.data_ptr(), s)
    torch.cuda.synchronize()
    return X.cpu().numpy().astype(np.complex128), y.cpu().numpy().astype(np.float64)


# TMA-fed column kernels of the 3*2^k, 5*2^k and short lengths, forced on
# both axes: n0 tiles (ragged: P not a multiple of the tile width) and n1 row
# pairs (odd H) or plain rows (even H); boxes of the largest divisor of the
# tile rows up to 256 for L > 256.
TMA_LEN_SHAPES = [(64, 3, 12), (2, 64, 32), (96, 5, 12), (2, 96, 32), (128, 3, 10), (2, 128, 34),
                  (160, 3, 12), (2, 160, 32), (192, 3, 12), (2, 192, 32), (320, 4, 14), (2, 320, 32),
                  (2, 320, 30), (384, 3, 12), (2, 384, 32), (640, 3, 10), (2, 640, 32), (768, 3, 10),
                  (2, 768, 32)]


@pytest.mark.parametrize("shape", TMA_LEN_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_tma_column_kernels_of_every_length_match_oracle(cuda_lib, shape):
    lib = cuda_lib
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    plan = lib.Plan(n0, n1, n2)
    assert lib.fft3d_set_choices(plan.handle, [0, 0, 0, 1, 1]) == lib.FFT3D_OK
    desc = plan.describe()
    long_axis = 0 if n0 > n1 else 1
    assert ("tma" in desc.split("n0[")[1].split("]")[0]) if long_axis == 0 else \
        ("tma" in desc.split("n1[")[1].split("]")[0]), desc
    x32 = synth.uniform_field(shape, seed=79).astype(np.float32)
    xd = torch.from_numpy(x32).cuda()
    X = torch.empty((n0, n1, H), dtype=torch.complex64, device="cuda")
    plan.r2c(xd.data_ptr(), X.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(X.cpu().numpy(), oracle.r2c3d(x32.astype(np.float64))) <= TOL
    Y = random_half_spectrum((n0, n1, H), seed=83)
    Yd = torch.from_numpy(Y).cuda()
    y = torch.empty_like(xd)
    plan.c2r(Yd.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(y.cpu().numpy(), oracle.c2r3d(Y.astype(np.complex128), n2)) <= TOL
    assert lib.fft3d_query_device_status(plan.handle) == lib.FFT3D_OK
    plan.close()


@pytest.mark.parametrize("shape", [(9, 32, 32), (10, 64, 64), (5, 128, 128), (6, 256, 256), (3, 512, 512),
                                   (4, 96, 96), (3, 160, 160), (2, 192, 192)],
                         ids=lambda s: "x".join(map(str, s)))
def test_plane_form_every_cluster_size_and_autotune(cuda_lib, shape):
    """Every instantiated cluster size of a plane shape (set through
    fft3d_set_plane_choice) and the separate-pass form match the oracle; the
    autotuner picks one of them and the tuned plan still matches."""
    lib = cuda_lib
    n0, n1, n2 = shape
    x32 = synth.uniform_field(shape, seed=67).astype(np.float32)
    Y = random_half_spectrum((n0, n1, n2 // 2 + 1), seed=68)
    Xo = oracle.r2c3d(x32.astype(np.float64))
    yo = oracle.c2r3d(Y.astype(np.complex128), n2)
    sizes = []
    for C in (0, 1, 2, 3, 4, 5, 8, 16):
        plan = lib.Plan(n0, n1, n2)
        st = lib.fft3d_set_plane_choice(plan.handle, C)
        if st != lib.FFT3D_OK:
            assert st == lib.FFT3D_ERR_UNSUPPORTED_SIZE
            assert lib.fft3d_get_plane_choice(plan.handle) == 0
            continue
        assert lib.fft3d_get_plane_choice(plan.handle) == C
        assert ("cluster-plane" in plan.describe()) == (C > 0)
        sizes.append(C)
        X, y = _plan_r2c_c2r(lib, plan, x32, Y, n2)
        assert rel_l2(X, Xo) <= TOL, C
        assert rel_l2(y, yo) <= TOL, C
    assert len(sizes) >= 2
    plan = lib.Plan(n0, n1, n2)
    real = torch.empty(n0 * n1 * n2, dtype=torch.float32, device="cuda").normal_()
    cplx = torch.empty(n0 * n1 * (n2 // 2 + 1), dtype=torch.complex64, device="cuda")
    assert lib.fft3d_autotune(plan.handle, real.data_ptr(), cplx.data_ptr(), 2,
                              torch.cuda.current_stream().cuda_stream) == lib.FFT3D_OK
    assert lib.fft3d_get_plane_choice(plan.handle) in sizes
    X, y = _plan_r2c_c2r(lib, plan, x32, Y, n2)
    assert rel_l2(X, Xo) <= TOL and rel_l2(y, yo) <= TOL
    # forms the choice does not apply to
    tp = lib.Plan(n0, n1, n2, flags=lib.FFT3D_FLAG_THREE_PASS)
    assert lib.fft3d_set_plane_choice(tp.handle, sizes[-1]) == lib.FFT3D_ERR_INVALID_ARG


PADDED_SHAPES = [(32, 32, 32), (64, 64, 64), (6, 512, 60), (8, 6, 1024), (3, 2, 2048), (2, 3, 4096), (48, 80, 96),
                 (5, 3, 2), (1, 8, 16), (4, 6, 9), (3, 5, 15), (4, 6, 26), (3, 11, 13), (4, 3, 768), (2, 5, 640)]


@pytest.mark.parametrize("extra", ["plain", "generic", "tc"])
@pytest.mark.parametrize("shape", PADDED_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_padded_real_layout_in_and_out_of_place(cuda_lib, shape, extra):
    """FFTW's padded real layout (rows of 2H floats): r2c and c2r out of place
    and in place match the oracle; r2c never reads the padding (NaN there) and
    an out-of-place c2r never writes it."""
    lib = cuda_lib
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    flags = lib.FFT3D_FLAG_PADDED_REAL | (lib.FFT3D_FLAG_GENERIC if extra == "generic" else 0)
    dtype = lib.FFT3D_F32_TC_BF16X3 if extra == "tc" else lib.FFT3D_F32
    tol = 1e-5 if extra == "tc" else TOL
    try:
        plan = lib.Plan(n0, n1, n2, dtype=dtype, flags=flags)
    except lib.Fft3dError as e:
        assert extra == "tc" and e.status == lib.FFT3D_ERR_UNSUPPORTED_SIZE  # no tensor-core axis at this size
        return
    s = torch.cuda.current_stream().cuda_stream
    x32 = synth.uniform_field(shape, seed=71).astype(np.float32)
    Xo = oracle.r2c3d(x32.astype(np.float64))
    xp = np.full((n0, n1, 2 * H), np.nan, dtype=np.float32)
    xp[..., :n2] = x32
    buf = torch.from_numpy(xp).cuda()
    X = torch.empty((n0, n1, H), dtype=torch.complex64, device="cuda")
    plan.r2c(buf.data_ptr(), X.data_ptr(), s)
    torch.cuda.synchronize()
    assert rel_l2(X.cpu().numpy(), Xo) <= tol
    plan.r2c(buf.data_ptr(), buf.data_ptr(), s)  # in place
    torch.cuda.synchronize()
    assert rel_l2(buf.view(torch.complex64).cpu().numpy(), Xo) <= tol
    Y = random_half_spectrum((n0, n1, H), seed=72)
    yo = oracle.c2r3d(Y.astype(np.complex128), n2)
    Yd = torch.from_numpy(Y).cuda()
    out = torch.full((n0, n1, 2 * H), 7.0, dtype=torch.float32, device="cuda")
    plan.c2r(Yd.data_ptr(), out.data_ptr(), s)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert rel_l2(o[..., :n2], yo) <= tol
    assert np.all(o[..., n2:] == 7.0)
    Yd = torch.from_numpy(Y).cuda()
    plan.c2r(Yd.data_ptr(), Yd.data_ptr(), s)  # in place
    torch.cuda.synchronize()
    assert rel_l2(Yd.view(torch.float32).cpu().numpy().reshape(n0, n1, 2 * H)[..., :n2], yo) <= tol
    # a partial overlap is still rejected
    assert lib.fft3d_r2c(plan.handle, buf.data_ptr(), buf.data_ptr() + 16, s) == lib.FFT3D_ERR_INVALID_ARG


@pytest.mark.parametrize("shape,plane", [((32, 32, 32), 0), ((5, 128, 128), 2), ((1, 8, 16), 0), ((4, 1, 8), 0),
                                         ((6, 512, 60), 0), ((64, 64, 64), 1), ((11, 13, 22), 0), ((7, 5, 9), 0)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else f"plane{v}")
def test_preserve_input_c2r(cuda_lib, shape, plane):
    """FFT3D_FLAG_PRESERVE_INPUT: c2r leaves its input bit for bit unchanged
    (the first column pass writes the plan's workspace) and still matches the
    oracle, with the separate passes or a cluster plane kernel."""
    lib = cuda_lib
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    for flags in (lib.FFT3D_FLAG_PRESERVE_INPUT, lib.FFT3D_FLAG_PRESERVE_INPUT | lib.FFT3D_FLAG_PADDED_REAL):
        plan = lib.Plan(n0, n1, n2, flags=flags)
        assert lib.fft3d_workspace_bytes(plan.handle) == n0 * n1 * H * 8
        if plane and not flags & lib.FFT3D_FLAG_PADDED_REAL:
            assert lib.fft3d_set_plane_choice(plan.handle, plane) == lib.FFT3D_OK
        s = torch.cuda.current_stream().cuda_stream
        Y = random_half_spectrum((n0, n1, H), seed=73)
        yo = oracle.c2r3d(Y.astype(np.complex128), n2)
        Yd = torch.from_numpy(Y).cuda()
        keep = Yd.clone()
        rw = 2 * H if flags & lib.FFT3D_FLAG_PADDED_REAL else n2
        out = torch.empty((n0, n1, rw), dtype=torch.float32, device="cuda")
        plan.c2r(Yd.data_ptr(), out.data_ptr(), s)
        torch.cuda.synchronize()
        assert torch.equal(Yd, keep)
        assert rel_l2(out.cpu().numpy()[..., :n2], yo) <= TOL
        assert lib.fft3d_c2r(plan.handle, Yd.data_ptr(), Yd.data_ptr(), s) == lib.FFT3D_ERR_INVALID_ARG


def test_padded_and_preserve_flag_combinations(cuda_lib):
    lib = cuda_lib
    for bad in (lib.FFT3D_FLAG_PADDED_REAL | lib.FFT3D_FLAG_EXPLICIT_TRANSPOSE,
                lib.FFT3D_FLAG_PRESERVE_INPUT | lib.FFT3D_FLAG_FUSED_PLANE):
        assert not lib.fft3d_plan_variant(32, 32, 32, lib.FFT3D_F32, 1, bad)
        assert lib.fft3d_last_error() == lib.FFT3D_ERR_INVALID_ARG
    plan = lib.Plan(32, 32, 32, flags=lib.FFT3D_FLAG_PADDED_REAL)
    assert lib.fft3d_set_plane_choice(plan.handle, 2) == lib.FFT3D_ERR_INVALID_ARG
    raw = lib.fft3d_plan_variant(32, 32, 32, lib.FFT3D_F32, 1, lib.FFT3D_FLAG_PRESERVE_INPUT)
    x = torch.empty(32 * 32 * 17, dtype=torch.complex64, device="cuda")
    y = torch.empty(32 ** 3, dtype=torch.float32, device="cuda")
    assert lib.fft3d_c2r(raw, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream) == \
        lib.FFT3D_ERR_NO_WORKSPACE
    lib.fft3d_destroy(raw)


@pytest.mark.parametrize("shape,chunking", [((32, 32, 32), (0, 1)), ((16, 32, 64), (0, 1)), ((64, 64, 64), (0, 1)),
                                            ((64, 64, 64), (16, 2)), ((16, 32, 64), (3, 1))],
                         ids=lambda v: "x".join(map(str, v)) if len(v) == 3 else "c%d_s%d" % v)
def test_navier_stokes_step_matches_oracle(cuda_lib, shape, chunking):
    """One Heun step of the pseudo-spectral Navier-Stokes equations (nonlinear
    term twice, two fused stage kernels, one captured graph) against the FP64
    oracle step: the new state within 1e-6, its increment within 5e-5 (both
    relative L2), bins outside the 2/3 rule bit for bit unchanged; launched
    directly on the legacy stream and as a replayed graph on a side stream."""
    lib = cuda_lib
    n0, n1, n2 = shape
    U64 = synth.spectral_velocity(n0, n1, n2, seed=93).astype(np.complex64)
    U = U64.astype(np.complex128)
    nu = 0.02
    r0 = oracle.ns_rhs(U, n2, nu)
    dt = float(0.01 * np.linalg.norm(U) / np.linalg.norm(r0))  # |increment| about 1 % of |u|
    ref = oracle.ns_step_rk2(U, n2, nu, np.float32(dt))
    ns = lib.NavierStokes(n0, n1, n2)
    assert lib.fft3d_ns_set_chunking(ns.handle, *chunking) == lib.FFT3D_OK
    # two nonlinear terms (n0 inverse; per chunk of planes n1 inverse, rows, n1
    # forward; the n0 forward over two kept k1 blocks) and two stage kernels
    chunks = -(-n0 // chunking[0]) if 0 < chunking[0] < n0 else 1
    launches = 2 * (1 + 3 * chunks + 2) + 2
    assert lib.fft3d_ns_launches(ns.handle) == launches
    mask = oracle.dealias_mask(n0, n1, n2)
    results = []
    u = torch.from_numpy(U64).cuda()
    ns.step(u, nu, dt, stream=False)  # legacy default stream: direct launches
    torch.cuda.synchronize()
    results.append(u.cpu().numpy())
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):  # first call captures the graph, the second replays it
            u = torch.from_numpy(U64).cuda()
            ns.step(u, nu, dt, stream=side)
            side.synchronize()
            results.append(u.cpu().numpy())
    assert lib.fft3d_ns_launches(ns.handle) == launches  # now the kernel nodes of the captured graph
    for got in results:
        got = got.astype(np.complex128)
        assert rel_l2(got, ref) <= 1e-6
        assert rel_l2(got - U, ref - U) <= 5e-5
        assert np.array_equal(got[:, ~mask], U64[:, ~mask].astype(np.complex128))
    ns.close()


def test_navier_stokes_rejects_bad_arguments(cuda_lib):
    lib = cuda_lib
    assert not lib.fft3d_ns_plan(30, 30, 30)  # n2/2 = 15 has no warp-resident row kernel
    assert lib.fft3d_last_error() == lib.FFT3D_ERR_UNSUPPORTED_SIZE
    h = lib.fft3d_ns_plan(16, 16, 16)
    u = torch.zeros((3, 16, 16, 9), dtype=torch.complex64, device="cuda")
    assert lib.fft3d_ns_step(h, u.data_ptr(), 0.01, 0.1, 0) == lib.FFT3D_ERR_NO_WORKSPACE
    ws = torch.empty(lib.fft3d_ns_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    assert lib.fft3d_ns_set_workspace(h, ws.data_ptr()) == lib.FFT3D_OK
    assert lib.fft3d_ns_step(h, u.data_ptr(), -1.0, 0.1, 0) == lib.FFT3D_ERR_INVALID_ARG
    assert lib.fft3d_ns_step(h, u.data_ptr(), 0.01, 0.0, 0) == lib.FFT3D_ERR_INVALID_ARG
    assert lib.fft3d_ns_step(h, ws.data_ptr(), 0.01, 0.1, 0) == lib.FFT3D_ERR_INVALID_ARG  # overlaps the workspace
    assert lib.fft3d_ns_step(h, u.data_ptr(), 0.01, 0.1, 0) == lib.FFT3D_OK
    torch.cuda.synchronize()
    lib.fft3d_ns_destroy(h)


@pytest.mark.parametrize("shape", [(8, 6, 15), (6, 10, 32)], ids=lambda s: "x".join(map(str, s)))
def test_energy_weights_follow_n2_parity(cuda_lib, shape):
    """Parseval on the device: the last bin weighs 1 only when it is a Nyquist
    bin (even n2)."""
    n0, n1, n2 = shape
    x32 = synth.uniform_field(shape, seed=95).astype(np.float32)
    plan = cuda_lib.Plan(n0, n1, n2)
    X = torch.empty((n0, n1, n2 // 2 + 1), dtype=torch.complex64, device="cuda")
    plan.r2c(torch.from_numpy(x32).cuda().data_ptr(), X.data_ptr(), torch.cuda.current_stream().cuda_stream)
    total, _ = plan.energy(X, 4)
    ref = oracle.half_energy(X.cpu().numpy(), n2)
    assert abs(total.item() - ref) <= 1e-9 * ref
    assert abs(total.item() / (n0 * n1 * n2) - np.sum(x32.astype(np.float64) ** 2)) <= 1e-5 * ref / (n0 * n1 * n2)


def test_bounded_wait_gives_up_without_hanging(cuda_lib):
    """Failure detection without a GPU fault: with the test hook, the
    producers of plane 0 never report, so the consumers' bounded waits give up
    (about a millisecond), the kernel returns, and the host reads
    FFT3D_ERR_TIMEOUT from the status word; the context stays usable."""
    lib = cuda_lib
    n = 32
    plan = lib.Plan(n, n, n, flags=lib.FFT3D_FLAG_FUSED_PLANE | lib.FFT3D_FLAG_TEST_SKIP_ARRIVAL)
    assert "plane[fused" in plan.describe()
    x = torch.zeros((n, n, n), dtype=torch.float32, device="cuda")
    X = torch.empty((n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.fft3d_r2c(plan.handle, x.data_ptr(), X.data_ptr(), s) == lib.FFT3D_OK
    assert lib.fft3d_query_device_status(plan.handle, s) == lib.FFT3D_ERR_TIMEOUT
    # the status word was cleared by the query, and the device still works
    assert lib.fft3d_query_device_status(plan.handle, s) == lib.FFT3D_OK
    x32 = synth.uniform_field((n, n, n), seed=63).astype(np.float32)
    assert rel_l2(gpu_r2c(lib, x32), oracle.r2c3d(x32.astype(np.float64))) <= TOL


def test_batched_tma_column_pass(cuda_lib):
    shape = (3, 256, 8, 12)
    x32 = synth.uniform_field(shape, seed=39).astype(np.float32)
    X = gpu_r2c(cuda_lib, x32)
    for b in range(3):
        assert rel_l2(X[b], oracle.r2c3d(x32[b].astype(np.float64))) <= TOL
    Y = random_half_spectrum((3 * 256, 8, 7), seed=40).reshape(3, 256, 8, 7)
    y = gpu_c2r(cuda_lib, Y, 12)
    for b in range(3):
        assert rel_l2(y[b], oracle.c2r3d(Y[b].astype(np.complex128), 12)) <= TOL


@pytest.mark.parametrize("shape", [(3, 16, 24, 20), (3, 11, 13, 22), (2, 6, 10, 15), (2, 5, 17, 9)],
                         ids=lambda s: "x".join(map(str, s)))
def test_batch_entries_do_not_bleed(cuda_lib, shape):
    """Batch offsets on specialised, Bluestein (11, 13, 17) and odd-n2 paths."""
    B, n0, n1, n2 = shape
    H = n2 // 2 + 1
    x32 = synth.uniform_field(shape, seed=37).astype(np.float32)
    X = gpu_r2c(cuda_lib, x32)
    for b in range(B):
        assert rel_l2(X[b], oracle.r2c3d(x32[b].astype(np.float64))) <= TOL
    Y = random_half_spectrum((B * n0, n1, H), seed=41).reshape(B, n0, n1, H)
    y = gpu_c2r(cuda_lib, Y, n2)
    for b in range(B):
        assert rel_l2(y[b], oracle.c2r3d(Y[b].astype(np.complex128), n2)) <= TOL


@pytest.mark.parametrize("shape", [(24, 40, 36), (11, 13, 26)], ids=lambda s: "x".join(map(str, s)))
def test_impulses_map_to_plane_waves(cuda_lib, shape):
    """A delta at (j0, j1, j2) transforms to exp(-2 pi i k.j/n): checks every
    index placement, including the rows and columns at the tile edges (and,
    at 11 x 13 x 26, the Bluestein chirp indices)."""
    n0, n1, n2 = shape
    for j in [(0, 0, 0), (n0 - 1, n1 - 1, n2 - 1), (5, 7, 1), (n0 // 2, n1 // 2, n2 // 2)]:
        x32 = synth.delta_field(*shape, *j).astype(np.float32)
        X = gpu_r2c(cuda_lib, x32)
        assert rel_l2(X, oracle.r2c3d(x32.astype(np.float64))) <= TOL


def test_c2r_ignores_imag_of_dc_and_nyquist_bins(cuda_lib):
    n0, n1, n2 = 8, 12, 16
    Y = random_half_spectrum((n0, n1, n2 // 2 + 1), seed=43)
    y = gpu_c2r(cuda_lib, Y, n2)
    assert rel_l2(y, oracle.c2r3d(Y.astype(np.complex128), n2)) <= TOL
    assert rel_l2(y, oracle.c2r3d_naive(Y.astype(np.complex128), n2)) <= TOL


@pytest.mark.parametrize("back", [False, True])
@pytest.mark.parametrize("shape", [(32, 48, 40), (11, 13, 22)], ids=lambda s: "x".join(map(str, s)))
def test_explicit_transpose_variant(cuda_lib, back, shape):
    n0, n1, n2 = shape
    f = cuda_lib.FFT3D_FLAG_EXPLICIT_TRANSPOSE | (cuda_lib.FFT3D_FLAG_TRANSPOSE_BACK if back else 0)
    x32 = synth.uniform_field((n0, n1, n2), seed=47).astype(np.float32)
    X = gpu_r2c(cuda_lib, x32, flags=f)
    Xo = oracle.r2c3d(x32.astype(np.float64))
    assert rel_l2(X, Xo if back else Xo.transpose(1, 0, 2)) <= TOL
    Y = random_half_spectrum((n0, n1, n2 // 2 + 1), seed=53)
    yo = oracle.c2r3d(Y.astype(np.complex128), n2)
    Yin = Y if back else np.ascontiguousarray(Y.transpose(1, 0, 2))
    assert rel_l2(gpu_c2r(cuda_lib, Yin, n2, flags=f), yo) <= TOL


def test_argument_errors_leave_output_untouched(cuda_lib):
    lib = cuda_lib
    plan = lib.Plan(8, 8, 8)
    x = torch.zeros(8 * 8 * 8 + 8, dtype=torch.float32, device="cuda")
    out = torch.full((8 * 8 * 5 * 2 + 8,), 7.0, dtype=torch.float32, device="cuda")
    assert lib.fft3d_r2c(plan.handle, x.data_ptr() + 4, out.data_ptr()) == lib.FFT3D_ERR_MISALIGNED
    assert lib.fft3d_r2c(plan.handle, x.data_ptr(), x.data_ptr() + 16) == lib.FFT3D_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
    xp = lib.fft3d_plan_variant(8, 8, 8, 0, 1, lib.FFT3D_FLAG_EXPLICIT_TRANSPOSE)
    assert lib.fft3d_workspace_bytes(xp) == 8 * 8 * 5 * 8
    assert lib.fft3d_r2c(xp, x.data_ptr(), out.data_ptr()) == lib.FFT3D_ERR_NO_WORKSPACE
    assert lib.fft3d_set_workspace(xp, out.data_ptr() + 16) == lib.FFT3D_ERR_MISALIGNED
    lib.fft3d_destroy(xp)


# ---------------------------------------------------------------------------
# Pseudo-spectral nonlinear term: tolerance 1e-5 rel-L2 per output field
# (three inverse and one forward FP32 transform compose).
# ---------------------------------------------------------------------------
TOL_NL = 1e-5


NL_CASES = [((32, 32, 32), (0, 1)), ((32, 48, 64), (0, 1)), ((256, 256, 256), (0, 1)), ((22, 13, 32), (0, 1)),
            # plane chunks of the middle passes: ragged last chunk, one plane per
            # chunk, two streams, a chunk larger than n0, the Bluestein axes
            ((32, 32, 32), (5, 1)), ((32, 48, 64), (1, 2)), ((32, 48, 64), (7, 2)), ((256, 256, 256), (16, 2)),
            ((256, 256, 256), (48, 1)), ((22, 13, 32), (4, 2)), ((16, 32, 64), (64, 2))]


@functools.lru_cache(maxsize=None)  # one oracle term per distinct shape of NL_CASES
def _nl_case(shape):
    n0, n1, n2 = shape
    U64 = synth.spectral_velocity(n0, n1, n2, seed=synth.seed_for_config(4)).astype(np.complex64)
    return U64, oracle.nonlinear_term(U64.astype(np.complex128), n2)


@pytest.mark.parametrize("shape,chunking", NL_CASES,
                         ids=lambda v: "x".join(map(str, v)) if len(v) == 3 else "c%d_s%d" % v)
def test_nonlinear_term_matches_oracle(cuda_lib, shape, chunking):
    n0, n1, n2 = shape
    U64, ref = _nl_case(shape)
    nl = cuda_lib.NonlinearTerm(n0, n1, n2)
    assert cuda_lib.fft3d_nonlinear_set_chunking(nl.handle, *chunking) == cuda_lib.FFT3D_OK
    assert cuda_lib.fft3d_nonlinear_get_chunking(nl.handle) == chunking
    planned = cuda_lib.fft3d_nonlinear_launches(nl.handle)
    ud = torch.from_numpy(U64).cuda()
    u_before = ud.clone()
    out = torch.empty((6, n0, n1, n2 // 2 + 1), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    results = []
    with torch.cuda.stream(stream):
        nl(ud, out=out, stream=stream)   # first call: captured into a graph and launched
        results.append(out.clone())
        out.zero_()
        nl(ud, out=out, stream=stream)   # same operands: the graph is replayed
        results.append(out.clone())
    stream.synchronize()
    assert cuda_lib.fft3d_nonlinear_launches(nl.handle) == planned  # the captured graph's kernel nodes
    results.append(nl(ud, stream=False))  # legacy default stream: direct launches
    torch.cuda.synchronize()
    assert torch.equal(ud, u_before)     # the input spectra are preserved
    for r in results:
        got = r.cpu().numpy().astype(np.complex128)
        for q in range(6):
            assert rel_l2(got[q], ref[q]) <= TOL_NL, q
    mask = oracle.dealias_mask(n0, n1, n2)
    assert np.all(results[0].cpu().numpy()[:, ~mask] == 0)
    nl.close()


def test_nonlinear_term_recaptures_for_new_buffers(cuda_lib):
    n = 32
    U = synth.spectral_velocity(n, n, n, seed=77).astype(np.complex64)
    V = synth.spectral_velocity(n, n, n, seed=78).astype(np.complex64)
    nl = cuda_lib.NonlinearTerm(n, n, n)
    Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        a = nl(Ud, stream=s)
        b = nl(Vd, stream=s)
    s.synchronize()
    for x, ref in ((a, oracle.nonlinear_term(U.astype(np.complex128), n)),
                   (b, oracle.nonlinear_term(V.astype(np.complex128), n))):
        got = x.cpu().numpy().astype(np.complex128)
        assert max(rel_l2(got[q], ref[q]) for q in range(6)) <= TOL_NL
    nl.close()


# ---------------------------------------------------------------------------
# Tensor-core radix-16 forms: split-BF16 (3 products) <= 1e-5, FP16 <= 3e-3.
# ---------------------------------------------------------------------------
TC_TOL = {1: 1e-5, 2: 3e-3}


def gpu_r2c_dtype(lib, x32, dtype):
    n0, n1, n2 = x32.shape[-3:]
    b = 1 if x32.ndim == 3 else x32.shape[0]
    plan = lib.Plan(n0, n1, n2, dtype, b)
    xd = torch.from_numpy(np.ascontiguousarray(x32)).cuda()
    out = torch.empty(x32.shape[:-1] + (n2 // 2 + 1,), dtype=torch.complex64, device="cuda")
    plan.r2c(xd.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    assert lib.fft3d_query_device_status(plan.handle) == lib.FFT3D_OK
    return out.cpu().numpy().astype(np.complex128), plan.describe()


def gpu_c2r_dtype(lib, Y64, n2, dtype):
    n0, n1 = Y64.shape[-3], Y64.shape[-2]
    b = 1 if Y64.ndim == 3 else Y64.shape[0]
    plan = lib.Plan(n0, n1, n2, dtype, b)
    Yd = torch.from_numpy(np.ascontiguousarray(Y64)).cuda()
    out = torch.empty(Y64.shape[:-3] + (n0, n1, n2), dtype=torch.float32, device="cuda")
    plan.c2r(Yd.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", [1, 2], ids=["bf16x3", "fp16"])
@pytest.mark.parametrize("shape", [(256, 256, 32), (512, 64, 16), (32, 512, 16), (1024, 16, 8), (2048, 4, 6),
                                   (256, 24, 20), (256, 11, 26)], ids=lambda s: "x".join(map(str, s)) if isinstance(s, tuple) else s)
def test_tensor_core_forms_match_oracle(cuda_lib, shape, dtype):
    n0, n1, n2 = shape
    x32 = synth.uniform_field(shape, seed=101).astype(np.float32)
    X, desc = gpu_r2c_dtype(cuda_lib, x32, dtype)
    assert "tensor-core" in desc
    err = rel_l2(X, oracle.r2c3d(x32.astype(np.float64)))
    assert err <= TC_TOL[dtype], err
    Y = random_half_spectrum((n0, n1, n2 // 2 + 1), seed=103)
    y = gpu_c2r_dtype(cuda_lib, Y, n2, dtype)
    err = rel_l2(y, oracle.c2r3d(Y.astype(np.complex128), n2))
    assert err <= TC_TOL[dtype], err


def test_tensor_core_form_batched_and_unsupported(cuda_lib):
    lib = cuda_lib
    x32 = synth.uniform_field((2, 256, 8, 12), seed=105).astype(np.float32)
    X, _ = gpu_r2c_dtype(lib, x32, 1)
    for b in range(2):
        assert rel_l2(X[b], oracle.r2c3d(x32[b].astype(np.float64))) <= TC_TOL[1]
    # no axis of length 256..2048 with a tensor-core kernel: the form is not offered
    assert not lib.fft3d_plan(32, 32, 32, 1, 1)
    assert lib.fft3d_last_error() == lib.FFT3D_ERR_UNSUPPORTED_SIZE
    assert not lib.fft3d_plan_variant(256, 8, 8, 1, 1, lib.FFT3D_FLAG_EXPLICIT_TRANSPOSE)


# ---------------------------------------------------------------------------
# Grouped uneven batch (64^3, 96^3, 128^3, 192^3, 160^3 x 4 fields) and the
# autotuner.
# ---------------------------------------------------------------------------
GROUP_DIMS = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (192, 192, 192), (160, 160, 160)]


@pytest.mark.parametrize("form", ["work_table", "streams"])
def test_grouped_uneven_batch_matches_oracle(cuda_lib, form):
    """Both group forms (the persistent work-table launch, and the per-size
    plans on forked streams): forward, inverse and the one-call round trip,
    captured and replayed, and on the legacy default stream; every field of
    every size against the oracle."""
    lib = cuda_lib
    counts = [4] * len(GROUP_DIMS)
    g = lib.Group(GROUP_DIMS, counts)
    assert g.form == lib.FFT3D_GROUP_STREAMS  # the default
    g.form = lib.FFT3D_GROUP_WORK_TABLE if form == "work_table" else lib.FFT3D_GROUP_STREAMS
    xs, Xs, refs, Xrefs = [], [], [], []
    for i, (n0, n1, n2) in enumerate(GROUP_DIMS):
        x32 = synth.uniform_field((4, n0, n1, n2), seed=synth.seed_for_config(4, field=i + 1)).astype(np.float32)
        xs.append(torch.from_numpy(x32).cuda())
        Xs.append(torch.empty((4, n0, n1, n2 // 2 + 1), dtype=torch.complex64, device="cuda"))
        refs.append(x32)
        Xrefs.append(oracle.r2c3d(x32.astype(np.float64)))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g.r2c(xs, Xs, stream=s.cuda_stream)   # captured into one graph
        g.r2c(xs, Xs, stream=s.cuda_stream)   # replayed
    s.synchronize()
    assert lib.fft3d_group_query_device_status(g.handle, 0) == lib.FFT3D_OK
    for i in range(len(GROUP_DIMS)):
        got = Xs[i].cpu().numpy().astype(np.complex128)
        for f in range(4):
            assert rel_l2(got[f], Xrefs[i][f]) <= TOL, (i, f)
    # inverse on the legacy default stream (launched directly), inputs clobbered
    Ys = [X.clone() for X in Xs]
    outs = [torch.empty_like(x) for x in xs]
    g.c2r(Ys, outs, stream=0)
    torch.cuda.synchronize()
    for i, (n0, n1, n2) in enumerate(GROUP_DIMS):
        y = outs[i].cpu().numpy().astype(np.float64)
        ref = oracle.c2r3d(Xs[i].cpu().numpy().astype(np.complex128), n2)
        for f in range(4):
            assert rel_l2(y[f], ref[f]) <= TOL, (i, f)
    # the round trip in one call (captured, replayed twice)
    mids = [torch.empty_like(X) for X in Xs]
    outs2 = [torch.full_like(x, float("nan")) for x in xs]
    with torch.cuda.stream(s):
        for _ in range(2):
            g.r2c_c2r(xs, mids, outs2, stream=s.cuda_stream)
    s.synchronize()
    for i, (n0, n1, n2) in enumerate(GROUP_DIMS):
        N = n0 * n1 * n2
        y = outs2[i].cpu().numpy().astype(np.float64)
        for f in range(4):
            assert rel_l2(y[f] / N, refs[i][f].astype(np.float64)) <= TOL_RT, (i, f)
    if form == "work_table":
        assert [lib.fft3d_group_launches(g.handle, d) for d in (-1, 1, 0)] == [1, 1, 1]
    else:
        assert lib.fft3d_group_launches(g.handle, -1) == 15 and lib.fft3d_group_launches(g.handle, 0) == 30
    g.close()


def test_group_work_table_availability_and_bounded_wait(cuda_lib):
    """A group with a size that has no work-table bodies keeps the streams
    form and refuses the work table; the test form with an unmeetable
    dependency gives up (bounded), reports FFT3D_ERR_TIMEOUT, and the same
    group then transforms correctly."""
    lib = cuda_lib
    g = lib.Group([(64, 64, 64), (250, 10, 12)], [1, 1])
    assert g.form == lib.FFT3D_GROUP_STREAMS
    assert lib.fft3d_group_set_form(g.handle, lib.FFT3D_GROUP_WORK_TABLE) == lib.FFT3D_ERR_INVALID_ARG
    g.close()
    dims = [(64, 64, 64), (96, 96, 96)]
    g = lib.Group(dims, [1, 2])
    xs = [torch.from_numpy(synth.uniform_field((c, *d), seed=70 + c).astype(np.float32)).cuda()
          for d, c in zip(dims, (1, 2))]
    Xs = [torch.empty((c, d[0], d[1], d[2] // 2 + 1), dtype=torch.complex64, device="cuda")
          for d, c in zip(dims, (1, 2))]
    g.form = lib.FFT3D_GROUP_WORK_TABLE_TEST_STALL
    g.r2c(xs, Xs, stream=0)
    assert lib.fft3d_group_query_device_status(g.handle, 0) == lib.FFT3D_ERR_TIMEOUT
    g.form = lib.FFT3D_GROUP_WORK_TABLE
    g.r2c(xs, Xs, stream=0)
    torch.cuda.synchronize()
    assert lib.fft3d_group_query_device_status(g.handle, 0) == lib.FFT3D_OK
    for x, X in zip(xs, Xs):
        ref = oracle.r2c3d(x.cpu().numpy().astype(np.float64))
        assert rel_l2(X.cpu().numpy().astype(np.complex128), ref) <= TOL
    g.close()


def test_autotune_keeps_parity_and_choices_roundtrip(cuda_lib):
    lib = cuda_lib
    n0, n1, n2 = 256, 96, 128
    plan = lib.Plan(n0, n1, n2)
    real = torch.randn(n0 * n1 * n2, device="cuda")
    cplx = torch.empty(n0 * n1 * (n2 // 2 + 1), dtype=torch.complex64, device="cuda")
    assert lib.fft3d_autotune(plan.handle, real.data_ptr(), cplx.data_ptr(), 2) == lib.FFT3D_OK
    ch = lib.fft3d_get_choices(plan.handle)
    assert len(ch) == 5 and ch[3] in (0, 1) and ch[4] in (0, 1)
    x32 = synth.uniform_field((n0, n1, n2), seed=91).astype(np.float32)
    xd = torch.from_numpy(x32).cuda()
    X = torch.empty((n0, n1, n2 // 2 + 1), dtype=torch.complex64, device="cuda")
    plan.r2c(xd.data_ptr(), X.data_ptr())
    assert rel_l2(X.cpu().numpy(), oracle.r2c3d(x32.astype(np.float64))) <= TOL
    # every candidate shape gives the same transform
    for choice in ([0, 0, 0, 1, 1], [4, 8, 2, 0, 0], [8, 16, 4, 0, 1], [0, 0, 0, 1, 0]):
        assert lib.fft3d_set_choices(plan.handle, choice) == lib.FFT3D_OK
        assert lib.fft3d_get_choices(plan.handle) == choice
        plan.r2c(xd.data_ptr(), X.data_ptr())
        assert rel_l2(X.cpu().numpy(), oracle.r2c3d(x32.astype(np.float64))) <= TOL
        Y = X.clone()
        y = torch.empty_like(xd)
        plan.c2r(Y.data_ptr(), y.data_ptr())
        assert rel_l2(y.cpu().numpy() / (n0 * n1 * n2), x32.astype(np.float64)) <= TOL_RT
    assert lib.fft3d_set_choices(plan.handle, [0, 0, 0, 2, 0]) == lib.FFT3D_ERR_INVALID_ARG


@pytest.mark.parametrize("shape", [(2048, 2, 6), (1536, 4, 12), (2, 2048, 32), (2, 2048, 30)],
                         ids=lambda s: "x".join(map(str, s)))
def test_long_axis_column_forms_match_oracle(cuda_lib, shape):
    """Every column-kernel form of the 1536- and 2048-long axes (the TMA ring,
    plain or row pairs; the plain kernel at full and half width) gives the
    oracle's transform, forward and back."""
    lib = cuda_lib
    n0, n1, n2 = shape
    plan = lib.Plan(n0, n1, n2)
    x32 = synth.uniform_field(shape, seed=57).astype(np.float32)
    ref = oracle.r2c3d(x32.astype(np.float64))
    xd = torch.from_numpy(x32).cuda()
    X = torch.empty((n0, n1, n2 // 2 + 1), dtype=torch.complex64, device="cuda")
    for choice in ([0, 0, 0, 1, 1], [4, 4, 0, 0, 0], [0, 0, 0, 0, 0]):
        assert lib.fft3d_set_choices(plan.handle, choice) == lib.FFT3D_OK
        plan.r2c(xd.data_ptr(), X.data_ptr())
        assert rel_l2(X.cpu().numpy(), ref) <= TOL, choice
        Y = X.clone()
        y = torch.empty_like(xd)
        plan.c2r(Y.data_ptr(), y.data_ptr())
        assert rel_l2(y.cpu().numpy() / (n0 * n1 * n2), x32.astype(np.float64)) <= TOL_RT, choice
    plan.close()


@pytest.mark.parametrize("shape,batch", [((2, 2048, 32), 1), ((2, 2048, 40), 1), ((3, 1024, 36), 2),
                                         ((2, 1024, 62), 1), ((4, 1024, 30), 1), ((3, 2048, 4), 1)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else f"b{v}")
def test_two_column_row_pair_form_matches_oracle(cuda_lib, shape, batch):
    """Column form 6 of the n1 pass (TMA row pairs, two columns per thread,
    16-byte exchange and even-row stores) gives the oracle's transform in
    both directions: odd H (row pairs) with a ragged last tile of one column,
    batches, and an even H, where the form falls back to the one-column TMA
    kernel."""
    lib = cuda_lib
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    lead = (batch,) if batch > 1 else ()
    x32 = synth.uniform_field(lead + shape, seed=71).astype(np.float32)
    ref = oracle.r2c3d(x32.astype(np.float64))
    Y64 = random_half_spectrum((batch * n0, n1, H), 73).reshape(lead + (n0, n1, H))
    yref = oracle.c2r3d(Y64.astype(np.complex128), n2)
    plan = lib.Plan(n0, n1, n2, lib.FFT3D_F32, batch, 0)
    assert lib.fft3d_set_choices(plan.handle, [0, 0, 0, 1, 6]) == lib.FFT3D_OK
    two = "2 cols/thread" in plan.describe()
    assert two == (H % 2 == 1 and H >= (4 if n1 == 2048 else 8)), plan.describe()
    xd = torch.from_numpy(x32).cuda()
    X = torch.empty(lead + (n0, n1, H), dtype=torch.complex64, device="cuda")
    plan.r2c(xd.data_ptr(), X.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(X.cpu().numpy(), ref) <= TOL
    Yd = torch.from_numpy(Y64).cuda()
    y = torch.empty_like(xd)
    plan.c2r(Yd.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(y.cpu().numpy(), yref) <= TOL
    assert lib.fft3d_query_device_status(plan.handle) == lib.FFT3D_OK
    plan.close()


@pytest.mark.parametrize("shape,batch", [((2048, 2, 6), 1), ((1024, 3, 10), 1), ((1536, 4, 12), 1),
                                         ((2, 2048, 32), 1), ((3, 1024, 30), 1), ((1024, 2, 8), 2),
                                         ((2048, 3, 4), 2), ((2048, 3, 10), 1), ((1024, 4, 12), 2),
                                         ((1536, 2, 30), 1), ((2, 2048, 30), 1), ((3, 1024, 36), 2),
                                         ((2, 2048, 40), 1)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else f"b{v}")
def test_cluster_split_column_forms_match_oracle(cuda_lib, shape, batch):
    """The cluster-split column kernels (forms 2 and 3 of the n0 and n1
    passes: the tile's rows split by residue over a 2- or 4-CTA cluster, the
    final radix-C step through distributed shared memory; form 4: the same
    split with 512-row TMA-fed sub-transforms on 2, 3 or 4 CTAs; form 5: the
    512-row residues of one CTA's tile, parked in L2 scratch, on the n1 axis
    with the odd-stride shift) give the
    oracle's transform in both directions: ragged column tiles, batches, the
    n1 axis, and the input-preserving inverse (its first pass writes
    elsewhere)."""
    lib = cuda_lib
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    lead = (batch,) if batch > 1 else ()
    x32 = synth.uniform_field(lead + shape, seed=61).astype(np.float32)
    ref = oracle.r2c3d(x32.astype(np.float64))
    Y64 = random_half_spectrum((batch * n0, n1, H), 63).reshape(lead + (n0, n1, H))
    yref = oracle.c2r3d(Y64.astype(np.complex128), n2)
    xd = torch.from_numpy(x32).cuda()
    tried = 0
    for flags in (0, lib.FFT3D_FLAG_PRESERVE_INPUT):
        plan = lib.Plan(n0, n1, n2, lib.FFT3D_F32, batch, flags)
        for f0 in (0, 2, 3, 4, 5):
            for f1 in (0, 2, 3, 4, 5):
                if f0 < 2 and f1 < 2:
                    continue
                if lib.fft3d_set_choices(plan.handle, [0, 0, 0, f0, f1]) != lib.FFT3D_OK:
                    continue  # no such form on this axis
                if "split" not in plan.describe():
                    continue  # form 4 on an axis whose stride it cannot take: the plain kernel runs
                tried += 1
                X = torch.empty(lead + (n0, n1, H), dtype=torch.complex64, device="cuda")
                plan.r2c(xd.data_ptr(), X.data_ptr())
                torch.cuda.synchronize()
                assert rel_l2(X.cpu().numpy(), ref) <= TOL, (f0, f1, flags)
                Yd = torch.from_numpy(Y64).cuda()
                y = torch.empty_like(xd)
                plan.c2r(Yd.data_ptr(), y.data_ptr())
                torch.cuda.synchronize()
                assert rel_l2(y.cpu().numpy(), yref) <= TOL, (f0, f1, flags)
                if flags:
                    assert np.array_equal(Yd.cpu().numpy(), Y64)  # the input survived
        plan.close()
    assert tried >= 2


# ---------------------------------------------------------------------------
# FP64 path (FFT3D_F64): every pass on the FP64 runtime-length kernels.
# ---------------------------------------------------------------------------
TOL_F64 = 1e-12

F64_SHAPES = [((32, 32, 32), 1), ((48, 80, 96), 1), ((6, 10, 15), 1), ((11, 13, 22), 1), ((3, 97, 8), 1),
              ((14, 7, 9), 2), ((64, 64, 64), 2), ((2, 2, 4094), 1), ((4096, 2, 2), 1), ((2, 2, 8192), 1)]


@pytest.mark.parametrize("shape,batch", F64_SHAPES, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else f"b{v}")
def test_fp64_path_matches_oracle(cuda_lib, shape, batch):
    """FFT3D_F64: r2c against the FP64 oracle, c2r of an arbitrary half
    spectrum against the oracle's c2r, and the round trip, at 1e-12 (the FP32
    path stays near 1e-7): direct and Bluestein lengths (11, 13, 97, 2047 =
    23 x 89), odd n2, batch, the longest lines (4096 points; a Bluestein line
    of 4096)."""
    lib = cuda_lib
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    plan = lib.Plan(n0, n1, n2, dtype=lib.FFT3D_F64, batch=batch)
    assert plan.describe().split()[2] == "fp64"
    x = synth.uniform_field((batch, n0, n1, n2), seed=83)
    xd = torch.from_numpy(x).cuda()
    X = torch.empty((batch, n0, n1, H), dtype=torch.complex128, device="cuda")
    plan.r2c(xd.data_ptr(), X.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(X.cpu().numpy(), oracle.r2c3d(x)) <= TOL_F64
    y = torch.empty_like(xd)
    plan.c2r(X.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(y.cpu().numpy() / (n0 * n1 * n2), x) <= TOL_F64
    Y = random_half_spectrum((batch * n0, n1, H), seed=84).astype(np.complex128).reshape(batch, n0, n1, H)
    Yd = torch.from_numpy(Y).cuda()
    plan.c2r(Yd.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(y.cpu().numpy(), oracle.c2r3d(Y, n2)) <= TOL_F64
    plan.close()


def test_fp64_entry_points_and_helpers(cuda_lib):
    """FP64 plans go through fft3d_r2c_f64 / fft3d_c2r_f64 only (and FP32
    plans never do); the forms built on FP32 spectra reject FP64 plans; rfft3
    / irfft3 pick the FP64 path for float64 / complex128 tensors."""
    lib = cuda_lib
    p64 = lib.Plan(8, 8, 8, dtype=lib.FFT3D_F64)
    p32 = lib.Plan(8, 8, 8)
    a = torch.zeros(8 * 8 * 8 * 2, dtype=torch.float64, device="cuda")
    b = torch.zeros(8 * 8 * 5 * 2, dtype=torch.float64, device="cuda")
    assert lib.fft3d_r2c(p64.handle, a.data_ptr(), b.data_ptr(), 0) == lib.FFT3D_ERR_INVALID_ARG
    assert lib.fft3d_c2r(p64.handle, b.data_ptr(), a.data_ptr(), 0) == lib.FFT3D_ERR_INVALID_ARG
    assert lib.fft3d_r2c_f64(p32.handle, a.data_ptr(), b.data_ptr(), 0) == lib.FFT3D_ERR_INVALID_ARG
    assert lib.fft3d_c2r_f64(p32.handle, b.data_ptr(), a.data_ptr(), 0) == lib.FFT3D_ERR_INVALID_ARG
    assert lib.fft3d_r2c_f64(p64.handle, a.data_ptr(), a.data_ptr() + 64, 0) == lib.FFT3D_ERR_INVALID_ARG
    with pytest.raises(lib.Fft3dError):
        p64.energy(torch.zeros((8, 8, 5), dtype=torch.complex64, device="cuda"), 4)
    assert lib.fft3d_autotune(p64.handle, a.data_ptr(), b.data_ptr(), 1) == lib.FFT3D_ERR_INVALID_ARG
    p64.close()
    p32.close()
    x = torch.from_numpy(synth.uniform_field((2, 12, 10, 14), seed=85)).cuda()
    X = lib.rfft3(x)
    assert X.dtype == torch.complex128
    assert rel_l2(X.cpu().numpy(), oracle.r2c3d(x.cpu().numpy())) <= TOL_F64
    y = lib.irfft3(X, 14)
    assert y.dtype == torch.float64
    assert rel_l2(y.cpu().numpy() / (12 * 10 * 14), x.cpu().numpy()) <= TOL_F64


def test_tuned_plan_uses_the_cache(cuda_lib, tmp_path):
    from paper_1406_5597_gb300 import tune
    path = str(tmp_path / "wisdom.json")
    p1, tuned = tune.tuned_plan(64, 48, 40, path=path, reps=1)
    assert tuned
    p2, tuned2 = tune.tuned_plan(64, 48, 40, path=path, reps=1)
    assert not tuned2
    assert cuda_lib.fft3d_get_choices(p1.handle) == cuda_lib.fft3d_get_choices(p2.handle)


# ---------------------------------------------------------------------------
# FP64 device diagnostics: Parseval sum and shell energies vs the oracle.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,batch", [((32, 32, 32), 1), ((24, 40, 36), 2), ((15, 12, 10), 1), ((64, 48, 40), 1)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_energy_matches_oracle(cuda_lib, shape, batch):
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    Y = random_half_spectrum((batch * n0, n1, H), seed=71).reshape(batch, n0, n1, H)
    plan = cuda_lib.Plan(n0, n1, n2, batch=batch)
    nbins = 40
    total, shells = plan.energy(torch.from_numpy(Y).cuda(), nbins)
    torch.cuda.synchronize()
    total = total.cpu().numpy()
    shells = shells.cpu().numpy()
    for b in range(batch):
        Yb = Y[b].astype(np.complex128)
        # |X|^2 is formed in FP32 on the device: relative error ~1e-7 per term
        assert abs(total[b] - oracle.half_energy(Yb, n2)) <= 1e-6 * oracle.half_energy(Yb, n2)
        ref = oracle.shell_energy(Yb, n0, n1, n2, nbins)
        assert np.all(np.abs(shells[b] - ref) <= 1e-6 * np.maximum(ref, 1e-30) + 1e-12)
        # every bin of shell < nbins is counted once
        assert abs(shells[b].sum() - ref.sum()) <= 1e-6 * ref.sum()


def test_energy_parseval_of_r2c(cuda_lib):
    n = 64
    x32 = synth.uniform_field((n, n, n), seed=73).astype(np.float32)
    plan = cuda_lib.Plan(n, n, n)
    xd = torch.from_numpy(x32).cuda()
    X = torch.empty((n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    plan.r2c(xd.data_ptr(), X.data_ptr(), torch.cuda.current_stream().cuda_stream)
    total, _ = plan.energy(X, 8)
    e = total.cpu().item() / n ** 3
    assert abs(e - np.sum(x32.astype(np.float64) ** 2)) <= 1e-5 * e


# ---------------------------------------------------------------------------
# Full size of the benchmark workload: 512^3 spectrum-shaped field (seed 1408).
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def field512():
    n = 512
    S = synth.spectral_velocity(n, n, n, seed=synth.seed_for_config(2), components=(0,))[0]
    x = oracle.c2r3d(S, n)
    return S, x


@pytest.mark.parametrize("dtype", [1, 2], ids=["bf16x3", "fp16"])
def test_512_tensor_core_forms(cuda_lib, field512, dtype):
    S, x = field512
    n = 512
    X, desc = gpu_r2c_dtype(cuda_lib, x.astype(np.float32), dtype)
    assert "tensor-core" in desc
    assert rel_l2(X, n ** 3 * S) <= TC_TOL[dtype]


@pytest.mark.parametrize("flags", [0, 1, 3], ids=["transpose-free", "explicit-transpose", "transpose-back"])
def test_512_spectrum_as_oracle_and_spot_bins(cuda_lib, field512, flags):
    """x = c2r(S) exactly (FP64), so r2c(x) = N S up to the FP32 rounding of x
    (~3e-8 relative): a full-size reference that needs no 512^3 forward oracle.
    Plus exact FP64 spot bins of the same FP32 input."""
    S, x = field512
    n = 512
    N = n ** 3
    x32 = x.astype(np.float32)
    X = gpu_r2c(cuda_lib, x32, flags=flags)
    if flags == 1:
        X = X.transpose(1, 0, 2)
    assert rel_l2(X, N * S) <= TOL
    rng = np.random.default_rng(5)
    ks = np.stack([rng.integers(0, n, 12), rng.integers(0, n, 12), rng.integers(0, n // 2 + 1, 12)], 1)
    ks = np.concatenate([ks, [[0, 0, 0], [4, 3, 0], [511, 1, 256], [1, 2, 3]]])
    ref = oracle.r2c_bins_f32(x32, ks)
    got = np.array([X[tuple(k)] for k in ks])
    # per-bin bound of the FP32 error model (tests/errmodel.py): the spread
    # part scales with the field's rms, the line part with the axis lines
    # through the bin, the local part with the bin
    rms = np.sqrt(np.mean(np.abs(X) ** 2))
    lines = line_rms(X, ks)
    assert np.all(np.abs(got - ref) <= spot_bound(ref, rms, 0, lines, n)), spot_report(got, ref, rms, 0, lines, n)


def test_512_inverse(cuda_lib, field512):
    S, x = field512
    n = 512
    N = n ** 3
    Y = (N * S).astype(np.complex64)
    y = gpu_c2r(cuda_lib, Y, n)
    assert rel_l2(y, N * x) <= TOL
    rng = np.random.default_rng(6)
    js = np.stack([rng.integers(0, n, 8), rng.integers(0, n, 8), rng.integers(0, n, 8)], 1)
    ref = oracle.c2r_points_c64(Y, n, js)
    got = np.array([y[tuple(j)] for j in js])
    rms = np.sqrt(np.mean(y ** 2))
    lines = line_rms(y, js)
    assert np.all(np.abs(got - ref) <= spot_bound(ref, rms, 0, lines, n)), spot_report(got, ref, rms, 0, lines, n)

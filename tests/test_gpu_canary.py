"""Out-of-bounds writes, without a sanitizer: every operand (input, output,
workspace) lies between guard margins filled with a canary word in one
allocation, every kernel family and form runs on it, and afterwards every
margin word must still hold the canary, and every read-only input must be bit
for bit unchanged.  The cases cover the specialised kernels (warp and
shared-memory rows, TMA and plain columns with ragged tiles), the runtime-radix
and Bluestein kernels, odd n2, the padded and input-preserving layouts, the
explicit-transpose comparator, the plane forms, the tensor-core forms and the
FP64 path.  Also the planner's environment switches (FFT3D_LOG,
FFT3D_FORCE_PASSES), in child processes.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import synth

CANARY = 0x7FC00BAD  # as a float: a NaN pattern that no transform writes
MARGIN = 64 * 1024   # bytes on each side of every operand
ALIGN = 256


class Arena:
    """One int32 CUDA allocation: [margin | operand | margin | operand | ... | margin]."""

    def __init__(self, sizes, device="cuda"):
        self.offsets = []
        off = MARGIN
        for n in sizes:
            self.offsets.append(off)
            off += -(-n // ALIGN) * ALIGN + MARGIN
        self.sizes = list(sizes)
        self.buf = torch.full((off // 4,), CANARY, dtype=torch.int32, device=device)
        assert device != "cuda" or self.buf.data_ptr() % ALIGN == 0

    def ptr(self, i):
        return self.buf.data_ptr() + self.offsets[i]

    def view(self, i, dtype, shape):
        n = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        assert n <= self.sizes[i]
        return self.buf[self.offsets[i] // 4: (self.offsets[i] + n) // 4].view(dtype).view(shape)

    def margins_intact(self):
        b = self.buf.cpu().numpy()
        mask = np.ones(b.shape, dtype=bool)
        for off, n in zip(self.offsets, self.sizes):
            mask[off // 4: (off + n + 3) // 4] = False
        bad = np.flatnonzero(mask & (b != CANARY))
        return bad.size == 0, bad[:8]


def test_arena_detects_a_write_next_to_an_operand():
    """The check itself: a write one word past an operand, or in the first
    margin, is found; writes inside the operands are not reported."""
    a = Arena([100, 4096], device="cpu")
    a.view(0, torch.float32, (25,)).fill_(1.0)
    a.view(1, torch.float64, (512,)).fill_(2.0)
    assert a.margins_intact()[0]
    a.buf[(a.offsets[1] + 4096) // 4] = 0
    ok, bad = a.margins_intact()
    assert not ok and bad.tolist() == [(a.offsets[1] + 4096) // 4]
    b = Arena([64], device="cpu")
    b.buf[0] = 1
    assert not b.margins_intact()[0]


CASES = [
    # (shape, batch, dtype name, flags name)
    ((64, 64, 64), 1, "f32", "none"),
    ((512, 6, 10), 1, "f32", "none"),          # TMA n0 pass, ragged tile
    ((6, 512, 60), 2, "f32", "none"),          # TMA row pairs, odd H
    ((48, 80, 96), 1, "f32", "none"),          # radix 3 / 5 kernels
    ((8, 6, 1024), 1, "f32", "none"),          # warp rows at n2 = 1024
    ((3, 2, 2048), 1, "f32", "none"),          # shared-memory rows
    ((2, 2048, 32), 1, "f32", "none"),         # 4-wide TMA row pairs at n1 = 2048
    ((6, 10, 15), 2, "f32", "none"),           # odd n2, runtime radices
    ((11, 13, 22), 1, "f32", "none"),          # Bluestein on every axis
    ((14, 7, 9), 1, "f32", "none"),            # radix 7, odd n2
    ((32, 48, 40), 1, "f32", "padded"),
    ((64, 64, 64), 1, "f32", "preserve"),
    ((32, 32, 32), 1, "f32", "transpose"),
    ((32, 32, 32), 1, "f32", "transpose_back"),
    ((64, 64, 64), 1, "f32", "cluster"),
    ((128, 128, 128), 1, "f32", "fused"),
    ((64, 64, 64), 1, "f32", "generic"),
    ((256, 24, 20), 1, "bf16x3", "none"),
    ((11, 13, 22), 2, "f64", "none"),
    ((48, 80, 96), 1, "f64", "none"),
    ((2048, 3, 4), 2, "f32", "split0"),         # cluster-split n0 pass, 2 CTAs, ragged tile
    ((2048, 3, 4), 1, "f32", "split1"),         # 4 CTAs per cluster
    ((1024, 3, 10), 1, "f32", "split1"),
    ((1536, 4, 12), 1, "f32", "split0"),
    ((2, 2048, 32), 1, "f32", "split0_n1"),     # the n1 pass, odd H
    ((2048, 3, 10), 2, "f32", "tsplit"),        # TMA-fed cluster split, 4 CTAs, ragged tile, batch
    ((1536, 2, 30), 1, "f32", "tsplit"),        # 3 CTAs
    ((1024, 4, 12), 1, "f32", "tsplit"),        # 2 CTAs
    ((2, 2048, 30), 1, "f32", "tsplit_n1"),     # the n1 pass (even H)
    ((2048, 3, 10), 2, "f32", "l2split"),       # residue split through L2 scratch, C = 4, ragged, batch
    ((1536, 2, 30), 1, "f32", "l2split"),       # C = 3
    ((1024, 4, 12), 1, "f32", "l2split"),       # C = 2
    ((2, 2048, 40), 1, "f32", "l2split_n1"),    # the n1 pass, odd H: odd residues' boxes shifted, C = 4
    ((3, 1024, 36), 2, "f32", "l2split_n1"),    # the n1 pass, odd H, C = 2, batch
    ((2, 2048, 30), 1, "f32", "l2split_n1"),    # the n1 pass, even H
]


# column-form choices {w0, w1, rows, form0, form1} of the split cases
SPLIT_CHOICES = {"split0": [0, 0, 0, 2, 0], "split1": [0, 0, 0, 3, 0], "split0_n1": [0, 0, 0, 0, 2],
                 "tsplit": [0, 0, 0, 4, 0], "tsplit_n1": [0, 0, 0, 0, 4], "l2split": [0, 0, 0, 5, 0],
                 "l2split_n1": [0, 0, 0, 0, 5]}


def _flags(lib, name):
    if name in SPLIT_CHOICES:
        return 0
    return {"none": 0, "padded": lib.FFT3D_FLAG_PADDED_REAL, "preserve": lib.FFT3D_FLAG_PRESERVE_INPUT,
            "transpose": lib.FFT3D_FLAG_EXPLICIT_TRANSPOSE,
            "transpose_back": lib.FFT3D_FLAG_EXPLICIT_TRANSPOSE | lib.FFT3D_FLAG_TRANSPOSE_BACK,
            "cluster": lib.FFT3D_FLAG_CLUSTER_PLANE, "fused": lib.FFT3D_FLAG_FUSED_PLANE,
            "generic": lib.FFT3D_FLAG_GENERIC}[name]


@pytest.mark.gpu
@pytest.mark.parametrize("shape,batch,dt,fl", CASES,
                         ids=["x".join(map(str, c[0])) + f"-b{c[1]}-{c[2]}-{c[3]}" for c in CASES])
def test_no_write_outside_the_operands(cuda_lib, shape, batch, dt, fl):
    lib = cuda_lib
    n0, n1, n2 = shape
    H = n2 // 2 + 1
    f64 = dt == "f64"
    dtype = {"f32": lib.FFT3D_F32, "bf16x3": lib.FFT3D_F32_TC_BF16X3, "f64": lib.FFT3D_F64}[dt]
    flags = _flags(lib, fl)
    plan = lib.Plan(n0, n1, n2, dtype=dtype, batch=batch, flags=flags)
    if fl in SPLIT_CHOICES:
        assert lib.fft3d_set_choices(plan.handle, SPLIT_CHOICES[fl]) == lib.FFT3D_OK
        assert "split" in plan.describe()
    rt = torch.float64 if f64 else torch.float32
    ct = torch.complex128 if f64 else torch.complex64
    row = 2 * H if fl == "padded" else n2
    real_shape = (batch, n0, n1, row)
    cplx_shape = (batch, n0, n1, H)
    esz = 8 if f64 else 4
    ws = lib.fft3d_workspace_bytes(plan.handle)
    sizes = [batch * n0 * n1 * row * esz, batch * n0 * n1 * H * 2 * esz, batch * n0 * n1 * row * esz]
    if ws:
        sizes.append(ws)
    arena = Arena(sizes)
    if ws:
        assert lib.fft3d_set_workspace(plan.handle, arena.ptr(3)) == lib.FFT3D_OK
    x = torch.from_numpy(synth.uniform_field((batch, n0, n1, n2), seed=97)).to(rt).cuda()
    xin = arena.view(0, rt, real_shape)
    if fl == "padded":
        xin.zero_()
    xin[..., :n2] = x
    x_before = xin.clone()
    s = torch.cuda.current_stream().cuda_stream
    plan.r2c(arena.ptr(0), arena.ptr(1), s)
    torch.cuda.synchronize()
    assert torch.equal(xin, x_before), "r2c wrote its input"
    X_before = arena.view(1, ct, cplx_shape).clone()
    plan.c2r(arena.ptr(1), arena.ptr(2), s)
    torch.cuda.synchronize()
    if fl == "preserve":
        assert torch.equal(arena.view(1, ct, cplx_shape), X_before), "the preserving c2r wrote its input"
    y = arena.view(2, rt, real_shape)[..., :n2].double().cpu().numpy() / (n0 * n1 * n2)
    err = np.linalg.norm(y - x.double().cpu().numpy()) / np.linalg.norm(x.double().cpu().numpy())
    assert err < (1e-12 if f64 else 2e-5), err
    ok, bad = arena.margins_intact()
    assert ok, f"canary overwritten at int32 words {bad.tolist()}"
    plan.close()


def _child(code, env):
    e = dict(os.environ)
    e.update(env)
    r = subprocess.run([sys.executable, "-c", code], env=e, capture_output=True, text=True, timeout=300,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stderr[-2000:]
    return r


@pytest.mark.gpu
def test_planner_environment_switches():
    """FFT3D_LOG=1 reports plan decisions on stderr; FFT3D_FORCE_PASSES ORs
    forms into every FP32 plan (not into FP64 plans, which take no flags)."""
    code = ("import paper_1406_5597_gb300 as f; "
            "p = f.Plan(64, 64, 64); print(p.describe()); "
            "q = f.Plan(16, 16, 16, dtype=f.FFT3D_F64); print(q.describe())")
    r = _child(code, {"FFT3D_LOG": "1", "FFT3D_FORCE_PASSES": "generic,three"})
    lines = r.stdout.strip().splitlines()
    assert "generic L=32" in lines[0] and "generic L=64" in lines[0]
    assert "fp64" in lines[1]
    assert "fft3d: plan 64x64x64 batch=1 dtype=0" in r.stderr
    r = _child(code, {"FFT3D_FORCE_PASSES": "transpose"})
    assert r.stdout.strip().splitlines()[0].endswith("explicit-transpose")
    assert "fft3d:" not in r.stderr
    r = _child(code, {})
    assert "generic" not in r.stdout.splitlines()[0]

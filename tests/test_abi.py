"""The C-ABI library builds for sm_103a, loads, and exports every function
include/fft3d.h declares; host-side argument checks answer without a GPU."""
import ctypes
import os

import pytest

import paper_1406_5597_gb300 as fft3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fft3d.build()
    return fft3d.load()


def test_exports_every_declared_function(lib):
    names = fft3d.declared_functions()
    assert "fft3d_plan" in names and "fft3d_r2c" in names and "fft3d_c2r" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in fft3d._SIGS, n


def test_error_strings(lib):
    for st in range(0, 8):
        assert fft3d.fft3d_error_string(st)
    assert "unknown" in fft3d.fft3d_error_string(99)


@pytest.mark.parametrize("dims,status", [
    ((0, 8, 8), fft3d.FFT3D_ERR_INVALID_ARG),
    ((8, 8, 1), fft3d.FFT3D_ERR_INVALID_ARG),
    ((8, 8, 8193), fft3d.FFT3D_ERR_UNSUPPORTED_SIZE),  # odd row longer than 4096
    ((4097, 8, 8), fft3d.FFT3D_ERR_UNSUPPORTED_SIZE),  # prime axis beyond 4096
    ((8, 8, 8194), fft3d.FFT3D_ERR_UNSUPPORTED_SIZE),  # n2/2 = 4097
    ((8192, 8, 8), fft3d.FFT3D_ERR_UNSUPPORTED_SIZE),
])
def test_plan_rejects_bad_sizes_before_touching_the_device(lib, dims, status):
    assert not fft3d.fft3d_plan(*dims, fft3d.FFT3D_F32, 1)
    assert fft3d.fft3d_last_error() == status


def test_plan_rejects_bad_dtype_batch_flags(lib):
    assert not fft3d.fft3d_plan(8, 8, 8, 4, 1)
    assert fft3d.fft3d_last_error() == fft3d.FFT3D_ERR_INVALID_ARG
    # FP64 plans take no flags, and no Bluestein length above 2048
    assert not fft3d.fft3d_plan_variant(8, 8, 8, fft3d.FFT3D_F64, 1, fft3d.FFT3D_FLAG_PADDED_REAL)
    assert fft3d.fft3d_last_error() == fft3d.FFT3D_ERR_INVALID_ARG
    assert not fft3d.fft3d_plan(2053, 8, 8, fft3d.FFT3D_F64, 1)
    assert fft3d.fft3d_last_error() == fft3d.FFT3D_ERR_UNSUPPORTED_SIZE
    assert not fft3d.fft3d_plan(8, 8, 8, 7, 1)
    assert fft3d.fft3d_last_error() == fft3d.FFT3D_ERR_INVALID_ARG
    assert not fft3d.fft3d_plan(8, 8, 8, 0, 0)
    assert fft3d.fft3d_last_error() == fft3d.FFT3D_ERR_INVALID_ARG
    assert not fft3d.fft3d_plan_variant(8, 8, 8, 0, 1, fft3d.FFT3D_FLAG_TRANSPOSE_BACK)
    assert fft3d.fft3d_last_error() == fft3d.FFT3D_ERR_INVALID_ARG
    assert not fft3d.fft3d_plan_variant(8, 8, 8, 0, 1, 0x100)


def test_nonlinear_plan_rejects_bad_sizes(lib):
    assert not fft3d.fft3d_nonlinear_plan(8, 8, 8194)
    assert fft3d.fft3d_last_error() == fft3d.FFT3D_ERR_UNSUPPORTED_SIZE
    assert fft3d.fft3d_nonlinear_exec(None, 16, 32) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_nonlinear_workspace_bytes(None) == 0
    fft3d.fft3d_nonlinear_destroy(None)


def test_null_handles(lib):
    assert fft3d.fft3d_r2c(None, 16, 32) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_c2r(None, 16, 32) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_r2c_f64(None, 16, 32) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_c2r_f64(None, 16, 32) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_workspace_bytes(None) == 0
    assert fft3d.fft3d_set_workspace(None, 0) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_launches_per_call(None) == fft3d.FFT3D_ERR_INVALID_ARG
    fft3d.fft3d_destroy(None)
    assert fft3d.fft3d_set_plane_choice(None, 2) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_ns_step(None, 16, 0.01, 0.1) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_ns_workspace_bytes(None) == 0
    assert fft3d.fft3d_ns_launches(None) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_ns_set_chunking(None, 8, 2) == fft3d.FFT3D_ERR_INVALID_ARG
    fft3d.fft3d_ns_destroy(None)
    assert fft3d.fft3d_nonlinear_launches(None) == fft3d.FFT3D_ERR_INVALID_ARG
    assert fft3d.fft3d_nonlinear_set_chunking(None, 8, 1) == fft3d.FFT3D_ERR_INVALID_ARG
    with pytest.raises(fft3d.Fft3dError):
        fft3d.fft3d_nonlinear_get_chunking(None)
    with pytest.raises(fft3d.Fft3dError):
        fft3d.fft3d_get_plane_choice(None)
    buf = ctypes.create_string_buffer(8)
    assert lib.fft3d_describe(None, buf, 8) == fft3d.FFT3D_ERR_INVALID_ARG


def test_binding_signatures_match_the_header():
    """Every prototype in include/fft3d.h has a binding entry with the same
    number of arguments and a matching return kind (void / int / size_t /
    pointer), so no argument is marshalled into the wrong slot."""
    import ctypes
    import re
    src = open(os.path.join(ROOT, "include", "fft3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = re.findall(r"([A-Za-z_][\w\s\*]*?)\b(fft3d_\w+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S)
    assert len(protos) >= 40
    for ret, name, params in protos:
        p = " ".join(params.split())
        nargs = 0 if p in ("", "void") else len(p.split(","))
        assert name in fft3d._SIGS, name
        argtypes, restype = fft3d._SIGS[name]
        assert len(argtypes) == nargs, (name, nargs, len(argtypes))
        ret = " ".join(ret.split())
        if ret == "void":
            assert restype is None, name
        elif ret == "int":
            assert restype is ctypes.c_int, name
        elif ret == "size_t":
            assert restype is ctypes.c_size_t, name
        elif ret == "double":
            assert restype is ctypes.c_double, name
        else:  # a handle or a string
            assert restype in (ctypes.c_void_p, ctypes.c_char_p), (name, ret)


def test_binding_objects_close_on_leaving_a_with_block():
    """Plan, Group, NonlinearTerm and NavierStokes release their handle at the
    end of a with-block; close() is idempotent (checked on handle-less objects,
    which needs no GPU)."""
    for cls in (fft3d.Plan, fft3d.Group, fft3d.NonlinearTerm, fft3d.NavierStokes):
        obj = object.__new__(cls)
        obj.handle = None
        with obj as o:
            assert o is obj
        obj.close()
        assert obj.handle is None


def _cuda_device_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_cuda_device_present(),
                    reason="host buffers stand in for device ones here; only run where nothing can launch")
def test_noalloc_energy_rejects_calls_beyond_its_scratch(lib):
    """fft3d_energy_noalloc checks the scratch a call needs against its fixed
    2^18-double array before anything touches the device: 8 x 8 x 2 with
    batch 4 and 8192 shells needs 4 * 8 * 8193 = 262176 doubles, 32 over.
    The buffers are sized for the whole call, and on a machine without a GPU
    a missing check could only fail (no device to launch on), never write."""
    import numpy as np
    spec = np.zeros(4 * 8 * 8 * 2 * 2 + 4, dtype=np.float32)
    total = np.full(4, 7.0)
    shells = np.full(4 * 8192, 7.0)
    sp = spec.ctypes.data + (-spec.ctypes.data) % 16  # 16-byte aligned start
    st = fft3d.fft3d_energy_noalloc(sp, 8, 8, 2, 4, total.ctypes.data, shells.ctypes.data, 8192, 0)
    assert st == fft3d.FFT3D_ERR_UNSUPPORTED_SIZE
    assert np.all(total == 7.0) and np.all(shells == 7.0)
    # one entry less fits (3 * 8 * 8193 doubles): it passes the size check and
    # fails only on the missing device
    st = fft3d.fft3d_energy_noalloc(sp, 8, 8, 2, 3, total.ctypes.data, shells.ctypes.data, 8192, 0)
    assert st == fft3d.FFT3D_ERR_CUDA
    assert np.all(total == 7.0) and np.all(shells == 7.0)

"""Python binding of libfft3d (transpose-free 3D r2c / c2r FFT on one GB300).

Argument marshalling only: every step of a transform runs in the library's
CUDA kernels.  The C functions keep their names (``fft3d_plan``,
``fft3d_r2c``, ``fft3d_c2r``, ``fft3d_destroy``, ...); data arguments are
device addresses (ints) and ``stream`` is a ``cudaStream_t`` address (0 for
the legacy default stream).  ``rfft3`` / ``irfft3`` wrap them for torch CUDA
tensors, which only provide the device memory and the stream.

There is no CPU path: if ``libfft3d.so`` is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfft3d.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "fft3d.h")

FFT3D_F32 = 0
FFT3D_F32_TC_BF16X3 = 1
FFT3D_F32_TC_F16 = 2
FFT3D_F64 = 3

FFT3D_OK = 0
FFT3D_ERR_INVALID_ARG = 1
FFT3D_ERR_UNSUPPORTED_SIZE = 2
FFT3D_ERR_MISALIGNED = 3
FFT3D_ERR_ALLOC = 4
FFT3D_ERR_CUDA = 5
FFT3D_ERR_TIMEOUT = 6
FFT3D_ERR_NO_WORKSPACE = 7

FFT3D_FLAG_EXPLICIT_TRANSPOSE = 0x1
FFT3D_FLAG_TRANSPOSE_BACK = 0x2
FFT3D_FLAG_THREE_PASS = 0x4
FFT3D_FLAG_GENERIC = 0x8
FFT3D_FLAG_TEST_SKIP_ARRIVAL = 0x10
FFT3D_FLAG_FUSED_PLANE = 0x20
FFT3D_FLAG_CLUSTER_PLANE = 0x40
FFT3D_FLAG_PADDED_REAL = 0x80
FFT3D_FLAG_PRESERVE_INPUT = 0x100

FFT3D_GROUP_STREAMS = 0
FFT3D_GROUP_WORK_TABLE = 1
FFT3D_GROUP_WORK_TABLE_TEST_STALL = 2

_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "fft3d_plan": ([_I, _I, _I, _I, _I], _P),
    "fft3d_plan_variant": ([_I, _I, _I, _I, _I, _I], _P),
    "fft3d_r2c": ([_P, _P, _P, _P], _I),
    "fft3d_c2r": ([_P, _P, _P, _P], _I),
    "fft3d_r2c_f64": ([_P, _P, _P, _P], _I),
    "fft3d_c2r_f64": ([_P, _P, _P, _P], _I),
    "fft3d_destroy": ([_P], None),
    "fft3d_last_error": ([], _I),
    "fft3d_error_string": ([_I], ctypes.c_char_p),
    "fft3d_query_device_status": ([_P, _P], _I),
    "fft3d_workspace_bytes": ([_P], ctypes.c_size_t),
    "fft3d_set_workspace": ([_P, _P], _I),
    "fft3d_describe": ([_P, ctypes.c_char_p, _I], _I),
    "fft3d_launches_per_call": ([_P, _I], _I),
    "fft3d_set_profiling": ([_P, _I], _I),
    "fft3d_profile_read": ([_P, _P, _P, _I], _I),
    "fft3d_pass_name": ([_I], ctypes.c_char_p),
    "fft3d_pass_bytes": ([_P, _I], ctypes.c_double),
    "fft3d_energy": ([_P, _P, _P, _P, _I, _P], _I),
    "fft3d_energy_noalloc": ([_P, _I, _I, _I, _I, _P, _P, _I, _P], _I),
    "fft3d_nonlinear_plan": ([_I, _I, _I], _P),
    "fft3d_nonlinear_workspace_bytes": ([_P], ctypes.c_size_t),
    "fft3d_nonlinear_set_workspace": ([_P, _P], _I),
    "fft3d_nonlinear_exec": ([_P, _P, _P, _P], _I),
    "fft3d_nonlinear_launches": ([_P], _I),
    "fft3d_nonlinear_set_chunking": ([_P, _I, _I], _I),
    "fft3d_nonlinear_get_chunking": ([_P, _P, _P], _I),
    "fft3d_nonlinear_destroy": ([_P], None),
    "fft3d_ns_plan": ([_I, _I, _I], _P),
    "fft3d_ns_workspace_bytes": ([_P], ctypes.c_size_t),
    "fft3d_ns_set_workspace": ([_P, _P], _I),
    "fft3d_ns_step": ([_P, _P, ctypes.c_float, ctypes.c_float, _P], _I),
    "fft3d_ns_launches": ([_P], _I),
    "fft3d_ns_set_chunking": ([_P, _I, _I], _I),
    "fft3d_ns_destroy": ([_P], None),
    "fft3d_autotune": ([_P, _P, _P, _I, _P], _I),
    "fft3d_get_choices": ([_P, _P], _I),
    "fft3d_set_choices": ([_P, _P], _I),
    "fft3d_get_plane_choice": ([_P], _I),
    "fft3d_set_plane_choice": ([_P, _I], _I),
    "fft3d_plan_group": ([_P, _P, _I, _I], _P),
    "fft3d_group_plan_at": ([_P, _I], _P),
    "fft3d_group_r2c": ([_P, _P, _P, _P], _I),
    "fft3d_group_c2r": ([_P, _P, _P, _P], _I),
    "fft3d_group_r2c_c2r": ([_P, _P, _P, _P, _P], _I),
    "fft3d_group_launches": ([_P, _I], _I),
    "fft3d_group_set_form": ([_P, _I], _I),
    "fft3d_group_get_form": ([_P], _I),
    "fft3d_group_query_device_status": ([_P, _P], _I),
    "fft3d_group_destroy": ([_P], None),
}


class Fft3dError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {error_string(status)} (status {status})")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library in-tree (see native_build.py)."""
    from . import native_build
    return native_build.build(force=force, verbose=verbose)


def declared_functions() -> list[str]:
    """Names of the functions include/fft3d.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fft3d_[a-z0-9_]+)\s*\(", text)))


def load():
    """Load libfft3d.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1406_5597_gb300.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _v(x):
    return None if x is None or x == 0 else ctypes.c_void_p(int(x))


# --- the C functions, same names ------------------------------------------------

def fft3d_plan(n0, n1, n2, dtype=FFT3D_F32, batch=1):
    return load().fft3d_plan(n0, n1, n2, dtype, batch)


def fft3d_plan_variant(n0, n1, n2, dtype=FFT3D_F32, batch=1, flags=0):
    return load().fft3d_plan_variant(n0, n1, n2, dtype, batch, flags)


def fft3d_r2c(plan, in_ptr, out_ptr, stream=0):
    return load().fft3d_r2c(_v(plan), _v(in_ptr), _v(out_ptr), _v(stream))


def fft3d_c2r(plan, in_ptr, out_ptr, stream=0):
    return load().fft3d_c2r(_v(plan), _v(in_ptr), _v(out_ptr), _v(stream))


def fft3d_r2c_f64(plan, in_ptr, out_ptr, stream=0):
    return load().fft3d_r2c_f64(_v(plan), _v(in_ptr), _v(out_ptr), _v(stream))


def fft3d_c2r_f64(plan, in_ptr, out_ptr, stream=0):
    return load().fft3d_c2r_f64(_v(plan), _v(in_ptr), _v(out_ptr), _v(stream))


def fft3d_destroy(plan):
    load().fft3d_destroy(_v(plan))


def fft3d_last_error():
    return load().fft3d_last_error()


def fft3d_error_string(status):
    return load().fft3d_error_string(status).decode()


def fft3d_query_device_status(plan, stream=0):
    return load().fft3d_query_device_status(_v(plan), _v(stream))


def fft3d_workspace_bytes(plan):
    return load().fft3d_workspace_bytes(_v(plan))


def fft3d_set_workspace(plan, dev_ptr):
    return load().fft3d_set_workspace(_v(plan), _v(dev_ptr))


def fft3d_describe(plan):
    buf = ctypes.create_string_buffer(512)
    st = load().fft3d_describe(_v(plan), buf, 512)
    if st != FFT3D_OK:
        raise Fft3dError(st, "fft3d_describe")
    return buf.value.decode()


def fft3d_launches_per_call(plan, direction=-1):
    return load().fft3d_launches_per_call(_v(plan), direction)


def fft3d_set_profiling(plan, enable=True):
    return load().fft3d_set_profiling(_v(plan), 1 if enable else 0)


def fft3d_pass_name(pass_id):
    r = load().fft3d_pass_name(pass_id)
    return r.decode() if r else None


def pass_names():
    names = []
    while True:
        n = fft3d_pass_name(len(names))
        if n is None:
            return names
        names.append(n)


def fft3d_profile_read(plan):
    """{pass name: (total ms, launches)} since the last read."""
    names = pass_names()
    n = len(names)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    st = load().fft3d_profile_read(_v(plan), ms, cnt, n)
    if st != FFT3D_OK:
        raise Fft3dError(st, "fft3d_profile_read")
    return {names[i]: (ms[i], cnt[i]) for i in range(n)}


def fft3d_pass_bytes(plan, pass_id):
    return load().fft3d_pass_bytes(_v(plan), pass_id)


def fft3d_energy(plan, spec_ptr, total_ptr, shells_ptr, nbins, stream=0):
    return load().fft3d_energy(_v(plan), _v(spec_ptr), _v(total_ptr), _v(shells_ptr), nbins, _v(stream))


def fft3d_energy_noalloc(spec_ptr, n0, n1, n2, batch, total_ptr, shells_ptr, nbins, stream=0):
    """fft3d_energy without a plan and without any device allocation (fixed
    library-owned scratch; see include/fft3d.h)."""
    return load().fft3d_energy_noalloc(_v(spec_ptr), n0, n1, n2, batch, _v(total_ptr), _v(shells_ptr), nbins,
                                       _v(stream))


def fft3d_nonlinear_plan(n0, n1, n2):
    return load().fft3d_nonlinear_plan(n0, n1, n2)


def fft3d_nonlinear_workspace_bytes(nl):
    return load().fft3d_nonlinear_workspace_bytes(_v(nl))


def fft3d_nonlinear_set_workspace(nl, dev_ptr):
    return load().fft3d_nonlinear_set_workspace(_v(nl), _v(dev_ptr))


def fft3d_nonlinear_exec(nl, uhat_ptr, nhat_ptr, stream=0):
    return load().fft3d_nonlinear_exec(_v(nl), _v(uhat_ptr), _v(nhat_ptr), _v(stream))


def fft3d_nonlinear_launches(nl):
    return load().fft3d_nonlinear_launches(_v(nl))


def fft3d_nonlinear_set_chunking(nl, planes, streams):
    return load().fft3d_nonlinear_set_chunking(_v(nl), planes, streams)


def fft3d_nonlinear_get_chunking(nl):
    a, b = ctypes.c_int(), ctypes.c_int()
    st = load().fft3d_nonlinear_get_chunking(_v(nl), ctypes.byref(a), ctypes.byref(b))
    if st != FFT3D_OK:
        raise Fft3dError(st, "fft3d_nonlinear_get_chunking")
    return a.value, b.value


def fft3d_nonlinear_destroy(nl):
    load().fft3d_nonlinear_destroy(_v(nl))


class _Closing:
    """Releases the handle on leaving a with-block (close() is idempotent)."""

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


class NonlinearTerm(_Closing):
    """Owning wrapper of fft3d_nonlinear_*: workspace from torch, then
    __call__(uhat (3, n0, n1, H) complex64 CUDA) -> (6, n0, n1, H) complex64."""

    def __init__(self, n0, n1, n2):
        import torch
        h = fft3d_nonlinear_plan(n0, n1, n2)
        if not h:
            raise Fft3dError(fft3d_last_error(), "fft3d_nonlinear_plan")
        self.handle = h
        self.shape = (n0, n1, n2)
        self._ws = torch.empty(fft3d_nonlinear_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        st = fft3d_nonlinear_set_workspace(h, self._ws.data_ptr())
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_nonlinear_set_workspace")

    def __call__(self, uhat, out=None, stream=None):
        import torch
        n0, n1, n2 = self.shape
        if out is None:
            out = torch.empty((6, n0, n1, n2 // 2 + 1), dtype=torch.complex64, device=uhat.device)
        st = fft3d_nonlinear_exec(self.handle, uhat.data_ptr(), out.data_ptr(),
                                  _stream_ptr(stream) if stream is not False else 0)
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_nonlinear_exec")
        return out

    def close(self):
        if self.handle:
            fft3d_nonlinear_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fft3d_autotune(plan, real_ptr, cplx_ptr, reps=5, stream=0):
    return load().fft3d_autotune(_v(plan), _v(real_ptr), _v(cplx_ptr), reps, _v(stream))


def fft3d_get_choices(plan):
    c = (ctypes.c_int * 5)()
    st = load().fft3d_get_choices(_v(plan), c)
    if st != FFT3D_OK:
        raise Fft3dError(st, "fft3d_get_choices")
    return list(c)


def fft3d_set_choices(plan, choices):
    if len(choices) != 5:
        raise ValueError("five choices: w0, w1, rows, tma0, tma1")
    c = (ctypes.c_int * 5)(*choices)
    return load().fft3d_set_choices(_v(plan), c)


def fft3d_ns_plan(n0, n1, n2):
    return load().fft3d_ns_plan(n0, n1, n2)


def fft3d_ns_workspace_bytes(ns):
    return load().fft3d_ns_workspace_bytes(_v(ns))


def fft3d_ns_set_workspace(ns, dev_ptr):
    return load().fft3d_ns_set_workspace(_v(ns), _v(dev_ptr))


def fft3d_ns_step(ns, uhat_ptr, nu, dt, stream=0):
    return load().fft3d_ns_step(_v(ns), _v(uhat_ptr), float(nu), float(dt), _v(stream))


def fft3d_ns_launches(ns):
    return load().fft3d_ns_launches(_v(ns))


def fft3d_ns_set_chunking(ns, planes, streams):
    return load().fft3d_ns_set_chunking(_v(ns), planes, streams)


def fft3d_ns_destroy(ns):
    load().fft3d_ns_destroy(_v(ns))


class NavierStokes(_Closing):
    """Owning wrapper of fft3d_ns_*: workspace from torch, then
    step(uhat, nu, dt) advances the (3, n0, n1, n2/2+1) complex64 CUDA tensor
    uhat in place by one Heun step."""

    def __init__(self, n0, n1, n2):
        import torch
        h = fft3d_ns_plan(n0, n1, n2)
        if not h:
            raise Fft3dError(fft3d_last_error(), "fft3d_ns_plan")
        self.handle = h
        self.shape = (n0, n1, n2)
        self._ws = torch.empty(fft3d_ns_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        st = fft3d_ns_set_workspace(h, self._ws.data_ptr())
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_ns_set_workspace")

    def step(self, uhat, nu, dt, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        s = stream.cuda_stream if stream is not False else 0
        st = fft3d_ns_step(self.handle, uhat.data_ptr(), nu, dt, s)
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_ns_step")
        return uhat

    def close(self):
        if self.handle:
            fft3d_ns_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fft3d_get_plane_choice(plan):
    """Cluster size of the plan's plane pass (0: separate row and n1 passes)."""
    c = load().fft3d_get_plane_choice(_v(plan))
    if c < 0:
        raise Fft3dError(-c, "fft3d_get_plane_choice")
    return c


def fft3d_set_plane_choice(plan, cluster):
    return load().fft3d_set_plane_choice(_v(plan), int(cluster))


def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[int(p) for p in ptrs])


def fft3d_plan_group(dims, counts, dtype=FFT3D_F32):
    d = (ctypes.c_int * (3 * len(dims)))(*[int(v) for t in dims for v in t])
    c = (ctypes.c_int * len(counts))(*[int(v) for v in counts])
    return load().fft3d_plan_group(d, c, len(dims), dtype)


def fft3d_group_plan_at(group, i):
    return load().fft3d_group_plan_at(_v(group), i)


def fft3d_group_r2c(group, in_ptrs, out_ptrs, stream=0):
    return load().fft3d_group_r2c(_v(group), _ptr_array(in_ptrs), _ptr_array(out_ptrs), _v(stream))


def fft3d_group_c2r(group, in_ptrs, out_ptrs, stream=0):
    return load().fft3d_group_c2r(_v(group), _ptr_array(in_ptrs), _ptr_array(out_ptrs), _v(stream))


def fft3d_group_r2c_c2r(group, in_ptrs, mid_ptrs, out_ptrs, stream=0):
    return load().fft3d_group_r2c_c2r(_v(group), _ptr_array(in_ptrs), _ptr_array(mid_ptrs), _ptr_array(out_ptrs),
                                      _v(stream))


def fft3d_group_launches(group, direction=-1):
    return load().fft3d_group_launches(_v(group), direction)


def fft3d_group_set_form(group, form):
    return load().fft3d_group_set_form(_v(group), form)


def fft3d_group_get_form(group):
    return load().fft3d_group_get_form(_v(group))


def fft3d_group_query_device_status(group, stream=0):
    return load().fft3d_group_query_device_status(_v(group), _v(stream))


def fft3d_group_destroy(group):
    load().fft3d_group_destroy(_v(group))


class Group(_Closing):
    """Owning wrapper of a grouped plan: dims [(n0, n1, n2), ...], counts
    [fields, ...].  r2c / c2r take lists of torch CUDA tensors, one per group
    (group i: counts[i] contiguous fields)."""

    def __init__(self, dims, counts, dtype=FFT3D_F32):
        h = fft3d_plan_group(dims, counts, dtype)
        if not h:
            raise Fft3dError(fft3d_last_error(), "fft3d_plan_group")
        self.handle = h
        self.dims = [tuple(d) for d in dims]
        self.counts = list(counts)

    def plan_at(self, i):
        return fft3d_group_plan_at(self.handle, i)

    def r2c(self, ins, outs, stream=0):
        st = fft3d_group_r2c(self.handle, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], stream)
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_group_r2c")

    def c2r(self, ins, outs, stream=0):
        st = fft3d_group_c2r(self.handle, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], stream)
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_group_c2r")

    def r2c_c2r(self, ins, mids, outs, stream=0):
        """Forward of ins into mids, then inverse of mids (clobbered) into outs, in one call."""
        st = fft3d_group_r2c_c2r(self.handle, [t.data_ptr() for t in ins], [t.data_ptr() for t in mids],
                                 [t.data_ptr() for t in outs], stream)
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_group_r2c_c2r")

    @property
    def form(self):
        return fft3d_group_get_form(self.handle)

    @form.setter
    def form(self, value):
        st = fft3d_group_set_form(self.handle, value)
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_group_set_form")

    def close(self):
        if self.handle:
            fft3d_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def error_string(status: int) -> str:
    try:
        return fft3d_error_string(status)
    except Exception:
        return "status %d" % status


# --- torch helpers (memory and streams only) -----------------------------------

class Plan(_Closing):
    """Owning wrapper of a plan handle (and of the workspace it may need)."""

    def __init__(self, n0, n1, n2, dtype=FFT3D_F32, batch=1, flags=0):
        h = fft3d_plan_variant(n0, n1, n2, dtype, batch, flags)
        if not h:
            raise Fft3dError(fft3d_last_error(), "fft3d_plan")
        self.handle = h
        self.shape = (n0, n1, n2)
        self.batch = batch
        self.flags = flags
        self.dtype = dtype
        self._ws = None
        nbytes = fft3d_workspace_bytes(h)
        if nbytes:
            import torch
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            st = fft3d_set_workspace(h, self._ws.data_ptr())
            if st != FFT3D_OK:
                raise Fft3dError(st, "fft3d_set_workspace")

    def describe(self):
        return fft3d_describe(self.handle)

    def r2c(self, in_ptr, out_ptr, stream=0):
        """Forward r2c through fft3d_r2c, or fft3d_r2c_f64 for an FFT3D_F64 plan."""
        f64 = self.dtype == FFT3D_F64
        st = (fft3d_r2c_f64 if f64 else fft3d_r2c)(self.handle, in_ptr, out_ptr, stream)
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_r2c_f64" if f64 else "fft3d_r2c")

    def c2r(self, in_ptr, out_ptr, stream=0):
        """Inverse c2r through fft3d_c2r, or fft3d_c2r_f64 for an FFT3D_F64 plan."""
        f64 = self.dtype == FFT3D_F64
        st = (fft3d_c2r_f64 if f64 else fft3d_c2r)(self.handle, in_ptr, out_ptr, stream)
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_c2r_f64" if f64 else "fft3d_c2r")

    def energy(self, spec, nbins):
        """(total, shells) FP64 CUDA tensors of a complex64 CUDA spectrum tensor."""
        import torch
        total = torch.empty(self.batch, dtype=torch.float64, device=spec.device)
        shells = torch.empty((self.batch, nbins), dtype=torch.float64, device=spec.device)
        st = fft3d_energy(self.handle, spec.data_ptr(), total.data_ptr(), shells.data_ptr(), nbins,
                          _stream_ptr(None))
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_energy")
        return total, shells

    def close(self):
        if self.handle:
            fft3d_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_plan_cache: dict = {}


def _cached_plan(shape, batch, dtype, flags):
    key = (tuple(shape), batch, dtype, flags)
    p = _plan_cache.get(key)
    if p is None:
        p = Plan(*shape, dtype=dtype, batch=batch, flags=flags)
        _plan_cache[key] = p
    return p


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def rfft3(x, dtype=FFT3D_F32, flags=0, stream=None):
    """Forward r2c of a float32 CUDA tensor (..., n0, n1, n2) -> complex64
    (..., n0, n1, n2/2+1); leading dimensions form the batch.  A float64
    tensor runs the FP64 path (FFT3D_F64) into complex128."""
    import torch
    if not (x.is_cuda and x.dtype in (torch.float32, torch.float64)):
        raise TypeError("rfft3 needs a float32 or float64 CUDA tensor")
    f64 = x.dtype == torch.float64
    if f64:
        dtype = FFT3D_F64
    elif dtype == FFT3D_F64:
        raise TypeError("FFT3D_F64 needs a float64 tensor")
    x = x.contiguous()
    n0, n1, n2 = x.shape[-3:]
    batch = int(x.numel() // (n0 * n1 * n2)) if x.numel() else 0
    out = torch.empty(x.shape[:-1] + (n2 // 2 + 1,), dtype=torch.complex128 if f64 else torch.complex64,
                      device=x.device)
    if batch == 0:
        return out
    _cached_plan((n0, n1, n2), batch, dtype, flags).r2c(x.data_ptr(), out.data_ptr(), _stream_ptr(stream))
    return out


def irfft3(X, n2, dtype=FFT3D_F32, flags=0, inplace_ok=False, stream=None):
    """Inverse c2r (unnormalised) of a complex64 CUDA tensor (..., n0, n1, n2/2+1);
    a complex128 tensor runs the FP64 path into float64.  The library clobbers
    its input, so X is cloned unless inplace_ok."""
    import torch
    if not (X.is_cuda and X.dtype in (torch.complex64, torch.complex128)):
        raise TypeError("irfft3 needs a complex64 or complex128 CUDA tensor")
    f64 = X.dtype == torch.complex128
    if f64:
        dtype = FFT3D_F64
    elif dtype == FFT3D_F64:
        raise TypeError("FFT3D_F64 needs a complex128 tensor")
    n0, n1, H = X.shape[-3:]
    if H != n2 // 2 + 1:
        raise ValueError("last dimension must be n2/2+1")
    X = X.contiguous() if inplace_ok else X.clone(memory_format=torch.contiguous_format)
    batch = int(X.numel() // (n0 * n1 * H)) if X.numel() else 0
    out = torch.empty(X.shape[:-1] + (n2,), dtype=torch.float64 if f64 else torch.float32, device=X.device)
    if batch == 0:
        return out
    _cached_plan((n0, n1, n2), batch, dtype, flags).c2r(X.data_ptr(), out.data_ptr(), _stream_ptr(stream))
    return out

"""Autotuning cache ("wisdom"): kernel shape choices per GPU and transform.

fft3d_autotune (C) times the candidate shapes of every pass on the caller's
buffers and keeps the fastest; this module stores the chosen six integers
{w0, w1, rows, tma0, tma1, plane cluster size} in a JSON file so later plans of
the same GPU model, driver and shape reuse them without tuning.  File: $FFT3D_TUNE_CACHE, else
~/.cache/fft3d_wisdom.json.
"""
from __future__ import annotations

import json
import os
import tempfile

from . import (FFT3D_F32, FFT3D_OK, Fft3dError, Plan, fft3d_autotune, fft3d_get_choices,
               fft3d_get_plane_choice, fft3d_set_choices, fft3d_set_plane_choice)


def cache_path() -> str:
    return os.environ.get("FFT3D_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                               "fft3d_wisdom.json")


def driver_version() -> int:
    """The CUDA driver's version number (cuDriverGetVersion), 0 if unknown."""
    import ctypes
    try:
        v = ctypes.c_int(0)
        if ctypes.CDLL("libcuda.so.1").cuDriverGetVersion(ctypes.byref(v)) != 0:
            return 0
        return v.value
    except OSError:
        return 0


def cache_key(gpu: str, shape, batch: int, dtype: int, flags: int, driver: int | None = None) -> str:
    """Entries are per GPU model and driver (a new driver may change which
    kernel shape is fastest), shape, batch, dtype and flags."""
    n0, n1, n2 = shape
    drv = driver_version() if driver is None else driver
    return f"{gpu}|drv{drv}|{n0}x{n1}x{n2}|b{batch}|d{dtype}|f{flags}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(entries: dict, path: str | None = None) -> None:
    """Merge entries into the cache file (atomic replace)."""
    path = path or cache_path()
    data = load_cache(path)
    data.update(entries)
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", prefix=".fft3d_wisdom")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned_plan(n0, n1, n2, batch=1, dtype=FFT3D_F32, flags=0, reps=5, path=None, retune=False):
    """A Plan whose kernel shapes come from the cache, or from fft3d_autotune
    on scratch torch buffers (then stored).  Returns (plan, tuned_now)."""
    import torch
    plan = Plan(n0, n1, n2, dtype=dtype, batch=batch, flags=flags)
    gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, (n0, n1, n2), batch, dtype, flags)
    cached = None if retune else load_cache(path).get(key)
    if cached is not None and len(cached) in (5, 6):
        st = fft3d_set_choices(plan.handle, cached[:5])
        if st != FFT3D_OK:
            raise Fft3dError(st, "fft3d_set_choices")
        if len(cached) == 6:
            st = fft3d_set_plane_choice(plan.handle, cached[5])
            if st != FFT3D_OK:
                raise Fft3dError(st, "fft3d_set_plane_choice")
        return plan, False
    real = torch.empty(batch * n0 * n1 * n2, dtype=torch.float32, device="cuda").normal_()
    cplx = torch.empty(batch * n0 * n1 * (n2 // 2 + 1), dtype=torch.complex64, device="cuda")
    st = fft3d_autotune(plan.handle, real.data_ptr(), cplx.data_ptr(), reps,
                        torch.cuda.current_stream().cuda_stream)
    if st != FFT3D_OK:
        raise Fft3dError(st, "fft3d_autotune")
    store_cache({key: fft3d_get_choices(plan.handle) + [fft3d_get_plane_choice(plan.handle)]}, path)
    return plan, True

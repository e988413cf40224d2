"""The allocation-free energy entry point (fft3d_energy_noalloc) against the
plan-based one (fft3d_energy).

fft3d_energy_noalloc serves callers that cannot allocate device memory
(their memory belongs to their own allocator or to a fixed budget): it keeps
its scratch in one fixed array inside the library.  This file is named so
that pytest collects it last; it needs nothing from the other test files and
passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

# The tolerance the energy tests use: |X|^2 in FP32, sums in FP64.
REL = 1e-6


def _spectrum(shape, batch, seed):
    n0, n1, H = shape
    re = synth.uniform_field((batch, n0, n1, H), seed)
    im = synth.uniform_field((batch, n0, n1, H), seed + 1)
    return torch.from_numpy((re + 1j * im).astype(np.complex64)).cuda()


def _noalloc(lib, spec, n0, n1, n2, batch, nbins):
    total = torch.full((batch,), -1.0, dtype=torch.float64, device="cuda")
    shells = torch.full((batch, nbins), -1.0, dtype=torch.float64, device="cuda")
    st = lib.fft3d_energy_noalloc(spec.data_ptr(), n0, n1, n2, batch, total.data_ptr(), shells.data_ptr(), nbins,
                                  torch.cuda.current_stream().cuda_stream)
    assert st == lib.FFT3D_OK, lib.error_string(st)
    torch.cuda.synchronize()
    return total.cpu().numpy(), shells.cpu().numpy()


def test_noalloc_energy_matches_plan_energy_on_two_calls(cuda_lib):
    lib = cuda_lib
    # two calls in a row, different inputs; then an odd n2 (no Nyquist bin)
    cases = [((64, 48, 40), 2, 30, 81), ((32, 32, 32), 1, 28, 83), ((12, 10, 15), 1, 9, 85)]
    for (n0, n1, n2), batch, nbins, seed in cases:
        spec = _spectrum((n0, n1, n2 // 2 + 1), batch, seed)
        plan = lib.Plan(n0, n1, n2, batch=batch)
        ref_total, ref_shells = plan.energy(spec, nbins)
        ref_total = ref_total.cpu().numpy()
        ref_shells = ref_shells.cpu().numpy()
        total, shells = _noalloc(lib, spec, n0, n1, n2, batch, nbins)
        assert np.all(np.abs(total - ref_total) <= REL * np.abs(ref_total))
        assert np.all(np.abs(shells - ref_shells) <= REL * np.abs(ref_shells) + 1e-12)
        plan.close()


def test_noalloc_energy_rejects_calls_beyond_its_scratch(cuda_lib):
    lib = cuda_lib
    out = torch.full((8193,), 7.0, dtype=torch.float64, device="cuda")
    spec = torch.zeros(16, dtype=torch.complex64, device="cuda")
    # 256 blocks * (8192 + 1) doubles exceed the fixed 2^18-double array
    st = lib.fft3d_energy_noalloc(spec.data_ptr(), 2048, 2048, 2048, 1, out.data_ptr(), out[1:].data_ptr(), 8192, 0)
    assert st == lib.FFT3D_ERR_UNSUPPORTED_SIZE
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())

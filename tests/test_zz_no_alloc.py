"""The allocation-free energy entry point (fft3d_energy_noalloc) against the
plan-based one (fft3d_energy).

fft3d_energy_noalloc serves callers that cannot allocate device memory
(their memory belongs to their own allocator or to a fixed budget): it keeps
its scratch in one fixed array inside the library.  Its rejection of calls
larger than that array is tested on the CPU (tests/test_abi.py), where the
check cannot launch anything.  This file is named so
that pytest collects it last; it needs nothing from the other test files and
passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
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


def _oracle(spec, n0, n1, n2, nbins):
    """oracle.half_energy / shell_energy of every batch entry (FP64)."""
    X = spec.cpu().numpy().astype(np.complex128)
    return (np.array([oracle.half_energy(Xb, n2) for Xb in X]),
            np.array([oracle.shell_energy(Xb, n0, n1, n2, nbins) for Xb in X]))


def test_noalloc_energy_matches_plan_energy_and_oracle_on_two_calls(cuda_lib):
    """Each case is two calls in a row on the shared scratch (the second on a
    new input), checked against fft3d_energy (the existing entry point) and
    against the FP64 oracle sums.  Cases: a batch, an odd n2 (no Nyquist bin)
    and nbins = 8192 (the histogram above 48 KB of shared memory)."""
    lib = cuda_lib
    cases = [((64, 48, 40), 2, 30, 81), ((32, 32, 32), 1, 28, 83), ((12, 10, 15), 1, 9, 85),
             ((12, 10, 15), 1, 8192, 87)]
    for (n0, n1, n2), batch, nbins, seed in cases:
        plan = lib.Plan(n0, n1, n2, batch=batch)
        for call in range(2):
            spec = _spectrum((n0, n1, n2 // 2 + 1), batch, seed + 10 * call)
            ref_total, ref_shells = plan.energy(spec, nbins)
            ref_total = ref_total.cpu().numpy()
            ref_shells = ref_shells.cpu().numpy()
            total, shells = _noalloc(lib, spec, n0, n1, n2, batch, nbins)
            assert np.all(np.abs(total - ref_total) <= REL * np.abs(ref_total))
            assert np.all(np.abs(shells - ref_shells) <= REL * np.abs(ref_shells) + 1e-12)
            o_total, o_shells = _oracle(spec, n0, n1, n2, nbins)
            assert np.all(np.abs(total - o_total) <= REL * o_total)
            assert np.all(np.abs(shells - o_shells) <= REL * o_shells + 1e-12)
        plan.close()


def test_noalloc_energy_batch_beyond_one_grid_dimension(cuda_lib):
    """70000 batch entries (more than a grid's y extent) of a 1 x 1 x 2 field:
    the launches are split over the batch; every entry against the oracle."""
    n0, n1, n2, batch, nbins = 1, 1, 2, 70000, 2
    spec = _spectrum((n0, n1, n2 // 2 + 1), batch, 91)
    for call in range(2):
        total, shells = _noalloc(cuda_lib, spec, n0, n1, n2, batch, nbins)
        o_total, o_shells = _oracle(spec, n0, n1, n2, nbins)
        assert np.all(np.abs(total - o_total) <= REL * o_total)
        assert np.all(np.abs(shells - o_shells) <= REL * o_shells + 1e-12)

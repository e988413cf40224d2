// FP64 spectral diagnostics (Parseval sum, shell-binned energies); see energy.cu.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace fft3d {

// Thread blocks per batch entry used by launch_energy for rows = n0*n1 rows.
int energy_blocks_per_entry(long long rows);
// Scratch (doubles) launch_energy needs: batch * blocks * (nbins + 1).
size_t energy_scratch_doubles(int batch, long long rows, int nbins);
// total[b] (may be NULL) and shells[b*nbins + bin] (may be NULL) for each batch entry b.
cudaError_t launch_energy(const void* X, int n0, int n1, int n2, int batch, int nbins, double* scratch,
                          double* total, double* shells, cudaStream_t s);

}  // namespace fft3d

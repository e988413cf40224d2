// fft3d_energy_noalloc: the FP64 spectral diagnostics of fft3d_energy for
// callers that cannot allocate device memory, e.g. applications whose device
// memory is owned entirely by their own allocator or by a budget fixed at
// start-up, or code called back from inside another library's memory
// management, where a cudaMalloc in a library call would fail, block, or
// break that budget.
//
// It needs no plan (the diagnostics use no twiddle tables) and allocates
// nothing: the block partials go to one file-scope device array of fixed
// size, which every GPU that loads this library holds until the process
// exits.  Host code cannot use the array's name as a device address, so
// every call looks up its address on the current device
// (cudaGetSymbolAddress, a host-side lookup).  The first call on a device is
// its set-up: the lookup may load this library's device code there, so it
// must not happen inside a stream capture.  Looking up again on later calls
// keeps the address right after anything that recreates the device's
// context (cudaDeviceReset).
#include <cstdint>

#include "energy.h"
#include "fft3d.h"

namespace {

// Scratch capacity in doubles: 2 MiB.
constexpr size_t kNoallocScratchDoubles = size_t(1) << 18;

static __device__ __align__(256) double g_energy_scratch[kNoallocScratchDoubles];

// Device address of g_energy_scratch on the current device.
cudaError_t scratch_for_current_device(double** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" int fft3d_energy_noalloc(const void* spec, int n0, int n1, int n2, int batch, double* total,
                                    double* shells, int nbins, void* stream)
{
    if (!spec || n0 < 1 || n1 < 1 || n2 < 2 || batch < 1 || nbins < 1 || nbins > 8192 ||
        (!total && !shells))
        return FFT3D_ERR_INVALID_ARG;
    if (((uintptr_t)spec & 15) || ((uintptr_t)total & 7) || ((uintptr_t)shells & 7)) return FFT3D_ERR_MISALIGNED;
    if (fft3d::energy_scratch_doubles(batch, (long long)n0 * n1, nbins) > kNoallocScratchDoubles)
        return FFT3D_ERR_UNSUPPORTED_SIZE;  // the fixed scratch array is too small for this call
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return FFT3D_ERR_CUDA;
    if (fft3d::launch_energy(spec, n0, n1, n2, batch, nbins, scratch, total, shells, (cudaStream_t)stream) !=
        cudaSuccess)
        return FFT3D_ERR_CUDA;
    return FFT3D_OK;
}

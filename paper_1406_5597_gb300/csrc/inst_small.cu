// Specialised kernels for short axes (8 .. 128).
#include "inst.cuh"

namespace fft3d {
const LenEntry* entries_small(int* n)
{
    static const LenEntry e[] = {
        FFT3D_ENTRY_COLROW(8, 8, 256, 8, 128),
        FFT3D_ENTRY_COLROW(16, 16, 256, 16, 128),
        FFT3D_ENTRY_COLROW(32, 8, 64, 8, 64),
        FFT3D_ENTRY_COLROW(64, 8, 32, 8, 32),
        FFT3D_ENTRY_COLROW(128, 8, 32, 8, 16),
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

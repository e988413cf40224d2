// Specialised kernels for axes with factors 3 and 5 (48 .. 1536).
#include "inst.cuh"

namespace fft3d {
const LenEntry* entries_mixed(int* n)
{
    static const LenEntry e[] = {
        FFT3D_ENTRY_COLROW(48, 12, 64, 12, 64),
        FFT3D_ENTRY_COLROW(80, 20, 64, 20, 32),
        FFT3D_ENTRY_COLROW(96, 24, 64, 24, 32),
        FFT3D_ENTRY_COL(160, 20, 32),
        FFT3D_ENTRY_COL(192, 24, 32),
        FFT3D_ENTRY_COL(1536, 24, 8),
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

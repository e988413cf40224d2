// Specialised kernels for 1024 and 2048.
#include "inst.cuh"

namespace fft3d {
const LenEntry* entries_1024_2048(int* n)
{
    static const LenEntry e[] = {
        FFT3D_ENTRY_COLROW(1024, 16, 8, 16, 4),
        FFT3D_ENTRY_COL(2048, 16, 8),
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

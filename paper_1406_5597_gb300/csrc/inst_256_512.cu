// Specialised kernels for 256 and 512.
#include "inst.cuh"

namespace fft3d {
const LenEntry* entries_256_512(int* n)
{
    static const LenEntry e[] = {
        FFT3D_ENTRY_COLROW(256, 8, 16, 8, 8),
        FFT3D_ENTRY_COLROW(512, 8, 16, 16, 8),
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

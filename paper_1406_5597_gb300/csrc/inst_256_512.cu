// Specialised kernels for 256 and 512.
#include "inst.cuh"

namespace fft3d {
const LenEntry* entries_256_512(int* n)
{
    static const LenEntry e[] = {
        {256, FFT3D_COL(256, 8, 16), FFT3D_TMA(256, 16, 16, 2, 0, 32, 3, 2), FFT3D_ROWW(256, 16, 4)},
        {512, FFT3D_COL(512, 8, 8), FFT3D_TMA(512, 32, 16, 2, 0, 32, 2, 2), FFT3D_ROWW(512, 16, 2)},
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

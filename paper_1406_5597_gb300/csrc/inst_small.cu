// Specialised kernels for short axes (8 .. 128).
#include "inst.cuh"

namespace fft3d {
const LenEntry* entries_small(int* n)
{
    static const LenEntry e[] = {
        {8, FFT3D_COL(8, 8, 256), FFT3D_NO_TMA, FFT3D_ROWW(8, 8, 64)},
        {16, FFT3D_COL(16, 16, 256), FFT3D_NO_TMA, FFT3D_ROWW(16, 16, 64)},
        {32, FFT3D_COL(32, 8, 64), FFT3D_NO_TMA, FFT3D_ROWW(32, 8, 16)},
        {64, FFT3D_COL(64, 8, 32), FFT3D_TMA(64, 8, 16, 3, 0, 8, 3, 0), FFT3D_ROWW(64, 8, 8)},
        {128, FFT3D_COL(128, 8, 32), FFT3D_TMA(128, 8, 16, 3, 0, 8, 3, 0), FFT3D_ROWW(128, 8, 4)},
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

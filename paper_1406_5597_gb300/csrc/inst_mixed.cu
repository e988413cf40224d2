// Specialised kernels for axes with factors 3 and 5 (48 .. 1536).
#include "inst.cuh"

namespace fft3d {
const LenEntry* entries_mixed(int* n)
{
    static const LenEntry e[] = {
        {48, FFT3D_COL(48, 12, 64), FFT3D_NO_TMA, FFT3D_ROWW(48, 12, 16)},
        {80, FFT3D_COL(80, 20, 64), FFT3D_NO_TMA, FFT3D_ROWW(80, 20, 16)},
        {96, FFT3D_COL(96, 24, 64), FFT3D_TMA(96, 24, 16, 3, 0, 24, 3, 0), FFT3D_ROWW(96, 12, 16)},
        {160, FFT3D_COL(160, 20, 32), FFT3D_TMA(160, 20, 16, 3, 0, 20, 3, 0), FFT3D_ROWW_NONL(160, 20, 8)},
        {192, FFT3D_COL(192, 24, 32), FFT3D_TMA(192, 24, 16, 3, 0, 24, 3, 0), FFT3D_ROWW_NONL(192, 12, 8)},
        {1536, FFT3D_COL(1536, 24, 8), FFT3D_TMA_NOPAIR(1536, 24, 8, 2, 0), FFT3D_NO_ROW},
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

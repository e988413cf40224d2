// Specialised kernels for the longer axes with a factor 3 or 5 (320 .. 1280):
// column passes in registers (20 or 24 values per thread, radices 8 / 4 / 2
// with one radix-5 or radix-3 stage) and warp-resident row transforms for the
// same lengths as n2/2.
#include "inst.cuh"

namespace fft3d {
const LenEntry* entries_mixed_wide(int* n)
{
    static const LenEntry e[] = {
        {320, FFT3D_COL(320, 20, 16), FFT3D_TMA(320, 20, 16, 2, 0, 20, 2, 0), FFT3D_ROWW_NONL(320, 20, 4)},
        {384, FFT3D_COL(384, 24, 16), FFT3D_TMA(384, 24, 16, 2, 0, 24, 2, 0), FFT3D_ROWW_NONL(384, 24, 4)},
        {640, FFT3D_COL(640, 20, 16), FFT3D_TMA(640, 20, 8, 2, 0, 20, 2, 0), FFT3D_ROWW_NONL(640, 20, 2)},
        {768, FFT3D_COL(768, 24, 16), FFT3D_TMA(768, 24, 8, 2, 0, 24, 2, 0), FFT3D_ROWW_NONL(768, 24, 2)},
        {1280, FFT3D_COL(1280, 20, 8), FFT3D_NO_TMA, FFT3D_NO_ROW},
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

// Specialised kernels for 1024 and 2048.
#include "inst.cuh"
#include "tma2.cuh"

namespace fft3d {
const LenEntry* entries_1024_2048(int* n)
{
    static const LenEntry e[] = {
        {1024, FFT3D_COL(1024, 32, 16), FFT3D_TMA(1024, 16, 8, 2, 0, 16, 2, 2), FFT3D_ROWW_NONL(1024, 32, 2),
         &launch_col_tma2<1024, 16, 8, 2, -1>, &launch_col_tma2<1024, 16, 8, 2, 1>},
        // 2048: 4-wide TMA tiles pay at the short n1 stride (row pairs, odd H:
        // 3.9 vs 3.5 TB/s for the plain 8-wide kernel), not at the n0 stride
        {2048, FFT3D_COL(2048, 32, 8), FFT3D_TMA(2048, 16, 4, 2, 0, 16, 2, 0), FFT3D_NO_ROW,
         &launch_col_tma2<2048, 16, 4, 2, -1>, &launch_col_tma2<2048, 16, 4, 2, 1>},
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}
}  // namespace fft3d

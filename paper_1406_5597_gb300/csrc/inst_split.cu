// Cluster-split column kernels of the long axes (colsplit.cuh): per length,
// the cluster size C, elements per thread E and columns per tile W.
#include "colsplit.cuh"

namespace fft3d {

#define FFT3D_SPLIT(L, C, E, W) \
    { L, C, E, W, &fft3d::launch_col_split<L, C, E, W, -1>, &fft3d::launch_col_split<L, C, E, W, 1> }

const SplitEntry* split_entries(int* n)
{
    static const SplitEntry e[] = {
        FFT3D_SPLIT(1024, 2, 32, 16),  // 512-row halves, 128-byte row segments
        FFT3D_SPLIT(1024, 4, 16, 16),  // 256-row quarters: smaller CTAs, more of them per SM
        FFT3D_SPLIT(1536, 2, 24, 8),   // 768-row halves (radix 8, 8, 4, 3)
        FFT3D_SPLIT(2048, 2, 32, 8),   // 1024-row halves, 64-byte row segments
        FFT3D_SPLIT(2048, 4, 32, 16),  // 512-row quarters, 128-byte row segments
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}

}  // namespace fft3d

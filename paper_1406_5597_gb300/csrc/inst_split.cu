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

const TmaSplitEntry* tma_split_entries(int* n)
{
    static const TmaSplitEntry e[] = {
        {1024, 2, &fft3d::launch_col_tma_split<2, -1>, &fft3d::launch_col_tma_split<2, 1>},
        {1536, 3, &fft3d::launch_col_tma_split<3, -1>, &fft3d::launch_col_tma_split<3, 1>},
        {2048, 4, &fft3d::launch_col_tma_split<4, -1>, &fft3d::launch_col_tma_split<4, 1>},
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}

template <int C, bool PARK>
int l2split_ctas()
{
    static PerDevice resident;
    int ctas = 0;
    return resident_ctas_per_device(resident, col_l2split_kernel<C, -1, PARK>, L2SplitGeom<C, PARK>::NT,
                                    L2SplitGeom<C, PARK>::smem, &ctas) == cudaSuccess
               ? ctas
               : 0;
}

#define FFT3D_L2SPLIT(L, C, PARK)                                                                       \
    { L, C, &launch_col_l2split<C, -1, PARK>, &launch_col_l2split<C, 1, PARK>,                          \
      &launch_col_l2split<C, -1, false, true>, &launch_col_l2split<C, 1, false, true>,                  \
      &l2split_scratch_values<C, PARK>, &l2split_ctas<C, PARK> }
#define FFT3D_L2SPLIT_NOSHIFT(L, C, PARK)                                                               \
    { L, C, &launch_col_l2split<C, -1, PARK>, &launch_col_l2split<C, 1, PARK>, nullptr, nullptr,        \
      &l2split_scratch_values<C, PARK>, &l2split_ctas<C, PARK> }

const L2SplitEntry* l2split_entries(int* n)
{
    static const L2SplitEntry e[] = {
        FFT3D_L2SPLIT(1024, 2, false),          // the other residue in L2
        FFT3D_L2SPLIT_NOSHIFT(1536, 3, true),   // residue 1 in shared memory, residue 0 in L2
        FFT3D_L2SPLIT(2048, 4, false),          // residues 0 .. 2 in L2
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}

}  // namespace fft3d

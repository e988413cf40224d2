// Column kernels with tensor-core radix-16 stages (split-BF16 and FP16).
#include "kernels.cuh"
#include "tc.cuh"

namespace fft3d {

#define FFT3D_TC(L, W)                                                                                      \
    {L, W, &launch_col_tc<L, W, TC_BF16X3, -1>, &launch_col_tc<L, W, TC_BF16X3, 1>,                       \
     &launch_col_tc<L, W, TC_F16, -1>, &launch_col_tc<L, W, TC_F16, 1>}

const TcEntry* tc_entries(int* n)
{
    static const TcEntry e[] = {
        FFT3D_TC(256, 16),
        FFT3D_TC(512, 16),
        FFT3D_TC(1024, 8),
        FFT3D_TC(2048, 8),
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}

}  // namespace fft3d

// Instantiation helpers: each inst_*.cu translation unit builds the
// specialised kernels for a group of lengths (compiled in parallel) and
// exposes them as a LenEntry table.
#pragma once
#include "kernels.cuh"

#define FFT3D_ENTRY_COLROW(L, CE, CW, RE, RR)                                                    \
    fft3d::LenEntry{L, CE, CW, RE, RR, &fft3d::launch_col<L, CE, CW, -1>,                       \
                    &fft3d::launch_col<L, CE, CW, 1>, &fft3d::launch_row<L, RE, RR, -1>,          \
                    &fft3d::launch_row<L, RE, RR, 1>}

#define FFT3D_ENTRY_COL(L, CE, CW)                                                               \
    fft3d::LenEntry{L, CE, CW, 0, 0, &fft3d::launch_col<L, CE, CW, -1>,                         \
                    &fft3d::launch_col<L, CE, CW, 1>, nullptr, nullptr}

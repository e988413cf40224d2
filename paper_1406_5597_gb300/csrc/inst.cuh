// Instantiation helpers: each inst_*.cu translation unit builds the
// specialised kernels for a group of lengths (compiled in parallel) and
// exposes them as a LenEntry table.
#pragma once
#include "kernels.cuh"

// plain column kernel: E elements per thread, W columns per CTA
#define FFT3D_COL(L, E, W) E, W, &fft3d::launch_col<L, E, W, -1>, &fft3d::launch_col<L, E, W, 1>
#define FFT3D_NO_TMA 0, 0, nullptr, nullptr, nullptr, nullptr, 0
// TMA-fed persistent column kernel: E elements per thread, W columns per
// tile, ring stages, L2 prefetch distance; the row-pair variant (odd axis
// stride) uses PE elements per thread, PST stages and prefetch distance PPF
#define FFT3D_TMA(L, E, W, ST, PF, PE, PST, PPF)                                                              \
    E, W, &fft3d::launch_col_tma<L, E, W, ST, -1, PF>, &fft3d::launch_col_tma<L, E, W, ST, 1, PF>,            \
        &fft3d::launch_col_tma<L, PE, W, PST, -1, PPF, true>, &fft3d::launch_col_tma<L, PE, W, PST, 1, PPF, true>, PE
#define FFT3D_TMA_NOPAIR(L, E, W, ST, PF) \
    E, W, &fft3d::launch_col_tma<L, E, W, ST, -1, PF>, &fft3d::launch_col_tma<L, E, W, ST, 1, PF>, nullptr, nullptr, 0
// warp-resident rows (T = L/E <= 32), ROWS rows per CTA
#define FFT3D_ROWW(L, E, R)                                                                              \
    E, R, true, &fft3d::launch_row_warp<L, E, R, -1>, &fft3d::launch_row_warp<L, E, R, 1>,              \
        &fft3d::launch_row_nonlinear<L, E, R>
// warp-resident rows without the fused nonlinear-term kernel (too many registers at this length)
#define FFT3D_ROWW_NONL(L, E, R) E, R, true, &fft3d::launch_row_warp<L, E, R, -1>, &fft3d::launch_row_warp<L, E, R, 1>, nullptr
// shared-memory staged rows
#define FFT3D_ROWS(L, E, R) E, R, false, &fft3d::launch_row<L, E, R, -1>, &fft3d::launch_row<L, E, R, 1>, nullptr
#define FFT3D_NO_ROW 0, 0, false, nullptr, nullptr, nullptr

// Cluster plane kernels (n2 rows + n1 columns of a plane in one cluster's
// distributed shared memory, or in one CTA's shared memory for clusters of
// one) for the (n2/2, n1) pairs of the cubic grids, at several cluster sizes.
#include "cplane.cuh"

namespace fft3d {

#define FFT3D_CPLANE(LR, ER, LC, C, NT, MINB) \
    {LR, LC, C, NT, &launch_cplane<LR, ER, LC, C, NT, -1, MINB>, &launch_cplane<LR, ER, LC, C, NT, 1, MINB>}

const CPlaneEntry* cplane_entries(int* n)
{
    // the first entry of a shape is its default; fft3d_autotune tries them all
    static const CPlaneEntry e[] = {
        FFT3D_CPLANE(16, 8, 32, 2, 32, 1),      // 32^3: 2 CTAs x 16 rows
        FFT3D_CPLANE(32, 8, 64, 1, 128, 2),     // 64^3: the plane in one CTA's shared memory
        FFT3D_CPLANE(64, 8, 128, 2, 256, 2),    // 128^3: 2 CTAs x 64 rows
        FFT3D_CPLANE(64, 8, 128, 1, 256, 2),    // 128^3: one CTA x 128 rows
        FFT3D_CPLANE(128, 8, 256, 4, 256, 2),   // 256^3: 4 CTAs x 64 rows
        FFT3D_CPLANE(128, 8, 256, 2, 512, 1),   // 256^3: 2 CTAs x 128 rows
        FFT3D_CPLANE(256, 16, 512, 8, 512, 1),  // 512^3: 8 CTAs x 64 rows
        FFT3D_CPLANE(48, 12, 96, 3, 128, 2),    // 96^3: 3 CTAs x 32 rows
        FFT3D_CPLANE(80, 20, 160, 5, 128, 2),   // 160^3: 5 CTAs x 32 rows
        FFT3D_CPLANE(96, 24, 192, 3, 256, 2),   // 192^3: 3 CTAs x 64 rows
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}

}  // namespace fft3d

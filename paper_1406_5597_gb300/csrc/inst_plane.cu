// Fused plane kernels (n2 rows + n1 columns in one persistent launch) for
// the (n2/2, n1) pairs of the common grid sizes.
#include "plane.cuh"

namespace fft3d {

#define FFT3D_PLANE(LR, ER, LC, EC, NT, MINB) \
    {LR, LC, ER, EC, NT, &launch_plane<LR, ER, LC, EC, NT, -1, MINB>, &launch_plane<LR, ER, LC, EC, NT, 1, MINB>}

const PlaneEntry* plane_entries(int* n)
{
    static const PlaneEntry e[] = {
        FFT3D_PLANE(16, 16, 32, 8, 128, 8),      // 32^3
        FFT3D_PLANE(64, 8, 128, 8, 256, 4),      // 128^3
        FFT3D_PLANE(128, 8, 256, 8, 256, 4),     // 256^3
        FFT3D_PLANE(256, 16, 512, 16, 256, 3),   // 512^3
        FFT3D_PLANE(512, 16, 1024, 16, 512, 1),  // 1024^3
    };
    *n = (int)(sizeof(e) / sizeof(e[0]));
    return e;
}

}  // namespace fft3d

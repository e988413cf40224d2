// Explicit n0 <-> n1 transpose of a complex (n0, n1, H) volume: the
// "transpose" of Sec. 2.1 step 2 ("axes 0 and 1 are flipped").  It exists
// only for the comparator variant (FFT3D_FLAG_EXPLICIT_TRANSPOSE); the
// transpose-free path never calls it.  With the n2 axis innermost every
// (j0, j1) row of H complex values moves as one contiguous unit:
//     out[b][j1][j0][:] = in[b][j0][j1][:].
#include "args.h"

namespace fft3d {

namespace {
__global__ void swap01_kernel(const float2* __restrict__ in, float2* __restrict__ out, long long n0, long long n1,
                              long long H, long long rows_total)
{
    // one warp per row; rows indexed in the SOURCE order (b, j0, j1)
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= rows_total) return;
    const long long j1 = warp % n1;
    const long long t = warp / n1;
    const long long j0 = t % n0;
    const long long b = t / n0;
    const float2* src = in + warp * H;
    float2* dst = out + ((b * n1 + j1) * n0 + j0) * H;
    for (long long k = lane; k < H; k += 32) dst[k] = src[k];
}
}  // namespace

cudaError_t launch_swap01(const float2* in, float2* out, long long batch, long long n0, long long n1, long long H,
                          cudaStream_t s)
{
    const long long rows = batch * n0 * n1;
    if (rows <= 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (rows * 32 + threads - 1) / threads;
    swap01_kernel<<<(unsigned)blocks, threads, 0, s>>>(in, out, n0, n1, H, rows);
    return cudaGetLastError();
}

}  // namespace fft3d

// FP64 spectral diagnostics of a half spectrum: the Parseval sum and the
// shell-binned energy spectrum.  They check a transform on the device and are
// the energy spectrum E(k) a turbulence solver reports (the pseudo-spectral
// context of Sec. 1).
//
// For X of shape batch x n0 x n1 x H (H = n2/2+1), per batch entry:
//   total    = sum over the half spectrum of c_k2 |X[k]|^2,
//              c_k2 = 1 at k2 = 0 and (even n2) k2 = n2/2, else 2  (= N sum_j x_j^2 when X = r2c(x));
//   shell[b] = the same sum restricted to the bins whose integer shell is b,
//              b = floor(|k| + 1/2) with |k_a| = min(j_a, n_a - j_a): shell 0
//              is k = 0 alone, shell b >= 1 is (2b-1)^2 <= 4|k|^2 < (2b+1)^2,
//              decided in integer arithmetic (no rounding picks a bin).
// |X|^2 is formed in FP32 and accumulated in FP64 (per thread, then per block
// in shared memory); block partials are summed in a fixed order by a second
// kernel, so the result does not depend on scheduling.
#include <cstdint>

#include "energy.h"

namespace fft3d {

namespace {

__device__ __forceinline__ int shell_of(long long kk4)
{
    // b = floor((sqrt(kk4) + 1) / 2), corrected in integers
    long long b = (long long)((sqrt((double)kk4) + 1.0) * 0.5);
    while (b > 0 && (2 * b - 1) * (2 * b - 1) > kk4) --b;
    while ((2 * b + 1) * (2 * b + 1) <= kk4) ++b;
    return (int)b;
}

// grid (blocks_per_entry, batch entries of this launch); batch entry b0 + blockIdx.y;
// partials: batch x blocks x (nbins + 1) doubles, slot nbins holds the block's total.
__global__ void energy_partials_kernel(const float2* __restrict__ X, int n0, int n1, int n2, int nbins,
                                       long long b0, double* __restrict__ partials)
{
    extern __shared__ double hist[];  // nbins + 1
    const int H = n2 / 2 + 1;
    const long long rows = (long long)n0 * n1;
    const long long b = b0 + blockIdx.y;
    const float2* Xb = X + b * rows * H;
    for (int i = threadIdx.x; i <= nbins; i += blockDim.x) hist[i] = 0.0;
    __syncthreads();
    double total = 0.0;
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long r = (long long)blockIdx.x * warps + warp; r < rows; r += (long long)gridDim.x * warps) {
        const int j0 = (int)(r / n1), j1 = (int)(r - (long long)j0 * n1);
        const long long a0 = min(j0, n0 - j0), a1 = min(j1, n1 - j1);
        const long long base = 4 * (a0 * a0 + a1 * a1);
        const float2* row = Xb + r * H;
        for (int k2 = lane; k2 < H; k2 += 32) {
            const float2 v = row[k2];
            const float c = (k2 == 0 || 2 * k2 == n2) ? 1.f : 2.f;
            const double e = (double)(c * fmaf(v.x, v.x, v.y * v.y));
            total += e;
            const int sb = shell_of(base + 4ll * k2 * k2);
            if (sb < nbins) atomicAdd(&hist[sb], e);
        }
    }
    // block total: warp shuffle in FP64, then one shared atomic per warp
    for (int o = 16; o > 0; o >>= 1) total += __shfl_down_sync(0xffffffffu, total, o);
    if (lane == 0) atomicAdd(&hist[nbins], total);
    __syncthreads();
    double* out = partials + (b * gridDim.x + blockIdx.x) * (long long)(nbins + 1);
    for (int i = threadIdx.x; i <= nbins; i += blockDim.x) out[i] = hist[i];
}

// One thread per (batch entry, bin): fixed-order sum over the block partials.
__global__ void energy_finalize_kernel(const double* __restrict__ partials, int blocks, int nbins, int batch,
                                       double* __restrict__ total, double* __restrict__ shells)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)batch * (nbins + 1)) return;
    const long long b = idx / (nbins + 1);
    const int bin = (int)(idx - b * (nbins + 1));
    const double* p = partials + b * blocks * (long long)(nbins + 1) + bin;
    double s = 0.0;
    for (int k = 0; k < blocks; ++k) s += p[(long long)k * (nbins + 1)];
    if (bin == nbins) {
        if (total) total[b] = s;
    } else if (shells) {
        shells[b * nbins + bin] = s;
    }
}

constexpr long long kMaxGridY = 65535;

}  // namespace

int energy_blocks_per_entry(long long rows)
{
    const long long want = (rows + 7) / 8;  // at least 8 rows per block
    return (int)(want < 256 ? (want < 1 ? 1 : want) : 256);
}

size_t energy_scratch_doubles(int batch, long long rows, int nbins)
{
    return (size_t)batch * energy_blocks_per_entry(rows) * (size_t)(nbins + 1);
}

cudaError_t launch_energy(const void* X, int n0, int n1, int n2, int batch, int nbins, double* scratch,
                          double* total, double* shells, cudaStream_t s)
{
    const long long rows = (long long)n0 * n1;
    const int blocks = energy_blocks_per_entry(rows);
    const size_t smem = (size_t)(nbins + 1) * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(energy_partials_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    // batch entries in launches of at most 65535 (the grid's y limit)
    for (long long b0 = 0; b0 < batch; b0 += kMaxGridY) {
        const unsigned nb = (unsigned)(batch - b0 < kMaxGridY ? batch - b0 : kMaxGridY);
        energy_partials_kernel<<<dim3(blocks, nb), 256, smem, s>>>(reinterpret_cast<const float2*>(X), n0, n1, n2,
                                                                   nbins, b0, scratch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const long long n = (long long)batch * (nbins + 1);
    energy_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(scratch, blocks, nbins, batch, total, shells);
    return cudaGetLastError();
}

}  // namespace fft3d

// Fused elementwise stage of the pseudo-spectral Navier-Stokes step (the
// solver of Sec. 1): divergence of the dealiased quadratic term, pressure
// projection, viscous term and the Heun update, one pass over the half
// spectrum per stage.  Each thread takes bins i, i + stride, ...; the bin's
// signed wavenumbers come from its flat index.
#include "launch_cache.h"
#include "ns.h"

namespace fft3d {

namespace {

__device__ __forceinline__ int signed_k(int j, int n) { return 2 * j < n ? j : j - n; }

template <int STAGE>
__global__ void __launch_bounds__(256) ns_stage_kernel(NsArgs a)
{
    const long long M = a.M;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += step) {
        const long long row = i / a.H;
        const int j2 = (int)(i - row * a.H);
        const int j1 = (int)(row % a.n1);
        const int j0 = (int)(row / a.n1);
        const int k0 = signed_k(j0, a.n0), k1 = signed_k(j1, a.n1), k2 = j2;
        const float2* src = (STAGE == 1) ? a.u : a.ustar;
        float2 u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = src[c * M + i];
        float2 r[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        // 2/3 rule: bins outside it do not change
        const bool keep = 3 * abs(k0) < a.n0 && 3 * abs(k1) < a.n1 && 3 * k2 < a.n2;
        if (keep) {
            float2 n[6];  // 00 01 02 11 12 22
#pragma unroll
            for (int q = 0; q < 6; ++q) n[q] = a.nhat[q * M + i];
            const float f0 = (float)k0, f1 = (float)k1, f2 = (float)k2;
            // a_l = sum_j k_j N_lj
            const float2 a0 = make_float2(f0 * n[0].x + f1 * n[1].x + f2 * n[2].x, f0 * n[0].y + f1 * n[1].y + f2 * n[2].y);
            const float2 a1 = make_float2(f0 * n[1].x + f1 * n[3].x + f2 * n[4].x, f0 * n[1].y + f1 * n[3].y + f2 * n[4].y);
            const float2 a2 = make_float2(f0 * n[2].x + f1 * n[4].x + f2 * n[5].x, f0 * n[2].y + f1 * n[4].y + f2 * n[5].y);
            const float kk = f0 * f0 + f1 * f1 + f2 * f2;
            const float inv = kk > 0.f ? 1.f / kk : 0.f;
            const float2 ka = make_float2((f0 * a0.x + f1 * a1.x + f2 * a2.x) * inv, (f0 * a0.y + f1 * a1.y + f2 * a2.y) * inv);
            const float2 av[3] = {a0, a1, a2};
            const float fk[3] = {f0, f1, f2};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // b = a - k (k.a)/|k|^2 (zero at k = 0); R = -i b - nu |k|^2 u
                const float2 b = kk > 0.f ? make_float2(av[c].x - fk[c] * ka.x, av[c].y - fk[c] * ka.y)
                                          : make_float2(0.f, 0.f);
                r[c] = make_float2(b.y - a.nu * kk * u[c].x, -b.x - a.nu * kk * u[c].y);
            }
        }
        if (STAGE == 1) {
            const float h = 0.5f * a.dt;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a.ustar[c * M + i] = make_float2(u[c].x + a.dt * r[c].x, u[c].y + a.dt * r[c].y);
                a.acc[c * M + i] = make_float2(u[c].x + h * r[c].x, u[c].y + h * r[c].y);
            }
        } else {
            const float h = 0.5f * a.dt;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 acc = a.acc[c * M + i];
                a.u[c * M + i] = make_float2(acc.x + h * r[c].x, acc.y + h * r[c].y);
            }
        }
    }
}

}  // namespace

cudaError_t launch_ns_stage(const NsArgs& a, int stage, cudaStream_t s)
{
    if (a.M <= 0) return cudaSuccess;
    static PerDevice sm_count;  // a few CTAs per SM, grid-stride over the bins
    int sms = 0;
    if (per_device(sm_count, &sms, [](int dev, int* v) {
            return cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev);
        }) != cudaSuccess)
        sms = 1;
    const long long blocks = 8ll * sms;
    long long need = (a.M + 255) / 256;
    const unsigned grid = (unsigned)(need < blocks ? need : blocks);
    if (stage == 1) ns_stage_kernel<1><<<grid, 256, 0, s>>>(a);
    else ns_stage_kernel<2><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fft3d

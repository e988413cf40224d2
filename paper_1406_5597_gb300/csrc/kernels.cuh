// Kernel templates of the transpose-free 3D r2c / c2r path.
//
//  * col_kernel: length-L c2c along a strided axis, IN PLACE.  Element
//    (b, j, c) of the volume sits at b*Bs + j*S + c; the c index is
//    contiguous.  For the n0 axis S = n1*(n2/2+1) and c runs over the flat
//    (k1, k2) plane, so a CTA that takes W adjacent c values reads W*8
//    contiguous bytes per n0 row: the strided n0 transform of Sec. 2.2 with
//    no transposed copy, coalesced because adjacent lanes take adjacent c.
//    The same kernel does the n1 axis (S = n2/2+1) when planes are processed
//    in separate passes.
//  * row_r2c_kernel: the n2-axis real transform of Sec. 2.1 step 1, as a
//    length-n2/2 complex FFT of the packed row z[m] = x[2m] + i x[2m+1]
//    followed by the Hermitian unpack
//        X[k] = (Z[k] + conj Z[L-k])/2 - (i/2) W^k (Z[k] - conj Z[L-k]),
//        W = exp(-2 pi i / n2), Z[L] = Z[0], k = 0..L (L = n2/2)
//    (the standard real-FFT packing; e.g. Sorensen et al., IEEE TASSP 1987).
//  * row_c2r_kernel: its inverse: drop Im of X[0] and X[L], pack
//        Z[k] = (X[k] + conj X[L-k]) + i W^{-k} (X[k] - conj X[L-k]),  k < L,
//    inverse length-L complex FFT, and the result read as float pairs is the
//    real row (unnormalised: twice the half-length scale, i.e. n2 x).
#pragma once
#include <cstdint>

#include "args.h"
#include "stockham.cuh"

namespace fft3d {

template <int L, int E, int DIR, int MAXT>
__global__ void __launch_bounds__(MAXT) col_kernel(ColArgs a, int W)
{
    extern __shared__ float2 sm[];
    constexpr int T = L / E;
    const int c = threadIdx.x;
    const int t = threadIdx.y;
    const long long ctiles = (a.C + W - 1) / W;
    const long long b = blockIdx.x / ctiles;
    const long long c0 = (blockIdx.x - b * ctiles) * W;
    const bool active = (c0 + c) < a.C;
    float2* base = a.data + b * a.Bs + c0 + c;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = active ? base[(long long)(t + T * m) * a.S] : make_float2(0.f, 0.f);
    ColExchange ex{sm, W, c};
    fft_group<L, E, DIR>(v, t, a.tw, ex);
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) base[(long long)(t + T * m) * a.S] = cscale(v[m], a.scale);
    }
}

// Row kernels: block = (T, ROWS) threads; group y handles one row.  The rows
// of a block are contiguous in memory on both sides, so loads and stores are
// linear copies between global memory and the padded shared rows.
template <int L>
struct RowLayout {
    static constexpr int H = L + 1;
    static constexpr int stride = (L + 1) + ((L + 1) >> 4) + 1;  // padded slots per row
};

template <int L, int E, int ROWS>
__global__ void __launch_bounds__((L / E) * ROWS) row_r2c_kernel(RowArgs a)
{
    extern __shared__ float2 sm[];
    constexpr int T = L / E;
    constexpr int H = L + 1;
    constexpr int RS = RowLayout<L>::stride;
    constexpr bool WS = (T <= 32);
    using Ex = RowExchange<WS>;
    const int t = threadIdx.x, r = threadIdx.y;
    const int tid = r * T + t;
    const long long row0 = (long long)blockIdx.x * ROWS;
    const int nrows = (int)min((long long)ROWS, a.rows - row0);
    const float2* in = reinterpret_cast<const float2*>(a.in) + row0 * L;  // packed z of each row
    float2* out = reinterpret_cast<float2*>(a.out) + row0 * H;

    for (int i = tid; i < ROWS * L; i += T * ROWS) {
        const int rr = i / L, p = i - rr * L;
        sm[rr * RS + Ex::pad(p)] = (rr < nrows) ? in[i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    Ex ex{sm + r * RS};
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = ex.get(t + T * m);
    ex.sync();
    fft_group<L, E, -1>(v, t, a.tw, ex);
    // Z to shared, then the Hermitian unpack.
#pragma unroll
    for (int m = 0; m < E; ++m) ex.put(t + T * m, v[m]);
    ex.sync();
    float2 x[E];
    float2 xl = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + T * m;
        const float2 zk = ex.get(k);
        const float2 zc = cconj(ex.get(k == 0 ? 0 : L - k));
        const float2 s = cadd(zk, zc);
        const float2 d = csub(zk, zc);
        // -(i/2) W^k d
        const float2 wd = cmul(d, __ldg(&a.twpack[k]));
        x[m] = make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
    }
    if (t == 0) {
        const float2 z0 = ex.get(0);
        xl = make_float2(z0.x - z0.y, 0.f);
    }
    ex.sync();
#pragma unroll
    for (int m = 0; m < E; ++m) ex.put(t + T * m, x[m]);
    if (t == 0) ex.put(L, xl);
    __syncthreads();
    for (int i = tid; i < nrows * H; i += T * ROWS) {
        const int rr = i / H, p = i - rr * H;
        out[i] = sm[rr * RS + Ex::pad(p)];
    }
}

template <int L, int E, int ROWS>
__global__ void __launch_bounds__((L / E) * ROWS) row_c2r_kernel(RowArgs a)
{
    extern __shared__ float2 sm[];
    constexpr int T = L / E;
    constexpr int H = L + 1;
    constexpr int RS = RowLayout<L>::stride;
    constexpr bool WS = (T <= 32);
    using Ex = RowExchange<WS>;
    const int t = threadIdx.x, r = threadIdx.y;
    const int tid = r * T + t;
    const long long row0 = (long long)blockIdx.x * ROWS;
    const int nrows = (int)min((long long)ROWS, a.rows - row0);
    const float2* in = reinterpret_cast<const float2*>(a.in) + row0 * H;
    float2* out = reinterpret_cast<float2*>(a.out) + row0 * L;  // real row as float pairs

    for (int i = tid; i < ROWS * H; i += T * ROWS) {
        const int rr = i / H, p = i - rr * H;
        sm[rr * RS + Ex::pad(p)] = (rr < nrows) ? in[i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    Ex ex{sm + r * RS};
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + T * m;
        float2 xk = ex.get(k);
        float2 xc = cconj(ex.get(L - k));
        if (k == 0) {  // Im of the DC and Nyquist bins is not part of a real row's spectrum
            xk.y = 0.f;
            xc.y = 0.f;
        }
        const float2 s = cadd(xk, xc);
        const float2 d = csub(xk, xc);
        // i W^{-k} d, W^{-k} = conj(twpack[k])
        const float2 wd = cmulc(d, __ldg(&a.twpack[k]));
        v[m] = make_float2(s.x - wd.y, s.y + wd.x);
    }
    ex.sync();
    fft_group<L, E, +1>(v, t, a.tw, ex);
#pragma unroll
    for (int m = 0; m < E; ++m) ex.put(t + T * m, v[m]);
    __syncthreads();
    for (int i = tid; i < nrows * L; i += T * ROWS) {
        const int rr = i / L, p = i - rr * L;
        out[i] = sm[rr * RS + Ex::pad(p)];
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers (one instantiation per supported length).
// ---------------------------------------------------------------------------
struct ColShape {
    int W;        // columns per CTA
    int threads;  // W * T
    size_t smem;  // dynamic shared bytes
};

template <int L, int E, int W>
inline ColShape col_shape()
{
    return ColShape{W, W * (L / E), (size_t)L * W * sizeof(float2)};
}

template <int L, int E, int W, int DIR>
inline cudaError_t launch_col(const ColArgs& a, cudaStream_t s)
{
    constexpr int T = L / E;
    constexpr int MAXT = W * T;
    static_assert(MAXT <= 1024, "too many threads");
    const size_t smem = (size_t)L * W * sizeof(float2);
    auto k = col_kernel<L, E, DIR, MAXT>;
    static bool attr_set = false;  // one attribute call per instantiation (per process)
    if (smem > 48 * 1024 && !attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const long long tiles = a.nb * ((a.C + W - 1) / W);
    if (tiles <= 0) return cudaSuccess;
    k<<<(unsigned)tiles, dim3(W, T), smem, s>>>(a, W);
    return cudaGetLastError();
}

template <int L, int E, int ROWS>
inline size_t row_smem()
{
    return (size_t)ROWS * RowLayout<L>::stride * sizeof(float2);
}

template <int L, int E, int ROWS, int DIR>
inline cudaError_t launch_row(const RowArgs& a, cudaStream_t s)
{
    constexpr int T = L / E;
    const size_t smem = row_smem<L, E, ROWS>();
    const long long blocks = (a.rows + ROWS - 1) / ROWS;
    if (blocks <= 0) return cudaSuccess;
    if constexpr (DIR < 0) {
        auto k = row_r2c_kernel<L, E, ROWS>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<(unsigned)blocks, dim3(T, ROWS), smem, s>>>(a);
    } else {
        auto k = row_c2r_kernel<L, E, ROWS>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<(unsigned)blocks, dim3(T, ROWS), smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace fft3d

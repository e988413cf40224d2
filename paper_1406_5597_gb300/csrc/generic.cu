// Runtime-length kernels: any transform length up to 4096, for the axis
// lengths that have no compile-time specialisation.  A CTA stages G lines in
// shared memory (two buffers) and runs the Stockham stages of a runtime radix
// list, one butterfly per thread iteration; a length with a prime factor above
// 7 runs Bluestein's chirp-z form around two such transforms of a power-of-two
// length M.  Same mathematics as the specialised kernels (see stockham.cuh and
// kernels.cuh); slower, but length-agnostic.
#include "args.h"
#include "radix.cuh"

namespace fft3d {

namespace {

// Index of position p of line g in a buffer of G interleaved lines.
__device__ __forceinline__ int gi(int p, int g, int G) { return p * G + g; }

// One Stockham stage of radix R (compile time, so the butterfly's values stay
// in registers) over the G lines of src, Ns = product of the earlier radices.
template <int DIR, int R>
__device__ __forceinline__ void generic_stage(int L, int Ns, const float2* src, float2* dst, int G,
                                              const float2* __restrict__ tw)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    const int nbf = L / R;
    const int step = L / (Ns * R);
    for (int i = tid; i < nbf * G; i += nthr) {
        const int line = i % G;
        const int j = i / G;
        const int jm = j % Ns;
        float2 a[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            float2 x = src[gi(j + k * nbf, line, G)];
            if (k > 0 && Ns > 1) x = twiddle<DIR>(x, __ldg(&tw[k * jm * step]));
            a[k] = x;
        }
        Dft<R, DIR>::run(a);
        const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int k = 0; k < R; ++k) dst[gi(base + k * Ns, line, G)] = a[k];
    }
}

// Runs the nst stages of radix[] (a length-L transform) on the G lines in
// b0; returns the buffer that holds the result (natural order).
template <int DIR>
__device__ float2* generic_stages(int L, int nst, const int* radix, float2* b0, float2* b1, int G,
                                  const float2* __restrict__ tw)
{
    float2* src = b0;
    float2* dst = b1;
    int Ns = 1;
    for (int s = 0; s < nst; ++s) {
        const int R = radix[s];
        switch (R) {
        case 2: generic_stage<DIR, 2>(L, Ns, src, dst, G, tw); break;
        case 3: generic_stage<DIR, 3>(L, Ns, src, dst, G, tw); break;
        case 4: generic_stage<DIR, 4>(L, Ns, src, dst, G, tw); break;
        case 5: generic_stage<DIR, 5>(L, Ns, src, dst, G, tw); break;
        case 7: generic_stage<DIR, 7>(L, Ns, src, dst, G, tw); break;
        default: generic_stage<DIR, 8>(L, Ns, src, dst, G, tw); break;
        }
        __syncthreads();
        float2* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// The length-g.L transform of the G lines in b0 (positions 0 .. L-1; the
// buffers hold gen_line_slots(g) positions per line); returns the buffer that
// holds the result in positions 0 .. L-1.  Bluestein (g.M > 0), forward:
// a = x c zero-padded to M, y = IFFT_M(FFT_M(a) bhat) (bhat carries 1/M),
// X[k] = c[k] y[k].  The inverse is the conjugate of the forward transform of
// the conjugate, i.e. the same steps with conj(c) and conj(bhat) (b is even, so
// its transform is even and conjugating b conjugates bhat).
template <int DIR>
__device__ float2* generic_line(const GenPlan& g, float2* b0, float2* b1, int G, const float2* __restrict__ tw)
{
    if (g.M == 0) return generic_stages<DIR>(g.L, g.nst, g.radix, b0, b1, G, tw);
    const int L = g.L, M = g.M;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    for (int i = tid; i < M * G; i += nthr) {
        const int n = i / G;
        float2 v = make_float2(0.f, 0.f);
        if (n < L) {
            const float2 c = __ldg(&g.chirp[n]);
            v = DIR < 0 ? cmul(b0[i], c) : cmulc(b0[i], c);
        }
        b0[i] = v;
    }
    __syncthreads();
    float2* A = generic_stages<-1>(M, g.mst, g.mradix, b0, b1, G, g.twm);
    for (int i = tid; i < M * G; i += nthr) {
        const float2 w = __ldg(&g.bhat[i / G]);
        A[i] = DIR < 0 ? cmul(A[i], w) : cmulc(A[i], w);
    }
    __syncthreads();
    float2* y = generic_stages<+1>(M, g.mst, g.mradix, A, A == b0 ? b1 : b0, G, g.twm);
    for (int i = tid; i < L * G; i += nthr) {
        const float2 c = __ldg(&g.chirp[i / G]);
        y[i] = DIR < 0 ? cmul(y[i], c) : cmulc(y[i], c);
    }
    __syncthreads();
    return y;
}

template <int DIR>
__global__ void generic_col_kernel(ColArgs a, GenPlan g, int G)
{
    extern __shared__ float2 sm[];
    const int L = g.L;
    float2* b0 = sm;
    float2* b1 = sm + (size_t)gen_line_slots(g) * G;
    const long long ctiles = (a.C + G - 1) / G;
    const long long b = blockIdx.x / ctiles;
    const long long c0 = (blockIdx.x - b * ctiles) * G;
    float2* base = a.data + b * a.Bs + c0;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    for (int i = tid; i < L * G; i += nthr) {
        const int line = i % G, p = i / G;
        b0[gi(p, line, G)] = (c0 + line < a.C) ? base[(long long)p * a.S + line] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = generic_line<DIR>(g, b0, b1, G, a.tw);
    float2* out = (a.dst ? a.dst : a.data) + b * a.Bs + c0;
    for (int i = tid; i < L * G; i += nthr) {
        const int line = i % G, p = i / G;
        if (c0 + line < a.C)
            out[(long long)p * a.S + line] = cscale(res[gi(p, line, G)], col_out_factor(p, L, a.scale, a.mask23));
    }
}

// Rows: G contiguous rows per CTA.  DIR = -1: r2c (packed row in, H bins
// out); DIR = +1: c2r (H bins in, packed real row out).  Buffers hold L+1
// positions per line so that the unpacked H = L+1 bins fit.
template <int DIR>
__global__ void generic_row_kernel(RowArgs a, GenPlan g, int G)
{
    extern __shared__ float2 sm[];
    const int L = g.L, H = L + 1;
    float2* b0 = sm;
    float2* b1 = sm + (size_t)gen_line_slots(g) * G;
    const long long row0 = (long long)blockIdx.x * G;
    const int nrows = (int)min((long long)G, a.rows - row0);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    if (DIR < 0) {
        const float2* in = reinterpret_cast<const float2*>(a.in) + row0 * a.rs;
        for (int i = tid; i < L * G; i += nthr) {
            const int line = i / L, p = i % L;
            b0[gi(p, line, G)] = line < nrows ? in[line * a.rs + p] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2* Z = generic_line<-1>(g, b0, b1, G, a.tw);
        float2* X = (Z == b0) ? b1 : b0;
        for (int i = tid; i < H * G; i += nthr) {
            const int line = i % G, k = i / G;
            float2 r;
            if (k == L) {
                const float2 z0 = Z[gi(0, line, G)];
                r = make_float2(z0.x - z0.y, 0.f);
            } else {
                const float2 zk = Z[gi(k, line, G)];
                const float2 zc = cconj(Z[gi(k == 0 ? 0 : L - k, line, G)]);
                const float2 s = cadd(zk, zc), d = csub(zk, zc);
                const float2 wd = cmul(d, __ldg(&a.twpack[k]));
                r = make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
            }
            X[gi(k, line, G)] = r;
        }
        __syncthreads();
        float2* out = reinterpret_cast<float2*>(a.out) + row0 * H;
        for (int i = tid; i < H * nrows; i += nthr) {
            const int line = i / H, k = i % H;
            out[i] = X[gi(k, line, G)];
        }
    } else {
        const float2* in = reinterpret_cast<const float2*>(a.in) + row0 * H;
        for (int i = tid; i < H * G; i += nthr) {
            const int line = i / H, k = i % H;
            b1[gi(k, line, G)] = line < nrows ? in[i] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int i = tid; i < L * G; i += nthr) {
            const int line = i % G, k = i / G;
            float2 xk = b1[gi(k, line, G)];
            float2 xc = cconj(b1[gi(L - k, line, G)]);
            if (k == 0) {
                xk.y = 0.f;
                xc.y = 0.f;
            }
            const float2 s = cadd(xk, xc), d = csub(xk, xc);
            const float2 wd = cmulc(d, __ldg(&a.twpack[k]));
            b0[gi(k, line, G)] = make_float2(s.x - wd.y, s.y + wd.x);
        }
        __syncthreads();
        float2* z = generic_line<+1>(g, b0, b1, G, a.tw);
        float2* out = reinterpret_cast<float2*>(a.out) + row0 * a.rs;
        for (int i = tid; i < L * nrows; i += nthr) {
            const int line = i / L, p = i % L;
            out[line * a.rs + p] = z[gi(p, line, G)];
        }
    }
}

// Rows of odd length n2 = g.L (no half-length packing): the r2c is the
// length-n2 complex FFT of the real row (imaginary parts zero), bins
// 0 .. (n2-1)/2 kept; the c2r builds the Hermitian extension of the
// (n2+1)/2 bins (Im of the DC bin dropped, no Nyquist bin) and keeps the real
// part of its length-n2 inverse FFT.  Real rows at a stride of a.rs floats.
template <int DIR>
__global__ void generic_row_odd_kernel(RowArgs a, GenPlan g, int G)
{
    extern __shared__ float2 sm[];
    const int L = g.L, H = L / 2 + 1;
    float2* b0 = sm;
    float2* b1 = sm + (size_t)gen_line_slots(g) * G;
    const long long row0 = (long long)blockIdx.x * G;
    const int nrows = (int)min((long long)G, a.rows - row0);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    if (DIR < 0) {
        const float* in = reinterpret_cast<const float*>(a.in) + row0 * a.rs;
        for (int i = tid; i < L * G; i += nthr) {
            const int line = i / L, p = i % L;
            b0[gi(p, line, G)] = make_float2(line < nrows ? in[line * a.rs + p] : 0.f, 0.f);
        }
        __syncthreads();
        float2* X = generic_line<-1>(g, b0, b1, G, a.tw);
        float2* out = reinterpret_cast<float2*>(a.out) + row0 * H;
        for (int i = tid; i < H * nrows; i += nthr) {
            const int line = i / H, k = i % H;
            out[i] = X[gi(k, line, G)];
        }
    } else {
        const float2* in = reinterpret_cast<const float2*>(a.in) + row0 * H;
        for (int i = tid; i < L * G; i += nthr) {
            const int line = i / L, k = i % L;
            float2 v = make_float2(0.f, 0.f);
            if (line < nrows) {
                if (k < H) {
                    v = in[line * H + k];
                    if (k == 0) v.y = 0.f;
                } else {
                    v = cconj(in[line * H + (L - k)]);
                }
            }
            b0[gi(k, line, G)] = v;
        }
        __syncthreads();
        float2* y = generic_line<+1>(g, b0, b1, G, a.tw);
        float* out = reinterpret_cast<float*>(a.out) + row0 * a.rs;
        for (int i = tid; i < L * nrows; i += nthr) {
            const int line = i / L, p = i % L;
            out[line * a.rs + p] = y[gi(p, line, G)].x;
        }
    }
}

// Lines per CTA: both buffers within 64 KB where a line allows it (a
// Bluestein line of M = 8192 points takes 128 KB on its own).
int lines_per_cta(const GenPlan& g)
{
    const int cap = 64 * 1024;
    int G = cap / (2 * gen_line_slots(g) * (int)sizeof(float2));
    if (G > 32) G = 32;
    if (G < 1) G = 1;
    return G;
}

}  // namespace

cudaError_t generic_col(const ColArgs& a, const GenPlan& g, int dir, cudaStream_t s)
{
    const int G = lines_per_cta(g);
    const size_t smem = 2 * (size_t)gen_line_slots(g) * G * sizeof(float2);
    const long long tiles = a.nb * ((a.C + G - 1) / G);
    if (tiles <= 0) return cudaSuccess;
    dim3 block(G, 256 / G > 0 ? 256 / G : 1);
    if (dir < 0) {
        cudaFuncSetAttribute(generic_col_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        generic_col_kernel<-1><<<(unsigned)tiles, block, smem, s>>>(a, g, G);
    } else {
        cudaFuncSetAttribute(generic_col_kernel<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        generic_col_kernel<+1><<<(unsigned)tiles, block, smem, s>>>(a, g, G);
    }
    return cudaGetLastError();
}

cudaError_t generic_row_odd(const RowArgs& a, const GenPlan& g, int dir, cudaStream_t s)
{
    const int G = lines_per_cta(g);
    const size_t smem = 2 * (size_t)gen_line_slots(g) * G * sizeof(float2);
    const long long blocks = (a.rows + G - 1) / G;
    if (blocks <= 0) return cudaSuccess;
    dim3 block(G, 256 / G > 0 ? 256 / G : 1);
    if (dir < 0) {
        cudaFuncSetAttribute(generic_row_odd_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        generic_row_odd_kernel<-1><<<(unsigned)blocks, block, smem, s>>>(a, g, G);
    } else {
        cudaFuncSetAttribute(generic_row_odd_kernel<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        generic_row_odd_kernel<+1><<<(unsigned)blocks, block, smem, s>>>(a, g, G);
    }
    return cudaGetLastError();
}

cudaError_t generic_row(const RowArgs& a, const GenPlan& g, int dir, cudaStream_t s)
{
    const int G = lines_per_cta(g);
    const size_t smem = 2 * (size_t)gen_line_slots(g) * G * sizeof(float2);
    const long long blocks = (a.rows + G - 1) / G;
    if (blocks <= 0) return cudaSuccess;
    dim3 block(G, 256 / G > 0 ? 256 / G : 1);
    if (dir < 0) {
        cudaFuncSetAttribute(generic_row_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        generic_row_kernel<-1><<<(unsigned)blocks, block, smem, s>>>(a, g, G);
    } else {
        cudaFuncSetAttribute(generic_row_kernel<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        generic_row_kernel<+1><<<(unsigned)blocks, block, smem, s>>>(a, g, G);
    }
    return cudaGetLastError();
}

}  // namespace fft3d

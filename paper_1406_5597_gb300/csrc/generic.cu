// Runtime-length kernels: any transform length up to 4096, for the axis
// lengths that have no compile-time specialisation, and the whole FP64 path.
// A CTA stages G lines in shared memory (two buffers) and runs the Stockham
// stages of a runtime radix list, one butterfly per thread iteration; a length
// with a prime factor above 7 runs Bluestein's chirp-z form around two such
// transforms of a power-of-two length M.  Same mathematics as the specialised
// kernels (see stockham.cuh and kernels.cuh); slower, but length-agnostic.
// Every kernel is a template over the complex type: float2 (the FP32 path,
// codelets of radix.cuh) or double2 (FP64, the codelets below).
#include <type_traits>

#include "args.h"
#include "radix.cuh"

namespace fft3d {

// double2 arithmetic, overloads of the float2 helpers of radix.cuh (same
// namespace, so that one unqualified call serves both types)
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 w)
{
    return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
// a * conj(w)
__device__ __forceinline__ double2 cmulc(double2 a, double2 w)
{
    return make_double2(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y));
}
template <int DIR>
__device__ __forceinline__ double2 twiddle(double2 a, double2 w_fwd)
{
    return DIR < 0 ? cmul(a, w_fwd) : cmulc(a, w_fwd);
}
// a * (DIR * i)
template <int DIR>
__device__ __forceinline__ double2 mul_i(double2 a)
{
    return DIR > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

namespace {

// ---------------------------------------------------------------------------
// double2 codelets
// ---------------------------------------------------------------------------
// cos and sin of 2 pi m / R for the odd radices, m in [1, (R-1)/2]
__device__ __forceinline__ constexpr double cos_r(int R, int m)
{
    return R == 3 ? -0.5
         : R == 5 ? (m == 1 ? 0.309016994374947424102293417183 : -0.809016994374947424102293417183)
         : (m == 1 ? 0.623489801858733530525004884004
            : m == 2 ? -0.222520933956314404288902564497 : -0.900968867902419126236102319507);
}
__device__ __forceinline__ constexpr double sin_r(int R, int m)
{
    return R == 3 ? 0.866025403784438646763723170753
         : R == 5 ? (m == 1 ? 0.951056516295153572116439333379 : 0.587785252292473129168705954639)
         : (m == 1 ? 0.781831482468029808708444526674
            : m == 2 ? 0.974927912181823607018131682994 : 0.433883739117558120475768332848);
}

// R-point DFT of a[0..R-1] in natural order, X[q] = sum_j a[j] exp(DIR 2 pi i j q / R).
template <int R, int DIR>
struct DftD {
    // odd R: pair j with R - j, s = a_j + a_{R-j}, d = a_j - a_{R-j};
    // X[q] = a_0 + sum_j (s cos t + DIR i d sin t), t = 2 pi j q / R
    __device__ __forceinline__ static void run(double2* a)
    {
        static_assert(R == 3 || R == 5 || R == 7, "odd radices 3, 5, 7");
        constexpr int Hh = (R - 1) / 2;
        double2 s[Hh], d[Hh];
#pragma unroll
        for (int j = 1; j <= Hh; ++j) {
            s[j - 1] = cadd(a[j], a[R - j]);
            d[j - 1] = csub(a[j], a[R - j]);
        }
        double2 y[R];
        y[0] = a[0];
#pragma unroll
        for (int j = 0; j < Hh; ++j) y[0] = cadd(y[0], s[j]);
#pragma unroll
        for (int q = 1; q < R; ++q) {
            double2 acc = a[0];
#pragma unroll
            for (int j = 1; j <= Hh; ++j) {
                const int m = (j * q) % R;
                const double c = cos_r(R, m <= Hh ? m : R - m);
                const double sn = (m <= Hh ? 1.0 : -1.0) * sin_r(R, m <= Hh ? m : R - m);
                acc.x = fma(s[j - 1].x, c, fma(-DIR * sn, d[j - 1].y, acc.x));
                acc.y = fma(s[j - 1].y, c, fma(DIR * sn, d[j - 1].x, acc.y));
            }
            y[q] = acc;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = y[q];
    }
};
template <int DIR>
struct DftD<2, DIR> {
    __device__ __forceinline__ static void run(double2* a)
    {
        const double2 t = a[1];
        a[1] = csub(a[0], t);
        a[0] = cadd(a[0], t);
    }
};
template <int DIR>
struct DftD<4, DIR> {
    __device__ __forceinline__ static void run(double2* a)
    {
        const double2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        const double2 s13 = cadd(a[1], a[3]), d13 = mul_i<DIR>(csub(a[1], a[3]));
        a[0] = cadd(s02, s13);
        a[2] = csub(s02, s13);
        a[1] = cadd(d02, d13);
        a[3] = csub(d02, d13);
    }
};
// 8 = 2 x 4: even and odd 4-point halves, combined with W_8^k = exp(DIR i pi k / 4)
template <int DIR>
struct DftD<8, DIR> {
    __device__ __forceinline__ static void run(double2* a)
    {
        constexpr double h = 0.707106781186547524400844362105;  // sqrt(2) / 2
        double2 e[4] = {a[0], a[2], a[4], a[6]}, o[4] = {a[1], a[3], a[5], a[7]};
        DftD<4, DIR>::run(e);
        DftD<4, DIR>::run(o);
        o[1] = cmul(o[1], make_double2(h, DIR * h));
        o[2] = mul_i<DIR>(o[2]);
        o[3] = cmul(o[3], make_double2(-h, DIR * h));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = cadd(e[k], o[k]);
            a[k + 4] = csub(e[k], o[k]);
        }
    }
};

template <typename T, int R, int DIR>
__device__ __forceinline__ void dft(T* a)
{
    if constexpr (std::is_same<T, float2>::value)
        Dft<R, DIR>::run(a);
    else
        DftD<R, DIR>::run(a);
}

// ---------------------------------------------------------------------------
// Stages and lines
// ---------------------------------------------------------------------------

// Index of position p of line g in a buffer of G interleaved lines.
__device__ __forceinline__ int gi(int p, int g, int G) { return p * G + g; }

// One Stockham stage of radix R (compile time, so the butterfly's values stay
// in registers) over the G lines of src, Ns = product of the earlier radices.
template <typename T, int DIR, int R>
__device__ __forceinline__ void generic_stage(int L, int Ns, const T* src, T* dst, int G, const T* __restrict__ tw)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    const int nbf = L / R;
    const int step = L / (Ns * R);
    for (int i = tid; i < nbf * G; i += nthr) {
        const int line = i % G;
        const int j = i / G;
        const int jm = j % Ns;
        T a[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            T x = src[gi(j + k * nbf, line, G)];
            if (k > 0 && Ns > 1) x = twiddle<DIR>(x, __ldg(&tw[k * jm * step]));
            a[k] = x;
        }
        dft<T, R, DIR>(a);
        const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int k = 0; k < R; ++k) dst[gi(base + k * Ns, line, G)] = a[k];
    }
}

// Runs the nst stages of radix[] (a length-L transform) on the G lines in
// b0; returns the buffer that holds the result (natural order).
template <typename T, int DIR>
__device__ T* generic_stages(int L, int nst, const int* radix, T* b0, T* b1, int G, const T* __restrict__ tw)
{
    T* src = b0;
    T* dst = b1;
    int Ns = 1;
    for (int s = 0; s < nst; ++s) {
        const int R = radix[s];
        switch (R) {
        case 2: generic_stage<T, DIR, 2>(L, Ns, src, dst, G, tw); break;
        case 3: generic_stage<T, DIR, 3>(L, Ns, src, dst, G, tw); break;
        case 4: generic_stage<T, DIR, 4>(L, Ns, src, dst, G, tw); break;
        case 5: generic_stage<T, DIR, 5>(L, Ns, src, dst, G, tw); break;
        case 7: generic_stage<T, DIR, 7>(L, Ns, src, dst, G, tw); break;
        default: generic_stage<T, DIR, 8>(L, Ns, src, dst, G, tw); break;
        }
        __syncthreads();
        T* t = src;
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
template <typename T, int DIR>
__device__ T* generic_line(const GenPlanT<T>& g, T* b0, T* b1, int G, const T* __restrict__ tw)
{
    if (g.M == 0) return generic_stages<T, DIR>(g.L, g.nst, g.radix, b0, b1, G, tw);
    const int L = g.L, M = g.M;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    for (int i = tid; i < M * G; i += nthr) {
        const int n = i / G;
        T v{};
        if (n < L) {
            const T c = __ldg(&g.chirp[n]);
            v = DIR < 0 ? cmul(b0[i], c) : cmulc(b0[i], c);
        }
        b0[i] = v;
    }
    __syncthreads();
    T* A = generic_stages<T, -1>(M, g.mst, g.mradix, b0, b1, G, g.twm);
    for (int i = tid; i < M * G; i += nthr) {
        const T w = __ldg(&g.bhat[i / G]);
        A[i] = DIR < 0 ? cmul(A[i], w) : cmulc(A[i], w);
    }
    __syncthreads();
    T* y = generic_stages<T, +1>(M, g.mst, g.mradix, A, A == b0 ? b1 : b0, G, g.twm);
    for (int i = tid; i < L * G; i += nthr) {
        const T c = __ldg(&g.chirp[i / G]);
        y[i] = DIR < 0 ? cmul(y[i], c) : cmulc(y[i], c);
    }
    __syncthreads();
    return y;
}

// ---------------------------------------------------------------------------
// Kernels (A = ColArgs / RowArgs for float2, ColArgs64 / RowArgs64 for double2)
// ---------------------------------------------------------------------------

// Columns: G adjacent columns (contiguous in memory) of one batch entry per CTA.
template <class A, typename T, int DIR>
__global__ void generic_col_kernel(A a, GenPlanT<T> g, int G)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int L = g.L;
    T* b0 = sm;
    T* b1 = sm + (size_t)gen_line_slots(g) * G;
    const long long ctiles = (a.C + G - 1) / G;
    const long long b = blockIdx.x / ctiles;
    const long long c0 = (blockIdx.x - b * ctiles) * G;
    T* base = a.data + b * a.Bs + c0;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    for (int i = tid; i < L * G; i += nthr) {
        const int line = i % G, p = i / G;
        b0[gi(p, line, G)] = (c0 + line < a.C) ? base[(long long)p * a.S + line] : T{};
    }
    __syncthreads();
    T* res = generic_line<T, DIR>(g, b0, b1, G, a.tw);
    T* out = (a.dst ? a.dst : a.data) + b * a.Bs + c0;
    for (int i = tid; i < L * G; i += nthr) {
        const int line = i % G, p = i / G;
        if (c0 + line < a.C) {
            if constexpr (std::is_same<T, float2>::value)
                out[(long long)p * a.S + line] =
                    cscale(res[gi(p, line, G)], col_out_factor(p, L, a.scale, a.mask23));
            else
                out[(long long)p * a.S + line] = res[gi(p, line, G)];
        }
    }
}

// Rows: G contiguous rows per CTA.  DIR = -1: r2c (packed row in, H bins
// out); DIR = +1: c2r (H bins in, packed real row out).  Buffers hold L+1
// positions per line so that the unpacked H = L+1 bins fit.
template <class A, typename T, int DIR>
__global__ void generic_row_kernel(A a, GenPlanT<T> g, int G)
{
    using S = decltype(T{}.x);
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int L = g.L, H = L + 1;
    T* b0 = sm;
    T* b1 = sm + (size_t)gen_line_slots(g) * G;
    const long long row0 = (long long)blockIdx.x * G;
    const int nrows = (int)min((long long)G, a.rows - row0);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    if (DIR < 0) {
        const T* in = reinterpret_cast<const T*>(a.in) + row0 * a.rs;
        for (int i = tid; i < L * G; i += nthr) {
            const int line = i / L, p = i % L;
            b0[gi(p, line, G)] = line < nrows ? in[line * a.rs + p] : T{};
        }
        __syncthreads();
        T* Z = generic_line<T, -1>(g, b0, b1, G, a.tw);
        T* X = (Z == b0) ? b1 : b0;
        for (int i = tid; i < H * G; i += nthr) {
            const int line = i % G, k = i / G;
            T r;
            if (k == L) {
                const T z0 = Z[gi(0, line, G)];
                r.x = z0.x - z0.y;
                r.y = S(0);
            } else {
                const T zk = Z[gi(k, line, G)];
                const T zc = cconj(Z[gi(k == 0 ? 0 : L - k, line, G)]);
                const T s = cadd(zk, zc), d = csub(zk, zc);
                const T wd = cmul(d, __ldg(&a.twpack[k]));
                r.x = S(0.5) * (s.x + wd.y);
                r.y = S(0.5) * (s.y - wd.x);
            }
            X[gi(k, line, G)] = r;
        }
        __syncthreads();
        T* out = reinterpret_cast<T*>(a.out) + row0 * H;
        for (int i = tid; i < H * nrows; i += nthr) {
            const int line = i / H, k = i % H;
            out[i] = X[gi(k, line, G)];
        }
    } else {
        const T* in = reinterpret_cast<const T*>(a.in) + row0 * H;
        for (int i = tid; i < H * G; i += nthr) {
            const int line = i / H, k = i % H;
            b1[gi(k, line, G)] = line < nrows ? in[i] : T{};
        }
        __syncthreads();
        for (int i = tid; i < L * G; i += nthr) {
            const int line = i % G, k = i / G;
            T xk = b1[gi(k, line, G)];
            T xc = cconj(b1[gi(L - k, line, G)]);
            if (k == 0) {
                xk.y = S(0);
                xc.y = S(0);
            }
            const T s = cadd(xk, xc), d = csub(xk, xc);
            const T wd = cmulc(d, __ldg(&a.twpack[k]));
            T r;
            r.x = s.x - wd.y;
            r.y = s.y + wd.x;
            b0[gi(k, line, G)] = r;
        }
        __syncthreads();
        T* z = generic_line<T, +1>(g, b0, b1, G, a.tw);
        T* out = reinterpret_cast<T*>(a.out) + row0 * a.rs;
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
// part of its length-n2 inverse FFT.  Real rows at a stride of a.rs scalars.
template <class A, typename T, int DIR>
__global__ void generic_row_odd_kernel(A a, GenPlanT<T> g, int G)
{
    using S = decltype(T{}.x);
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int L = g.L, H = L / 2 + 1;
    T* b0 = sm;
    T* b1 = sm + (size_t)gen_line_slots(g) * G;
    const long long row0 = (long long)blockIdx.x * G;
    const int nrows = (int)min((long long)G, a.rows - row0);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    if (DIR < 0) {
        const S* in = reinterpret_cast<const S*>(a.in) + row0 * a.rs;
        for (int i = tid; i < L * G; i += nthr) {
            const int line = i / L, p = i % L;
            T v{};
            if (line < nrows) v.x = in[line * a.rs + p];
            b0[gi(p, line, G)] = v;
        }
        __syncthreads();
        T* X = generic_line<T, -1>(g, b0, b1, G, a.tw);
        T* out = reinterpret_cast<T*>(a.out) + row0 * H;
        for (int i = tid; i < H * nrows; i += nthr) {
            const int line = i / H, k = i % H;
            out[i] = X[gi(k, line, G)];
        }
    } else {
        const T* in = reinterpret_cast<const T*>(a.in) + row0 * H;
        for (int i = tid; i < L * G; i += nthr) {
            const int line = i / L, k = i % L;
            T v{};
            if (line < nrows) {
                if (k < H) {
                    v = in[line * H + k];
                    if (k == 0) v.y = S(0);
                } else {
                    v = cconj(in[line * H + (L - k)]);
                }
            }
            b0[gi(k, line, G)] = v;
        }
        __syncthreads();
        T* y = generic_line<T, +1>(g, b0, b1, G, a.tw);
        S* out = reinterpret_cast<S*>(a.out) + row0 * a.rs;
        for (int i = tid; i < L * nrows; i += nthr) {
            const int line = i / L, p = i % L;
            out[line * a.rs + p] = y[gi(p, line, G)].x;
        }
    }
}

// Lines per CTA: both buffers within 64 KB where a line allows it (a
// Bluestein line of M = 8192 points takes 128 KB in FP32, 256 KB in FP64:
// too long for one CTA, rejected by the FP64 planner).
template <typename T>
int lines_per_cta(const GenPlanT<T>& g)
{
    const int cap = 64 * 1024;
    int G = cap / (2 * gen_line_slots(g) * (int)sizeof(T));
    if (G > 32) G = 32;
    if (G < 1) G = 1;
    return G;
}

template <typename T>
size_t generic_smem(const GenPlanT<T>& g, int G)
{
    return 2 * (size_t)gen_line_slots(g) * G * sizeof(T);
}

template <class A, typename T>
cudaError_t run_generic_col(const A& a, const GenPlanT<T>& g, int dir, cudaStream_t s)
{
    const int G = lines_per_cta(g);
    const size_t smem = generic_smem(g, G);
    const long long tiles = a.nb * ((a.C + G - 1) / G);
    if (tiles <= 0) return cudaSuccess;
    auto k = dir < 0 ? generic_col_kernel<A, T, -1> : generic_col_kernel<A, T, +1>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)tiles, dim3(G, 256 / G > 0 ? 256 / G : 1), smem, s>>>(a, g, G);
    return cudaGetLastError();
}

template <class A, typename T>
cudaError_t run_generic_row(const A& a, const GenPlanT<T>& g, int dir, bool odd, cudaStream_t s)
{
    const int G = lines_per_cta(g);
    const size_t smem = generic_smem(g, G);
    const long long blocks = (a.rows + G - 1) / G;
    if (blocks <= 0) return cudaSuccess;
    auto k = odd ? (dir < 0 ? generic_row_odd_kernel<A, T, -1> : generic_row_odd_kernel<A, T, +1>)
                 : (dir < 0 ? generic_row_kernel<A, T, -1> : generic_row_kernel<A, T, +1>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)blocks, dim3(G, 256 / G > 0 ? 256 / G : 1), smem, s>>>(a, g, G);
    return cudaGetLastError();
}

}  // namespace

cudaError_t generic_col(const ColArgs& a, const GenPlan& g, int dir, cudaStream_t s)
{
    return run_generic_col(a, g, dir, s);
}
cudaError_t generic_row(const RowArgs& a, const GenPlan& g, int dir, cudaStream_t s)
{
    return run_generic_row(a, g, dir, false, s);
}
cudaError_t generic_row_odd(const RowArgs& a, const GenPlan& g, int dir, cudaStream_t s)
{
    return run_generic_row(a, g, dir, true, s);
}
cudaError_t generic_col64(const ColArgs64& a, const GenPlan64& g, int dir, cudaStream_t s)
{
    return run_generic_col(a, g, dir, s);
}
cudaError_t generic_row64(const RowArgs64& a, const GenPlan64& g, int dir, cudaStream_t s)
{
    return run_generic_row(a, g, dir, false, s);
}
cudaError_t generic_row_odd64(const RowArgs64& a, const GenPlan64& g, int dir, cudaStream_t s)
{
    return run_generic_row(a, g, dir, true, s);
}

}  // namespace fft3d

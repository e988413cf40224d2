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
#include "launch_cache.h"
#include "stockham.cuh"
#include "tma.cuh"

namespace fft3d {

template <int L, int E, int DIR, int MAXT>
__global__ void __launch_bounds__(MAXT) col_kernel(ColArgs a, int W)
{
    extern __shared__ float2 sm[];
    constexpr int T = L / E;
    const int c = threadIdx.x;
    const int t = threadIdx.y;
    const long long ctiles = (a.C + W - 1) / W;
    const long long bb = blockIdx.x / ctiles;  // batch entry b of group b2
    const long long c0 = (blockIdx.x - bb * ctiles) * W;
    const long long b2 = bb / a.nb, b = bb - b2 * a.nb;
    const long long boff = b2 * a.Bs2 + b * a.Bs;
    const bool active = (c0 + c) < a.C;
    float2* base = a.data + boff + c0 + c;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = active ? base[(long long)(t + T * m) * a.S] : make_float2(0.f, 0.f);
    ColExchange ex{sm, W, c};
    fft_group<L, E, DIR>(v, t, a.tw, ex);
    if (active) {
        float2* out = (a.dst ? a.dst : a.data) + boff + c0 + c;
        if (a.mask23 == 0 && a.scale == 1.0f) {
#pragma unroll
            for (int m = 0; m < E; ++m) out[(long long)(t + T * m) * a.S] = v[m];
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m)
                out[(long long)(t + T * m) * a.S] = cscale(v[m], col_out_factor(t + T * m, L, a.scale, a.mask23));
        }
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
    const float2* in = reinterpret_cast<const float2*>(a.in) + row0 * a.rs;  // packed z of each row
    float2* out = reinterpret_cast<float2*>(a.out) + row0 * H;

    for (int i = tid; i < ROWS * L; i += T * ROWS) {
        const int rr = i / L, p = i - rr * L;
        sm[rr * RS + Ex::pad(p)] = (rr < nrows) ? in[rr * a.rs + p] : make_float2(0.f, 0.f);
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
    float2* out = reinterpret_cast<float2*>(a.out) + row0 * a.rs;  // real row as float pairs

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
        out[rr * a.rs + p] = sm[rr * RS + Ex::pad(p)];
    }
}

// ---------------------------------------------------------------------------
// Warp-resident row kernels (T = L/E <= 32 threads per row, rows packed into
// warps).  Each thread reads its positions t + T*m straight from global memory
// (adjacent lanes, adjacent addresses), so only the Stockham exchanges touch
// shared memory.  The Hermitian unpack/pack needs, next to bin k = t + T*m,
// bin L-k: for t > 0 that is position (T-t) + T*(E-1-m), held by lane T-t of
// the same row in register E-1-m; for t = 0 it is T*(E-m), the thread's own
// register (E-m) mod E.  One warp shuffle per value replaces a shared-memory
// round trip.  The unpack twiddle W_{2L}^k is formed as W_{2L}^t * W_{2L}^{T m}.
// ---------------------------------------------------------------------------
// Load policy of the row / column bodies: 0 read-only path (__ldg), 1 L2 only
// (__ldcg: data another CTA wrote during this launch), 2 plain load (shared
// memory, through a generic pointer).
constexpr int kLdNc = 0, kLdCg = 1, kLdPlain = 2;
template <int CG>
__device__ __forceinline__ float2 ld2(const float2* p)
{
    if constexpr (CG == kLdCg) return __ldcg(p);
    else if constexpr (CG == kLdPlain) return *p;
    else return __ldg(p);
}

// r2c of one packed real row held in registers (v[m] = samples 2p, 2p+1 at
// position p = t + T*m): forward FFT, Hermitian unpack, then store of the H
// bins to out_row, with bins k2 >= k2_keep set to zero (k2_keep = L+1 keeps
// all; the 2/3 rule keeps 3*k2 < n2).  t in [0, T); lane = the thread's lane;
// the T threads of a row are consecutive lanes.  sm_row: RowLayout<L>::stride
// float2 of exchange space.
// Ex: the exchange policy over sm_row (the warp-synchronous padded row by default).
// TW: the twiddle table (const float2*) or a TwCache of this transform.
template <int L, int E, class Ex = RowExchange<true>, class TW>
__device__ __forceinline__ void row_r2c_regs(float2 (&v)[E], float2* out_row, bool active, int t, int lane,
                                             float2* sm_row, const TW& tw,
                                             const float2* __restrict__ twpack, int k2_keep = L + 1)
{
    constexpr int T = L / E;
    static_assert(T <= 32 && (32 % T) == 0, "rows must pack into warps");
    Ex ex{sm_row};
    fft_group<L, E, -1>(v, t, tw, ex);
    const int partner = lane - t + ((T - t) & (T - 1));
#pragma unroll
    for (int m = 0; m < E; ++m) {
        float2 g;
        g.x = __shfl_sync(0xffffffffu, v[E - 1 - m].x, partner);
        g.y = __shfl_sync(0xffffffffu, v[E - 1 - m].y, partner);
        const float2 zk = v[m];
        const float2 zc = cconj(t == 0 ? v[(E - m) % E] : g);
        const float2 s = cadd(zk, zc);
        const float2 d = csub(zk, zc);
        const float2 w = __ldg(&twpack[t + T * m]);  // W^k, k = t + T*m
        const float2 wd = cmul(d, w);  // X = s/2 - (i/2) W^k d
        const int k = t + T * m;
        if (active)
            out_row[k] = (k < k2_keep) ? make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x)) : make_float2(0.f, 0.f);
    }
    if (active && t == 0) out_row[L] = (L < k2_keep) ? make_float2(v[0].x - v[0].y, 0.f) : make_float2(0.f, 0.f);
}

// r2c of one row: in_row = packed row (L float2), out_row = H bins.
template <int L, int E, int CG>
__device__ __forceinline__ void row_r2c_body(const float2* in_row, float2* out_row, bool active, int t, int lane,
                                             float2* sm_row, const float2* __restrict__ tw,
                                             const float2* __restrict__ twpack)
{
    constexpr int T = L / E;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = active ? ld2<CG>(&in_row[t + T * m]) : make_float2(0.f, 0.f);
    row_r2c_regs<L, E>(v, out_row, active, t, lane, sm_row, tw, twpack);
}

// Loads of one row of H bins for row_c2r_from: x[m] = bin t + T*m, nyq = the
// Nyquist bin L (thread t = 0 only).  Split from the transform so that a
// kernel can issue the loads of several rows before the first one's shuffles.
template <int L, int E, int CG>
__device__ __forceinline__ void row_c2r_load(const float2* in_row, bool active, int t, float2 (&x)[E], float2& nyq)
{
    constexpr int T = L / E;
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = active ? ld2<CG>(&in_row[t + T * m]) : make_float2(0.f, 0.f);
    nyq = (active && t == 0) ? ld2<CG>(&in_row[L]) : make_float2(0.f, 0.f);
}

// c2r of one row whose H bins are in registers (row_c2r_load's x, nyq):
// v[m] = the real samples 2p, 2p+1 at position p = t + T*m (unnormalised).
template <int L, int E, class Ex = RowExchange<true>, class TW>
__device__ __forceinline__ void row_c2r_from(const float2 (&x)[E], float2 nyq, int t, int lane, float2* sm_row,
                                             const TW& tw, const float2* __restrict__ twpack, float2 (&v)[E])
{
    constexpr int T = L / E;
    static_assert(T <= 32 && (32 % T) == 0, "rows must pack into warps");
    const int partner = lane - t + ((T - t) & (T - 1));
#pragma unroll
    for (int m = 0; m < E; ++m) {
        float2 g;
        g.x = __shfl_sync(0xffffffffu, x[E - 1 - m].x, partner);
        g.y = __shfl_sync(0xffffffffu, x[E - 1 - m].y, partner);
        float2 xk = x[m];
        float2 xc;
        if (t == 0) {
            // bin L - T*m: the Nyquist bin for m = 0, else own register E - m
            xc = cconj(m == 0 ? nyq : x[(E - m) % E]);
            if (m == 0) {  // Im of the DC and Nyquist bins is not part of a real row's spectrum
                xk.y = 0.f;
                xc.y = 0.f;
            }
        } else {
            xc = cconj(g);
        }
        const float2 s = cadd(xk, xc);
        const float2 d = csub(xk, xc);
        const float2 w = __ldg(&twpack[t + T * m]);  // W^k, k = t + T*m
        const float2 wd = cmulc(d, w);  // Z = s + i W^{-k} d
        v[m] = make_float2(s.x - wd.y, s.y + wd.x);
    }
    Ex ex{sm_row};
    ex.sync();
    fft_group<L, E, +1>(v, t, tw, ex);
}

// c2r of one row of H bins into registers: v[m] = the real samples 2p, 2p+1
// at position p = t + T*m (unnormalised).
// Ex: the exchange policy over sm_row; sm_row may alias in_row (every lane's
// reads of in_row complete before the first exchange write).
template <int L, int E, int CG, class Ex = RowExchange<true>>
__device__ __forceinline__ void row_c2r_regs(const float2* in_row, bool active, int t, int lane, float2* sm_row,
                                             const float2* __restrict__ tw, const float2* __restrict__ twpack,
                                             float2 (&v)[E])
{
    float2 x[E], nyq;
    row_c2r_load<L, E, CG>(in_row, active, t, x, nyq);
    row_c2r_from<L, E, Ex>(x, nyq, t, lane, sm_row, tw, twpack, v);
}

// c2r of one row: in_row = H bins, out_row = packed real row (L float2).
template <int L, int E, int CG>
__device__ __forceinline__ void row_c2r_body(const float2* in_row, float2* out_row, bool active, int t, int lane,
                                             float2* sm_row, const float2* __restrict__ tw,
                                             const float2* __restrict__ twpack)
{
    constexpr int T = L / E;
    float2 v[E];
    row_c2r_regs<L, E, CG>(in_row, active, t, lane, sm_row, tw, twpack, v);
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) out_row[t + T * m] = v[m];
    }
}

// Pseudo-spectral quadratic products of one row set (the nonlinear term of a
// velocity field, Sec. 1's solver context): the three velocity rows (after
// their n0 and n1 inverse passes) are taken to real space (c2r), the six
// products u_i u_j (ij = 00, 01, 02, 11, 12, 22) formed sample by sample in
// registers, and each product row transformed back (r2c) with the 2/3 rule on
// k2 applied.  in: 3 fields of rows x H bins (field stride fs); out: 6 fields.

// The six products of one row set's velocity samples u (registers), each
// taken back to bins with the k2 part of the 2/3 rule and stored.
template <int L, int E, class TW>
__device__ __forceinline__ void nl_products_r2c(const float2 (&u)[3][E], const NlRowArgs& a, long long row,
                                                bool active, int t, int lane, float2* smr, const TW& tw)
{
    constexpr int H = L + 1;
    constexpr int PI[6] = {0, 0, 0, 1, 1, 2};
    constexpr int PJ[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float2 z[E];
#pragma unroll
        for (int m = 0; m < E; ++m)
            z[m] = make_float2(u[PI[q]][m].x * u[PJ[q]][m].x, u[PI[q]][m].y * u[PJ[q]][m].y);
        row_r2c_regs<L, E>(z, a.out + q * a.fs + row * H, active, t, lane, smr, tw, a.twpack, a.k2_keep);
    }
}

// Short rows (E <= 8): 128 registers, so that eight CTAs fit an SM; the
// kernel is issue-bound, and more resident warps hide the shuffle and
// exchange latencies.
template <int L, int E, int ROWS>
__global__ void __launch_bounds__((L / E) * ROWS, E <= 8 ? 8 : 1) row_nonlinear_kernel(NlRowArgs a)
{
    extern __shared__ float2 sm[];
    constexpr int T = L / E;
    constexpr int H = L + 1;
    const int t = threadIdx.x, r = threadIdx.y;
    const int lane = (r * T + t) & 31;
    const long long row = (long long)blockIdx.x * ROWS + r;
    const bool active = row < a.rows;
    float2* smr = sm + r * RowLayout<L>::stride;
    float2 u[3][E];
    if constexpr (E <= 8) {
        // the loads of all three rows first, so that three rows' worth of
        // requests are in flight before the first c2r (few registers per row)
        float2 x[3][E], nyq[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) row_c2r_load<L, E, false>(a.in + f * a.fs + row * H, active, t, x[f], nyq[f]);
        // the nine transforms of the thread share their twiddles: formed once
        TwCache<L, E> twc;
        twc.fill(a.tw, t);
#pragma unroll
        for (int f = 0; f < 3; ++f) row_c2r_from<L, E>(x[f], nyq[f], t, lane, smr, twc, a.twpack, u[f]);
        nl_products_r2c<L, E>(u, a, row, active, t, lane, smr, twc);
    } else {
#pragma unroll
        for (int f = 0; f < 3; ++f)
            row_c2r_regs<L, E, false>(a.in + f * a.fs + row * H, active, t, lane, smr, a.tw, a.twpack, u[f]);
        nl_products_r2c<L, E>(u, a, row, active, t, lane, smr, a.tw);
    }
}

template <int L, int E, int ROWS>
inline size_t row_smem();

template <int L, int E, int ROWS>
inline cudaError_t launch_row_nonlinear(const NlRowArgs& a, cudaStream_t s)
{
    constexpr int T = L / E;
    static_assert((T * ROWS) % 32 == 0, "the shuffles need whole warps");
    const size_t smem = row_smem<L, E, ROWS>();
    const long long blocks = (a.rows + ROWS - 1) / ROWS;
    if (blocks <= 0) return cudaSuccess;
    row_nonlinear_kernel<L, E, ROWS><<<(unsigned)blocks, dim3(T, ROWS), smem, s>>>(a);
    return cudaGetLastError();
}

template <int L, int E, int ROWS>
__global__ void __launch_bounds__((L / E) * ROWS) row_r2c_warp_kernel(RowArgs a)
{
    extern __shared__ float2 sm[];
    constexpr int T = L / E;
    constexpr int H = L + 1;
    const int t = threadIdx.x, r = threadIdx.y;
    const long long row = (long long)blockIdx.x * blockDim.y + r;
    row_r2c_body<L, E, kLdCg>(reinterpret_cast<const float2*>(a.in) + row * a.rs,
                              reinterpret_cast<float2*>(a.out) + row * H, row < a.rows, t, (r * T + t) & 31,
                              sm + r * RowLayout<L>::stride, a.tw, a.twpack);
}

// The c2r rows with 32 values per thread (L = 1024) take 147 registers
// uncapped: 6 CTAs of 64 threads per SM, too few warps to cover the loads of
// the half-spectrum rows (long-scoreboard stalls); capped at 128, 8 CTAs fit,
// as for the r2c rows.
template <int L, int E, int ROWS>
constexpr int row_c2r_min_ctas()
{
    return (E >= 32 && (L / E) * ROWS <= 64) ? 8 : 1;
}

template <int L, int E, int ROWS>
__global__ void __launch_bounds__((L / E) * ROWS, row_c2r_min_ctas<L, E, ROWS>()) row_c2r_warp_kernel(RowArgs a)
{
    extern __shared__ float2 sm[];
    constexpr int T = L / E;
    constexpr int H = L + 1;
    const int t = threadIdx.x, r = threadIdx.y;
    const long long row = (long long)blockIdx.x * blockDim.y + r;
    // read-only cached loads: every other half-spectrum row starts 8 bytes
    // off a 16-byte boundary, so a warp's 256-byte load shares its last
    // sector with the next one, which L1 then serves (2048^3 row c2r 11.9 ->
    // 11.3 ms).  Safe in place (padded layout): a row's threads hold all
    // their inputs before any store, and no row reads another's bytes.
    row_c2r_body<L, E, kLdNc>(reinterpret_cast<const float2*>(a.in) + row * H,
                              reinterpret_cast<float2*>(a.out) + row * a.rs, row < a.rows, t, (r * T + t) & 31,
                              sm + r * RowLayout<L>::stride, a.tw, a.twpack);
}

// Column transform of one tile column: base points at element (j = 0) of the
// column, positions t + T*m at stride S; exchange through ex.
// Out-of-place variant: reads the column at src, writes the result at dst
// (same layout and stride).
template <int L, int E, int DIR, bool CG>
__device__ __forceinline__ void col_body_to(const float2* src, float2* dst, long long S, bool active, int t,
                                            const float2* __restrict__ tw, const ColExchange& ex)
{
    constexpr int T = L / E;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = active ? ld2<CG>(&src[(long long)(t + T * m) * S]) : make_float2(0.f, 0.f);
    fft_group<L, E, DIR>(v, t, tw, ex);
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) dst[(long long)(t + T * m) * S] = v[m];
    }
}

template <int L, int E, int DIR, bool CG>
__device__ __forceinline__ void col_body(float2* base, long long S, bool active, int t, const float2* __restrict__ tw,
                                         float scale, const ColExchange& ex)
{
    constexpr int T = L / E;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = active ? ld2<CG>(&base[(long long)(t + T * m) * S]) : make_float2(0.f, 0.f);
    fft_group<L, E, DIR>(v, t, tw, ex);
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) base[(long long)(t + T * m) * S] = cscale(v[m], scale);
    }
}

// ---------------------------------------------------------------------------
// Persistent, pipelined column kernel.  Each CTA walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; the elements of the tile STAGES-1 steps ahead
// are copied global -> shared with cp.async while the current tile is
// transformed, so loads, butterflies and stores of different tiles overlap.
// A thread copies exactly the elements it later reads (positions t + T*m of
// its column), so a stage buffer needs no barrier: cp.async.wait_group on the
// thread's own copy groups is enough.  Only the Stockham exchange buffer is
// shared between threads.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int L, int E, int DIR, int W, int STAGES>
__global__ void __launch_bounds__(W*(L / E)) col_pipe_kernel(ColArgs a, long long ntiles)
{
    extern __shared__ __align__(16) float2 sm[];
    constexpr int T = L / E;
    const int c = threadIdx.x;
    const int t = threadIdx.y;
    const long long ctiles = (a.C + W - 1) / W;
    float2* ex_buf = sm + (size_t)STAGES * L * W;

    auto issue = [&](long long tile, int stage) {
        if (tile < ntiles) {
            const long long b = tile / ctiles;
            const long long c0 = (tile - b * ctiles) * W;
            if (c0 + c < a.C) {
                const float2* src = a.data + b * a.Bs + c0 + c;
                float2* dst = sm + (size_t)stage * L * W + c;
#pragma unroll
                for (int m = 0; m < E; ++m) cp_async8(dst + (t + T * m) * W, src + (long long)(t + T * m) * a.S);
            }
        }
        cp_async_commit();  // one group per tile slot, possibly empty, keeps the counting uniform
    };

    long long tile = blockIdx.x;
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) issue(tile + (long long)s * gridDim.x, s);
    int stage = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        issue(tile + (long long)(STAGES - 1) * gridDim.x, (stage + STAGES - 1) % STAGES);
        cp_async_wait<STAGES - 1>();
        const long long b = tile / ctiles;
        const long long c0 = (tile - b * ctiles) * W;
        const bool active = (c0 + c) < a.C;
        const float2* buf = sm + (size_t)stage * L * W + c;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = active ? buf[(t + T * m) * W] : make_float2(0.f, 0.f);
        ColExchange exch{ex_buf, W, c};
        fft_group<L, E, DIR>(v, t, a.tw, exch);
        if (active) {
            float2* dst = a.data + b * a.Bs + c0 + c;
#pragma unroll
            for (int m = 0; m < E; ++m) dst[(long long)(t + T * m) * a.S] = cscale(v[m], a.scale);
        }
        stage = (stage + 1) % STAGES;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// TMA-fed persistent column kernel (the n0 pass).  The volume is seen as a 2D
// FP32 tensor: inner extent 2*C floats (the flat (k1, k2) plane), outer extent
// nb*L rows at a byte stride of 8*S.  A tile (W columns x L rows) arrives with
// L/256 bulk tensor copies into one slot of a STAGES-deep shared-memory ring;
// one elected thread keeps STAGES-1 tiles in flight, completion is counted on
// the slot's mbarrier (transaction bytes), so the copies hold no registers and
// no thread issue slots.  After the threads have read their values from the
// slot, the slot doubles as the Stockham exchange buffer; results go straight
// from registers to global memory.  Every mbarrier wait is bounded: a wait
// that gives up sets kStatusTimeout in the device status word, and the CTA
// drains its outstanding copies (again bounded) before returning.
// Requirements (checked by the host): the base address 16-byte aligned,
// Bs == L*S, W*8 a multiple of 16, and 8*S a multiple of 16.
//
// PAIR mode lifts the last one (an odd axis stride S, e.g. the n1 pass with
// H = n2/2+1 odd): the volume is viewed as PAIRS of rows (stride 16*S bytes,
// inner extent 2*S complex), the even rows of a tile come as a box starting
// at column c0, the odd rows as a box starting at column c0-1 of the second
// row of the pair (H + c0 - 1 is even, so the start stays 16-byte aligned);
// both boxes are W+2 columns wide and the reads index past the offset.
// ---------------------------------------------------------------------------
constexpr unsigned kMbarMaxTries = 1u << 20;

// XB: a dedicated exchange buffer next to the ring, so reading the slot and
// the first exchange write need no barrier between them, and the next tile's
// barrier orders the buffer's reuse (two CTA barriers per tile with a single
// exchange instead of four).  Used where the ring alone already limits the
// SM to one CTA and the buffer still fits.
template <int L, int E, int W, int STAGES, bool PAIR>
constexpr bool col_tma_xbuf()
{
    constexpr size_t ring = (size_t)STAGES * L * (PAIR ? W + 2 : W) * 8 + 64;
    return ring > 113 * 1024 && ring + (size_t)L * W * 8 <= 227 * 1024;
}

template <int L, int E, int DIR, int W, int STAGES, int PF = 0, bool PAIR = false,
          bool XB = col_tma_xbuf<L, E, W, STAGES, PAIR>()>
__global__ void __launch_bounds__(W*(L / E)) col_tma_kernel(const __grid_constant__ CUtensorMap tmap, ColArgs a,
                                                           long long ntiles)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    constexpr int T = L / E;
    constexpr int ROWS_IN_MAP = PAIR ? L / 2 : L;  // tensor rows per tile (row pairs in PAIR mode)
    constexpr int BOXR = tma_box_rows(ROWS_IN_MAP);
    constexpr int NBOX = ROWS_IN_MAP / BOXR;
    static_assert(ROWS_IN_MAP % BOXR == 0, "tile rows must split into boxes of <= 256 rows");
    static_assert(!PAIR || (L % 2 == 0 && W % 2 == 0), "row pairs need even L and W");
    static_assert(STAGES >= 2, "one slot is consumed while the next is in flight: at least two slots");
    constexpr int WS = PAIR ? W + 2 : W;  // slot row width (complex values)
    constexpr unsigned TILE_BYTES = (unsigned)L * WS * sizeof(float2);
    constexpr size_t XBYTES = XB ? (size_t)L * W * sizeof(float2) : 0;
    float2* ring = reinterpret_cast<float2*>(smraw);
    float2* xbuf = reinterpret_cast<float2*>(smraw + (size_t)STAGES * TILE_BYTES);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smraw + (size_t)STAGES * TILE_BYTES + XBYTES);
    const int c = threadIdx.x;
    const int t = threadIdx.y;
    const bool leader = (c == 0 && t == 0);
    const long long ctiles = (a.C + W - 1) / W;
    // leader: copies issued so far; the k-th goes to slot k % STAGES with
    // phase parity (k / STAGES) & 1 (bookkeeping for the drain)
    long long n_issued = 0;

    if (leader) {
        prefetch_tensormap(&tmap);
#pragma unroll
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](long long tile, int s) {
        if (tile >= ntiles) return;
        const long long b = tile / ctiles;
        const long long c0 = (tile - b * ctiles) * W;
        const int x = (int)(2 * c0);
        mbar_arrive_expect_tx(&bars[s], TILE_BYTES);
        float2* slot = ring + (size_t)s * L * WS;
#pragma unroll
        for (int k = 0; k < NBOX; ++k) {
            const int y = (int)(b * ROWS_IN_MAP + k * BOXR);
            tma_load_2d(slot + (size_t)k * BOXR * WS, &tmap, x, y, &bars[s]);
            if constexpr (PAIR)
                tma_load_2d(slot + (size_t)(L / 2) * WS + (size_t)k * BOXR * WS, &tmap, (int)(2 * (a.S + c0 - 1)), y,
                            &bars[s]);
        }
        ++n_issued;
        if constexpr (PF > 0) {  // warm L2 with the tile PF ring-lengths further on
            const long long pt = tile + (long long)PF * gridDim.x;
            if (pt < ntiles) {
                const long long pb = pt / ctiles;
                const long long pc0 = (pt - pb * ctiles) * W;
#pragma unroll
                for (int k = 0; k < NBOX; ++k) {
                    const int y = (int)(pb * ROWS_IN_MAP + k * BOXR);
                    tma_prefetch_l2_2d(&tmap, (int)(2 * pc0), y);
                    if constexpr (PAIR) tma_prefetch_l2_2d(&tmap, (int)(2 * (a.S + pc0 - 1)), y);
                }
            }
        }
    };

    if (leader) {
#pragma unroll
        for (int s = 0; s < STAGES - 1; ++s) issue(blockIdx.x + (long long)s * gridDim.x, s);
    }
    // the butterfly positions of a thread are the same in every tile: its
    // twiddles are formed once
    TwCache<L, E> twc;
    twc.fill(a.tw, t);
    int stage = 0;
    unsigned phase = 0;
    long long n_consumed = 0;
    bool failed = false;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const bool ok = mbar_wait_bounded(&bars[stage], phase, kMbarMaxTries);
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        ++n_consumed;
        // the slot consumed in the previous iteration is free again: refill it
        if (leader) issue(tile + (long long)(STAGES - 1) * gridDim.x, (stage + STAGES - 1) % STAGES);
        const long long b = tile / ctiles;
        const long long c0 = (tile - b * ctiles) * W;
        const bool active = (c0 + c) < a.C;
        float2* buf = ring + (size_t)stage * L * WS;
        float2 v[E];
        if constexpr (PAIR && T % 2 == 0) {
            // row parity is the thread's own (t + T*m has the parity of t):
            // even rows from the box at c0, odd rows from the box at c0 - 1
            const float2* src = (t & 1) ? buf + (L / 2) * WS + c + 1 : buf + c;
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = src[((t >> 1) + (T / 2) * m) * WS];
        } else if constexpr (PAIR) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int j = t + T * m;  // even rows: box from c0; odd rows: box from c0 - 1
                v[m] = (j & 1) ? buf[(L / 2) * WS + (j >> 1) * WS + c + 1] : buf[(j >> 1) * WS + c];
            }
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = buf[(t + T * m) * W + c];
        }
        if constexpr (XB) {
            fft_group<L, E, DIR>(v, t, twc, ColExchangeNoTail{xbuf, W, c});
        } else {
            __syncthreads();  // the slot now serves as the exchange buffer
            fft_group<L, E, DIR>(v, t, twc, ColExchange{buf, W, c});
        }
        fence_proxy_async_smem();  // order this thread's shared accesses before the slot's next bulk copy
        if (active) {
            float2* dst = (a.dst ? a.dst : a.data) + b * a.Bs + c0 + c;
            if (a.mask23 == 0 && a.scale == 1.0f) {
#pragma unroll
                for (int m = 0; m < E; ++m) dst[(long long)(t + T * m) * a.S] = v[m];
            } else {
#pragma unroll
                for (int m = 0; m < E; ++m)
                    dst[(long long)(t + T * m) * a.S] = cscale(v[m], col_out_factor(t + T * m, L, a.scale, a.mask23));
            }
        }
        if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
        }
    }
    if (failed && leader) {
        atomicOr(a.status, kStatusTimeout);
        // drain: wait (bounded) for every copy issued but not consumed
        for (long long k = n_consumed; k < n_issued; ++k)
            mbar_wait_bounded(&bars[k % STAGES], (unsigned)((k / STAGES) & 1), kMbarMaxTries);
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
inline cudaError_t launch_col(const ColArgs& a, int w, cudaStream_t s)
{
    constexpr int T = L / E;
    constexpr int MAXT = W * T;
    static_assert(MAXT <= 1024, "too many threads");
    const int wr = (w > 0 && w <= W) ? w : W;  // runtime columns per CTA
    const size_t smem_max = (size_t)L * W * sizeof(float2);
    const size_t smem = (size_t)L * wr * sizeof(float2);
    auto k = col_kernel<L, E, DIR, MAXT>;
    static PerDevice limit;  // the shared memory limit, raised once per device
    if (smem_max > 48 * 1024) {
        cudaError_t e = smem_limit_per_device(limit, k, smem_max);
        if (e != cudaSuccess) return e;
    }
    const long long tiles = a.nb2 * a.nb * ((a.C + wr - 1) / wr);
    if (tiles <= 0) return cudaSuccess;
    k<<<(unsigned)tiles, dim3(wr, T), smem, s>>>(a, wr);
    return cudaGetLastError();
}

template <int L, int E, int ROWS>
inline size_t row_smem()
{
    return (size_t)ROWS * RowLayout<L>::stride * sizeof(float2);
}

template <int L, int E, int ROWS, int DIR>
inline cudaError_t launch_row(const RowArgs& a, int /*rows: fixed for the staged kernel*/, cudaStream_t s)
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

template <int L, int E, int ROWS, int DIR>
inline cudaError_t launch_row_warp(const RowArgs& a, int rows, cudaStream_t s)
{
    constexpr int T = L / E;
    static_assert((T * ROWS) % 32 == 0, "the shuffles need whole warps");
    // runtime rows per CTA: at most ROWS, whole warps
    const int rr = (rows > 0 && rows <= ROWS && (T * rows) % 32 == 0) ? rows : ROWS;
    const size_t smem_max = (num_stages(L, E) > 1) ? row_smem<L, E, ROWS>() : 0;
    const size_t smem = smem_max / ROWS * rr;
    const long long blocks = (a.rows + rr - 1) / rr;
    if (blocks <= 0) return cudaSuccess;
    auto k = (DIR < 0) ? row_r2c_warp_kernel<L, E, ROWS> : row_c2r_warp_kernel<L, E, ROWS>;
    static PerDevice limit;  // the shared memory limit, raised once per device
    if (smem_max > 48 * 1024) {
        cudaError_t e = smem_limit_per_device(limit, k, smem_max);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)blocks, dim3(T, rr), smem, s>>>(a);
    return cudaGetLastError();
}

template <int L, int E, int W, int STAGES, int DIR>
inline cudaError_t launch_col_pipe(const ColArgs& a, cudaStream_t s)
{
    constexpr int T = L / E;
    const size_t smem = (size_t)(STAGES + 1) * L * W * sizeof(float2);
    auto k = col_pipe_kernel<L, E, DIR, W, STAGES>;
    static PerDevice resident;  // resident CTAs on the device, queried once per device
    int ctas = 0;
    cudaError_t e = resident_ctas_per_device(resident, k, W * T, smem, &ctas);
    if (e != cudaSuccess) return e;
    const long long ntiles = a.nb * ((a.C + W - 1) / W);
    if (ntiles <= 0) return cudaSuccess;
    long long grid = ctas;
    if (grid > ntiles) grid = ntiles;
    k<<<(unsigned)grid, dim3(W, T), smem, s>>>(a, ntiles);
    return cudaGetLastError();
}

template <int L, int E, int W, int STAGES, int DIR, int PF = 0, bool PAIR = false>
inline cudaError_t launch_col_tma(const ColArgs& a, const CUtensorMap& map, cudaStream_t s)
{
    constexpr int T = L / E;
    constexpr int WS = PAIR ? W + 2 : W;
    constexpr bool XB = col_tma_xbuf<L, E, W, STAGES, PAIR>();
    const size_t smem = (size_t)STAGES * L * WS * sizeof(float2) + (XB ? (size_t)L * W * sizeof(float2) : 0) +
                        STAGES * sizeof(unsigned long long);
    auto k = col_tma_kernel<L, E, DIR, W, STAGES, PF, PAIR>;
    static PerDevice resident;  // resident CTAs on the device, queried once per device
    int ctas = 0;
    cudaError_t e = resident_ctas_per_device(resident, k, W * T, smem, &ctas);
    if (e != cudaSuccess) return e;
    const long long ntiles = a.nb * ((a.C + W - 1) / W);
    if (ntiles <= 0) return cudaSuccess;
    long long grid = ctas;
    if (grid > ntiles) grid = ntiles;
    k<<<(unsigned)grid, dim3(W, T), smem, s>>>(map, a, ntiles);
    return cudaGetLastError();
}

inline cudaError_t col_tensor_map(CUtensorMap* map, const ColArgs& a, int L, int W, bool pair = false)
{
    return col_tensor_map_host(map, a, L, W, pair);
}

}  // namespace fft3d

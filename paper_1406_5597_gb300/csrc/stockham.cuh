// Compile-time Stockham FFT of length L held in registers by a group of
// T = L/E threads, E elements each, exchanging through shared memory.
//
// Thread t of the group always holds the elements at positions t + T*m,
// m in [0, E).  A stage of radix R (R divides E) with Ns = product of the
// earlier radices runs the butterflies j = t + T*q, q in [0, E/R): butterfly j
// reads positions j + k*L/R = t + T*(q + k*E/R), i.e. register q + k*E/R, so
// every stage reads a thread's own registers; it twiddles input k by
// W_{Ns*R}^{k*(j mod Ns)}, takes the radix-R DFT and writes output k to
// position (j div Ns)*Ns*R + (j mod Ns) + k*Ns (the self-sorting Stockham
// order).  Those writes go through shared memory; after a barrier each
// thread reloads positions t + T*m.  In the last stage (Ns*R = L) the output
// positions are the input positions again, so the result stays in registers,
// in natural order, with no final exchange.
//
// Twiddles come from a table of W_L^m = exp(-2 pi i m / L), m in [0, L),
// computed in FP64 on the host and rounded to FP32 (W_{Ns*R}^{x} = W_L^{x*L/(Ns*R)}).
#pragma once
#include <type_traits>

#include "radix.cuh"

namespace fft3d {

constexpr int pick_radix(int rem, int E)
{
    constexpr int order[8] = {32, 16, 8, 4, 2, 5, 3, 7};
    for (int i = 0; i < 8; ++i)
        if (E % order[i] == 0 && rem % order[i] == 0) return order[i];
    return 0;
}

constexpr int num_stages(int L, int E)
{
    int s = 0, rem = L;
    while (rem > 1) {
        int R = pick_radix(rem, E);
        if (R == 0) return -1;
        rem /= R;
        ++s;
    }
    return s;
}

constexpr int radix_at(int L, int E, int s)
{
    int rem = L, R = 1;
    for (int i = 0; i <= s; ++i) {
        R = pick_radix(rem, E);
        rem /= R;
    }
    return R;
}

constexpr int ns_at(int L, int E, int s)
{
    int ns = 1;
    for (int i = 0; i < s; ++i) ns *= radix_at(L, E, i);
    return ns;
}

// Exchange policies: where position p of the group's vector lives in shared
// memory, and which barrier orders the group.
//
// Column exchange: W columns side by side, position p of column c at
// sm[p*W + c]; lanes run along c, so every access is a contiguous run.
struct ColExchange {
    float2* sm;
    int W;
    int c;
    __device__ __forceinline__ void put(int p, float2 v) const { sm[p * W + c] = v; }
    __device__ __forceinline__ float2 get(int p) const { return sm[p * W + c]; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// The same, for a caller that orders the buffer's next use itself: the
// barrier after the reads of the last exchange (which only protects the
// buffer against a following put) is left out.
struct ColExchangeNoTail {
    float2* sm;
    int W;
    int c;
    static constexpr bool kSkipLastTrailingSync = true;
    __device__ __forceinline__ void put(int p, float2 v) const { sm[p * W + c] = v; }
    __device__ __forceinline__ float2 get(int p) const { return sm[p * W + c]; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

template <class Ex, class = void>
struct TrailingSync {
    static constexpr bool value = true;
};
template <class Ex>
struct TrailingSync<Ex, std::void_t<decltype(Ex::kSkipLastTrailingSync)>> {
    static constexpr bool value = !Ex::kSkipLastTrailingSync;
};

// Row exchange: one row per group, position p at sm[p + p/16] (one pad slot
// per 16 complex values spreads the strided Stockham writes over the banks).
template <bool WARP_SYNC>
struct RowExchange {
    float2* sm;
    __device__ __forceinline__ static int pad(int p) { return p + (p >> 4); }
    __device__ __forceinline__ void put(int p, float2 v) const { sm[pad(p)] = v; }
    __device__ __forceinline__ float2 get(int p) const { return sm[pad(p)]; }
    __device__ __forceinline__ void sync() const
    {
        if constexpr (WARP_SYNC) __syncwarp();
        else __syncthreads();
    }
};

// Twiddles of a radix-R butterfly, inputs 1..R-1 by W^{k*base} (table
// units).  Only the powers W^{base}, W^{2 base}, W^{4 base} (W^{8 base},
// W^{16 base}) are read from the FP32 table; the others are products of two
// to four of them (each product adds one FP32 rounding).
template <int R>
constexpr int n_powers()
{
    return R == 2 ? 1 : R == 3 || R == 4 ? 2 : R == 5 || R == 7 || R == 8 ? 3 : R == 16 ? 4 : 5;
}

template <int R>
__device__ __forceinline__ void load_powers(float2 (&p)[5], const float2* __restrict__ tw, int base)
{
#pragma unroll
    for (int i = 0; i < n_powers<R>(); ++i) p[i] = __ldg(&tw[(1 << i) * base]);
}

// w[k] = W^{k base}, k in [1, R), from the powers p[i] = W^{2^i base}.
template <int R>
__device__ __forceinline__ void twiddle_set(const float2 (&p)[5], float2* w)
{
    w[1] = p[0];
    if constexpr (R >= 3) w[2] = p[1];
    if constexpr (R >= 4) w[3] = cmul(p[0], p[1]);
    if constexpr (R >= 5) w[4] = p[2];
    if constexpr (R >= 6) w[5] = cmul(w[1], w[4]);
    if constexpr (R >= 7) w[6] = cmul(w[2], w[4]);
    if constexpr (R >= 8) w[7] = cmul(w[3], w[4]);
    if constexpr (R == 16) {
        w[8] = p[3];
        const float2 w12 = cmul(w[4], w[8]);
        w[9] = cmul(w[1], w[8]);
        w[10] = cmul(w[2], w[8]);
        w[11] = cmul(w[3], w[8]);
        w[12] = w12;
        w[13] = cmul(w[1], w12);
        w[14] = cmul(w[2], w12);
        w[15] = cmul(w[3], w12);
    }
    if constexpr (R == 32) {
        w[8] = p[3];
        w[16] = p[4];
#pragma unroll
        for (int k = 9; k < 16; ++k) w[k] = cmul(w[k - 8], w[8]);
#pragma unroll
        for (int k = 17; k < 32; ++k) w[k] = cmul(w[k - 16], w[16]);
    }
}

template <int R, int DIR>
__device__ __forceinline__ void twiddle_apply(float2* a, const float2* w)
{
#pragma unroll
    for (int k = 1; k < R; ++k) a[k] = twiddle<DIR>(a[k], w[k]);
}

template <int R, int DIR>
__device__ __forceinline__ void twiddle_inputs(float2* a, const float2* __restrict__ tw, int base)
{
    float2 p[5];
    load_powers<R>(p, tw, base);
    float2 w[R];
    twiddle_set<R>(p, w);
    twiddle_apply<R, DIR>(a, w);
}

// Per-thread twiddle cache of a whole transform (every stage after the
// first, every butterfly of the thread), for persistent kernels whose
// butterfly positions depend on the thread alone: filled once, it replaces
// the table reads and products of every later transform.
template <int L, int E, int TS = 1>
struct TwCache {
    static constexpr int NS = num_stages(L, E);
    static constexpr int T = L / E;
    float2 w[NS][E][32];  // [stage][butterfly][k]; only the entries in use become registers
    template <int S>
    __device__ __forceinline__ void fill_from(const float2* __restrict__ tw, int t)
    {
        if constexpr (S < NS) {
            constexpr int R = radix_at(L, E, S);
            constexpr int Ns = ns_at(L, E, S);
            constexpr int Q = E / R;
            constexpr int step = L / (Ns * R);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int jm = (t + T * q) % Ns;
                float2 p[5];
                load_powers<R>(p, tw, jm * step * TS);
                twiddle_set<R>(p, w[S][q]);
            }
            fill_from<S + 1>(tw, t);
        }
    }
    __device__ __forceinline__ void fill(const float2* __restrict__ tw, int t) { fill_from<1>(tw, t); }
};

template <class TW>
struct IsTwCache {
    static constexpr bool value = false;
};
template <int L, int E, int TS>
struct IsTwCache<TwCache<L, E, TS>> {
    static constexpr bool value = true;
};

// TS: the twiddle table has length L*TS (W_L^x = table[x*TS]).
template <int L, int E, int DIR, int S, int TS = 1>
struct Stage {
    // TW: the twiddle table (const float2*) or a TwCache of this transform
    template <class Ex, class TW>
    __device__ __forceinline__ static void run(float2 (&v)[E], int t, const TW& tw, const Ex& ex)
    {
        constexpr int NS = num_stages(L, E);
        constexpr int R = radix_at(L, E, S);
        constexpr int Ns = ns_at(L, E, S);
        constexpr int T = L / E;
        constexpr int Q = E / R;
        constexpr bool last = (S == NS - 1);
        static_assert(R > 0 && E % R == 0, "radix must divide E");
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float2 a[R];
#pragma unroll
            for (int k = 0; k < R; ++k) a[k] = v[q + k * Q];
            const int j = t + T * q;
            const int jm = j % Ns;
            if constexpr (Ns > 1) {
                if constexpr (IsTwCache<TW>::value) {
                    twiddle_apply<R, DIR>(a, tw.w[S][q]);
                } else {
                    constexpr int step = L / (Ns * R);
                    twiddle_inputs<R, DIR>(a, tw, jm * step * TS);
                }
            }
            Dft<R, DIR>::run(a);
            if constexpr (last) {
#pragma unroll
                for (int k = 0; k < R; ++k) v[q + k * Q] = a[k];
            } else {
                const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
                for (int k = 0; k < R; ++k) ex.put(base + k * Ns, a[k]);
            }
        }
        if constexpr (!last) {
            ex.sync();
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = ex.get(t + T * m);
            if constexpr (S + 2 < NS || TrailingSync<Ex>::value) ex.sync();
            Stage<L, E, DIR, S + 1, TS>::run(v, t, tw, ex);
        }
    }
};

// Full transform: v holds positions t + T*m on entry and their DFT on exit.
// TS > 1: the twiddle table belongs to a TS times longer transform.
template <int L, int E, int DIR, int TS = 1, class Ex, class TW>
__device__ __forceinline__ void fft_group(float2 (&v)[E], int t, const TW& tw, const Ex& ex)
{
    static_assert(num_stages(L, E) > 0, "L must factor into radices dividing E");
    Stage<L, E, DIR, 0, TS>::run(v, t, tw, ex);
}

}  // namespace fft3d

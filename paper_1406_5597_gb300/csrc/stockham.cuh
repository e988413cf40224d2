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
#include "radix.cuh"

namespace fft3d {

constexpr int pick_radix(int rem, int E)
{
    constexpr int order[7] = {32, 16, 8, 4, 2, 5, 3};
    for (int i = 0; i < 7; ++i)
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

// Twiddle inputs 1..R-1 of a radix-R butterfly by W^{k*base} (table units).
// Only the powers 1, 2, 4 (8, 16) are read from the FP32 table; the others
// are products of two to four of them (each product adds one FP32 rounding).
template <int R, int DIR>
__device__ __forceinline__ void twiddle_inputs(float2* a, const float2* __restrict__ tw, int base)
{
    const float2 w1 = __ldg(&tw[base]);
    if constexpr (R == 2) {
        a[1] = twiddle<DIR>(a[1], w1);
    } else if constexpr (R == 3) {
        a[1] = twiddle<DIR>(a[1], w1);
        a[2] = twiddle<DIR>(a[2], __ldg(&tw[2 * base]));
    } else if constexpr (R == 4) {
        const float2 w2 = __ldg(&tw[2 * base]);
        a[1] = twiddle<DIR>(a[1], w1);
        a[2] = twiddle<DIR>(a[2], w2);
        a[3] = twiddle<DIR>(a[3], cmul(w1, w2));
    } else if constexpr (R == 5) {
        const float2 w2 = __ldg(&tw[2 * base]);
        const float2 w4 = __ldg(&tw[4 * base]);
        a[1] = twiddle<DIR>(a[1], w1);
        a[2] = twiddle<DIR>(a[2], w2);
        a[3] = twiddle<DIR>(a[3], cmul(w1, w2));
        a[4] = twiddle<DIR>(a[4], w4);
    } else if constexpr (R == 32) {
        // powers 1, 2, 4, 8, 16 from the table, the rest as products
        float2 w[32];
        w[1] = w1;
        w[2] = __ldg(&tw[2 * base]);
        w[4] = __ldg(&tw[4 * base]);
        w[8] = __ldg(&tw[8 * base]);
        w[16] = __ldg(&tw[16 * base]);
        w[3] = cmul(w[1], w[2]);
#pragma unroll
        for (int k = 5; k < 8; ++k) w[k] = cmul(w[k - 4], w[4]);
#pragma unroll
        for (int k = 9; k < 16; ++k) w[k] = cmul(w[k - 8], w[8]);
#pragma unroll
        for (int k = 17; k < 32; ++k) w[k] = cmul(w[k - 16], w[16]);
#pragma unroll
        for (int k = 1; k < 32; ++k) a[k] = twiddle<DIR>(a[k], w[k]);
    } else if constexpr (R == 8 || R == 16) {
        const float2 w2 = __ldg(&tw[2 * base]);
        const float2 w4 = __ldg(&tw[4 * base]);
        const float2 w3 = cmul(w1, w2);
        a[1] = twiddle<DIR>(a[1], w1);
        a[2] = twiddle<DIR>(a[2], w2);
        a[3] = twiddle<DIR>(a[3], w3);
        a[4] = twiddle<DIR>(a[4], w4);
        a[5] = twiddle<DIR>(a[5], cmul(w1, w4));
        a[6] = twiddle<DIR>(a[6], cmul(w2, w4));
        a[7] = twiddle<DIR>(a[7], cmul(w3, w4));
        if constexpr (R == 16) {
            const float2 w8 = __ldg(&tw[8 * base]);
            const float2 w12 = cmul(w4, w8);
            a[8] = twiddle<DIR>(a[8], w8);
            a[9] = twiddle<DIR>(a[9], cmul(w1, w8));
            a[10] = twiddle<DIR>(a[10], cmul(w2, w8));
            a[11] = twiddle<DIR>(a[11], cmul(w3, w8));
            a[12] = twiddle<DIR>(a[12], w12);
            a[13] = twiddle<DIR>(a[13], cmul(w1, w12));
            a[14] = twiddle<DIR>(a[14], cmul(w2, w12));
            a[15] = twiddle<DIR>(a[15], cmul(w3, w12));
        }
    }
}

// TS: the twiddle table has length L*TS (W_L^x = table[x*TS]).
template <int L, int E, int DIR, int S, int TS = 1>
struct Stage {
    template <class Ex>
    __device__ __forceinline__ static void run(float2 (&v)[E], int t, const float2* __restrict__ tw, const Ex& ex)
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
                constexpr int step = L / (Ns * R);
                twiddle_inputs<R, DIR>(a, tw, jm * step * TS);
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
            ex.sync();
            Stage<L, E, DIR, S + 1, TS>::run(v, t, tw, ex);
        }
    }
};

// Full transform: v holds positions t + T*m on entry and their DFT on exit.
// TS > 1: the twiddle table belongs to a TS times longer transform.
template <int L, int E, int DIR, int TS = 1, class Ex>
__device__ __forceinline__ void fft_group(float2 (&v)[E], int t, const float2* __restrict__ tw, const Ex& ex)
{
    static_assert(num_stages(L, E) > 0, "L must factor into radices dividing E");
    Stage<L, E, DIR, 0, TS>::run(v, t, tw, ex);
}

}  // namespace fft3d

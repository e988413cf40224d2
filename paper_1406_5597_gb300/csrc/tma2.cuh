// TMA-fed column pass over row pairs with two columns per thread (the n1
// pass of Sec. 2.1 at an odd axis stride S, e.g. H = n2/2 + 1).
//
// The tile, ring and row-pair view are those of col_tma_kernel in PAIR mode
// (even rows of a W-column tile from a box at column c0, odd rows from a box
// at c0 - 1 of the row pair's second row, W + 2 columns wide).  What differs
// is the thread's share: thread (cp, t) holds columns 2cp and 2cp + 1 at the
// rows t + T*m, so its shared-memory and global accesses move two complex
// values at a time (16 bytes) where the one-column kernel moves one: the
// even rows' reads from the slot, every exchange, and the even rows' global
// stores (an odd row starts 8 bytes off a 16-byte boundary, so its reads and
// stores stay 8-byte pairs).  The one-column kernel at L = 2048 is bound by
// the issue of those memory instructions (MIO and LSU queues), not by DRAM.
// The two columns' butterflies run the same float2 codelets one after the
// other; the Stockham indexing is that of Stage in stockham.cuh.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace fft3d {

// Exchange of column pairs: position p of pair cp at sm[pad(p) * WP + cp]
// (16 bytes each).  A first radix-16 stage writes a warp's positions 16
// apart; one pad slot per 16 positions spreads them to the four-wavefront
// minimum of a 512-byte warp access.  Needs (L + L/16) * WP float4.
struct ColPairExchange {
    float4* sm;
    int WP;
    int cp;
    __device__ __forceinline__ static int pad(int p) { return p + (p >> 4); }
    __device__ __forceinline__ void put(int p, float2 a, float2 b) const
    {
        sm[pad(p) * WP + cp] = make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ __forceinline__ void get(int p, float2& a, float2& b) const
    {
        const float4 v = sm[pad(p) * WP + cp];
        a = make_float2(v.x, v.y);
        b = make_float2(v.z, v.w);
    }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// One Stockham stage of two columns (va, vb) with a per-thread twiddle cache;
// the order of butterflies, twiddles and exchange positions is Stage's.
template <int L, int E, int DIR, int S>
struct PairStage {
    __device__ __forceinline__ static void run(float2 (&va)[E], float2 (&vb)[E], int t, const TwCache<L, E>& tw,
                                               const ColPairExchange& ex)
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
            float2 a[R], b[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                a[k] = va[q + k * Q];
                b[k] = vb[q + k * Q];
            }
            const int j = t + T * q;
            const int jm = j % Ns;
            if constexpr (Ns > 1) {
                twiddle_apply<R, DIR>(a, tw.w[S][q]);
                twiddle_apply<R, DIR>(b, tw.w[S][q]);
            }
            Dft<R, DIR>::run(a);
            Dft<R, DIR>::run(b);
            if constexpr (last) {
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    va[q + k * Q] = a[k];
                    vb[q + k * Q] = b[k];
                }
            } else {
                const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
                for (int k = 0; k < R; ++k) ex.put(base + k * Ns, a[k], b[k]);
            }
        }
        if constexpr (!last) {
            ex.sync();
#pragma unroll
            for (int m = 0; m < E; ++m) ex.get(t + T * m, va[m], vb[m]);
            ex.sync();
            PairStage<L, E, DIR, S + 1>::run(va, vb, t, tw, ex);
        }
    }
};

// Persistent: one CTA per resident slot, tiles blockIdx.x + k * gridDim.x,
// a ring of STAGES slots filled by 2D bulk tensor copies (mbarrier
// transaction counts, bounded waits that set kStatusTimeout and drain the
// copies in flight), the exchange in the consumed slot.  Requirements
// (checked by the host, as for col_tma_kernel in PAIR mode): S odd, Bs even,
// the base address 16-byte aligned; W even.
template <int L, int E, int DIR, int W, int STAGES>
__global__ void __launch_bounds__((W / 2) * (L / E)) col_tma2_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                    ColArgs a, long long ntiles)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    constexpr int T = L / E;
    constexpr int WP = W / 2;
    constexpr int ROWS_IN_MAP = L / 2;  // row pairs per tile
    constexpr int BOXR = ROWS_IN_MAP < 256 ? ROWS_IN_MAP : 256;
    constexpr int NBOX = ROWS_IN_MAP / BOXR;
    constexpr int WS = W + 2;  // slot row width (complex values)
    constexpr unsigned TILE_BYTES = (unsigned)L * WS * sizeof(float2);
    static_assert(ROWS_IN_MAP % BOXR == 0, "tile rows must split into boxes of <= 256 rows");
    static_assert(W % 2 == 0 && T % 2 == 0 && STAGES >= 2, "column pairs, row parity per thread, a two-slot ring");
    static_assert((size_t)(L + (L >> 4)) * WP * 16 <= TILE_BYTES, "the padded pair exchange must fit the slot");
    static_assert((WS * sizeof(float2)) % 16 == 0, "even rows' column pairs must stay 16-byte aligned in the slot");
    float2* ring = reinterpret_cast<float2*>(smraw);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smraw + (size_t)STAGES * TILE_BYTES);
    const int cp = threadIdx.x;
    const int t = threadIdx.y;
    const bool leader = (cp == 0 && t == 0);
    const long long ctiles = (a.C + W - 1) / W;
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
        mbar_arrive_expect_tx(&bars[s], TILE_BYTES);
        float2* slot = ring + (size_t)s * L * WS;
#pragma unroll
        for (int k = 0; k < NBOX; ++k) {
            const int y = (int)(b * ROWS_IN_MAP + k * BOXR);
            tma_load_2d(slot + (size_t)k * BOXR * WS, &tmap, (int)(2 * c0), y, &bars[s]);
            tma_load_2d(slot + (size_t)(L / 2) * WS + (size_t)k * BOXR * WS, &tmap, (int)(2 * (a.S + c0 - 1)), y,
                        &bars[s]);
        }
        ++n_issued;
    };

    if (leader) {
#pragma unroll
        for (int s = 0; s < STAGES - 1; ++s) issue(blockIdx.x + (long long)s * gridDim.x, s);
    }
    TwCache<L, E> twc;  // a thread's butterfly positions are the same in every tile
    twc.fill(a.tw, t);
    int stage = 0;
    unsigned phase = 0;
    long long n_consumed = 0;
    bool failed = false;
    const bool odd = t & 1;  // the parity of every row t + T*m of this thread
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
        const bool act_a = (c0 + 2 * cp) < a.C, act_b = (c0 + 2 * cp + 1) < a.C;
        float2* buf = ring + (size_t)stage * L * WS;
        float2 va[E], vb[E];
        if (!odd) {  // even rows: the box from c0, the pair 16-byte aligned
            const float4* src = reinterpret_cast<const float4*>(buf + 2 * cp);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const float4 x = src[((t >> 1) + (T / 2) * m) * (WS / 2)];
                va[m] = make_float2(x.x, x.y);
                vb[m] = make_float2(x.z, x.w);
            }
        } else {  // odd rows: the box from c0 - 1
            const float2* src = buf + (L / 2) * WS + 2 * cp + 1;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                va[m] = src[((t >> 1) + (T / 2) * m) * WS];
                vb[m] = src[((t >> 1) + (T / 2) * m) * WS + 1];
            }
        }
        __syncthreads();  // the slot now serves as the exchange buffer
        PairStage<L, E, DIR, 0>::run(va, vb, t, twc, ColPairExchange{reinterpret_cast<float4*>(buf), WP, cp});
        fence_proxy_async_smem();  // order this thread's shared accesses before the slot's next bulk copy
        float2* dst = (a.dst ? a.dst : a.data) + b * a.Bs + c0 + 2 * cp;
        const bool plain = a.mask23 == 0 && a.scale == 1.0f;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + T * m;
            float2 x = va[m], y = vb[m];
            if (!plain) {
                const float f = col_out_factor(j, L, a.scale, a.mask23);
                x = cscale(x, f);
                y = cscale(y, f);
            }
            float2* row = dst + (long long)j * a.S;
            if (!odd && act_b) {  // even row, both columns: one 16-byte store
                *reinterpret_cast<float4*>(row) = make_float4(x.x, x.y, y.x, y.y);
            } else {
                if (act_a) row[0] = x;
                if (act_b) row[1] = y;
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

template <int L, int E, int W, int STAGES, int DIR>
inline cudaError_t launch_col_tma2(const ColArgs& a, const CUtensorMap& map, cudaStream_t s)
{
    constexpr int T = L / E;
    // the even rows' 16-byte stores need an odd axis stride, an even batch
    // stride and 16-byte aligned bases
    if (!(a.S & 1) || (a.Bs & 1) || ((uintptr_t)a.data & 15) || ((uintptr_t)a.dst & 15)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)STAGES * L * (W + 2) * sizeof(float2) + STAGES * sizeof(unsigned long long);
    auto k = col_tma2_kernel<L, E, DIR, W, STAGES>;
    static PerDevice resident;  // resident CTAs on the device, queried once per device
    int ctas = 0;
    cudaError_t e = resident_ctas_per_device(resident, k, (W / 2) * T, smem, &ctas);
    if (e != cudaSuccess) return e;
    const long long ntiles = a.nb * ((a.C + W - 1) / W);
    if (ntiles <= 0) return cudaSuccess;
    const long long grid = ntiles < ctas ? ntiles : ctas;
    k<<<(unsigned)grid, dim3(W / 2, T), smem, s>>>(map, a, ntiles);
    return cudaGetLastError();
}

}  // namespace fft3d

// Radix-16 Stockham stages on the tensor cores (tcgen05, sm_100 family).
//
// A 16-point complex DFT y = F x is the real 32 x 32 product
//     [Re y; Im y] = G [Re x; Im x],   G = [[Fr, -Fi], [Fi, Fr]],
// so a stage of independent 16-point DFTs is a matrix product D = A B with
// A = one row [Re x, Im x] per DFT (K = 32), B = G^T, D in FP32 in tensor
// memory.  Operands are 16-bit, so FP32 values are split:
//   * split-BF16 (3 products): a = a_hi + a_lo with a_hi = bf16(a),
//     a_lo = bf16(a - a_hi); the same for G (split on the host from FP64);
//     D = A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 (the dropped
//     A_lo B_lo term and the split residuals are ~2^-16 relative);
//   * FP16 (1 product): each row scaled by a power of two so that its largest
//     |value| sits near 2^14, D = A_s B, the scale divided out again.
// Thread r of the CTA owns butterfly row r: it writes its row of A into
// shared memory in the K-major "no swizzle" layout (8-row x 16-byte core
// matrices, K-adjacent core matrices 128 bytes apart, row-adjacent ones 512
// bytes apart), one elected thread issues the MMAs of every 128-row tile and
// commits them to an mbarrier, and thread r reads row r of D back with
// tcgen05.ld (warp w reads TMEM lanes 32*(w%4).., tile w/4).  Twiddles between
// stages and any stage of another radix stay on the CUDA cores (FP32).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#include "launch_cache.h"
#include "stockham.cuh"
#include "tma.cuh"

namespace fft3d {

enum TcMode { TC_BF16X3 = 1, TC_F16 = 2 };

// Host-built operand tables: for each direction, the real 32 x 32 matrix G
// stored n-major (row n = output component, 32 k values), 16-bit values:
// [fwd hi][fwd lo][inv hi][inv lo] for BF16, [fwd][inv] (+ unused) for FP16.
constexpr int kTcTableElems = 4 * 32 * 32;

__device__ __forceinline__ int tc_kmaj_off(int row, int k)
{
    return ((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t tc_desc(unsigned saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;  // leading byte offset: next core matrix along K
    d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset: next 8 rows
    d |= (uint64_t)1 << 46;           // descriptor version
    return d;                         // no swizzle, base offset 0
}

__device__ __forceinline__ void tc_mma(unsigned dtmem, uint64_t da, uint64_t db, unsigned idesc, int accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_ld32(unsigned addr, float (&d)[32])
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) d[j] = __uint_as_float(r[j]);
}

// Per-CTA tensor-core context.
struct TcCtx {
    uint8_t* a_hi;               // tiles x 8 KB (A rows, high parts / FP16 scaled)
    uint8_t* a_lo;               // tiles x 8 KB (A rows, low parts; BF16 mode)
    uint8_t* b;                  // 2 (hi, lo) x 2 KB: G of this direction
    unsigned long long* bar;     // MMA completion
    unsigned tmem;               // base TMEM address (tiles x 32 columns)
    int tiles;                   // nthreads / 128
    unsigned* phase;             // mbarrier phase parity (shared)
    int* status;
    bool* failed;                // shared flag: a bounded wait gave up
};

template <int MODE>
__device__ __forceinline__ unsigned tc_idesc()
{
    // D F32 (bits 4-5 = 1); A/B BF16 (bits 7-9, 10-12 = 1) or F16 (0); both K-major;
    // N = 32 (bits 17-22: N >> 3); M = 128 (bits 24-28: M >> 4)
    constexpr unsigned ab = (MODE == TC_BF16X3) ? 1u : 0u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ uint16_t f2bf_bits(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }
__device__ __forceinline__ float bf_bits2f(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// One batched 16-point DFT stage on the tensor cores: every thread of the
// CTA passes its 16 (already twiddled) inputs in a[] and gets the DFT back.
// All threads of the CTA must call it (it synchronises the CTA).
template <int MODE>
__device__ __forceinline__ void tc_dft16(float2 (&a)[16], const TcCtx& c)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int tile = tid >> 7, row = tid & 127;
    uint8_t* ah = c.a_hi + tile * 8192;
    uint8_t* al = c.a_lo + tile * 8192;
    float scale = 1.f;
    if constexpr (MODE == TC_F16) {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) mx = fmaxf(mx, fmaxf(fabsf(a[k].x), fabsf(a[k].y)));
        int e = 0;
        frexpf(mx, &e);                      // mx in [2^(e-1), 2^e)
        scale = (mx > 0.f) ? ldexpf(1.f, 14 - e) : 1.f;  // largest |value| lands in [2^13, 2^14)
    }
    // write row `row` of A: k = 0..15 real parts, 16..31 imaginary parts; 4 chunks of 8 values
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        uint16_t hi[8], lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = kb * 8 + j;
            const float v = (k < 16) ? a[k].x : a[k - 16].y;
            if constexpr (MODE == TC_BF16X3) {
                hi[j] = f2bf_bits(v);
                lo[j] = f2bf_bits(v - bf_bits2f(hi[j]));
            } else {
                hi[j] = __half_as_ushort(__float2half_rn(v * scale));
                lo[j] = 0;
            }
        }
        const int off = tc_kmaj_off(row, kb * 8);
        uint4 vh, vl;
        vh.x = hi[0] | ((unsigned)hi[1] << 16);
        vh.y = hi[2] | ((unsigned)hi[3] << 16);
        vh.z = hi[4] | ((unsigned)hi[5] << 16);
        vh.w = hi[6] | ((unsigned)hi[7] << 16);
        *reinterpret_cast<uint4*>(ah + off) = vh;
        if constexpr (MODE == TC_BF16X3) {
            vl.x = lo[0] | ((unsigned)lo[1] << 16);
            vl.y = lo[2] | ((unsigned)lo[3] << 16);
            vl.z = lo[4] | ((unsigned)lo[5] << 16);
            vl.w = lo[6] | ((unsigned)lo[7] << 16);
            *reinterpret_cast<uint4*>(al + off) = vl;
        }
    }
    fence_proxy_async_smem();  // A rows written by threads, read by the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
        const unsigned idesc = tc_idesc<MODE>();
        const unsigned bh = smem_u32(c.b), bl = smem_u32(c.b + 2048);
        for (int q = 0; q < c.tiles; ++q) {
            const unsigned d = c.tmem + 32u * q;
            const unsigned ahq = smem_u32(c.a_hi + q * 8192), alq = smem_u32(c.a_lo + q * 8192);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) tc_mma(d, tc_desc(ahq + ks * 256), tc_desc(bh + ks * 256), idesc, ks);
            if constexpr (MODE == TC_BF16X3) {
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) tc_mma(d, tc_desc(ahq + ks * 256), tc_desc(bl + ks * 256), idesc, 1);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) tc_mma(d, tc_desc(alq + ks * 256), tc_desc(bh + ks * 256), idesc, 1);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(c.bar))
                     : "memory");
    }
    const unsigned ph = *c.phase;
    const bool ok = mbar_wait_bounded(c.bar, ph, 1u << 20);
    if (!ok) *c.failed = true;  // racy but idempotent: any thread may set it
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float d[32];
    const int warp = tid >> 5;
    tc_ld32(c.tmem + ((unsigned)(32 * (warp & 3)) << 16) + 32u * tile, d);
    const float inv = 1.f / scale;
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = make_float2(d[k] * inv, d[16 + k] * inv);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // every thread has read D and its A row may be rewritten
    if (tid == 0) *c.phase = ph ^ 1u;
    __syncthreads();
}

// Stockham stages as in stockham.cuh with E = 16 (one butterfly per thread
// per stage); radix-16 stages go to the tensor cores.
template <int L, int DIR, int MODE, int S>
struct TcStage {
    template <class Ex>
    __device__ __forceinline__ static void run(float2 (&v)[16], int t, const float2* __restrict__ tw, const Ex& ex,
                                               const TcCtx& c)
    {
        constexpr int E = 16;
        constexpr int NS = num_stages(L, E);
        constexpr int R = radix_at(L, E, S);
        constexpr int Ns = ns_at(L, E, S);
        constexpr int T = L / E;
        constexpr int Q = E / R;
        constexpr bool last = (S == NS - 1);
        if constexpr (R == 16) {
            float2 a[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = v[k];
            const int j = t;
            const int jm = j % Ns;
            if constexpr (Ns > 1) twiddle_inputs<16, DIR>(a, tw, jm * (L / (Ns * 16)));
            tc_dft16<MODE>(a, c);
            if constexpr (last) {
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = a[k];
            } else {
                const int base = (j / Ns) * Ns * 16 + jm;
#pragma unroll
                for (int k = 0; k < 16; ++k) ex.put(base + k * Ns, a[k]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                float2 a[R];
#pragma unroll
                for (int k = 0; k < R; ++k) a[k] = v[q + k * Q];
                const int j = t + T * q;
                const int jm = j % Ns;
                if constexpr (Ns > 1) twiddle_inputs<R, DIR>(a, tw, jm * (L / (Ns * R)));
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
        }
        if constexpr (!last) {
            ex.sync();
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = ex.get(t + T * m);
            ex.sync();
            TcStage<L, DIR, MODE, S + 1>::run(v, t, tw, ex, c);
        }
    }
};

// Column pass with tensor-core radix-16 stages: the plain column kernel's
// data movement (lanes along the contiguous columns) with E = 16.
// Shared memory: max(exchange L*W*8, A tiles) + G (4 KB) + barrier.
template <int L, int DIR, int MODE, int W>
__global__ void __launch_bounds__(W*(L / 16)) col_tc_kernel(ColArgs a, const uint16_t* __restrict__ gtab)
{
    extern __shared__ __align__(1024) uint8_t smraw[];
    constexpr int E = 16, T = L / E, NT = W * T;
    static_assert(NT % 128 == 0, "the CTA must fill whole 128-row MMA tiles");
    constexpr int TILES = NT / 128;
    constexpr size_t EX_BYTES = (size_t)L * W * sizeof(float2);
    constexpr size_t A_BYTES = (size_t)TILES * 8192 * (MODE == TC_BF16X3 ? 2 : 1);
    constexpr size_t REGION = EX_BYTES > A_BYTES ? EX_BYTES : A_BYTES;
    float2* exbuf = reinterpret_cast<float2*>(smraw);
    uint8_t* a_hi = smraw;
    uint8_t* a_lo = smraw + TILES * 8192;
    uint8_t* bmat = smraw + REGION;  // 4 KB
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(bmat + 4096);
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bar + 1);
    unsigned* phase = tmem_slot + 1;
    bool* failed = reinterpret_cast<bool*>(phase + 1);

    const int c = threadIdx.x, t = threadIdx.y;
    const int tid = t * W + c;
    // G of this direction into shared memory (K-major core layout, n rows)
    const uint16_t* g = gtab + (DIR < 0 ? 0 : 2 * 1024);
    for (int i = tid; i < 2 * 1024; i += NT) {
        const int part = i >> 10, n = (i >> 5) & 31, k = i & 31;
        *reinterpret_cast<uint16_t*>(bmat + part * 2048 + tc_kmaj_off(n, k)) = g[i];
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        *phase = 0;
        *failed = false;
    }
    if (tid < 32) {  // warp 0 allocates TILES * 32 TMEM columns
        constexpr unsigned cols = TILES * 32 <= 32 ? 32 : (TILES * 32 <= 64 ? 64 : (TILES * 32 <= 128 ? 128 : 256));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    TcCtx ctx{a_hi, a_lo, bmat, bar, *tmem_slot, TILES, phase, a.status, failed};

    const long long ctiles = (a.C + W - 1) / W;
    const long long b = blockIdx.x / ctiles;
    const long long c0 = (blockIdx.x - b * ctiles) * W;
    const bool active = (c0 + c) < a.C;
    float2* base = a.data + b * a.Bs + c0 + c;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = active ? base[(long long)(t + T * m) * a.S] : make_float2(0.f, 0.f);
    ColExchange ex{exbuf, W, c};
    TcStage<L, DIR, MODE, 0>::run(v, t, a.tw, ex, ctx);
    if (active && !*failed) {
        float2* out = (a.dst ? a.dst : a.data) + b * a.Bs + c0 + c;
#pragma unroll
        for (int m = 0; m < E; ++m)
            out[(long long)(t + T * m) * a.S] = cscale(v[m], col_out_factor(t + T * m, L, a.scale, a.mask23));
    }
    if (tid == 0 && *failed) atomicOr(a.status, kStatusTimeout);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid < 32) {
        constexpr unsigned cols = TILES * 32 <= 32 ? 32 : (TILES * 32 <= 64 ? 64 : (TILES * 32 <= 128 ? 128 : 256));
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(ctx.tmem), "n"(cols) : "memory");
    }
}

template <int L, int DIR, int MODE, int W>
inline size_t col_tc_smem()
{
    constexpr int TILES = W * (L / 16) / 128;
    constexpr size_t EX_BYTES = (size_t)L * W * sizeof(float2);
    constexpr size_t A_BYTES = (size_t)TILES * 8192 * (MODE == TC_BF16X3 ? 2 : 1);
    constexpr size_t REGION = EX_BYTES > A_BYTES ? EX_BYTES : A_BYTES;
    return REGION + 4096 + 64;
}

template <int L, int W, int MODE, int DIR>
inline cudaError_t launch_col_tc(const ColArgs& a, const uint16_t* gtab, cudaStream_t s)
{
    constexpr int T = L / 16;
    const size_t smem = col_tc_smem<L, DIR, MODE, W>();
    auto k = col_tc_kernel<L, DIR, MODE, W>;
    static PerDevice limit;  // the shared memory limit, raised once per device
    cudaError_t e = smem_limit_per_device(limit, k, smem);
    if (e != cudaSuccess) return e;
    const long long tiles = a.nb * ((a.C + W - 1) / W);
    if (tiles <= 0) return cudaSuccess;
    k<<<(unsigned)tiles, dim3(W, T), smem, s>>>(a, gtab);
    return cudaGetLastError();
}

}  // namespace fft3d

// Fused plane kernel: the 2D transform of every n0-plane (Sec. 2.1 step 1:
// the n2-axis real transform of each row and the n1-axis complex transform of
// each column) in ONE persistent launch, with the plane kept on chip (L2)
// between its two halves.
//
// A plane (n1 x H complex values; 1 MiB at 512^3) does not fit in one SM's
// shared memory, so the two halves run as separate work items of one grid:
//   forward: row items (r2c of RPI rows, DRAM -> L2) produce plane p;
//            column items (n1-axis c2c of WC columns, in place, L2 -> L2)
//            consume it;
//   inverse: column items (n1-axis c2c, in place, DRAM -> L2) produce plane
//            p; row items (c2r, L2 -> DRAM) consume it.
// Items are numbered slot by slot: slot s holds the producer items of plane s
// followed by the consumer items of plane s - lag, and every CTA walks item
// indices blockIdx.x, blockIdx.x + gridDim.x, ...  A consumer item first
// waits until the per-plane counter shows all producer items of its plane
// done; since producers of plane p sit lag slots earlier in the order, the
// wait is normally already satisfied, and the plane's data is still in L2, so
// DRAM sees one read and one write per element for the whole 2D step.
//
// Co-residency of all CTAs is guaranteed by a cooperative launch, and the
// item order only ever waits on lower-numbered items, so progress is assured;
// still, every wait is bounded: a wait that gives up sets kStatusTimeout in
// the device status word and the CTA returns (the plane's output is then
// undefined, the host sees FFT3D_ERR_TIMEOUT from fft3d_query_device_status).
#pragma once
#include "kernels.cuh"
#include "plane.h"

namespace fft3d {

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int LR>
struct PlaneSmem {
    // row items need RPI padded rows; column items need LC * WC values
    static constexpr size_t bytes(int rpi, int lc, int wc)
    {
        const size_t r = (size_t)rpi * RowLayout<LR>::stride * sizeof(float2);
        const size_t c = (size_t)lc * wc * sizeof(float2);
        return r > c ? r : c;
    }
};

// LR = n2/2 (row complex length), ER its elements per thread; LC = n1 (column
// length), EC its elements per thread; NT threads per CTA; DIR -1 forward.
template <int LR, int ER, int LC, int EC, int NT, int DIR, int MINB = 1024 / NT>
__global__ void __launch_bounds__(NT, MINB) plane_kernel(PlaneArgs a)
{
    extern __shared__ __align__(16) float2 sm[];
    constexpr int TR = LR / ER;
    constexpr int RPI = NT / TR;  // rows per row item
    constexpr int TC = LC / EC;
    constexpr int WC = NT / TC;   // columns per column item
    static_assert(NT % TR == 0 && NT % TC == 0 && NT % 32 == 0, "item shapes must tile the CTA");
    const int tid = threadIdx.x;
    const int H = a.H;
    const int RI = (LC + RPI - 1) / RPI;  // row items per plane
    const int CI = (H + WC - 1) / WC;     // column items per plane
    const int NP = DIR < 0 ? RI : CI;     // producer items per plane
    const int Z = RI + CI;
    const long long nitems = (a.planes + a.lag) * Z;
    __shared__ int s_fail;
    __shared__ long long s_item;
    if (tid == 0) s_fail = 0;
    int* ticket = a.counters + ((a.planes + 1) & ~1LL);  // 8-byte aligned
    const int NC = Z - NP;                                // consumer items per plane
    const bool ring = DIR > 0 && a.ring_planes > 0;

    for (;;) {
        // claim the next item: item i starts only after every item < i started
        if (tid == 0) s_item = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(ticket), 1ull);
        __syncthreads();
        const long long i = s_item;
        if (i >= nitems) break;
        const long long slot = i / Z;
        const int j = (int)(i - slot * Z);
        const bool producer = j < NP;
        const long long p = producer ? slot : slot - a.lag;
        if (p >= 0 && p < a.planes) {
            const int sub = producer ? j : j - NP;
            // consumers wait for their plane's producers; with the inverse
            // ring, producers wait until the slot's previous plane is consumed
            const long long wp = producer ? p - a.ring_planes : p;
            const int need = producer ? NP + NC : NP;
            if (!producer || (ring && wp >= 0)) {
                if (tid == 0) {
                    unsigned n = 0;
                    while (ld_acquire_gpu(&a.counters[wp]) < need) {
                        if (++n > a.wait_limit) {
                            s_fail = 1;
                            atomicOr(a.status, kStatusTimeout);
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                __syncthreads();
                if (s_fail) return;
            }
            // inverse with a ring: the n1 results of plane p live in ring slot p mod ring_planes
            float2* mid = (DIR < 0 || a.ring_planes == 0)
                              ? reinterpret_cast<float2*>(DIR < 0 ? a.out : const_cast<void*>(a.in)) + p * LC * H
                              : a.ring + (p % a.ring_planes) * LC * H;
            const bool row_item = (DIR < 0) == producer;
            if (row_item) {
                const int rr = tid / TR, t = tid - rr * TR;
                const int r = sub * RPI + rr;
                const long long row = p * LC + r;
                float2* smr = sm + rr * RowLayout<LR>::stride;
                if (DIR < 0)
                    row_r2c_body<LR, ER, false>(reinterpret_cast<const float2*>(a.in) + row * LR, mid + (long long)r * H,
                                                r < LC, t, tid & 31, smr, a.tw_row, a.twpack);
                else
                    row_c2r_body<LR, ER, true>(mid + (long long)r * H, reinterpret_cast<float2*>(a.out) + row * LR,
                                               r < LC, t, tid & 31, smr, a.tw_row, a.twpack);
            } else {
                const int tc = tid / WC, c = tid - tc * WC;
                const int c0 = sub * WC;
                ColExchange ex{sm, WC, c};
                if (DIR < 0) {
                    col_body<LC, EC, DIR, true>(mid + c0 + c, H, c0 + c < H, tc, a.tw_col, 1.0f, ex);
                } else {
                    // read the plane from the input, write the ring slot (or in place)
                    float2* src = reinterpret_cast<float2*>(const_cast<void*>(a.in)) + p * LC * H + c0 + c;
                    if (ring)  // the input is only read in this launch: read-only path
                        col_body_to<LC, EC, DIR, false>(src, mid + c0 + c, H, c0 + c < H, tc, a.tw_col, ex);
                    else
                        col_body_to<LC, EC, DIR, true>(src, mid + c0 + c, H, c0 + c < H, tc, a.tw_col, ex);
                }
            }
            if (producer || ring) {
                __threadfence();  // this thread's stores (and reads) complete before the count
                __syncthreads();
                if (tid == 0 && p != a.skip_plane) atomicAdd(&a.counters[p], 1);
            }
        }
        __syncthreads();  // shared memory and s_item are reused by the next item
    }
}

template <int LR, int ER, int LC, int EC, int NT, int DIR, int MINB = 1024 / NT>
inline cudaError_t launch_plane(const PlaneArgs& a, cudaStream_t s)
{
    constexpr int TR = LR / ER, RPI = NT / TR, TC = LC / EC, WC = NT / TC;
    const size_t smem = PlaneSmem<LR>::bytes(RPI, LC, WC);
    auto k = plane_kernel<LR, ER, LC, EC, NT, DIR, MINB>;
    static PerDevice resident;  // resident CTAs on the device, queried once per device
    int ctas = 0;
    cudaError_t e = resident_ctas_per_device(resident, k, NT, smem, &ctas);
    if (e != cudaSuccess) return e;
    const int RI = (LC + RPI - 1) / RPI, CI = (a.H + WC - 1) / WC;
    const int Z = RI + CI;
    // The resident CTAs span about grid/Z slots of the item order at any time;
    // the consumers must trail the producers by more than that, or they wait.
    PlaneArgs b = a;
    const long long span = ((long long)ctas + Z - 1) / Z;
    b.lag = (int)(span + a.lag);
    if (b.ring_planes <= 2 * b.lag) b.ring_planes = 0;  // ring too short to trail the consumers: work in place
    const long long nitems = (b.planes + b.lag) * (long long)Z;
    long long grid = ctas;
    if (grid > nitems) grid = nitems;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident: waits can always be met
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, b);
}

}  // namespace fft3d

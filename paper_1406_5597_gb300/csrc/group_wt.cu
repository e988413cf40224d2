// Work-table kernel of a grouped transform of uneven sizes: the passes of all
// sizes (each size: row r2c, n1 pass, n0 pass forward; the reverse inverse,
// Sec. 2.1) run in ONE persistent launch.  The work is a table of segments
// (one pass of one size), each a list of items (a tile of rows or columns of
// 256 threads' worth); CTAs take items in table order from a global ticket.
// An item of a pass may start only when every item of the same size's
// previous pass is done: its CTA waits on that segment's completion counter
// (bounded: a wait that gives up sets kStatusTimeout and the CTA stops).
// Table order puts every segment after the one it depends on, so the items a
// waiting CTA needs were handed out earlier to CTAs that are running (the grid
// is no larger than the resident CTAs), and the small sizes' passes overlap
// the large sizes' ones instead of each pass being a launch of its own.
// Data written by one item is read by later items of other CTAs in the same
// launch, so the bodies load through L2 (ld.global.cg), and a completed item
// is published with a device-scope fence before its counter is raised.
#include "group_wt.h"
#include "kernels.cuh"

namespace fft3d {

namespace {

constexpr int kWtThreads = 256;
constexpr unsigned kWtMaxWaits = 1u << 22;  // ~1 s of polling at 256 ns

template <int L, int E, int DIR>
__device__ __forceinline__ void wt_col(const WtSeg& g, long long item, float2* sm)
{
    constexpr int T = L / E, W = kWtThreads / T;
    static_assert(kWtThreads % T == 0, "columns of whole thread groups");
    const int tid = threadIdx.x, c = tid % W, t = tid / W;
    const long long ctiles = (g.C + W - 1) / W;
    const long long b = item / ctiles;
    const long long c0 = (item - b * ctiles) * W;
    const bool active = (c0 + c) < g.C;
    col_body<L, E, DIR, true>(g.data + b * g.Bs + c0 + c, g.S, active, t, g.tw, 1.0f, ColExchange{sm, W, c});
}

template <int L, int E, int DIR>
__device__ __forceinline__ void wt_row(const WtSeg& g, long long item, float2* sm)
{
    constexpr int T = L / E, R = kWtThreads / T, H = L + 1;
    static_assert(T <= 32 && 32 % T == 0, "warp-resident rows");
    const int tid = threadIdx.x, r = tid / T, t = tid % T;
    const long long row = item * R + r;
    const bool active = row < g.rows;
    float2* smr = sm + r * RowLayout<L>::stride;
    if constexpr (DIR < 0)
        row_r2c_body<L, E, kLdCg>(reinterpret_cast<const float2*>(g.in) + row * g.rs,
                                  reinterpret_cast<float2*>(g.out) + row * H, active, t, tid & 31, smr, g.tw,
                                  g.twpack);
    else
        row_c2r_body<L, E, kLdCg>(reinterpret_cast<const float2*>(g.in) + row * H,
                                  reinterpret_cast<float2*>(g.out) + row * g.rs, active, t, tid & 31, smr, g.tw,
                                  g.twpack);
}

// The bodies: rows of length n2/2 in {32, 48, 64, 80, 96} and columns of length
// {64, 96, 128, 160, 192} (the 2^k, 3 2^k and 5 2^k grids of a multi-size
// group), each forward and inverse, with the element counts per thread of
// the specialised single-size kernels.
struct BodyDesc {
    bool row;
    int L, E, dir;
};
constexpr BodyDesc kBodies[] = {
    {true, 32, 8, -1},   {true, 32, 8, 1},   {true, 48, 12, -1},  {true, 48, 12, 1},  {true, 64, 8, -1},
    {true, 64, 8, 1},    {true, 80, 20, -1}, {true, 80, 20, 1},   {true, 96, 24, -1}, {true, 96, 24, 1},
    {false, 64, 8, -1},  {false, 64, 8, 1},  {false, 96, 24, -1}, {false, 96, 24, 1}, {false, 128, 8, -1},
    {false, 128, 8, 1},  {false, 160, 20, -1}, {false, 160, 20, 1}, {false, 192, 24, -1}, {false, 192, 24, 1},
};
constexpr int kNumBodies = sizeof(kBodies) / sizeof(kBodies[0]);

template <int I>
__device__ __forceinline__ void run_body(const WtSeg& g, long long item, float2* sm)
{
    constexpr BodyDesc d = kBodies[I];
    if constexpr (d.row) wt_row<d.L, d.E, d.dir>(g, item, sm);
    else wt_col<d.L, d.E, d.dir>(g, item, sm);
}

template <int I = 0>
__device__ __forceinline__ void dispatch(int body, const WtSeg& g, long long item, float2* sm)
{
    if constexpr (I < kNumBodies) {
        if (body == I) run_body<I>(g, item, sm);
        else dispatch<I + 1>(body, g, item, sm);
    }
}

template <int I = 0>
constexpr size_t body_smem_max()
{
    if constexpr (I == kNumBodies) {
        return 0;
    } else {
        constexpr BodyDesc d = kBodies[I];
        constexpr int T = d.L / d.E;
        constexpr size_t here = d.row ? (size_t)(kWtThreads / T) * (size_t)(d.L + 1 + ((d.L + 1) >> 4) + 1) * 8
                                      : (size_t)d.L * (kWtThreads / T) * 8;
        constexpr size_t rest = body_smem_max<I + 1>();
        return here > rest ? here : rest;
    }
}
constexpr size_t kWtSmem = body_smem_max();

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kWtThreads, 3) wt_kernel(const __grid_constant__ WtTable tab, WtCounters* ctr)
{
    extern __shared__ __align__(16) float2 sm[];
    __shared__ long long s_item;
    __shared__ int s_seg;
    __shared__ int s_ok;
    // thread 0 takes the next ticket while the current item runs, so the
    // atomic's round trip is hidden behind the item's work
    long long next = threadIdx.x == 0 ? (long long)atomicAdd(&ctr->ticket, 1ull) : 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long it = next;
            if (it < tab.total) next = (long long)atomicAdd(&ctr->ticket, 1ull);
            int sg = -1, ok = 1;
            if (it < tab.total) {
                sg = 0;
                while (sg + 1 < tab.nseg && it >= tab.seg[sg + 1].first) ++sg;
                const int d = tab.seg[sg].dep;
                if (d >= 0) {
                    const int need = (int)tab.seg[sg].need;
                    unsigned tries = 0;
                    while (ld_acquire(&ctr->done[d]) < need) {
                        if (++tries > kWtMaxWaits || ld_acquire(&ctr->status) != 0) {
                            ok = 0;
                            atomicOr(&ctr->status, kStatusTimeout);
                            break;
                        }
                        __nanosleep(256);
                    }
                }
            }
            s_item = it;
            s_seg = sg;
            s_ok = ok;
        }
        __syncthreads();
        const long long it = s_item;
        const int sg = s_seg;
        if (it >= tab.total || !s_ok) break;
        const WtSeg& g = tab.seg[sg];
        dispatch(g.body, g, it - g.first, sm);
        __threadfence();  // publish this thread's results device-wide
        __syncthreads();  // every thread of the item is done (and done with s_item and sm)
        if (threadIdx.x == 0) atomicAdd(&ctr->done[sg], 1);
    }
}

}  // namespace

int wt_body_index(bool row, int L, int dir, int* per_item)
{
    for (int i = 0; i < kNumBodies; ++i)
        if (kBodies[i].row == row && kBodies[i].L == L && kBodies[i].dir == dir) {
            if (per_item) *per_item = kWtThreads / (kBodies[i].L / kBodies[i].E);
            return i;
        }
    return -1;
}

cudaError_t launch_wt(const WtTable& tab, WtCounters* ctr, cudaStream_t s)
{
    static PerDevice resident;  // resident CTAs on the device, queried once per device
    int ctas = 0;
    cudaError_t e = resident_ctas_per_device(resident, wt_kernel, kWtThreads, kWtSmem, &ctas);
    if (e != cudaSuccess) return e;
    if (tab.total <= 0) return cudaSuccess;
    const long long grid = tab.total < ctas ? tab.total : ctas;
    wt_kernel<<<(unsigned)grid, kWtThreads, kWtSmem, s>>>(tab, ctr);
    return cudaGetLastError();
}

}  // namespace fft3d

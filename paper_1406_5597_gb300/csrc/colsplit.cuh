// Column transform of a long strided axis split over a thread-block cluster:
// the n0 pass of Sec. 2.2 (the axis transformed where it lies, at stride
// n1*(n2/2+1)) for L >= 1024, where a tile of W adjacent columns x L rows is
// too big for one SM to hold while a second tile is in flight (2048 x 8
// complex values = 128 KB).
//
// The C CTAs of a cluster share one tile, split the decimation-in-time way
// (W = exp(-2 pi i / L), k = k' + (L/C) s, k' in [0, L/C), s in [0, C)):
//
//   X[k' + (L/C) s] = sum_b F_C^{b s} . W^{b k'} . sum_a x[C a + b] W_{L/C}^{a k'}
//
// CTA b loads the rows C a + b (a in [0, L/C)) of the W columns, runs the
// L/C-point transforms in registers (exchanges in its own shared memory) and
// multiplies by W^{b k'}.  The final radix-C step of the outputs k' in
// [r L/C^2, (r+1) L/C^2) belongs to CTA r; thread (c, t) holds k' = t + T m,
// so those k' are its registers m in [r E/C, (r+1) E/C), and it pushes them
// into CTA r's receive buffer (st.shared::cluster, thread to the same thread
// index: conflict-free).  After a cluster barrier every CTA forms the
// radix-C DFTs of its k' range and writes C output rows per k'.
//
// A CTA holds L/C x W values (64 KB at L/C = 1024, W = 8), so two CTAs of
// different clusters share an SM and one CTA's loads overlap the other's
// butterflies and stores: the plain one-tile-per-CTA kernel at L = 2048 has a
// single 512-thread CTA per SM (25 % of the warp slots) and its loads wait on
// its own butterflies.  DRAM still sees one read and one write per element.
// Two hardware cluster barriers per tile (the first one's arrival is made at
// the start, so that every CTA of the cluster runs before any remote store);
// no spin-waits.
#pragma once
#include "cluster.cuh"
#include "kernels.cuh"

namespace fft3d {

template <int L, int C, int E, int W>
struct ColSplitGeom {
    static constexpr int LC = L / C;  // rows per CTA
    static constexpr int T = LC / E;  // threads per column
    static constexpr int NT = W * T;  // threads per CTA
    static constexpr int EC = E / C;  // registers each destination CTA takes
    static constexpr size_t xbytes = (size_t)LC * W * sizeof(float2);
    static constexpr size_t rbytes = (size_t)(C - 1) * EC * NT * sizeof(float2);
    static constexpr size_t smem = xbytes + rbytes;
    static_assert(L % C == 0 && LC % E == 0, "C CTAs of E values per thread must cover the axis");
    static_assert(E % C == 0, "every destination CTA takes E/C registers of each thread");
    static_assert(C >= 2 && C <= 8, "portable cluster sizes");
    static_assert(NT <= 1024, "too many threads");
};

template <int L, int C, int E, int W, int DIR>
__global__ void __launch_bounds__(ColSplitGeom<L, C, E, W>::NT, 2) col_split_kernel(ColArgs a)
{
    using G = ColSplitGeom<L, C, E, W>;
    constexpr int LC = G::LC, T = G::T, NT = G::NT, EC = G::EC;
    extern __shared__ __align__(16) float2 sm[];
    float2* xbuf = sm;           // LC x W: exchanges of the sub-transforms
    float2* rbuf = sm + LC * W;  // (C-1) x EC x NT: values pushed here by the other CTAs
    const int c = threadIdx.x, t = threadIdx.y;
    const int tid = t * W + c;
    const int rank = (int)cluster_ctarank();
    cluster_arrive_relaxed();  // paired with the wait before the first remote store
    const long long ctiles = (a.C + W - 1) / W;
    const long long tile = blockIdx.x / C;
    const long long b = tile / ctiles;
    const long long c0 = (tile - b * ctiles) * W;
    const bool active = (c0 + c) < a.C;
    const float2* src = a.data + b * a.Bs + c0 + c;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = active ? src[(long long)(C * (t + T * m) + rank) * a.S] : make_float2(0.f, 0.f);
    // L/C-point transforms of the rows C a + rank; the table holds W_L, so the
    // sub-transform reads every C-th entry
    fft_group<LC, E, DIR, C>(v, t, a.tw, ColExchange{xbuf, W, c});
    if (rank > 0) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = twiddle<DIR>(v[m], __ldg(&a.tw[rank * (t + T * m)]));
    }
    cluster_wait_acquire();  // every CTA of the cluster has started
    // registers m in [r EC, (r+1) EC) go to CTA r, into its slot for this CTA
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int r = m / EC;
        if (r != rank) {
            const int slot = rank - (rank > r ? 1 : 0);
            dsmem_st(dsmem_map(&rbuf[(slot * EC + m % EC) * NT + tid], (unsigned)r), v[m]);
        }
    }
    cluster_arrive_release();
    cluster_wait_acquire();  // every CTA's pushes are visible
    float2* dst = (a.dst ? a.dst : a.data) + b * a.Bs + c0 + c;
#pragma unroll
    for (int r = 0; r < C; ++r) {
        if (r != rank) continue;
#pragma unroll
        for (int q = 0; q < EC; ++q) {
            float2 z[C];
#pragma unroll
            for (int s = 0; s < C; ++s)
                z[s] = (s == r) ? v[r * EC + q] : rbuf[((s - (s > r ? 1 : 0)) * EC + q) * NT + tid];
            Dft<C, DIR>::run(z);
            const int kp = t + T * (r * EC + q);
            if (active) {
                if (a.mask23 == 0 && a.scale == 1.0f) {
#pragma unroll
                    for (int s = 0; s < C; ++s) dst[(long long)(kp + LC * s) * a.S] = z[s];
                } else {
#pragma unroll
                    for (int s = 0; s < C; ++s)
                        dst[(long long)(kp + LC * s) * a.S] =
                            cscale(z[s], col_out_factor(kp + LC * s, L, a.scale, a.mask23));
                }
            }
        }
    }
}

// One tile of W columns per cluster of C CTAs; w (the runtime width of the
// plain kernel) does not apply.
template <int L, int C, int E, int W, int DIR>
inline cudaError_t launch_col_split(const ColArgs& a, int /*w*/, cudaStream_t s)
{
    using G = ColSplitGeom<L, C, E, W>;
    auto k = col_split_kernel<L, C, E, W, DIR>;
    static PerDevice limit;  // the shared memory limit, raised once per device
    cudaError_t e = smem_limit_per_device(limit, k, G::smem);
    if (e != cudaSuccess) return e;
    const long long tiles = a.nb * ((a.C + W - 1) / W);
    if (tiles <= 0) return cudaSuccess;
    if (tiles > 0x7fffffffLL / C) return cudaErrorInvalidConfiguration;  // grid x extent
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tiles * C));
    cfg.blockDim = dim3(W, G::T);
    cfg.dynamicSmemBytes = G::smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace fft3d

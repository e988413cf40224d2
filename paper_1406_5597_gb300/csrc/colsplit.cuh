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

// ---------------------------------------------------------------------------
// TMA-fed form of the split: every CTA of the cluster runs the 512-row
// sub-transform of the persistent TMA column kernel (16-column tiles of
// 128-byte rows, a two-slot ring kept full by one elected thread, bulk tensor
// copies counted on mbarriers), L = 512 C.  The residue-r rows of a tile are
// rows 512 b + a of a 2D view of the volume with base r*P (P = n1 (n2/2+1))
// and row stride C*P, so each CTA reads its own tensor map.  Clusters are
// persistent: cluster i takes tiles i, i + nclusters, ...
//
// Per tile: wait for the slot (bounded), agree across the cluster that every
// CTA's copies arrived (each CTA writes its flag into every peer's shared
// memory before the first cluster barrier; a failed wait on any CTA makes
// the whole cluster stop after that barrier, so no CTA is left waiting at a
// later one), refill the other slot, transform in registers with the slot as
// exchange buffer, twiddle, push the peers' k' ranges (thread to thread),
// second cluster barrier, radix-C step of the own k' range, stores straight
// from registers.  The first barrier of the next tile also tells a CTA that
// its peers have read the previous tile's pushes.  A wait that gives up sets
// kStatusTimeout and the CTA drains its own copies (bounded) before it ends.
// Requirements (checked by the host): P even (16-byte aligned residue
// bases), Bs = L*P.
// ---------------------------------------------------------------------------
constexpr int kSplitLC = 512;  // rows per CTA
constexpr int kSplitE = 32;    // values per thread
constexpr int kSplitW = 16;    // columns per tile (128-byte rows)

template <int C>
struct TmaSplitGeom {
    static constexpr int L = kSplitLC * C;
    static constexpr int T = kSplitLC / kSplitE;  // 16 threads per column
    static constexpr int NT = kSplitW * T;         // 256 threads
    static constexpr int STAGES = 2;
    static constexpr unsigned TILE_BYTES = (unsigned)kSplitLC * kSplitW * sizeof(float2);  // 64 KB
    // k' split: CTA r takes registers m in [mlo(r), mlo(r+1))
    __host__ __device__ static constexpr int mlo(int r) { return r * kSplitE / C; }
    static constexpr int MAXEC = (kSplitE + C - 1) / C;
    __host__ __device__ static constexpr int owner(int m)
    {
        int r = 0;
        while (r + 1 < C && m >= mlo(r + 1)) ++r;
        return r;
    }
    static constexpr size_t ring = (size_t)STAGES * TILE_BYTES;
    static constexpr size_t rbytes = (size_t)(C - 1) * MAXEC * NT * sizeof(float2);
    static constexpr size_t smem = ring + rbytes + 64 + 16 * C;  // + mbarriers + agreement flags
};

template <int C, int DIR>
__global__ void __launch_bounds__(TmaSplitGeom<C>::NT) col_tma_split_kernel(const __grid_constant__ SplitMaps maps,
                                                                           ColArgs a, long long ntiles)
{
    using G = TmaSplitGeom<C>;
    constexpr int L = G::L, LC = kSplitLC, E = kSplitE, W = kSplitW, T = G::T, NT = G::NT, STAGES = G::STAGES;
    constexpr int MAXEC = G::MAXEC;
    constexpr int BOXR = 256, NBOX = LC / BOXR;
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2* ring = reinterpret_cast<float2*>(smraw);
    float2* rbuf = reinterpret_cast<float2*>(smraw + G::ring);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smraw + G::ring + G::rbytes);
    int* okf = reinterpret_cast<int*>(smraw + G::ring + G::rbytes + 64);
    const int c = threadIdx.x, t = threadIdx.y;
    const int tid = t * W + c;
    const bool leader = (tid == 0);
    const int rank = (int)cluster_ctarank();
    const CUtensorMap* map = &maps.map[rank];
    const long long ctiles = (a.C + W - 1) / W;
    const long long cl = cluster_index(), ncl = cluster_count();
    long long n_issued = 0;

    if (leader) {
        prefetch_tensormap(map);
#pragma unroll
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    cluster_sync_all();  // every CTA of the cluster runs before the first remote store

    auto issue = [&](long long tile, int s) {
        if (tile >= ntiles) return;
        const long long b = tile / ctiles;
        const long long c0 = (tile - b * ctiles) * W;
        mbar_arrive_expect_tx(&bars[s], G::TILE_BYTES);
        float2* slot = ring + (size_t)s * LC * W;
#pragma unroll
        for (int k = 0; k < NBOX; ++k)
            tma_load_2d(slot + (size_t)k * BOXR * W, map, (int)(2 * c0), (int)(b * LC + k * BOXR), &bars[s]);
        ++n_issued;
    };

    if (leader) issue(cl, 0);
    TwCache<LC, E, C> twc;  // the sub-transform's twiddles (table of length L: every C-th entry)
    twc.fill(a.tw, t);
    int stage = 0;
    unsigned phase = 0;
    long long n_consumed = 0;
    bool failed = false;
    for (long long tile = cl; tile < ntiles; tile += ncl) {
        const bool ok = __syncthreads_and(mbar_wait_bounded(&bars[stage], phase, kMbarMaxTries));
        // cluster-wide agreement that every CTA has its tile
        if (leader) {
#pragma unroll
            for (int p = 0; p < C; ++p) {
                if (p == rank) okf[rank] = ok;
                else asm volatile("st.shared::cluster.u32 [%0], %1;\n" ::"r"(dsmem_map(&okf[rank], (unsigned)p)),
                                  "r"((unsigned)ok)
                                  : "memory");
            }
        }
        cluster_arrive_release();
        cluster_wait_acquire();
        bool all_ok = true;
#pragma unroll
        for (int p = 0; p < C; ++p) all_ok = all_ok && (okf[p] != 0);
        if (!all_ok) {
            failed = true;
            if (ok) ++n_consumed;
            break;
        }
        ++n_consumed;
        if (leader) issue(tile + ncl, stage ^ 1);  // the other slot was consumed in the previous iteration
        const long long b = tile / ctiles;
        const long long c0 = (tile - b * ctiles) * W;
        const bool active = (c0 + c) < a.C;
        float2* buf = ring + (size_t)stage * LC * W;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = buf[(t + T * m) * W + c];
        __syncthreads();  // the slot now serves as the exchange buffer
        fft_group<LC, E, DIR, C>(v, t, twc, ColExchange{buf, W, c});
        fence_proxy_async_smem();  // order this thread's shared accesses before the slot's next bulk copy
        if (rank > 0) {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = twiddle<DIR>(v[m], __ldg(&a.tw[rank * (t + T * m)]));
        }
        // push registers m to their owner CTA (its slot for this CTA)
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int r = G::owner(m);
            if (r != rank) {
                const int slot = rank - (rank > r ? 1 : 0);
                dsmem_st(dsmem_map(&rbuf[(slot * MAXEC + (m - G::mlo(r))) * NT + tid], (unsigned)r), v[m]);
            }
        }
        cluster_arrive_release();
        cluster_wait_acquire();  // every peer's pushes are visible
        float2* dst = (a.dst ? a.dst : a.data) + b * a.Bs + c0 + c;
#pragma unroll
        for (int r = 0; r < C; ++r) {
            if (r != rank) continue;
#pragma unroll
            for (int m = G::mlo(r); m < G::mlo(r + 1); ++m) {
                float2 z[C];
#pragma unroll
                for (int s = 0; s < C; ++s)
                    z[s] = (s == r) ? v[m] : rbuf[((s - (s > r ? 1 : 0)) * MAXEC + (m - G::mlo(r))) * NT + tid];
                Dft<C, DIR>::run(z);
                const int kp = t + T * m;
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
        stage ^= 1;
        if (stage == 0) phase ^= 1u;
    }
    if (failed && leader) {
        atomicOr(a.status, kStatusTimeout);
        // drain: wait (bounded) for every copy issued but not consumed
        for (long long k = n_consumed; k < n_issued; ++k)
            mbar_wait_bounded(&bars[k % STAGES], (unsigned)((k / STAGES) & 1), kMbarMaxTries);
    }
}

// Persistent clusters of C CTAs, as many as are co-resident; one tensor map
// per residue.  Requirements: P = a.S / C even, a.Bs = L * a.S / C.
template <int C, int DIR>
inline cudaError_t launch_col_tma_split(const ColArgs& a, const SplitMaps& maps, cudaStream_t s)
{
    using G = TmaSplitGeom<C>;
    auto k = col_tma_split_kernel<C, DIR>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kSplitW, G::T);
    cfg.dynamicSmemBytes = G::smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static PerDevice resident;  // co-resident clusters, queried once per device
    int max_clusters = 0;
    cudaError_t e = per_device(resident, &max_clusters, [&](int, int* v) {
        cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
        if (r != cudaSuccess) return r;
        cfg.gridDim = dim3(C * 64);
        return cudaOccupancyMaxActiveClusters(v, k, &cfg);
    });
    if (e != cudaSuccess) return e;
    const long long ntiles = a.nb * ((a.C + kSplitW - 1) / kSplitW);
    if (ntiles <= 0) return cudaSuccess;
    const long long ncl = ntiles < max_clusters ? ntiles : max_clusters;
    cfg.gridDim = dim3((unsigned)(ncl * C));
    return cudaLaunchKernelEx(&cfg, k, maps, a, ntiles);
}

// ---------------------------------------------------------------------------
// Residue split through L2 (one CTA per tile, no cluster): a persistent CTA
// takes the W = 16 columns x L rows of a tile (L = 512 C) as C residue
// sub-tiles of 512 rows (rows C a + r), each fed by bulk tensor copies through
// the two-slot ring of the TMA column kernel, one sub-tile ahead, so the next
// tile's first sub-tile arrives while the current tile is combined.  For
// residue r < C-1 the CTA runs the 512-point transform, twiddles by W^{r k'}
// and parks the values in the CTA's own scratch region (device memory that
// stays in L2: up to C-1 sub-tiles per CTA, up to 30 MB per GPU), or, with
// PARK, residue C-2 in shared memory next to the ring (measured: faster at
// C = 3, slower at C = 2 and 4, where the larger shared-memory carve-out
// costs more than the L2 round trip saves); after the last residue
// it reads them back (ld.global.cg: L2, never a stale L1 line; the loads of 8
// outputs at a time issued together) and forms the radix-C outputs
// X[k' + 512 s] from the last residue, written back into its slot.  Thread
// (c, t) reads only the values it parked itself, so no barrier orders them.
// DRAM sees one read and one write of the tile; the scratch traffic
// (2 (C-2) sub-tiles per tile) stays in L2.  Every mbarrier wait is
// bounded (a wait that gives up sets kStatusTimeout; the CTA drains its own
// copies, bounded, and ends).
// Requirements (checked by the host): P even, Bs = L*P, at least 16 columns.
// ---------------------------------------------------------------------------
// SHIFT: an odd axis stride S (the n1 pass, S = n2/2 + 1): the rows of an odd
// residue start 8 bytes past a 16-byte boundary, so their tensor map starts
// one complex value early, and every box is two columns wider (WS = W + 2),
// the thread reading its column at offset (r S) mod 2.
template <int C, bool PARK, bool SHIFT = false>
struct L2SplitGeom {
    static constexpr int L = kSplitLC * C;
    static constexpr int T = kSplitLC / kSplitE;  // 16 threads per column
    static constexpr int NT = kSplitW * T;         // 256 threads
    // ring depth: at C = 2 (unshifted) three slots, which keep two residues'
    // copies in flight while the third serves the exchange and the combine
    // (1024^3 n0 pass 1.95 -> 1.80 ms); measured slower at C = 4 (2048^3
    // forward 17.05 -> 17.6 ms) and for the shifted maps (up to 1.5x), and
    // with a residue parked in shared memory only two fit
    static constexpr int STAGES = (C == 2 && !SHIFT && !PARK) ? 3 : 2;
    static constexpr int WS = SHIFT ? kSplitW + 2 : kSplitW;                          // slot row width
    static constexpr unsigned SUB_BYTES = (unsigned)kSplitLC * WS * sizeof(float2);  // 64 / 72 KB
    static_assert(!SHIFT || C % 2 == 0, "an odd stride needs an even C for 16-byte row strides");
    static_assert(kSplitW * sizeof(float2) == 128 && NT % 32 == 0 && 32 % kSplitW == 0,
                  "a parked row is one 128-byte L2 line, read by the lanes of one warp");
    // PARK: residue C-2 is parked in shared memory next to the ring, the
    // others (0 .. C-3, or 0 .. C-2 without PARK) in L2 scratch
    static constexpr int NL2 = PARK ? C - 2 : C - 1;  // residues parked in L2
    static constexpr size_t smem = (size_t)(STAGES + (PARK ? 1 : 0)) * SUB_BYTES + 64;
    static constexpr size_t scratch_per_cta = (size_t)(NL2 > 0 ? NL2 : 1) * kSplitLC * kSplitW;  // float2 values
};

template <int C, int DIR, bool PARK, bool SHIFT = false>
__global__ void __launch_bounds__(L2SplitGeom<C, PARK, SHIFT>::NT) col_l2split_kernel(
    const __grid_constant__ SplitMaps maps, ColArgs a, float2* scratch, long long ntiles)
{
    using G = L2SplitGeom<C, PARK, SHIFT>;
    constexpr int NL2 = G::NL2, WS = G::WS;
    constexpr int L = G::L, LC = kSplitLC, E = kSplitE, W = kSplitW, T = G::T, STAGES = G::STAGES;
    constexpr int BOXR = 256, NBOX = LC / BOXR;
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2* ring = reinterpret_cast<float2*>(smraw);
    float2* park = ring + (size_t)STAGES * LC * WS;  // PARK: residue C-2 (each thread's own positions)
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(smraw + (size_t)(STAGES + (PARK ? 1 : 0)) * G::SUB_BYTES);
    const int c = threadIdx.x, t = threadIdx.y;
    const bool leader = (c == 0 && t == 0);
    const long long ctiles = (a.C + W - 1) / W;
    float2* mine = scratch + (size_t)blockIdx.x * G::scratch_per_cta + (size_t)t * W + c;  // + (r LC + T m) W
    long long n_issued = 0;

    if (leader) {
#pragma unroll
        for (int r = 0; r < C; ++r) prefetch_tensormap(&maps.map[r]);
#pragma unroll
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // the CTA's n-th sub-tile: tile blockIdx.x + (n / C) gridDim.x, residue n % C
    auto issue = [&](long long n) {
        const long long tile = blockIdx.x + (n / C) * (long long)gridDim.x;
        if (tile >= ntiles) return;
        const int r = (int)(n % C), s = (int)(n % STAGES);
        const long long b = tile / ctiles;
        const long long c0 = (tile - b * ctiles) * W;
        mbar_arrive_expect_tx(&bars[s], G::SUB_BYTES);
        float2* slot = ring + (size_t)s * LC * WS;
#pragma unroll
        for (int k = 0; k < NBOX; ++k)
            tma_load_2d(slot + (size_t)k * BOXR * WS, &maps.map[r], (int)(2 * c0), (int)(b * LC + k * BOXR), &bars[s]);
        ++n_issued;
    };

    if (leader) {
#pragma unroll
        for (int k = 0; k < STAGES - 1; ++k) issue(k);
    }
    long long n_consumed = 0;
    bool failed = false;
    for (long long n = 0;; ++n) {
        const long long tile = blockIdx.x + (n / C) * (long long)gridDim.x;
        if (tile >= ntiles) break;
        const int r = (int)(n % C), s = (int)(n % STAGES);
        const bool ok = mbar_wait_bounded(&bars[s], (unsigned)((n / STAGES) & 1), kMbarMaxTries);
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        ++n_consumed;
        if (leader) issue(n + STAGES - 1);  // into the slot consumed at n - 1
        const long long b = tile / ctiles;
        const long long c0 = (tile - b * ctiles) * W;
        const bool active = (c0 + c) < a.C;
        float2* buf = ring + (size_t)s * LC * WS;
        const int off = SHIFT ? (int)((r * a.S) & 1) : 0;  // the odd residues' maps start one value early
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = buf[(t + T * m) * WS + c + off];
        __syncthreads();  // the slot now serves as the exchange buffer (W-wide rows from here on)
        // (twiddles from the table: registers go to the combine's loads below)
        fft_group<LC, E, DIR, C>(v, t, a.tw, ColExchange{buf, W, c});
        if (r > 0) {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = twiddle<DIR>(v[m], __ldg(&a.tw[r * (t + T * m)]));
        }
        if (PARK && r == C - 2) {  // parked in shared memory
#pragma unroll
            for (int m = 0; m < E; ++m) park[(t + T * m) * W + c] = v[m];
            fence_proxy_async_smem();  // order this thread's shared accesses before the slot's next bulk copy
            continue;
        }
        if (r < NL2) {  // parked in L2
#pragma unroll
            for (int m = 0; m < E; ++m) __stcg(&mine[((size_t)r * LC + T * m) * W], v[m]);
            fence_proxy_async_smem();
            continue;
        }
        // last residue: its values go back into the slot (each thread to the
        // positions it alone reads), then the radix-C step with the parked
        // residues, their L2 loads issued MB registers at a time so that they
        // are in flight together
#pragma unroll
        for (int m = 0; m < E; ++m) buf[(t + T * m) * W + c] = v[m];
        float2* dst = (a.dst ? a.dst : a.data) + b * a.Bs + c0 + c;
        // The parked values are loaded MB positions at a time.  At C = 2 the
        // batches are double buffered, the next batch's loads issued before
        // this batch is combined, so that one L2 round trip is exposed instead
        // of E/MB (1024^3 n0 pass 1.80 -> 1.77 ms); at C = 4 that spills, and
        // neither it nor smaller batches were faster there or at C = 3.
        constexpr int MB = 8;
        constexpr bool DB = C == 2;
        float2 zn[DB ? MB : 1][DB ? NL2 : 1];  // DB: the next batch
        if constexpr (DB) {
#pragma unroll
            for (int mm = 0; mm < MB; ++mm)
#pragma unroll
                for (int q = 0; q < NL2; ++q) zn[mm][q] = __ldcg(&mine[((size_t)q * LC + T * mm) * W]);
        }
#pragma unroll
        for (int m0 = 0; m0 < E; m0 += MB) {
            float2 z[MB][C];
            if constexpr (DB) {
#pragma unroll
                for (int mm = 0; mm < MB; ++mm)
#pragma unroll
                    for (int q = 0; q < NL2; ++q) z[mm][q] = zn[mm][q];
                if (m0 + MB < E) {
#pragma unroll
                    for (int mm = 0; mm < MB; ++mm)
#pragma unroll
                        for (int q = 0; q < NL2; ++q)
                            zn[mm][q] = __ldcg(&mine[((size_t)q * LC + T * (m0 + MB + mm)) * W]);
                }
            } else {
#pragma unroll
                for (int mm = 0; mm < MB; ++mm)
#pragma unroll
                    for (int q = 0; q < NL2; ++q) z[mm][q] = __ldcg(&mine[((size_t)q * LC + T * (m0 + mm)) * W]);
            }
#pragma unroll
            for (int mm = 0; mm < MB; ++mm) {
                if constexpr (PARK) z[mm][C - 2] = park[(t + T * (m0 + mm)) * W + c];
                z[mm][C - 1] = buf[(t + T * (m0 + mm)) * W + c];
                Dft<C, DIR>::run(z[mm]);
                const int kp = t + T * (m0 + mm);
                if (active) {
                    if (a.mask23 == 0 && a.scale == 1.0f) {
#pragma unroll
                        for (int q = 0; q < C; ++q) dst[(long long)(kp + LC * q) * a.S] = z[mm][q];
                    } else {
#pragma unroll
                        for (int q = 0; q < C; ++q)
                            dst[(long long)(kp + LC * q) * a.S] =
                                cscale(z[mm][q], col_out_factor(kp + LC * q, L, a.scale, a.mask23));
                    }
                }
            }
            // the parked rows just combined are dead: a row (one 128-byte line
            // of W values) is read by the W lanes of one warp, so once the warp
            // has them its first lane drops the lines from L2 unwritten (the
            // next tile parks whole lines again)
            __syncwarp();
            if (c == 0) {
#pragma unroll
                for (int mm = 0; mm < MB; ++mm)
#pragma unroll
                    for (int q = 0; q < NL2; ++q) discard_l2_line(&mine[((size_t)q * LC + T * (m0 + mm)) * W]);
            }
        }
        fence_proxy_async_smem();  // order this thread's shared accesses before the slot's next bulk copy
    }
    if (failed && leader) {
        atomicOr(a.status, kStatusTimeout);
        for (long long k = n_consumed; k < n_issued; ++k)
            mbar_wait_bounded(&bars[k % STAGES], (unsigned)((k / STAGES) & 1), kMbarMaxTries);
    }
}

// Persistent: one CTA per resident slot (one per SM).  scratch: at least
// l2split_scratch_values<C>(ctas) float2 values of device memory, ctas = the
// grid size this launcher uses (l2split_ctas).
template <int C, bool PARK>
inline size_t l2split_scratch_values(int ctas)
{
    return (size_t)ctas * L2SplitGeom<C, PARK>::scratch_per_cta;
}

template <int C, int DIR, bool PARK, bool SHIFT = false>
inline cudaError_t launch_col_l2split(const ColArgs& a, const SplitMaps& maps, float2* scratch, int ctas,
                                      cudaStream_t s)
{
    using G = L2SplitGeom<C, PARK, SHIFT>;
    auto k = col_l2split_kernel<C, DIR, PARK, SHIFT>;
    static PerDevice limit;  // the shared memory limit, raised once per device
    cudaError_t e = smem_limit_per_device(limit, k, G::smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = a.nb * ((a.C + kSplitW - 1) / kSplitW);
    if (ntiles <= 0) return cudaSuccess;
    const long long grid = ntiles < ctas ? ntiles : ctas;
    k<<<(unsigned)grid, dim3(kSplitW, G::T), G::smem, s>>>(maps, a, scratch, ntiles);
    return cudaGetLastError();
}

}  // namespace fft3d

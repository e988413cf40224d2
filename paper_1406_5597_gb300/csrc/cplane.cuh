// Cluster plane kernel: the 2D transform of each n0-plane (Sec. 2.1 step 1:
// the n2-axis real transform of every row, then the n1-axis complex transform
// of every column) with the whole plane held in the distributed shared
// memory of one thread-block cluster, so DRAM sees one read of the real plane
// and one write of its half spectrum (forward), or the reverse (inverse).
//
// A plane is n1 x H complex values (H = n2/2 + 1; 1.05 MB at 512^3), more
// than one SM holds, so C CTAs of a cluster share it: CTA b keeps the rows
// j1 = C*a + b, a in [0, RC), RC = n1/C, in a padded slab in its own shared
// memory.  The n1 transform is split the decimation-in-time way over that
// row assignment (F = exp(-2 pi i / n1), k = k' + RC*s, k' in [0, RC)):
//
//   X[k' + RC s] = sum_b F_C^{b s} . F^{b k'} . sum_a x[C a + b] F_RC^{a k'}
//
// so each CTA first runs RC-point column transforms over its own rows (no
// exchange), multiplies by F^{b k'}, and only the final radix-C step needs
// the other CTAs' slabs: CTA q takes the outputs k' in [q*RC/C, (q+1)*RC/C)
// of every column, reads the C values it needs straight from the C slabs
// (ld.shared::cluster; adjacent lanes take adjacent k2, so every remote read
// and every DRAM write is a contiguous run) and writes C full output rows.
//
// The inverse runs the same steps mirrored (Sec. 2.1: reverse order): the
// radix-C step first, reading the spectrum rows from DRAM and storing each
// result, times conj F^{b k'}, into the slab of CTA b (st.shared::cluster);
// then the RC-point inverse column transforms in place; then the c2r of each
// slab row straight to DRAM.
//
// Clusters are persistent: cluster i takes planes i, i + nclusters, ...
// Two cluster barriers per plane order the slab hand-overs (hardware
// barriers that every thread of the cluster reaches on every plane; the
// kernel has no spin-waits).
#pragma once
#include "cluster.cuh"
#include "cplane.h"
#include "kernels.cuh"
#include "tma.cuh"

namespace fft3d {

// Row transform exchange inside the row's own slab row (the row's values are
// in registers by then): position p at p + p/32, which stays inside a padded
// slab row and puts the two rows of a warp on opposite bank halves.
struct SlabRowExchange {
    float2* sm;
    __device__ __forceinline__ static int pad(int p) { return p + (p >> 5); }
    __device__ __forceinline__ void put(int p, float2 v) const { sm[pad(p)] = v; }
    __device__ __forceinline__ float2 get(int p) const { return sm[pad(p)]; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// Column transform exchange in place: position p of the thread's column
// (slab column k2, owned by one warp) at base[p * SH], base = slab + k2.
template <int SH>
struct SlabColExchange {
    float2* base;
    __device__ __forceinline__ void put(int p, float2 v) const { base[p * SH] = v; }
    __device__ __forceinline__ float2 get(int p) const { return base[p * SH]; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// Shapes derived from (n2/2, n1, cluster size, threads).
template <int LR, int ER, int LC, int C, int NT>
struct CPlaneGeom {
    static constexpr int H = LR + 1;
    static constexpr int RC = LC / C;                      // slab rows per CTA
    static constexpr int SH = H + (24 - H % 16) % 16;      // slab row stride: 64 bytes past a 128-byte multiple
    static constexpr int TR = LR / ER;                     // threads per row transform
    static constexpr int RPR = NT / TR;                    // rows per wave (wave 0 comes through the stage)
    static constexpr int ROUNDS = RC / RPR;
    static constexpr int EC = (RC <= 32 && num_stages(RC, RC) == 1) ? RC : 16;  // column transform: elements
                                                           // per thread (one thread per column when a single
                                                           // stage covers RC)
    static constexpr int TC = RC / EC;                     // threads per column
    static constexpr int GC = 32 / TC;                     // columns per warp
    static constexpr int NG = (H + GC - 1) / GC;           // column groups
    static constexpr int NW = NT / 32;
    static constexpr int KPC = RC / C;                     // k' rows per CTA in the radix-C step (at least;
                                                           // CTA q takes [q*RC/C, (q+1)*RC/C))
    static constexpr int NX = KPC * H;                     // radix-C items of the smallest share
    static constexpr int XI = NX / NT;                     // items every thread takes (the rest: a tail)
    static constexpr int XP0 = XI < 16 / C ? XI : 16 / C;  // inverse: items loaded one plane ahead
    static constexpr int XPRE = XP0 > 0 ? XP0 : (XI > 0 ? 1 : 0);  // (at most 16 values in registers)
    static constexpr int SLAB = RC * SH;                   // complex values
    static constexpr unsigned ROW_BYTES = LR * sizeof(float2);
    static constexpr unsigned STAGE_BYTES = RPR * ROW_BYTES;
    static constexpr unsigned SLAB_LOAD_BYTES = (RC - RPR) * ROW_BYTES;
    static constexpr size_t smem_fwd = (size_t)SLAB * sizeof(float2) + STAGE_BYTES + 2 * sizeof(unsigned long long);
    static constexpr size_t smem_inv = (size_t)SLAB * sizeof(float2);
    static_assert(LC % C == 0 && RC >= C, "n1 must split evenly over the cluster");
    static_assert(TR <= 32 && 32 % TR == 0 && NT % 32 == 0, "rows must pack into warps");
    static_assert(RPR <= RC && RC % RPR == 0, "row waves must tile the slab rows");
    static_assert(RC % EC == 0 && TC <= 32 && 32 % TC == 0, "column transform must pack into warps");
    static_assert(num_stages(RC, EC) > 0, "RC must factor into radices dividing 16");
    static_assert((LR - 1) + (LR - 1) / 32 < SH, "row exchange must fit a slab row");
    static_assert(NG * GC <= SH || num_stages(RC, EC) == 1, "column exchange must stay inside the slab rows");
    static_assert(ROW_BYTES % 16 == 0 && (SH * sizeof(float2)) % 16 == 0, "bulk copies need 16-byte rows");
};

template <int LR, int ER, int LC, int C, int NT, int DIR, int MINB>
__global__ void __launch_bounds__(NT, MINB) cplane_kernel(CPlaneArgs a)
{
    using G = CPlaneGeom<LR, ER, LC, C, NT>;
    constexpr int H = G::H, RC = G::RC, SH = G::SH, TR = G::TR, RPR = G::RPR;
    constexpr int EC = G::EC, TC = G::TC, GC = G::GC, XI = G::XPRE;
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2* slab = reinterpret_cast<float2*>(smraw);
    const unsigned rank = cluster_ctarank();
    const long long cid = cluster_index(), ncl = cluster_count();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned rs[C];  // the slabs of the cluster's CTAs, as shared::cluster addresses
#pragma unroll
    for (int b = 0; b < C; ++b) rs[b] = dsmem_map(slab, (unsigned)b);
    // this CTA's k' rows in the radix-C step
    const int kbase = (int)rank * RC / C;
    const int NX = ((int)rank + 1) * RC / C * H - kbase * H;
    // row waves: thread (rr, tr) transforms slab row r*RPR + rr
    const int rr = tid / TR, tr = tid - (tid / TR) * TR;
    // column groups: lane (cc, tc) of a warp, GC columns per group
    const int cc = lane % GC, tc = lane / GC;

    // RC-point column transforms over the slab rows, in place; the forward
    // multiplies output k' by F^{rank k'} on the way out.
    auto local_columns = [&]() {
        for (int g = warp; g < G::NG; g += G::NW) {
            const int k2 = g * GC + cc;
            const bool act = k2 < H;
            float2* col = slab + k2;
            float2 v[EC];
#pragma unroll
            for (int m = 0; m < EC; ++m) v[m] = act ? col[(tc + TC * m) * SH] : make_float2(0.f, 0.f);
            __syncwarp();  // the group's values are in registers before the exchange reuses its columns
            fft_group<RC, EC, DIR, LC / RC>(v, tc, a.tw_col, SlabColExchange<SH>{col});
            if (act) {
#pragma unroll
                for (int m = 0; m < EC; ++m) {
                    const int k = tc + TC * m;
                    float2 r = v[m];
                    if (DIR < 0 && rank != 0) r = cmul(r, __ldg(&a.tw_col[((int)rank * k) % LC]));
                    col[k * SH] = r;
                }
            }
            __syncwarp();
        }
    };

    if constexpr (DIR < 0) {
        // Forward.  Input rows of a plane: wave 0 arrives by bulk copies in
        // the stage buffer during the previous plane; waves 1.. arrive in
        // place, each real row in the slab row that later holds its spectrum.
        float2* stage = reinterpret_cast<float2*>(smraw + (size_t)G::SLAB * sizeof(float2));
        unsigned long long* bars = reinterpret_cast<unsigned long long*>(smraw + (size_t)G::SLAB * sizeof(float2) +
                                                                       G::STAGE_BYTES);
        const bool leader = tid == 0;
        if (leader) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        bool failed = false;
        auto wait = [&](int i, unsigned parity) {
            if (failed) return;
            if (!mbar_wait_bounded(&bars[i], parity, kMbarMaxTries)) {
                failed = true;
                atomicOr(a.status, kStatusTimeout);
            }
        };
        auto in_row = [&](long long p, int ar) {
            return reinterpret_cast<const float2*>(a.in) + (p * LC + (long long)C * ar + rank) * LR;
        };
        auto issue_stage = [&](long long p) {
            mbar_arrive_expect_tx(&bars[0], G::STAGE_BYTES);
            for (int ar = 0; ar < RPR; ++ar) bulk_load(stage + ar * LR, in_row(p, ar), G::ROW_BYTES, &bars[0]);
        };
        if (leader && cid < a.planes) issue_stage(cid);
        unsigned it = 0;
        for (long long p = cid; p < a.planes; p += ncl, ++it) {
            const unsigned par = it & 1u;
            if (leader && RC > RPR) {
                mbar_arrive_expect_tx(&bars[1], G::SLAB_LOAD_BYTES);
                for (int ar = RPR; ar < RC; ++ar) bulk_load(slab + ar * SH, in_row(p, ar), G::ROW_BYTES, &bars[1]);
            }
            // 1. n2-axis r2c: wave 0 from the stage, then the rows in the slab
            wait(0, par);
            {
                float2 v[ER];
                const float2* srow = stage + rr * LR;
#pragma unroll
                for (int m = 0; m < ER; ++m) v[m] = srow[tr + TR * m];
                fence_proxy_async_smem();  // these reads precede the stage's next bulk refill
                __syncwarp();
                float2* row = slab + rr * SH;
                row_r2c_regs<LR, ER, SlabRowExchange>(v, row, true, tr, lane, row, a.tw_row, a.twpack);
            }
            __syncthreads();  // stage consumed: prefetch the next plane's wave 0
            if (leader && p + ncl < a.planes) issue_stage(p + ncl);
            if (RC > RPR) wait(1, par);
#pragma unroll 1
            for (int r = 1; r < G::ROUNDS; ++r) {
                float2* row = slab + (r * RPR + rr) * SH;
                float2 v[ER];
#pragma unroll
                for (int m = 0; m < ER; ++m) v[m] = row[tr + TR * m];
                __syncwarp();  // the real row is in registers before its slab row becomes the exchange
                row_r2c_regs<LR, ER, SlabRowExchange>(v, row, true, tr, lane, row, a.tw_row, a.twpack);
            }
            __syncthreads();
            // 2. RC-point n1 transforms of the slab columns, times F^{rank k'}
            local_columns();
            fence_proxy_async_smem();  // slab accesses precede the next plane's bulk copies into it
            cluster_sync_all();
            // 3. radix-C step across the cluster's slabs -> DRAM rows k' + RC s (two items per pass)
            float2* out = reinterpret_cast<float2*>(a.out) + p * LC * (long long)H;
#pragma unroll 1
            for (int i = tid; i < NX; i += 2 * NT) {
                const int i2 = i + NT;
                const bool two = i2 < NX;
                const int kl = i / H, k2 = i - kl * H;
                const int kl2 = two ? i2 / H : kl, k22 = two ? i2 - kl2 * H : k2;
                const unsigned off = (unsigned)(((kbase + kl) * SH + k2) * sizeof(float2));
                const unsigned off2 = (unsigned)(((kbase + kl2) * SH + k22) * sizeof(float2));
                float2 z[C], z2[C];
#pragma unroll
                for (int b = 0; b < C; ++b) z[b] = dsmem_ld(rs[b] + off);
#pragma unroll
                for (int b = 0; b < C; ++b) z2[b] = dsmem_ld(rs[b] + off2);
                Dft<C, -1>::run(z);
                Dft<C, -1>::run(z2);
                float2* o = out + (long long)(kbase + kl) * H + k2;
#pragma unroll
                for (int s = 0; s < C; ++s) o[(long long)s * RC * H] = z[s];
                if (two) {
                    float2* o2 = out + (long long)(kbase + kl2) * H + k22;
#pragma unroll
                    for (int s = 0; s < C; ++s) o2[(long long)s * RC * H] = z2[s];
                }
            }
            cluster_sync_all();  // no slab is refilled while another CTA may still read it
        }
    } else {
        // Inverse.  The spectrum values of the first XI radix-C items of a
        // thread are loaded into registers one plane ahead, across the
        // barrier that ends the previous plane; the others in the step itself.
        const float2* in = reinterpret_cast<const float2*>(a.in);
        float2 pre[XI > 0 ? XI : 1][C];
        auto load_items = [&](long long p) {
#pragma unroll
            for (int j = 0; j < XI; ++j) {
                const int i = tid + j * NT;
                const int kl = i / H, k2 = i - kl * H;
                const float2* q = in + p * LC * (long long)H + (long long)(kbase + kl) * H + k2;
#pragma unroll
                for (int s = 0; s < C; ++s) pre[j][s] = __ldg(q + (long long)s * RC * H);
            }
        };
        // radix-C of one item, times conj F^{b k'}, into slab row k' of CTA b
        auto scatter = [&](float2 (&z)[C], int i) {
            const int kl = i / H, k2 = i - kl * H;
            const int kp = kbase + kl;
            Dft<C, +1>::run(z);
            const unsigned off = (unsigned)((kp * SH + k2) * sizeof(float2));
#pragma unroll
            for (int b = 0; b < C; ++b) {
                const float2 r = (b == 0) ? z[b] : cmulc(z[b], __ldg(&a.tw_col[(b * kp) % LC]));
                dsmem_st(rs[b] + off, r);
            }
        };
        if (cid < a.planes) load_items(cid);
        cluster_sync_all();  // every CTA of the cluster runs before the first remote store
        for (long long p = cid; p < a.planes; p += ncl) {
            // 1. radix-C step: DRAM rows k' + RC s -> slab row k' of every CTA
#pragma unroll
            for (int j = 0; j < XI; ++j) scatter(pre[j], tid + j * NT);
            for (int i = XI * NT + tid; i < NX; i += NT) {
                const int kl = i / H, k2 = i - kl * H;
                const float2* q = in + p * LC * (long long)H + (long long)(kbase + kl) * H + k2;
                float2 z[C];
#pragma unroll
                for (int s = 0; s < C; ++s) z[s] = __ldg(q + (long long)s * RC * H);
                scatter(z, i);
            }
            cluster_sync_all();
            // 2. RC-point inverse n1 transforms of the slab columns, in place
            local_columns();
            __syncthreads();
            // 3. n2-axis c2r of each slab row -> DRAM
            float2* out = reinterpret_cast<float2*>(a.out) + p * LC * (long long)LR;
#pragma unroll 1
            for (int r = 0; r < G::ROUNDS; ++r) {
                const int ar = r * RPR + rr;
                float2* row = slab + ar * SH;
                float2 v[ER];
                row_c2r_regs<LR, ER, kLdPlain, SlabRowExchange>(row, true, tr, lane, row, a.tw_row, a.twpack, v);
                float2* orow = out + ((long long)C * ar + rank) * LR;
#pragma unroll
                for (int m = 0; m < ER; ++m) orow[tr + TR * m] = v[m];
            }
            if (p + ncl < a.planes) load_items(p + ncl);
            cluster_sync_all();  // slabs are read out before the next plane's remote stores
        }
    }
}

// MINB: CTAs per SM the register budget is sized for (two when the shared
// memory of two fits, so that two clusters' planes overlap on every SM).
template <int LR, int ER, int LC, int C, int NT, int DIR, int MINB>
inline cudaError_t launch_cplane(const CPlaneArgs& a, cudaStream_t s)
{
    using G = CPlaneGeom<LR, ER, LC, C, NT>;
    constexpr size_t smem = DIR < 0 ? G::smem_fwd : G::smem_inv;
    auto k = cplane_kernel<LR, ER, LC, C, NT, DIR, MINB>;
    static PerDevice resident;  // co-resident clusters, queried once per device
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int max_clusters = 0;
    cudaError_t e = per_device(resident, &max_clusters, [&](int, int* v) {
        cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        if (C > 8) {
            r = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (r != cudaSuccess) return r;
        }
        cfg.gridDim = dim3(C * 64);
        return cudaOccupancyMaxActiveClusters(v, k, &cfg);
    });
    if (e != cudaSuccess) return e;
    if (a.planes <= 0) return cudaSuccess;
    const long long ncl = a.planes < max_clusters ? a.planes : max_clusters;
    cfg.gridDim = dim3((unsigned)(ncl * C));
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace fft3d

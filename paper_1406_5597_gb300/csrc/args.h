// Kernel argument blocks and the launcher registry shared by the device
// translation units and the host planner.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace fft3d {

struct ColArgs {
    float2* data;        // in place
    long long S;         // axis stride (complex elements)
    long long C;         // contiguous columns per batch entry
    long long nb;        // batch entries
    long long Bs;        // batch stride (complex elements)
    const float2* tw;    // W_L^m, m in [0, L)
    float scale;         // multiplies the result (1 for a plain pass)
    int* status;         // device status word (bounded waits that give up set bits here)
    float2* dst;         // result goes here (same layout) instead of in place; nullptr: in place
    int mask23;          // nonzero: zero the outputs whose signed index k has 3|k| >= L (2/3 rule)
    // outer batch (plain column kernel only): nb2 groups of the nb entries, group stride Bs2
    long long nb2 = 1;
    long long Bs2 = 0;
};

// Rows per 2D bulk tensor copy of a column tile of `rows` rows: the largest
// divisor of rows that is at most 256 (the box limit), so that whole boxes
// tile it (rows <= 256: one box; 512 / 1024: 256; 384: 192; 640: 128).
__host__ __device__ constexpr int tma_box_rows(int rows)
{
    for (int b = rows < 256 ? rows : 256; b > 1; --b)
        if (rows % b == 0) return b;
    return 1;
}

// Output factor of a column pass for output index k of a length-L axis:
// scale, or 0 where the 2/3 rule drops k (signed k in [-L/2, L/2), so the
// Nyquist bin is always dropped).
__host__ __device__ inline float col_out_factor(int k, int L, float scale, int mask23)
{
    if (!mask23) return scale;
    const int ks = (2 * k < L) ? k : k - L;
    const int ak = ks < 0 ? -ks : ks;
    return (3 * ak < L) ? scale : 0.f;
}

// Device status bits.
constexpr int kStatusTimeout = 1;

struct RowArgs {
    const void* in;
    void* out;
    long long rows;
    const float2* tw;      // W_L^m, m in [0, L), L = n2/2
    const float2* twpack;  // exp(-2 pi i k / n2), k in [0, L]
    long long rs;          // real-side row stride: in float pairs for even n2, L (dense) or L + 1 (padded
                           // rows of 2H floats); in floats for odd n2 (n2 dense, 2H = n2 + 1 padded)
};

// Runtime plan for the generic (any length) kernels, over the complex type T
// (float2, or double2 for the FP64 path).  A length whose prime factors are
// 2, 3, 5 and 7 runs its Stockham stages directly (radix list).  Any other
// length runs Bluestein's chirp-z form (M > 0): with c[n] = exp(-i pi n^2 / L),
// the DFT is X[k] = c[k] sum_n (x[n] c[n]) conj(c[k - n]), a cyclic
// convolution of length M (a power of two >= 2L - 1) done by two length-M
// transforms and a pointwise product with the transformed chirp.
template <typename T>
struct GenPlanT {
    int L;
    int nst;
    int radix[24];
    int M;           // 0: direct stages; else the convolution length
    int mst;         // stages of the length-M transforms
    int mradix[24];
    const T* chirp;  // c[n], n < L (device)
    const T* bhat;   // (1/M) FFT_M of b, b[m] = b[M - m] = conj(c[m]) for m < L, else 0 (device)
    const T* twm;    // W_M^x = exp(-2 pi i x / M), x < M (device)
};
using GenPlan = GenPlanT<float2>;
using GenPlan64 = GenPlanT<double2>;

// Slots per line of a generic kernel's shared buffers: the L + 1 bins of an
// unpacked row, or the M points of a Bluestein convolution.
template <typename T>
__host__ __device__ inline int gen_line_slots(const GenPlanT<T>& g)
{
    return g.M > g.L + 1 ? g.M : g.L + 1;
}

// Arguments of the FP64 passes (runtime-length kernels only): as ColArgs and
// RowArgs, in double precision, without scaling, masking or status word.
struct ColArgs64 {
    double2* data;       // in place
    long long S;         // axis stride (complex elements)
    long long C;         // contiguous columns per batch entry
    long long nb;        // batch entries
    long long Bs;        // batch stride (complex elements)
    const double2* tw;   // W_L^m, m in [0, L)
    double2* dst;        // nullptr: in place
};
struct RowArgs64 {
    const void* in;
    void* out;
    long long rows;
    const double2* tw;      // W_L^m, m in [0, L), L = n2/2 (even n2) or n2 (odd n2)
    const double2* twpack;  // exp(-2 pi i k / n2), k in [0, L] (even n2)
    long long rs;           // real-side row stride: in double pairs for even n2, in doubles for odd n2
};

// Launchers take a runtime shape choice: w = columns per CTA (0 or > compiled
// maximum: the compiled value), rows = rows per CTA (same rule).
using ColFn = cudaError_t (*)(const ColArgs&, int w, cudaStream_t);
using ColTmaFn = cudaError_t (*)(const ColArgs&, const CUtensorMap&, cudaStream_t);
using RowFn = cudaError_t (*)(const RowArgs&, int rows, cudaStream_t);
struct NlRowArgs {
    const float2* in;
    float2* out;
    long long rows;
    long long fs;  // field stride (complex elements)
    const float2* tw;
    const float2* twpack;
    int k2_keep;   // bins k2 >= k2_keep are set to zero
};

using NlFn = cudaError_t (*)(const NlRowArgs&, cudaStream_t);

// Compile-time specialised kernels for one transform length.
struct LenEntry {
    int L;
    int col_E, col_W;  // plain column kernel: elements per thread, columns per CTA
    ColFn col_fwd, col_inv;
    int tma_E, tma_W;  // TMA-fed persistent column kernel (tma_W = 0: none)
    ColTmaFn tma_fwd, tma_inv;
    ColTmaFn tma_pair_fwd, tma_pair_inv;  // same, for an odd axis stride (row-pair view)
    int tma_pair_E;                       // its elements per thread
    int row_E, row_rows;  // row kernels (row_E = 0: none)
    bool row_warp;        // rows resident in warps (shuffle unpack) or staged in shared memory
    RowFn r2c, c2r;
    NlFn nl;              // fused nonlinear-term row kernel (warp rows only)
    // TMA row pairs with two columns per thread (column form 6; nullptr: none)
    ColTmaFn tma_pair2_fwd = nullptr, tma_pair2_inv = nullptr;
};

const LenEntry* find_len(int L);

struct PlaneArgs;
using PlaneFn = cudaError_t (*)(const PlaneArgs&, cudaStream_t);

// Fused plane kernel for one (n2/2, n1) pair.
struct PlaneEntry {
    int LR, LC;  // n2/2 and n1
    int ER, EC, NT;
    PlaneFn fwd, inv;
};
const PlaneEntry* plane_entries(int* n);

// Column kernels with radix-16 stages on the tensor cores.
using ColTcFn = cudaError_t (*)(const ColArgs&, const uint16_t* gtab, cudaStream_t);
struct TcEntry {
    int L, W;
    ColTcFn bf16_fwd, bf16_inv, f16_fwd, f16_inv;
};
const TcEntry* tc_entries(int* n);

// Column kernels of a long axis split over a thread-block cluster of C CTAs
// (colsplit.cuh): E elements per thread, W columns per tile.
struct SplitEntry {
    int L, C, E, W;
    ColFn fwd, inv;
};
const SplitEntry* split_entries(int* n);

// TMA-fed split (colsplit.cuh): L = 512 C, one tensor map per residue r of
// the rows (base + r S, row stride C S).
struct SplitMaps {
    CUtensorMap map[4];
};
using ColTmaSplitFn = cudaError_t (*)(const ColArgs&, const SplitMaps&, cudaStream_t);
struct TmaSplitEntry {
    int L, C;
    ColTmaSplitFn fwd, inv;
};
const TmaSplitEntry* tma_split_entries(int* n);

// Residue split through L2 (colsplit.cuh): L = 512 C, one CTA per tile, the
// residues parked in a scratch region of device memory (scratch_values(ctas)
// float2 values for a grid of ctas CTAs).
using ColL2SplitFn = cudaError_t (*)(const ColArgs&, const SplitMaps&, float2* scratch, int ctas, cudaStream_t);
struct L2SplitEntry {
    int L, C;
    ColL2SplitFn fwd, inv;
    ColL2SplitFn fwd_shift, inv_shift;  // odd axis stride (even C only; else nullptr)
    size_t (*scratch_values)(int ctas);
    int (*ctas)();  // grid size on the current device (resident CTAs)
};
const L2SplitEntry* l2split_entries(int* n);

// Generic kernels: dir = -1 forward, +1 inverse.
cudaError_t generic_col(const ColArgs& a, const GenPlan& g, int dir, cudaStream_t s);
cudaError_t generic_row(const RowArgs& a, const GenPlan& g, int dir, cudaStream_t s);
cudaError_t generic_row_odd(const RowArgs& a, const GenPlan& g, int dir, cudaStream_t s);
cudaError_t generic_col64(const ColArgs64& a, const GenPlan64& g, int dir, cudaStream_t s);
cudaError_t generic_row64(const RowArgs64& a, const GenPlan64& g, int dir, cudaStream_t s);
cudaError_t generic_row_odd64(const RowArgs64& a, const GenPlan64& g, int dir, cudaStream_t s);

}  // namespace fft3d

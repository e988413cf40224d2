// Kernel argument blocks and the launcher registry shared by the device
// translation units and the host planner.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

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
};

// Device status bits.
constexpr int kStatusTimeout = 1;

struct RowArgs {
    const void* in;
    void* out;
    long long rows;
    const float2* tw;      // W_L^m, m in [0, L), L = n2/2
    const float2* twpack;  // exp(-2 pi i k / n2), k in [0, L]
};

// Runtime radix plan for the generic (any 2/3/5-smooth length) kernels.
struct GenPlan {
    int L;
    int nst;
    int radix[24];
};

using ColFn = cudaError_t (*)(const ColArgs&, cudaStream_t);
using ColTmaFn = cudaError_t (*)(const ColArgs&, const CUtensorMap&, cudaStream_t);
using RowFn = cudaError_t (*)(const RowArgs&, cudaStream_t);

// Compile-time specialised kernels for one transform length.
struct LenEntry {
    int L;
    int col_E, col_W;  // plain column kernel: elements per thread, columns per CTA
    ColFn col_fwd, col_inv;
    int tma_E, tma_W;  // TMA-fed persistent column kernel (tma_W = 0: none)
    ColTmaFn tma_fwd, tma_inv;
    int row_E, row_rows;  // row kernels (row_E = 0: none)
    bool row_warp;        // rows resident in warps (shuffle unpack) or staged in shared memory
    RowFn r2c, c2r;
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

// Generic kernels: dir = -1 forward, +1 inverse.
cudaError_t generic_col(const ColArgs& a, const GenPlan& g, int dir, cudaStream_t s);
cudaError_t generic_row(const RowArgs& a, const GenPlan& g, int dir, cudaStream_t s);

}  // namespace fft3d

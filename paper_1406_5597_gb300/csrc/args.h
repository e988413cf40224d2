// Kernel argument blocks and the launcher registry shared by the device
// translation units and the host planner.
#pragma once
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
};

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
using RowFn = cudaError_t (*)(const RowArgs&, cudaStream_t);

// Compile-time specialised kernels for one transform length.
struct LenEntry {
    int L;
    int col_E, col_W;    // column kernel: elements per thread, columns per CTA
    int row_E, row_rows; // row kernels (0 when not instantiated for this L)
    ColFn col_fwd, col_inv;
    RowFn r2c, c2r;
};

const LenEntry* find_len(int L);

// Generic kernels: dir = -1 forward, +1 inverse.
cudaError_t generic_col(const ColArgs& a, const GenPlan& g, int dir, cudaStream_t s);
cudaError_t generic_row(const RowArgs& a, const GenPlan& g, int dir, cudaStream_t s);

}  // namespace fft3d

// Host view of the cluster plane kernel (device code: cplane.cuh).
#pragma once
#include "args.h"

namespace fft3d {

struct CPlaneArgs {
    const void* in;        // forward: real planes; inverse: half-spectrum planes (only read)
    void* out;             // forward: half-spectrum planes; inverse: real planes
    long long planes;      // batch * n0
    const float2* tw_row;  // W_{n2/2}^m, m in [0, n2/2)
    const float2* twpack;  // exp(-2 pi i k / n2), k in [0, n2/2]
    const float2* tw_col;  // W_{n1}^m, m in [0, n1)
    int* status;           // device status word (a bounded copy wait that gives up sets kStatusTimeout)
};

using CPlaneFn = cudaError_t (*)(const CPlaneArgs&, cudaStream_t);

// Cluster plane kernel for one (n2/2, n1) pair: C CTAs per plane.
struct CPlaneEntry {
    int LR, LC;  // n2/2 and n1
    int C, NT;   // cluster size, threads per CTA
    CPlaneFn fwd, inv;
};
const CPlaneEntry* cplane_entries(int* n);

}  // namespace fft3d

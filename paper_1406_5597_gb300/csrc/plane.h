// Host view of the fused plane kernel's arguments (device code: plane.cuh).
#pragma once
#include "args.h"

namespace fft3d {

struct PlaneArgs {
    const void* in;
    void* out;
    long long planes;        // batch * n0
    int H;                   // n2/2 + 1
    const float2* tw_row;    // W_{n2/2}^m table
    const float2* twpack;    // exp(-2 pi i k / n2), k in [0, n2/2]
    const float2* tw_col;    // W_{n1}^m table
    int* counters;           // one per plane, then one work ticket; all zero at launch
    float2* ring;            // inverse: ring of ring_planes planes holding the n1 results (L2 resident)
    int ring_planes;         // 0: the inverse works in place on its input
    int* status;             // device status word
    int lag;                 // extra planes of lead beyond what the resident CTAs span
    unsigned wait_limit;     // polls (about 0.1-0.2 us each) before a wait gives up
    long long skip_plane;    // test hook: this plane's producers never report (-1: none)
};

}  // namespace fft3d

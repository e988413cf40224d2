// Work-table form of a grouped transform of uneven sizes (group_wt.cu): the
// row, n1 and n0 passes of every size in one persistent launch.
#pragma once
#include <cstddef>

#include "args.h"

namespace fft3d {

// One segment: the items (tiles of rows or columns) of one pass of one size.
struct WtSeg {
    int body;         // compiled item body (wt_body_index)
    int dep;          // segment whose items must all be done before any of this one starts, or -1
    long long first;  // first ticket of the segment
    long long items;  // items of the segment
    long long need;   // completed items of dep to wait for (its item count)
    // column pass: in place at data, element (b, j, c) at b*Bs + j*S + c
    float2* data;
    long long S, C, nb, Bs;
    // row pass: rows of the real side (stride rs float pairs) and of the half spectrum (H values)
    const void* in;
    void* out;
    long long rows, rs;
    const float2* tw;      // W_L^m, m in [0, L) of the pass's axis
    const float2* twpack;  // row passes: exp(-2 pi i k / n2), k in [0, L]
};

constexpr int kWtMaxSeg = 40;

struct WtTable {
    int nseg;
    long long total;  // tickets (items) of all segments
    WtSeg seg[kWtMaxSeg];
};

// Device counters of one launch; zeroed before it.
struct WtCounters {
    unsigned long long ticket;
    int status;  // kStatusTimeout when a dependency wait gave up
    int pad;
    int done[kWtMaxSeg];
};

// The compiled item body of a row pass (row = true; L = n2/2) or a column pass
// (L = the axis length) in direction dir (-1 forward, +1 inverse), or -1 if
// this length has none.  *items_per_tile: rows (row pass) or columns per item.
int wt_body_index(bool row, int L, int dir, int* per_item);

// One persistent launch over the table (grid: the resident CTAs of the device).
cudaError_t launch_wt(const WtTable& tab, WtCounters* ctr, cudaStream_t s);

}  // namespace fft3d

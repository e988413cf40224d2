// Host-side tensor-map encoding (see tma_host.cpp).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace fft3d {

// Host: encode a 2D FP32 tensor map (inner dimension contiguous).
// dims/strides in elements/bytes as cuTensorMapEncodeTiled expects.
cudaError_t encode_tensor_map_2d(CUtensorMap* map, const void* base, unsigned long long inner,
                                 unsigned long long outer, unsigned long long row_stride_bytes, unsigned box_inner,
                                 unsigned box_outer);

struct ColArgs;
// Tensor map of a column pass for the TMA column kernel: 2D FP32 view, inner
// 2*C floats, outer nb*L rows of byte stride 8*S, box (2*W floats) x min(L, 256);
// pair mode: inner 4*S floats (a row pair), outer nb*L/2 pairs of byte
// stride 16*S, box (2*(W+2) floats) x min(L/2, 256).
cudaError_t col_tensor_map_host(CUtensorMap* map, const ColArgs& a, int L, int W, bool pair = false);

}  // namespace fft3d

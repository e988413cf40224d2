// Host-side tensor-map encoding through the driver entry point.
#include <cudaTypedefs.h>

#include "args.h"
#include "tma_host.h"

namespace fft3d {

cudaError_t encode_tensor_map_2d(CUtensorMap* map, const void* base, unsigned long long inner,
                                 unsigned long long outer, unsigned long long row_stride_bytes, unsigned box_inner,
                                 unsigned box_outer)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t gdim[2] = {inner, outer};
    const cuuint64_t gstride[1] = {row_stride_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estride[2] = {1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), gdim, gstride, box, estride,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t col_tensor_map_host(CUtensorMap* map, const ColArgs& a, int L, int W, bool pair)
{
    if (!pair)
        return encode_tensor_map_2d(map, a.data, 2ull * a.C, (unsigned long long)a.nb * L, 8ull * a.S, 2u * W,
                                    (unsigned)tma_box_rows(L));
    const int rows = L / 2;
    return encode_tensor_map_2d(map, a.data, 4ull * a.S, (unsigned long long)a.nb * rows, 16ull * a.S,
                                2u * (W + 2), (unsigned)tma_box_rows(rows));
}

}  // namespace fft3d

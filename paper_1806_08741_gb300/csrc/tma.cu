// tma.cu -- host-side construction of TMA tensor maps for image tiles.
//
// The image is described to the TMA unit as bytes: [N_2][N_1][N_0 * C *
// sizeof(T)], so one tiled copy moves a tile of TX x TY x TZ voxels with
// all their channels, rows kept contiguous, and out-of-image voxels filled
// with zeros.  The driver's encoder is reached through the runtime's
// entry-point query, so the library does not link the driver library.
#include <cuda.h>

#include "common.cuh"

namespace sslic {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

bool image_tma_ok(const Geom& g, const void* img, int esz)
{
    const uint64_t row = (uint64_t)g.N[0] * g.C * esz;
    return ((uintptr_t)img & 15) == 0 && row % 16 == 0 && encoder() != nullptr;
}

int encode_image_map(void* map, const Geom& g, const void* img, int esz, int tx, int ty, int tz)
{
    EncodeTiledFn fn = encoder();
    if (!fn) return SSLIC_EUNSUPPORTED;
    const cuuint64_t row = (cuuint64_t)g.N[0] * g.C * esz;
    const cuuint64_t dims[3] = {row, (cuuint64_t)g.N[1], (cuuint64_t)g.N[2]};
    const cuuint64_t strides[2] = {row, row * (cuuint64_t)g.N[1]};
    const cuuint32_t box[3] = {(cuuint32_t)(tx * g.C * esz), (cuuint32_t)ty, (cuuint32_t)tz};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t rank = g.n == 3 ? 3 : 2;
    const CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT8, rank,
                          const_cast<void*>(img), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SSLIC_OK : SSLIC_EUNSUPPORTED;
}

}  // namespace sslic

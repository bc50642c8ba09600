// Host side of the record tensor maps (tma.cuh): encoded with the driver's
// cuTensorMapEncodeTiled, looked up once through the runtime's driver entry
// point query (no link against the driver library).
#include <mutex>

#include "tma.cuh"

namespace gs {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

gs_status_t make_record_map(const float *rec, int64_t rows, CUtensorMap *map)
{
    if (!rec || rows < 1 || rows >= (int64_t(1) << 31) || (reinterpret_cast<uintptr_t>(rec) & 15))
        return GS_ERR_INVALID_ARG;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return GS_ERR_UNSUPPORTED;
    const cuuint64_t dims[2] = {(cuuint64_t)kRecFloats, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kRecBytes};  // bytes between rows, a multiple of 16
    const cuuint32_t box[2] = {(cuuint32_t)kRecFloats, 1u};  // one row of 48 bytes (gather4 boxes are one row high)
    const cuuint32_t estrides[2] = {1u, 1u};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(rec), dims, strides, box,
                          estrides, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GS_OK : GS_ERR_INVALID_ARG;
}

gs_status_t make_tensor_map_4d(const float *base, const uint64_t dims[4], const uint64_t strides[3],
                               const uint32_t box[4], CUtensorMap *map)
{
    if (!base || (reinterpret_cast<uintptr_t>(base) & 15)) return GS_ERR_INVALID_ARG;
    for (int k = 0; k < 3; k++)
        if (strides[k] % 16 || strides[k] == 0) return GS_ERR_INVALID_ARG;
    for (int k = 0; k < 4; k++)
        if (dims[k] == 0 || box[k] == 0 || box[k] > 256) return GS_ERR_INVALID_ARG;
    if ((box[0] * sizeof(float)) % 16) return GS_ERR_INVALID_ARG;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return GS_ERR_UNSUPPORTED;
    cuuint64_t d[4], st[3];
    cuuint32_t b[4], es[4] = {1u, 1u, 1u, 1u};
    for (int k = 0; k < 4; k++) {
        d[k] = dims[k];
        b[k] = box[k];
    }
    for (int k = 0; k < 3; k++) st[k] = strides[k];
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), d, st, b, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GS_OK : GS_ERR_INVALID_ARG;
}

}  // namespace gs

// Host-side tensor-map encoding for the TMA kernels, through the driver
// entry point cuTensorMapEncodeTiled (resolved once at run time).
#include "tma.cuh"

#include <mutex>

namespace cgdir {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

bool encode_tensor_map(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                       const uint32_t *box, int elem) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || rank < 1 || rank > 5) return false;
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
    cuuint64_t gdim[5], gstride[4];
    cuuint32_t bdim[5], estr[5];
    uint64_t stride = (uint64_t)elem;
    for (int i = 0; i < rank; ++i) {
        if (dims[i] == 0 || box[i] == 0 || box[i] > 256) return false;
        gdim[i] = dims[i];
        bdim[i] = box[i];
        estr[i] = 1;
    }
    for (int i = 1; i < rank; ++i) {
        stride *= dims[i - 1];
        if (stride % 16 != 0) return false;
        gstride[i - 1] = stride;
    }
    if ((box[0] * (uint32_t)elem) % 16 != 0) return false;
    CUtensorMapDataType dt;
    if (elem == 4) dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    else if (elem == 2) dt = CU_TENSOR_MAP_DATA_TYPE_UINT16;
    else if (elem == 1) dt = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    else return false;
    const CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void *>(base), gdim, gstride, bdim, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace cgdir

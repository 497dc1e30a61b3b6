// tmap.cu -- host-side encoding of the TMA tensor maps of the operand planes.
// The driver's cuTensorMapEncodeTiled is reached through the runtime's
// driver entry-point query, so the library does not link libcuda directly.
#include <cudaTypedefs.h>

#include <mutex>

#include "cgemm_tc.cuh"

namespace tc {
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_mu;

tc_status get_encode(PFN_cuTensorMapEncodeTiled_v12000* fn) {
    // The encoder is a driver call and wants the device's context current on
    // this thread.  A thread that has made no runtime call that binds it yet
    // (a framework's worker thread, say) gets it bound here, once.
    thread_local bool bound = false;
    if (!bound) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess)
            return fail(TC_ERR_CUDA, "no CUDA device for the tensor-map encoder");
        bound = true;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_encode) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return fail(TC_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    *fn = g_encode;
    return TC_OK;
}
}  // namespace

tc_status make_part_map(CUtensorMap* map, const void* base, int Np, int planes, int precision) {
    return make_part_map_rows(map, base, Np, planes, precision, 32);
}

tc_status make_part_map_rows(CUtensorMap* map, const void* base, int Np, int planes, int precision, int row_bytes) {
    if (row_bytes != 32 && row_bytes != 64 && row_bytes != 128)
        return fail(TC_ERR_INVALID_ARG, "tensor map: rows of 32, 64 or 128 bytes");
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    TC_TRY(get_encode(&enc));
    const size_t E = cgemm_elem_bytes(precision);
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || (Np * E) % 16 != 0)
        return fail(TC_ERR_INVALID_ARG, "operand planes must be 16-byte aligned with 16-byte row pitch");
    cuuint64_t dims[3] = {(cuuint64_t)Np, (cuuint64_t)Np, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)Np * E, (cuuint64_t)Np * (cuuint64_t)Np * E};
    cuuint32_t box[3] = {(cuuint32_t)(row_bytes / E), 128u, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUtensorMapDataType dt = E == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     row_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                     : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TC_OK;
}

}  // namespace tc

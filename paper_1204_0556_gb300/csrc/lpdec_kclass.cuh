// Instantiates the decode and projection kernels of one degree class.
// Each lpdec_kD.cu defines LPDEC_D and includes this file, so the classes
// compile as separate translation units (in parallel).
#include "lpdec_internal.h"

#ifndef LPDEC_D
#error "define LPDEC_D before including lpdec_kclass.cuh"
#endif

#define LPDEC_CAT2(a, b) a##b
#define LPDEC_CAT(a, b) LPDEC_CAT2(a, b)

namespace lpdec {

namespace {
constexpr int kD = LPDEC_D;
constexpr int kMaxT = kD <= 8 ? 1024 : 512;

template <typename S>
const void *decode_fn() {
    return reinterpret_cast<const void *>(&decode_kernel<kD, S, kMaxT>);
}

const void *decode_fn_for(int dtype) {
    switch (dtype) {
        case 0: return decode_fn<float>();
        case 1: return decode_fn<__nv_bfloat16>();
        case 2: return decode_fn<__half>();
        default: return nullptr;
    }
}
}  // namespace

cudaError_t LPDEC_CAT(prepare_decode_, LPDEC_D)(int dtype, size_t smem) {
    const void *fn = decode_fn_for(dtype);
    if (!fn) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t LPDEC_CAT(occupancy_decode_, LPDEC_D)(int dtype, int block, size_t smem, int *blocks_per_sm) {
    const void *fn = decode_fn_for(dtype);
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

cudaError_t LPDEC_CAT(launch_decode_, LPDEC_D)(int dtype, const DecodeArgs &a, const LaunchCfg &lc) {
    if (lc.block > kMaxT) return cudaErrorInvalidConfiguration;
    switch (dtype) {
        case 0: decode_kernel<kD, float, kMaxT><<<lc.grid, lc.block, lc.smem, lc.stream>>>(a); break;
        case 1: decode_kernel<kD, __nv_bfloat16, kMaxT><<<lc.grid, lc.block, lc.smem, lc.stream>>>(a); break;
        case 2: decode_kernel<kD, __half, kMaxT><<<lc.grid, lc.block, lc.smem, lc.stream>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t LPDEC_CAT(launch_project_, LPDEC_D)(int d, long long count, const float *v, float *z,
                                                 cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int block = 256;
    const long long grid = (count + block - 1) / block;
    project_kernel<kD><<<(unsigned)grid, block, 0, s>>>(d, count, v, z);
    return cudaGetLastError();
}

}  // namespace lpdec

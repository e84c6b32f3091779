// Instantiates the decode and projection kernels of one degree class.
// Each lpdec_kD.cu defines LPDEC_D and includes this file, so the classes
// compile as separate translation units (in parallel).
#include <atomic>

#include "lpdec_internal.h"

#ifndef LPDEC_D
#error "define LPDEC_D before including lpdec_kclass.cuh"
#endif

#define LPDEC_CAT2(a, b) a##b
#define LPDEC_CAT(a, b) LPDEC_CAT2(a, b)

namespace lpdec {

namespace {
constexpr int kD = LPDEC_D;
constexpr int kL = class_lanes(kD);
constexpr int kMaxT = class_max_threads_D(kD);
// Variable degree of the regular-code kernel built for this class: (3,6)-type
// codes for D = 6, (4,8) for D = 8, and degree-3 variables with any common
// check degree for the wide classes.
constexpr int kRegDV = kD == 8 ? 4 : 3;

// Kernel forms of this class: 0 generic, 1 regular (indices from global
// memory), 2 regular with the indices staged in shared memory; 3-5 the same
// three as STREAMED ring kernels (decode_kernel_ring).
constexpr int kForms = 6;

template <int DV, bool STAGE, bool RING, typename S>
const void *decode_fn() {
    if constexpr (RING) return reinterpret_cast<const void *>(&decode_kernel_ring<kD, kL, DV, S, kMaxT, STAGE>);
    else return reinterpret_cast<const void *>(&decode_kernel<kD, kL, DV, S, kMaxT, STAGE>);
}

template <int DV, bool STAGE, bool RING>
const void *decode_fn_dtype(int dtype) {
    switch (dtype) {
        case 0: return decode_fn<DV, STAGE, RING, float>();
        case 1: return decode_fn<DV, STAGE, RING, __nv_bfloat16>();
        case 2: return decode_fn<DV, STAGE, RING, __half>();
        case 3: return decode_fn<DV, STAGE, RING, q16_t>();
        default: return nullptr;
    }
}

int form_of(int reg_dv, bool stage, bool ring) {
    const int f = (kRegDV > 0 && reg_dv == kRegDV) ? (stage ? 2 : 1) : 0;
    return ring ? f + 3 : f;
}

const void *decode_fn_for(int dtype, int form) {
    switch (form) {
        case 5: return decode_fn_dtype<kRegDV, true, true>(dtype);
        case 4: return decode_fn_dtype<kRegDV, false, true>(dtype);
        case 3: return decode_fn_dtype<0, false, true>(dtype);
        case 2: return decode_fn_dtype<kRegDV, true, false>(dtype);
        case 1: return decode_fn_dtype<kRegDV, false, false>(dtype);
        default: return decode_fn_dtype<0, false, false>(dtype);
    }
}

template <int DV, bool STAGE, bool RING, typename S>
void launch_one(const DecodeArgs &a, const LaunchCfg &lc) {
    if constexpr (RING) decode_kernel_ring<kD, kL, DV, S, kMaxT, STAGE><<<lc.grid, lc.block, lc.smem, lc.stream>>>(a);
    else decode_kernel<kD, kL, DV, S, kMaxT, STAGE><<<lc.grid, lc.block, lc.smem, lc.stream>>>(a);
}

template <int DV, bool STAGE, bool RING>
cudaError_t launch_dv(int dtype, const DecodeArgs &a, const LaunchCfg &lc) {
    switch (dtype) {
        case 0: launch_one<DV, STAGE, RING, float>(a, lc); break;
        case 1: launch_one<DV, STAGE, RING, __nv_bfloat16>(a, lc); break;
        case 2: launch_one<DV, STAGE, RING, __half>(a, lc); break;
        case 3: launch_one<DV, STAGE, RING, q16_t>(a, lc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
}  // namespace

// Largest dynamic shared memory already granted to each kernel of this class
// ([dtype][form]); the attribute is set only when a launch needs more, so
// decodes in a steady state (and under CUDA-graph capture) make no attribute
// calls.  Per device: a kernel attribute is per device.
static std::atomic<int> g_smem_granted[64][4][kForms];

cudaError_t LPDEC_CAT(prepare_decode_, LPDEC_D)(int dtype, int reg_dv, bool stage, bool ring, size_t smem) {
    const int form = form_of(reg_dv, stage, ring);
    const void *fn = decode_fn_for(dtype, form);
    if (!fn) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    std::atomic<int> &granted = g_smem_granted[dev][dtype][form];
    if ((int)smem <= granted.load()) return cudaSuccess;
    err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess) {
        int cur = granted.load();
        while ((int)smem > cur && !granted.compare_exchange_weak(cur, (int)smem)) {
        }
    }
    return err;
}

cudaError_t LPDEC_CAT(occupancy_decode_, LPDEC_D)(int dtype, int reg_dv, bool stage, bool ring, int block,
                                                   size_t smem, int *blocks_per_sm) {
    const void *fn = decode_fn_for(dtype, form_of(reg_dv, stage, ring));
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

cudaError_t LPDEC_CAT(launch_decode_, LPDEC_D)(int dtype, int reg_dv, const DecodeArgs &a, const LaunchCfg &lc) {
    if (lc.block > kMaxT) return cudaErrorInvalidConfiguration;
    const bool ring = a.ring_slots > 0;
    if (ring && !a.k_state) return cudaErrorInvalidValue;  // the ring streams parked state
    switch (form_of(reg_dv, a.slice_base > 0, ring)) {
        case 5: return launch_dv<kRegDV, true, true>(dtype, a, lc);
        case 4: return launch_dv<kRegDV, false, true>(dtype, a, lc);
        case 3: return launch_dv<0, false, true>(dtype, a, lc);
        case 2: return launch_dv<kRegDV, true, false>(dtype, a, lc);
        case 1: return launch_dv<kRegDV, false, false>(dtype, a, lc);
        default: return launch_dv<0, false, false>(dtype, a, lc);
    }
}

cudaError_t LPDEC_CAT(launch_project_, LPDEC_D)(int d, long long count, const float *v, float *z,
                                                 cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int block = 256;
    const long long lanes = kL;  // threads per vector (project_kernel)
    const long long grid = (count * lanes + block - 1) / block;
    project_kernel<kD><<<(unsigned)grid, block, 0, s>>>(d, count, v, z);
    return cudaGetLastError();
}

}  // namespace lpdec

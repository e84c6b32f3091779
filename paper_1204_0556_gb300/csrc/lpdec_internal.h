// Internal interface between the C-ABI layer and the per-degree kernel units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "lpdec_device.cuh"

namespace lpdec {

// Degree classes: a check of degree d runs in the class D >= d (unused lanes
// are padded).  D <= 8 sorts the breakpoints with a network; larger D uses
// the sort-free fixed point.
constexpr int kNumClasses = 5;
constexpr int kClassD[kNumClasses] = {6, 8, 16, 20, 32};

inline int degree_class(int max_dc) {
    for (int i = 0; i < kNumClasses; ++i)
        if (max_dc <= kClassD[i]) return i;
    return -1;
}

// Largest CTA the decode kernel of a class is compiled for.  The classes
// D = 20 and 32 hold 10 and 16 entries per lane in registers: compiled for
// at most 896 threads they get 72 registers a thread instead of 64, and spill
// less (D = 32: 112 -> 60 bytes).  C4000 (2 x 416 threads) runs 7.6% faster,
// C8000 (1 x 800) 1%.
constexpr int class_max_threads_D(int D) { return D >= 20 ? 896 : 1024; }
inline int class_max_threads(int cls) { return class_max_threads_D(kClassD[cls]); }

struct LaunchCfg {
    int grid;
    int block;
    size_t smem;
    cudaStream_t stream;
    int slice_base = 0;  // staged regular form: shared-memory offset of the first slice (after the
                         // 16-bit index block at offset 0); 0 when the indices are not staged
    // ring kernel (STREAMED): slots, slot size and the offsets of the slots,
    // the groups' scratch and the slot metadata; ring_slots = 0 otherwise
    int ring_slots = 0, ring_slot_bytes = 0, ring_off_slots = 0, ring_off_scratch = 0, ring_off_meta = 0;
    int ring_llr_off = 0;  // byte offset of the LLR row within a slot, 0 when the slots hold none
};

// Per-class entry points, defined in lpdec_kD.cu.
// reg_dv: the code's variable degree when it is regular with check degree
// exactly D (selects the regular-code kernel where one is built), else 0.
#define LPDEC_DECLARE_CLASS(D)                                                                           \
    cudaError_t launch_decode_##D(int dtype, int reg_dv, const DecodeArgs &a, const LaunchCfg &lc);      \
    cudaError_t occupancy_decode_##D(int dtype, int reg_dv, bool stage, bool ring, int block, size_t smem, \
                                     int *blocks_per_sm);                                                 \
    cudaError_t prepare_decode_##D(int dtype, int reg_dv, bool stage, bool ring, size_t smem);           \
    cudaError_t launch_project_##D(int d, long long count, const float *v, float *z, cudaStream_t s);
LPDEC_DECLARE_CLASS(6)
LPDEC_DECLARE_CLASS(8)
LPDEC_DECLARE_CLASS(16)
LPDEC_DECLARE_CLASS(20)
LPDEC_DECLARE_CLASS(32)
#undef LPDEC_DECLARE_CLASS

}  // namespace lpdec

// Mixed-code persistent decode: frames of up to eight codes with different
// check degrees in one launch (RESIDENT schedule, per-frame early exit).
//
// A CTA works on one code at a time, with that code's tile: `groups` frames
// decoded concurrently, each by `group_threads` threads, in slices of shared
// memory laid out for that code.  Groups pull frame ids from the code's work
// queue; when the queue is empty the CTA synchronizes, picks another code that
// still has frames, re-carves its shared memory and continues.  Early-exiting
// frames therefore free their slice for the next frame of any code, and CTAs
// rebalance across codes by themselves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lpdec.h"
#include "lpdec_api_internal.h"
#include "lpdec_internal.h"

namespace lpdec {
namespace {

// Batch-wide pointers a group needs to run frames of the current code.
struct MixedIO {
    const long long *offset;
    const float *llr;
    float *x_out;
    uint8_t *bits_out;
    int32_t *iters_out;
    uint8_t *cert_out;
    int *queue;  // this code's work-queue counter
};

// One group's share of a round: pull frames of the current code until its
// queue is empty.  Two kernels use it.  The FAST kernel inlines the three most
// common forms ((3,6), (4,8), and checks of degree 21..32 with degree-3
// variables) and serves batches whose codes each take one of them, each form
// at most once; the host then puts the code of form s in slot s, so the
// kernel names its descriptor by a constant index and the descriptor's fields
// are read from the kernel's parameter space at fixed offsets.  The general
// kernel calls every form through mixed_round_call, not inlined, so that each
// gets the whole register budget (inlining five forms spilled 232 B), with
// the descriptor of the current code copied to shared memory.
template <int D, int L, int DV, typename S>
__device__ __forceinline__ void mixed_round(const MixedCode &mc, const CodeView &cv, MixedIO b,
                                            unsigned char *smem_raw, int g, int t) {
    const int T = mc.group_threads;
    const int bar = 1 + g;
    unsigned char *base = smem_raw + (size_t)g * mc.smem_per_group;
    Slice<S> sm;
    sm.w = reinterpret_cast<S *>(base);
    sm.l = sm.w + cv.Ep;
    sm.x = reinterpret_cast<float *>(base + mc.off_x);
    sm.red = reinterpret_cast<float *>(base + mc.off_red);
    sm.flags = reinterpret_cast<int *>(sm.red + 2 * (T >> 5));
    sm.mbar = reinterpret_cast<uint64_t *>(sm.flags + 6);
    uint32_t phase = 0;
    int par = 0;
    for (;;) {
        if (t == 0) sm.flags[4 + par] = atomicAdd(b.queue, 1);
        group_sync(bar, T);
        const int idx = sm.flags[4 + par];
        par ^= 1;
        if (idx >= mc.n_frames) break;
        const int f = mc.frames[idx];
        const size_t off = (size_t)b.offset[f];
        FrameIO io;
        io.llr = b.llr + off;
        io.x = b.x_out + off;
        io.bits = b.bits_out ? b.bits_out + off : nullptr;
        io.iters = b.iters_out ? b.iters_out + f : nullptr;
        io.cert = b.cert_out ? b.cert_out + f : nullptr;
        io.w_state = io.l_state = nullptr;
        io.k_state = nullptr;
        // (3,6) codes stage their 16-bit indices in the mixed CTA; the others,
        // whose frames fill the shared memory, read them from global memory
        // with the x-update's prefetch (as the single-code kernels do)
        frame_run<D, L, DV, S, false, !(DV == 3 && D <= 8)>(cv, mc.cfg, mc.cfg.max_iter, io, sm, t, T, bar, phase);
    }
}

// General kernel: the descriptor (with its staged index pointers) is in shared memory.
template <int D, int L, int DV, typename S>
__device__ __noinline__ void mixed_round_call(const MixedCode *mc, MixedIO b, unsigned char *smem_raw, int g, int t) {
    mixed_round<D, L, DV, S>(*mc, mc->view, b, smem_raw, g, t);
}

// FAST kernel: mc is a descriptor of the kernel's parameter block.  STAGED:
// the code's 16-bit indices were copied to shared memory at mc.idx_off (the
// pointers are rebuilt here); otherwise they stay the global ones, so each
// instantiation knows the memory its index loads go to.
template <int D, int L, int DV, typename S, bool STAGED>
__device__ __forceinline__ void fast_round(const MixedCode &mc, MixedIO b, unsigned char *smem_raw, int g, int t) {
    CodeView cv = mc.view;
    if constexpr (STAGED) {
        cv.col16 = reinterpret_cast<const uint16_t *>(smem_raw + mc.idx_off);
        cv.csc16 = cv.col16 + mc.view.col16_elems;
    }
    mixed_round<D, L, DV, S>(mc, cv, b, smem_raw, g, t);
}

template <typename S, bool FAST>
__global__ void __launch_bounds__(kMixedMaxThreads, 1) mixed_kernel(const MixedArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int next_code;
    __shared__ MixedCode cur_code;  // descriptor of the code this CTA works on
    // Longest frames first: every CTA starts on the code with the most edges
    // per frame and moves through the codes in that order, so the frames still
    // running when the batch drains are those of the shortest code.
    int cur = -1;
    for (int q = 0; q < a.n_codes && cur < 0; ++q)
        if (a.code[a.order[q]].n_frames > 0) cur = a.order[q];
    if (cur < 0) return;
    for (;;) {
        if (threadIdx.x == 0) cur_code = a.code[cur];
        __syncthreads();
        if (cur_code.idx_off >= 0) {
            // stage this code's 16-bit indices after its slices, then point the
            // view at the copy (every thread has read the global pointer first)
            copy16(smem_raw + cur_code.idx_off, cur_code.view.col16, cur_code.view.idx16_bytes, threadIdx.x,
                   blockDim.x);
            __syncthreads();
            if (threadIdx.x == 0) {
                cur_code.view.col16 = reinterpret_cast<const uint16_t *>(smem_raw + cur_code.idx_off);
                cur_code.view.csc16 = cur_code.view.col16 + cur_code.view.col16_elems;
            }
            __syncthreads();
        }
        const int T = cur_code.group_threads;
        const int g = threadIdx.x / T;
        if (g < cur_code.groups) {
            MixedIO b{a.offset, a.llr, a.x_out, a.bits_out, a.iters_out, a.cert_out, a.queues + cur};
            const int t = threadIdx.x - g * T;
            if constexpr (FAST) {
                switch (cur) {  // slot s holds the code of FAST form s; slots 1 and 2 never stage
                    case 0:
                        if (a.code[0].idx_off >= 0) fast_round<6, 1, 3, S, true>(a.code[0], b, smem_raw, g, t);
                        else fast_round<6, 1, 3, S, false>(a.code[0], b, smem_raw, g, t);
                        break;
                    case 1: fast_round<8, 1, 4, S, false>(a.code[1], b, smem_raw, g, t); break;
                    default: fast_round<32, class_lanes(32), 3, S, false>(a.code[2], b, smem_raw, g, t); break;
                }
            } else {
                switch (cur_code.kind) {
                    case kK6R3: mixed_round_call<6, 1, 3, S>(&cur_code, b, smem_raw, g, t); break;
                    case kK6: mixed_round_call<6, 1, 0, S>(&cur_code, b, smem_raw, g, t); break;
                    case kK8R4: mixed_round_call<8, 1, 4, S>(&cur_code, b, smem_raw, g, t); break;
                    case kK8: mixed_round_call<8, 1, 0, S>(&cur_code, b, smem_raw, g, t); break;
                    case kK16: mixed_round_call<16, class_lanes(16), 0, S>(&cur_code, b, smem_raw, g, t); break;
                    case kK20: mixed_round_call<20, class_lanes(20), 0, S>(&cur_code, b, smem_raw, g, t); break;
                    case kK16R3: mixed_round_call<16, class_lanes(16), 3, S>(&cur_code, b, smem_raw, g, t); break;
                    case kK20R3: mixed_round_call<20, class_lanes(20), 3, S>(&cur_code, b, smem_raw, g, t); break;
                    case kK32R3: mixed_round_call<32, class_lanes(32), 3, S>(&cur_code, b, smem_raw, g, t); break;
                    default: mixed_round_call<32, class_lanes(32), 0, S>(&cur_code, b, smem_raw, g, t); break;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // the first code, in the order above, that still has frames
            int nx = -1;
            for (int q = 0; q < a.n_codes; ++q) {
                const int c = a.order[q];
                if (atomicAdd(a.queues + c, 0) < a.code[c].n_frames) { nx = c; break; }
            }
            next_code = nx;
        }
        __syncthreads();
        const int nx = next_code;
        if (nx < 0) break;
        cur = nx;
        // thread 0 rewrites cur_code and next_code only after the barrier at the
        // top of the next round, which every thread reaches after reading them
    }
}

template <bool FAST>
const void *mixed_fn_t(int dtype) {
    switch (dtype) {
        case 0: return reinterpret_cast<const void *>(&mixed_kernel<float, FAST>);
        case 1: return reinterpret_cast<const void *>(&mixed_kernel<__nv_bfloat16, FAST>);
        case 2: return reinterpret_cast<const void *>(&mixed_kernel<__half, FAST>);
        case 3: return reinterpret_cast<const void *>(&mixed_kernel<q16_t, FAST>);
        default: return nullptr;
    }
}

// The FAST kernel serves batches whose codes all run one of its three inlined forms.
const void *mixed_fn(int dtype, bool fast) { return fast ? mixed_fn_t<true>(dtype) : mixed_fn_t<false>(dtype); }

int kind_of(const lpdec_code *c) {
    switch (kClassD[c->cls]) {
        case 6: return c->reg_dv == 3 ? kK6R3 : kK6;
        case 8: return c->reg_dv == 4 ? kK8R4 : kK8;
        case 16: return c->reg_dv == 3 ? kK16R3 : kK16;
        case 20: return c->reg_dv == 3 ? kK20R3 : kK20;
        default: return c->reg_dv == 3 ? kK32R3 : kK32;
    }
}

// Everything a mixed launch needs except the batch buffers: argument block,
// launch shape, and the host copies of the per-frame offsets and per-code
// frame lists.
struct MixedSetup {
    MixedArgs a;
    int grid = 0, block = 0;
    size_t smem = 0;
    const void *fn = nullptr;
    int n_frames = 0;
    std::vector<long long> offset;
    std::vector<int> flat;
    std::vector<int> list_start;
    long long *d_offset = nullptr;  // device copies, set by mixed_bind
    int *d_flat = nullptr;
    size_t work_bytes() const {
        return 256 + ((offset.size() * 8 + 255) & ~(size_t)255) + flat.size() * 4;
    }
};

int mixed_setup(const char *who, const lpdec_code *const *codes, int32_t n_codes, int32_t n_frames,
                const int32_t *frame_code, const lpdec_params *p, MixedSetup &S) {
    if (!codes || n_codes < 1 || n_codes > kMaxMixedCodes)
        return set_error(LPDEC_EINVAL, "%s: n_codes=%d must be in [1, %d]", who, n_codes, kMaxMixedCodes);
    if (n_frames < 0) return set_error(LPDEC_EINVAL, "%s: n_frames=%d < 0", who, n_frames);
    int rc = validate_params(p);
    if (rc) return rc;
    if (p->schedule == LPDEC_SCHED_STREAMED) return set_error(LPDEC_EINVAL, "%s: runs the RESIDENT schedule only", who);
    for (int c = 0; c < n_codes; ++c)
        if (!codes[c]) return set_error(LPDEC_EINVAL, "%s: codes[%d] is NULL", who, c);
    if (n_frames > 0 && !frame_code) return set_error(LPDEC_EINVAL, "%s: frame_code must not be NULL", who);
    const int dev = codes[0]->device;
    for (int c = 1; c < n_codes; ++c)
        if (codes[c]->device != dev) return set_error(LPDEC_EINVAL, "%s: codes on different devices", who);
    for (int f = 0; f < n_frames; ++f)
        if (frame_code[f] < 0 || frame_code[f] >= n_codes)
            return set_error(LPDEC_EINVAL, "%s: frame_code[%d]=%d out of range", who, f, frame_code[f]);

    // FAST batches: every code takes one of the FAST kernel's three forms, each
    // form at most once.  The codes then move to the slot of their form (a form
    // no code takes keeps an empty slot: no frames, no CTA starts or moves there).
    int used[3] = {-1, -1, -1};
    bool fast = true;
    for (int c = 0; c < n_codes && fast; ++c) {
        const int k = kind_of(codes[c]);
        const int sl = k == kK6R3 ? 0 : (k == kK8R4 ? 1 : (k == kK32R3 ? 2 : -1));
        if (sl < 0 || used[sl] >= 0) fast = false;
        else used[sl] = c;
    }
    const lpdec_code *slot_codes[3];
    std::vector<int32_t> slot_frame_code;
    if (fast) {
        for (int sl = 0; sl < 3; ++sl) slot_codes[sl] = codes[used[sl] >= 0 ? used[sl] : 0];
        int slot_of[kMaxMixedCodes];
        for (int sl = 0; sl < 3; ++sl)
            if (used[sl] >= 0) slot_of[used[sl]] = sl;
        slot_frame_code.resize((size_t)n_frames);
        for (int f = 0; f < n_frames; ++f) slot_frame_code[f] = slot_of[frame_code[f]];
        codes = slot_codes;
        n_codes = 3;
        frame_code = slot_frame_code.data();
    }

    // per-frame offsets and per-code frame lists
    S.n_frames = n_frames;
    S.offset.assign((size_t)n_frames, 0);
    std::vector<std::vector<int>> lists((size_t)n_codes);
    long long off = 0;
    for (int f = 0; f < n_frames; ++f) {
        const int c = frame_code[f];
        if (c < 0 || c >= n_codes) return set_error(LPDEC_EINVAL, "%s: frame_code[%d]=%d out of range", who, f, c);
        S.offset[f] = off;
        off += codes[c]->n;
        lists[c].push_back(f);
    }
    S.flat.clear();
    S.list_start.assign((size_t)n_codes, 0);
    for (int c = 0; c < n_codes; ++c) {
        S.list_start[c] = (int)S.flat.size();
        S.flat.insert(S.flat.end(), lists[c].begin(), lists[c].end());
    }

    MixedArgs &a = S.a;
    std::memset(&a, 0, sizeof(a));
    a.n_codes = n_codes;
    int block = 32;
    size_t smem = 0;
    const int cap = device_smem_optin(dev);
    std::vector<SliceLayout> layouts((size_t)n_codes);
    for (int c = 0; c < n_codes; ++c) {
        const lpdec_code *cc = codes[c];
        Tile tile = cc->tuned[p->state_dtype].valid ? cc->tuned[p->state_dtype] : default_tile(cc, p->state_dtype);
        if (tile.group_threads > kMixedMaxThreads) tile = default_tile(cc, p->state_dtype, kMixedMaxThreads);
        if (tile.group_threads > kMixedMaxThreads)
            return set_error(LPDEC_EINVAL, "%s: code %d needs %d threads per frame (limit %d)", who, c,
                             tile.group_threads, kMixedMaxThreads);
        const SliceLayout L = slice_layout(cc, p->state_dtype, tile.group_threads);
        if ((int)L.bytes > cap)
            return set_error(LPDEC_EINVAL, "%s: code %d's frame state does not fit in shared memory", who, c);
        layouts[c] = L;
        MixedCode &mc = a.code[c];
        mc.view = make_view(cc);
        mc.cfg = make_cfg(cc, p);
        mc.kind = kind_of(cc);
        mc.group_threads = tile.group_threads;
        mc.smem_per_group = (int)L.bytes;
        mc.off_x = (int)L.off_x;
        mc.off_red = (int)L.off_red;
        mc.n_frames = (int)lists[c].size();
        smem = std::max(smem, L.bytes);  // at least one frame of every code must fit in the CTA
    }
    // One CTA per SM serves every code in turn, so each code gets as many
    // frames per CTA as the CTA's threads and shared memory allow (the CTA
    // takes the largest single-code footprint, capped by the device).
    for (int c = 0; c < n_codes; ++c) {
        const int g = std::min(15, kMixedMaxThreads / a.code[c].group_threads);
        smem = std::max(smem, std::min<size_t>((size_t)cap / layouts[c].bytes, (size_t)g) * layouts[c].bytes);
    }
    for (int c = 0; c < n_codes; ++c) {
        MixedCode &mc = a.code[c];
        const int g = std::min({15, kMixedMaxThreads / mc.group_threads, (int)(smem / layouts[c].bytes)});
        mc.groups = std::max(1, g);
        block = std::max(block, mc.groups * mc.group_threads);
    }
    // Regular codes stage their 16-bit index block after their slices when it
    // fits in the device's shared memory (the CTA's footprint may grow to it).
    for (int c = 0; c < n_codes; ++c) {
        MixedCode &mc = a.code[c];
        mc.idx_off = -1;
        if (codes[c]->reg_dv > 0 && codes[c]->idx16_bytes > 0) {
            const size_t off = ((size_t)mc.groups * layouts[c].bytes + 127) & ~(size_t)127;
            if (off + (size_t)codes[c]->idx16_bytes <= (size_t)cap) {
                mc.idx_off = (int)off;
                smem = std::max(smem, off + (size_t)codes[c]->idx16_bytes);
            }
        }
    }
    // FAST: an empty slot stages nothing, and the (4,8) and wide slots never
    // stage (their frames fill the shared memory; their kernel forms read the
    // indices from global memory with the x-update's prefetch)
    if (fast)
        for (int sl = 0; sl < 3; ++sl)
            if (used[sl] < 0 || sl > 0) a.code[sl].idx_off = -1;
    S.fn = mixed_fn(p->state_dtype, fast);
    cudaError_t err = cudaFuncSetAttribute(S.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return cuda_error(err, "mixed decode: cudaFuncSetAttribute");
    int bps = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, S.fn, block, smem);
    if (err != cudaSuccess) return cuda_error(err, "mixed decode: occupancy");
    if (bps < 1) return set_error(LPDEC_EINVAL, "%s: tile does not fit on an SM", who);
    S.grid = bps * device_sm_count(dev);
    S.block = block;
    S.smem = smem;
    // the order in which CTAs take the codes: most edges per frame first
    for (int c = 0; c < n_codes; ++c) a.order[c] = c;
    std::stable_sort(a.order, a.order + n_codes, [&](int x, int y) { return codes[x]->E > codes[y]->E; });
    return LPDEC_OK;
}

// Point the argument block at a device workspace laid out as
// [256 B queue counters | offsets | frame lists].
void mixed_bind(MixedSetup &S, char *work, const float *llr, float *x_out, uint8_t *bits_out, int32_t *iters_out,
                uint8_t *cert_out) {
    const size_t ob = (S.offset.size() * 8 + 255) & ~(size_t)255;
    S.a.queues = reinterpret_cast<int *>(work);
    S.d_offset = reinterpret_cast<long long *>(work + 256);
    S.d_flat = reinterpret_cast<int *>(work + 256 + ob);
    S.a.offset = S.d_offset;
    for (int c = 0; c < S.a.n_codes; ++c) S.a.code[c].frames = S.d_flat + S.list_start[c];
    S.a.llr = llr;
    S.a.x_out = x_out;
    S.a.bits_out = bits_out;
    S.a.iters_out = iters_out;
    S.a.cert_out = cert_out;
}

// Queue the launch: zero the counters, run the kernel.  No host memory is
// touched and nothing is allocated, so this can be captured in a CUDA graph.
int mixed_launch(MixedSetup &S, cudaStream_t stream) {
    cudaError_t err = cudaMemsetAsync(S.a.queues, 0, 256, stream);
    if (err != cudaSuccess) return cuda_error(err, "mixed decode: cudaMemsetAsync");
    void *args[] = {&S.a};
    err = cudaLaunchKernel(S.fn, dim3(S.grid), dim3(S.block), args, S.smem, stream);
    if (err != cudaSuccess) return cuda_error(err, "mixed decode: launch");
    return LPDEC_OK;
}

}  // namespace
}  // namespace lpdec

struct lpdec_mixed_plan {
    lpdec::MixedSetup setup;
    void *work = nullptr;
};

extern "C" int lpdec_decode_mixed(const lpdec_code *const *codes, int32_t n_codes, int32_t n_frames,
                                  const int32_t *frame_code, const float *llr, const lpdec_params *p,
                                  float *x_out, uint8_t *bits_out, int32_t *iters_out, uint8_t *cert_out,
                                  void *cuda_stream) {
    using namespace lpdec;
    MixedSetup S;
    int rc = mixed_setup("lpdec_decode_mixed", codes, n_codes, n_frames, frame_code, p, S);
    if (rc) return rc;
    if (n_frames == 0) return LPDEC_OK;
    if (!llr || !x_out) return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: llr and x_out must not be NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    char *work = nullptr;
    cudaError_t err = lib_alloc(reinterpret_cast<void **>(&work), S.work_bytes(), stream);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode_mixed: allocation of the workspace");
    mixed_bind(S, work, llr, x_out, bits_out, iters_out, cert_out);
    err = cudaMemcpyAsync(S.d_offset, S.offset.data(), S.offset.size() * 8, cudaMemcpyHostToDevice, stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(S.d_flat, S.flat.data(), S.flat.size() * 4, cudaMemcpyHostToDevice, stream);
    rc = err != cudaSuccess ? cuda_error(err, "lpdec_decode_mixed: workspace upload") : mixed_launch(S, stream);
    err = cudaFreeAsync(work, stream);
    if (!rc && err != cudaSuccess) rc = cuda_error(err, "lpdec_decode_mixed: cudaFreeAsync");
    return rc;
}

extern "C" int lpdec_mixed_plan_create(const lpdec_code *const *codes, int32_t n_codes, int32_t n_frames,
                                       const int32_t *frame_code, const lpdec_params *p, lpdec_mixed_plan **out) {
    using namespace lpdec;
    if (!out) return set_error(LPDEC_EINVAL, "lpdec_mixed_plan_create: out is NULL");
    if (n_frames < 1) return set_error(LPDEC_EINVAL, "lpdec_mixed_plan_create: n_frames must be >= 1");
    auto *plan = new (std::nothrow) lpdec_mixed_plan();
    if (!plan) return set_error(LPDEC_ENOMEM, "lpdec_mixed_plan_create: host allocation failed");
    int rc = mixed_setup("lpdec_mixed_plan_create", codes, n_codes, n_frames, frame_code, p, plan->setup);
    if (rc) {
        delete plan;
        return rc;
    }
    MixedSetup &S = plan->setup;
    cudaError_t err = cudaMalloc(&plan->work, S.work_bytes());
    if (err != cudaSuccess) {
        delete plan;
        return cuda_error(err, "lpdec_mixed_plan_create: cudaMalloc");
    }
    char *w = static_cast<char *>(plan->work);
    mixed_bind(S, w, nullptr, nullptr, nullptr, nullptr, nullptr);
    err = cudaMemcpy(S.d_offset, S.offset.data(), S.offset.size() * 8, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(S.d_flat, S.flat.data(), S.flat.size() * 4, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        cudaFree(plan->work);
        delete plan;
        return cuda_error(err, "lpdec_mixed_plan_create: upload");
    }
    *out = plan;
    return LPDEC_OK;
}

extern "C" int lpdec_mixed_plan_decode(lpdec_mixed_plan *plan, const float *llr, float *x_out, uint8_t *bits_out,
                                       int32_t *iters_out, uint8_t *cert_out, void *cuda_stream) {
    using namespace lpdec;
    if (!plan) return set_error(LPDEC_EINVAL, "lpdec_mixed_plan_decode: plan is NULL");
    if (!llr || !x_out) return set_error(LPDEC_EINVAL, "lpdec_mixed_plan_decode: llr and x_out must not be NULL");
    MixedSetup &S = plan->setup;
    mixed_bind(S, static_cast<char *>(plan->work), llr, x_out, bits_out, iters_out, cert_out);
    return mixed_launch(S, static_cast<cudaStream_t>(cuda_stream));
}

extern "C" int lpdec_mixed_plan_destroy(lpdec_mixed_plan *plan) {
    if (!plan) return lpdec::set_error(LPDEC_EINVAL, "lpdec_mixed_plan_destroy: plan is NULL");
    const cudaError_t err = cudaFree(plan->work);
    delete plan;
    if (err != cudaSuccess) return lpdec::cuda_error(err, "lpdec_mixed_plan_destroy: cudaFree");
    return LPDEC_OK;
}

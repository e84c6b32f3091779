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
// queue is empty.  Not inlined, so that each kernel form gets the whole
// register budget instead of the union of all forms.
template <int D, int L, int DV, typename S>
__device__ __noinline__ void mixed_round(const MixedCode *mc, MixedIO b, unsigned char *smem_raw, int g, int t) {
    const int T = mc->group_threads;
    const int bar = 1 + g;
    unsigned char *base = smem_raw + (size_t)g * mc->smem_per_group;
    Slice<S> sm;
    sm.z = reinterpret_cast<S *>(base);
    sm.l = sm.z + mc->view.Ep;
    sm.x = reinterpret_cast<float *>(base + mc->off_x);
    sm.red = reinterpret_cast<float *>(base + mc->off_red);
    sm.flags = reinterpret_cast<int *>(sm.red + 2 * (T >> 5));
    sm.mbar = reinterpret_cast<uint64_t *>(sm.flags + 6);
    uint32_t phase = 0;
    int par = 0;
    for (;;) {
        if (t == 0) sm.flags[4 + par] = atomicAdd(b.queue, 1);
        group_sync(bar, T);
        const int idx = sm.flags[4 + par];
        par ^= 1;
        if (idx >= mc->n_frames) break;
        const int f = mc->frames[idx];
        const size_t off = (size_t)b.offset[f];
        FrameIO io;
        io.llr = b.llr + off;
        io.x = b.x_out + off;
        io.bits = b.bits_out ? b.bits_out + off : nullptr;
        io.iters = b.iters_out ? b.iters_out + f : nullptr;
        io.cert = b.cert_out ? b.cert_out + f : nullptr;
        io.z_state = io.l_state = nullptr;
        io.k_state = nullptr;
        frame_run<D, L, DV, S>(mc->view, mc->cfg, mc->cfg.max_iter, io, sm, t, T, bar, phase);
    }
}

template <typename S>
__global__ void __launch_bounds__(kMixedMaxThreads, 1) mixed_kernel(const MixedArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int next_code;
    __shared__ MixedCode cur_code;  // descriptor of the code this CTA works on
    int cur = 0;
    while (cur < a.n_codes - 1 && (int)blockIdx.x >= a.home_end[cur]) ++cur;
    for (;;) {
        if (threadIdx.x == 0) cur_code = a.code[cur];
        __syncthreads();
        const int T = cur_code.group_threads;
        const int g = threadIdx.x / T;
        if (g < cur_code.groups) {
            MixedIO b{a.offset, a.llr, a.x_out, a.bits_out, a.iters_out, a.cert_out, a.queues + cur};
            const int t = threadIdx.x - g * T;
            switch (cur_code.kind) {
                case kK6R3: mixed_round<6, 1, 3, S>(&cur_code, b, smem_raw, g, t); break;
                case kK6: mixed_round<6, 1, 0, S>(&cur_code, b, smem_raw, g, t); break;
                case kK8R4: mixed_round<8, 1, 4, S>(&cur_code, b, smem_raw, g, t); break;
                case kK8: mixed_round<8, 1, 0, S>(&cur_code, b, smem_raw, g, t); break;
                case kK16: mixed_round<16, 2, 0, S>(&cur_code, b, smem_raw, g, t); break;
                case kK20: mixed_round<20, 4, 0, S>(&cur_code, b, smem_raw, g, t); break;
                default: mixed_round<32, 4, 0, S>(&cur_code, b, smem_raw, g, t); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // next code with frames left, starting after the current one
            int nx = -1;
            for (int q = 1; q <= a.n_codes; ++q) {
                const int c = (cur + q) % a.n_codes;
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

const void *mixed_fn(int dtype) {
    switch (dtype) {
        case 0: return reinterpret_cast<const void *>(&mixed_kernel<float>);
        case 1: return reinterpret_cast<const void *>(&mixed_kernel<__nv_bfloat16>);
        case 2: return reinterpret_cast<const void *>(&mixed_kernel<__half>);
        default: return nullptr;
    }
}

int kind_of(const lpdec_code *c) {
    switch (kClassD[c->cls]) {
        case 6: return c->reg_dv == 3 ? kK6R3 : kK6;
        case 8: return c->reg_dv == 4 ? kK8R4 : kK8;
        case 16: return kK16;
        case 20: return kK20;
        default: return kK32;
    }
}

}  // namespace
}  // namespace lpdec

extern "C" int lpdec_decode_mixed(const lpdec_code *const *codes, int32_t n_codes, int32_t n_frames,
                                  const int32_t *frame_code, const float *llr, const lpdec_params *p,
                                  float *x_out, uint8_t *bits_out, int32_t *iters_out, uint8_t *cert_out,
                                  void *cuda_stream) {
    using namespace lpdec;
    if (!codes || n_codes < 1 || n_codes > kMaxMixedCodes)
        return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: n_codes=%d must be in [1, %d]", n_codes, kMaxMixedCodes);
    if (n_frames < 0) return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: n_frames=%d < 0", n_frames);
    int rc = validate_params(p);
    if (rc) return rc;
    if (p->schedule == LPDEC_SCHED_STREAMED)
        return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: runs the RESIDENT schedule only");
    for (int c = 0; c < n_codes; ++c)
        if (!codes[c]) return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: codes[%d] is NULL", c);
    if (n_frames == 0) return LPDEC_OK;
    if (!frame_code || !llr || !x_out)
        return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: frame_code, llr and x_out must not be NULL");
    const int dev = codes[0]->device;
    for (int c = 1; c < n_codes; ++c)
        if (codes[c]->device != dev) return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: codes on different devices");

    // per-frame offsets and per-code frame lists
    std::vector<long long> offset((size_t)n_frames);
    std::vector<std::vector<int>> lists((size_t)n_codes);
    long long off = 0;
    for (int f = 0; f < n_frames; ++f) {
        const int c = frame_code[f];
        if (c < 0 || c >= n_codes)
            return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: frame_code[%d]=%d out of range", f, c);
        offset[f] = off;
        off += codes[c]->n;
        lists[c].push_back(f);
    }

    MixedArgs a;
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
            return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: code %d needs %d threads per frame (limit %d)", c,
                             tile.group_threads, kMixedMaxThreads);
        const SliceLayout L = slice_layout(cc, p->state_dtype, tile.group_threads);
        if ((int)L.bytes > cap)
            return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: code %d's frame state does not fit in shared memory", c);
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
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const void *fn = mixed_fn(p->state_dtype);
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode_mixed: cudaFuncSetAttribute");
    int bps = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, block, smem);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode_mixed: occupancy");
    if (bps < 1) return set_error(LPDEC_EINVAL, "lpdec_decode_mixed: tile does not fit on an SM");
    const int grid = bps * device_sm_count(dev);
    // home codes: CTAs split in proportion to each code's edge work
    double total = 0.0;
    for (int c = 0; c < n_codes; ++c) total += (double)a.code[c].n_frames * codes[c]->E;
    int acc = 0;
    double run = 0.0;
    for (int c = 0; c < n_codes; ++c) {
        run += (double)a.code[c].n_frames * codes[c]->E;
        acc = (int)std::lround(grid * (total > 0 ? run / total : 1.0));
        a.home_end[c] = c == n_codes - 1 ? grid : acc;
    }

    // workspace: queues, offsets, frame lists
    const size_t qb = 256, ob = ((size_t)n_frames * 8 + 255) & ~(size_t)255, lb = (size_t)n_frames * 4;
    char *work = nullptr;
    err = cudaMallocAsync(reinterpret_cast<void **>(&work), qb + ob + lb, stream);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode_mixed: cudaMallocAsync");
    a.queues = reinterpret_cast<int *>(work);
    a.offset = reinterpret_cast<const long long *>(work + qb);
    int *flat = reinterpret_cast<int *>(work + qb + ob);
    std::vector<int> flat_h;
    flat_h.reserve((size_t)n_frames);
    for (int c = 0; c < n_codes; ++c) {
        a.code[c].frames = flat + flat_h.size();
        flat_h.insert(flat_h.end(), lists[c].begin(), lists[c].end());
    }
    a.llr = llr;
    a.x_out = x_out;
    a.bits_out = bits_out;
    a.iters_out = iters_out;
    a.cert_out = cert_out;
    rc = LPDEC_OK;
    err = cudaMemsetAsync(work, 0, qb, stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(work + qb, offset.data(), (size_t)n_frames * 8, cudaMemcpyHostToDevice, stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(flat, flat_h.data(), (size_t)n_frames * 4, cudaMemcpyHostToDevice, stream);
    if (err != cudaSuccess) rc = cuda_error(err, "lpdec_decode_mixed: workspace upload");
    if (!rc) {
        void *args[] = {&a};
        err = cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, stream);
        if (err != cudaSuccess) rc = cuda_error(err, "lpdec_decode_mixed: launch");
    }
    err = cudaFreeAsync(work, stream);
    if (!rc && err != cudaSuccess) rc = cuda_error(err, "lpdec_decode_mixed: cudaFreeAsync");
    return rc;
}

// lpdec_decode_noalloc: the batch decoder for callers that must not allocate
// device memory while they run.
//
// lpdec_decode takes its scratch space (work-queue counters and, for the
// STREAMED schedule, the parked w/lambda state) from the library's
// stream-ordered memory pool on every call: an allocator call each time, and
// pool memory that stays mapped until lpdec_release_memory trims it.  Some
// callers cannot allow either: a receive loop with a fixed memory footprint
// and a latency budget that rules out allocator calls, or a host framework
// that owns all device memory through its own allocator and forbids side
// allocations.  This entry point runs the same kernels with their scratch in
// one fixed, file-scope device array instead, and makes no allocator call.
//
// The array is kLpdecNoallocScratchBytes (32 MiB) and every GPU that loads this
// library keeps it until the process exits.  It is shared by every call: the
// parts that must start at zero are cleared on the call's stream before the
// kernels run, so calls must not overlap on the GPU (two calls in flight at
// once, e.g. on different streams, race on the array).
#include <cuda_runtime.h>

#include <mutex>

#include "lpdec.h"
#include "lpdec_api_internal.h"

namespace {

constexpr size_t kLpdecNoallocScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kLpdecNoallocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (the host-side name of the array is only a stand-in).
std::mutex g_setup_mu;
void *g_scratch_ptr[64] = {nullptr};

int scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return lpdec::cuda_error(err, "lpdec_decode_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return lpdec::set_error(LPDEC_EINVAL, "lpdec_decode_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (err != cudaSuccess) return lpdec::cuda_error(err, "lpdec_decode_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return LPDEC_OK;
}

}  // namespace

extern "C" int lpdec_decode_noalloc(const lpdec_code *c, int32_t n_frames, const float *llr,
                                    const lpdec_params *p, float *x_out, uint8_t *bits_out, int32_t *iters_out,
                                    uint8_t *cert_out, void *cuda_stream) {
    if (!c) return lpdec::set_error(LPDEC_EINVAL, "lpdec_decode_noalloc: code is NULL");
    if (n_frames < 0) return lpdec::set_error(LPDEC_EINVAL, "lpdec_decode_noalloc: n_frames=%d < 0", n_frames);
    int rc = lpdec::validate_params(p);
    if (rc) return rc;
    if (n_frames == 0) return LPDEC_OK;
    if (!llr || !x_out) return lpdec::set_error(LPDEC_EINVAL, "lpdec_decode_noalloc: llr and x_out must not be NULL");
    const lpdec::Tile tile = lpdec::chosen_tile(c, p);
    const int schedule = lpdec::resolve_schedule(c, p, tile);
    const size_t need =
        lpdec::workspace_bytes(c, n_frames, schedule, p->state_dtype, p->max_iter, p->iters_per_launch);
    if (need > kLpdecNoallocScratchBytes)
        return lpdec::set_error(LPDEC_ENOMEM,
                                "lpdec_decode_noalloc: this decode needs %zu bytes of scratch but the fixed "
                                "scratch array holds %zu; use fewer frames per call or the RESIDENT schedule",
                                need, kLpdecNoallocScratchBytes);
    void *work = nullptr;
    rc = scratch_for_current_device(&work);
    if (rc) return rc;
    return lpdec::enqueue_decode(c, n_frames, llr, p, x_out, bits_out, iters_out, cert_out,
                                 static_cast<cudaStream_t>(cuda_stream), work, schedule, tile, nullptr);
}

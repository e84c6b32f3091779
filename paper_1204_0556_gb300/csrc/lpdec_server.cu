// Continuous-batching decode server (lpdec_server_*).
//
// Each code added to the server owns a pool of frame slots in device memory:
// LLRs, x/bits/iteration/certificate outputs and the parked w = z - lambda/mu and lambda/mu
// state of every frame in flight.  Each code runs its own rounds, on a stream
// of its own, and a scheduler thread keeps every code's rounds going:
//   1. for a code with no round in flight, admit pending frames (FIFO over
//      requests) into free slots: one pinned host->device copy of the new LLR
//      rows and a scatter kernel that places them and marks the slots fresh;
//   2. launch the code's round: advance every active slot by `iters_per_launch`
//      ADMM iterations with the decode kernel (STREAMED form, indexed by a slot
//      list), then copy back which slots finished (converged or reached
//      max_iter);
//   3. when a code's round completes, gather the outputs of its finished slots
//      into one compact buffer, copy it to the host, free the slots, complete
//      requests whose frames are all done, and start the code's next round.
// The codes' rounds do not wait for one another: a code with long frames
// (many iterations, many edges) does not hold back the others, and its own
// rounds follow each other with only its own bookkeeping in between.
// A frame's arithmetic depends only on its own state, and the kernel runs the
// same iterations whatever the round boundaries, so a result is identical
// whether the frame was decoded alone or among others.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lpdec.h"
#include "lpdec_api_internal.h"
#include "lpdec_internal.h"

namespace lpdec {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxSlotsPerCode = 4096;

__global__ void scatter_new_frames(int n, int count, const int *__restrict__ slots, const float *__restrict__ src,
                                   float *__restrict__ llr, int32_t *__restrict__ kst) {
    const int i = blockIdx.x;
    if (i >= count) return;
    const int s = slots[i];
    for (int t = threadIdx.x; t < n; t += blockDim.x) llr[(size_t)s * n + t] = src[(size_t)i * n + t];
    if (threadIdx.x == 0) kst[s] = 0;
}

__global__ void gather_k_state(int count, const int *__restrict__ active, const int32_t *__restrict__ kst,
                               int32_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = kst[active[i]];
}

__global__ void gather_outputs(int n, int count, const int *__restrict__ fin, const float *__restrict__ x,
                               const uint8_t *__restrict__ bits, const int32_t *__restrict__ iters,
                               const uint8_t *__restrict__ cert, float *__restrict__ xo, uint8_t *__restrict__ bo,
                               int32_t *__restrict__ io, uint8_t *__restrict__ co) {
    const int i = blockIdx.x;
    if (i >= count) return;
    const int s = fin[i];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        xo[(size_t)i * n + t] = x[(size_t)s * n + t];
        bo[(size_t)i * n + t] = bits[(size_t)s * n + t];
    }
    if (threadIdx.x == 0) {
        io[i] = iters[s];
        co[i] = cert[s];
    }
}

struct Request {
    uint64_t id = 0;
    int code_id = 0;
    int n_frames = 0;
    std::vector<float> llr;
    std::vector<float> x;
    std::vector<uint8_t> bits;
    std::vector<int32_t> iters;
    std::vector<uint8_t> cert;
    int next_frame = 0;  // frames admitted so far
    int done_frames = 0;
    Clock::time_point t_submit;
    bool done = false;
};

struct Pool {
    const lpdec_code *code = nullptr;
    lpdec_params params{};
    bool have_params = false;
    Tile tile;
    int cap = 0;
    size_t bytes = 0;
    void *dev = nullptr;  // one device allocation
    void *host = nullptr; // one pinned host allocation
    float *llr = nullptr, *x = nullptr, *d_new_llr = nullptr, *d_xo = nullptr;
    uint8_t *bits = nullptr, *cert = nullptr, *d_bo = nullptr, *d_co = nullptr;
    int32_t *iters = nullptr, *kst = nullptr, *d_kc = nullptr, *d_io = nullptr;
    void *wst = nullptr, *lst = nullptr;  // parked w = z - lambda/mu and lambda/mu, [slots x Ep]
    int *d_active = nullptr, *d_new_slots = nullptr, *d_fin = nullptr, *d_queue = nullptr;
    float *h_new_llr = nullptr, *h_xo = nullptr;
    int *h_new_slots = nullptr, *h_active = nullptr, *h_fin = nullptr;
    int32_t *h_kc = nullptr, *h_io = nullptr;
    uint8_t *h_bo = nullptr, *h_co = nullptr;
    std::vector<int> free_slots;
    std::vector<int> active;
    std::vector<std::pair<Request *, int>> owner;
    std::deque<Request *> pending;
    int n_new = 0;
    cudaStream_t stream = nullptr;  // this code's rounds run here, overlapping the other codes
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // a round's first launch; its status copy
    bool in_flight = false;                    // a round is queued; active is the list it runs on
    std::atomic<int> queued{0};  // frames in pending (read without the lock by the scheduler's wait)
    float last_end = -1e30f;     // device time [ms] at which this code's last completed round ended
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Merge device-time intervals into disjoint ones (their union is unchanged).
void merge_intervals(std::vector<std::pair<float, float>> &v) {
    std::sort(v.begin(), v.end());
    size_t k = 0;
    for (size_t i = 0; i < v.size(); ++i) {
        if (k > 0 && v[i].first <= v[k - 1].second) v[k - 1].second = std::max(v[k - 1].second, v[i].second);
        else v[k++] = v[i];
    }
    v.resize(k);
}

}  // namespace
}  // namespace lpdec

struct lpdec_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, used = 0;
    std::vector<std::unique_ptr<lpdec::Pool>> pools;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, std::unique_ptr<lpdec::Request>> reqs;
    uint64_t next_id = 1;
    bool stop = false, closed = false;
    int failed = 0;
    std::string fail_msg;
    std::thread worker;
    bool worker_started = false;
    size_t pending_frames = 0;
    // statistics of completed requests
    std::vector<double> lat_ms;
    int64_t frames_done = 0;
    double info_bits = 0.0;
    lpdec::Clock::time_point t_first, t_last;
    bool have_first = false;
    // round accounting
    int64_t rounds = 0;          // rounds of all codes
    double round_wall_ms = 0.0;  // host time of scheduler steps that had a round in flight
    cudaEvent_t ev_ref = nullptr;                 // device-time origin of the busy intervals
    std::vector<std::pair<float, float>> busy;    // device intervals [ms] of recent rounds
    double busy_settled_ms = 0.0;                 // union length of older rounds, which no later round overlaps
    size_t busy_merge_at = 256;                   // merge when busy reaches this size (doubling: amortized cost)
};

namespace lpdec {
namespace {

int pool_alloc(lpdec_server *sv, Pool &P, int slots) {
    const lpdec_code *c = P.code;
    const int n = c->n;
    const size_t sb = (size_t)c->Ep * (P.params.state_dtype == LPDEC_STATE_F32 ? 4 : 2);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align256(b); return o; };
    const size_t o_llr = take((size_t)slots * n * 4), o_x = take((size_t)slots * n * 4), o_bits = take((size_t)slots * n),
                 o_iters = take((size_t)slots * 4), o_cert = take((size_t)slots), o_w = take((size_t)slots * sb),
                 o_l = take((size_t)slots * sb), o_k = take((size_t)slots * 4), o_act = take((size_t)slots * 4),
                 o_ns = take((size_t)slots * 4), o_nl = take((size_t)slots * n * 4), o_kc = take((size_t)slots * 4),
                 o_fin = take((size_t)slots * 4), o_xo = take((size_t)slots * n * 4), o_bo = take((size_t)slots * n),
                 o_io = take((size_t)slots * 4), o_co = take((size_t)slots), o_q = take(4);
    P.bytes = off;
    cudaError_t err = cudaMalloc(&P.dev, off);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_server_add_code: cudaMalloc of the slot pool");
    char *d = static_cast<char *>(P.dev);
    P.llr = reinterpret_cast<float *>(d + o_llr);
    P.x = reinterpret_cast<float *>(d + o_x);
    P.bits = reinterpret_cast<uint8_t *>(d + o_bits);
    P.iters = reinterpret_cast<int32_t *>(d + o_iters);
    P.cert = reinterpret_cast<uint8_t *>(d + o_cert);
    P.wst = d + o_w;
    P.lst = d + o_l;
    P.kst = reinterpret_cast<int32_t *>(d + o_k);
    P.d_active = reinterpret_cast<int *>(d + o_act);
    P.d_new_slots = reinterpret_cast<int *>(d + o_ns);
    P.d_new_llr = reinterpret_cast<float *>(d + o_nl);
    P.d_kc = reinterpret_cast<int32_t *>(d + o_kc);
    P.d_fin = reinterpret_cast<int *>(d + o_fin);
    P.d_xo = reinterpret_cast<float *>(d + o_xo);
    P.d_bo = reinterpret_cast<uint8_t *>(d + o_bo);
    P.d_io = reinterpret_cast<int32_t *>(d + o_io);
    P.d_co = reinterpret_cast<uint8_t *>(d + o_co);
    P.d_queue = reinterpret_cast<int *>(d + o_q);
    // pinned staging
    size_t hoff = 0;
    auto htake = [&](size_t b) { size_t o = hoff; hoff += align256(b); return o; };
    const size_t h_nl = htake((size_t)slots * n * 4), h_ns = htake((size_t)slots * 4), h_act = htake((size_t)slots * 4),
                 h_kc = htake((size_t)slots * 4), h_fin = htake((size_t)slots * 4), h_xo = htake((size_t)slots * n * 4),
                 h_bo = htake((size_t)slots * n), h_io = htake((size_t)slots * 4), h_co = htake((size_t)slots);
    err = cudaMallocHost(&P.host, hoff);
    if (err != cudaSuccess) {
        cudaFree(P.dev);
        P.dev = nullptr;
        return cuda_error(err, "lpdec_server_add_code: cudaMallocHost of the staging buffers");
    }
    char *h = static_cast<char *>(P.host);
    P.h_new_llr = reinterpret_cast<float *>(h + h_nl);
    P.h_new_slots = reinterpret_cast<int *>(h + h_ns);
    P.h_active = reinterpret_cast<int *>(h + h_act);
    P.h_kc = reinterpret_cast<int32_t *>(h + h_kc);
    P.h_fin = reinterpret_cast<int *>(h + h_fin);
    P.h_xo = reinterpret_cast<float *>(h + h_xo);
    P.h_bo = reinterpret_cast<uint8_t *>(h + h_bo);
    P.h_io = reinterpret_cast<int32_t *>(h + h_io);
    P.h_co = reinterpret_cast<uint8_t *>(h + h_co);
    err = cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreate(&P.ev0);
    if (err == cudaSuccess) err = cudaEventCreate(&P.ev1);
    if (err != cudaSuccess) {
        cudaFree(P.dev);
        cudaFreeHost(P.host);
        P.dev = P.host = nullptr;
        return cuda_error(err, "lpdec_server_add_code: stream creation");
    }
    // the code's first round follows whatever the caller queued on the server stream
    cudaEvent_t after;
    if (cudaEventCreateWithFlags(&after, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(after, sv->stream);
        cudaStreamWaitEvent(P.stream, after, 0);
        cudaEventDestroy(after);
    }
    P.cap = slots;
    P.free_slots.resize(slots);
    for (int s = 0; s < slots; ++s) P.free_slots[s] = slots - 1 - s;
    P.owner.assign(slots, {nullptr, 0});
    sv->used += off;
    return LPDEC_OK;
}

// Admission for a code with no round in flight (the caller holds the lock).
void admit_locked(lpdec_server *sv, Pool &P) {
    P.n_new = 0;
    const int n = P.code->n;
    while (!P.pending.empty() && !P.free_slots.empty()) {
        Request *r = P.pending.front();
        while (r->next_frame < r->n_frames && !P.free_slots.empty()) {
            const int s = P.free_slots.back();
            P.free_slots.pop_back();
            std::memcpy(P.h_new_llr + (size_t)P.n_new * n, r->llr.data() + (size_t)r->next_frame * n, (size_t)n * 4);
            P.h_new_slots[P.n_new++] = s;
            P.owner[s] = {r, r->next_frame};
            P.active.push_back(s);
            ++r->next_frame;
            --sv->pending_frames;
            P.queued.fetch_sub(1, std::memory_order_relaxed);
        }
        if (r->next_frame == r->n_frames) P.pending.pop_front();
    }
}

// Queue one round of a code on its stream (no lock held; the scheduler thread
// alone touches a pool's device buffers and its active list while in flight).
int launch_round(lpdec_server *sv, Pool &P) {
    cudaStream_t st = P.stream;
    cudaError_t err;
    if (!sv->ev_ref) {
        // the origin of the busy intervals, recorded on a stream of its own so
        // that it completes at once (the code streams may wait on the caller's work)
        cudaStream_t s0 = nullptr;
        err = cudaEventCreate(&sv->ev_ref);
        if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventRecord(sv->ev_ref, s0);
        if (err == cudaSuccess) err = cudaEventSynchronize(sv->ev_ref);
        if (s0) cudaStreamDestroy(s0);
        if (err != cudaSuccess) return cuda_error(err, "server: reference event");
    }
    cudaEventRecord(P.ev0, st);
    const int n = P.code->n;
    if (P.n_new > 0) {
        err = cudaMemcpyAsync(P.d_new_llr, P.h_new_llr, (size_t)P.n_new * n * 4, cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(P.d_new_slots, P.h_new_slots, (size_t)P.n_new * 4, cudaMemcpyHostToDevice, st);
        if (err != cudaSuccess) return cuda_error(err, "server: admission copy");
        scatter_new_frames<<<P.n_new, 128, 0, st>>>(n, P.n_new, P.d_new_slots, P.d_new_llr, P.llr, P.kst);
    }
    const int na = (int)P.active.size();
    std::memcpy(P.h_active, P.active.data(), (size_t)na * 4);
    err = cudaMemcpyAsync(P.d_active, P.h_active, (size_t)na * 4, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(P.d_queue, 0, 4, st);
    if (err != cudaSuccess) return cuda_error(err, "server: round set-up");
    DecodeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.code = make_view(P.code);
    a.cfg = make_cfg(P.code, &P.params);
    a.n_frames = na;
    a.llr = P.llr;
    a.x_out = P.x;
    a.bits_out = P.bits;
    a.iters_out = P.iters;
    a.cert_out = P.cert;
    a.w_state = P.wst;
    a.l_state = P.lst;
    a.k_state = P.kst;
    a.iters_this_launch = P.params.iters_per_launch;
    a.frame_list = P.d_active;
    a.queue = P.d_queue;
    int rc = launch_once(P.code, P.params.state_dtype, P.tile, a, st);
    if (rc) return rc;
    gather_k_state<<<(na + 255) / 256, 256, 0, st>>>(na, P.d_active, P.kst, P.d_kc);
    err = cudaMemcpyAsync(P.h_kc, P.d_kc, (size_t)na * 4, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaEventRecord(P.ev1, st);
    if (err != cudaSuccess) return cuda_error(err, "server: status copy");
    P.in_flight = true;
    return LPDEC_OK;
}

// A code's round has completed (ev1 reached): retire its finished slots and
// hand their outputs to their requests.
int finish_round(lpdec_server *sv, Pool &P) {
    cudaError_t err;
    float t0 = 0.0f, t1 = 0.0f;
    const bool timed = cudaEventElapsedTime(&t0, sv->ev_ref, P.ev0) == cudaSuccess &&
                       cudaEventElapsedTime(&t1, sv->ev_ref, P.ev1) == cudaSuccess;
    const int na = (int)P.active.size();
    int nf = 0;
    for (int i = 0; i < na; ++i)
        if (P.h_kc[i] < 0) P.h_fin[nf++] = P.active[i];
    const int n = P.code->n;
    if (nf) {
        cudaStream_t st = P.stream;
        err = cudaMemcpyAsync(P.d_fin, P.h_fin, (size_t)nf * 4, cudaMemcpyHostToDevice, st);
        if (err != cudaSuccess) return cuda_error(err, "server: finished list copy");
        gather_outputs<<<nf, 128, 0, st>>>(n, nf, P.d_fin, P.x, P.bits, P.iters, P.cert, P.d_xo, P.d_bo, P.d_io,
                                           P.d_co);
        err = cudaMemcpyAsync(P.h_xo, P.d_xo, (size_t)nf * n * 4, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(P.h_bo, P.d_bo, (size_t)nf * n, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(P.h_io, P.d_io, (size_t)nf * 4, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(P.h_co, P.d_co, (size_t)nf, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) return cuda_error(err, "server: output gather");
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    const auto now = Clock::now();
    bool any_done = false;
    for (int i = 0; i < nf; ++i) {
        const int s = P.h_fin[i];
        Request *r = P.owner[s].first;
        const int fr = P.owner[s].second;
        std::memcpy(r->x.data() + (size_t)fr * n, P.h_xo + (size_t)i * n, (size_t)n * 4);
        std::memcpy(r->bits.data() + (size_t)fr * n, P.h_bo + (size_t)i * n, (size_t)n);
        r->iters[fr] = P.h_io[i];
        r->cert[fr] = P.h_co[i];
        P.owner[s] = {nullptr, 0};
        P.free_slots.push_back(s);
        if (++r->done_frames == r->n_frames) {
            r->done = true;
            any_done = true;
            const double ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
            sv->lat_ms.push_back(ms);
            sv->frames_done += r->n_frames;
            sv->info_bits += (double)r->n_frames * (P.code->n - P.code->m);
            sv->t_last = now;
        }
    }
    if (nf) {  // drop finished slots from the active list
        std::vector<int> keep;
        keep.reserve(P.active.size());
        for (int i = 0; i < na; ++i)
            if (P.h_kc[i] >= 0) keep.push_back(P.active[i]);
        P.active.swap(keep);
    }
    P.in_flight = false;
    if (any_done) sv->cv_done.notify_all();
    sv->rounds += 1;
    if (timed) {
        sv->busy.emplace_back(t0, t1);
        P.last_end = t1;
    }
    if (sv->busy.size() >= sv->busy_merge_at) {
        // A round not yet completed runs on its code's stream after that code's
        // last completed round, and a round launched later starts later still:
        // no future interval begins before the earliest last_end of the codes
        // in flight.  The merged intervals that end before it are settled.
        merge_intervals(sv->busy);
        float horizon = 1e30f;
        for (auto &pp : sv->pools)
            if (pp->in_flight) horizon = std::min(horizon, pp->last_end);
        size_t k = 0;
        while (k < sv->busy.size() && sv->busy[k].second <= horizon) {
            sv->busy_settled_ms += (double)(sv->busy[k].second - sv->busy[k].first);
            ++k;
        }
        sv->busy.erase(sv->busy.begin(), sv->busy.begin() + (long)k);
        sv->busy_merge_at = std::max<size_t>(256, 2 * sv->busy.size());
    }
    return LPDEC_OK;
}

// One scheduler step: start a round for every code that has none in flight and
// has frames to run, then wait until some round completes (or new frames
// arrive for an idle code) and retire the completed rounds.  Returns an LPDEC
// status; the caller holds no lock.  lpdec_server_add_code may append to
// sv->pools at any time (under the lock), so the step works on a copy of the
// pool pointers taken under the lock; the Pool objects themselves never move.
int run_step(lpdec_server *sv) {
    const auto t_step = Clock::now();
    std::vector<Pool *> pools, start;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        pools.reserve(sv->pools.size());
        for (auto &pp : sv->pools) pools.push_back(pp.get());
        for (Pool *pp : pools) {
            if (pp->in_flight) continue;
            admit_locked(sv, *pp);
            if (!pp->active.empty()) start.push_back(pp);
        }
    }
    for (Pool *pp : start) {
        const int rc = launch_round(sv, *pp);
        if (rc) return rc;
    }
    bool any_flight = false;
    for (Pool *pp : pools) any_flight |= pp->in_flight;
    if (!any_flight) return LPDEC_OK;
    // wait for a completed round, or for frames that an idle code could start on
    std::vector<Pool *> done;
    for (;;) {
        for (Pool *pp : pools) {
            if (!pp->in_flight) continue;
            const cudaError_t q = cudaEventQuery(pp->ev1);
            if (q == cudaSuccess) done.push_back(pp);
            else if (q != cudaErrorNotReady) return cuda_error(q, "server: round");
        }
        if (!done.empty()) break;
        // (without the lock, which the submitting threads need: in_flight
        // changes only on this thread, queued is atomic, and free_slots, sized
        // by the code's first submit before it raises queued, changes only on
        // this thread afterwards)
        bool idle_work = false;
        for (Pool *pp : pools)
            if (!pp->in_flight && pp->queued.load(std::memory_order_acquire) > 0 && !pp->free_slots.empty())
                idle_work = true;
        if (idle_work) break;
        // spin (yielding the core): a sleep of even 20 us measurably delays
        // every round of a code whose rounds are short
        std::this_thread::yield();
    }
    for (Pool *pp : done) {
        const int rc = finish_round(sv, *pp);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->round_wall_ms += std::chrono::duration<double, std::milli>(Clock::now() - t_step).count();
    return LPDEC_OK;
}

void worker_main(lpdec_server *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] {
                if (sv->stop) return true;
                for (auto &pp : sv->pools)
                    if (!pp->active.empty() || !pp->pending.empty()) return true;
                return false;
            });
            bool busy = false;
            for (auto &pp : sv->pools)
                if (!pp->active.empty() || !pp->pending.empty()) busy = true;
            if (sv->stop && !busy) return;
        }
        const int rc = run_step(sv);
        if (rc) {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->failed = rc;
            sv->fail_msg = lpdec_last_error();
            sv->cv_done.notify_all();
            return;
        }
    }
}

}  // namespace
}  // namespace lpdec

using lpdec::set_error;

extern "C" int lpdec_server_create(size_t device_budget_bytes, void *cuda_stream, lpdec_server **out) {
    if (!out) return set_error(LPDEC_EINVAL, "lpdec_server_create: out is NULL");
    if (device_budget_bytes == 0) return set_error(LPDEC_EINVAL, "lpdec_server_create: budget must be > 0");
    auto *sv = new (std::nothrow) lpdec_server();
    if (!sv) return set_error(LPDEC_ENOMEM, "lpdec_server_create: host allocation failed");
    cudaError_t err = cudaGetDevice(&sv->device);
    if (err != cudaSuccess) {
        delete sv;
        return lpdec::cuda_error(err, "lpdec_server_create: cudaGetDevice");
    }
    sv->budget = device_budget_bytes;
    if (cuda_stream) {
        sv->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        err = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) {
            delete sv;
            return lpdec::cuda_error(err, "lpdec_server_create: cudaStreamCreate");
        }
        sv->own_stream = true;
    }
    *out = sv;
    return LPDEC_OK;
}

extern "C" int lpdec_server_add_code(lpdec_server *sv, const lpdec_code *code, int32_t *code_id) {
    if (!sv || !code || !code_id) return set_error(LPDEC_EINVAL, "lpdec_server_add_code: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->closed) return set_error(LPDEC_ECLOSED, "lpdec_server_add_code: server is shut down");
    if (code->device != sv->device) return set_error(LPDEC_EINVAL, "lpdec_server_add_code: code on another device");
    auto P = std::make_unique<lpdec::Pool>();
    P->code = code;
    *code_id = (int32_t)sv->pools.size();
    sv->pools.push_back(std::move(P));
    return LPDEC_OK;
}

extern "C" int lpdec_server_submit(lpdec_server *sv, int32_t code_id, int32_t n_frames, const float *llr_host,
                                   const lpdec_params *p, uint64_t *request_id) {
    if (!sv || !llr_host || !request_id) return set_error(LPDEC_EINVAL, "lpdec_server_submit: NULL argument");
    if (n_frames < 1) return set_error(LPDEC_EINVAL, "lpdec_server_submit: n_frames=%d must be >= 1", n_frames);
    int rc = lpdec::validate_params(p);
    if (rc) return rc;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->closed) return set_error(LPDEC_ECLOSED, "lpdec_server_submit: server is shut down");
    if (sv->failed) return set_error(sv->failed, "lpdec_server_submit: server failed: %s", sv->fail_msg.c_str());
    if (code_id < 0 || code_id >= (int)sv->pools.size())
        return set_error(LPDEC_EINVAL, "lpdec_server_submit: unknown code_id %d", code_id);
    lpdec::Pool &P = *sv->pools[code_id];
    if (!P.have_params) {
        // first request fixes the code's parameters and sizes its slot pool
        lpdec::Tile tile = P.code->tuned[p->state_dtype].valid ? P.code->tuned[p->state_dtype]
                                                                 : lpdec::default_tile(P.code, p->state_dtype);
        const lpdec::SliceLayout L = lpdec::slice_layout(P.code, p->state_dtype, tile.group_threads);
        if ((int)L.bytes > lpdec::device_smem_optin(sv->device))
            return set_error(LPDEC_EINVAL, "lpdec_server_submit: frame state of code %d does not fit in shared memory",
                             code_id);
        P.params = *p;
        P.tile = tile;
        const int n = P.code->n;
        const size_t per_slot = 2 * (size_t)P.code->Ep * (p->state_dtype == LPDEC_STATE_F32 ? 4 : 2) +
                                (size_t)n * 4 * 3 + (size_t)n * 2 + 64;
        const size_t left = sv->budget > sv->used ? sv->budget - sv->used : 0;
        const int slots = (int)std::min<size_t>(lpdec::kMaxSlotsPerCode, left / per_slot);
        if (slots < 1)
            return set_error(LPDEC_ENOMEM, "lpdec_server_submit: device budget exhausted (%zu of %zu bytes used)",
                             sv->used, sv->budget);
        rc = lpdec::pool_alloc(sv, P, slots);  // under the lock: one sizing per code
        if (rc) return rc;
        P.have_params = true;
    } else if (std::memcmp(&P.params, p, sizeof(*p)) != 0) {
        return set_error(LPDEC_EINVAL, "lpdec_server_submit: a code's requests must share one parameter set");
    }
    const size_t max_pending = 4 * (size_t)P.cap + 16;
    if (sv->pending_frames + (size_t)n_frames > max_pending * sv->pools.size())
        return set_error(LPDEC_EBUSY, "lpdec_server_submit: %zu frames already queued", sv->pending_frames);
    auto r = std::make_unique<lpdec::Request>();
    const int n = P.code->n;
    r->id = sv->next_id++;
    r->code_id = code_id;
    r->n_frames = n_frames;
    r->llr.assign(llr_host, llr_host + (size_t)n_frames * n);
    r->x.resize((size_t)n_frames * n);
    r->bits.resize((size_t)n_frames * n);
    r->iters.resize(n_frames);
    r->cert.resize(n_frames);
    r->t_submit = lpdec::Clock::now();
    if (!sv->have_first) {
        sv->t_first = r->t_submit;
        sv->have_first = true;
    }
    P.pending.push_back(r.get());
    P.queued.fetch_add(n_frames, std::memory_order_release);  // after the pool's first sizing
    sv->pending_frames += n_frames;
    *request_id = r->id;
    sv->reqs.emplace(r->id, std::move(r));
    if (!sv->worker_started) {
        sv->worker = std::thread(lpdec::worker_main, sv);
        sv->worker_started = true;
    }
    sv->cv_work.notify_one();
    return LPDEC_OK;
}

extern "C" int lpdec_server_poll(lpdec_server *sv, uint64_t request_id, int32_t timeout_ms, float *x, uint8_t *bits,
                                 int32_t *iters, uint8_t *cert) {
    if (!sv) return set_error(LPDEC_EINVAL, "lpdec_server_poll: server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(request_id);
    if (it == sv->reqs.end()) return set_error(LPDEC_EINVAL, "lpdec_server_poll: unknown request %llu",
                                               (unsigned long long)request_id);
    lpdec::Request *r = it->second.get();
    const auto pred = [&] { return r->done || sv->failed != 0; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, pred);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        return set_error(LPDEC_ETIMEOUT, "lpdec_server_poll: request %llu not done within %d ms",
                         (unsigned long long)request_id, timeout_ms);
    }
    if (!r->done) return set_error(sv->failed, "lpdec_server_poll: server failed: %s", sv->fail_msg.c_str());
    if (x) std::memcpy(x, r->x.data(), r->x.size() * 4);
    if (bits) std::memcpy(bits, r->bits.data(), r->bits.size());
    if (iters) std::memcpy(iters, r->iters.data(), r->iters.size() * 4);
    if (cert) std::memcpy(cert, r->cert.data(), r->cert.size());
    sv->reqs.erase(it);
    return LPDEC_OK;
}

extern "C" int lpdec_server_stats(lpdec_server *sv, double *p50_ms, double *p99_ms, double *bits_per_s,
                                  int64_t *frames) {
    if (!sv) return set_error(LPDEC_EINVAL, "lpdec_server_stats: server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::vector<double> v = sv->lat_ms;
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
        std::nth_element(v.begin(), v.begin() + k, v.end());
        return v[k];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (bits_per_s) {
        const double s = sv->have_first ? std::chrono::duration<double>(sv->t_last - sv->t_first).count() : 0.0;
        *bits_per_s = s > 0 ? sv->info_bits / s : 0.0;
    }
    if (frames) *frames = sv->frames_done;
    return LPDEC_OK;
}

extern "C" int lpdec_server_counters(lpdec_server *sv, int64_t *rounds, double *round_wall_ms,
                                     double *round_gpu_ms) {
    if (!sv) return set_error(LPDEC_EINVAL, "lpdec_server_counters: server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (rounds) *rounds = sv->rounds;
    if (round_wall_ms) *round_wall_ms = sv->round_wall_ms;
    if (round_gpu_ms) {
        lpdec::merge_intervals(sv->busy);
        double ms = sv->busy_settled_ms;
        for (const auto &iv : sv->busy) ms += (double)(iv.second - iv.first);
        *round_gpu_ms = ms;
    }
    return LPDEC_OK;
}

extern "C" int lpdec_server_destroy(lpdec_server *sv) {
    if (!sv) return set_error(LPDEC_EINVAL, "lpdec_server_destroy: server is NULL");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->closed = true;
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker_started) sv->worker.join();  // drains the frames already submitted
    int rc = LPDEC_OK;
    for (auto &pp : sv->pools) {
        if (pp->stream) cudaStreamSynchronize(pp->stream);
        if (pp->dev && cudaFree(pp->dev) != cudaSuccess) rc = LPDEC_ECUDA;
        if (pp->host && cudaFreeHost(pp->host) != cudaSuccess) rc = LPDEC_ECUDA;
        if (pp->ev0) cudaEventDestroy(pp->ev0);
        if (pp->ev1) cudaEventDestroy(pp->ev1);
        if (pp->stream) cudaStreamDestroy(pp->stream);
    }
    if (sv->ev_ref) cudaEventDestroy(sv->ev_ref);
    if (sv->own_stream) cudaStreamDestroy(sv->stream);
    delete sv;
    if (rc) return set_error(rc, "lpdec_server_destroy: freeing device memory failed");
    return LPDEC_OK;
}

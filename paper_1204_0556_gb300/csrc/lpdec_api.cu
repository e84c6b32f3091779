// C-ABI layer of liblpdec: argument validation, the code object, workspace,
// tile selection and kernel launches.  Declarations and error semantics are
// in include/lpdec.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lpdec.h"
#include "lpdec_api_internal.h"
#include "lpdec_internal.h"

using lpdec::DecodeArgs;

// ---------------------------------------------------------------------------
// errors
namespace {
thread_local std::string g_last_error;
}

namespace lpdec {
int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}
int cuda_error(cudaError_t e, const char *what) {
    return set_error(e == cudaErrorMemoryAllocation ? LPDEC_ENOMEM : LPDEC_ECUDA, "%s: %s (%s)", what,
                     cudaGetErrorString(e), cudaGetErrorName(e));
}
}  // namespace lpdec

using lpdec::cuda_error;
using lpdec::set_error;

extern "C" const char *lpdec_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *lpdec_version(void) { return "liblpdec 0.1 (sm_103a)"; }

extern "C" void lpdec_params_default(lpdec_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->mu = 3.0;
    p->rho = 1.9;
    p->eps = 1e-5;
    p->max_iter = 1000;
    p->state_dtype = LPDEC_STATE_F32;
    p->cert_tol = 1e-2;
    p->schedule = LPDEC_SCHED_AUTO;
    p->iters_per_launch = 1;
}

// ---------------------------------------------------------------------------
// code object

// n - rank over GF(2) of H, by Gaussian elimination on packed rows.
static int gf2_k_rank(int n, int m, const int32_t *row_ptr, const int32_t *col_idx) {
    const int W = (n + 63) / 64;
    std::vector<uint64_t> a((size_t)m * W, 0);
    for (int j = 0; j < m; ++j)
        for (int e = row_ptr[j]; e < row_ptr[j + 1]; ++e)
            a[(size_t)j * W + col_idx[e] / 64] |= 1ull << (col_idx[e] % 64);
    int rank = 0;
    for (int col = 0; col < n && rank < m; ++col) {
        const int wd = col / 64;
        const uint64_t bit = 1ull << (col % 64);
        int piv = -1;
        for (int r = rank; r < m; ++r)
            if (a[(size_t)r * W + wd] & bit) { piv = r; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int q = 0; q < W; ++q) std::swap(a[(size_t)piv * W + q], a[(size_t)rank * W + q]);
        for (int r = 0; r < m; ++r)
            if (r != rank && (a[(size_t)r * W + wd] & bit))
                for (int q = wd; q < W; ++q) a[(size_t)r * W + q] ^= a[(size_t)rank * W + q];
        ++rank;
    }
    return n - rank;
}

// Order each variable's edges within its index slots so that the 32 variables
// a warp handles together touch as few shared-memory banks twice as possible in
// every slot: the x-update gathers w (and, folding, scatters u) slot by slot, and
// w[e] of FP32 state sits in bank e mod 32.  Greedy over the permutations of each
// variable's edges, three passes per block of 32 variables.  Only the order of a
// variable's (commutative) sum changes.
static void order_edge_slots(uint16_t *csc, int n, int dv) {
    for (int b0 = 0; b0 < n; b0 += 32) {
        const int b1 = std::min(n, b0 + 32);
        int cnt[4][32] = {};
        for (int i = b0; i < b1; ++i)
            for (int s = 0; s < dv; ++s) ++cnt[s][csc[(size_t)i * 4 + s] & 31];
        for (int pass = 0; pass < 3; ++pass) {
            for (int i = b0; i < b1; ++i) {
                uint16_t *v = csc + (size_t)i * 4;
                for (int s = 0; s < dv; ++s) --cnt[s][v[s] & 31];
                uint16_t cur[4] = {v[0], v[1], v[2], v[3]};
                uint16_t best[4] = {v[0], v[1], v[2], v[3]};
                int best_cost = 0;
                for (int s = 0; s < dv; ++s) best_cost += cnt[s][cur[s] & 31];
                std::sort(cur, cur + dv);
                do {
                    int cost = 0;
                    for (int s = 0; s < dv; ++s) cost += cnt[s][cur[s] & 31];
                    if (cost < best_cost) {
                        best_cost = cost;
                        std::copy(cur, cur + dv, best);
                    }
                } while (std::next_permutation(cur, cur + dv));
                std::copy(best, best + dv, v);
                for (int s = 0; s < dv; ++s) ++cnt[s][v[s] & 31];
            }
        }
    }
}

// Processing order of the checks of a wide code whose check degrees differ.
// A warp's 16 lane pairs take 16 consecutive entries of the order, and pair p
// reads words e0_p + 2k and e0_p + 2k + 1 of the edge state (e0_p: its check's
// first edge), so the warp's accesses fall in distinct banks when the 16
// offsets share a parity and are distinct mod 32.  The checks are bucketed by
// e0 mod 32 and dealt out in groups of 16, one per bucket of a parity, fullest
// buckets first; groups are padded from the fullest buckets when a parity runs
// short.  (C8000: 2.7 -> 1.2 wavefronts per check-update access, simulated;
// 2.67e11 -> 2.74e11 edge-iterations/s measured at 300 iterations.)
// Only the order in which checks are taken changes, not what is computed.
static void check_order_for_banks(int m, const int32_t *row_ptr, int32_t *order) {
    std::vector<std::vector<int32_t>> bucket(32);
    for (int j = m - 1; j >= 0; --j) bucket[row_ptr[j] & 31].push_back(j);  // popped in index order
    int pos = 0;
    for (int par = 0; par < 2; ++par) {
        auto left = [&] {
            for (int r = par; r < 32; r += 2)
                if (!bucket[r].empty()) return true;
            return false;
        };
        while (left()) {
            int rs[16], nr = 0;
            for (int r = par; r < 32; r += 2) rs[nr++] = r;
            std::stable_sort(rs, rs + nr, [&](int a, int b) { return bucket[a].size() > bucket[b].size(); });
            int taken = 0;
            for (int q = 0; q < nr && taken < 16; ++q)
                if (!bucket[rs[q]].empty()) {
                    order[pos++] = bucket[rs[q]].back();
                    bucket[rs[q]].pop_back();
                    ++taken;
                }
            while (taken < 16) {  // this parity runs short: fill from its fullest buckets
                int best = -1;
                for (int r = par; r < 32; r += 2)
                    if (!bucket[r].empty() && (best < 0 || bucket[r].size() > bucket[best].size())) best = r;
                if (best < 0) break;
                order[pos++] = bucket[best].back();
                bucket[best].pop_back();
                ++taken;
            }
        }
    }
}

extern "C" int lpdec_code_create(int32_t n, int32_t m, const int32_t *row_ptr, const int32_t *col_idx,
                                 const int32_t *col_ptr, const int32_t *row_idx, const int32_t *edge_perm,
                                 lpdec_code **out) {
    if (!out) return set_error(LPDEC_EINVAL, "lpdec_code_create: out is NULL");
    if (n <= 0 || m <= 0) return set_error(LPDEC_EINVAL, "lpdec_code_create: n=%d m=%d must be positive", n, m);
    if (!row_ptr || !col_idx || !col_ptr || !row_idx || !edge_perm)
        return set_error(LPDEC_EINVAL, "lpdec_code_create: NULL index array");
    if (row_ptr[0] != 0 || col_ptr[0] != 0)
        return set_error(LPDEC_EINVAL, "lpdec_code_create: row_ptr[0] and col_ptr[0] must be 0");
    int max_dc = 0;
    for (int j = 0; j < m; ++j) {
        const int d = row_ptr[j + 1] - row_ptr[j];
        if (d < 1 || d > 32)
            return set_error(LPDEC_EINVAL, "lpdec_code_create: check %d has degree %d (must be 1..32)", j, d);
        max_dc = std::max(max_dc, d);
    }
    const int64_t E = row_ptr[m];
    if (E > (int64_t)1 << 30) return set_error(LPDEC_EINVAL, "lpdec_code_create: too many edges");
    if (col_ptr[n] != E) return set_error(LPDEC_EINVAL, "lpdec_code_create: col_ptr[n]=%d != E=%lld", col_ptr[n], (long long)E);
    for (int j = 0; j < m; ++j)
        for (int e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
            if (col_idx[e] < 0 || col_idx[e] >= n)
                return set_error(LPDEC_EINVAL, "lpdec_code_create: col_idx[%d]=%d out of range", e, col_idx[e]);
            if (e > row_ptr[j] && col_idx[e] <= col_idx[e - 1])
                return set_error(LPDEC_EINVAL, "lpdec_code_create: columns of check %d not strictly ascending", j);
        }
    for (int i = 0; i < n; ++i)
        if (col_ptr[i + 1] < col_ptr[i] || col_ptr[i + 1] > E)
            return set_error(LPDEC_EINVAL, "lpdec_code_create: col_ptr is not nondecreasing within [0, E]");
    std::vector<int32_t> edge_row((size_t)E);
    for (int j = 0; j < m; ++j)
        for (int e = row_ptr[j]; e < row_ptr[j + 1]; ++e) edge_row[e] = j;
    std::vector<uint8_t> seen((size_t)E, 0);
    for (int i = 0; i < n; ++i) {
        const int d = col_ptr[i + 1] - col_ptr[i];
        if (d < 1) return set_error(LPDEC_EINVAL, "lpdec_code_create: variable %d has degree %d (must be >= 1)", i, d);
        for (int s = col_ptr[i]; s < col_ptr[i + 1]; ++s) {
            const int e = edge_perm[s];
            if (e < 0 || e >= E || seen[e])
                return set_error(LPDEC_EINVAL, "lpdec_code_create: edge_perm[%d]=%d invalid or repeated", s, e);
            seen[e] = 1;
            if (col_idx[e] != i || edge_row[e] != row_idx[s])
                return set_error(LPDEC_EINVAL, "lpdec_code_create: CSC slot %d disagrees with CSR edge %d", s, e);
            if (s > col_ptr[i] && row_idx[s] <= row_idx[s - 1])
                return set_error(LPDEC_EINVAL, "lpdec_code_create: rows of variable %d not strictly ascending", i);
        }
    }

    lpdec_code *c = new (std::nothrow) lpdec_code();
    if (!c) return set_error(LPDEC_ENOMEM, "lpdec_code_create: host allocation failed");
    c->n = n;
    c->m = m;
    c->E = (int)E;
    c->Ep = (int)((E + 7) / 8 * 8);
    c->max_dc = max_dc;
    c->k_rank = gf2_k_rank(n, m, row_ptr, col_idx);
    c->cls = lpdec::degree_class(max_dc);
    // Regular codes (one check degree, one variable degree) run the regular-code
    // kernel, which takes variable edges from i*dv slots and check edges from
    // j*dc: (3,6)-type codes in the class D = 6 and (4,8) in D = 8 (check degree
    // equal to the class width); in the wide classes, any code whose variables
    // all have degree 3 (reg_dc = 0 when the check degrees differ: the check
    // update then takes its edge range from row_ptr).
    {
        const int dc0 = row_ptr[1] - row_ptr[0], dv0 = col_ptr[1] - col_ptr[0];
        bool reg_c = true, reg_v = true;
        for (int j = 0; j < m && reg_c; ++j) reg_c = (row_ptr[j + 1] - row_ptr[j]) == dc0;
        for (int i = 0; i < n && reg_v; ++i) reg_v = (col_ptr[i + 1] - col_ptr[i]) == dv0;
        const int D = lpdec::kClassD[c->cls];
        if (D <= 8) {
            const bool reg = reg_c && reg_v && dv0 == (D == 8 ? 4 : 3) && dc0 == D;
            c->reg_dv = reg ? dv0 : 0;
            c->reg_dc = reg ? dc0 : 0;
        } else {
            c->reg_dv = (reg_v && dv0 == 3) ? 3 : 0;
            c->reg_dc = (c->reg_dv && reg_c) ? dc0 : 0;
        }
    }
    cudaError_t err = cudaGetDevice(&c->device);
    if (err != cudaSuccess) { delete c; return cuda_error(err, "lpdec_code_create: cudaGetDevice"); }
    // Four index arrays in one allocation, each starting on a 16-byte boundary,
    // plus (wide classes with differing check degrees) the check order.
    auto pad4 = [](size_t w) { return (w + 3) & ~(size_t)3; };
    const bool ordered = lpdec::kClassD[c->cls] > 8 && c->reg_dc == 0;
    const size_t o_row = 0, o_col = pad4((size_t)m + 1), o_cptr = o_col + pad4((size_t)E),
                 o_csc = o_cptr + pad4((size_t)n + 1), o_ord = o_csc + pad4((size_t)E),
                 words = o_ord + (ordered ? pad4((size_t)m) : 0);
    err = cudaMalloc(&c->dev_block, words * sizeof(int32_t));
    if (err != cudaSuccess) { delete c; return cuda_error(err, "lpdec_code_create: cudaMalloc"); }
    int32_t *p = static_cast<int32_t *>(c->dev_block);
    c->row_ptr = p + o_row;
    c->col_idx = p + o_col;
    c->col_ptr = p + o_cptr;
    c->csc_edge = p + o_csc;
    c->check_order = ordered ? p + o_ord : nullptr;
    std::vector<int32_t> host(words, 0);
    if (ordered) check_order_for_banks(m, row_ptr, host.data() + o_ord);
    std::copy(row_ptr, row_ptr + m + 1, host.begin() + o_row);
    std::copy(col_idx, col_idx + E, host.begin() + o_col);
    std::copy(col_ptr, col_ptr + n + 1, host.begin() + o_cptr);
    std::copy(edge_perm, edge_perm + E, host.begin() + o_csc);
    err = cudaMemcpy(c->dev_block, host.data(), words * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        cudaFree(c->dev_block);
        delete c;
        return cuda_error(err, "lpdec_code_create: cudaMemcpy");
    }
    // Regular codes: 16-bit index block for the regular-form kernels.  Codes
    // whose indices need more than 16 bits run the generic form instead.
    if (c->reg_dv > 0 && (E > 65535 || n > 65535 || c->reg_dv > 4)) c->reg_dv = c->reg_dc = 0;
    if (c->reg_dv > 0) {
        c->col16_elems = (int)((E + 7) / 8 * 8);
        c->idx16_bytes = (int)((size_t)c->col16_elems * 2 + (((size_t)n * 8 + 15) & ~(size_t)15));  // copy16 moves 16-byte units
        std::vector<uint16_t> h16((size_t)c->idx16_bytes / 2, 0);
        for (int64_t e = 0; e < E; ++e) h16[(size_t)e] = (uint16_t)col_idx[e];
        uint16_t *csc = h16.data() + c->col16_elems;
        // (4,8) form: the edge state sits at the swizzled position of each
        // edge (lpdec::state_pos), so the variable phase gathers from there.
        const bool swz = lpdec::kClassD[c->cls] == 8;
        for (int i = 0; i < n; ++i)
            for (int s = col_ptr[i]; s < col_ptr[i + 1]; ++s) {
                const int e = edge_perm[s];
                csc[(size_t)i * 4 + (s - col_ptr[i])] = (uint16_t)(swz ? lpdec::state_pos8(e) : e);
            }
        order_edge_slots(csc, n, c->reg_dv);
        err = cudaMalloc(&c->dev_idx16, (size_t)c->idx16_bytes);
        if (err == cudaSuccess)
            err = cudaMemcpy(c->dev_idx16, h16.data(), (size_t)c->idx16_bytes, cudaMemcpyHostToDevice);
        if (err != cudaSuccess) {
            cudaFree(c->dev_idx16);
            cudaFree(c->dev_block);
            delete c;
            return cuda_error(err, "lpdec_code_create: 16-bit index block");
        }
    }
    *out = c;
    return LPDEC_OK;
}

extern "C" int lpdec_code_info(const lpdec_code *c, int32_t *n, int32_t *m, int64_t *E, int32_t *max_dc,
                               int32_t *k_rank) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_code_info: code is NULL");
    if (n) *n = c->n;
    if (m) *m = c->m;
    if (E) *E = c->E;
    if (max_dc) *max_dc = c->max_dc;
    if (k_rank) *k_rank = c->k_rank;
    return LPDEC_OK;
}

extern "C" int lpdec_code_destroy(lpdec_code *c) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_code_destroy: code is NULL");
    cudaError_t err = cudaFree(c->dev_block);
    if (c->dev_idx16) {
        cudaError_t e2 = cudaFree(c->dev_idx16);
        if (err == cudaSuccess) err = e2;
    }
    delete c;
    if (err != cudaSuccess) return cuda_error(err, "lpdec_code_destroy: cudaFree");
    return LPDEC_OK;
}

// ---------------------------------------------------------------------------
// launch plumbing
namespace lpdec {

// Stream-ordered allocations of the library come from one memory pool per
// device that keeps freed memory for the next call (no release threshold):
// a call that synchronizes then does not hand its buffers back to the driver
// and map them again on the next call.  lpdec_release_memory trims the pools.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

cudaError_t lib_alloc(void **ptr, size_t bytes, cudaStream_t stream) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(ptr, bytes, stream);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props;
            std::memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t p = nullptr;
            err = cudaMemPoolCreate(&p, &props);
            if (err != cudaSuccess) return err;
            uint64_t keep = ~0ull;
            err = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
            if (err != cudaSuccess) {
                cudaMemPoolDestroy(p);
                return err;
            }
            g_pool[dev] = p;
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(ptr, bytes, pool, stream);
}

static cudaError_t class_prepare(const lpdec_code *c, int dtype, bool stage, bool ring, size_t smem) {
    switch (kClassD[c->cls]) {
        case 6: return prepare_decode_6(dtype, c->reg_dv, stage, ring, smem);
        case 8: return prepare_decode_8(dtype, c->reg_dv, stage, ring, smem);
        case 16: return prepare_decode_16(dtype, c->reg_dv, stage, ring, smem);
        case 20: return prepare_decode_20(dtype, c->reg_dv, stage, ring, smem);
        default: return prepare_decode_32(dtype, c->reg_dv, stage, ring, smem);
    }
}
static cudaError_t class_occupancy(const lpdec_code *c, int dtype, bool stage, bool ring, int block, size_t smem,
                                   int *bps) {
    switch (kClassD[c->cls]) {
        case 6: return occupancy_decode_6(dtype, c->reg_dv, stage, ring, block, smem, bps);
        case 8: return occupancy_decode_8(dtype, c->reg_dv, stage, ring, block, smem, bps);
        case 16: return occupancy_decode_16(dtype, c->reg_dv, stage, ring, block, smem, bps);
        case 20: return occupancy_decode_20(dtype, c->reg_dv, stage, ring, block, smem, bps);
        default: return occupancy_decode_32(dtype, c->reg_dv, stage, ring, block, smem, bps);
    }
}
static cudaError_t class_launch(const lpdec_code *c, int dtype, const DecodeArgs &a, const LaunchCfg &lc) {
    switch (kClassD[c->cls]) {
        case 6: return launch_decode_6(dtype, c->reg_dv, a, lc);
        case 8: return launch_decode_8(dtype, c->reg_dv, a, lc);
        case 16: return launch_decode_16(dtype, c->reg_dv, a, lc);
        case 20: return launch_decode_20(dtype, c->reg_dv, a, lc);
        default: return launch_decode_32(dtype, c->reg_dv, a, lc);
    }
}

static size_t dtype_size(int dtype) { return dtype == LPDEC_STATE_F32 ? 4 : 2; }

// Byte layout of one group's shared-memory slice (must match decode_kernel):
// w and lambda/mu, x, the reduction scratch, and 8 ints of flags (the last two
// hold the mbarrier of the bulk loads).
SliceLayout slice_layout(const lpdec_code *c, int dtype, int group_threads) {
    SliceLayout L;
    size_t off = (2 * (size_t)c->Ep * dtype_size(dtype) + 15) & ~(size_t)15;
    L.off_x = off;
    off += ((size_t)c->n * 4 + 15) & ~(size_t)15;
    L.off_red = off;
    off += (size_t)(group_threads / 32) * 2 * 4 + 8 * 4;
    L.bytes = (off + 127) & ~(size_t)127;
    return L;
}

int device_smem_optin(int device) {
    static std::mutex mu;
    static int cached[64] = {0};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64) return 0;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) v = 48 * 1024;
        cached[device] = v;
    }
    return cached[device];
}

int device_sm_count(int device) {
    static std::mutex mu;
    static int cached[64] = {0};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64) return 1;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) v = 1;
        cached[device] = v;
    }
    return cached[device];
}

// Default tile: groups of at most 256 threads (each thread owns one check per
// pass), as many groups per CTA as threads, named barriers and shared memory
// allow.  Several frames per SM keep warps busy across the group barriers.
Tile default_tile(const lpdec_code *c, int dtype, int max_threads) {
    Tile t;
    const int maxT = max_threads > 0 ? std::min(max_threads, class_max_threads(c->cls)) : class_max_threads(c->cls);
    const int lanes = class_lanes(kClassD[c->cls]);
    const long long slots = (long long)c->m * lanes;  // thread slots one pass over the checks needs
    // One thread per check: several small groups per CTA (more frames in
    // flight across the group barriers).  Segmented checks: one wide group,
    // which measured fastest for the wide-check codes.
    const int cap = lanes == 1 ? std::min(256, maxT) : maxT;
    const int passes = (int)((slots + cap - 1) / cap);
    int gt = (int)(((slots + passes - 1) / passes + 31) / 32 * 32);
    gt = std::max(32, std::min(gt, cap));
    const SliceLayout L = slice_layout(c, dtype, gt);
    const int smem_cap = device_smem_optin(c->device);
    int g = std::min(15, maxT / gt);
    g = std::max(1, std::min<int>(g, (int)(smem_cap / std::max<size_t>(L.bytes, 1))));
    t.group_threads = gt;
    t.groups = g;
    return t;
}

Tile chosen_tile(const lpdec_code *c, const lpdec_params *p) {
    const int dt = p->state_dtype;
    if (p->schedule == LPDEC_SCHED_STREAMED && c->tuned_streamed[dt].valid) return c->tuned_streamed[dt];
    if (c->tuned[dt].valid) return c->tuned[dt];
    return default_tile(c, dt);
}

// Ring kernel layout (must match decode_kernel_ring): [16-bit index block,
// when staged] [R slots: w, lambda/mu, and the frame's LLR row when the slots
// hold it] [G scratch areas: x, the reduction scratch and 8 ints of flags]
// [R slot records of 32 bytes, then two ints: the consumers' sequence counter
// and the stop flag].
struct RingLayout {
    size_t slot_bytes = 0, llr_off = 0, off_slots = 0, off_scratch = 0, off_meta = 0, total = 0;
    SliceLayout scratch;  // off_x = 0
};
static RingLayout ring_layout(const lpdec_code *c, int dtype, const Tile &tile, size_t base, bool llr) {
    RingLayout R;
    const size_t state = 2 * (size_t)c->Ep * dtype_size(dtype);  // a multiple of 32
    R.llr_off = llr ? state : 0;
    R.slot_bytes = (state + (llr ? (size_t)c->n * 4 : 0) + 127) & ~(size_t)127;
    R.scratch.off_x = 0;
    R.scratch.off_red = ((size_t)c->n * 4 + 15) & ~(size_t)15;
    R.scratch.bytes = (R.scratch.off_red + (size_t)(tile.group_threads / 32) * 2 * 4 + 8 * 4 + 127) & ~(size_t)127;
    R.off_slots = base;
    R.off_scratch = R.off_slots + (size_t)tile.ring * R.slot_bytes;
    R.off_meta = R.off_scratch + (size_t)tile.groups * R.scratch.bytes;
    R.total = R.off_meta + (size_t)tile.ring * 32 + 16;
    return R;
}

size_t ring_smem_bytes(const lpdec_code *c, int dtype, const Tile &tile) {
    if (tile.ring <= tile.groups || tile.ring > 64) return 0;
    return ring_layout(c, dtype, tile, 0, false).total;
}

static int plan_ring(const lpdec_code *c, int dtype, const Tile &tile, int n_frames, cudaStream_t stream,
                     LaunchCfg *lc, SliceLayout *layout) {
    const int block = tile.groups * tile.group_threads + 32;  // + the producer warp
    if (block > class_max_threads(c->cls) || tile.groups < 1 || tile.groups > 15 || tile.group_threads % 32 ||
        tile.group_threads < 32 || tile.ring <= tile.groups || tile.ring > 64)
        return set_error(LPDEC_EINVAL, "invalid ring tile: %d groups x %d threads, %d slots", tile.groups,
                         tile.group_threads, tile.ring);
    const size_t cap = (size_t)device_smem_optin(c->device);
    // The first layout that fits, in this order: LLR rows in the slots (each
    // launch then reads them with one bulk copy per frame instead of a load
    // per variable; the copy needs 4n to be a multiple of 16) with and
    // without the staged indices, then without the LLR rows.
    const size_t idx_base = ((size_t)c->idx16_bytes + 127) & ~(size_t)127;
    const bool can_stage = c->reg_dv > 0 && c->idx16_bytes > 0, can_llr = c->n % 4 == 0;
    const bool opts[4][2] = {{true, true}, {false, true}, {true, false}, {false, false}};  // {stage, llr}
    RingLayout R;
    bool stage = false;
    for (const auto &o : opts) {
        if ((o[0] && !can_stage) || (o[1] && !can_llr)) continue;
        R = ring_layout(c, dtype, tile, o[0] ? idx_base : 0, o[1]);
        stage = o[0];
        if (R.total <= cap) break;
    }
    if (R.total > cap)
        return set_error(LPDEC_EINVAL, "ring of %d slots of %zu bytes and %d groups does not fit in shared memory (%zu bytes)",
                         tile.ring, R.slot_bytes, tile.groups, cap);
    cudaError_t err = class_prepare(c, dtype, stage, true, R.total);
    if (err != cudaSuccess) return cuda_error(err, "cudaFuncSetAttribute");
    int bps = 0;
    err = class_occupancy(c, dtype, stage, true, block, R.total, &bps);
    if (err != cudaSuccess) return cuda_error(err, "occupancy query");
    if (bps < 1) return set_error(LPDEC_EINVAL, "ring tile does not fit on an SM (%d threads, %zu bytes)", block, R.total);
    const long long need = ((long long)n_frames + tile.groups - 1) / tile.groups;
    const long long persistent = (long long)bps * device_sm_count(c->device);
    lc->grid = (int)std::max<long long>(1, std::min(need, persistent));
    lc->block = block;
    lc->smem = R.total;
    lc->stream = stream;
    lc->slice_base = stage ? (int)idx_base : 0;
    lc->ring_slots = tile.ring;
    lc->ring_slot_bytes = (int)R.slot_bytes;
    lc->ring_off_slots = (int)R.off_slots;
    lc->ring_off_scratch = (int)R.off_scratch;
    lc->ring_off_meta = (int)R.off_meta;
    lc->ring_llr_off = (int)R.llr_off;
    if (layout) *layout = R.scratch;
    return LPDEC_OK;
}

void apply_plan(DecodeArgs &a, const Tile &tile, const LaunchCfg &lc, const SliceLayout &L) {
    a.group_threads = tile.group_threads;
    a.smem_per_group = (int)L.bytes;
    a.off_x = (int)L.off_x;
    a.off_red = (int)L.off_red;
    a.slice_base = lc.slice_base;
    a.ring_slots = lc.ring_slots;
    a.ring_groups = lc.ring_slots > 0 ? tile.groups : 0;
    a.ring_slot_bytes = lc.ring_slot_bytes;
    a.ring_off_slots = lc.ring_off_slots;
    a.ring_off_scratch = lc.ring_off_scratch;
    a.ring_off_meta = lc.ring_off_meta;
    // the LLR rows are copied in bulk: the batch must start on a 16-byte boundary
    a.ring_llr_off = (reinterpret_cast<uintptr_t>(a.llr) & 15) ? 0 : lc.ring_llr_off;
}

int plan_launch(const lpdec_code *c, int dtype, const Tile &tile, int n_frames, cudaStream_t stream,
                LaunchCfg *lc, SliceLayout *layout) {
    *lc = LaunchCfg();
    if (tile.ring > 0) return plan_ring(c, dtype, tile, n_frames, stream, lc, layout);
    const SliceLayout L = slice_layout(c, dtype, tile.group_threads);
    size_t smem = L.bytes * (size_t)tile.groups;
    if ((int)smem > device_smem_optin(c->device) || tile.groups < 1)
        return set_error(LPDEC_EINVAL, "frame state (%zu bytes per group x %d groups) does not fit in shared memory (%d bytes)",
                         L.bytes, tile.groups, device_smem_optin(c->device));
    const int block = tile.groups * tile.group_threads;
    if (block > class_max_threads(c->cls) || tile.groups > 15 || tile.group_threads % 32)
        return set_error(LPDEC_EINVAL, "invalid tile: %d groups x %d threads", tile.groups, tile.group_threads);
    // Regular form: stage the 16-bit index block at the start of shared memory
    // (the slices follow it) when it fits.
    lc->slice_base = 0;
    const size_t idx_aligned = ((size_t)c->idx16_bytes + 127) & ~(size_t)127;
    if (c->reg_dv > 0 && c->idx16_bytes > 0 && smem + idx_aligned <= (size_t)device_smem_optin(c->device)) {
        lc->slice_base = (int)idx_aligned;
        smem += idx_aligned;
    }
    const bool stage = lc->slice_base > 0;
    cudaError_t err = class_prepare(c, dtype, stage, false, smem);
    if (err != cudaSuccess) return cuda_error(err, "cudaFuncSetAttribute");
    int bps = 0;
    err = class_occupancy(c, dtype, stage, false, block, smem, &bps);
    if (err != cudaSuccess) return cuda_error(err, "occupancy query");
    if (bps < 1) return set_error(LPDEC_EINVAL, "tile does not fit on an SM (%d threads, %zu bytes)", block, smem);
    const long long need = ((long long)n_frames + tile.groups - 1) / tile.groups;
    const long long persistent = (long long)bps * device_sm_count(c->device);
    lc->grid = (int)std::max<long long>(1, std::min(need, persistent));
    lc->block = block;
    lc->smem = smem;
    lc->stream = stream;
    if (layout) *layout = L;
    return LPDEC_OK;
}

int validate_params(const lpdec_params *p) {
    if (!p) return set_error(LPDEC_EINVAL, "params is NULL");
    if (!(p->mu > 0.0) || !std::isfinite(p->mu)) return set_error(LPDEC_EINVAL, "mu=%g must be > 0", p->mu);
    if (!(p->rho >= 1.0 && p->rho < 2.0)) return set_error(LPDEC_EINVAL, "rho=%g must be in [1, 2)", p->rho);
    if (!(p->eps >= 0.0) || !std::isfinite(p->eps)) return set_error(LPDEC_EINVAL, "eps=%g must be >= 0", p->eps);
    if (p->max_iter < 1) return set_error(LPDEC_EINVAL, "max_iter=%d must be >= 1", p->max_iter);
    if (p->state_dtype < 0 || p->state_dtype > 3) return set_error(LPDEC_EINVAL, "unknown state_dtype %d", p->state_dtype);
    if (!(p->cert_tol > 0.0 && p->cert_tol < 0.5)) return set_error(LPDEC_EINVAL, "cert_tol=%g must be in (0, 0.5)", p->cert_tol);
    if (p->schedule < 0 || p->schedule > 2) return set_error(LPDEC_EINVAL, "unknown schedule %d", p->schedule);
    if (p->iters_per_launch < 1) return set_error(LPDEC_EINVAL, "iters_per_launch=%d must be >= 1", p->iters_per_launch);
    for (int i = 0; i < 6; ++i)
        if (p->reserved[i]) return set_error(LPDEC_EINVAL, "reserved fields must be zero");
    return LPDEC_OK;
}

// Limit of the first wait on a copy or a ring slot in STREAMED launches
// (lpdec_set_wait_limit); the device-side default is kWaitClocks.
static std::atomic<long long> g_wait_clocks{kWaitClocks};

IterCfg make_cfg(const lpdec_code *c, const lpdec_params *p) {
    IterCfg cfg;
    cfg.wait_clocks = g_wait_clocks.load();
    cfg.mu_inv = (float)(1.0 / p->mu);
    cfg.rho = (float)p->rho;
    cfg.rho_inv = (float)(1.0 / p->rho);
    cfg.omr = (float)(1.0 - p->rho);
    cfg.tmr = (float)(2.0 - p->rho);
    cfg.cert_tol = (float)p->cert_tol;
    cfg.eps2E = p->eps * p->eps * (double)c->E;
    const double epsc = std::max(p->eps, 1e-5);
    cfg.epsc2E = epsc * epsc * (double)c->E;
    cfg.max_iter = p->max_iter;
    cfg.check_stop = p->eps > 0.0 ? 1 : 0;
    // Q16 state: the smallest power of two s with 32767 s >= 1 + 6/mu, a bound on
    // |w| = |z - lambda/mu| and |lambda/mu| (|lambda| stayed below 5.5 in FP64
    // runs of the benchmark codes from 0 to 9 dB); mu = 3 gives s = 2^-13.
    const double bound = 1.0 + 6.0 / p->mu;
    const int e = (int)std::ceil(std::log2(bound / 32767.0));
    cfg.q.s = (float)std::ldexp(1.0, e);
    cfg.q.inv = (float)std::ldexp(1.0, -e);
    cfg.q.off = -12615680.0f * cfg.q.s;
    return cfg;
}

CodeView make_view(const lpdec_code *c) {
    CodeView v;
    v.n = c->n;
    v.m = c->m;
    v.E = c->E;
    v.Ep = c->Ep;
    v.row_ptr = c->row_ptr;
    v.check_order = c->check_order;
    v.col_idx = c->col_idx;
    v.col_ptr = c->col_ptr;
    v.csc_edge = c->csc_edge;
    v.col16 = static_cast<const uint16_t *>(c->dev_idx16);
    v.csc16 = c->dev_idx16 ? v.col16 + c->col16_elems : nullptr;
    v.idx16_bytes = c->idx16_bytes;
    v.col16_elems = c->col16_elems;
    v.reg_dc = c->reg_dc;
    return v;
}

// After the last STREAMED launch every frame has k_state = -1; a frame that a
// stopped group or producer left behind is marked abandoned, so that its stale
// outputs are never taken for results.
__global__ void mark_unfinished(int n, const int32_t *__restrict__ k_state, int32_t *iters_out, uint8_t *cert_out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n && k_state[f] >= 0) {
        if (iters_out) iters_out[f] = kFrameTimeout;
        if (cert_out) cert_out[f] = 0;
    }
}

// Enqueue the decode of n_frames frames.  `work` must hold workspace_bytes().
size_t workspace_bytes(const lpdec_code *c, int n_frames, int schedule, int dtype, int max_iter, int ipl) {
    size_t b = 256;  // queue counters for the launches, padded
    const int launches = schedule == LPDEC_SCHED_STREAMED ? (max_iter + ipl - 1) / ipl : 1;
    b += (size_t)launches * 4;
    b = (b + 255) & ~(size_t)255;
    if (schedule == LPDEC_SCHED_STREAMED) {
        b += 2 * (size_t)n_frames * c->Ep * dtype_size(dtype);
        b += ((size_t)n_frames * 4 + 255) & ~(size_t)255;
    }
    return b;
}

int resolve_schedule(const lpdec_code *c, const lpdec_params *p, const Tile &tile) {
    if (p->schedule != LPDEC_SCHED_AUTO) return p->schedule;
    const SliceLayout L = slice_layout(c, p->state_dtype, tile.group_threads);
    return (int)L.bytes <= device_smem_optin(c->device) ? LPDEC_SCHED_RESIDENT : LPDEC_SCHED_STREAMED;
}

int enqueue_decode(const lpdec_code *c, int n_frames, const float *llr, const lpdec_params *p, float *x_out,
                   uint8_t *bits_out, int32_t *iters_out, uint8_t *cert_out, cudaStream_t stream, void *work,
                   int schedule, const Tile &tile_in, int *launches_out) {
    Tile tile = tile_in;
    if (schedule != LPDEC_SCHED_STREAMED) tile.ring = 0;  // the ring streams parked state
    LaunchCfg lc;
    SliceLayout L;
    int rc = plan_launch(c, p->state_dtype, tile, n_frames, stream, &lc, &L);
    if (rc) return rc;
    DecodeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.code = make_view(c);
    a.cfg = make_cfg(c, p);
    a.n_frames = n_frames;
    a.llr = llr;
    a.x_out = x_out;
    a.bits_out = bits_out;
    a.iters_out = iters_out;
    a.cert_out = cert_out;
    apply_plan(a, tile, lc, L);
    const int ipl = schedule == LPDEC_SCHED_STREAMED ? p->iters_per_launch : p->max_iter;
    const int launches = schedule == LPDEC_SCHED_STREAMED ? (p->max_iter + ipl - 1) / ipl : 1;
    char *w = static_cast<char *>(work);
    int *queues = reinterpret_cast<int *>(w + 256);
    size_t off = (256 + (size_t)launches * 4 + 255) & ~(size_t)255;
    if (schedule == LPDEC_SCHED_STREAMED) {
        const size_t sb = (size_t)n_frames * c->Ep * dtype_size(p->state_dtype);
        a.w_state = w + off;
        a.l_state = w + off + sb;
        a.k_state = reinterpret_cast<int32_t *>(w + off + 2 * sb);
        cudaError_t err = cudaMemsetAsync(a.k_state, 0, (size_t)n_frames * 4, stream);
        if (err != cudaSuccess) return cuda_error(err, "cudaMemsetAsync");
    }
    cudaError_t err = cudaMemsetAsync(queues, 0, (size_t)launches * 4, stream);
    if (err != cudaSuccess) return cuda_error(err, "cudaMemsetAsync");
    a.iters_this_launch = ipl;
    for (int L_ = 0; L_ < launches; ++L_) {
        a.queue = queues + L_;
        err = class_launch(c, p->state_dtype, a, lc);
        if (err != cudaSuccess) return cuda_error(err, "decode kernel launch");
    }
    if (schedule == LPDEC_SCHED_STREAMED && n_frames > 0) {
        mark_unfinished<<<(n_frames + 255) / 256, 256, 0, stream>>>(n_frames, a.k_state, iters_out, cert_out);
        err = cudaGetLastError();
        if (err != cudaSuccess) return cuda_error(err, "mark_unfinished launch");
    }
    if (launches_out) *launches_out = launches;
    return LPDEC_OK;
}

// Plan and launch the decode kernel once with caller-filled arguments (frame
// buffers, state, queue, frame list); fills the tile fields of `a`.
int launch_once(const lpdec_code *c, int dtype, const Tile &tile_in, DecodeArgs &a, cudaStream_t stream) {
    Tile tile = tile_in;
    if (!a.k_state) tile.ring = 0;  // the ring streams parked state
    LaunchCfg lc;
    SliceLayout L;
    int rc = plan_launch(c, dtype, tile, a.n_frames, stream, &lc, &L);
    if (rc) return rc;
    apply_plan(a, tile, lc, L);
    cudaError_t err = class_launch(c, dtype, a, lc);
    if (err != cudaSuccess) return cuda_error(err, "decode kernel launch");
    return LPDEC_OK;
}

}  // namespace lpdec

// ---------------------------------------------------------------------------
// decode entry points

extern "C" int lpdec_decode(const lpdec_code *c, int32_t n_frames, const float *llr, const lpdec_params *p,
                            float *x_out, uint8_t *bits_out, int32_t *iters_out, uint8_t *cert_out,
                            void *cuda_stream) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_decode: code is NULL");
    if (n_frames < 0) return set_error(LPDEC_EINVAL, "lpdec_decode: n_frames=%d < 0", n_frames);
    int rc = lpdec::validate_params(p);
    if (rc) return rc;
    if (n_frames == 0) return LPDEC_OK;
    if (!llr || !x_out) return set_error(LPDEC_EINVAL, "lpdec_decode: llr and x_out must not be NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const lpdec::Tile tile = lpdec::chosen_tile(c, p);
    const int schedule = lpdec::resolve_schedule(c, p, tile);
    const size_t wb = lpdec::workspace_bytes(c, n_frames, schedule, p->state_dtype, p->max_iter, p->iters_per_launch);
    void *work = nullptr;
    cudaError_t err = lpdec::lib_alloc(&work, wb, stream);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode: allocation of the workspace");
    rc = lpdec::enqueue_decode(c, n_frames, llr, p, x_out, bits_out, iters_out, cert_out, stream, work, schedule,
                               tile, nullptr);
    err = cudaFreeAsync(work, stream);
    if (rc) return rc;
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode: cudaFreeAsync");
    return LPDEC_OK;
}

namespace {
// Frames the decode kernel holds in flight at once for this batch (CTAs x
// groups), or 0 if the launch cannot be planned.
int frames_in_flight(const lpdec_code *c, const lpdec_params *p, int n_frames, cudaStream_t stream) {
    lpdec::Tile tile = lpdec::chosen_tile(c, p);
    const int schedule = lpdec::resolve_schedule(c, p, tile);
    if (schedule != LPDEC_SCHED_STREAMED) tile.ring = 0;
    lpdec::LaunchCfg lc;
    lpdec::SliceLayout L;
    if (lpdec::plan_launch(c, p->state_dtype, tile, n_frames, stream, &lc, &L)) return 0;
    return lc.grid * tile.groups;
}
}  // namespace

extern "C" int lpdec_decode_host(const lpdec_code *c, int32_t n_frames, const float *llr, const lpdec_params *p,
                                 float *x_out, uint8_t *bits_out, int32_t *iters_out, uint8_t *cert_out,
                                 void *cuda_stream) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_decode_host: code is NULL");
    if (n_frames < 0) return set_error(LPDEC_EINVAL, "lpdec_decode_host: n_frames=%d < 0", n_frames);
    int rc = lpdec::validate_params(p);
    if (rc) return rc;
    if (n_frames == 0) return LPDEC_OK;
    if (!llr || !x_out) return set_error(LPDEC_EINVAL, "lpdec_decode_host: llr and x_out must not be NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)c->n;
    const size_t nx = (size_t)n_frames * n;
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t bytes = align(nx * 4) * 2 + align(nx) + align((size_t)n_frames * 4) + align((size_t)n_frames);
    char *buf = nullptr;
    cudaError_t err = lpdec::lib_alloc(reinterpret_cast<void **>(&buf), bytes, stream);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode_host: allocation of device buffers");
    float *d_llr = reinterpret_cast<float *>(buf);
    float *d_x = reinterpret_cast<float *>(buf + align(nx * 4));
    uint8_t *d_bits = reinterpret_cast<uint8_t *>(buf + align(nx * 4) * 2);
    int32_t *d_iters = reinterpret_cast<int32_t *>(buf + align(nx * 4) * 2 + align(nx));
    uint8_t *d_cert = reinterpret_cast<uint8_t *>(buf + align(nx * 4) * 2 + align(nx) + align((size_t)n_frames * 4));

    // Pipelining: a large batch is cut into chunks of whole waves (the frames the
    // kernel holds in flight), decoded alternately on the caller's stream and a
    // second stream, so that each chunk's LLR copy overlaps the previous chunk's
    // decode and its output copy the next one's.  The first and last chunks are
    // one wave each, so that little is copied before the first decode or after
    // the last.  Each frame's arithmetic does not depend on the batch, so the
    // results are those of one decode.
    const int wave = frames_in_flight(c, p, n_frames, stream);
    std::vector<int> cut{0};  // chunk k holds frames [cut[k], cut[k+1])
    if (wave > 0 && n_frames >= 8 * wave) {
        const int waves = (n_frames + wave - 1) / wave;
        const int mid = waves - 2, k = std::min(6, std::max(1, mid / 4));
        const int per = (mid + k - 1) / k;
        cut.push_back(wave);
        for (int w = 1 + per; w < waves - 1; w += per) cut.push_back(w * wave);
        cut.push_back((waves - 1) * wave);
    }
    cut.push_back(n_frames);
    int chunks = (int)cut.size() - 1;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (chunks > 1) {
        err = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventRecord(fork, stream);  // after the allocation
        if (err == cudaSuccess) err = cudaStreamWaitEvent(side, fork, 0);
        if (err != cudaSuccess) {
            rc = cuda_error(err, "lpdec_decode_host: second stream");
            chunks = 0;
        }
    }
    for (int k = 0; k < chunks && !rc; ++k) {
        const int f0 = cut[k], nf = cut[k + 1] - cut[k];
        cudaStream_t s = (k & 1) ? side : stream;
        const size_t o = (size_t)f0 * n, cnt = (size_t)nf * n;
        err = cudaMemcpyAsync(d_llr + o, llr + o, cnt * 4, cudaMemcpyHostToDevice, s);
        if (err != cudaSuccess) { rc = cuda_error(err, "lpdec_decode_host: copy of llr"); break; }
        rc = lpdec_decode(c, nf, d_llr + o, p, d_x + o, bits_out ? d_bits + o : nullptr,
                          iters_out ? d_iters + f0 : nullptr, cert_out ? d_cert + f0 : nullptr, s);
        if (rc) break;
        err = cudaMemcpyAsync(x_out + o, d_x + o, cnt * 4, cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess && bits_out) err = cudaMemcpyAsync(bits_out + o, d_bits + o, cnt, cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess && iters_out)
            err = cudaMemcpyAsync(iters_out + f0, d_iters + f0, (size_t)nf * 4, cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess && cert_out)
            err = cudaMemcpyAsync(cert_out + f0, d_cert + f0, (size_t)nf, cudaMemcpyDeviceToHost, s);
        if (err != cudaSuccess) rc = cuda_error(err, "lpdec_decode_host: copy of outputs");
    }
    if (side) {  // join the second stream back before the buffer is freed
        cudaError_t ej = cudaEventRecord(join, side);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(stream, join, 0);
        if (ej != cudaSuccess) cudaStreamSynchronize(side);
        if (!rc && ej != cudaSuccess) rc = cuda_error(ej, "lpdec_decode_host: join");
    }
    cudaError_t e2 = cudaFreeAsync(buf, stream);
    cudaError_t e3 = cudaStreamSynchronize(stream);
    if (side) cudaStreamDestroy(side);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (rc) return rc;
    if (e2 != cudaSuccess) return cuda_error(e2, "lpdec_decode_host: cudaFreeAsync");
    if (e3 != cudaSuccess) return cuda_error(e3, "lpdec_decode_host: cudaStreamSynchronize");
    return LPDEC_OK;
}

// ---------------------------------------------------------------------------
// autotuner: time candidate tiles on the caller's sample and keep the fastest

extern "C" int lpdec_autotune(lpdec_code *c, const lpdec_params *p, int32_t n_frames, const float *llr,
                              void *cuda_stream, int32_t *group_threads_out, int32_t *groups_out,
                              double *ms_per_frame_out) {
    if (!c || !llr) return set_error(LPDEC_EINVAL, "lpdec_autotune: code and llr must not be NULL");
    if (n_frames < 1) return set_error(LPDEC_EINVAL, "lpdec_autotune: n_frames must be >= 1");
    int rc = lpdec::validate_params(p);
    if (rc) return rc;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    lpdec_params q = *p;
    const bool streamed = p->schedule == LPDEC_SCHED_STREAMED;
    if (!streamed) q.schedule = LPDEC_SCHED_RESIDENT;
    const int lanes = lpdec::class_lanes(lpdec::kClassD[c->cls]);
    const int maxT = lpdec::class_max_threads(c->cls);
    const int cap = lpdec::device_smem_optin(c->device);
    std::vector<lpdec::Tile> cand;
    for (int passes = 1; passes <= 32; ++passes) {
        const long long slots = (long long)c->m * lanes;
        int gt = (int)(((slots + passes - 1) / passes + 31) / 32 * 32);
        if (gt > maxT || gt < 32) continue;
        const lpdec::SliceLayout L = lpdec::slice_layout(c, q.state_dtype, gt);
        const int gmax = std::min({15, maxT / gt, (int)(cap / L.bytes)});
        for (int g = 1; g <= gmax; ++g) {
            lpdec::Tile t;
            t.group_threads = gt;
            t.groups = g;
            bool dup = false;
            for (auto &o : cand) dup |= (o.group_threads == gt && o.groups == g);
            if (!dup) cand.push_back(t);
        }
    }
    if (lanes > 1) {
        // Wide checks: also groups as wide as one or two per CTA allow, whose
        // last pass over the checks is ragged (C8000: 1 x 896 runs 1% faster
        // than 1 x 800, the widest even split).
        for (int g = 1; g <= 2; ++g) {
            const int gt = maxT / g / 32 * 32;
            if ((long long)gt > (long long)c->m * lanes + 31) continue;
            const lpdec::SliceLayout L = lpdec::slice_layout(c, q.state_dtype, gt);
            if ((size_t)g * L.bytes > (size_t)cap) continue;
            bool dup = false;
            for (auto &o : cand) dup |= (o.group_threads == gt && o.groups == g);
            if (!dup) {
                lpdec::Tile t;
                t.group_threads = gt;
                t.groups = g;
                cand.push_back(t);
            }
        }
    }
    if (streamed) {
        // Ring tiles: G groups and a producer warp, R = G+1 .. G+4 slots, and
        // the most slots that fit.
        const size_t plain = cand.size();
        for (size_t i = 0; i < plain; ++i) {
            lpdec::Tile t = cand[i];
            if (t.groups * t.group_threads + 32 > maxT) continue;
            int last_fit = 0;
            for (int r = t.groups + 1; r <= 64; ++r) {
                t.ring = r;
                if (lpdec::ring_smem_bytes(c, q.state_dtype, t) > (size_t)cap) break;
                last_fit = r;
                if (r <= t.groups + 4) cand.push_back(t);
            }
            if (last_fit > t.groups + 4) {
                t.ring = last_fit;
                cand.push_back(t);
            }
        }
    }
    if (cand.empty()) return set_error(LPDEC_EINVAL, "lpdec_autotune: no tile fits this code");
    const size_t nx = (size_t)n_frames * c->n;
    char *buf = nullptr;
    const size_t wb = lpdec::workspace_bytes(c, n_frames, q.schedule, q.state_dtype, q.max_iter, q.iters_per_launch);
    cudaError_t err = lpdec::lib_alloc(reinterpret_cast<void **>(&buf), nx * 4 + 256 + wb, stream);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_autotune: allocation of device buffers");
    float *x = reinterpret_cast<float *>(buf);
    void *work = buf + ((nx * 4 + 255) & ~(size_t)255);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaFreeAsync(buf, stream);
        return cuda_error(err, "lpdec_autotune: cudaEventCreate");
    }
    double best = 1e30;
    lpdec::Tile best_t = cand[0];
    rc = LPDEC_OK;
    for (const auto &t : cand) {
        rc = lpdec::enqueue_decode(c, n_frames, llr, &q, x, nullptr, nullptr, nullptr, stream, work,
                                   q.schedule, t, nullptr);  // warm-up
        if (rc) break;
        cudaEventRecord(e0, stream);
        for (int r = 0; r < 2 && !rc; ++r)
            rc = lpdec::enqueue_decode(c, n_frames, llr, &q, x, nullptr, nullptr, nullptr, stream, work,
                                       q.schedule, t, nullptr);
        cudaEventRecord(e1, stream);
        if (rc) break;
        err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) { rc = cuda_error(err, "lpdec_autotune: timing"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / 2.0 / n_frames;
        if (per < best) { best = per; best_t = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, stream);
    cudaStreamSynchronize(stream);
    if (rc) return rc;
    best_t.valid = true;
    (streamed ? c->tuned_streamed : c->tuned)[q.state_dtype] = best_t;
    if (group_threads_out) *group_threads_out = best_t.group_threads;
    if (groups_out) *groups_out = best_t.groups;
    if (ms_per_frame_out) *ms_per_frame_out = best;
    return LPDEC_OK;
}

extern "C" int lpdec_set_tile(lpdec_code *c, int32_t state_dtype, int32_t group_threads, int32_t groups) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_set_tile: code is NULL");
    if (state_dtype < 0 || state_dtype > 3) return set_error(LPDEC_EINVAL, "lpdec_set_tile: unknown state_dtype");
    if (group_threads == 0 && groups == 0) {  // back to the built-in default
        c->tuned[state_dtype] = lpdec::Tile();
        c->tuned_streamed[state_dtype] = lpdec::Tile();
        return LPDEC_OK;
    }
    const int maxT = lpdec::class_max_threads(c->cls);
    if (group_threads < 32 || group_threads % 32 || groups < 1 || groups > 15 || group_threads * groups > maxT)
        return set_error(LPDEC_EINVAL, "lpdec_set_tile: %d groups x %d threads is not a valid tile", groups,
                         group_threads);
    const lpdec::SliceLayout L = lpdec::slice_layout(c, state_dtype, group_threads);
    if ((int)(L.bytes * groups) > lpdec::device_smem_optin(c->device))
        return set_error(LPDEC_EINVAL, "lpdec_set_tile: %d slices of %zu bytes exceed shared memory", groups, L.bytes);
    lpdec::Tile t;
    t.group_threads = group_threads;
    t.groups = groups;
    t.valid = true;
    c->tuned[state_dtype] = t;
    c->tuned_streamed[state_dtype] = t;
    return LPDEC_OK;
}

extern "C" int lpdec_set_streamed_tile(lpdec_code *c, int32_t state_dtype, int32_t group_threads, int32_t groups,
                                       int32_t ring_slots) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_set_streamed_tile: code is NULL");
    if (state_dtype < 0 || state_dtype > 3) return set_error(LPDEC_EINVAL, "lpdec_set_streamed_tile: unknown state_dtype");
    if (group_threads == 0 && groups == 0 && ring_slots == 0) {
        c->tuned_streamed[state_dtype] = lpdec::Tile();
        return LPDEC_OK;
    }
    const int maxT = lpdec::class_max_threads(c->cls);
    const int producer = ring_slots > 0 ? 32 : 0;
    if (group_threads < 32 || group_threads % 32 || groups < 1 || groups > 15 ||
        group_threads * groups + producer > maxT)
        return set_error(LPDEC_EINVAL, "lpdec_set_streamed_tile: %d groups x %d threads is not a valid tile", groups,
                         group_threads);
    lpdec::Tile t;
    t.group_threads = group_threads;
    t.groups = groups;
    t.ring = ring_slots;
    t.valid = true;
    if (ring_slots != 0) {
        if (ring_slots <= groups || ring_slots > 64)
            return set_error(LPDEC_EINVAL, "lpdec_set_streamed_tile: ring_slots=%d must be in (groups, 64]", ring_slots);
        const size_t need = lpdec::ring_smem_bytes(c, state_dtype, t);
        if (need > (size_t)lpdec::device_smem_optin(c->device))
            return set_error(LPDEC_EINVAL, "lpdec_set_streamed_tile: a ring of %d slots needs %zu bytes of shared memory",
                             ring_slots, need);
    } else {
        const lpdec::SliceLayout L = lpdec::slice_layout(c, state_dtype, group_threads);
        if ((int)(L.bytes * groups) > lpdec::device_smem_optin(c->device))
            return set_error(LPDEC_EINVAL, "lpdec_set_streamed_tile: %d slices of %zu bytes exceed shared memory",
                             groups, L.bytes);
    }
    c->tuned_streamed[state_dtype] = t;
    return LPDEC_OK;
}

extern "C" int lpdec_get_tile(const lpdec_code *c, int32_t state_dtype, int32_t schedule, int32_t *group_threads,
                              int32_t *groups, int32_t *ring_slots) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_get_tile: code is NULL");
    if (state_dtype < 0 || state_dtype > 3) return set_error(LPDEC_EINVAL, "lpdec_get_tile: unknown state_dtype");
    if (schedule < 0 || schedule > 2) return set_error(LPDEC_EINVAL, "lpdec_get_tile: unknown schedule");
    lpdec_params p;
    lpdec_params_default(&p);
    p.state_dtype = state_dtype;
    p.schedule = schedule;
    const lpdec::Tile t = lpdec::chosen_tile(c, &p);
    if (group_threads) *group_threads = t.group_threads;
    if (groups) *groups = t.groups;
    if (ring_slots) *ring_slots = schedule == LPDEC_SCHED_RESIDENT ? 0 : t.ring;
    return LPDEC_OK;
}

extern "C" int lpdec_release_memory(void) {
    std::lock_guard<std::mutex> lk(lpdec::g_pool_mu);
    for (int d = 0; d < 64; ++d) {
        if (!lpdec::g_pool[d]) continue;
        cudaError_t err = cudaMemPoolTrimTo(lpdec::g_pool[d], 0);
        if (err != cudaSuccess) return cuda_error(err, "lpdec_release_memory: cudaMemPoolTrimTo");
    }
    return LPDEC_OK;
}

extern "C" int lpdec_project(int32_t d, int64_t count, const float *v, float *z, void *cuda_stream) {
    if (d < 1 || d > 32) return set_error(LPDEC_EINVAL, "lpdec_project: d=%d must be in [1, 32]", d);
    if (count < 0) return set_error(LPDEC_EINVAL, "lpdec_project: count < 0");
    if (count == 0) return LPDEC_OK;
    if (!v || !z) return set_error(LPDEC_EINVAL, "lpdec_project: NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t err;
    switch (lpdec::kClassD[lpdec::degree_class(d)]) {
        case 6: err = lpdec::launch_project_6(d, count, v, z, s); break;
        case 8: err = lpdec::launch_project_8(d, count, v, z, s); break;
        case 16: err = lpdec::launch_project_16(d, count, v, z, s); break;
        case 20: err = lpdec::launch_project_20(d, count, v, z, s); break;
        default: err = lpdec::launch_project_32(d, count, v, z, s); break;
    }
    if (err != cudaSuccess) return cuda_error(err, "lpdec_project launch");
    return LPDEC_OK;
}

extern "C" int lpdec_set_wait_limit(int64_t clocks) {
    lpdec::g_wait_clocks.store(clocks > 0 ? (long long)clocks : lpdec::kWaitClocks);
    return LPDEC_OK;
}

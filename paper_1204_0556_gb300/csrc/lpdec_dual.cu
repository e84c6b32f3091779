// Dual subgradient ascent decoder (the paper's appendix): the un-augmented
// Lagrangian L_0 = gamma^T x + sum_j lambda_j^T (P_j x - z_j) is minimized
// over x in [0,1]^n (a Heaviside step per variable) and over z_j in PP_d
// (Algorithm 3, a sign pattern plus a parity repair per check), both from
// lambda^k, and lambda_j += mu (P_j x - z_j).
//
// Integer form.  Every subgradient entry x_i - z_e is -1, 0 or +1, so from
// lambda^0 = 0 every lambda_e is mu times an integer k_e with |k_e| <= k.  The
// kernel keeps k_e (int16; max_iter <= 32767).  Algorithm 3 depends on lambda
// only through signs and comparisons, which k reproduces exactly (mu > 0).  The
// Heaviside step x_i = [-gamma_i - mu S_i > 0], S_i = sum of k over the edges
// of i, is x_i = [S_i < c_i] with c_i = ceil(-gamma_i / mu) computed once per
// frame in FP64 and corrected with two exactly-signed fused multiply-adds, so
// every decision of the iteration is the exact real-number decision.
//
// Layout: a persistent CTA of G groups x T threads; each group decodes one
// frame at a time in its shared-memory slice (k[Ep] int16, c[n] int32, x[n]
// u8, flags), pulling frame ids from a global counter.  When the code's index
// arrays fit 16 bits they are staged once per CTA in shared memory as u16.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdint>

#include "lpdec.h"
#include "lpdec_api_internal.h"
#include "lpdec_device.cuh"

namespace lpdec {
namespace {

constexpr int kDualMaxThreads = 1024;
constexpr int kDualMaxIter = 32767;  // |k_e| <= iterations must fit int16
constexpr double kThrClamp = 4194304.0;  // 2^22 > max |S_i| = 32 * 32767

struct DualArgs {
    int n, m, E, Ep;
    const int *row_ptr, *col_idx, *col_ptr, *csc_edge;  // device copies of the code
    int n_frames;
    const float *llr;  // [F x n]
    double mu;
    int max_iter;
    float *x_out;        // [F x n]
    uint8_t *bits_out;   // [F x n] or null
    int32_t *iters_out;  // [F] or null
    uint8_t *cert_out;   // [F] or null
    int *queue;          // frame counter, zero at launch
    int group_threads;
    int slice_bytes;
    int off_thr, off_x, off_flags;        // within a slice
    int idx_bytes;                        // CTA-wide u16 index copy (0: indices read from global)
    int o_col, o_csc, o_rowp, o_colp;     // offsets of the u16 arrays in the copy
};

// Index access: u16 copies in shared memory, or the int32 arrays in global memory.
template <bool IDX16>
struct Idx {
    const void *col, *csc, *rowp, *colp;
    __device__ __forceinline__ int get(const void *p, int i) const {
        if constexpr (IDX16) return reinterpret_cast<const uint16_t *>(p)[i];
        else return __ldg(reinterpret_cast<const int *>(p) + i);
    }
    __device__ __forceinline__ int col_of(int e) const { return get(col, e); }
    __device__ __forceinline__ int csc_of(int s) const { return get(csc, s); }
    __device__ __forceinline__ int row_start(int j) const { return get(rowp, j); }
    __device__ __forceinline__ int col_start(int i) const { return get(colp, i); }
};

// Algorithm 3 on the integer costs k[0..d): the edge (index into the row)
// whose z differs from [k > 0], or -1 when the positive set is already even.
// Odd positive set: add the largest non-positive entry when k_ip + k_in > 0,
// else drop the smallest positive entry; ties pick the lowest index.
struct LpMax {
    int r = 0, kp = INT_MAX, ip = -1, kn = INT_MIN, in = -1;
    __device__ __forceinline__ void see(int v, int q) {
        if (v > 0) {
            ++r;
            if (v < kp) { kp = v; ip = q; }
        } else if (v > kn) {
            kn = v;
            in = q;
        }
    }
    __device__ __forceinline__ int flip() const {
        if (!(r & 1)) return -1;
        return (in >= 0 && kp + kn > 0) ? in : ip;
    }
};

// c_i = min { S integer : mu S + gamma_i >= 0 }, so that x_i = [S_i < c_i].
__device__ __forceinline__ int heaviside_threshold(float g, double mu) {
    double q = -(double)g / mu;
    if (q >= kThrClamp) return (int)kThrClamp;
    if (q <= -kThrClamp) return -(int)kThrClamp;
    double c = ceil(q);
    // The quotient is within one unit of the exact ceiling; fma rounds once, so
    // the sign of mu*c + gamma is exact.
    if (fma(mu, c, (double)g) < 0.0) c += 1.0;
    else if (fma(mu, c - 1.0, (double)g) >= 0.0) c -= 1.0;
    return (int)c;
}

// D > 0: every check has degree D and check j owns edges j*D..j*D+D-1; DV > 0:
// every variable has degree DV and its CSC slots are i*DV..i*DV+DV-1.
template <int D, int DV, bool IDX16>
__global__ void __launch_bounds__(kDualMaxThreads, 1) dual_kernel(const DualArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Idx<IDX16> ix;
    if constexpr (IDX16) {
        uint16_t *col = reinterpret_cast<uint16_t *>(smem_raw + a.o_col);
        uint16_t *csc = reinterpret_cast<uint16_t *>(smem_raw + a.o_csc);
        uint16_t *rowp = reinterpret_cast<uint16_t *>(smem_raw + a.o_rowp);
        uint16_t *colp = reinterpret_cast<uint16_t *>(smem_raw + a.o_colp);
        for (int e = threadIdx.x; e < a.E; e += blockDim.x) {
            col[e] = (uint16_t)__ldg(a.col_idx + e);
            csc[e] = (uint16_t)__ldg(a.csc_edge + e);
        }
        for (int j = threadIdx.x; j <= a.m; j += blockDim.x) rowp[j] = (uint16_t)__ldg(a.row_ptr + j);
        for (int i = threadIdx.x; i <= a.n; i += blockDim.x) colp[i] = (uint16_t)__ldg(a.col_ptr + i);
        ix.col = col; ix.csc = csc; ix.rowp = rowp; ix.colp = colp;
        __syncthreads();
    } else {
        ix.col = a.col_idx; ix.csc = a.csc_edge; ix.rowp = a.row_ptr; ix.colp = a.col_ptr;
    }

    const int T = a.group_threads;
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    const int lane = t & 31;
    const int bar = 1 + g;
    unsigned char *base = smem_raw + a.idx_bytes + (size_t)g * a.slice_bytes;
    int16_t *kst = reinterpret_cast<int16_t *>(base);
    int *thr = reinterpret_cast<int *>(base + a.off_thr);
    uint8_t *xs = base + a.off_x;
    volatile int *flags = reinterpret_cast<int *>(base + a.off_flags);
    // flags[0], flags[1]: "some subgradient entry is nonzero" of even / odd
    // iterations; flags[2], flags[3]: double-buffered frame id; flags[4]: bad LLR.

    int par = 0;
    for (;;) {
        if (t == 0) flags[2 + par] = atomicAdd(a.queue, 1);
        group_sync(bar, T);
        const int f = flags[2 + par];
        par ^= 1;
        if (f >= a.n_frames) break;
        if (t == 0) { flags[0] = 0; flags[1] = 0; flags[4] = 0; }

        // ---- lambda^0 = 0 and the per-variable Heaviside thresholds
        const float *gam = a.llr + (size_t)f * a.n;
        int bad = 0;
        for (int i = t; i < a.n; i += T) {
            const float gi = __ldg(gam + i);
            bad |= !isfinite(gi);
            thr[i] = heaviside_threshold(gi, a.mu);
        }
        zero16(kst, a.Ep * 2, t, T);
        bad = __any_sync(0xffffffffu, bad);
        group_sync(bar, T);
        if (bad && lane == 0) flags[4] = 1;
        group_sync(bar, T);
        float *xo = a.x_out + (size_t)f * a.n;
        uint8_t *bo = a.bits_out ? a.bits_out + (size_t)f * a.n : nullptr;
        if (flags[4]) {
            for (int i = t; i < a.n; i += T) {
                xo[i] = 0.0f;
                if (bo) bo[i] = 0;
            }
            if (t == 0) {
                if (a.iters_out) a.iters_out[f] = LPDEC_FRAME_BAD_LLR;
                if (a.cert_out) a.cert_out[f] = 0;
            }
            continue;
        }

        int k = 0;
        bool done = false;
        while (k < a.max_iter) {
            // ---- x-update: Heaviside step of -gamma - sum_j P_j^T lambda_j
            for (int i = t; i < a.n; i += T) {
                int S = 0;
                if constexpr (DV > 0) {
#pragma unroll
                    for (int s = 0; s < DV; ++s) S += kst[ix.csc_of(i * DV + s)];
                } else {
                    const int s1 = ix.col_start(i + 1);
                    for (int s = ix.col_start(i); s < s1; ++s) S += kst[ix.csc_of(s)];
                }
                xs[i] = S < thr[i] ? 1 : 0;
            }
            group_sync(bar, T);
            if (t == 0) flags[(k + 1) & 1] = 0;  // every reader of it finished before this iteration's barrier
            // ---- z-update (Algorithm 3) and lambda-update, one check per thread
            int mism = 0;
            for (int j = t; j < a.m; j += T) {
                if constexpr (D > 0) {
                    int16_t *kj = kst + j * D;
                    int v[D];
#pragma unroll
                    for (int q = 0; q < D; q += 2) {
                        const uint32_t w = *reinterpret_cast<const uint32_t *>(kj + q);
                        v[q] = (int)(int16_t)(w & 0xffffu);
                        v[q + 1] = (int)(int16_t)(w >> 16);
                    }
                    LpMax lm;
#pragma unroll
                    for (int q = 0; q < D; ++q) lm.see(v[q], q);
                    const int fl = lm.flip();
#pragma unroll
                    for (int q = 0; q < D; ++q) {
                        const int z = (v[q] > 0) ^ (q == fl);
                        const int s = (int)xs[ix.col_of(j * D + q)] - z;
                        mism |= s;
                        v[q] += s;
                    }
#pragma unroll
                    for (int q = 0; q < D; q += 2)
                        *reinterpret_cast<uint32_t *>(kj + q) = (uint32_t)(uint16_t)v[q] | ((uint32_t)(uint16_t)v[q + 1] << 16);
                } else {
                    const int e0 = ix.row_start(j), e1 = ix.row_start(j + 1);
                    LpMax lm;
                    for (int e = e0; e < e1; ++e) lm.see(kst[e], e - e0);
                    const int fl = lm.flip();
                    for (int e = e0; e < e1; ++e) {
                        const int v = kst[e];
                        const int z = (v > 0) ^ (e - e0 == fl);
                        const int s = (int)xs[ix.col_of(e)] - z;
                        mism |= s;
                        kst[e] = (int16_t)(v + s);
                    }
                }
            }
            if (__any_sync(0xffffffffu, mism != 0) && lane == 0) flags[k & 1] = 1;
            group_sync(bar, T);
            done = flags[k & 1] == 0;
            ++k;
            if (done) break;  // zero subgradient: lambda is dual optimal, x an LP optimum
        }

        // ---- outputs (x^k is in shared memory; the last barrier ordered it)
        for (int i = t; i < a.n; i += T) {
            const uint8_t b = xs[i];
            xo[i] = (float)b;
            if (bo) bo[i] = b;
        }
        if (t == 0) {
            if (a.iters_out) a.iters_out[f] = k;
            if (a.cert_out) a.cert_out[f] = done ? 1 : 0;
        }
    }
}

enum DualForm { kForm63 = 0, kForm84, kFormGeneric16, kFormGeneric32, kNumForms };

const void *dual_fn(int form) {
    switch (form) {
        case kForm63: return reinterpret_cast<const void *>(&dual_kernel<6, 3, true>);
        case kForm84: return reinterpret_cast<const void *>(&dual_kernel<8, 4, true>);
        case kFormGeneric16: return reinterpret_cast<const void *>(&dual_kernel<0, 0, true>);
        default: return reinterpret_cast<const void *>(&dual_kernel<0, 0, false>);
    }
}

struct DualLayout {
    int idx_bytes = 0, o_col = 0, o_csc = 0, o_rowp = 0, o_colp = 0;
    int slice_bytes = 0, off_thr = 0, off_x = 0, off_flags = 0;
    int form = kFormGeneric32;
};

size_t pad16(size_t v) { return (v + 15) & ~(size_t)15; }

DualLayout dual_layout(const lpdec_code *c) {
    DualLayout L;
    size_t off = pad16((size_t)c->Ep * 2);
    L.off_thr = (int)off;
    off += pad16((size_t)c->n * 4);
    L.off_x = (int)off;
    off += pad16((size_t)c->n);
    L.off_flags = (int)off;
    off += 8 * 4;
    L.slice_bytes = (int)((off + 127) & ~(size_t)127);
    const bool fits16 = c->E <= 65535 && c->n <= 65535;
    size_t o = 0;
    L.o_col = 0;
    o += pad16((size_t)c->E * 2);
    L.o_csc = (int)o;
    o += pad16((size_t)c->E * 2);
    L.o_rowp = (int)o;
    o += pad16(((size_t)c->m + 1) * 2);
    L.o_colp = (int)o;
    o += pad16(((size_t)c->n + 1) * 2);
    const bool stage = fits16 && (int)(o + L.slice_bytes) <= device_smem_optin(c->device);
    L.idx_bytes = stage ? (int)((o + 127) & ~(size_t)127) : 0;
    const int D = kClassD[c->cls];
    if (!stage) L.form = kFormGeneric32;
    else if (D == 6 && c->reg_dv == 3) L.form = kForm63;
    else if (D == 8 && c->reg_dv == 4) L.form = kForm84;
    else L.form = kFormGeneric16;
    return L;
}

// Default tile: one check per thread per pass with groups of at most 128
// threads (128 x 8 and 96 x 10 measured fastest on C1056; 192 x 5 was 2.5 %
// slower), as many groups (frames) per CTA as threads, barriers and shared
// memory allow.
Tile dual_default_tile(const lpdec_code *c, const DualLayout &L) {
    const int passes = (c->m + 127) / 128;
    int gt = ((c->m + passes - 1) / passes + 31) / 32 * 32;
    gt = std::max(32, std::min(gt, 128));
    const int room = device_smem_optin(c->device) - L.idx_bytes;
    int g = std::min(15, kDualMaxThreads / gt);
    g = std::max(1, std::min(g, room / std::max(L.slice_bytes, 1)));
    Tile t;
    t.group_threads = gt;
    t.groups = g;
    return t;
}

std::atomic<int> g_dual_smem_granted[64][kNumForms];

cudaError_t dual_prepare(int form, size_t smem) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const void *fn = dual_fn(form);
    if (dev < 0 || dev >= 64) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    std::atomic<int> &granted = g_dual_smem_granted[dev][form];
    if ((int)smem <= granted.load()) return cudaSuccess;
    err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess) {
        int cur = granted.load();
        while ((int)smem > cur && !granted.compare_exchange_weak(cur, (int)smem)) {
        }
    }
    return err;
}

cudaError_t dual_launch(int form, int grid, int block, size_t smem, cudaStream_t s, const DualArgs &a) {
    switch (form) {
        case kForm63: dual_kernel<6, 3, true><<<grid, block, smem, s>>>(a); break;
        case kForm84: dual_kernel<8, 4, true><<<grid, block, smem, s>>>(a); break;
        case kFormGeneric16: dual_kernel<0, 0, true><<<grid, block, smem, s>>>(a); break;
        default: dual_kernel<0, 0, false><<<grid, block, smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace lpdec

using lpdec::cuda_error;
using lpdec::set_error;

extern "C" int lpdec_dual_set_tile(lpdec_code *c, int32_t group_threads, int32_t groups) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_dual_set_tile: code is NULL");
    if (group_threads == 0 && groups == 0) {
        c->dual_tile = lpdec::Tile();
        return LPDEC_OK;
    }
    if (group_threads < 32 || group_threads % 32 || groups < 1 || groups > 15 ||
        group_threads * groups > lpdec::kDualMaxThreads)
        return set_error(LPDEC_EINVAL, "lpdec_dual_set_tile: %d groups x %d threads is not a valid tile", groups,
                         group_threads);
    const lpdec::DualLayout L = lpdec::dual_layout(c);
    if (L.idx_bytes + (long long)L.slice_bytes * groups > lpdec::device_smem_optin(c->device))
        return set_error(LPDEC_EINVAL, "lpdec_dual_set_tile: %d slices of %d bytes exceed shared memory", groups,
                         L.slice_bytes);
    c->dual_tile.group_threads = group_threads;
    c->dual_tile.groups = groups;
    c->dual_tile.valid = true;
    return LPDEC_OK;
}

extern "C" int lpdec_decode_dual(const lpdec_code *c, int32_t n_frames, const float *llr, double mu,
                                 int32_t max_iter, float *x_out, uint8_t *bits_out, int32_t *iters_out,
                                 uint8_t *cert_out, void *cuda_stream) {
    if (!c) return set_error(LPDEC_EINVAL, "lpdec_decode_dual: code is NULL");
    if (n_frames < 0) return set_error(LPDEC_EINVAL, "lpdec_decode_dual: n_frames=%d < 0", n_frames);
    if (!(mu > 0.0) || !std::isfinite(mu)) return set_error(LPDEC_EINVAL, "lpdec_decode_dual: mu=%g must be > 0", mu);
    if (max_iter < 1 || max_iter > lpdec::kDualMaxIter)
        return set_error(LPDEC_EINVAL, "lpdec_decode_dual: max_iter=%d must be in [1, %d]", max_iter,
                         lpdec::kDualMaxIter);
    if (n_frames == 0) return LPDEC_OK;
    if (!llr || !x_out) return set_error(LPDEC_EINVAL, "lpdec_decode_dual: llr and x_out must not be NULL");
    const lpdec::DualLayout L = lpdec::dual_layout(c);
    const lpdec::Tile tile = c->dual_tile.valid ? c->dual_tile : lpdec::dual_default_tile(c, L);
    const size_t smem = (size_t)L.idx_bytes + (size_t)L.slice_bytes * tile.groups;
    if ((int)smem > lpdec::device_smem_optin(c->device))
        return set_error(LPDEC_EINVAL, "lpdec_decode_dual: frame state (%d bytes) does not fit in shared memory",
                         L.slice_bytes);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t err = lpdec::dual_prepare(L.form, smem);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode_dual: cudaFuncSetAttribute");
    const int block = tile.groups * tile.group_threads;
    int bps = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, lpdec::dual_fn(L.form), block, smem);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode_dual: occupancy query");
    if (bps < 1) return set_error(LPDEC_EINVAL, "lpdec_decode_dual: tile does not fit on an SM");
    const long long need = ((long long)n_frames + tile.groups - 1) / tile.groups;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)bps * lpdec::device_sm_count(c->device)));

    int *queue = nullptr;
    err = lpdec::lib_alloc(reinterpret_cast<void **>(&queue), sizeof(int), stream);
    if (err != cudaSuccess) return cuda_error(err, "lpdec_decode_dual: allocation of the queue");
    err = cudaMemsetAsync(queue, 0, sizeof(int), stream);
    int rc = LPDEC_OK;
    if (err != cudaSuccess) rc = cuda_error(err, "lpdec_decode_dual: cudaMemsetAsync");
    if (!rc) {
        lpdec::DualArgs a;
        a.n = c->n; a.m = c->m; a.E = c->E; a.Ep = c->Ep;
        a.row_ptr = c->row_ptr; a.col_idx = c->col_idx; a.col_ptr = c->col_ptr; a.csc_edge = c->csc_edge;
        a.n_frames = n_frames;
        a.llr = llr;
        a.mu = mu;
        a.max_iter = max_iter;
        a.x_out = x_out; a.bits_out = bits_out; a.iters_out = iters_out; a.cert_out = cert_out;
        a.queue = queue;
        a.group_threads = tile.group_threads;
        a.slice_bytes = L.slice_bytes;
        a.off_thr = L.off_thr; a.off_x = L.off_x; a.off_flags = L.off_flags;
        a.idx_bytes = L.idx_bytes;
        a.o_col = L.o_col; a.o_csc = L.o_csc; a.o_rowp = L.o_rowp; a.o_colp = L.o_colp;
        err = lpdec::dual_launch(L.form, grid, block, smem, stream, a);
        if (err != cudaSuccess) rc = cuda_error(err, "lpdec_decode_dual: kernel launch");
    }
    err = cudaFreeAsync(queue, stream);
    if (!rc && err != cudaSuccess) rc = cuda_error(err, "lpdec_decode_dual: cudaFreeAsync");
    return rc;
}

// Device code of liblpdec: the check-side projection onto the parity polytope
// and the per-frame ADMM iteration (Algorithm 1, Section 3.3), for sm_103a.
//
// Work decomposition.  A *group* of GT threads (a whole number of warps)
// decodes one frame at a time; a CTA holds G groups, each with its own slice
// of shared memory and its own named barrier.  Inside a group:
//   - variable phase: thread t owns variables t, t+GT, ...; it sums
//     w_e = z_e - lambda_e/mu over the variable's edges (CSC order, gathered
//     through the edge permutation) and writes x_i (Algorithm 1, x-update);
//   - check phase: thread t owns checks t, t+GT, ...; it gathers x over the
//     check's edges, recovers z_old = w + lambda/mu, forms the over-relaxed v,
//     projects it onto PP_d in registers and writes lambda/mu = v - z and
//     w = z - lambda/mu back (Algorithm 1, z- and lambda-updates);
//   - stopping test: FP32 per-thread partials, FP32 warp shuffles, FP64 sum
//     over the group's warps (the only FP64 on the GPU).
// The edge state (w, lambda/mu) is stored as S (float, bf16 or fp16); all
// arithmetic is FP32.  lambda is kept pre-scaled as lambda/mu (the scaled
// dual of Section 3.4), so the lambda-update is lambda' <- v - z.  Keeping w
// rather than z halves the x-update's gathers; it is the same iteration.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace lpdec {

// Lanes per check in the decode kernel of a class: one thread per check for
// D <= 8 (sorted breakpoints), L adjacent lanes for wider checks
// (check_update_w).
#ifndef LPDEC_L16
#define LPDEC_L16 2
#endif
#ifndef LPDEC_L20
#define LPDEC_L20 2
#endif
#ifndef LPDEC_L32
#define LPDEC_L32 2
#endif
__host__ __device__ constexpr int class_lanes(int D) {
    return D <= 8 ? 1 : (D <= 16 ? LPDEC_L16 : (D <= 20 ? LPDEC_L20 : LPDEC_L32));
}

constexpr float kPadV = -1.0e30f;  // value of an unused lane of a check (clips to 0)
constexpr float kBigKappa = 1.0e30f;

// ---------------------------------------------------------------------------
// storage conversions
//
// q16_t: 16-bit fixed point.  A stored value is k * s with k a signed 16-bit
// integer kept biased (b = k + 32768) and s = 2^e a per-decode power of two
// (QScale, chosen on the host from mu).  With b in the low half of a word
// whose high half is 0x4B40, the word is the float 1.5 * 2^23 + b exactly, so
// a load is one byte permute and one FFMA, (f - (1.5 * 2^23 + 32768)) * s,
// exact; a store is one FFMA, v / s + 1.5 * 2^23 + 32768 rounded to the
// nearest integer by the addition, clamped to the 16-bit range (values beyond
// +-32767 s saturate), whose low half is b.
struct q16_t {
    uint16_t b;
};
struct QScale {
    float s;    // 2^e
    float off;  // -(1.5 * 2^23 + 32768) * s
    float inv;  // 1 / s
};
constexpr float kQMagic = 12615680.0f;  // 1.5 * 2^23 + 32768
constexpr float kQLo = 12582912.0f;     // b = 0
constexpr float kQHi = 12648447.0f;     // b = 65535

__device__ __forceinline__ float q16_decode(unsigned word, unsigned sel, const QScale &q) {
    return fmaf(__int_as_float((int)__byte_perm(word, 0x4B400000u, sel)), q.s, q.off);
}
__device__ __forceinline__ unsigned q16_encode(float v, const QScale &q) {
    return (unsigned)__float_as_int(fminf(fmaxf(fmaf(v, q.inv, kQMagic), kQLo), kQHi));
}

template <typename S> __device__ __forceinline__ float ld(S v, const QScale &q);
template <> __device__ __forceinline__ float ld<float>(float v, const QScale &) { return v; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(__nv_bfloat16 v, const QScale &) {
    return __bfloat162float(v);
}
template <> __device__ __forceinline__ float ld<__half>(__half v, const QScale &) { return __half2float(v); }
template <> __device__ __forceinline__ float ld<q16_t>(q16_t v, const QScale &q) { return q16_decode(v.b, 0x7610, q); }

template <typename S> __device__ __forceinline__ S st(float v, const QScale &q);
template <> __device__ __forceinline__ float st<float>(float v, const QScale &) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 st<__nv_bfloat16>(float v, const QScale &) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half st<__half>(float v, const QScale &) { return __float2half_rn(v); }
template <> __device__ __forceinline__ q16_t st<q16_t>(float v, const QScale &q) {
    q16_t r;
    r.b = (uint16_t)(q16_encode(v, q) & 0xffffu);
    return r;
}

// Two adjacent state elements (for even-aligned pairs of edges of a check).
template <typename S> __device__ __forceinline__ float2 ld2(const S *p, const QScale &q);
template <> __device__ __forceinline__ float2 ld2<float>(const float *p, const QScale &) {
    return *reinterpret_cast<const float2 *>(p);
}
template <> __device__ __forceinline__ float2 ld2<__half>(const __half *p, const QScale &) {
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
template <> __device__ __forceinline__ float2 ld2<__nv_bfloat16>(const __nv_bfloat16 *p, const QScale &) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}
template <> __device__ __forceinline__ float2 ld2<q16_t>(const q16_t *p, const QScale &q) {
    const unsigned w = *reinterpret_cast<const unsigned *>(p);
    const float2 f = make_float2(__int_as_float((int)__byte_perm(w, 0x4B400000u, 0x7610)),
                                 __int_as_float((int)__byte_perm(w, 0x4B400000u, 0x7632)));
    return __ffma2_rn(f, make_float2(q.s, q.s), make_float2(q.off, q.off));  // each lane exact, as q16_decode
}
template <typename S> __device__ __forceinline__ void st2(S *p, float a, float b, const QScale &q);
template <> __device__ __forceinline__ void st2<float>(float *p, float a, float b, const QScale &) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
template <> __device__ __forceinline__ void st2<__half>(__half *p, float a, float b, const QScale &) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
}
template <> __device__ __forceinline__ void st2<__nv_bfloat16>(__nv_bfloat16 *p, float a, float b, const QScale &) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}
template <> __device__ __forceinline__ void st2<q16_t>(q16_t *p, float a, float b, const QScale &q) {
    *reinterpret_cast<unsigned *>(p) = __byte_perm(q16_encode(a, q), q16_encode(b, q), 0x5410);
}

// Bit pattern of two stored zeros (the initial z = lambda = 0).
template <typename S> __host__ __device__ constexpr unsigned state_zero2() {
    return std::is_same<S, q16_t>::value ? 0x80008000u : 0u;
}

// ---------------------------------------------------------------------------
// Batcher odd-even merge sort network (ascending) on a register array of N
// values, N padded up to a power of two with +inf lanes whose comparators are
// dropped (a comparator against +inf at the higher index never swaps).
__host__ __device__ constexpr int pow2ceil(int n) { return n <= 1 ? 1 : 2 * pow2ceil((n + 1) / 2); }

template <int N>
__device__ __forceinline__ void sort_asc(float (&a)[N]) {
    constexpr int P2 = pow2ceil(N);
#pragma unroll
    for (int p = 1; p < P2; p <<= 1) {
#pragma unroll
        for (int k = p; k >= 1; k >>= 1) {
#pragma unroll
            for (int j = k % p; j <= P2 - 1 - k; j += 2 * k) {
#pragma unroll
                for (int i = 0; i <= k - 1; ++i) {
                    if ((i + j) / (p * 2) == (i + j + k) / (p * 2)) {
                        const int lo = i + j, hi = i + j + k;
                        if (hi < N) {
                            const float x = a[lo], y = a[hi];
                            a[lo] = fminf(x, y);
                            a[hi] = fmaxf(x, y);
                        }
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// beta_opt of the two-slice projection.
//
// With S the odd set of the violated facet (f_k = +1 on S, -1 off S) and
// kappa_k = v_k - 1 on S, kappa_k = -v_k off S (the breakpoints E1 and E2 of
// Section 4.4), f^T clip(v - beta f) = |S| - 1 on the range where no entry
// leaves the active set (Proposition in Section 4.4) reads
//     sum_k max(0, beta - kappa_k) = 1,
// a concave, decreasing, piecewise-linear equation whose root is
//     beta* = min_m (1 + kappa_(1) + ... + kappa_(m)) / m
// over the ascending order kappa_(1) <= kappa_(2) <= ...
//
// Small D: sort kappa with the network above, then take the minimum over m.
template <int D>
__device__ __forceinline__ float beta_sorted(float (&kap)[D], int d) {
    sort_asc<D>(kap);
    float P = 1.0f + kap[0];
    float best = P;
#pragma unroll
    for (int m = 2; m <= D; ++m) {
        P += kap[m - 1];
        if (m <= d) best = fminf(best, P * (1.0f / (float)m));  // 1/m folds to a constant
    }
    return fmaxf(best, 0.0f);
}

// ---------------------------------------------------------------------------
// Euclidean projection of v (entries k < d; entries k >= d must hold kPadV)
// onto the parity polytope PP_d (Section 4.4, Algorithm 2).
//
//  1. cube clip zh = Pi_[0,1](v).
//  2. the only odd-set facet sum_S z - sum_{S^c} z <= |S| - 1 that a cube
//     point can violate is the most violated one: S = {k : zh_k > 1/2}, with
//     the entry closest to 1/2 flipped when |S| is even.  When it is violated
//     it is the facet f_r of eq. (fr-def) (S = the r+1 largest entries).
//  3. not violated: zh is in PP_d (Corollary 1 / Lemma 4) and is the answer.
//  4. violated: z = Pi_[0,1](v - beta* f_S) (Lemma 4) with beta* from the
//     two-slice breakpoint equation above.
//
// The result is returned implicitly: z_k = Pi_[0,1](v_k - beta f_k) with
// f_k = +1 where bit k of `facet` is set and -1 elsewhere; beta = 0 means
// z = zh.  Callers form z on the fly, so no z array stays live.
struct Proj {
    unsigned facet;
    float beta;
};

__device__ __forceinline__ float proj_z(float v, const Proj &pr, int k) {
    return __saturatef(((pr.facet >> k) & 1u) ? v - pr.beta : v + pr.beta);
}
//
// Facet and violation test in one pass.  With zh = clip(v) and
// delta_k = |zh_k - 1/2|, zh_k = 1/2 + delta_k on S and 1/2 - delta_k off S, so
// for the odd set S the facet value is g = |S| - d/2 + sum_k delta_k, and
// g > |S| - 1 reads  sum_k delta_k > d/2 - 1.  Flipping entry kb (when the
// set {zh > 1/2} is even) lowers the left side by 2 delta_kb either way.  The
// entry closest to 1/2 is found with one integer min over keys holding
// delta's bit pattern (nonnegative floats order as integers) with its low
// bits replaced by the index; entries whose distances agree to within those
// bits are tied and the lowest index wins.
template <int D>
__device__ __forceinline__ Proj project_pp(const float (&v)[D], int d) {
    static_assert(D >= 1 && D <= 8, "wider checks use project_wide");
    constexpr int kIdxBits = 3;
    constexpr int kIdxMask = (1 << kIdxBits) - 1;
    unsigned th = 0u;
    int key = 0x7fffffff;
    float sdist = 0.0f;
    // zh_k > 1/2 exactly when v_k > 1/2; tz = zh - 1/2 in packed FP32 pairs
    // (each lane rounds as the scalar subtraction); |tz| is taken in the sum
    // and, as the cleared sign bit, in the key.
    float tz[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (v[k] > 0.5f) th |= 1u << k;
        tz[k] = __saturatef(v[k]);
    }
#pragma unroll
    for (int k = 0; k + 1 < D; k += 2) {
        const float2 t2 = __fadd2_rn(make_float2(tz[k], tz[k + 1]), make_float2(-0.5f, -0.5f));
        tz[k] = t2.x;
        tz[k + 1] = t2.y;
    }
    if (D & 1) tz[D - 1] = tz[D - 1] - 0.5f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (k < d) {
            sdist += fabsf(tz[k]);
            key = min(key, (__float_as_int(tz[k]) & (0x7fffffff & ~kIdxMask)) | k);
        }
    }
    if ((__popc(th) & 1) == 0) {
        th ^= 1u << (key & kIdxMask);
        sdist -= 2.0f * __int_as_float(key & ~kIdxMask);
    }
    Proj pr;
    pr.facet = th;
    pr.beta = 0.0f;
    if (sdist <= 0.5f * (float)d - 1.0f) return pr;  // zh already in PP_d

    {
        float kap[D];
#pragma unroll
        for (int k = 0; k < D; ++k)
            kap[k] = (k < d) ? (((th >> k) & 1u) ? v[k] - 1.0f : -v[k]) : kBigKappa;
        // One active breakpoint: with kappa_(1) <= kappa_(2) the two smallest,
        // beta* = 1 + kappa_(1) exactly when kappa_(2) >= 1 + kappa_(1) (then only
        // kappa_(1) lies below beta*).  This holds for most violated checks once a
        // frame has settled, and skips the sort; otherwise sort and scan.
        float k1 = fminf(kap[0], D > 1 ? kap[1] : kBigKappa);
        float k2 = D > 1 ? fmaxf(kap[0], kap[1]) : kBigKappa;
#pragma unroll
        for (int k = 2; k < D; ++k) {
            k2 = fminf(k2, fmaxf(k1, kap[k]));
            k1 = fminf(k1, kap[k]);
        }
        const float c1 = 1.0f + k1;
        pr.beta = k2 >= c1 ? fmaxf(c1, 0.0f) : beta_sorted<D>(kap, d);
    }
    return pr;
}

// ---------------------------------------------------------------------------
// Code graph and per-launch arguments (passed by value).
struct CodeView {
    int n, m, E, Ep;          // Ep: E rounded up to a multiple of 8 (state row stride)
    const int *row_ptr;       // [m+1] CSR
    const int *col_idx;       // [E]   variable of each CSR edge
    const int *col_ptr;       // [n+1] CSC
    const int *csc_edge;      // [E]   CSR edge id of each CSC slot
    // Regular codes only (null otherwise): 16-bit copies of the indices, in one
    // block of idx16_bytes (a multiple of 16): col16[col16_elems] = col_idx
    // (CSR order, padded to a multiple of 8 entries), then csc16[4n] = the CSR
    // edge ids of each variable's edges in 4 slots (unused slots 0).  Global
    // memory, or the CTA's shared-memory copy (generic pointers).
    const uint16_t *col16;
    const uint16_t *csc16;
    int idx16_bytes;
    int col16_elems;
    int reg_dc;               // regular-code kernels: the common check degree (check j owns edges
                              // j*reg_dc ...), or 0 when check degrees differ (wide classes only)
    const int *check_order;   // wide classes with differing check degrees: the order in which the
                              // check phase takes the checks (a permutation of 0..m-1), else null
};

struct IterCfg {
    float mu_inv;       // 1/mu
    float rho;          // over-relaxation
    float rho_inv;      // 1/rho
    float omr;          // 1 - rho
    float tmr;          // 2 - rho
    float cert_tol;
    double eps2E;       // eps^2 * E
    double epsc2E;      // max(eps, 1e-5)^2 * E
    int max_iter;
    int check_stop;     // eps > 0
    QScale q;           // q16_t state only: the fixed-point scale
    long long wait_clocks;  // STREAMED: limit of a first wait on a copy or a ring slot (kWaitClocks)
};

struct DecodeArgs {
    CodeView code;
    IterCfg cfg;
    int n_frames;
    const float *llr;        // [F x n]
    float *x_out;            // [F x n]
    uint8_t *bits_out;       // [F x n] or null
    int32_t *iters_out;      // [F] or null
    uint8_t *cert_out;       // [F] or null
    // STREAMED schedule: state kept in device memory between launches (null when RESIDENT)
    void *w_state;           // [F x Ep] of S (w = z - lambda/mu)
    void *l_state;           // [F x Ep] of S (lambda/mu)
    int32_t *k_state;        // [F] iterations done; -1 once the frame is finished
    int iters_this_launch;   // RESIDENT: max_iter
    const int *frame_list;   // [n_frames] ids of the frames to run, or null for 0..n_frames-1
    int *queue;              // frame work-queue counter, zero at launch
    int group_threads;       // GT, a multiple of 32
    int smem_per_group;      // bytes of one group's slice
    int off_x;               // byte offset of x in a slice
    int off_red;             // byte offset of the reduction scratch in a slice
    int slice_base;          // byte offset of the first slice: 0, or (staged regular form) the
                             // 128-aligned size of the 16-bit index block copied to offset 0
    // STREAMED ring (decode_kernel_ring): R state slots for G compute groups;
    // smem_per_group / off_red then describe a group's scratch (x at 0).
    int ring_slots;          // R (0: not a ring launch)
    int ring_groups;         // G
    int ring_slot_bytes;     // bytes of one slot (w, lambda/mu, then the LLR row), a multiple of 128
    int ring_off_slots, ring_off_scratch, ring_off_meta;
    int ring_llr_off;        // byte offset of the frame's LLR row in a slot; 0: LLRs read from global memory
};

// Named barrier for one group (ids 1..15; id 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}


// One check update (Algorithm 1 z- and lambda-update with over-relaxation),
// by one thread, in registers.  The edge state is (w, l) = (z - lambda/mu,
// lambda/mu); z_old = w + l.  For small D the gathered x and old z stay in
// registers; for large D they are re-read from shared memory in the store
// pass to keep the register footprint at one D-array.
// DV > 0: the code is regular (every check has degree D, so check j owns
// edges j*D .. j*D+D-1, and every variable has degree DV); the edge state of a
// check is then read and written in aligned pairs.
// The regular form with FP32 state folds x into the edge state in iterations
// without residuals (see frame_run); 16-bit state would round
// u = rho x + (1 - rho) w, so it gathers x.
template <typename S>
constexpr bool kFoldX = std::is_same<S, float>::value;

// Position of an edge's state in the (4,8) regular form.  With one thread per
// check, a warp's checks j0..j0+31 start 8 words apart, so the paired 8-byte
// accesses of the check update would meet the same banks every fourth check
// (a 4-way conflict).  The pair slot of edge k of check j is therefore XORed
// with (j >> 2) & 3: within each half warp, the four checks that share a bank
// group use four different pair slots, and every paired load and store of the
// check update takes the minimum of two wavefronts.  The variable phase
// gathers through the 16-bit edge ids, which hold these positions.
__host__ __device__ constexpr int state_pos8(int e) {
    return (e & ~7) | ((((e >> 1) & 3) ^ ((e >> 5) & 3)) << 1) | (e & 1);
}

// RES: also accumulate the primal and dual residual terms (iterations that run
// the stopping test or produce the certificate); without them z_old is not
// needed and v = rho x + (1 - rho) w + (2 - rho) lambda/mu directly.
template <int D, int DV, typename S, bool RES>
__device__ __forceinline__ void check_update(const CodeView &c, const IterCfg &p, int j,
                                             S *ws, S *ls, const float *xs, float &rp, float &rd) {
    constexpr bool kKeep = RES && D <= 8;
    constexpr bool kReg = DV > 0;
    constexpr bool kPairs = kReg && (D % 2 == 0);
    const int e0 = kReg ? j * D : __ldg(c.row_ptr + j);
    const int d = kReg ? D : __ldg(c.row_ptr + j + 1) - e0;
    float v[D];
    float xv[kKeep ? D : 1], zo[kKeep ? D : 1];
    // (4,8) form: pair slot k/2 of check j sits at slot (k/2) ^ ((j >> 2) & 3) (state_pos8)
    constexpr bool kSwz = kPairs && D == 8;
    const int sw = kSwz ? ((j >> 2) & 3) : 0;
    if constexpr (kPairs) {
        const uint32_t *ci = reinterpret_cast<const uint32_t *>(c.col16 + e0);
#pragma unroll
        for (int k = 0; k < D; k += 2) {
            const int ks = kSwz ? 2 * ((k >> 1) ^ sw) : k;
            const float2 w2 = ld2<S>(ws + e0 + ks, p.q);  // u = rho x + (1 - rho) w when folded
            const float2 l2 = ld2<S>(ls + e0 + ks, p.q);
            if constexpr (!RES && kFoldX<S>) {  // regular form (kPairs): ws holds u
                const float2 vv = __ffma2_rn(make_float2(p.tmr, p.tmr), l2, w2);  // packed pair, lane = fmaf
                v[k] = vv.x;
                v[k + 1] = vv.y;
                continue;
            }
            const uint32_t cc = ci[k / 2];
            const float x0 = xs[cc & 0xffffu], x1 = xs[cc >> 16];
            if constexpr (RES) {
                const float z0 = w2.x + l2.x, z1 = w2.y + l2.y;  // z_old
                if constexpr (kKeep) { xv[k] = x0; xv[k + 1] = x1; zo[k] = z0; zo[k + 1] = z1; }
                v[k] = fmaf(p.rho, x0, p.omr * z0) + l2.x;
                v[k + 1] = fmaf(p.rho, x1, p.omr * z1) + l2.y;
            } else {
                v[k] = fmaf(p.rho, x0, fmaf(p.omr, w2.x, p.tmr * l2.x));
                v[k + 1] = fmaf(p.rho, x1, fmaf(p.omr, w2.y, p.tmr * l2.y));
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < d) {
                const int e = e0 + k;
                const float lk = ld<S>(ls[e], p.q);
                const float xk = xs[__ldg(c.col_idx + e)];
                if constexpr (RES) {
                    const float zk = ld<S>(ws[e], p.q) + lk;  // z_j^old
                    if constexpr (kKeep) { xv[k] = xk; zo[k] = zk; }
                    const float q = fmaf(p.rho, xk, p.omr * zk);  // rho P_j x + (1 - rho) z_j^old
                    v[k] = q + lk;                                 // v_j = q + lambda_j / mu
                } else {
                    v[k] = fmaf(p.rho, xk, fmaf(p.omr, ld<S>(ws[e], p.q), p.tmr * lk));
                }
            } else {
                v[k] = kPadV;
            }
        }
    }
    const Proj pr = project_pp<D>(v, d);
    if constexpr (kPairs) {
#pragma unroll
        for (int k = 0; k < D; k += 2) {
            const float z0 = proj_z(v[k], pr, k), z1 = proj_z(v[k + 1], pr, k + 1);
            // lambda/mu = v - z and w = z - lambda/mu as packed FP32 pairs (a
            // product with -1 is exact, so each lane rounds as the subtraction)
            const float2 m1 = make_float2(-1.0f, -1.0f);
            const float2 zz = make_float2(z0, z1);
            const float2 ll = __ffma2_rn(zz, m1, make_float2(v[k], v[k + 1]));
            const float2 ww = __ffma2_rn(ll, m1, zz);
            const int ks = kSwz ? 2 * ((k >> 1) ^ sw) : k;
            st2<S>(ls + e0 + ks, ll.x, ll.y, p.q);
            st2<S>(ws + e0 + ks, ww.x, ww.y, p.q);
            if constexpr (RES) {
                float a = xv[k] - z0, b = z0 - zo[k];
                rp = fmaf(a, a, rp);
                rd = fmaf(b, b, rd);
                a = xv[k + 1] - z1;
                b = z1 - zo[k + 1];
                rp = fmaf(a, a, rp);
                rd = fmaf(b, b, rd);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < d) {
                const int e = e0 + k;
                const float z = proj_z(v[k], pr, k);
                float xk = 0.0f, zk = 0.0f;
                if constexpr (kKeep) { xk = xv[k]; zk = zo[k]; }
                else if constexpr (RES) { xk = xs[__ldg(c.col_idx + e)]; zk = ld<S>(ws[e], p.q) + ld<S>(ls[e], p.q); }
                const float l = v[k] - z;  // lambda/mu += q - z, i.e. lambda/mu = v - z
                ls[e] = st<S>(l, p.q);
                ws[e] = st<S>(z - l, p.q);
                if constexpr (RES) {
                    const float a = xk - z;
                    const float b = z - zk;
                    rp = fmaf(a, a, rp);
                    rd = fmaf(b, b, rd);
                }
            }
        }
    }
}

// Check update for wide checks (D > 8): L = 1 or 2 adjacent lanes per check,
// lane r holding entries r, r + L, r + 2L, ... in registers (V = D / L of
// them), so every load and store is at a compile-time offset from the check's
// first edge and the lanes combine their partial results with one xor-shuffle
// each.  Entries q >= d hold kPadV: they clip to 0, are never in the facet set,
// and their breakpoint is +1e30, so they never become active.
//
// After the facet choice the registers hold the breakpoints kappa_q = v_q - 1
// on the facet set and -v_q off it; v and z are rebuilt from kappa: v = kappa + 1,
// z = clip(v - beta) on the set; v = -kappa, z = clip(v + beta) off it.  beta*
// solves sum_q max(0, beta - kappa_q) = 1 (see beta_sorted): h(beta) =
// sum_q max(0, beta - kappa_q) - 1 is convex and increasing, so Newton's step
// beta <- (1 + sum_{kappa < beta} kappa) / #{kappa < beta} from any point above
// the root decreases monotonically to it (the tangent lies below h) and stops
// when the active set stops changing.  The pass that takes a step also finds
// the largest active breakpoint; when the new point lies above it, the active
// set cannot change and the step is final without another pass (the pass it
// saves would return the same value).  It starts from the smaller of two
// points above the root: (1 + sum_q kappa_q) / d, exact when every breakpoint
// is active, and 1 + kappa_(1), exact when only the smallest one is.
// DV > 0: the regular form (16-bit column indices; with FP32 state and no
// residuals ws holds u = rho x + (1 - rho) w, see frame_run).  Check j's
// edges start at j*reg_dc when every check has degree reg_dc, else at
// row_ptr[j].  Both lanes of a pair must call this with the same j; a pair
// whose check index is out of range passes valid = false and stores nothing.
// Reductions over the L adjacent lanes (L = 1, 2 or 4) that share a check.
template <int L>
__device__ __forceinline__ float pair_sum(float x) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
template <int L>
__device__ __forceinline__ int pair_sum_i(int x) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
template <int L>
__device__ __forceinline__ int pair_min_i(int x) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
template <int L>
__device__ __forceinline__ float pair_min(float x) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// The projection of one wide check.  On entry kap[k] holds v of this lane's
// entry q = k*L + r (kPadV for q >= d; dr = d - r); on return it holds the
// breakpoint kappa_q, bit k of th marks the facet set, and the result is beta
// (0 when clip(v) is already in PP_d).  Every lane of the warp must call this
// (the pair reductions are warp-wide shuffles); a pair with d = 0 does no work
// that matters.
template <int D, int L>
__device__ __forceinline__ float project_wide(float (&kap)[D / L], int d, int dr, int r, unsigned &th_out) {
    constexpr int V = D / L;
    // facet S = {v > 1/2}, the entry closest to 1/2 flipped when |S| is even;
    // violation test sum_q |clip(v_q) - 1/2| (- 2 min when flipped) > d/2 - 1.
    // Padded entries add 1/2 each to the sum, as they do to the right side
    // (taken over all D entries).  Keys hold the entry index q = k*L + r.
    unsigned th = 0u;  // bit k: this lane's entry k is in the facet set
    int key = 0x7fffffff;
    float sdist = 0.0f;
#pragma unroll
    for (int k = 0; k < V; k += 2) {
        const float a = kap[k], b = k + 1 < V ? kap[k + 1] : kPadV;
        if (a > 0.5f) th |= 1u << k;
        if (b > 0.5f) th |= 1u << (k + 1);
        const float2 t2 = __fadd2_rn(make_float2(__saturatef(a), __saturatef(b)), make_float2(-0.5f, -0.5f));
        sdist += fabsf(t2.x);
        key = min(key, (__float_as_int(t2.x) & 0x7fffffe0) | (k * L + r));
        if (k + 1 < V) {
            sdist += fabsf(t2.y);
            key = min(key, (__float_as_int(t2.y) & 0x7fffffe0) | ((k + 1) * L + r));
        }
    }
    key = pair_min_i<L>(key);
    sdist = pair_sum<L>(sdist);
    if ((pair_sum_i<L>(__popc(th)) & 1) == 0) {
        const int qb = key & 31;
        if (qb % L == r) th ^= 1u << (qb / L);
        sdist -= 2.0f * __int_as_float(key & ~31);
    }
    const bool violated = d > 0 && sdist > 0.5f * (float)D - 1.0f;
    // breakpoints in place; their sum over the real entries, and the smallest
    float ksum = 0.0f, k1 = kBigKappa;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        kap[k] = ((th >> k) & 1u) ? kap[k] - 1.0f : -kap[k];
        if (k * L < dr) ksum += kap[k];
        k1 = fminf(k1, kap[k]);
    }
    ksum = pair_sum<L>(ksum);
    k1 = pair_min<L>(k1);
    th_out = th;
    float beta = 0.0f;
    if (violated) {  // the same for both lanes of a pair
        const unsigned pm = ((1u << L) - 1u) << (threadIdx.x & (32 - L));  // the check's lanes
        beta = fminf(__fdividef(1.0f + ksum, (float)d), 1.0f + k1);
        for (int it = 0; it <= D; ++it) {
            float s1 = 0.0f, kmax = -kBigKappa;
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (kap[k] < beta) { s1 += kap[k]; ++cnt; kmax = fmaxf(kmax, kap[k]); }
#pragma unroll
            for (int o = 1; o < L; o <<= 1) {
                s1 += __shfl_xor_sync(pm, s1, o);
                cnt += __shfl_xor_sync(pm, cnt, o);
                kmax = fmaxf(kmax, __shfl_xor_sync(pm, kmax, o));
            }
            const float nb = __fdividef(1.0f + s1, (float)cnt);  // cnt >= 1: beta > kappa_(1)
            if (!(nb < beta)) break;
            beta = nb;
            // no breakpoint in [nb, old beta): the active set at nb is the same,
            // so a further step would return nb again (the same sum, bit for bit)
            if (nb > kmax) break;
        }
        beta = fmaxf(beta, 0.0f);
    }
    return beta;
}

// v and z of entry k after project_wide.
__device__ __forceinline__ void wide_vz(float kap, bool on, float beta, float &v, float &z) {
    v = on ? kap + 1.0f : -kap;
    z = __saturatef(on ? v - beta : v + beta);
}

template <int D, int L, int DV, typename S, bool RES>
__device__ __forceinline__ void check_update_w(const CodeView &c, const IterCfg &p, int j, bool valid, S *ws, S *ls,
                                               const float *xs, float &rp, float &rd) {
    static_assert(D > 8 && D <= 32 && (L == 1 || L == 2 || L == 4) && D % L == 0, "wide class");
    constexpr int V = D / L;
    const int r = threadIdx.x & (L - 1);
    int e0 = 0, d = 0;
    if (valid) {
        if (DV > 0 && c.reg_dc > 0) {
            d = c.reg_dc;
            e0 = j * d;
        } else {
            e0 = __ldg(c.row_ptr + j);
            d = __ldg(c.row_ptr + j + 1) - e0;
        }
    }
    auto col_of = [&](int e) -> int {
        if constexpr (DV > 0) return c.col16[e];
        else return __ldg(c.col_idx + e);
    };
    constexpr bool kFold = kFoldX<S> && DV > 0 && !RES;
    const int eb = e0 + r;   // this lane's first entry; entry k of the lane is edge eb + k*L
    const int dr = d - r;    // entry k of the lane is real when k*L < dr
    const S *wsj = ws + eb;
    const S *lsj = ls + eb;
    float kap[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        if (k * L < dr) {
            if constexpr (kFold) {
                kap[k] = fmaf(p.tmr, ld<S>(lsj[k * L], p.q), ld<S>(wsj[k * L], p.q));
            } else {
                const float xk = xs[col_of(eb + k * L)];
                kap[k] = fmaf(p.rho, xk, fmaf(p.omr, ld<S>(wsj[k * L], p.q), p.tmr * ld<S>(lsj[k * L], p.q)));
            }
        } else {
            kap[k] = kPadV;
        }
    }
    unsigned th;
    const float beta = project_wide<D, L>(kap, d, dr, r, th);
    // z, lambda/mu = v - z and w = z - lambda/mu
    // Every entry is computed and only the stores (and the residual terms) are
    // guarded: with the whole entry under the guard the compiler branched
    // around it, and the divergent branches and their reconvergence cost
    // C8000 8% of its time.
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const bool real = k * L < dr;
        float v, z;
        wide_vz(kap[k], (th >> k) & 1u, beta, v, z);
        const float l = v - z;
        const float w = z - l;
        const int e = eb + k * L;
        if constexpr (RES) {
            // x_i(e) from v = rho x + (1 - rho) w_old + (2 - rho) lambda_old/mu
            // rather than a second gather (equal up to FP32 rounding)
            float wo = 0.0f, lo = 0.0f;
            if (real) {
                wo = ld<S>(ws[e], p.q);
                lo = ld<S>(ls[e], p.q);
            }
            const float xk = (v - fmaf(p.omr, wo, p.tmr * lo)) * p.rho_inv;
            const float a = xk - z;
            const float b = z - (wo + lo);
            rp = real ? fmaf(a, a, rp) : rp;
            rd = real ? fmaf(b, b, rd) : rd;
        }
        if (real) {
            ls[e] = st<S>(l, p.q);
            ws[e] = st<S>(w, p.q);
        }
    }
}

// Shared-memory slice of one group: w[Ep], l[Ep] (type S), x[n] (float),
// red[2 * nwarps] (float), flags[8] (int; the last two hold an mbarrier).
// The edge state is kept as w = z - lambda/mu and l = lambda/mu: the x-update
// needs only the sum of w over a variable's edges (one gather per edge), and
// the check update recovers z_old = w + l.
template <typename S>
struct Slice {
    S *w, *l;
    float *x, *red;
    int *flags;      // [0] converged, [1] residual ok, [2] bad LLR, [3] copy ok, [4..5] frame ids
    uint64_t *mbar;  // flags[6..7]: completion barrier of the bulk loads
    const float *llr = nullptr;  // ring kernel: the frame's LLRs copied into its slot (else read from io.llr)
};


// Copy nbytes (a multiple of 16) between 16-byte aligned buffers, cooperatively.
__device__ __forceinline__ void copy16(void *dst, const void *src, int nbytes, int t, int T) {
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int i = t; i < (nbytes >> 4); i += T) d[i] = s[i];
}
// Fill nbytes (a multiple of 16) with a repeated 32-bit pattern, cooperatively.
__device__ __forceinline__ void fill16(void *dst, int nbytes, unsigned pattern, int t, int T) {
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 zz = make_uint4(pattern, pattern, pattern, pattern);
    for (int i = t; i < (nbytes >> 4); i += T) d[i] = zz;
}
__device__ __forceinline__ void zero16(void *dst, int nbytes, int t, int T) { fill16(dst, nbytes, 0u, t, T); }

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine, non-tensor form) between global and
// shared memory, completed through an mbarrier (loads) or a bulk group
// (stores).  Addresses must be 16-byte aligned and sizes multiples of 16.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// LLR i of the frame: from its row copied into shared memory (ring kernel,
// gs != null; an ordinary load, so it stays after the wait for the copy),
// else a read-only global load.
template <bool READY>
__device__ __forceinline__ float llr_at(const float *g, const float *gs, int i) {
    if constexpr (READY)
        if (gs) return gs[i];
    return __ldg(g + i);
}

// Wait for the mbarrier phase with the given parity, for at most ~1 s of SM
// clocks; returns false on timeout (the caller reports it, never spins forever).
// The first wait on a copy or a slot takes the decode's limit
// (IterCfg::wait_clocks, normally kWaitClocks); the wait for copies still in
// flight after a timeout always takes kWaitClocks, so no CTA leaves while a
// copy into its shared memory may still land.
constexpr long long kWaitClocks = 1ll << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit = kWaitClocks) {
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > limit) return false;
    }
    return true;
}
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst_gmem, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until every committed bulk store has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Order this thread's generic-proxy shared-memory accesses (and, after a
// barrier, the group's) before later async-proxy accesses.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr int kFrameTimeout = -2;  // iters_out value of a frame abandoned after a copy timed out (LPDEC_FRAME_ABANDONED)

// Decode frame f (RESIDENT) or advance it by up to iters_this_launch
// iterations (STREAMED), with one group of T threads; t is the thread's rank.
// Every thread of the group calls this; all branches on shared data are
// group-uniform.
// Where one frame's inputs, outputs and (STREAMED) parked state live.
struct FrameIO {
    const float *llr;   // [n]
    float *x;           // [n]
    uint8_t *bits;      // [n] or null
    int32_t *iters;     // one value or null
    uint8_t *cert;      // one value or null
    void *w_state;      // STREAMED: [Ep] of S
    void *l_state;      // STREAMED: [Ep] of S
    int32_t *k_state;   // STREAMED: iterations done (-1: finished); null when RESIDENT
};

// L = 1: one thread per check; L > 1: L lanes per check (segmented update).
// Returns false only if a bulk copy timed out; the group must then stop.
// READY (STREAMED ring): a parked frame's state is already in sm (the caller
// waited for its copies), so no copy is issued or awaited here.
// PF (regular form with the 16-bit indices in global memory): the x-update
// loads the next variable's edge ids and LLR while it processes this one.
template <int D, int L, int DV, typename S, bool READY = false, bool PF = false>
__device__ __forceinline__ bool frame_run(const CodeView &c, const IterCfg &p, int iters_this_launch, const FrameIO &io,
                          const Slice<S> &sm, int t, int T, int bar, uint32_t &phase) {
    const int lane = t & 31, w = t >> 5, nw = T >> 5;
    volatile int *flags = sm.flags;
    const float *gam = io.llr;
    const float *gam_s = READY ? sm.llr : nullptr;
    const bool streamed = io.k_state != nullptr;
    const int state_bytes = c.Ep * (int)sizeof(S);

    int k = streamed ? *io.k_state : 0;
    if (k < 0) return true;  // finished in an earlier launch
    if (t == 0) { flags[0] = 0; flags[1] = 0; flags[2] = 0; }

    if (k == 0) {
        // Algorithm 1 initialization: z = lambda = 0 (w = 0).  Also reject non-finite LLRs.
        int bad = 0;
        for (int i = t; i < c.n; i += T) bad |= !isfinite(llr_at<READY>(gam, gam_s, i));
        fill16(sm.w, 2 * state_bytes, state_zero2<S>(), t, T);
        bad = __any_sync(0xffffffffu, bad);
        group_sync(bar, T);
        if (bad && lane == 0) atomicOr((int *)&flags[2], 1);
        group_sync(bar, T);
        if (flags[2]) {
            for (int i = t; i < c.n; i += T) {
                io.x[i] = 0.0f;
                if (io.bits) io.bits[i] = 0;
            }
            if (t == 0) {
                if (io.iters) *io.iters = -1;
                if (io.cert) *io.cert = 0;
                if (streamed) *io.k_state = -1;
            }
            return true;
        }
    } else if constexpr (!READY) {
        // STREAMED: bring the parked w and lambda/mu back with two bulk copies.
        const void *zg = io.w_state;
        const void *lg = io.l_state;
        if (t == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(sm.mbar, 2u * (uint32_t)state_bytes);
            bulk_load(sm.w, zg, (uint32_t)state_bytes, sm.mbar);
            bulk_load(sm.l, lg, (uint32_t)state_bytes, sm.mbar);
            flags[3] = mbar_wait_bounded(sm.mbar, phase, p.wait_clocks) ? 1 : 0;
        }
        group_sync(bar, T);
        if (flags[3] == 0) {
            if (t == 0) {
                mbar_wait_bounded(sm.mbar, phase);  // one more bounded wait for the copies in flight
                if (io.iters) *io.iters = kFrameTimeout;
                if (io.cert) *io.cert = 0;
                *io.k_state = -1;
            }
            return false;
        }
        mbar_wait_bounded(sm.mbar, phase);  // already complete: each thread acquires the copied data
        phase ^= 1u;
    }

    const int k_end = min(p.max_iter, k + iters_this_launch);
    bool conv = false, rok = false;
    while (k < k_end) {
        // Residual terms are needed by the stopping test and, on the last
        // iteration, by the certificate.
        const bool need_res = p.check_stop || (k + 1 == p.max_iter);
        // Regular form with FP32 state, iterations without residuals: after
        // computing x_i the variable thread folds it into its edges,
        // overwriting w_e with u_e = rho x_i + (1 - rho) w_e, so the check
        // update forms v = u + (2 - rho) lambda/mu without gathering x.  (The
        // generic form would need a second pass over each variable's edges.)
        const bool fold = kFoldX<S> && DV > 0 && !need_res;
        // ---- x-update (Algorithm 1; Section 3.2): sum over the edges of w = z - lambda/mu
        uint2 pk_next = make_uint2(0u, 0u);
        float g_next = 0.0f;
        if constexpr (DV > 0 && PF) {
            if (t < c.n) {
                pk_next = *reinterpret_cast<const uint2 *>(c.csc16 + 4 * t);
                g_next = llr_at<READY>(gam, gam_s, t);
            }
        }
        for (int i = t; i < c.n; i += T) {
            float acc = 0.0f, inv_dv;
            if constexpr (DV > 0) {
                static_assert(DV <= 4, "regular form holds up to 4 edges per variable");
                uint2 pk;
                float gi;
                if constexpr (PF) {
                    pk = pk_next;
                    gi = g_next;
                    if (i + T < c.n) {
                        pk_next = *reinterpret_cast<const uint2 *>(c.csc16 + 4 * (i + T));
                        g_next = llr_at<READY>(gam, gam_s, i + T);
                    }
                } else {
                    pk = *reinterpret_cast<const uint2 *>(c.csc16 + 4 * i);
                    gi = llr_at<READY>(gam, gam_s, i);
                }
                const unsigned es[4] = {pk.x & 0xffffu, pk.x >> 16, pk.y & 0xffffu, pk.y >> 16};
                float wv[DV];
#pragma unroll
                for (int s = 0; s < DV; ++s) {
                    wv[s] = ld<S>(sm.w[es[s]], p.q);
                    acc += wv[s];
                }
                inv_dv = 1.0f / (float)DV;
                const float x = __saturatef((acc - gi * p.mu_inv) * inv_dv);
                // x is read only by the check update of a residual iteration and
                // by the outputs, which follow a residual iteration (the last
                // one, or the one that stops); a folded iteration need not store it
                if (!fold) sm.x[i] = x;
                if (fold) {
                    const float rx = p.rho * x;
#pragma unroll
                    for (int s = 0; s + 1 < DV; s += 2) {  // packed FP32 pairs (each lane rounds as fmaf)
                        const float2 uu = __ffma2_rn(make_float2(p.omr, p.omr), make_float2(wv[s], wv[s + 1]),
                                                     make_float2(rx, rx));
                        sm.w[es[s]] = st<S>(uu.x, p.q);
                        sm.w[es[s + 1]] = st<S>(uu.y, p.q);
                    }
                    if (DV & 1) sm.w[es[DV - 1]] = st<S>(fmaf(p.omr, wv[DV - 1], rx), p.q);
                }
            } else {
                const int s0 = __ldg(c.col_ptr + i), s1 = __ldg(c.col_ptr + i + 1);
                for (int s = s0; s < s1; ++s) {
                    const int e = __ldg(c.csc_edge + s);
                    acc += ld<S>(sm.w[e], p.q);
                }
                inv_dv = __frcp_rn((float)(s1 - s0));
                const float gi = llr_at<READY>(gam, gam_s, i);
                const float x = __saturatef((acc - gi * p.mu_inv) * inv_dv);
                sm.x[i] = x;
            }
        }
        group_sync(bar, T);
        // ---- z- and lambda-updates (Algorithm 1; Section 5.2 over-relaxation)
        float rp = 0.0f, rd = 0.0f;
        if constexpr (D > 8) {
            // L lanes per check; every lane of the group runs the same number of passes
            // (with check_order, a warp's 16 lane pairs take 16 consecutive entries
            // of it: see check_order_for_banks)
            const int per_pass = T / L;
            if (need_res) {
                for (int j0 = 0; j0 < c.m; j0 += per_pass) {
                    const int jj = j0 + t / L;
                    const int j = (jj < c.m && c.check_order) ? __ldg(c.check_order + jj) : jj;
                    check_update_w<D, L, DV, S, true>(c, p, j, jj < c.m, sm.w, sm.l, sm.x, rp, rd);
                }
            } else {
                for (int j0 = 0; j0 < c.m; j0 += per_pass) {
                    const int jj = j0 + t / L;
                    const int j = (jj < c.m && c.check_order) ? __ldg(c.check_order + jj) : jj;
                    check_update_w<D, L, DV, S, false>(c, p, j, jj < c.m, sm.w, sm.l, sm.x, rp, rd);
                }
            }
        } else {
            static_assert(L == 1, "checks of degree <= 8 take one thread each");
            if (need_res) {
                for (int j = t; j < c.m; j += T) check_update<D, DV, S, true>(c, p, j, sm.w, sm.l, sm.x, rp, rd);
            } else {
                for (int j = t; j < c.m; j += T) check_update<D, DV, S, false>(c, p, j, sm.w, sm.l, sm.x, rp, rd);
            }
        }
        ++k;
        if (need_res) {
            // ---- stopping test (Algorithm 1; Section 3.3)
            rp = warp_sum(rp);
            rd = warp_sum(rd);
            if (lane == 0) { sm.red[2 * w] = rp; sm.red[2 * w + 1] = rd; }
            group_sync(bar, T);
            if (w == 0) {
                // the warps' partial sums added in FP64 across the lanes of warp 0
                double Rp = lane < nw ? (double)sm.red[2 * lane] : 0.0;
                double Rd = lane < nw ? (double)sm.red[2 * lane + 1] : 0.0;
                for (int o = 1; o < nw; o <<= 1) {
                    Rp += __shfl_xor_sync(0xffffffffu, Rp, o);
                    Rd += __shfl_xor_sync(0xffffffffu, Rd, o);
                }
                if (lane == 0) {
                    flags[0] = (p.check_stop && Rp < p.eps2E && Rd < p.eps2E) ? 1 : 0;
                    flags[1] = (Rp < p.epsc2E && Rd < p.epsc2E) ? 1 : 0;
                }
            }
            group_sync(bar, T);
            conv = flags[0] != 0;
            rok = flags[1] != 0;
            if (conv) break;
        } else {
            group_sync(bar, T);
        }
    }

    if (!conv && k < p.max_iter) {
        // STREAMED: park the state in device memory for the next launch with two
        // bulk stores (the group barrier at the end of the iteration ordered every
        // thread's shared-memory writes before them).  The next user of this
        // slice waits for the stores to finish reading it.
        if (t == 0) {
            fence_proxy_async_smem();
            bulk_store(io.w_state, sm.w, (uint32_t)state_bytes);
            bulk_store(io.l_state, sm.l, (uint32_t)state_bytes);
            bulk_commit();
            *io.k_state = k;
        }
        return true;
    }

    // ---- outputs: x, hard decision, certificate
    float frac = 0.0f;
    float *xo = io.x;
    uint8_t *bo = io.bits;
    for (int i = t; i < c.n; i += T) {
        const float x = sm.x[i];
        xo[i] = x;
        if (bo) bo[i] = x > 0.5f ? 1 : 0;
        frac = fmaxf(frac, fminf(x, 1.0f - x));
    }
    int synd = 0;
    for (int j = t; j < c.m; j += T) {
        const int e0 = __ldg(c.row_ptr + j), e1 = __ldg(c.row_ptr + j + 1);
        int par = 0;
        for (int e = e0; e < e1; ++e) par ^= sm.x[__ldg(c.col_idx + e)] > 0.5f ? 1 : 0;
        synd |= par;
    }
    frac = warp_max(frac);
    synd = __any_sync(0xffffffffu, synd);
    if (lane == 0) { sm.red[2 * w] = frac; sm.red[2 * w + 1] = synd ? 1.0f : 0.0f; }
    group_sync(bar, T);
    if (t == 0) {
        float fr = 0.0f;
        bool sy = false;
        for (int q = 0; q < nw; ++q) { fr = fmaxf(fr, sm.red[2 * q]); sy |= sm.red[2 * q + 1] != 0.0f; }
        if (io.iters) *io.iters = k;
        if (io.cert) *io.cert = (rok && fr <= p.cert_tol && !sy) ? 1 : 0;
        if (streamed) *io.k_state = -1;
    }
    return true;
}

// Where frame f's inputs, outputs and parked state live.
template <typename S>
__device__ __forceinline__ FrameIO frame_io(const DecodeArgs &a, int f) {
    FrameIO io;
    const size_t off = (size_t)f * a.code.n;
    io.llr = a.llr + off;
    io.x = a.x_out + off;
    io.bits = a.bits_out ? a.bits_out + off : nullptr;
    io.iters = a.iters_out ? a.iters_out + f : nullptr;
    io.cert = a.cert_out ? a.cert_out + f : nullptr;
    if (a.k_state) {
        const size_t sb = (size_t)a.code.Ep * sizeof(S);
        io.w_state = reinterpret_cast<char *>(a.w_state) + (size_t)f * sb;
        io.l_state = reinterpret_cast<char *>(a.l_state) + (size_t)f * sb;
        io.k_state = a.k_state + f;
    } else {
        io.w_state = io.l_state = nullptr;
        io.k_state = nullptr;
    }
    return io;
}

// Persistent decode kernel: each group pulls frame ids from a global counter
// until the batch is exhausted.  DV > 0 selects the regular-code form (check
// degree D, variable degree DV); L is the number of lanes per check.  MAXT:
// largest CTA size the kernel is built for.  STAGE (regular form only): the
// CTA first copies the code's 16-bit index block to the start of its shared
// memory and reads the indices from there; the slices follow at slice_base.
template <int D, int L, int DV, typename S, int MAXT, bool STAGE>
__global__ void __launch_bounds__(MAXT, 1) decode_kernel(const DecodeArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    static_assert(!STAGE || DV > 0, "index staging is built for the regular form");
    CodeView cv = a.code;
    if constexpr (STAGE) {
        copy16(smem_raw, a.code.col16, a.code.idx16_bytes, threadIdx.x, blockDim.x);
        __syncthreads();
        cv.col16 = reinterpret_cast<const uint16_t *>(smem_raw);
        cv.csc16 = cv.col16 + a.code.col16_elems;
    }
    const int T = a.group_threads;
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    const int bar = 1 + g;
    unsigned char *base = smem_raw + a.slice_base + (size_t)g * a.smem_per_group;
    Slice<S> sm;
    sm.w = reinterpret_cast<S *>(base);
    sm.l = sm.w + a.code.Ep;
    sm.x = reinterpret_cast<float *>(base + a.off_x);
    sm.red = reinterpret_cast<float *>(base + a.off_red);
    sm.flags = reinterpret_cast<int *>(sm.red + 2 * (T >> 5));
    sm.mbar = reinterpret_cast<uint64_t *>(sm.flags + 6);
    if (t == 0) {
        mbar_init(sm.mbar, 1);
        fence_proxy_async_smem();
    }
    uint32_t phase = 0;
    int par = 0;
    for (;;) {
        // frame ids are double-buffered (flags[4], flags[5]) so that a slow
        // thread still reading this id is never overtaken by the next fetch.
        // Before the slice is reused, the previous frame's bulk stores must
        // have finished reading it.
        if (t == 0) {
            bulk_wait_read_all();
            sm.flags[4 + par] = atomicAdd(a.queue, 1);
        }
        group_sync(bar, T);
        const int q = sm.flags[4 + par];
        par ^= 1;
        if (q >= a.n_frames) break;
        const int f = a.frame_list ? a.frame_list[q] : q;
        const FrameIO io = frame_io<S>(a, f);
        if (!frame_run<D, L, DV, S, false, !STAGE>(cv, a.cfg, a.iters_this_launch, io, sm, t, T, bar, phase)) break;
    }
    if (t == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// STREAMED schedule with a producer warp and a ring of state slots.
//
// The CTA holds G compute groups and one producer warp.  The producer claims
// frames from the launch's work queue in order and, for each, waits until the
// next of R > G ring slots is free, then starts the bulk copies of the frame's
// parked w and lambda/mu into it (or, for a frame's first launch, publishes it
// at once).  Compute groups take slots in sequence order, wait for the slot's
// copies, run the frame's iterations (frame_run, READY), park it from the slot
// and release the slot once the parking copies have read it.  The loads of the
// next R - G frames are thus in flight while the groups compute.  The producer
// ends with one sentinel slot per group.  Every wait is bounded; a group whose
// wait runs out reports its frame as abandoned (after a bounded wait for the
// copies in flight) and stops, and a producer whose wait runs out drains its
// copies and stops.
struct RingMeta {
    uint64_t full;   // phase k completes when the slot's k-th frame is ready
    uint64_t empty;  // phase k completes when the slot's k-th frame is released
    int frame;       // frame id of the slot's current sequence number, or -1 (no more frames)
    int seq;         // that sequence number
    int pad[2];
};

// Wait (bounded like mbar_wait_bounded) until a slot's tag holds `seq`.
__device__ __forceinline__ bool ring_wait_tag(const int *tag, int seq, long long limit) {
    const long long start = clock64();
    while (*reinterpret_cast<const volatile int *>(tag) != seq) {
        if (clock64() - start > limit) return false;
    }
    return true;
}

template <typename S>
__device__ __forceinline__ S *ring_slot(const DecodeArgs &a, unsigned char *smem_raw, int s) {
    return reinterpret_cast<S *>(smem_raw + a.ring_off_slots + (size_t)s * a.ring_slot_bytes);
}

constexpr int kRingClaim = 4;  // frames the producer claims per atomic while many remain

// Publish frame f (k iterations done; f < 0: no more frames) as sequence
// number seq of the ring: wait until its slot is free, then start the bulk
// copies of the parked state (k > 0) and of the frame's LLRs (when the slots
// hold them), or mark the slot ready at once.  Run by one thread.  Returns
// kPubNone if nothing was published (the wait for the slot ran out or a group
// had stopped), kPubOk, or kPubStop: published, but a group has stopped.
//
// A group that gives up on its slot's tag sets the stop flag and then reads
// the tag; the producer writes the tag and then reads the stop flag.  With a
// block-scope SC fence between the write and the read on both sides, at least
// one of them sees the other's write: the group (tag seen) waits for the
// copies itself, or the producer (stop seen) counts the publish among those
// whose copies it waits for before leaving.
constexpr int kPubNone = 0, kPubOk = 1, kPubStop = 2;
template <typename S>
__device__ __forceinline__ int ring_publish(const DecodeArgs &a, unsigned char *smem_raw, RingMeta *meta,
                                            volatile int *abort_flag, int seq, int f, int k) {
    const int R = a.ring_slots;
    const int s = seq % R;
    if (seq >= R && !mbar_wait_bounded(&meta[s].empty, (uint32_t)(seq / R - 1) & 1u, a.cfg.wait_clocks)) {
        *abort_flag = 1;
        return kPubNone;
    }
    if (*abort_flag) return kPubNone;
    meta[s].frame = f;
    *reinterpret_cast<volatile int *>(&meta[s].seq) = seq;  // the tag groups wait for (ring_wait_tag)
    const uint32_t sbytes = (uint32_t)((size_t)a.code.Ep * sizeof(S));
    const uint32_t lbytes = a.ring_llr_off ? (uint32_t)a.code.n * 4u : 0u;  // a multiple of 16 (host checks)
    const uint32_t tx = f < 0 ? 0u : (k > 0 ? 2u * sbytes : 0u) + lbytes;
    if (tx) {
        S *w = ring_slot<S>(a, smem_raw, s);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&meta[s].full, tx);
        if (k > 0) {
            const size_t off = (size_t)f * sbytes;
            bulk_load(w, reinterpret_cast<const char *>(a.w_state) + off, sbytes, &meta[s].full);
            bulk_load(w + a.code.Ep, reinterpret_cast<const char *>(a.l_state) + off, sbytes, &meta[s].full);
        }
        if (lbytes)
            bulk_load(reinterpret_cast<char *>(w) + a.ring_llr_off, a.llr + (size_t)f * a.code.n, lbytes,
                      &meta[s].full);
    } else {
        mbar_arrive(&meta[s].full);
    }
    __threadfence_block();
    return *abort_flag ? kPubStop : kPubOk;
}

// The producer warp: claims frames in batches (one atomic per batch, the
// batch's iteration counts read by its lanes at once), publishes those not
// finished in order, then one sentinel per group.  Near the end of the queue
// it claims one frame at a time, so no CTA holds a batch while others idle.
template <typename S>
__device__ void ring_produce(const DecodeArgs &a, unsigned char *smem_raw, RingMeta *meta, volatile int *abort_flag,
                             int lane) {
    const unsigned full = 0xffffffffu;
    const int R = a.ring_slots, G = a.ring_groups;
    int seq = 0, batch = kRingClaim, ok = 1;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(a.queue, batch);
        base = __shfl_sync(full, base, 0);
        if (base >= a.n_frames) break;
        const int nb = batch;
        batch = a.n_frames - base > 2 * (int)gridDim.x * kRingClaim ? kRingClaim : 1;
        int f = -1, k = -1;
        if (lane < nb && base + lane < a.n_frames) {
            f = a.frame_list ? a.frame_list[base + lane] : base + lane;
            k = a.k_state[f];
        }
        unsigned live = __ballot_sync(full, k >= 0);
        while (live && ok) {
            const int src = __ffs(live) - 1;
            live &= live - 1;
            const int fs = __shfl_sync(full, f, src);
            const int ks = __shfl_sync(full, k, src);
            int st = kPubNone;
            if (lane == 0) st = ring_publish<S>(a, smem_raw, meta, abort_flag, seq, fs, ks);
            st = __shfl_sync(full, st, 0);
            seq += st != kPubNone;
            ok = st == kPubOk;
        }
        if (!ok) break;
    }
    if (lane != 0) return;
    for (int i = 0; i < G && ok; ++i) {  // one "no more frames" slot per group
        const int st = ring_publish<S>(a, smem_raw, meta, abort_flag, seq, -1, 0);
        seq += st != kPubNone;
        ok = st == kPubOk;
    }
    // After a stop, the copies of the last R published slots may be in flight:
    // wait for them (bounded) before the CTA can exit.
    if (!ok)
        for (int j = seq > R ? seq - R : 0; j < seq; ++j) mbar_wait_bounded(&meta[j % R].full, (uint32_t)(j / R) & 1u);
}

template <int D, int L, int DV, typename S, int MAXT, bool STAGE>
__global__ void __launch_bounds__(MAXT, 1) decode_kernel_ring(const DecodeArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    static_assert(!STAGE || DV > 0, "index staging is built for the regular form");
    CodeView cv = a.code;
    if constexpr (STAGE) {
        copy16(smem_raw, a.code.col16, a.code.idx16_bytes, threadIdx.x, blockDim.x);
        cv.col16 = reinterpret_cast<const uint16_t *>(smem_raw);
        cv.csc16 = cv.col16 + a.code.col16_elems;
    }
    const int R = a.ring_slots, T = a.group_threads;
    RingMeta *meta = reinterpret_cast<RingMeta *>(smem_raw + a.ring_off_meta);
    int *ctr = reinterpret_cast<int *>(meta + R);  // [0] consumer sequence counter, [1] stop flag
    if (threadIdx.x == 0) {
        for (int s = 0; s < R; ++s) {
            mbar_init(&meta[s].full, 1);
            mbar_init(&meta[s].empty, 1);
            meta[s].frame = -1;
            meta[s].seq = -1;
        }
        ctr[0] = 0;
        ctr[1] = 0;
        fence_proxy_async_smem();
    }
    __syncthreads();
    volatile int *abort_flag = ctr + 1;
    if ((int)threadIdx.x >= a.ring_groups * T) {  // the producer warp
        ring_produce<S>(a, smem_raw, meta, abort_flag, threadIdx.x & 31);
        return;
    }
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    const int bar = 1 + g;
    unsigned char *scr = smem_raw + a.ring_off_scratch + (size_t)g * a.smem_per_group;
    Slice<S> sm;
    sm.x = reinterpret_cast<float *>(scr);
    sm.red = reinterpret_cast<float *>(scr + a.off_red);
    sm.flags = reinterpret_cast<int *>(sm.red + 2 * (T >> 5));
    sm.mbar = nullptr;
    uint32_t unused_phase = 0;
    int par = 0;
    for (;;) {
        if (t == 0) sm.flags[4 + par] = atomicAdd(&ctr[0], 1);
        group_sync(bar, T);
        const int my = sm.flags[4 + par];
        par ^= 1;
        const int s = my % R;
        const uint32_t ph = (uint32_t)(my / R) & 1u;
        // A parity wait cannot tell this round from the round two before it.
        // Copies land out of order, so when this group claims `my` the slot may
        // still be in its previous round (my - R published, copies in flight),
        // or already past this one.  So first wait until the slot's tag reads
        // `my`: the producer writes it before publishing, and publishes `my`
        // only after my - R was released, so the slot is then in this round or
        // just past it, which the parity wait tells apart.  After the wait the
        // tag must still read `my` (the producer retags the slot only after this
        // group releases it); a mismatch is a broken invariant and stops the
        // group like a timeout.
        if (t == 0)
            sm.flags[3] = (ring_wait_tag(&meta[s].seq, my, a.cfg.wait_clocks) &&
                           mbar_wait_bounded(&meta[s].full, ph, a.cfg.wait_clocks) &&
                           *reinterpret_cast<const volatile int *>(&meta[s].seq) == my)
                              ? 1
                              : 0;
        group_sync(bar, T);
        if (sm.flags[3] == 0) {
            if (t == 0) {
                *abort_flag = 1;
                __threadfence_block();  // pairs with the producer's fence in ring_publish
                if (*reinterpret_cast<const volatile int *>(&meta[s].seq) == my && meta[s].frame >= 0) {
                    // published, copies late
                    mbar_wait_bounded(&meta[s].full, ph);
                    const int f = meta[s].frame;
                    if (a.iters_out) a.iters_out[f] = kFrameTimeout;
                    if (a.cert_out) a.cert_out[f] = 0;
                    a.k_state[f] = -1;
                }
            }
            break;
        }
        mbar_wait_bounded(&meta[s].full, ph);  // complete: every thread acquires the slot
        const int f = meta[s].frame;
        if (f < 0) break;  // no more frames
        sm.w = ring_slot<S>(a, smem_raw, s);
        sm.l = sm.w + a.code.Ep;
        sm.llr = a.ring_llr_off ? reinterpret_cast<const float *>(reinterpret_cast<const char *>(sm.w) + a.ring_llr_off)
                                : nullptr;
        const FrameIO io = frame_io<S>(a, f);
        frame_run<D, L, DV, S, true, !STAGE>(cv, a.cfg, a.iters_this_launch, io, sm, t, T, bar, unused_phase);
        if (t == 0) {
            // the group's writes to the slot (ordered by its last barrier) and
            // the parking copies' reads of it are done before the producer
            // starts the next copies into it
            fence_proxy_async_smem();
            bulk_wait_read_all();
            mbar_arrive(&meta[s].empty);
        }
    }
    if (t == 0) bulk_wait_all();
}

// Projection of `count` vectors of dimension d (d <= D): one thread per vector
// for D <= 8, the decoder's lane pairs (project_wide) for wider classes, so
// the results are the decoder's own.
template <int D>
__global__ void __launch_bounds__(256) project_kernel(int d, long long count, const float *__restrict__ v,
                                                     float *__restrict__ z) {
    constexpr int L = class_lanes(D);
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long i = tid / L;
    if constexpr (L == 1) {
        if (i >= count) return;
        float vv[D];
#pragma unroll
        for (int k = 0; k < D; ++k) vv[k] = (k < d) ? v[i * d + k] : kPadV;
        const Proj pr = project_pp<D>(vv, d);
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (k < d) z[i * d + k] = proj_z(vv[k], pr, k);
    } else {
        // every lane takes part in the pair reductions; out-of-range pairs have d = 0
        constexpr int V = D / L;
        const int r = threadIdx.x & (L - 1);
        const int dd = i < count ? d : 0;
        const int dr = dd - r;
        float kap[V];
#pragma unroll
        for (int k = 0; k < V; ++k) kap[k] = (k * L < dr) ? v[i * d + k * L + r] : kPadV;
        unsigned th;
        const float beta = project_wide<D, L>(kap, dd, dr, r, th);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            if (k * L < dr) {
                float vk, zk;
                wide_vz(kap[k], (th >> k) & 1u, beta, vk, zk);
                z[i * d + k * L + r] = zk;
            }
        }
    }
}

}  // namespace lpdec

namespace lpdec {

// ---------------------------------------------------------------------------
// Mixed-code batches: one persistent launch decodes frames of several codes.
constexpr int kMaxMixedCodes = 8;
// CTA size bound of the mixed kernel: 896 threads, 72 registers a thread.
// The FAST kernel's inlined wide form spills 44-60 bytes there instead of
// 120-128 at 1024 threads (64 registers), and a C1056/C2640/C4000 batch runs
// in 313 ms instead of 354 ms.  (768 threads with 80 registers measured
// slower than 1024 threads in the general kernel.)  Codes whose tile is wider
// run fewer frames per CTA in a mixed launch.
#ifndef LPDEC_MIXED_MAX_THREADS
#define LPDEC_MIXED_MAX_THREADS 896
#endif
constexpr int kMixedMaxThreads = LPDEC_MIXED_MAX_THREADS;

// Kernel forms a code can run in (check degree class D, lanes per check L,
// regular variable degree DV or 0).
enum MixedKind : int {
    kK6R3 = 0, kK6 = 1, kK8R4 = 2, kK8 = 3, kK16 = 4, kK20 = 5, kK32 = 6,
    kK16R3 = 7, kK20R3 = 8, kK32R3 = 9,  // regular codes with degree-3 variables in the wide classes
    kNumKinds = 10
};

struct MixedCode {
    CodeView view;
    IterCfg cfg;         // per code: the stopping constants scale with its E
    int kind;            // MixedKind
    int groups;          // frames decoded at once by a CTA working on this code
    int group_threads;   // threads per frame
    int smem_per_group;  // bytes of one slice
    int off_x, off_red;  // slice layout
    int n_frames;        // frames of this code in the batch
    const int *frames;   // [n_frames] their frame ids
    int idx_off;         // regular codes: shared-memory offset where a CTA working on this code
                         // stages its 16-bit index block (after the slices), or -1
};

struct MixedArgs {
    int n_codes;
    MixedCode code[kMaxMixedCodes];
    int order[kMaxMixedCodes];     // codes by decreasing edges per frame: CTAs take them in this order
    const long long *offset;       // [F] element offset of frame f in llr, x_out and bits_out
    const float *llr;
    float *x_out;
    uint8_t *bits_out;
    int32_t *iters_out;
    uint8_t *cert_out;
    int *queues;                   // [n_codes] work-queue counters, zero at launch
};

}  // namespace lpdec

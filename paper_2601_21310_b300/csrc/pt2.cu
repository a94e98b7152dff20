// Epstein-Nesbet PT2 over the connected space (Eq. pt2_correction; Algorithm 1 step 4).
//
// For each hash bucket b (the high 32 bits of a SplitMix64 hash of the det, scaled to [0, B)):
//   1. emit (key x', H_x'y psi_y) for every excitation x' of every y in S with bucket(x') = b:
//      with B = 1 the position of every emission is fixed (y ascending, then canonical
//      excitation index), otherwise a count pass and a scan give them; the screened form
//      appends its emissions through per-warp staging in one traversal;
//   2. stable LSD radix sort by key (2 norb bits), so equal keys keep their emission order;
//   3. count the run heads per chunk and scan the counts (each chunk's first run index); each
//      warp then sums the runs that start in its chunk, lane by lane along runs, carrying the
//      open run across lanes and steps -> c(x') for every unique x': in FP64 in emission order
//      for the unscreened form (fixed positions, so a fixed order), in exact 128-bit fixed
//      point (fx128.cuh, independent of the order of the run's terms) for the screened form,
//      whose appended emissions have no fixed order; a per-unique pass sends members of S to
//      the internal term (c(x) is the off-diagonal part of (H_SS psi)_x) and turns the others
//      into c^2 / (D (E - H_x'x')) with H_x'x' from the Slater-Condon diagonal;
//   4. compensated sums of the external terms, and of the internal terms of the dets of S in
//      bucket b: r_x = H_xx psi_x + c(x) - E psi_x, r_x^2 / (D (E - H_xx)).
// D = psi.psi, compensated. Keys are the 2 norb-bit number (a << norb) | b: uint32 when
// 2 norb <= 32, uint64 when <= 64, two words above.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "excite.cuh"
#include "fx128.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

#define PT_THREADS 256
#define PT_WARPS (PT_THREADS / 32)

__device__ __forceinline__ bool in_bucket(uint64_t a, uint64_t b, uint64_t B, uint64_t bucket) {
    return B == 1 || det_bucket(a, b, B) == bucket;
}

__global__ void __launch_bounds__(PT_THREADS) k_pt2_count(ProblemDev P,
                                                           const ulonglong2* __restrict__ S,
                                                           int64_t nS, uint64_t B,
                                                           uint64_t bucket, int64_t* cnt) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const uint32_t nexc = (uint32_t)P.nexc;
    for (int64_t det = (int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * PT_WARPS) {
        ulonglong2 x = S[det];
        fill_ctx(P, x.x, x.y, ctx, lane);
        int c = 0;
        EnumPos q;
        q.cls = -1;
        const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                       o4 = o3 + (uint32_t)P.dBB;
        for (uint32_t e = lane; e < nexc; e += 32) {
            uint64_t a2, b2;
            step_key(P, T, *ctx, x.x, x.y, e, o2, o3, o4, q, a2, b2);
            c += in_bucket(a2, b2, B, bucket);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL_MASK, c, o);
        if (lane == 0) cnt[det] = c;
        __syncwarp();
    }
}

// All buckets in one pass: cnt[b * nS + det] = number of excitations of det in bucket b, from a
// per-warp shared-memory histogram over the B buckets (B <= PT_HIST_MAX).
#define PT_HIST_MAX 1024
__global__ void __launch_bounds__(PT_THREADS) k_pt2_count_all(ProblemDev P,
                                                               const ulonglong2* __restrict__ S,
                                                               int64_t nS, uint32_t B,
                                                               int64_t* __restrict__ cnt) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    uint32_t* hist = (uint32_t*)(smem + pair_table_bytes(P) + PT_WARPS * sizeof(DetCtx)) +
                     (threadIdx.x >> 5) * B;
    const int lane = threadIdx.x & 31;
    const uint32_t nexc = (uint32_t)P.nexc;
    const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                   o4 = o3 + (uint32_t)P.dBB;
    for (int64_t det = (int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * PT_WARPS) {
        ulonglong2 x = S[det];
        for (uint32_t k = lane; k < B; k += 32) hist[k] = 0;
        fill_ctx(P, x.x, x.y, ctx, lane);  // ends with __syncwarp
        EnumPos q;
        q.cls = -1;
        for (uint32_t e = lane; e < nexc; e += 32) {
            uint64_t a2, b2;
            step_key(P, T, *ctx, x.x, x.y, e, o2, o3, o4, q, a2, b2);
            atomicAdd(&hist[det_bucket(a2, b2, B)], 1u);
        }
        __syncwarp();
        for (uint32_t k = lane; k < B; k += 32) cnt[(int64_t)k * nS + det] = hist[k];
        __syncwarp();
    }
}

// offs == nullptr: every excitation is emitted at det * nexc + e (B = 1). With B > 1 only the
// key is decoded first; the full decode and the element are computed for in-bucket ones.
template <class K>
__global__ void __launch_bounds__(PT_THREADS, 4) k_pt2_emit(ProblemDev P,
                                                          const ulonglong2* __restrict__ S,
                                                          const double* __restrict__ psi,
                                                          int64_t nS, uint64_t B, uint64_t bucket,
                                                          const int64_t* __restrict__ offs,
                                                          K* __restrict__ keys,
                                                          double* __restrict__ vals) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    const AbTab abt = ab_tab_at(smem + pair_table_bytes(P) + PT_WARPS * sizeof(DetCtx) +
                                    (threadIdx.x >> 5) * ab_tab_bytes(P),
                                P);
    __shared__ uint32_t queue[PT_WARPS * 64];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const uint32_t nexc = (uint32_t)P.nexc;
    const int norb = P.norb;
    for (int64_t det = (int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * PT_WARPS) {
        ulonglong2 x = S[det];
        fill_ctx(P, x.x, x.y, ctx, lane);
        const double py = psi[det];
        int64_t run = offs ? offs[det] : det * (int64_t)nexc;
        if (B == 1) {
            const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                           o4 = o3 + (uint32_t)P.dBB;
            fill_ab_tab(P, *ctx, x.y, abt, lane);
            EnumPos q;
            q.cls = -1;
            AbState ab;
            ab.on = 0;
            for (uint32_t r0 = 0; r0 < nexc; r0 += 32) {
                const uint32_t e = r0 + lane;
                const bool take = e < nexc;
                const unsigned m = __ballot_sync(FULL_MASK, take);
                if (take) {
                    uint64_t a2, b2;
                    double hv;
                    if (e >= o4) {  // alpha-beta doubles from the tables
                        ab_fast_step(P, *ctx, x.x, e - o4, ab);
                        hv = ab_fast_element(P, abt, ab, b2);
                        a2 = ab.a2;
                    } else {
                        Exc ex;
                        step_exc(P, T, *ctx, x.x, x.y, e, o2, o3, o4, q, ex);
                        a2 = ex.a2;
                        b2 = ex.b2;
                        hv = exc_element(P, *ctx, ex);
                    }
                    const int64_t pos = run + __popc(m & lt);
                    keys[pos] = key_make<K>(a2, b2, norb);
                    vals[pos] = __dmul_rn(hv, py);
                }
                run += __popc(m);
            }
            __syncwarp();  // the tables are rewritten for the next configuration
        } else {
            // Only the key is decoded for every excitation. In-bucket indices are appended, in
            // canonical order, to a per-warp queue; each time it holds 32 the whole warp decodes
            // and evaluates them together, so the expensive part runs without divergence.
            uint32_t* q = queue + (threadIdx.x >> 5) * 64;
            uint32_t qn = 0;
            EnumPos pos;
            pos.cls = -1;
            const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                           o4 = o3 + (uint32_t)P.dBB;
            for (uint32_t r0 = 0; r0 < nexc; r0 += 32) {
                const uint32_t e = r0 + lane;
                bool take = false;
                if (e < nexc) {
                    uint64_t a2, b2;
                    step_key(P, T, *ctx, x.x, x.y, e, o2, o3, o4, pos, a2, b2);
                    take = in_bucket(a2, b2, B, bucket);
                }
                const unsigned m = __ballot_sync(FULL_MASK, take);
                if (take) q[qn + __popc(m & lt)] = e;
                qn += __popc(m);
                __syncwarp();
                if (qn >= 32 || (r0 + 32 >= nexc && qn > 0)) {
                    const uint32_t nt = qn < 32 ? qn : 32;
                    if ((uint32_t)lane < nt) {
                        Exc ex;
                        decode_exc(P, T, *ctx, x.x, x.y, q[lane], ex);
                        keys[run + lane] = key_make<K>(ex.a2, ex.b2, norb);
                        vals[run + lane] = __dmul_rn(exc_element(P, *ctx, ex), py);
                    }
                    run += nt;
                    const uint32_t rest = qn - nt;  // < 32
                    const uint32_t moved = (uint32_t)lane < rest ? q[32 + lane] : 0u;
                    __syncwarp();
                    if ((uint32_t)lane < rest) q[lane] = moved;
                    qn = rest;
                    __syncwarp();
                }
            }
            // a last partial batch can remain only if the final flush took exactly 32
            if (qn > 0) {
                if ((uint32_t)lane < qn) {
                    Exc ex;
                    decode_exc(P, T, *ctx, x.x, x.y, q[lane], ex);
                    keys[run + lane] = key_make<K>(ex.a2, ex.b2, norb);
                    vals[run + lane] = __dmul_rn(exc_element(P, *ctx, ex), py);
                }
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

// All buckets in one pass: excitation e of det goes to bucket b = det_bucket(x', B), at
// start[b] + offs[b * nS + det] + (its rank among det's excitations in bucket b, canonical
// order). Every excitation is decoded once (incrementally); per-warp counters in shared memory
// carry each bucket's rank across rounds of 32.
template <class K>
__global__ void __launch_bounds__(PT_THREADS) k_pt2_emit_all(ProblemDev P,
                                                              const ulonglong2* __restrict__ S,
                                                              const double* __restrict__ psi,
                                                              int64_t nS, uint32_t B,
                                                              const int64_t* __restrict__ start,
                                                              const int64_t* __restrict__ offs,
                                                              K* __restrict__ keys,
                                                              double* __restrict__ vals) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    const AbTab abt = ab_tab_at(smem + pair_table_bytes(P) + PT_WARPS * sizeof(DetCtx) +
                                    (threadIdx.x >> 5) * ab_tab_bytes(P),
                                P);
    uint32_t* ctr = (uint32_t*)(smem + pair_table_bytes(P) +
                                PT_WARPS * (sizeof(DetCtx) + ab_tab_bytes(P))) +
                    (threadIdx.x >> 5) * B;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const uint32_t nexc = (uint32_t)P.nexc;
    const int norb = P.norb;
    const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                   o4 = o3 + (uint32_t)P.dBB;
    for (int64_t det = (int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * PT_WARPS) {
        const ulonglong2 x = S[det];
        for (uint32_t k = lane; k < B; k += 32) ctr[k] = 0;
        fill_ctx(P, x.x, x.y, ctx, lane);  // ends with __syncwarp
        fill_ab_tab(P, *ctx, x.y, abt, lane);
        const double py = psi[det];
        EnumPos q;
        q.cls = -1;
        AbState ab;
        ab.on = 0;
        for (uint32_t r0 = 0; r0 < nexc; r0 += 32) {
            const uint32_t e = r0 + lane;
            const bool take = e < nexc;
            uint64_t a2 = 0, b2 = 0;
            double hv = 0.0;
            uint32_t b = 0xffffffffu;
            if (take) {
                if (e >= o4) {  // alpha-beta doubles from the tables
                    ab_fast_step(P, *ctx, x.x, e - o4, ab);
                    hv = ab_fast_element(P, abt, ab, b2);
                    a2 = ab.a2;
                } else {
                    Exc ex;
                    step_exc(P, T, *ctx, x.x, x.y, e, o2, o3, o4, q, ex);
                    a2 = ex.a2;
                    b2 = ex.b2;
                    hv = exc_element(P, *ctx, ex);
                }
                b = det_bucket(a2, b2, B);
            }
            const unsigned peers = __match_any_sync(FULL_MASK, b);
            uint32_t base = 0;
            if (take) {
                base = ctr[b];
                const int64_t pos = start[b] + offs[(int64_t)b * nS + det] + base +
                                    __popc(peers & lt);
                keys[pos] = key_make<K>(a2, b2, norb);
                vals[pos] = __dmul_rn(hv, py);
            }
            __syncwarp();
            if (take && lane == __ffs(peers) - 1) ctr[b] = base + __popc(peers);
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------------------------------
// Run reduction over the sorted (key, value) pairs. The pairs are cut into chunks of SEG_CHUNK;
// a chunk owns the runs of equal keys whose first element (head) lies in it.
//   k_seg_heads  number of heads per chunk (an exclusive scan gives each chunk's first run
//                index and the total number of unique keys);
//   k_seg_sum    one warp per chunk: from the chunk's first head to the first head at or past
//                the chunk's end, 32 x SEG_ITEMS elements per step (16-byte loads, SEG_ITEMS
//                consecutive elements per lane). Each lane adds its elements along runs (one FP64
//                add per element); the open run at each lane's end is passed to the next lane (a
//                segmented shuffle scan only when some lane holds no head) and, across steps, to
//                lane 0. The last element of a run writes the run's sum and key at the run index.
// Two forms: FP64 sums in element order (emissions at fixed positions), and exact 128-bit
// fixed-point sums converted to FP64 once per run (emissions appended in timing order), whose
// c(x') does not depend on the order of the run's terms.
// ------------------------------------------------------------------------------------------
#define SEG_CHUNK 2048
#define SEG_ITEMS 8

// SEG_ITEMS consecutive keys from i0 (a multiple of SEG_ITEMS); past `end` reads key zero
template <class K>
__device__ __forceinline__ void seg_load_keys(const K* __restrict__ keys, int64_t i0, int64_t end,
                                              K (&kk)[SEG_ITEMS]) {
    if (i0 + SEG_ITEMS <= end) {  // SEG_ITEMS * sizeof(K) is a multiple of 16 bytes
        constexpr int NV = SEG_ITEMS * (int)sizeof(K) / 16;
        uint4 t[NV];
        const uint4* src = reinterpret_cast<const uint4*>(keys + i0);
#pragma unroll
        for (int q = 0; q < NV; ++q) t[q] = __ldg(src + q);
        memcpy(kk, t, sizeof(t));
    } else {
#pragma unroll
        for (int j = 0; j < SEG_ITEMS; ++j) kk[j] = i0 + j < end ? keys[i0 + j] : key_zero<K>();
    }
}

__device__ __forceinline__ void seg_load_vals(const double* __restrict__ vals, int64_t i0,
                                              int64_t end, double (&v)[SEG_ITEMS]) {
    if (i0 + SEG_ITEMS <= end) {
        const double2* src = reinterpret_cast<const double2*>(vals + i0);
#pragma unroll
        for (int q = 0; q < SEG_ITEMS / 2; ++q) {
            const double2 t = __ldg(src + q);
            v[2 * q] = t.x;
            v[2 * q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < SEG_ITEMS; ++j) v[j] = i0 + j < end ? vals[i0 + j] : 0.0;
    }
}

template <class K>
__global__ void __launch_bounds__(256) k_seg_heads(const K* __restrict__ keys, int64_t n,
                                                   uint32_t* __restrict__ hc) {
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (n + SEG_CHUNK - 1) / SEG_CHUNK;
    for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; ch < nchunks;
         ch += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t c0 = ch * SEG_CHUNK, c1 = min(n, c0 + SEG_CHUNK);
        K last = c0 > 0 ? keys[c0 - 1] : key_zero<K>();
        uint32_t cnt = 0;
        for (int64_t b = c0; b < c1; b += 32 * SEG_ITEMS) {
            const int64_t i0 = b + (int64_t)SEG_ITEMS * lane;
            K kk[SEG_ITEMS];
            seg_load_keys(keys, i0, c1, kk);
            const K up = key_shfl_up(kk[SEG_ITEMS - 1], 1);
            K kp = lane == 0 ? last : up;
#pragma unroll
            for (int j = 0; j < SEG_ITEMS; ++j) {
                const int64_t i = i0 + j;
                cnt += (i < c1 && (i == 0 || kk[j] != kp)) ? 1u : 0u;
                kp = kk[j];
            }
            last = key_shfl(kk[SEG_ITEMS - 1], 31);
        }
        cnt = __reduce_add_sync(FULL_MASK, cnt);
        if (lane == 0) hc[ch] = cnt;
    }
}

// FP64 run sums in element order within a lane and lane order across lanes (the form for
// emissions at fixed positions, whose order is then fixed too)
template <class K>
__global__ void __launch_bounds__(256) k_seg_sum(const K* __restrict__ keys,
                                                 const double* __restrict__ vals,
                                                 const uint32_t* __restrict__ rbase, int64_t n,
                                                 double* __restrict__ cU, K* __restrict__ keyU) {
    const int lane = threadIdx.x & 31;
    constexpr int W = 32 * SEG_ITEMS;  // elements per warp step
    const unsigned lt = lanemask_lt();
    const int64_t nchunks = (n + SEG_CHUNK - 1) / SEG_CHUNK;
    for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; ch < nchunks;
         ch += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t c0 = ch * SEG_CHUNK, c1 = min(n, c0 + SEG_CHUNK);
        // first head inside [c0, c1)
        int64_t s0 = -1;
        for (int64_t b = c0; b < c1 && s0 < 0; b += 32) {
            const int64_t i = b + lane;
            const bool h = i < c1 && (i == 0 || keys[i] != keys[i - 1]);
            const unsigned m = __ballot_sync(FULL_MASK, h);
            if (m) s0 = b + __ffs(m) - 1;
        }
        if (s0 < 0) continue;  // every element continues a run owned by an earlier chunk
        const int64_t b0 = s0 & ~(int64_t)(SEG_ITEMS - 1);
        K kbefore = b0 > 0 ? keys[b0 - 1] : key_zero<K>();
        uint32_t ridx0 = rbase[ch];  // run index of the next head
        double carry = 0.0;          // the open run entering lane 0
        for (int64_t b = b0; b < n; b += W) {
            const int64_t i0 = b + (int64_t)SEG_ITEMS * lane;
            K kk[SEG_ITEMS];
            double v[SEG_ITEMS];
            seg_load_keys(keys, i0, n, kk);
            seg_load_vals(vals, i0, n, v);
            const K knext = b + W < n ? keys[b + W] : key_zero<K>();
            const K up = key_shfl_up(kk[SEG_ITEMS - 1], 1);
            // heads, and the first element that ends the walk (a head at or past c1, or past n)
            const int ja = (b == b0 && lane == 0) ? (int)(s0 - b0) : 0;
            unsigned hm = 0;
            int jstop = SEG_ITEMS;
            K kp = lane == 0 ? kbefore : up;
#pragma unroll
            for (int j = 0; j < SEG_ITEMS; ++j) {
                const int64_t i = i0 + j;
                const bool in = i < n;
                const bool h = in && (i == 0 || kk[j] != kp);
                if (h) hm |= 1u << j;
                if ((!in || (h && i >= c1)) && jstop == SEG_ITEMS) jstop = j;
                kp = kk[j];
            }
            const unsigned sm = __ballot_sync(FULL_MASK, jstop < SEG_ITEMS);
            const int L = sm ? __ffs(sm) - 1 : 32;
            const int jL = sm ? __shfl_sync(FULL_MASK, jstop, L) : 0;
            const int je = lane < L ? SEG_ITEMS : (lane == L ? jL : 0);  // active: [ja, je)
            const unsigned am = (je >= SEG_ITEMS ? 0xffu : ((1u << je) - 1u)) & ~((1u << ja) - 1u);
            hm &= am;
            // lane pass: running sums along runs, one FP64 add per element; fsum is the sum of
            // the lane's first segment (its elements before the lane's first head)
            double run = 0.0, tv[SEG_ITEMS], fsum = 0.0;
#pragma unroll
            for (int j = 0; j < SEG_ITEMS; ++j) {
                if ((hm >> j) & 1u) {
                    if ((hm & ((1u << j) - 1u)) == 0u) fsum = run;
                    run = v[j];
                } else if ((am >> j) & 1u) {
                    run = run + v[j];
                }
                tv[j] = run;
            }
            if (hm == 0u) fsum = run;
            const bool act = am != 0;
            const bool lh = hm != 0;
            const double lsum = act ? run : 0.0;
            // the open run entering this lane: from the previous lane, or a segmented scan when
            // some active lane holds no head (a run crosses whole lanes)
            double inc;
            double nextcarry;
            if (!__any_sync(FULL_MASK, act && !lh)) {
                const double prev = __shfl_up_sync(FULL_MASK, lsum, 1);
                inc = lane == 0 ? carry : prev;
                nextcarry = __shfl_sync(FULL_MASK, lsum, 31);
            } else {
                double sv = lsum;
                int sf = lh ? 1 : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double yv = __shfl_up_sync(FULL_MASK, sv, o);
                    const int yf = __shfl_up_sync(FULL_MASK, sf, o);
                    if (lane >= o && !sf) sv = yv + sv;
                    if (lane >= o) sf |= yf;
                }
                double ex = __shfl_up_sync(FULL_MASK, sv, 1);
                int exf = __shfl_up_sync(FULL_MASK, sf, 1);
                if (lane == 0) {
                    ex = 0.0;
                    exf = 0;
                }
                inc = exf ? ex : carry + ex;
                const double sv31 = __shfl_sync(FULL_MASK, sv, 31);
                const int sf31 = __shfl_sync(FULL_MASK, sf, 31);
                nextcarry = sf31 ? sv31 : carry + sv31;
            }
            // run index of each tail: heads before this lane (warp prefix) + heads up to it
            const uint32_t nh = (uint32_t)__popc(hm);
            uint32_t hpre = nh;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL_MASK, hpre, o);
                if (lane >= o) hpre += y;
            }
            const uint32_t htot = __shfl_sync(FULL_MASK, hpre, 31);
            hpre -= nh;
            // does the run at the lane's last active element end there?
            const int first_ends = (!act || (hm & 1u)) ? 1 : 0;
            const int next_first_ends = __shfl_down_sync(FULL_MASK, first_ends, 1);
            bool end_after;
            if (je < SEG_ITEMS) end_after = true;
            else if (lane < 31) end_after = next_first_ends != 0;
            else end_after = (b + W >= n) || (knext != kk[SEG_ITEMS - 1]);
            // the first segment's run continues one entering the lane: one add per lane
            const double first_total = inc + fsum;
#pragma unroll
            for (int j = 0; j < SEG_ITEMS; ++j) {
                if ((am >> j) & 1u) {
                    const bool tail = (j + 1 < je) ? ((hm >> (j + 1)) & 1u) != 0 : end_after;
                    if (tail) {
                        const unsigned upto = hm & ((2u << j) - 1u);  // heads at or before j
                        const uint32_t r = ridx0 + hpre + (uint32_t)__popc(upto) - 1u;
                        cU[r] = upto ? tv[j] : first_total;
                        keyU[r] = kk[j];
                    }
                }
            }
            ridx0 += htot;
            carry = nextcarry;
            kbefore = key_shfl(kk[SEG_ITEMS - 1], 31);
            if (L < 32) break;
        }
    }
}

// The same reduction with exact 128-bit fixed-point run sums (fx128.cuh): the form for
// emissions appended in timing order, whose run sums must not depend on the order of their
// terms. Converting each term costs integer instructions (the kernel is ALU-bound on this part,
// about twice the FP64 form's time), so the FP64 form is used wherever the order is fixed.
template <class K>
__global__ void __launch_bounds__(256) k_seg_sum_fx(const K* __restrict__ keys,
                                                 const double* __restrict__ vals,
                                                 const uint32_t* __restrict__ rbase, int64_t n,
                                                 const unsigned long long* __restrict__ vmax_bits,
                                                 double hoff_max, double run_max,
                                                 double* __restrict__ cU, K* __restrict__ keyU) {
    const int lane = threadIdx.x & 31;
    constexpr int W = 32 * SEG_ITEMS;  // elements per warp step
    // the fixed-point grid: every term is |H_x'y psi_y| <= hoff_max * max|psi| and a run has at
    // most run_max terms
    const double vmax = __dmul_ru(hoff_max, __longlong_as_double((long long)*vmax_bits));
    const bool finite = vmax <= 1.7976931348623157e308;
    const int F = fx_scale(finite ? vmax : 1.0, run_max);
    const int64_t nchunks = (n + SEG_CHUNK - 1) / SEG_CHUNK;
    for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; ch < nchunks;
         ch += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t c0 = ch * SEG_CHUNK, c1 = min(n, c0 + SEG_CHUNK);
        // first head inside [c0, c1)
        int64_t s0 = -1;
        for (int64_t b = c0; b < c1 && s0 < 0; b += 32) {
            const int64_t i = b + lane;
            const bool h = i < c1 && (i == 0 || keys[i] != keys[i - 1]);
            const unsigned m = __ballot_sync(FULL_MASK, h);
            if (m) s0 = b + __ffs(m) - 1;
        }
        if (s0 < 0) continue;  // every element continues a run owned by an earlier chunk
        const int64_t b0 = s0 & ~(int64_t)(SEG_ITEMS - 1);
        K kbefore = b0 > 0 ? keys[b0 - 1] : key_zero<K>();
        uint32_t ridx0 = rbase[ch];  // run index of the next head
        Fx128 carry = fx_zero();     // the open run entering lane 0
        for (int64_t b = b0; b < n; b += W) {
            const int64_t i0 = b + (int64_t)SEG_ITEMS * lane;
            K kk[SEG_ITEMS];
            double v[SEG_ITEMS];
            seg_load_keys(keys, i0, n, kk);
            seg_load_vals(vals, i0, n, v);
            const K knext = b + W < n ? keys[b + W] : key_zero<K>();
            const K up = key_shfl_up(kk[SEG_ITEMS - 1], 1);
            // heads, and the first element that ends the walk (a head at or past c1, or past n)
            const int ja = (b == b0 && lane == 0) ? (int)(s0 - b0) : 0;
            unsigned hm = 0;
            int jstop = SEG_ITEMS;
            K kp = lane == 0 ? kbefore : up;
#pragma unroll
            for (int j = 0; j < SEG_ITEMS; ++j) {
                const int64_t i = i0 + j;
                const bool in = i < n;
                const bool h = in && (i == 0 || kk[j] != kp);
                if (h) hm |= 1u << j;
                if ((!in || (h && i >= c1)) && jstop == SEG_ITEMS) jstop = j;
                kp = kk[j];
            }
            const unsigned sm = __ballot_sync(FULL_MASK, jstop < SEG_ITEMS);
            const int L = sm ? __ffs(sm) - 1 : 32;
            const int jL = sm ? __shfl_sync(FULL_MASK, jstop, L) : 0;
            const int je = lane < L ? SEG_ITEMS : (lane == L ? jL : 0);  // active: [ja, je)
            const unsigned am = (je >= SEG_ITEMS ? 0xffu : ((1u << je) - 1u)) & ~((1u << ja) - 1u);
            hm &= am;
            const bool act = am != 0;
            const bool lh = hm != 0;
            // run index of each tail: heads before this lane (warp prefix) + heads up to it
            const uint32_t nh = (uint32_t)__popc(hm);
            uint32_t hpre = nh;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL_MASK, hpre, o);
                if (lane >= o) hpre += y;
            }
            const uint32_t htot = __shfl_sync(FULL_MASK, hpre, 31);
            hpre -= nh;
            // does the run at the lane's last active element end there?
            const int first_ends = (!act || (hm & 1u)) ? 1 : 0;
            const int next_first_ends = __shfl_down_sync(FULL_MASK, first_ends, 1);
            bool end_after;
            if (je < SEG_ITEMS) end_after = true;
            else if (lane < 31) end_after = next_first_ends != 0;
            else end_after = (b + W >= n) || (knext != kk[SEG_ITEMS - 1]);
            // tails: active elements followed by a head (or by the end of the walk)
            const unsigned tm = am & ((hm >> 1) | (end_after ? (1u << (je - 1)) : 0u));
            // lane pass: running sums along runs, one exact integer add per element. A run that
            // starts in this lane is complete at its tail and written there; the lane's first
            // segment (its elements before its first head) continues a run entering the lane and
            // is finished after the scan below. fsum is that first segment's sum.
            Fx128 run = fx_zero(), fsum = fx_zero();
            bool tfirst = false;  // the first segment's run ends in this lane, at key kfirst
            K kfirst = key_zero<K>();
#pragma unroll
            for (int j = 0; j < SEG_ITEMS; ++j) {
                if ((am >> j) & 1u) {
                    const Fx128 fv = fx_from_double(v[j], F);
                    const bool head = (hm >> j) & 1u;
                    if (head && (hm & ((1u << j) - 1u)) == 0u) fsum = run;
                    run = head ? fv : fx_add(run, fv);
                    if ((tm >> j) & 1u) {
                        const unsigned upto = hm & ((2u << j) - 1u);  // heads at or before j
                        if (upto) {
                            const uint32_t r = ridx0 + hpre + (uint32_t)__popc(upto) - 1u;
                            cU[r] = finite ? fx_to_double(run, F) : vmax;
                            keyU[r] = kk[j];
                        } else {
                            tfirst = true;
                            kfirst = kk[j];
                        }
                    }
                }
            }
            if (hm == 0u) fsum = run;
            const Fx128 lsum = act ? run : fx_zero();
            // the open run entering this lane: from the previous lane, or a segmented scan when
            // some active lane holds no head (a run crosses whole lanes)
            Fx128 inc, nextcarry;
            if (!__any_sync(FULL_MASK, act && !lh)) {
                const Fx128 prev = fx_shfl_up(lsum, 1);
                inc = lane == 0 ? carry : prev;
                nextcarry = fx_shfl(lsum, 31);
            } else {
                Fx128 sv = lsum;
                int sf = lh ? 1 : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const Fx128 yv = fx_shfl_up(sv, o);
                    const int yf = __shfl_up_sync(FULL_MASK, sf, o);
                    if (lane >= o && !sf) sv = fx_add(yv, sv);
                    if (lane >= o) sf |= yf;
                }
                Fx128 ex = fx_shfl_up(sv, 1);
                int exf = __shfl_up_sync(FULL_MASK, sf, 1);
                if (lane == 0) {
                    ex = fx_zero();
                    exf = 0;
                }
                inc = exf ? ex : fx_add(carry, ex);
                const Fx128 sv31 = fx_shfl(sv, 31);
                const int sf31 = __shfl_sync(FULL_MASK, sf, 31);
                nextcarry = sf31 ? sv31 : fx_add(carry, sv31);
            }
            if (tfirst) {  // the first segment's run ends in this lane: one add
                const uint32_t r = ridx0 + hpre - 1u;
                cU[r] = finite ? fx_to_double(fx_add(inc, fsum), F) : vmax;
                keyU[r] = kfirst;
            }
            ridx0 += htot;
            carry = nextcarry;
            kbefore = key_shfl(kk[SEG_ITEMS - 1], 31);
            if (L < 32) break;
        }
    }
}

// bit pattern of max |psi| (non-negative doubles order like their bit patterns)
__global__ void k_absmax_bits(const double* __restrict__ x, int64_t n,
                              unsigned long long* __restrict__ out) {
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(fabs(x[i])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

template <class K>
__global__ void k_unique_terms(ProblemDev P, HashS H, const K* __restrict__ keyU,
                               const double* __restrict__ cU, int64_t nuniq,
                               const double* __restrict__ Dp, double E, double* __restrict__ cS,
                               double* __restrict__ eterm, unsigned long long* __restrict__ next,
                               uint32_t* __restrict__ ext_flag, int outside) {
    // outside != 0: every key is known to lie outside S (the screened emission leaves S out),
    // so no probe is needed
    const double D = *Dp;
    const int norb = P.norb;
    unsigned long long local = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nuniq;
         u += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a, b;
        key_split(keyU[u], norb, a, b);
        const double c = cU[u];
        const int32_t s = outside ? -1 : hash_lookup(H, a, b);
        if (ext_flag) ext_flag[u] = s >= 0 ? 0u : 1u;
        if (s >= 0) {
            cS[s] = c;
            eterm[u] = 0.0;
        } else {
            const double hxx = diag_element_bytes(P, a, b);
            eterm[u] = __ddiv_rn(__dmul_rn(c, c), __dmul_rn(D, __dsub_rn(E, hxx)));
            ++local;
        }
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(FULL_MASK, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(next, local);
}

// every stride-th configuration of S and its amplitude (the sample that sizes the screened
// single traversal)
__global__ void k_gather_stride(const ulonglong2* __restrict__ S, const double* __restrict__ psi,
                                int64_t ns, int64_t stride, ulonglong2* __restrict__ So,
                                double* __restrict__ po) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x) {
        So[i] = S[i * stride];
        po[i] = psi[i * stride];
    }
}

// the external unique set of one bucket, in key order: configuration and c(x')
template <class K>
__global__ void k_unique_out(const K* __restrict__ keyU, const double* __restrict__ cU,
                             const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                             int64_t nuniq, int norb, ulonglong2* __restrict__ dets_out,
                             double* __restrict__ c_out) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nuniq;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[u]) continue;
        uint64_t a, b;
        key_split(keyU[u], norb, a, b);
        dets_out[pos[u]] = make_ulonglong2(a, b);
        c_out[pos[u]] = cU[u];
    }
}

// cS[x] = sum over the excitations y of x that lie in S of <x|H|y> psi_y (the off-diagonal part
// of (H_SS psi)_x), by enumerating x's own connected set; one warp per x, lanes keep partial
// sums in canonical order, then a fixed shuffle tree. Used by the screened form, whose
// emissions leave out the configurations of S.
__global__ void __launch_bounds__(PT_THREADS) k_pt2_hss_psi(ProblemDev P, HashS H,
                                                             const ulonglong2* __restrict__ S,
                                                             const double* __restrict__ psi,
                                                             int64_t nS, double* __restrict__ cS) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const uint32_t nexc = (uint32_t)P.nexc;
    for (int64_t det = (int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * PT_WARPS) {
        const ulonglong2 x = S[det];
        fill_ctx(P, x.x, x.y, ctx, lane);
        double acc = 0.0;
        EnumPos q;
        q.cls = -1;
        const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                       o4 = o3 + (uint32_t)P.dBB;
        for (uint32_t e = lane; e < nexc; e += 32) {
            uint64_t a2, b2;
            step_key(P, T, *ctx, x.x, x.y, e, o2, o3, o4, q, a2, b2);
            const int32_t hit = hash_lookup(H, a2, b2);
            if (hit >= 0) {
                Exc ex;
                decode_exc(P, T, *ctx, x.x, x.y, e, ex);
                acc = __dadd_rn(acc, __dmul_rn(exc_element(P, *ctx, ex), psi[hit]));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(FULL_MASK, acc, o));
        if (lane == 0) cS[det] = acc;
        __syncwarp();
    }
}

__global__ void k_pt2_internal(ProblemDev P, const ulonglong2* __restrict__ S,
                               const double* __restrict__ psi, const double* __restrict__ cS,
                               int64_t nS, const double* __restrict__ Dp, double E, uint64_t B,
                               uint64_t bucket, double* __restrict__ eterm) {
    const double D = *Dp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nS;
         i += (int64_t)gridDim.x * blockDim.x) {
        ulonglong2 x = S[i];
        if (!in_bucket(x.x, x.y, B, bucket)) {
            eterm[i] = 0.0;
            continue;
        }
        double hxx = diag_element_impl(P, x.x, x.y);
        double vx = __dadd_rn(__dmul_rn(hxx, psi[i]), cS[i]);
        double r = __dsub_rn(vx, __dmul_rn(E, psi[i]));
        eterm[i] = __ddiv_rn(__dmul_rn(r, r), __dmul_rn(D, __dsub_rn(E, hxx)));
    }
}

// ------------------------------------------------------------------------------------------
// PT2 over a connected space whose unique set does not fit in device memory (hashed passes).
// Fine buckets fb(x') = det_hash(x') mod FB; a pass takes a contiguous range of fine buckets and
// accumulates every emission (x', H_x'y psi_y) of that range into a hash table of
// configurations in exact 128-bit fixed point (FxSlot: 128-bit CAS for the key, 64-bit atomics
// for the sum), so the table holds one slot per unique x' instead of one entry per emitted
// pair and the connected space is traversed once per pass. The table is then compacted, the
// unique keys sorted, and the sums reduced as any bucket is.
// ------------------------------------------------------------------------------------------
#define PT_FB 256
#define PT_HASHED_MIN_BUCKETS 8  // sorted buckets above which the hashed passes are used

// emitted pairs per fine bucket: per-warp shared-memory histograms over all of the warp's
// configurations, added to tot[PT_FB] at the end
__global__ void __launch_bounds__(PT_THREADS) k_pt2_fine_totals(ProblemDev P,
                                                                 const ulonglong2* __restrict__ S,
                                                                 int64_t nS,
                                                                 unsigned long long* __restrict__ tot) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    uint32_t* hist = (uint32_t*)(smem + pair_table_bytes(P) + PT_WARPS * sizeof(DetCtx)) +
                     (threadIdx.x >> 5) * PT_FB;
    const int lane = threadIdx.x & 31;
    const uint32_t nexc = (uint32_t)P.nexc;
    const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                   o4 = o3 + (uint32_t)P.dBB;
    for (uint32_t k = lane; k < PT_FB; k += 32) hist[k] = 0;
    __syncwarp();
    for (int64_t det = (int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * PT_WARPS) {
        ulonglong2 x = S[det];
        fill_ctx(P, x.x, x.y, ctx, lane);  // ends with __syncwarp
        EnumPos q;
        q.cls = -1;
        for (uint32_t e = lane; e < nexc; e += 32) {
            uint64_t a2, b2;
            step_key(P, T, *ctx, x.x, x.y, e, o2, o3, o4, q, a2, b2);
            atomicAdd(&hist[det_hash(a2, b2) % PT_FB], 1u);
        }
        __syncwarp();
    }
    for (uint32_t k = lane; k < PT_FB; k += 32)
        if (hist[k]) atomicAdd(&tot[k], (unsigned long long)hist[k]);
}

__global__ void k_fx_table_clear(FxSlot* __restrict__ t, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        t[i] = FxSlot{FX_EMPTY, FX_EMPTY, 0ull, 0ull};
}

// The emissions of the fine buckets [lo, hi) into the table (capacity mask + 1): only the key is
// decoded for every excitation; in-range ones are queued per warp and, 32 at a time, fully
// decoded, evaluated (H_x'y psi_y in FP64, as the emission kernels do), converted to fixed
// point on the grid 2^-F and added. A key that finds no slot within FX_PROBES probes sets
// *overflow (the pass is then repeated on a smaller range).
#define FX_PROBES 4096
__global__ void __launch_bounds__(PT_THREADS, 4) k_pt2_insert(ProblemDev P,
                                                            const ulonglong2* __restrict__ S,
                                                            const double* __restrict__ psi,
                                                            int64_t nS, uint32_t lo, uint32_t hi,
                                                            FxSlot* __restrict__ tab,
                                                            uint64_t mask, int F,
                                                            int* __restrict__ overflow) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    __shared__ uint32_t queue[PT_WARPS * 64];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const uint32_t nexc = (uint32_t)P.nexc;
    const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                   o4 = o3 + (uint32_t)P.dBB;
    uint32_t* q = queue + (threadIdx.x >> 5) * 64;
    for (int64_t det = (int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * PT_WARPS) {
        const ulonglong2 x = S[det];
        fill_ctx(P, x.x, x.y, ctx, lane);
        const double py = psi[det];
        // one batch of up to 32 queued excitations: decode, evaluate, add into the table
        auto insert_batch = [&](uint32_t nt) {
            if ((uint32_t)lane < nt) {
                Exc ex;
                decode_exc(P, T, *ctx, x.x, x.y, q[lane], ex);
                const Fx128 v = fx_from_double(__dmul_rn(exc_element(P, *ctx, ex), py), F);
                uint64_t slot = hash_slot(s_hash(ex.a2, ex.b2), mask);
                bool done = false;
                for (int it = 0; it < FX_PROBES && !done; ++it) {
                    unsigned long long oa, ob;
                    fx_cas_key(tab + slot, ex.a2, ex.b2, oa, ob);
                    if ((oa == FX_EMPTY && ob == FX_EMPTY) || (oa == ex.a2 && ob == ex.b2)) {
                        fx_atomic_add(tab + slot, v);
                        done = true;
                    } else {
                        slot = (slot + 1) & mask;
                    }
                }
                if (!done) atomicOr(overflow, 1);
            }
        };
        uint32_t qn = 0;
        EnumPos pos;
        pos.cls = -1;
        for (uint32_t r0 = 0; r0 < nexc; r0 += 32) {
            const uint32_t e = r0 + lane;
            bool take = false;
            if (e < nexc) {
                uint64_t a2, b2;
                step_key(P, T, *ctx, x.x, x.y, e, o2, o3, o4, pos, a2, b2);
                const uint32_t fb = (uint32_t)(det_hash(a2, b2) % PT_FB);
                take = fb >= lo && fb < hi;
            }
            const unsigned m = __ballot_sync(FULL_MASK, take);
            if (take) q[qn + __popc(m & lt)] = e;
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                insert_batch(32);
                const uint32_t rest = qn - 32;
                const uint32_t moved = (uint32_t)lane < rest ? q[32 + lane] : 0u;
                __syncwarp();
                if ((uint32_t)lane < rest) q[lane] = moved;
                qn = rest;
                __syncwarp();
            }
        }
        if (qn > 0) insert_batch(qn);
        __syncwarp();  // the queue and the context are rewritten for the next configuration
    }
}

// occupied slots -> (packed key, c(x')) in an order that depends on timing (sorted afterwards)
template <class K>
__global__ void k_fx_table_compact(const FxSlot* __restrict__ t, uint64_t n, int F, int norb,
                                   K* __restrict__ keys, double* __restrict__ vals,
                                   unsigned long long* __restrict__ cursor, uint64_t cap) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    for (uint64_t i0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~(uint64_t)31; i0 < n;
         i0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = i0 + lane;
        FxSlot sl = FxSlot{FX_EMPTY, FX_EMPTY, 0ull, 0ull};
        if (i < n) sl = t[i];
        const bool occ = !(sl.a == FX_EMPTY && sl.b == FX_EMPTY);
        const unsigned m = __ballot_sync(FULL_MASK, occ);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd(cursor, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL_MASK, base, 0);
        if (occ) {
            const uint64_t p = base + __popc(m & lt);
            if (p < cap) {
                keys[p] = key_make<K>(sl.a, sl.b, norb);
                vals[p] = fx_to_double(Fx128{sl.lo, sl.hi}, F);
            }
        }
    }
}

// the emission kernels also hold each warp's alpha-beta tables
static size_t pt_smem_emit(const ProblemDev& P) {
    return pair_table_bytes(P) + PT_WARPS * (sizeof(DetCtx) + ab_tab_bytes(P));
}
static size_t pt_smem(const ProblemDev& P) {
    return pair_table_bytes(P) + PT_WARPS * sizeof(DetCtx);
}
static unsigned pt_grid(int64_t nS) {
    int64_t g = (nS + PT_WARPS - 1) / PT_WARPS;
    if (g > 148 * 16) g = 148 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

// host-side compensated sum (bucket partials)
static double host_ksum(const std::vector<double>& v) {
    double s = 0, c = 0;
    for (double x : v) {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    return s + c;
}

// What every bucket's reduction needs besides its pairs.
struct Pt2Ctx {
    const HashS* H;
    double* cS;                      // device [nS]: c(x) of the members of S
    double* D_dev;                   // device: psi.psi
    unsigned long long* vmax_bits;   // device: bit pattern of max |psi|
    double run_max;                  // longest possible run (terms of one c(x'))
    double E_var;
    bool exact;                      // fixed-point run sums (screened emissions)
    // optional: the external unique set of the bucket (nqs_pt2_unique)
    bool uq_on;
    uint64_t* uq_dets;  // device [uq_cap][2] (may be null: size only)
    double* uq_c;       // device [uq_cap]
    int64_t uq_cap;
    int64_t uq_n;       // host: size of the set (written by pt2_reduce)
};

// sort, deduplicate and reduce one bucket's n emitted pairs (keys, vals; keys2 / vals2 are the
// sort's second buffers, n long), adding its external sum on the device
template <class K>
static int pt2_reduce(nqs_problem* p, K* keys, double* vals, K* keys2, double* vals2, int64_t n,
                      Pt2Ctx& cx, double* ext_dev, unsigned long long* nuniq_dev,
                      cudaStream_t s) {
    const ProblemDev& P = p->d;
    Scratch bs(p, s);
    if (sizeof(K) == 4)
        NQS_TRY(radix_sort_pairs32(p, bs, (uint32_t*&)keys, vals, (uint32_t*&)keys2, vals2, n,
                                   2 * P.norb, s));
    else if (sizeof(K) == 8)
        NQS_TRY(radix_sort_pairs(p, bs, (uint64_t*&)keys, vals, (uint64_t*&)keys2, vals2, n,
                                 2 * P.norb, s));
    else
        NQS_TRY(radix_sort_pairs128(p, bs, (Key128*&)keys, vals, (Key128*&)keys2, vals2, n,
                                    2 * P.norb, s));
    // heads per chunk and their exclusive scan (the chunks' first run indices)
    const int64_t nchunks = (n + SEG_CHUNK - 1) / SEG_CHUNK;
    uint32_t *hc, *rbase;
    NQS_TRY(bs.get(&hc, nchunks > 0 ? nchunks : 1));
    NQS_TRY(bs.get(&rbase, nchunks > 0 ? nchunks : 1));
    int64_t nuniq = 0;
    if (n > 0) {
        {
            ProfScope prof_(PROF_HEADS, s);
            k_seg_heads<K><<<grid_for(nchunks * 32, 256, 148 * 16), 256, 0, s>>>(keys, n, hc);
        }
        NQS_CK_LAUNCH();
        NQS_TRY(scan_exclusive_u32(p, bs, hc, rbase, nchunks, s));
        uint32_t last_base = 0, last_count = 0;
        NQS_CK(cudaMemcpyAsync(&last_base, rbase + nchunks - 1, 4, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaMemcpyAsync(&last_count, hc + nchunks - 1, 4, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        nuniq = (int64_t)last_base + last_count;
    }
    double *cU, *eterm;
    K* keyU;
    uint32_t *flag = nullptr, *pos = nullptr;
    NQS_TRY(bs.get(&cU, nuniq));
    NQS_TRY(bs.get(&keyU, nuniq));
    NQS_TRY(bs.get(&eterm, nuniq));
    if (cx.uq_on) {
        NQS_TRY(bs.get(&flag, nuniq));
        NQS_TRY(bs.get(&pos, nuniq));
    }
    if (nuniq > 0) {
        {
            ProfScope prof_(PROF_SEG_REDUCE, s);
            if (cx.exact)
                k_seg_sum_fx<K><<<grid_for(nchunks * 32, 256, 148 * 16), 256, 0, s>>>(
                    keys, vals, rbase, n, cx.vmax_bits, P.hoff_max, cx.run_max, cU, keyU);
            else
                k_seg_sum<K><<<grid_for(nchunks * 32, 256, 148 * 16), 256, 0, s>>>(
                    keys, vals, rbase, n, cU, keyU);
        }
        NQS_CK_LAUNCH();
        {
            ProfScope prof_(PROF_UNIQUE, s);
            k_unique_terms<K><<<grid_for(nuniq, 256), 256, 0, s>>>(
                P, *cx.H, keyU, cU, nuniq, cx.D_dev, cx.E_var, cx.cS, eterm, nuniq_dev, flag,
                cx.exact ? 1 : 0);
        }
        NQS_CK_LAUNCH();
    }
    if (cx.uq_on) {
        cx.uq_n = 0;
        if (nuniq > 0) {
            NQS_TRY(scan_exclusive_u32(p, bs, flag, pos, nuniq, s));
            uint32_t lp = 0, lf = 0;
            NQS_CK(cudaMemcpyAsync(&lp, pos + nuniq - 1, 4, cudaMemcpyDeviceToHost, s));
            NQS_CK(cudaMemcpyAsync(&lf, flag + nuniq - 1, 4, cudaMemcpyDeviceToHost, s));
            NQS_CK(cudaStreamSynchronize(s));
            cx.uq_n = (int64_t)lp + lf;
            if (cx.uq_dets && cx.uq_n <= cx.uq_cap) {
                k_unique_out<K><<<grid_for(nuniq, 256), 256, 0, s>>>(
                    keyU, cU, flag, pos, nuniq, P.norb, (ulonglong2*)cx.uq_dets, cx.uq_c);
                NQS_CK_LAUNCH();
            }
        }
    }
    NQS_TRY(ksum_f64(p, bs, eterm, nuniq, ext_dev, s));
    return NQS_OK;
}

// one bucket of the pipeline with key type K: emit its pairs, then reduce them
template <class K>
static int pt2_bucket(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                      int64_t B, int64_t b, const int64_t* offs, int64_t n, Pt2Ctx& cx,
                      double* ext_dev, unsigned long long* nuniq_dev, double eps,
                      cudaStream_t s) {
    const ProblemDev& P = p->d;
    Scratch bs(p, s);
    K *keys, *keys2;
    double *vals, *vals2;
    NQS_TRY(bs.get(&keys, n));
    NQS_TRY(bs.get(&vals, n));
    NQS_TRY(bs.get(&keys2, n));
    NQS_TRY(bs.get(&vals2, n));
    if (eps > 0.0) {
        NQS_TRY(hb_pt2_pass(p, *cx.H, dets, psi, nS, eps, (uint64_t)B, (uint64_t)b, nullptr, offs,
                            keys, vals, s));
    } else {
        {
            ProfScope prof_(PROF_PT2_EMIT, s);
            k_pt2_emit<K><<<pt_grid(nS), PT_THREADS, pt_smem_emit(P), s>>>(
                P, (const ulonglong2*)dets, psi, nS, (uint64_t)B, (uint64_t)b, offs, keys, vals);
        }
        NQS_CK_LAUNCH();
    }
    return pt2_reduce<K>(p, keys, vals, keys2, vals2, n, cx, ext_dev, nuniq_dev, s);
}

// The screened emissions of the whole connected space in one traversal, appended into buffers
// of cap pairs, then reduced as one bucket. *needed receives the number of pairs; when it
// exceeds cap nothing is reduced (the caller splits into buckets).
template <class K>
static int pt2_screened_append(nqs_problem* p, const uint64_t* dets, const double* psi,
                               int64_t nS, double eps, int64_t cap, Pt2Ctx& cx, double* ext_dev,
                               unsigned long long* nuniq_dev, int64_t* needed, cudaStream_t s) {
    Scratch bs(p, s);
    K* keys;
    double* vals;
    unsigned long long* cur;
    NQS_TRY(bs.get(&keys, cap));
    NQS_TRY(bs.get(&vals, cap));
    NQS_TRY(bs.get(&cur, 1));
    NQS_TRY(hb_pt2_append(p, *cx.H, dets, psi, nS, eps, keys, vals, cap, cur, s));
    unsigned long long n = 0;
    NQS_CK(cudaMemcpyAsync(&n, cur, sizeof n, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    *needed = (int64_t)n;
    if ((int64_t)n > cap) return NQS_OK;
    K* keys2;
    double* vals2;
    NQS_TRY(bs.get(&keys2, n));
    NQS_TRY(bs.get(&vals2, n));
    return pt2_reduce<K>(p, keys, vals, keys2, vals2, (int64_t)n, cx, ext_dev, nuniq_dev, s);
}

// The internal term of bucket b: r_x^2 / (D (E - H_xx)) over the dets of S in bucket b, summed
// into dev_scalars[2 + 2b] (zero without the internal term)
static int pt2_internal_bucket(nqs_problem* p, const uint64_t* dets, const double* psi,
                               const double* cS, int64_t nS, double* dev_scalars, double E_var,
                               int64_t B, int64_t b, double* eint, bool with_int,
                               cudaStream_t s) {
    if (!with_int) {
        NQS_CK(cudaMemsetAsync(dev_scalars + 2 + 2 * b, 0, sizeof(double), s));
        return NQS_OK;
    }
    k_pt2_internal<<<grid_for(nS, 256), 256, 0, s>>>(p->d, (const ulonglong2*)dets, psi, cS, nS,
                                                     dev_scalars, E_var, (uint64_t)B, (uint64_t)b,
                                                     eint);
    NQS_CK_LAUNCH();
    Scratch sc(p, s);
    return ksum_f64(p, sc, eint, nS, dev_scalars + 2 + 2 * b, s);
}

// All buckets resident at once (unscreened, counts of every bucket known): one emission pass
// writes each pair into its bucket's region (bucket regions start on 16-element boundaries), then
// the buckets are reduced one after another with one pair of sort buffers of the largest
// bucket's size. total_emitted receives the number of pairs.
template <class K>
static int pt2_resident(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                        int64_t B, const std::vector<int64_t>& nb, const int64_t* offs_all,
                        Pt2Ctx& cx, double* dev_scalars, unsigned long long* next_dev,
                        double* eint, bool with_int, int64_t* total_emitted, cudaStream_t s) {
    const ProblemDev& P = p->d;
    std::vector<int64_t> start(B);
    int64_t at = 0, nmax = 1;
    for (int64_t b = 0; b < B; ++b) {
        start[b] = at;
        at += (nb[b] + 15) & ~(int64_t)15;
        if (nb[b] > nmax) nmax = nb[b];
    }
    Scratch rs(p, s);
    K *keys, *keys2;
    double *vals, *vals2;
    int64_t* start_dev;
    NQS_TRY(rs.get(&keys, at > 0 ? at : 1));
    NQS_TRY(rs.get(&vals, at > 0 ? at : 1));
    NQS_TRY(rs.get(&keys2, nmax));
    NQS_TRY(rs.get(&vals2, nmax));
    NQS_TRY(rs.get(&start_dev, B));
    NQS_CK(cudaMemcpyAsync(start_dev, start.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice,
                           s));
    const size_t smem_all = pt_smem_emit(P) + (size_t)PT_WARPS * B * sizeof(uint32_t);
    if (smem_all > 48 * 1024)
        NQS_CK(cudaFuncSetAttribute(k_pt2_emit_all<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_all));
    {
        ProfScope prof_(PROF_PT2_EMIT, s);
        k_pt2_emit_all<K><<<pt_grid(nS), PT_THREADS, smem_all, s>>>(
            P, (const ulonglong2*)dets, psi, nS, (uint32_t)B, start_dev, offs_all, keys, vals);
    }
    NQS_CK_LAUNCH();
    *total_emitted = 0;
    for (int64_t b = 0; b < B; ++b) {
        *total_emitted += nb[b];
        NQS_TRY(pt2_reduce<K>(p, keys + start[b], vals + start[b], keys2, vals2, nb[b], cx,
                              dev_scalars + 1 + 2 * b, next_dev + b, s));
        NQS_TRY(pt2_internal_bucket(p, dets, psi, cx.cS, nS, dev_scalars, cx.E_var, B, b, eint,
                                    with_int, s));
    }
    return NQS_OK;
}

// Hashed passes over the fine buckets (see k_pt2_insert): each pass takes the next range of fine
// buckets whose estimated unique count fits the table (unique / emitted ratio: 0.3 until a pass
// has measured it, then the largest seen x 1.15), accumulates its emissions in the table,
// compacts and sorts the unique keys and reduces them (runs of one: the sums are final), adding
// the pass's external sum into dev_scalars[1 + 2 pass]. A pass whose table overflows is
// repeated on half its range. *passes and *total_emitted receive the pass count and the
// number of emitted pairs.
template <class K>
static int pt2_hashed(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                      Pt2Ctx& cx, double* dev_scalars, unsigned long long* next_dev,
                      int64_t nslots, double avail, int64_t chunk, int* passes,
                      int64_t* total_emitted, cudaStream_t s) {
    const ProblemDev& P = p->d;
    Scratch sc(p, s);
    // emitted pairs per fine bucket
    unsigned long long* tot_dev;
    NQS_TRY(sc.get(&tot_dev, PT_FB));
    NQS_CK(cudaMemsetAsync(tot_dev, 0, PT_FB * sizeof(unsigned long long), s));
    const size_t smem_t = pt_smem(P) + (size_t)PT_WARPS * PT_FB * sizeof(uint32_t);
    if (smem_t > 48 * 1024)
        NQS_CK(cudaFuncSetAttribute(k_pt2_fine_totals, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_t));
    {
        ProfScope prof_(PROF_PT2_COUNT, s);
        k_pt2_fine_totals<<<pt_grid(nS), PT_THREADS, smem_t, s>>>(P, (const ulonglong2*)dets, nS,
                                                                  tot_dev);
    }
    NQS_CK_LAUNCH();
    std::vector<unsigned long long> tot(PT_FB);
    unsigned long long vbits = 0;
    NQS_CK(cudaMemcpyAsync(tot.data(), tot_dev, PT_FB * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaMemcpyAsync(&vbits, cx.vmax_bits, sizeof vbits, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    // the fixed-point grid (as k_seg_sum_fx chooses it)
    double vmax;
    memcpy(&vmax, &vbits, sizeof vmax);
    vmax *= P.hoff_max * (1.0 + 1e-15);
    int F = 100;
    if (vmax > 0.0 && vmax < 1e300) {
        int k;
        frexp(vmax * cx.run_max, &k);
        F = 125 - k;
    }
    // table capacity: the table (32 B per slot) and the compacted keys (key + value per unique,
    // 0.75 per slot) during compaction; then key and value twice for the sort plus the per-unique
    // arrays of the reduction (key + 16 B), at most 0.75 of the slots
    const double kb = (double)sizeof(K);
    const double per_slot = fmax(32.0 + 0.75 * (kb + 8.0), 0.75 * (3.0 * kb + 32.0));
    double cmax = 0.8 * avail / per_slot;
    if (chunk > 0 && (double)chunk < cmax) cmax = (double)chunk;  // the caller's cap
    uint64_t C = 1024;
    while ((double)(C * 2) <= cmax) C *= 2;
    const double ucap = 0.75 * (double)C;
    const size_t smem_i = pt_smem(P);
    if (smem_i > 48 * 1024)
        NQS_CK(cudaFuncSetAttribute(k_pt2_insert, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_i));
    double ratio = 0.3;
    int pass = 0;
    *total_emitted = 0;
    uint32_t lo = 0;
    while (lo < PT_FB) {
        // the next range: fine buckets while the estimated unique count fits
        uint32_t hi = lo;
        double pairs = 0.0;
        while (hi < PT_FB && (hi == lo || (pairs + (double)tot[hi]) * ratio <= ucap)) {
            pairs += (double)tot[hi];
            ++hi;
        }
        if (pass >= nslots) {
            nqs_record_message("nqs_pt2: more hashed passes than result slots");
            return NQS_ERR_UNSUPPORTED;
        }
        Scratch ps(p, s);
        FxSlot* tab;
        int* ovf;
        unsigned long long* cur;
        NQS_TRY(ps.get(&tab, C));
        NQS_TRY(ps.get(&ovf, 1));
        NQS_TRY(ps.get(&cur, 1));
        k_fx_table_clear<<<grid_for((int64_t)C, 256), 256, 0, s>>>(tab, C);
        NQS_CK_LAUNCH();
        NQS_CK(cudaMemsetAsync(ovf, 0, sizeof(int), s));
        NQS_CK(cudaMemsetAsync(cur, 0, sizeof(unsigned long long), s));
        {
            ProfScope prof_(PROF_PT2_EMIT, s);
            k_pt2_insert<<<pt_grid(nS), PT_THREADS, smem_i, s>>>(P, (const ulonglong2*)dets, psi, nS,
                                                                 lo, hi, tab, C - 1, F, ovf);
        }
        NQS_CK_LAUNCH();
        int ovh = 0;
        NQS_CK(cudaMemcpyAsync(&ovh, ovf, sizeof ovh, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        if (ovh) {
            if (hi - lo == 1) {
                nqs_record_message("nqs_pt2: one fine bucket's unique set exceeds the table");
                return NQS_ERR_OOM;
            }
            ratio *= 2.0;  // plan again on a smaller range
            continue;
        }
        // compact into arrays of the table's occupancy bound, then free the table
        const uint64_t ucapn = (uint64_t)ucap + 1024;
        K *keys, *keys2;
        double *vals, *vals2;
        Scratch rs(p, s);
        NQS_TRY(rs.get(&keys, ucapn));
        NQS_TRY(rs.get(&vals, ucapn));
        k_fx_table_compact<K><<<grid_for((int64_t)C, 256), 256, 0, s>>>(tab, C, F, P.norb, keys,
                                                                          vals, cur, ucapn);
        NQS_CK_LAUNCH();
        unsigned long long nu = 0;
        NQS_CK(cudaMemcpyAsync(&nu, cur, sizeof nu, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        if (nu > ucapn) {  // fuller than planned: everything is in the table, but not compacted
            ratio = fmax(ratio * 2.0, (double)nu / fmax(pairs, 1.0) * 1.15);
            continue;
        }
        ps.release();  // the table: its memory serves the sort
        NQS_TRY(rs.get(&keys2, nu));
        NQS_TRY(rs.get(&vals2, nu));
        NQS_TRY(pt2_reduce<K>(p, keys, vals, keys2, vals2, (int64_t)nu, cx,
                              dev_scalars + 1 + 2 * pass, next_dev + pass, s));
        NQS_CK(cudaMemsetAsync(dev_scalars + 2 + 2 * pass, 0, sizeof(double), s));
        *total_emitted += (int64_t)pairs;
        ratio = fmax(pass == 0 ? 0.0 : ratio / 1.15, (double)nu / fmax(pairs, 1.0)) * 1.15;
        ++pass;
        lo = hi;
    }
    *passes = pass;
    return NQS_OK;
}

// optional output of nqs_pt2_unique: the external unique set of one bucket
struct UniqReq {
    int64_t bucket;
    uint64_t* dets;
    double* c;
    int64_t cap;
    int64_t n;  // out
};

static int pt2_impl(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                    double E_var, const nqs_csr* hss, const nqs_opts* opts, double* out,
                    double* bucket_partials, cudaStream_t stream, UniqReq* uq);

extern "C" int nqs_pt2(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                       double E_var, const nqs_opts* opts, double* out, double* bucket_partials,
                       nqs_stream_t stream) {
    return pt2_impl(p, dets, psi, nS, E_var, nullptr, opts, out, bucket_partials,
                    (cudaStream_t)stream, nullptr);
}

extern "C" int nqs_pt2_hss(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                           double E_var, const nqs_csr* hss, const nqs_opts* opts, double* out,
                           double* bucket_partials, nqs_stream_t stream) {
    if (!hss || hss->n_rows != nS || !hss->row_ptr || !hss->col || !hss->val) return NQS_ERR_ARG;
    return pt2_impl(p, dets, psi, nS, E_var, hss, opts, out, bucket_partials,
                    (cudaStream_t)stream, nullptr);
}

static int pt2_unique_impl(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                           double eps, int buckets, int bucket, uint64_t* dets_out,
                           double* c_out, int64_t capacity, int64_t* n_unique,
                           nqs_stream_t stream) {
    if (!p || !n_unique || buckets < 1 || bucket < 0 || bucket >= buckets || capacity < 0)
        return NQS_ERR_ARG;
    if (capacity > 0 && (!dets_out || !c_out || (((uintptr_t)dets_out) & 15))) return NQS_ERR_ARG;
    nqs_opts o;
    nqs_opts_default(&o);
    o.buckets = buckets;
    o.validate = 0;
    o.eps_pt2 = eps;
    UniqReq uq{bucket, dets_out, c_out, capacity, 0};
    double res[5];
    const int st = pt2_impl(p, dets, psi, nS, 0.0, nullptr, &o, res, nullptr,
                            (cudaStream_t)stream, &uq);
    *n_unique = uq.n;
    if (st < 0) return st;
    if (uq.n > capacity) {
        nqs_record_message("nqs_pt2_unique: capacity smaller than the unique set; *n_unique holds "
                           "the size needed");
        return NQS_ERR_ARG;
    }
    return NQS_OK;
}

extern "C" int nqs_pt2_unique(nqs_problem* p, const uint64_t* dets, const double* psi,
                              int64_t nS, int buckets, int bucket, uint64_t* dets_out,
                              double* c_out, int64_t capacity, int64_t* n_unique,
                              nqs_stream_t stream) {
    return pt2_unique_impl(p, dets, psi, nS, 0.0, buckets, bucket, dets_out, c_out, capacity,
                           n_unique, stream);
}

extern "C" int nqs_pt2_unique_screened(nqs_problem* p, const uint64_t* dets, const double* psi,
                                       int64_t nS, double eps_pt2, int buckets, int bucket,
                                       uint64_t* dets_out, double* c_out, int64_t capacity,
                                       int64_t* n_unique, nqs_stream_t stream) {
    if (!(eps_pt2 > 0.0) || !(eps_pt2 < INFINITY)) return NQS_ERR_ARG;
    return pt2_unique_impl(p, dets, psi, nS, eps_pt2, buckets, bucket, dets_out, c_out, capacity,
                           n_unique, stream);
}

static int pt2_impl(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                    double E_var, const nqs_csr* hss, const nqs_opts* opts, double* out,
                    double* bucket_partials, cudaStream_t stream, UniqReq* uq) {
    if (!p || !dets || !psi || !out || nS <= 0) return NQS_ERR_ARG;
    if (((uintptr_t)dets) & 15) return NQS_ERR_ARG;
    if (nS >= ((int64_t)1 << 31)) return NQS_ERR_UNSUPPORTED;
    cudaStream_t s = stream;
    if (opts && opts->buckets <= 0 && bucket_partials) return NQS_ERR_ARG;
    nqs_opts def;
    if (!opts) {
        nqs_opts_default(&def);
        opts = &def;
    }
    const double eps = opts->eps_pt2;
    if (!(eps >= 0.0)) return NQS_ERR_ARG;
    const bool screened = eps > 0.0;
    int64_t B = opts->buckets;
    Scratch sc(p, s);
    if (opts->validate) NQS_TRY(validate_dets(p, sc, dets, nS, true, s));
    HashS H;
    NQS_TRY(hash_build(p, sc, dets, nS, &H, s));
    const ProblemDev& P = p->d;
    size_t smem = pt_smem(P);
    if (smem > 48 * 1024)
        NQS_CK(cudaFuncSetAttribute(k_pt2_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    const size_t sme = pt_smem_emit(P);
    if (sme > 48 * 1024) {
        NQS_CK(cudaFuncSetAttribute(k_pt2_emit<uint32_t>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sme));
        NQS_CK(cudaFuncSetAttribute(k_pt2_emit<uint64_t>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sme));
        NQS_CK(cudaFuncSetAttribute(k_pt2_emit<Key128>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sme));
    }
    const int kbits = 2 * P.norb;  // 32-bit, 64-bit or two-word keys
    const double kb = kbits <= 32 ? 4.0 : (kbits <= 64 ? 8.0 : 16.0);
    // device memory available to this call: free memory plus what the library's pool holds
    // unused
    auto avail_bytes = [&](double* av) -> int {
        size_t fr = 0, tot = 0;
        NQS_CK(cudaMemGetInfo(&fr, &tot));
        uint64_t reserved = 0, used = 0;
        NQS_CK(cudaMemPoolGetAttribute(p->pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
        NQS_CK(cudaMemPoolGetAttribute(p->pool, cudaMemPoolAttrUsedMemCurrent, &used));
        *av = (double)fr + (double)(reserved > used ? reserved - used : 0);
        return NQS_OK;
    };

    bool hashed = false;
    if (!screened && B <= 0) {
        // automatic: enough buckets that one bucket's pairs (keys and values twice, plus 8 bytes
        // per pair toward the per-unique arrays) use at most half of the free device memory,
        // and stay below 2^31
        double av = 0;
        NQS_TRY(avail_bytes(&av));
        double capb = 0.5 * av / (2.0 * (kb + 8.0) + 8.0);
        if (capb > 2147483647.0) capb = 2147483647.0;
        if (opts->chunk > 0 && (double)opts->chunk < capb) capb = (double)opts->chunk;
        B = (int64_t)ceil((double)nS * (double)P.nexc / capb);
        if (B < 1) B = 1;
        // when the sorted buckets would traverse the connected space many times, accumulate
        // into hash tables of unique configurations instead (one traversal per pass, memory per
        // unique x' rather than per emitted pair)
        hashed = B > PT_HASHED_MIN_BUCKETS && !uq;
    }
    // per-bucket slots: the bucket count is known here, except for the automatic screened form
    // (one bucket unless its single traversal overflows; at most 1024 then)
    const int64_t nslots = B > 1024 ? B : 1024;
    double* dev_scalars;  // [0] = D, then per bucket (ext, int)
    NQS_TRY(sc.get(&dev_scalars, 1 + 2 * nslots));
    unsigned long long* next_dev;
    NQS_TRY(sc.get(&next_dev, nslots));
    unsigned long long* vmax_bits;
    NQS_TRY(sc.get(&vmax_bits, 1));
    NQS_CK(cudaMemsetAsync(next_dev, 0, nslots * sizeof(unsigned long long), s));
    NQS_CK(cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned long long), s));
    NQS_TRY(kdot2_f64(p, sc, psi, psi, nS, dev_scalars, s));  // dev_scalars[0] = psi.psi
    k_absmax_bits<<<grid_for(nS, 256, 148 * 4), 256, 0, s>>>(psi, nS, vmax_bits);
    NQS_CK_LAUNCH();
    double* cS;
    NQS_TRY(sc.get(&cS, nS));
    NQS_CK(cudaMemsetAsync(cS, 0, nS * sizeof(double), s));
    double* eint;
    NQS_TRY(sc.get(&eint, nS));
    Pt2Ctx cx{&H, cS, dev_scalars, vmax_bits,
              (double)(nS < P.nexc ? nS : P.nexc), E_var, screened, uq != nullptr,
              uq ? uq->dets : nullptr, uq ? uq->c : nullptr, uq ? uq->cap : 0, 0};

    if (screened && opts->internal_pt2 && hss) {
        // the screened emissions leave S out: the internal term takes the off-diagonal part of
        // H_SS psi from the caller's H_SS
        NQS_TRY(csr_spmv_offdiag(hss, psi, cS, s));
    } else if (screened && opts->internal_pt2) {
        // ... or from the connected sets of S, enumerated again
        if (smem > 48 * 1024)
            NQS_CK(cudaFuncSetAttribute(k_pt2_hss_psi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
        k_pt2_hss_psi<<<pt_grid(nS), PT_THREADS, smem, s>>>(P, H, (const ulonglong2*)dets, psi,
                                                             nS, cS);
        NQS_CK_LAUNCH();
    }

    int64_t total_emitted = 0;
    bool done = false;
    if (hashed) {
        double av = 0;
        NQS_TRY(avail_bytes(&av));
        int passes = 0;
        int st = kbits <= 32 ? pt2_hashed<uint32_t>(p, dets, psi, nS, cx, dev_scalars, next_dev,
                                                    nslots, av, opts->chunk, &passes, &total_emitted, s)
               : kbits <= 64 ? pt2_hashed<uint64_t>(p, dets, psi, nS, cx, dev_scalars, next_dev,
                                                    nslots, av, opts->chunk, &passes, &total_emitted, s)
                             : pt2_hashed<Key128>(p, dets, psi, nS, cx, dev_scalars, next_dev,
                                                  nslots, av, opts->chunk, &passes, &total_emitted, s);
        NQS_TRY(st);
        B = passes;
        // the internal term over all of S once every pass has filled its c(x) of S
        NQS_TRY(pt2_internal_bucket(p, dets, psi, cS, nS, dev_scalars, E_var, 1, 0, eint,
                                    opts->internal_pt2 != 0, s));
        done = true;
    }
    if (screened && B <= 0) {
        // automatic: one traversal appending into buffers sized from a counted sample of S
        // (every stride-th configuration, x1.5 + 2^16), at most what memory allows (pairs, sort
        // buffers and per-unique arrays: 3 key widths + 36 bytes per pair, 90% of what is
        // available). The traversal counts every pair, so one that overflows is repeated with
        // the exact size when that fits; otherwise the emissions are split into counted buckets.
        double av = 0;
        NQS_TRY(avail_bytes(&av));
        double memcap = 0.9 * av / (3.0 * kb + 36.0);
        if (memcap > 4294967295.0) memcap = 4294967295.0;
        const int64_t stride = nS > 4096 ? nS / 4096 : 1;
        const int64_t ns = (nS + stride - 1) / stride;
        double est;
        {
            Scratch es(p, s);
            uint64_t* ds;
            double* ps;
            int64_t *c1, *o1, *t1;
            NQS_TRY(es.get(&ds, 2 * ns));
            NQS_TRY(es.get(&ps, ns));
            NQS_TRY(es.get(&c1, ns));
            NQS_TRY(es.get(&o1, ns));
            NQS_TRY(es.get(&t1, 1));
            k_gather_stride<<<grid_for(ns, 256), 256, 0, s>>>((const ulonglong2*)dets, psi, ns,
                                                               stride, (ulonglong2*)ds, ps);
            NQS_CK_LAUNCH();
            NQS_TRY(hb_pt2_pass(p, H, ds, ps, ns, eps, 1, 0, c1, nullptr, nullptr, nullptr, s));
            NQS_TRY(scan_exclusive_i64(p, es, c1, o1, ns, t1, s));
            int64_t tot = 0;
            NQS_CK(cudaMemcpyAsync(&tot, t1, sizeof tot, cudaMemcpyDeviceToHost, s));
            NQS_CK(cudaStreamSynchronize(s));
            est = (double)tot * ((double)nS / (double)ns);
        }
        double capd = fmin(1.5 * est + 65536.0, (double)nS * (double)P.nexc);
        capd = fmin(capd, memcap);
        int64_t cap = (int64_t)capd;
        int64_t needed = 0;
        for (int attempt = 0; attempt < 2 && !done; ++attempt) {
            int st = kbits <= 32
                         ? pt2_screened_append<uint32_t>(p, dets, psi, nS, eps, cap, cx,
                                                         dev_scalars + 1, next_dev, &needed, s)
                     : kbits <= 64
                         ? pt2_screened_append<uint64_t>(p, dets, psi, nS, eps, cap, cx,
                                                         dev_scalars + 1, next_dev, &needed, s)
                         : pt2_screened_append<Key128>(p, dets, psi, nS, eps, cap, cx,
                                                       dev_scalars + 1, next_dev, &needed, s);
            NQS_TRY(st);
            if (needed <= cap) {
                B = 1;
                total_emitted = needed;
                NQS_TRY(pt2_internal_bucket(p, dets, psi, cS, nS, dev_scalars, E_var, 1, 0, eint,
                                            opts->internal_pt2 != 0, s));
                done = true;
            } else if ((double)needed <= memcap) {
                cap = needed;  // the exact size: one more traversal
            } else {
                B = (int64_t)ceil((double)needed / memcap);
                break;
            }
        }
    }
    if (B > nslots) {
        nqs_record_message("nqs_pt2: the screened emissions need more than 1024 buckets; raise "
                           "eps_pt2 or pass opts->buckets");
        return NQS_ERR_UNSUPPORTED;
    }
    if (uq && (uq->bucket >= B)) return NQS_ERR_ARG;
    int64_t* cnt = nullptr;
    int64_t* offs = nullptr;
    int64_t* total_dev = nullptr;
    // one counting pass for every bucket when the B x nS count table stays below 2 GiB
    const bool count_all = !done && !screened && B > 1 && B <= PT_HIST_MAX &&
                           (double)nS * (double)B * sizeof(int64_t) <= 2147483648.0;
    if (!done && (B > 1 || screened)) {
        NQS_TRY(sc.get(&cnt, count_all ? (size_t)nS * B : (size_t)nS));
        NQS_TRY(sc.get(&offs, nS));
        NQS_TRY(sc.get(&total_dev, 1));
    }
    if (count_all) {
        const size_t smem_all = smem + (size_t)PT_WARPS * B * sizeof(uint32_t);
        if (smem_all > 48 * 1024)
            NQS_CK(cudaFuncSetAttribute(k_pt2_count_all,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_all));
        {
            ProfScope prof_(PROF_PT2_COUNT, s);
            k_pt2_count_all<<<pt_grid(nS), PT_THREADS, smem_all, s>>>(
                P, (const ulonglong2*)dets, nS, (uint32_t)B, cnt);
        }
        NQS_CK_LAUNCH();
    }
    const int64_t cap = opts->chunk > 0 ? opts->chunk : ((int64_t)1 << 32) - 1;
    if (count_all && !uq) {
        // every bucket's pairs resident at once when they fit: per-bucket offsets, then one
        // emission pass instead of one decoding pass over all excitations per bucket
        int64_t* offs_all;
        int64_t* nb_dev;
        NQS_TRY(sc.get(&offs_all, (size_t)nS * B));
        NQS_TRY(sc.get(&nb_dev, B));
        for (int64_t b = 0; b < B; ++b) {
            Scratch ts(p, s);
            NQS_TRY(scan_exclusive_i64(p, ts, cnt + (size_t)b * nS, offs_all + (size_t)b * nS,
                                       nS, nb_dev + b, s));
        }
        std::vector<int64_t> nb(B);
        NQS_CK(cudaMemcpyAsync(nb.data(), nb_dev, B * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        double tot = 0.0, nmax = 0.0;
        bool fits_sort = true;
        for (int64_t b = 0; b < B; ++b) {
            tot += (double)nb[b] + 16.0;
            nmax = fmax(nmax, (double)nb[b]);
            if (nb[b] > cap) fits_sort = false;
        }
        // pairs of all buckets + one pair of sort buffers + the largest bucket's unique arrays
        const double need = tot * (kb + 8.0) + nmax * (kb + 8.0) + nmax * (kb + 16.0);
        double av = 0;
        NQS_TRY(avail_bytes(&av));
        if (fits_sort && need <= 0.9 * av) {
            done = true;
            const bool wi = opts->internal_pt2 != 0;
            int st = kbits <= 32
                         ? pt2_resident<uint32_t>(p, dets, psi, nS, B, nb, offs_all, cx,
                                                  dev_scalars, next_dev, eint, wi,
                                                  &total_emitted, s)
                     : kbits <= 64
                         ? pt2_resident<uint64_t>(p, dets, psi, nS, B, nb, offs_all, cx,
                                                  dev_scalars, next_dev, eint, wi,
                                                  &total_emitted, s)
                         : pt2_resident<Key128>(p, dets, psi, nS, B, nb, offs_all, cx,
                                                dev_scalars, next_dev, eint, wi, &total_emitted,
                                                s);
            NQS_TRY(st);
        }
    }
    for (int64_t b = 0; b < B && !done; ++b) {
        if (uq && b != uq->bucket) {
            NQS_CK(cudaMemsetAsync(dev_scalars + 1 + 2 * b, 0, 2 * sizeof(double), s));
            continue;
        }
        int64_t n;
        if (B == 1 && !screened) {
            n = nS * P.nexc;
        } else {
            Scratch cs(p, s);
            if (screened) {
                NQS_TRY(hb_pt2_pass(p, H, dets, psi, nS, eps, (uint64_t)B, (uint64_t)b, cnt,
                                    nullptr, nullptr, nullptr, s));
            } else if (!count_all) {
                {
                    ProfScope prof_(PROF_PT2_COUNT, s);
                    k_pt2_count<<<pt_grid(nS), PT_THREADS, smem, s>>>(
                        P, (const ulonglong2*)dets, nS, (uint64_t)B, (uint64_t)b, cnt);
                }
                NQS_CK_LAUNCH();
            }
            NQS_TRY(scan_exclusive_i64(p, cs, count_all ? cnt + (size_t)b * nS : cnt, offs, nS,
                                       total_dev, s));
            NQS_CK(cudaMemcpyAsync(&n, total_dev, sizeof n, cudaMemcpyDeviceToHost, s));
            NQS_CK(cudaStreamSynchronize(s));
        }
        if (n > cap) return NQS_ERR_OOM;  // more buckets needed
        total_emitted += n;
        const int64_t* o = (B == 1 && !screened) ? nullptr : offs;
        int st = kbits <= 32
                     ? pt2_bucket<uint32_t>(p, dets, psi, nS, B, b, o, n, cx,
                                            dev_scalars + 1 + 2 * b, next_dev + b, eps, s)
                 : kbits <= 64
                     ? pt2_bucket<uint64_t>(p, dets, psi, nS, B, b, o, n, cx,
                                            dev_scalars + 1 + 2 * b, next_dev + b, eps, s)
                     : pt2_bucket<Key128>(p, dets, psi, nS, B, b, o, n, cx,
                                          dev_scalars + 1 + 2 * b, next_dev + b, eps, s);
        NQS_TRY(st);
        NQS_TRY(pt2_internal_bucket(p, dets, psi, cS, nS, dev_scalars, E_var, B, b, eint,
                                    opts->internal_pt2 != 0, s));
    }
    if (uq) uq->n = cx.uq_n;
    std::vector<double> hs(1 + 2 * B);
    std::vector<unsigned long long> hn(B);
    NQS_CK(cudaMemcpyAsync(hs.data(), dev_scalars, hs.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaMemcpyAsync(hn.data(), next_dev, B * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    std::vector<double> ext(B), in(B);
    double nu = 0;
    for (int64_t b = 0; b < B; ++b) {
        ext[b] = hs[1 + 2 * b];
        in[b] = hs[2 + 2 * b];
        nu += (double)hn[b];
        if (bucket_partials) {
            bucket_partials[2 * b] = ext[b];
            bucket_partials[2 * b + 1] = in[b];
        }
    }
    out[0] = host_ksum(ext);
    out[1] = host_ksum(in);
    out[2] = nu;
    out[3] = (double)total_emitted;
    out[4] = (double)B;
    return NQS_OK;
}

// H_SS construction (Sec. 3.1 combinatorial kernel, Eq. connected_set, Algorithm 1 step 1):
// every single and double excitation of every det of S, in canonical order, is resolved as a
// member of S or not (through an open-addressing hash table of S, and in nqs_connections
// through indices of S by alpha and by beta string that settle whole blocks at once), and the
// hits become CSR entries.
//
// One warp per det. Pass 1 counts the hits of each row and records them as ballot words; an
// exclusive scan gives row_ptr; pass 2 walks the ballot words in canonical order and writes
// each row without any sort. The matrix element is computed only for hits.
#include <stdlib.h>
#include <string.h>

#include "excite.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

// Pass 1: count the hits of each row. With bits != nullptr the hit pattern is also stored, one
// 32-bit ballot word per 32 canonical indices ([nS][ceil(nexc/32)], written with streaming
// stores so that it does not push the hash table of S out of L2), so that pass 2 only revisits
// hits.
//
// The kernel is instruction-issue bound, so the work per index is kept small: each lane handles
// two indices per round (e and e + 32) and issues both first probes before resolving either,
// and the doubles are decoded incrementally: a lane keeps the positions of its current index
// (hole-pair / particle-pair positions for same-spin doubles, positions in the occupied and
// virtual lists for alpha-beta doubles) and steps them by 32 without dividing.
__global__ void __launch_bounds__(CONN_THREADS, 5) k_conn_count(ProblemDev P, HashS H,
                                                              const ulonglong2* __restrict__ S,
                                                              int64_t nS, int64_t* rowcnt,
                                                              uint32_t* __restrict__ bits) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const uint32_t nexc = (uint32_t)P.nexc;
    const uint32_t nwords = (nexc + 31) / 32;
    const uint32_t o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                   o4 = o3 + (uint32_t)P.dBB;
    for (int64_t det = (int64_t)blockIdx.x * CONN_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * CONN_WARPS) {
        ulonglong2 x = S[det];
        fill_ctx(P, x.x, x.y, ctx, lane);
        int cnt = 0;
        EnumPos q;
        q.cls = -1;
        for (uint32_t r0 = 0; r0 < nexc; r0 += 64) {
            const uint32_t e0 = r0 + lane, e1 = e0 + 32;
            const bool v0 = e0 < nexc, v1 = e1 < nexc;
            uint64_t a0 = 0, b0 = 0, a1 = 0, b1 = 0, s0 = 0, s1 = 0;
            uint16_t f0 = 0, f1 = 0, g0 = 0, g1 = 0;
            if (v0) {
                step_key(P, T, *ctx, x.x, x.y, e0, o2, o3, o4, q, a0, b0);
                const uint64_t hh = s_hash(a0, b0);
                s0 = hash_slot(hh, H.mask);
                f0 = hash_fingerprint(hh);
                g0 = __ldg(&H.fp[s0]);
            }
            if (v1) {
                step_key(P, T, *ctx, x.x, x.y, e1, o2, o3, o4, q, a1, b1);
                const uint64_t hh = s_hash(a1, b1);
                s1 = hash_slot(hh, H.mask);
                f1 = hash_fingerprint(hh);
                g1 = __ldg(&H.fp[s1]);
            }
            // resolve both probe sequences (fingerprints first; a key only on a match)
            bool h0 = false, h1 = false;
            for (uint64_t it = 0; v0 && g0 != 0 && it <= H.mask; ++it) {
                if (g0 == f0) {
                    const ulonglong2 k = __ldg(&H.set[__ldg(&H.idx[s0])]);
                    if (k.x == a0 && k.y == b0) {
                        h0 = true;
                        break;
                    }
                }
                s0 = (s0 + 1) & H.mask;
                g0 = __ldg(&H.fp[s0]);
            }
            for (uint64_t it = 0; v1 && g1 != 0 && it <= H.mask; ++it) {
                if (g1 == f1) {
                    const ulonglong2 k = __ldg(&H.set[__ldg(&H.idx[s1])]);
                    if (k.x == a1 && k.y == b1) {
                        h1 = true;
                        break;
                    }
                }
                s1 = (s1 + 1) & H.mask;
                g1 = __ldg(&H.fp[s1]);
            }
            const unsigned m0 = __ballot_sync(FULL_MASK, h0);
            const unsigned m1 = __ballot_sync(FULL_MASK, h1);
            if (lane == 0) {
                cnt += __popc(m0) + __popc(m1);
                if (bits) {
                    __stcs(&bits[det * nwords + r0 / 32], m0);
                    if (r0 / 32 + 1 < nwords) __stcs(&bits[det * nwords + r0 / 32 + 1], m1);
                }
            }
        }
        if (lane == 0) rowcnt[det] = cnt + 1;  // + diagonal
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// Pass 1 with indices of S (nqs_connections). S is sorted by (a, b), so the configurations of
// S that share an alpha string form one contiguous run; a second index groups the alpha strings
// of S by beta string. For x = (A, B) the count pass then resolves
//   - the alpha-beta doubles per alpha single a' of A (the block of all beta singles that go
//     with it): one lookup of a' in the alpha index; nothing to do when a' is not an alpha
//     string of S; a scan of a''s run when it is short (length <= 4 x the beta singles), a
//     member's beta string b_y being a beta single of B exactly when popcount(B ^ b_y) == 2,
//     the two differing bits giving j_b and b_b and hence the canonical index; otherwise a
//     probe of the hash of S for each beta single, as the plain pass does;
//   - the beta singles and beta-beta doubles (same alpha string A) by one scan of x's own
//     alpha run: popcount(B ^ b_y) == 2 or 4;
//   - the alpha singles and alpha-alpha doubles (same beta string B) by one scan of x's own
//     beta group: popcount(A ^ a_y) == 2 or 4;
// falling back to the plain probe pass for a class whenever its run or group is long. Every
// canonical index resolves to the same hit or miss as a lookup of its x' in S, so the ballot
// words are bit for bit those of k_conn_count. The row's words are cleared first and hits are
// ORed in (order-free).
// ------------------------------------------------------------------------------------------
struct AlphaIdx {
    const uint64_t* key;  // [cap] alpha string, 0 = empty (alpha strings of S are nonzero)
    const int2* run;      // [cap] {start in S, length}
    uint64_t mask;        // cap - 1
};

__device__ __forceinline__ uint64_t alpha_slot(uint64_t a, uint64_t mask) {
    uint64_t h = a * 0x9E3779B97F4A7C15ull;
    return (h ^ (h >> 29)) & mask;
}

// one thread per configuration; the first of each alpha run inserts (a, start, length)
__global__ void k_alpha_index(const ulonglong2* __restrict__ S, int64_t nS, uint64_t* key,
                              int2* run, uint64_t mask) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nS;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = S[i].x;
        if (i > 0 && S[i - 1].x == a) continue;
        int64_t lo = i + 1, hi = nS;  // first position after the run (S ascending by a)
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (S[mid].x == a) lo = mid + 1;
            else hi = mid;
        }
        uint64_t slot = alpha_slot(a, mask);
        for (uint64_t it = 0; it <= mask; ++it) {
            if (atomicCAS((unsigned long long*)&key[slot], 0ull, (unsigned long long)a) == 0ull) {
                run[slot] = make_int2((int)i, (int)(lo - i));
                break;
            }
            slot = (slot + 1) & mask;
        }
    }
}

__device__ __forceinline__ bool alpha_find(const AlphaIdx& X, uint64_t a, int2& r) {
    uint64_t slot = alpha_slot(a, X.mask);
    for (uint64_t it = 0; it <= X.mask; ++it) {
        const uint64_t k = __ldg(&X.key[slot]);
        if (k == a) {
            r = __ldg(&X.run[slot]);
            return true;
        }
        if (k == 0ull) return false;
        slot = (slot + 1) & X.mask;
    }
    return false;
}

// Index of S by beta string: the alpha strings of the configurations that share a beta string,
// grouped in one list (the order inside a group is arbitrary: the count pass only tests
// membership). Built by counting per beta string, an exclusive scan over the table and a fill.
// Beta strings are nonzero whenever the beta electrons have somewhere to go (nb >= 1, mb >= 1),
// which is the only case in which it is used.
struct BetaIdx {
    const uint64_t* key;    // [cap] beta string, 0 = empty
    const uint32_t* off;    // [cap] start of the group in alist
    const uint32_t* cnt;    // [cap] group size
    const uint64_t* alist;  // [nS] alpha strings, grouped by beta string
    uint64_t mask;          // cap - 1
};

__device__ __forceinline__ int64_t beta_slot_insert(uint64_t* key, uint64_t b, uint64_t mask) {
    uint64_t slot = alpha_slot(b, mask);
    for (uint64_t it = 0; it <= mask; ++it) {
        const unsigned long long prev =
            atomicCAS((unsigned long long*)&key[slot], 0ull, (unsigned long long)b);
        if (prev == 0ull || prev == b) return (int64_t)slot;
        slot = (slot + 1) & mask;
    }
    return -1;
}

__global__ void k_beta_count(const ulonglong2* __restrict__ S, int64_t nS, uint64_t* key,
                             uint32_t* cnt, uint64_t mask) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nS;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = beta_slot_insert(key, S[i].y, mask);
        if (slot >= 0) atomicAdd(&cnt[slot], 1u);
    }
}

__global__ void k_beta_fill(const ulonglong2* __restrict__ S, int64_t nS, uint64_t* key,
                            const uint32_t* __restrict__ off, uint32_t* fill, uint64_t* alist,
                            uint64_t mask) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nS;
         i += (int64_t)gridDim.x * blockDim.x) {
        const ulonglong2 x = S[i];
        const int64_t slot = beta_slot_insert(key, x.y, mask);  // present: finds its slot
        if (slot >= 0) alist[off[slot] + atomicAdd(&fill[slot], 1u)] = x.x;
    }
}

__device__ __forceinline__ bool beta_find(const BetaIdx& Y, uint64_t b, uint32_t& off,
                                          uint32_t& n) {
    uint64_t slot = alpha_slot(b, Y.mask);
    for (uint64_t it = 0; it <= Y.mask; ++it) {
        const uint64_t k = __ldg(&Y.key[slot]);
        if (k == b) {
            off = __ldg(&Y.off[slot]);
            n = __ldg(&Y.cnt[slot]);
            return true;
        }
        if (k == 0ull) return false;
        slot = (slot + 1) & Y.mask;
    }
    return false;
}

// OR a 32-bit ballot whose bit k stands for canonical index base + k into the row's words
__device__ __forceinline__ void or_ballot(uint32_t* wb, uint32_t base, unsigned m) {
    if (!m) return;
    const uint32_t w = base >> 5, sh = base & 31u;
    atomicOr(&wb[w], m << sh);
    if (sh) {
        const unsigned hi = m >> (32u - sh);
        if (hi) atomicOr(&wb[w + 1], hi);
    }
}

// The plain probe pass over the canonical indices [lo, hi) of one class range (singles decode
// directly; same-spin doubles step incrementally from a fresh position). Returns, in lane 0,
// the number of hits; ballots are ORed into the row's (cleared) words.
__device__ __noinline__ int probe_range(const ProblemDev& P, const PairTables& T,
                                           const DetCtx& c, const HashS& H, ulonglong2 x,
                                           uint32_t lo, uint32_t hi, uint32_t o2, uint32_t o3,
                                           uint32_t o4, uint32_t* wb, int lane) {
    int cnt = 0;
    EnumPos q;
    q.cls = -1;
    for (uint32_t r0 = lo; r0 < hi; r0 += 64) {
        const uint32_t e0 = r0 + lane, e1 = e0 + 32;
        const bool v0 = e0 < hi, v1 = e1 < hi;
        uint64_t a0 = 0, b0 = 0, a1 = 0, b1 = 0, s0 = 0, s1 = 0;
        uint16_t f0 = 0, f1 = 0, g0 = 0, g1 = 0;
        if (v0) {
            step_key(P, T, c, x.x, x.y, e0, o2, o3, o4, q, a0, b0);
            const uint64_t hh = s_hash(a0, b0);
            s0 = hash_slot(hh, H.mask);
            f0 = hash_fingerprint(hh);
            g0 = __ldg(&H.fp[s0]);
        }
        if (v1) {
            step_key(P, T, c, x.x, x.y, e1, o2, o3, o4, q, a1, b1);
            const uint64_t hh = s_hash(a1, b1);
            s1 = hash_slot(hh, H.mask);
            f1 = hash_fingerprint(hh);
            g1 = __ldg(&H.fp[s1]);
        }
        bool h0 = false, h1 = false;
        for (uint64_t it = 0; v0 && g0 != 0 && it <= H.mask; ++it) {
            if (g0 == f0) {
                const ulonglong2 k = __ldg(&H.set[__ldg(&H.idx[s0])]);
                if (k.x == a0 && k.y == b0) {
                    h0 = true;
                    break;
                }
            }
            s0 = (s0 + 1) & H.mask;
            g0 = __ldg(&H.fp[s0]);
        }
        for (uint64_t it = 0; v1 && g1 != 0 && it <= H.mask; ++it) {
            if (g1 == f1) {
                const ulonglong2 k = __ldg(&H.set[__ldg(&H.idx[s1])]);
                if (k.x == a1 && k.y == b1) {
                    h1 = true;
                    break;
                }
            }
            s1 = (s1 + 1) & H.mask;
            g1 = __ldg(&H.fp[s1]);
        }
        const unsigned m0 = __ballot_sync(FULL_MASK, h0);
        const unsigned m1 = __ballot_sync(FULL_MASK, h1);
        if (lane == 0) {
            cnt += __popc(m0) + __popc(m1);
            or_ballot(wb, r0, m0);
            or_ballot(wb, r0 + 32, m1);
        }
    }
    return cnt;
}

// position of the pair (r1 < r2) in the lexicographic list of pairs of n items
__device__ __forceinline__ uint32_t pair_pos(uint32_t r1, uint32_t r2, uint32_t n) {
    return r1 * (2 * n - r1 - 1) / 2 + (r2 - r1 - 1);
}

// S: the rows to resolve; R: the sorted set they are resolved against (the array the alpha
// index's runs point into; R = S for H_SS, the sorted target set for the proxy Hamiltonian)
// the alpha-beta work of one lane of k_conn_count_ab: its first item in the warp's item range,
// the start of the alpha run it scans in R (-1: probe the beta singles instead) and the alpha
// string of its single
struct __align__(16) OwnerRec {
    uint32_t first;
    int32_t start;
    uint64_t a2;
};

// PART 0: the row's words cleared, then the singles and same-spin doubles (scans of x's own
// beta group and alpha run); PART 1, launched after it: the alpha-beta block, adding to the
// row's count. Two kernels, so that each keeps fewer values live than the whole pass would.
#define CONN_AB_BLOCKS0 7  // blocks per SM of each part (a sweep: 5, 6 and 8 no faster)
#define CONN_AB_BLOCKS1 7
template <int PART>
__global__ void __launch_bounds__(CONN_THREADS, PART == 0 ? CONN_AB_BLOCKS0 : CONN_AB_BLOCKS1)
    k_conn_count_ab(ProblemDev P, HashS H,
                                                                 AlphaIdx X, BetaIdx Y,
                                                                 const ulonglong2* __restrict__ S,
                                                                 int64_t nS,
                                                                 const ulonglong2* __restrict__ R,
                                                                 int64_t* rowcnt,
                                                                 uint32_t* __restrict__ bits) {
    extern __shared__ __align__(16) uint8_t smem[];
    // per warp, for the alpha-beta block: each lane's work record and the lane of each rank
    // among the lanes that have work
    __shared__ OwnerRec orec[CONN_WARPS][32];
    __shared__ uint8_t orank[CONN_WARPS][32];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    OwnerRec* rec = orec[threadIdx.x >> 5];
    uint8_t* rank_lane = orank[threadIdx.x >> 5];
    const uint32_t nexc = (uint32_t)P.nexc;
    const uint32_t nwords = (nexc + 31) / 32;
    const uint32_t o1 = (uint32_t)P.sA, o2 = (uint32_t)(P.sA + P.sB), o3 = o2 + (uint32_t)P.dAA,
                   o4 = o3 + (uint32_t)P.dBB;
    const uint32_t sA = (uint32_t)P.sA, sB = (uint32_t)P.sB;
    const uint32_t scan_max = 4 * sB;
    const uint32_t own_scan_max = 4 * (sB + (uint32_t)P.dBB);
    const uint32_t nb = (uint32_t)P.nb, mb = (uint32_t)P.mb, Qb = (uint32_t)choose2(P.mb);
    const uint32_t na = (uint32_t)P.na, ma = (uint32_t)P.ma, Qa = (uint32_t)choose2(P.ma);
    const uint32_t own_a_scan_max = 4 * (sA + (uint32_t)P.dAA);
    for (int64_t det = (int64_t)blockIdx.x * CONN_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * CONN_WARPS) {
        ulonglong2 x = S[det];
        fill_ctx(P, x.x, x.y, ctx, lane);
        uint32_t* wb = bits + det * nwords;
        int cnt = 0;
        if (PART == 0) {
        for (uint32_t w = lane; w < nwords; w += 32) wb[w] = 0u;
        __syncwarp();
        // alpha singles and alpha-alpha doubles of x keep its beta string: they are the alpha
        // strings a_y of x's own beta group with popcount(A ^ a_y) = 2 (single) or 4 (double)
        uint32_t boff = 0, blen = 0;
        if (Y.key && beta_find(Y, x.y, boff, blen) && blen <= own_a_scan_max) {
            for (uint32_t k0 = 0; k0 < blen; k0 += 32) {
                const uint32_t k = k0 + lane;
                bool hit = false;
                uint32_t e = 0;
                if (k < blen) {
                    const uint64_t ay = __ldg(&Y.alist[boff + k]);
                    const uint64_t d = ay ^ x.x;
                    const int pc = __popcll(d);
                    if (pc == 2) {
                        const uint64_t ibit = x.x & d, abit = ay & d;
                        const uint32_t xa = (uint32_t)__popcll(x.x & (ibit - 1ull));
                        const uint32_t ya = (uint32_t)__popcll(~x.x & (abit - 1ull));
                        e = xa * ma + ya;
                        hit = true;
                    } else if (pc == 4) {
                        const uint64_t holes = x.x & d, parts = ay & d;
                        const uint64_t i1 = holes & (~holes + 1ull), i2 = holes ^ i1;
                        const uint64_t a1 = parts & (~parts + 1ull), a2 = parts ^ a1;
                        const uint32_t r1 = (uint32_t)__popcll(x.x & (i1 - 1ull)),
                                       r2 = (uint32_t)__popcll(x.x & (i2 - 1ull));
                        const uint32_t v1 = (uint32_t)__popcll(~x.x & (a1 - 1ull)),
                                       v2 = (uint32_t)__popcll(~x.x & (a2 - 1ull));
                        e = o2 + pair_pos(r1, r2, na) * Qa + pair_pos(v1, v2, ma);
                        hit = true;
                    }
                }
                if (hit) atomicOr(&wb[e >> 5], 1u << (e & 31));
                const unsigned mh = __ballot_sync(FULL_MASK, hit);
                if (lane == 0) cnt += __popc(mh);
            }
        } else {
            cnt += probe_range(P, T, *ctx, H, x, 0, o1, o2, o3, o4, wb, lane);
            cnt += probe_range(P, T, *ctx, H, x, o2, o3, o2, o3, o4, wb, lane);
        }
        // beta singles and beta-beta doubles of x keep its alpha string: they are the members
        // y of x's own alpha run with popcount(B ^ b_y) = 2 (single) or 4 (double)
        int2 own = make_int2(0, 0);
        const bool have_own = alpha_find(X, x.x, own);  // x is in S: always found
        if (have_own && (uint32_t)own.y <= own_scan_max) {
            for (uint32_t k0 = 0; k0 < (uint32_t)own.y; k0 += 32) {
                const uint32_t k = k0 + lane;
                bool hit = false;
                uint32_t e = 0;
                if (k < (uint32_t)own.y) {
                    const uint64_t by = __ldg(&R[own.x + k].y);
                    const uint64_t d = by ^ x.y;
                    const int pc = __popcll(d);
                    if (pc == 2) {
                        const uint64_t jbit = x.y & d, bbit = by & d;
                        const uint32_t xb = (uint32_t)__popcll(x.y & (jbit - 1ull));
                        const uint32_t yb = (uint32_t)__popcll(~x.y & (bbit - 1ull));
                        e = o1 + xb * mb + yb;
                        hit = true;
                    } else if (pc == 4) {
                        const uint64_t holes = x.y & d, parts = by & d;
                        const uint64_t j1 = holes & (~holes + 1ull), j2 = holes ^ j1;
                        const uint64_t b1 = parts & (~parts + 1ull), b2 = parts ^ b1;
                        const uint32_t r1 = (uint32_t)__popcll(x.y & (j1 - 1ull)),
                                       r2 = (uint32_t)__popcll(x.y & (j2 - 1ull));
                        const uint32_t v1 = (uint32_t)__popcll(~x.y & (b1 - 1ull)),
                                       v2 = (uint32_t)__popcll(~x.y & (b2 - 1ull));
                        e = o3 + pair_pos(r1, r2, nb) * Qb + pair_pos(v1, v2, mb);
                        hit = true;
                    }
                }
                if (hit) atomicOr(&wb[e >> 5], 1u << (e & 31));
                const unsigned mh = __ballot_sync(FULL_MASK, hit);
                if (lane == 0) cnt += __popc(mh);
            }
        } else {
            cnt += probe_range(P, T, *ctx, H, x, o1, o2, o2, o3, o4, wb, lane);
            cnt += probe_range(P, T, *ctx, H, x, o3, o4, o2, o3, o4, wb, lane);
        }
        }  // PART 0
        __syncwarp();
        for (uint32_t sa0 = 0; PART == 1 && sa0 < sA; sa0 += 32) {
            const uint32_t si = sa0 + lane;
            uint64_t a2 = 0;
            int2 r = make_int2(0, 0);
            uint32_t w = 0;
            bool scan = false;
            if (si < sA) {
                const uint32_t xa = si / (uint32_t)P.ma, ya = si - xa * (uint32_t)P.ma;
                a2 = x.x ^ (1ull << ctx->occA[xa]) ^ (1ull << ctx->virA[ya]);
                if (alpha_find(X, a2, r)) {
                    scan = (uint32_t)r.y <= scan_max;
                    w = scan ? (uint32_t)r.y : sB;
                }
            }
            uint32_t incl = w;  // inclusive prefix of the work over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
            const uint32_t excl = incl - w;
            // work item t belongs to the last lane with work whose first item is at or before t
            // (those first items are strictly increasing over such lanes). Per chunk of 32
            // items: the lanes with work starting at or before the chunk, plus a mask of the
            // starts inside it, give each item the rank of its owner; the owner's record comes
            // from shared memory.
            const unsigned has = __ballot_sync(FULL_MASK, w > 0u);
            if (w > 0u) {
                OwnerRec o;
                o.first = excl;
                o.start = scan ? r.x : -1;
                o.a2 = a2;
                rec[lane] = o;
                rank_lane[__popc(has & lt)] = (uint8_t)lane;
            }
            __syncwarp();
            for (uint32_t t0 = 0; t0 < total; t0 += 32) {
                const int dj = (int)(excl - t0);  // excl, t0 < 2^31
                const unsigned before = __ballot_sync(FULL_MASK, w > 0u && dj <= 0);
                const unsigned inside = __reduce_or_sync(
                    FULL_MASK, (w > 0u && dj > 0 && dj < 32) ? (1u << dj) : 0u);
                const int c = __popc(before) + __popc(inside & ((2u << lane) - 1u));
                const int own = rank_lane[c - 1];
                const OwnerRec o = rec[own];
                const uint32_t t = t0 + lane;
                bool hit = false;
                uint32_t lb = 0;
                if (t < total) {
                    const uint32_t k = t - o.first;
                    if (o.start >= 0) {
                        const uint64_t by = __ldg(&R[o.start + k].y);
                        const uint64_t d = by ^ x.y;
                        if (__popcll(d) == 2) {
                            const uint64_t jbit = x.y & d, bbit = by & d;
                            const uint32_t xb = (uint32_t)__popcll(x.y & (jbit - 1ull));
                            const uint32_t yb = (uint32_t)__popcll(~x.y & (bbit - 1ull));
                            lb = xb * (uint32_t)P.mb + yb;
                            hit = true;
                        }
                    } else {
                        const uint32_t xb = k / (uint32_t)P.mb, yb = k - xb * (uint32_t)P.mb;
                        const uint64_t b2 =
                            x.y ^ (1ull << ctx->occB[xb]) ^ (1ull << ctx->virB[yb]);
                        hit = hash_lookup(H, o.a2, b2) >= 0;
                        lb = k;
                    }
                }
                if (hit) {
                    const uint32_t e = o4 + (sa0 + (uint32_t)own) * sB + lb;
                    atomicOr(&wb[e / 32], 1u << (e & 31));
                }
                const unsigned mh = __ballot_sync(FULL_MASK, hit);
                if (lane == 0) cnt += __popc(mh);
            }
            __syncwarp();  // the records are rewritten by the next round of alpha singles
        }
        if (lane == 0) {
            if (PART == 0) rowcnt[det] = cnt + 1;  // + diagonal
            else rowcnt[det] += cnt;
        }
        __syncwarp();
    }
}

// Pass 2: write each row in canonical order: the diagonal, then the hits. With bits the warp
// walks the stored ballot words (skipping empty ones) and decodes, probes and evaluates only
// the hits; without bits it re-enumerates every excitation.
__global__ void __launch_bounds__(CONN_THREADS, 6) k_conn_fill(ProblemDev P, HashS H,
                                                             const ulonglong2* __restrict__ S,
                                                             int64_t nS,
                                                             const int64_t* __restrict__ row_ptr,
                                                             int32_t* __restrict__ col,
                                                             double* __restrict__ val,
                                                             const uint32_t* __restrict__ bits) {
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables T = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    __shared__ uint32_t queue[CONN_WARPS * 64];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const uint32_t nexc = (uint32_t)P.nexc;
    const uint32_t nwords = (nexc + 31) / 32;
    // the diagonal of every row, one thread per configuration (each a sequential FP64 sum; one
    // lane per warp doing it would hold the FP64 pipe for a whole warp per operation)
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < nS;
         d += (int64_t)gridDim.x * blockDim.x) {
        const ulonglong2 x = S[d];
        const int64_t b = row_ptr[d];
        col[b] = (int32_t)d;
        val[b] = diag_element_impl(P, x.x, x.y);
    }
    for (int64_t det = (int64_t)blockIdx.x * CONN_WARPS + (threadIdx.x >> 5); det < nS;
         det += (int64_t)gridDim.x * CONN_WARPS) {
        ulonglong2 x = S[det];
        fill_ctx(P, x.x, x.y, ctx, lane);
        const int64_t base = row_ptr[det];
        int64_t run = base + 1;
        if (bits) {
            // The hits of the stored ballot words are appended, in canonical order, to a per-warp
            // queue; each time it holds 32 the whole warp decodes, probes and evaluates them
            // together (hits are ~10% of the excitations: one word at a time would leave most
            // lanes idle).
            const uint32_t* wb = bits + det * nwords;
            uint32_t* qu = queue + (threadIdx.x >> 5) * 64;
            uint32_t qn = 0;
            auto flush = [&](uint32_t nt) {
                if ((uint32_t)lane < nt) {
                    Exc ex;
                    decode_exc(P, T, *ctx, x.x, x.y, qu[lane], ex);
                    col[run + lane] = hash_lookup_member(H, ex.a2, ex.b2);  // a hit: in S
                    val[run + lane] = exc_element(P, *ctx, ex);
                }
                run += nt;
                const uint32_t rest = qn - nt;
                const uint32_t moved = (uint32_t)lane < rest ? qu[nt + lane] : 0u;
                __syncwarp();
                if ((uint32_t)lane < rest) qu[lane] = moved;
                qn = rest;
                __syncwarp();
            };
            // the next 32 ballot words are loaded before this chunk's hits are queued and
            // resolved, so the load's latency overlaps the work
            uint32_t nxt = lane < nwords ? __ldcs(&wb[lane]) : 0u;
            for (uint32_t w0 = 0; w0 < nwords; w0 += 32) {
                const uint32_t my = nxt;
                nxt = (w0 + 32 + lane < nwords) ? __ldcs(&wb[w0 + 32 + lane]) : 0u;
                unsigned nz = __ballot_sync(FULL_MASK, my != 0u);
                while (nz) {
                    const int src = __ffs(nz) - 1;
                    nz &= nz - 1;
                    const uint32_t m = __shfl_sync(FULL_MASK, my, src);
                    if ((m >> lane) & 1u) qu[qn + __popc(m & lt)] = (w0 + src) * 32 + lane;
                    qn += __popc(m);
                    __syncwarp();
                    if (qn >= 32) flush(32);
                }
            }
            if (qn > 0) flush(qn);
        } else {
            for (uint32_t r0 = 0; r0 < nexc; r0 += 32) {
                uint32_t e = r0 + lane;
                int32_t hit = -1;
                Exc ex;
                if (e < nexc) {
                    decode_exc(P, T, *ctx, x.x, x.y, e, ex);
                    hit = hash_lookup(H, ex.a2, ex.b2);
                }
                unsigned m = __ballot_sync(FULL_MASK, hit >= 0);
                if (hit >= 0) {
                    int64_t pos = run + __popc(m & lt);
                    col[pos] = hit;
                    val[pos] = exc_element(P, *ctx, ex);
                }
                run += __popc(m);
            }
        }
        __syncwarp();
    }
}

static size_t conn_smem(const ProblemDev& P) {
    return pair_table_bytes(P) + CONN_WARPS * sizeof(DetCtx);
}

static unsigned conn_grid(int64_t nS) {
    int64_t g = (nS + CONN_WARPS - 1) / CONN_WARPS;
    if (g > 148 * 16) g = 148 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

size_t conn_smem_bytes(const ProblemDev& P) { return conn_smem(P); }
unsigned conn_grid_size(int64_t nS) { return conn_grid(nS); }

// The count pass over `rows` (nrows configurations) against the sorted, unique set R (nR
// configurations, hashed in H; every row must be a member of R): the indices of R by alpha
// string and by beta string, then k_conn_count_ab (k_conn_count when there are no alpha-beta
// doubles). rowcnt [nrows] receives the row lengths (diagonal included) and bits
// [nrows][ceil(nexc / 32)] the hit ballots.
int conn_count_indexed(nqs_problem* p, Scratch& sc, const HashS& H, const uint64_t* rows,
                       int64_t nrows, const uint64_t* Rset, int64_t nR, int64_t* rowcnt,
                       uint32_t* bits, cudaStream_t s) {
    const size_t smem = conn_smem(p->d);
    if (smem > 48 * 1024) {
        NQS_CK(cudaFuncSetAttribute(k_conn_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
        NQS_CK(cudaFuncSetAttribute(k_conn_count_ab<0>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NQS_CK(cudaFuncSetAttribute(k_conn_count_ab<1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    // index of R by alpha string (runs of the sorted R), for the alpha-beta block of pass 1
    const bool use_ab = p->d.dAB > 0;
    AlphaIdx X;
    memset(&X, 0, sizeof X);
    if (use_ab) {
        uint64_t cap = 1024;
        while (cap < 2 * (uint64_t)nR) cap <<= 1;
        uint64_t* akey;
        int2* arun;
        NQS_TRY(sc.get(&akey, cap));
        NQS_TRY(sc.get(&arun, cap));
        NQS_CK(cudaMemsetAsync(akey, 0, cap * sizeof(uint64_t), s));
        k_alpha_index<<<grid_for(nR, 256), 256, 0, s>>>((const ulonglong2*)Rset, nR, akey, arun,
                                                        cap - 1);
        NQS_CK_LAUNCH();
        X.key = akey;
        X.run = arun;
        X.mask = cap - 1;
    }
    // index of R by beta string, for the alpha singles and alpha-alpha doubles of pass 1
    BetaIdx Y;
    memset(&Y, 0, sizeof Y);
    if (use_ab && p->d.nb >= 1 && p->d.mb >= 1) {
        uint64_t cap = 1024;
        while (cap < 2 * (uint64_t)nR) cap <<= 1;
        uint64_t *bkey, *alist;
        uint32_t *bcnt, *boff, *bfill;
        NQS_TRY(sc.get(&bkey, cap));
        NQS_TRY(sc.get(&bcnt, cap));
        NQS_TRY(sc.get(&boff, cap));
        NQS_TRY(sc.get(&bfill, cap));
        NQS_TRY(sc.get(&alist, nR));
        NQS_CK(cudaMemsetAsync(bkey, 0, cap * sizeof(uint64_t), s));
        NQS_CK(cudaMemsetAsync(bcnt, 0, cap * sizeof(uint32_t), s));
        NQS_CK(cudaMemsetAsync(bfill, 0, cap * sizeof(uint32_t), s));
        k_beta_count<<<grid_for(nR, 256), 256, 0, s>>>((const ulonglong2*)Rset, nR, bkey, bcnt,
                                                       cap - 1);
        NQS_CK_LAUNCH();
        NQS_TRY(scan_exclusive_u32(p, sc, bcnt, boff, (int64_t)cap, s));
        k_beta_fill<<<grid_for(nR, 256), 256, 0, s>>>((const ulonglong2*)Rset, nR, bkey, boff,
                                                      bfill, alist, cap - 1);
        NQS_CK_LAUNCH();
        Y.key = bkey;
        Y.off = boff;
        Y.cnt = bcnt;
        Y.alist = alist;
        Y.mask = cap - 1;
    }
    {
        ProfScope prof_(PROF_CONN_COUNT, s);
        if (use_ab) {
            k_conn_count_ab<0><<<conn_grid(nrows), CONN_THREADS, smem, s>>>(
                p->d, H, X, Y, (const ulonglong2*)rows, nrows, (const ulonglong2*)Rset, rowcnt,
                bits);
            k_conn_count_ab<1><<<conn_grid(nrows), CONN_THREADS, smem, s>>>(
                p->d, H, X, Y, (const ulonglong2*)rows, nrows, (const ulonglong2*)Rset, rowcnt,
                bits);
        } else
            k_conn_count<<<conn_grid(nrows), CONN_THREADS, smem, s>>>(
                p->d, H, (const ulonglong2*)rows, nrows, rowcnt, bits);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

extern "C" int nqs_connections(nqs_problem* p, const uint64_t* dets, int64_t nS,
                               const nqs_opts* opts, nqs_csr* out, int64_t* n_enumerated,
                               nqs_stream_t stream) {
    if (!p || !out || nS <= 0 || !dets) return NQS_ERR_ARG;
    if (nS >= ((int64_t)1 << 31)) return NQS_ERR_UNSUPPORTED;
    if (((uintptr_t)dets) & 15) return NQS_ERR_ARG;
    memset(out, 0, sizeof *out);
    cudaStream_t s = (cudaStream_t)stream;
    nqs_opts def;
    if (!opts) {
        nqs_opts_default(&def);
        opts = &def;
    }
    Scratch sc(p, s);
    if (opts->validate) NQS_TRY(validate_dets(p, sc, dets, nS, true, s));
    HashS H;
    NQS_TRY(hash_build(p, sc, dets, nS, &H, s));
    size_t smem = conn_smem(p->d);
    if (smem > 48 * 1024)
        NQS_CK(cudaFuncSetAttribute(k_conn_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    int64_t* rowcnt;
    NQS_TRY(sc.get(&rowcnt, nS));
    uint32_t* bits;
    NQS_TRY(sc.get(&bits, (size_t)nS * ((p->d.nexc + 31) / 32)));
    // the matrix comes from the problem's stream-ordered pool: no device-wide synchronisation
    // to allocate it, and nqs_csr_free_async returns it in stream order
    int64_t* row_ptr = nullptr;
    NQS_TRY(nqs_scratch_alloc(p, (void**)&row_ptr, (nS + 1) * sizeof(int64_t), s));
    auto fail = [&](int code) {
        nqs_scratch_free(p, row_ptr, s);
        return code;
    };
    int st = conn_count_indexed(p, sc, H, dets, nS, dets, nS, rowcnt, bits, s);
    if (st < 0) return fail(st);
    st = scan_exclusive_i64(p, sc, rowcnt, row_ptr, nS, row_ptr + nS, s);
    if (st < 0) return fail(st);
    int64_t nnz = 0;
    if (cudaMemcpyAsync(&nnz, row_ptr + nS, sizeof nnz, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(NQS_ERR_CUDA);
    int32_t* col = nullptr;
    double* val = nullptr;
    if (nqs_scratch_alloc(p, (void**)&col, (nnz > 0 ? nnz : 1) * sizeof(int32_t), s) != NQS_OK ||
        nqs_scratch_alloc(p, (void**)&val, (nnz > 0 ? nnz : 1) * sizeof(double), s) != NQS_OK) {
        nqs_scratch_free(p, col, s);
        return fail(NQS_ERR_OOM);
    }
    {
        ProfScope prof_(PROF_CONN_FILL, s);
        k_conn_fill<<<conn_grid(nS), CONN_THREADS, smem, s>>>(p->d, H, (const ulonglong2*)dets, nS,
                                                              row_ptr, col, val, bits);
    }
    nqs_note_launch();
    if (cudaGetLastError() != cudaSuccess) {
        nqs_scratch_free(p, col, s);
        nqs_scratch_free(p, val, s);
        return fail(NQS_ERR_CUDA);
    }
    out->row_ptr = row_ptr;
    out->col = col;
    out->val = val;
    out->nnz = nnz;
    out->n_rows = nS;
    if (n_enumerated) *n_enumerated = nS * p->d.nexc;
    return NQS_OK;
}

extern "C" int nqs_csr_free(nqs_csr* csr) {
    if (!csr) return NQS_ERR_ARG;
    // after every stream of the device is idle, a free in any stream order is safe
    cudaError_t e = cudaDeviceSynchronize();
    if (csr->row_ptr) cudaFreeAsync(csr->row_ptr, 0);
    if (csr->col) cudaFreeAsync(csr->col, 0);
    if (csr->val) cudaFreeAsync(csr->val, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    memset(csr, 0, sizeof *csr);
    if (e != cudaSuccess) {
        nqs_record_error("nqs_csr_free", e, __FILE__, __LINE__);
        return NQS_ERR_CUDA;
    }
    return NQS_OK;
}

extern "C" int nqs_csr_free_async(nqs_csr* csr, nqs_stream_t stream) {
    if (!csr) return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (csr->row_ptr) cudaFreeAsync(csr->row_ptr, s);
    if (csr->col) cudaFreeAsync(csr->col, s);
    if (csr->val) cudaFreeAsync(csr->val, s);
    memset(csr, 0, sizeof *csr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        nqs_record_error("nqs_csr_free_async", e, __FILE__, __LINE__);
        return NQS_ERR_CUDA;
    }
    return NQS_OK;
}

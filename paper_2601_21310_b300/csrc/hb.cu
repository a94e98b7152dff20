// Heat-bath screened perturbative set, Eq. (hb_screen) of Sec. 3.3:
//   P = { x' not in S : max over x in S of |H_x'x psi(x)| >= eps }.
//
// Sec. 3.3 accelerates the test with integral tables: for every pair of occupied orbitals the
// particle pairs are sorted by descending |<ij||ab>|, and the walk over them stops at the first
// entry below the cutoff. Doubles are exactly those entries (|H_x'x| = |<ij||ab>|), so with the
// cutoff tested as the product |<ij||ab>| * |psi_x| >= eps (FP64, monotone in the table value)
// the early exit drops nothing that the definition keeps. Singles have an element that depends
// on x; they are few (n (norb - n) per spin) and are all evaluated exactly.
//
// Tables (built once per problem, on first use):
//   same spin     one list per orbital pair i<j: particle pairs a<b with {a,b} and {i,j}
//                 disjoint, value |(ia|jb) - (ib|ja)|, length C(norb-2, 2);
//   opposite spin one list per (i alpha, j beta): (a alpha, b beta) with a != i, b != j,
//                 value |(ia|jb)|, length (norb-1)^2.
// Each list is sorted descending in shared memory by one CTA (bitonic network).
//
// Selection: one warp per x of S. A count pass and an emit pass run the same traversal
// (singles, same-spin pairs, opposite-spin pairs; lists whose head fails the cutoff are skipped
// from a ballot over 32 hole pairs). Kept configurations are probed in the hash table of S and
// dropped when present. The emitted (key, |H psi|) pairs are radix-sorted by key; each run
// becomes one output configuration with the maximum of its couplings.
#include <math.h>

#include "excite.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

#define HB_THREADS 256
#define HB_WARPS (HB_THREADS / 32)
#define HB_SORT_THREADS 512

struct HbTab {
    const double* val;    // [lists][len] descending
    const uint16_t* code; // a | b << 8
    int Lss, Los;         // list lengths
    int64_t os_base;      // index of the first opposite-spin entry
};

// index of the orbital pair i < j among all C(norb, 2) pairs, lexicographic
__device__ __forceinline__ int pair_index(int i, int j, int n) {
    return i * (2 * n - i - 1) / 2 + (j - i - 1);
}

// x comes before y in a descending list (ties by ascending code)
__device__ __forceinline__ bool hb_before(double vx, uint16_t cx, double vy, uint16_t cy) {
    return vx > vy || (vx == vy && cx < cy);
}

// One CTA per list. Slots cover every candidate particle pair; those that share an orbital with
// the hole pair get the value -1 and sort behind every real entry (all >= 0).
__global__ void __launch_bounds__(HB_SORT_THREADS) k_hb_tables(int n, const double* __restrict__ eri,
                                                               int n_ss_lists, int Lss, int Los,
                                                               int Np, double* __restrict__ val,
                                                               uint16_t* __restrict__ code) {
    extern __shared__ __align__(16) uint8_t smem[];
    double* sv = (double*)smem;
    uint16_t* sc = (uint16_t*)(sv + Np);
    const int list = blockIdx.x;
    const bool same = list < n_ss_lists;
    int i, j, nslots;
    if (same) {
        int lo = 0, rem = list;
        while (rem >= n - 1 - lo) {
            rem -= n - 1 - lo;
            ++lo;
        }
        i = lo;
        j = lo + 1 + rem;
        nslots = n * (n - 1) / 2;
    } else {
        const int q = list - n_ss_lists;
        i = q / n;
        j = q - i * n;
        nslots = n * n;
    }
    for (int t = threadIdx.x; t < Np; t += blockDim.x) {
        double v = -1.0;
        int a = 0, b = 0;
        if (t < nslots) {
            if (same) {
                int lo = 0, rem = t;
                while (rem >= n - 1 - lo) {
                    rem -= n - 1 - lo;
                    ++lo;
                }
                a = lo;
                b = lo + 1 + rem;
                if (a != i && a != j && b != i && b != j) {
                    const double t1 = eri[(((size_t)i * n + a) * n + j) * n + b];
                    const double t2 = eri[(((size_t)i * n + b) * n + j) * n + a];
                    v = fabs(t1 - t2);
                }
            } else {
                a = t / n;
                b = t - a * n;
                if (a != i && b != j) v = fabs(eri[(((size_t)i * n + a) * n + j) * n + b]);
            }
        }
        sv[t] = v;
        sc[t] = (uint16_t)(a | (b << 8));
    }
    __syncthreads();
    for (int k = 2; k <= Np; k <<= 1) {
        for (int s = k >> 1; s > 0; s >>= 1) {
            for (int t = threadIdx.x; t < Np; t += blockDim.x) {
                const int u = t ^ s;
                if (u > t) {
                    const bool first_half = (t & k) == 0;
                    const bool out_of_order = first_half ? hb_before(sv[u], sc[u], sv[t], sc[t])
                                                         : hb_before(sv[t], sc[t], sv[u], sc[u]);
                    if (out_of_order) {
                        const double tv = sv[t];
                        sv[t] = sv[u];
                        sv[u] = tv;
                        const uint16_t tc = sc[t];
                        sc[t] = sc[u];
                        sc[u] = tc;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int L = same ? Lss : Los;
    const int64_t base = same ? (int64_t)list * Lss
                              : (int64_t)n_ss_lists * Lss + (int64_t)(list - n_ss_lists) * Los;
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        val[base + t] = sv[t];
        code[base + t] = sc[t];
    }
}

static int hb_tables(nqs_problem* p, HbTab* out) {
    const int n = p->d.norb;
    const int n_ss = n * (n - 1) / 2, n_os = n * n;
    const int Lss = (n - 2) * (n - 3) / 2 > 0 ? (n - 2) * (n - 3) / 2 : 0;
    const int Los = (n - 1) * (n - 1);
    if (!p->hb_val) {
        const int64_t total = (int64_t)n_ss * Lss + (int64_t)n_os * Los;
        int Np = 1;
        while (Np < n * n) Np <<= 1;
        const size_t smem = (size_t)Np * (sizeof(double) + sizeof(uint16_t));
        if (smem > 48 * 1024)
            NQS_CK(cudaFuncSetAttribute(k_hb_tables, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
        double* val = nullptr;
        uint16_t* code = nullptr;
        if (cudaMalloc(&val, (total > 0 ? total : 1) * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&code, (total > 0 ? total : 1) * sizeof(uint16_t)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(val);
            return NQS_ERR_OOM;
        }
        k_hb_tables<<<n_ss + n_os, HB_SORT_THREADS, smem>>>(n, p->d.eri, n_ss, Lss, Los, Np, val,
                                                             code);
        nqs_note_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cudaFree(val);
            cudaFree(code);
            nqs_record_error("k_hb_tables", e, __FILE__, __LINE__);
            return NQS_ERR_CUDA;
        }
        p->hb_val = val;
        p->hb_code = code;
    }
    out->val = p->hb_val;
    out->code = p->hb_code;
    out->Lss = Lss;
    out->Los = Los;
    out->os_base = (int64_t)n_ss * Lss;
    return NQS_OK;
}

__device__ __forceinline__ bool in_bucket_of(uint64_t a, uint64_t b, uint64_t B, uint64_t bucket) {
    return B == 1 || det_bucket(a, b, B) == bucket;
}

// The screening test fl(v |psi_x|) >= eps for v >= 0 (a table entry or |<x'|H|x>|), without an
// FP64 multiply per candidate: the rounded product is non-decreasing in v, so it holds exactly
// when v >= v*, the smallest double that passes, and non-negative doubles order like their bit
// patterns (an integer compare). v* is found once per x: a few ulp steps from eps / |psi_x|,
// else a bisection over the bit patterns of [0, inf] (exact, at most 63 products).
struct HbCut {
    unsigned long long thr;  // bit pattern of v*
    __device__ __forceinline__ bool pass(double v) const {
        return (unsigned long long)__double_as_longlong(v) >= thr;
    }
};

// the FP64 element of a single near the cut (rare): out of line, so that the traversal keeps
// its registers for the common path
__device__ __noinline__ double single_element_near_cut(const ProblemDev& P, const DetCtx& c,
                                                       const Exc& x) {
    return exc_element(P, c, x);
}

// The same cut for a single's element from its fixed-point value F (units 2^-e): |F| at or above
// hi passes and at or below lo fails whatever FP64 rounding the exact element has (the margin
// covers the table roundings and the FP64 sum's own error); in between the FP64 element is
// formed exactly and tested.
struct HbCutFx {
    long long lo, hi;  // fail surely when |F| <= lo (lo = -1: never), pass surely when |F| >= hi
    bool all;          // eps = 0: every single passes
};

__device__ __forceinline__ HbCutFx hb_cut_fx(const HbCut& c, const ProblemDev& P) {
    const long long never_pass = 0x7fffffffffffffffll;
    HbCutFx r;
    r.all = c.thr == 0ull;
    r.lo = -1;
    r.hi = never_pass;
    if (r.all) return r;
    // margin in grid units: 49 roundings of table entries (half a unit each), the FP64 sum's
    // error (48 ulps of at most hoff_max, i.e. 48 * 2^-53 hoff_max 2^e <= 48 * 2^9 units), and
    // 2048 for the rounding of t +- margin in FP64 (spacing at most 2^10 below 2^62)
    const double margin = 24.5 + 48.0 * 512.0 + 2048.0;
    const double t = ldexp(__longlong_as_double((long long)c.thr), P.sfx_e);
    const double two62 = 4611686018427387904.0;
    if (t + margin < two62) r.hi = (long long)ceil(t + margin);
    if (t - margin >= two62) r.lo = never_pass;  // no element reaches the cut
    else if (t - margin > 0.0) r.lo = (long long)floor(t - margin);
    return r;
}

__device__ __noinline__ unsigned long long hb_cut_bisect(double eps, double ap) {
    unsigned long long lo = 0ull, hi = 0x7ff0000000000000ull;  // fails at lo, passes at hi
    while (hi - lo > 1ull) {
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        if (__dmul_rn(__longlong_as_double((long long)mid), ap) >= eps) hi = mid;
        else lo = mid;
    }
    return hi;
}

// requires eps > 0 or returns the pass-all cut; ap > 0 and finite
__device__ __forceinline__ HbCut hb_cut(double eps, double ap) {
    HbCut c;
    c.thr = 0ull;
    if (!(eps > 0.0)) return c;  // every v >= 0 passes
    const double t = __ddiv_rn(eps, ap);
    const unsigned long long inf = 0x7ff0000000000000ull;
    if (!(t < __longlong_as_double((long long)inf))) {
        c.thr = inf;  // no finite v passes
        return c;
    }
    unsigned long long b = (unsigned long long)__double_as_longlong(t);
    int steps = 0;
    if (__dmul_rn(t, ap) >= eps) {
        while (b > 0 && steps < 8 && __dmul_rn(__longlong_as_double((long long)(b - 1)), ap) >= eps) {
            --b;
            ++steps;
        }
    } else {
        do {
            ++b;
            ++steps;
        } while (b < inf && steps < 8 && __dmul_rn(__longlong_as_double((long long)b), ap) < eps);
    }
    c.thr = steps >= 8 ? hb_cut_bisect(eps, ap) : b;
    return c;
}

// signed <x'|H|x> of a double read from its orbitals, with the same terms and signs as
// exc_element: same spin (grp 0 alpha, 1 beta) holes i<j -> particles a<b, sign of i->a then
// j->b; opposite spin i->a (alpha), j->b (beta)
__device__ __forceinline__ double double_element(const ProblemDev& P, int grp, uint64_t wA,
                                                 uint64_t wB, int i, int j, int a, int b) {
    if (grp < 2) {
        const uint64_t w = grp == 0 ? wA : wB;
        const int s1 = exc_sign(w, i, a);
        const uint64_t w1 = w ^ (1ull << i) ^ (1ull << a);
        const int s2 = exc_sign(w1, j, b);
        const double v = eri_at(P, i, a, j, b) - eri_at(P, j, a, i, b);
        return s1 * s2 < 0 ? -v : v;
    }
    const double v = eri_at(P, i, a, j, b);
    return exc_sign(wA, i, a) * exc_sign(wB, j, b) < 0 ? -v : v;
}

// The screened traversal of one x per warp, in six modes:
//   HB_COUNT / HB_EMIT  heat-bath set: cnt[det] = number of kept pairs, or the pairs
//                       (key, |H_x'x psi_x|) written from offs[det] on;
//   PT_COUNT / PT_EMIT  screened PT2 emissions of one hash bucket: the same test plus
//                       bucket(x') == bucket, emitting the signed H_x'x psi_x;
//   HB_APPEND / PT_APPEND  one traversal without counts: each warp stages its kept pairs in
//                       shared memory and appends them 32 at a time at a position taken from
//                       the global cursor (*cursor counts every pair; pairs at or past `cap`
//                       are not written, so *cursor > cap tells the host to retry with more
//                       room). The order of the output then depends on timing; everything
//                       downstream is order independent (a sort, exact run sums, a maximum).
// examined (may be null) accumulates the number of candidates whose coupling was tested.
enum { HB_COUNT = 0, HB_EMIT = 1, PT_COUNT = 2, PT_EMIT = 3, HB_APPEND = 5, PT_APPEND = 7 };
#define HB_STAGE 64  // staged pairs per warp (append modes)
#define HB_CQ 64     // queued double-excitation candidates per warp
#define HB_CQ_BYTES (HB_CQ * (sizeof(uint32_t) + sizeof(double)))

// shared memory of k_hb_select: pair tables, per-warp contexts and candidate queues, and in
// the append modes the per-warp staging of kept pairs
template <class K>
static size_t hb_smem(const ProblemDev& P, bool append) {
    return pair_table_bytes(P) + HB_WARPS * (sizeof(DetCtx) + HB_CQ_BYTES) +
           (append ? (size_t)HB_WARPS * HB_STAGE * (sizeof(K) + sizeof(double)) : 0);
}

template <int MODE, class K>
__global__ void __launch_bounds__(HB_THREADS, 4) k_hb_select(ProblemDev P, HashS H, HbTab T,
                                                          const ulonglong2* __restrict__ S,
                                                          const double* __restrict__ psi,
                                                          int64_t nS, double eps, uint64_t B,
                                                          uint64_t bucket,
                                                          int64_t* __restrict__ cnt,
                                                          const int64_t* __restrict__ offs,
                                                          K* __restrict__ keys,
                                                          double* __restrict__ vals,
                                                          unsigned long long* examined,
                                                          unsigned long long* __restrict__ cursor,
                                                          uint64_t cap, int nparts) {
    constexpr bool EMIT = (MODE & 1) != 0;
    constexpr bool PTM = (MODE & 2) != 0;
    constexpr bool APPEND = (MODE & 4) != 0;
    extern __shared__ __align__(16) uint8_t smem[];
    PairTables PT = setup_pair_tables(P, (uint16_t*)smem);
    DetCtx* ctx = (DetCtx*)(smem + pair_table_bytes(P)) + (threadIdx.x >> 5);
    // candidate queue of this warp (HB_CQ codes, then HB_CQ table values), after the contexts
    uint8_t* cqb = smem + pair_table_bytes(P) + HB_WARPS * sizeof(DetCtx) +
                   (threadIdx.x >> 5) * HB_CQ_BYTES;
    uint32_t* cq = (uint32_t*)cqb;
    double* cqv = (double*)(cqb + HB_CQ * sizeof(uint32_t));
    // append staging: HB_STAGE keys then HB_STAGE values per warp, after the queues
    uint8_t* stage = smem + pair_table_bytes(P) + HB_WARPS * (sizeof(DetCtx) + HB_CQ_BYTES) +
                     (threadIdx.x >> 5) * HB_STAGE * (sizeof(K) + sizeof(double));
    K* sk = (K*)stage;
    double* sv = (double*)(stage + HB_STAGE * sizeof(K));
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int n = P.norb;
    const uint32_t nsing = (uint32_t)(P.sA + P.sB);
    int qn = 0;  // staged pairs of this warp (append modes)
    // write the first `cnt_` staged pairs at a reserved position and move the rest down
    auto flush = [&](int cnt_) {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)cnt_);
        base = __shfl_sync(FULL_MASK, base, 0);
        if (lane < cnt_ && base + lane < cap) {
            keys[base + lane] = sk[lane];
            vals[base + lane] = sv[lane];
        }
        const int rest = qn - cnt_;
        K k2 = key_zero<K>();
        double v2 = 0.0;
        if (lane < rest) {
            k2 = sk[cnt_ + lane];
            v2 = sv[cnt_ + lane];
        }
        __syncwarp();
        if (lane < rest) {
            sk[lane] = k2;
            sv[lane] = v2;
        }
        __syncwarp();
        qn = rest;
    };
    // work items: (x, part) with part < nparts; part p takes the singles (p = 0) and the p-th of
    // every nparts chunks of 32 hole pairs, so the lists of one x with much work are walked by
    // several warps at once (count and append modes; the emit modes write each x's pairs in
    // order from offs[x] and take nparts = 1). Counts of several parts are added atomically
    // into cnt, which the caller zeroes.
    if (EMIT) nparts = 1;  // emit and append modes: one warp per x, without the split's cost
    const int64_t nitems = nS * (int64_t)nparts;
    for (int64_t item = (int64_t)blockIdx.x * HB_WARPS + (threadIdx.x >> 5); item < nitems;
         item += (int64_t)gridDim.x * HB_WARPS) {
        const int64_t det = nparts == 1 ? item : item / nparts;
        const int part = nparts == 1 ? 0 : (int)(item - det * nparts);
        const ulonglong2 x = S[det];
        const double py = psi[det];
        const double ap = fabs(py);
        int64_t run = (EMIT && !APPEND) ? offs[det] : 0;
        unsigned long long tested = 0;
        // m = |H| |psi| >= eps fails for every coupling when |psi| = 0 < eps, and when psi is
        // not a number: nothing to do for this x
        if (!(ap >= 0.0) || (ap == 0.0 && eps > 0.0)) {
            if (!EMIT && lane == 0 && nparts == 1) cnt[det] = 0;
            continue;
        }
        fill_ctx(P, x.x, x.y, ctx, lane);
        const HbCut cut = hb_cut(eps, ap);
        auto keep = [&](bool take, uint64_t a2, uint64_t b2, double m) {
            const unsigned bal = __ballot_sync(FULL_MASK, take);
            if (APPEND) {
                if (take) {
                    const int slot = qn + __popc(bal & lt);
                    sk[slot] = key_make<K>(a2, b2, n);
                    sv[slot] = m;
                }
                qn += __popc(bal);
                if (qn >= 32) flush(32);
            } else if (EMIT && take) {
                const int64_t pos = run + __popc(bal & lt);
                keys[pos] = key_make<K>(a2, b2, n);
                vals[pos] = m;
            }
            run += __popc(bal);
        };
        // singles: every one, with its exact element
        const HbCutFx cutfx = hb_cut_fx(cut, P);
        for (uint32_t r0 = 0; part == 0 && r0 < nsing; r0 += 32) {
            const uint32_t e = r0 + lane;
            bool take = false;
            Exc ex;
            ex.a2 = ex.b2 = 0;
            double m = 0.0;
            if (e < nsing) {
                decode_exc(P, PT, *ctx, x.x, x.y, e, ex);
                if (PTM) {
                    // the element in exact fixed point; the FP64 element only near the cut
                    const long long F = single_element_fx(P, x.x, x.y, ex);
                    const long long aF = F < 0 ? -F : F;
                    bool ok;
                    double hv = 0.0;
                    bool have_hv = false;
                    if (cutfx.all || aF >= cutfx.hi) {
                        ok = true;
                    } else if (aF <= cutfx.lo) {
                        ok = false;
                    } else {
                        hv = single_element_near_cut(P, *ctx, ex);
                        have_hv = true;
                        ok = cut.pass(fabs(hv));
                    }
                    take = ok && in_bucket_of(ex.a2, ex.b2, B, bucket) &&
                           hash_lookup(H, ex.a2, ex.b2) < 0;
                    if (EMIT && take) {
                        if (!have_hv) {  // the fixed-point element with the excitation's sign
                            const double f = ldexp(__ll2double_rn(F), -P.sfx_e);
                            hv = ex.sign < 0 ? -f : f;
                        }
                        m = __dmul_rn(hv, py);
                    }
                } else {
                    const double hv = exc_element(P, *ctx, ex);
                    const bool ok = cut.pass(fabs(hv));
                    take = ok && hash_lookup(H, ex.a2, ex.b2) < 0;
                    if (EMIT && take) m = __dmul_rn(fabs(hv), ap);
                }
            }
            keep(take, ex.a2, ex.b2, m);
        }
        if (!(APPEND && PTM) && part == 0) tested += nsing;
        // doubles: three groups of hole pairs; each lane tests the head of one list. A list is
        // walked 32 entries at a time; the entries that pass the cut and whose particles are
        // empty in x are queued (hole and particle orbitals and group in one word, with the
        // table value), and the queue is resolved 32 at a time: the configuration, the bucket
        // test, the probe into S and the element, each at full warp width
        const uint64_t wA = x.x, wB = x.y;
        int cn = 0;  // queued candidates of this warp
        auto drain = [&](int cnt_) {
            __syncwarp();
            bool take = false;
            uint64_t a2 = 0, b2 = 0;
            double m = 0.0;
            uint32_t code = 0;
            double tq = 0.0;
            if (lane < cnt_) {
                code = cq[lane];
                tq = cqv[lane];
            }
            const int rest = cn - cnt_;
            uint32_t c2 = 0;
            double t2 = 0.0;
            if (lane < rest) {
                c2 = cq[cnt_ + lane];
                t2 = cqv[cnt_ + lane];
            }
            __syncwarp();
            if (lane < rest) {
                cq[lane] = c2;
                cqv[lane] = t2;
            }
            cn = rest;
            if (lane < cnt_) {
                const int hi = code & 63, hj = (code >> 6) & 63, a = (code >> 12) & 63,
                          b = (code >> 18) & 63, grp = (int)(code >> 24);
                if (grp < 2) {
                    const uint64_t w = grp == 0 ? wA : wB;
                    const uint64_t w2 =
                        w ^ (1ull << hi) ^ (1ull << hj) ^ (1ull << a) ^ (1ull << b);
                    a2 = grp == 0 ? w2 : wA;
                    b2 = grp == 0 ? wB : w2;
                } else {
                    a2 = wA ^ (1ull << hi) ^ (1ull << a);
                    b2 = wB ^ (1ull << hj) ^ (1ull << b);
                }
                const bool inb = PTM ? in_bucket_of(a2, b2, B, bucket) : true;
                take = inb && hash_lookup(H, a2, b2) < 0;
                if (PTM && EMIT && take)
                    m = __dmul_rn(double_element(P, grp, wA, wB, hi, hj, a, b), py);
                else if (!PTM && EMIT && take)
                    m = __dmul_rn(tq, ap);
            }
            keep(take, a2, b2, m);
            __syncwarp();
        };
        for (int grp = 0; grp < 3; ++grp) {
            const int npairs = grp == 0 ? (int)choose2(P.na)
                             : grp == 1 ? (int)choose2(P.nb) : P.na * P.nb;
            const int L = grp < 2 ? T.Lss : T.Los;
            if (L == 0) continue;
            for (int p0 = 32 * part; p0 < npairs; p0 += 32 * nparts) {
                const int pi = p0 + lane;
                int i = 0, j = 0;
                int64_t base = 0;
                bool head = false;
                if (pi < npairs) {
                    if (grp < 2) {
                        const uint16_t pr = grp == 0 ? PT.occA[pi] : PT.occB[pi];
                        const uint8_t* occ = grp == 0 ? ctx->occA : ctx->occB;
                        i = occ[pr & 0xff];
                        j = occ[pr >> 8];
                        base = (int64_t)pair_index(i, j, n) * L;
                    } else {
                        const int xa = pi / P.nb, xb = pi - xa * P.nb;
                        i = ctx->occA[xa];
                        j = ctx->occB[xb];
                        base = T.os_base + (int64_t)(i * n + j) * L;
                    }
                    head = cut.pass(__ldg(&T.val[base]));
                }
                unsigned hm = __ballot_sync(FULL_MASK, head);
                while (hm) {
                    const int src = __ffs(hm) - 1;
                    hm &= hm - 1;
                    const int hi = __shfl_sync(FULL_MASK, i, src);
                    const int hj = __shfl_sync(FULL_MASK, j, src);
                    const int64_t hb = __shfl_sync(FULL_MASK, base, src);
                    // particles must be empty in x: in the alpha (grp 0) or beta (grp 1)
                    // string for same-spin pairs, a in alpha and b in beta for grp 2
                    const uint64_t wa = grp == 1 ? wB : wA, wb = grp == 0 ? wA : wB;
                    const uint32_t hcode = (uint32_t)hi | ((uint32_t)hj << 6) | ((uint32_t)grp << 24);
                    // software-pipelined walk: the next 32 entries are loaded before this
                    // chunk's candidates are tested, so the two L2 round trips overlap
                    double tv = lane < L ? __ldg(&T.val[hb + lane]) : 0.0;
                    uint16_t cd = lane < L ? __ldg(&T.code[hb + lane]) : (uint16_t)0;
                    for (int c0 = 0; c0 < L; c0 += 32) {
                        const int t = c0 + lane;
                        const bool pass = t < L && cut.pass(tv);
                        const unsigned stop = __ballot_sync(FULL_MASK, !pass);
                        double tvn = 0.0;
                        uint16_t cdn = 0;
                        if (!stop && t + 32 < L) {
                            tvn = __ldg(&T.val[hb + t + 32]);
                            cdn = __ldg(&T.code[hb + t + 32]);
                        }
                        const int a = cd & 0xff, b = cd >> 8;
                        const bool valid = pass && !((wa >> a) & 1ull) && !((wb >> b) & 1ull);
                        const unsigned vb = __ballot_sync(FULL_MASK, valid);
                        if (valid) {
                            const int slot = cn + __popc(vb & lt);
                            cq[slot] = hcode | ((uint32_t)a << 12) | ((uint32_t)b << 18);
                            if (!PTM) cqv[slot] = tv;
                        }
                        cn += __popc(vb);
                        if (cn >= 32) drain(32);
                        if (!(APPEND && PTM)) tested += stop ? (unsigned)(__ffs(stop) - 1) : 32u;
                        if (stop) break;  // sorted: every later entry fails too
                        tv = tvn;
                        cd = cdn;
                    }
                }
            }
        }
        if (cn > 0) drain(cn);
        if (!EMIT && lane == 0) {
            if (nparts == 1) cnt[det] = run;
            else atomicAdd((unsigned long long*)&cnt[det], (unsigned long long)run);
        }
        if (examined && lane == 0) atomicAdd(examined, tested);
        __syncwarp();
    }
    if (APPEND && qn > 0) flush(qn);
}

// output: one configuration per run of equal keys, with the maximum coupling of the run
// (non-negative doubles order like their bit patterns, so an integer atomicMax is exact)
template <class K>
__global__ void k_hb_out(const K* __restrict__ keys, const double* __restrict__ vals,
                         const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                         int64_t n, int norb, ulonglong2* __restrict__ out,
                         unsigned long long* __restrict__ mx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = (int64_t)pos[i] + flags[i] - 1;
        if (flags[i]) {
            uint64_t a, b;
            key_split(keys[i], norb, a, b);
            out[u] = make_ulonglong2(a, b);
        }
        atomicMax(&mx[u], (unsigned long long)__double_as_longlong(vals[i]));
    }
}

template <class K>
__global__ void k_hb_heads(const K* __restrict__ keys, int64_t n, uint32_t* __restrict__ f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// parts per configuration for the count passes: with few configurations (the strided samples
// that size the one-traversal buffers) the warps that walk the heaviest ones set the duration,
// so their lists are split over 8 warps; with many, one warp per configuration
static int hb_count_parts(int64_t n) { return n <= 32768 ? 8 : 1; }

static unsigned hb_grid(int64_t nS) {
    int64_t g = (nS + HB_WARPS - 1) / HB_WARPS;
    if (g > 148 * 16) g = 148 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

// every stride-th configuration of S and its amplitude (the sample that sizes the buffers of
// the one-traversal emission)
__global__ void k_hb_gather_stride(const ulonglong2* __restrict__ S, const double* __restrict__ psi,
                                   int64_t ns, int64_t stride, ulonglong2* __restrict__ So,
                                   double* __restrict__ po) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x) {
        So[i] = S[i * stride];
        po[i] = psi[i * stride];
    }
}

template <class K>
static int hb_run(nqs_problem* p, Scratch& sc, const HashS& H, const HbTab& T,
                  const uint64_t* dets, const double* psi, int64_t nS, double eps,
                  nqs_detset* out, cudaStream_t s) {
    const ProblemDev& P = p->d;
    const size_t smem = hb_smem<K>(P, false);
    if (smem > 48 * 1024) {
        NQS_CK(cudaFuncSetAttribute(k_hb_select<HB_COUNT, K>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NQS_CK(cudaFuncSetAttribute(k_hb_select<HB_EMIT, K>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    // One traversal appending the kept pairs (their order is then timing-dependent; the
    // reduction below, a sort and a maximum per run, is not), into buffers sized from a counted
    // sample of S (every stride-th configuration, x1.5) and enlarged once if they overflow.
    const size_t smem_a = hb_smem<K>(P, true);
    if (smem_a > 48 * 1024)
        NQS_CK(cudaFuncSetAttribute(k_hb_select<HB_APPEND, K>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a));
    unsigned long long *examined, *cursor;
    NQS_TRY(sc.get(&examined, 1));
    NQS_TRY(sc.get(&cursor, 1));
    double est;
    {
        const int64_t stride = nS > 4096 ? nS / 4096 : 1;
        const int64_t ns = (nS + stride - 1) / stride;
        Scratch es(p, s);
        ulonglong2* ds;
        double* ps;
        int64_t *c1, *o1, *t1;
        NQS_TRY(es.get(&ds, ns));
        NQS_TRY(es.get(&ps, ns));
        NQS_TRY(es.get(&c1, ns));
        NQS_TRY(es.get(&o1, ns));
        NQS_TRY(es.get(&t1, 1));
        k_hb_gather_stride<<<grid_for(ns, 256), 256, 0, s>>>((const ulonglong2*)dets, psi, ns,
                                                              stride, ds, ps);
        NQS_CK_LAUNCH();
        const int np = hb_count_parts(ns);
        if (np > 1) NQS_CK(cudaMemsetAsync(c1, 0, ns * sizeof(int64_t), s));
        {
            ProfScope prof_(PROF_HB_SELECT, s);
            k_hb_select<HB_COUNT, K><<<hb_grid(ns * np), HB_THREADS, smem, s>>>(
                P, H, T, ds, ps, ns, eps, 1, 0, c1, nullptr, nullptr, nullptr, nullptr, nullptr,
                0, np);
        }
        NQS_CK_LAUNCH();
        NQS_TRY(scan_exclusive_i64(p, es, c1, o1, ns, t1, s));
        int64_t tot = 0;
        NQS_CK(cudaMemcpyAsync(&tot, t1, sizeof tot, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        est = (double)tot * ((double)nS / (double)ns);
    }
    size_t fr = 0, totm = 0;
    NQS_CK(cudaMemGetInfo(&fr, &totm));
    uint64_t reserved = 0, used = 0;
    NQS_CK(cudaMemPoolGetAttribute(p->pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
    NQS_CK(cudaMemPoolGetAttribute(p->pool, cudaMemPoolAttrUsedMemCurrent, &used));
    const double avail = (double)fr + (double)(reserved > used ? reserved - used : 0);
    // pairs, sort buffers and the output: 2 (key + 8) + 12 bytes per pair, 90% of what is free
    const double memcap = fmin(0.9 * avail / (2.0 * (sizeof(K) + 8.0) + 12.0), 4294967295.0);
    int64_t cap = (int64_t)fmin(fmin(1.5 * est + 65536.0, (double)nS * (double)P.nexc), memcap);
    int64_t n = 0;
    K *keys = nullptr, *keys2;
    double *vals = nullptr, *vals2;
    for (int attempt = 0; attempt < 2; ++attempt) {
        NQS_TRY(sc.get(&keys, cap));
        NQS_TRY(sc.get(&vals, cap));
        NQS_CK(cudaMemsetAsync(examined, 0, sizeof(unsigned long long), s));
        NQS_CK(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s));
        {
            ProfScope prof_(PROF_HB_SELECT, s);
            k_hb_select<HB_APPEND, K><<<hb_grid(nS), HB_THREADS, smem_a, s>>>(
                P, H, T, (const ulonglong2*)dets, psi, nS, eps, 1, 0, nullptr, nullptr, keys,
                vals, examined, cursor, (uint64_t)cap, 1);
        }
        NQS_CK_LAUNCH();
        unsigned long long nc = 0, nexam = 0;
        NQS_CK(cudaMemcpyAsync(&nc, cursor, sizeof nc, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaMemcpyAsync(&nexam, examined, sizeof nexam, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        n = (int64_t)nc;
        out->n_emitted = n;
        out->n_examined = (int64_t)nexam;
        if (n <= cap) break;
        if ((double)n > memcap || n >= ((int64_t)1 << 32)) {
            nqs_record_message("nqs_hb_select: the kept pairs do not fit in device memory (or "
                               "exceed 2^32); raise eps_hb");
            return NQS_ERR_UNSUPPORTED;
        }
        cap = n;  // the exact size: one more traversal
    }
    if (n == 0) return NQS_OK;
    NQS_TRY(sc.get(&keys2, n));
    NQS_TRY(sc.get(&vals2, n));
    if (sizeof(K) == 4)
        NQS_TRY(radix_sort_pairs32(p, sc, (uint32_t*&)keys, vals, (uint32_t*&)keys2, vals2, n,
                                   2 * P.norb, s));
    else if (sizeof(K) == 8)
        NQS_TRY(radix_sort_pairs(p, sc, (uint64_t*&)keys, vals, (uint64_t*&)keys2, vals2, n,
                                 2 * P.norb, s));
    else
        NQS_TRY(radix_sort_pairs128(p, sc, (Key128*&)keys, vals, (Key128*&)keys2, vals2, n,
                                    2 * P.norb, s));
    uint32_t* flags = (uint32_t*)vals2;
    uint32_t* pos = flags + n;
    k_hb_heads<K><<<grid_for(n, 256), 256, 0, s>>>(keys, n, flags);
    NQS_CK_LAUNCH();
    NQS_TRY(scan_exclusive_u32(p, sc, flags, pos, n, s));
    uint32_t last_pos = 0, last_flag = 0;
    NQS_CK(cudaMemcpyAsync(&last_pos, pos + n - 1, 4, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaMemcpyAsync(&last_flag, flags + n - 1, 4, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    const int64_t nu = (int64_t)last_pos + last_flag;
    uint64_t* od = nullptr;
    double* om = nullptr;
    if (cudaMalloc(&od, nu * 2 * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&om, nu * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(od);
        return NQS_ERR_OOM;
    }
    out->dets = od;
    out->value = om;
    out->n = nu;
    NQS_CK(cudaMemsetAsync(om, 0, nu * sizeof(double), s));
    k_hb_out<K><<<grid_for(n, 256), 256, 0, s>>>(keys, vals, flags, pos, n, P.norb,
                                                 (ulonglong2*)od, (unsigned long long*)om);
    NQS_CK_LAUNCH();
    NQS_CK(cudaStreamSynchronize(s));
    return NQS_OK;
}

// One pass of the screened PT2 emission for bucket `bucket` of B: with cnt, the per-x counts;
// otherwise the (key, H_x'x psi_x) pairs written at offs (keys of the width 2 norb needs).
template <class K>
static int hb_pt2_pass_k(nqs_problem* p, const HbTab& T, const HashS& H, const uint64_t* dets,
                         const double* psi, int64_t nS, double eps, uint64_t B, uint64_t bucket,
                         int64_t* cnt, const int64_t* offs, void* keys, double* vals,
                         cudaStream_t s) {
    const ProblemDev& P = p->d;
    const size_t smem = hb_smem<K>(P, false);
    if (smem > 48 * 1024) {
        NQS_CK(cudaFuncSetAttribute(k_hb_select<PT_COUNT, K>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NQS_CK(cudaFuncSetAttribute(k_hb_select<PT_EMIT, K>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (cnt) {
        const int np = hb_count_parts(nS);
        if (np > 1) NQS_CK(cudaMemsetAsync(cnt, 0, nS * sizeof(int64_t), s));
        ProfScope prof_(PROF_PT2_COUNT, s);
        k_hb_select<PT_COUNT, K><<<hb_grid(nS * np), HB_THREADS, smem, s>>>(
            P, H, T, (const ulonglong2*)dets, psi, nS, eps, B, bucket, cnt, nullptr, nullptr,
            nullptr, nullptr, nullptr, 0, np);
    } else {
        ProfScope prof_(PROF_PT2_EMIT, s);
        k_hb_select<PT_EMIT, K><<<hb_grid(nS), HB_THREADS, smem, s>>>(
            P, H, T, (const ulonglong2*)dets, psi, nS, eps, B, bucket, nullptr, offs, (K*)keys,
            vals, nullptr, nullptr, 0, 1);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int hb_pt2_pass(nqs_problem* p, const HashS& H, const uint64_t* dets, const double* psi,
                int64_t nS, double eps, uint64_t B, uint64_t bucket, int64_t* cnt,
                const int64_t* offs, void* keys, double* vals, cudaStream_t s) {
    HbTab T;
    NQS_TRY(hb_tables(p, &T));
    const int kbits = 2 * p->d.norb;
    if (kbits <= 32)
        return hb_pt2_pass_k<uint32_t>(p, T, H, dets, psi, nS, eps, B, bucket, cnt, offs, keys,
                                       vals, s);
    if (kbits <= 64)
        return hb_pt2_pass_k<uint64_t>(p, T, H, dets, psi, nS, eps, B, bucket, cnt, offs, keys,
                                       vals, s);
    return hb_pt2_pass_k<Key128>(p, T, H, dets, psi, nS, eps, B, bucket, cnt, offs, keys, vals,
                                 s);
}

// The screened PT2 emissions of all of C\S in one traversal (PT_APPEND): the pairs go to
// keys / vals [cap] in an order that depends on timing; *cursor_dev (zeroed here) receives the
// number of pairs, which exceeds cap when the buffers were too small (then nothing past cap
// was written and the caller must retry or split into buckets).
template <class K>
static int hb_pt2_append_k(nqs_problem* p, const HbTab& T, const HashS& H, const uint64_t* dets,
                           const double* psi, int64_t nS, double eps, void* keys, double* vals,
                           int64_t cap, unsigned long long* cursor_dev, cudaStream_t s) {
    const ProblemDev& P = p->d;
    const size_t smem = hb_smem<K>(P, true);
    if (smem > 48 * 1024)
        NQS_CK(cudaFuncSetAttribute(k_hb_select<PT_APPEND, K>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    NQS_CK(cudaMemsetAsync(cursor_dev, 0, sizeof(unsigned long long), s));
    {
        ProfScope prof_(PROF_PT2_EMIT, s);
        k_hb_select<PT_APPEND, K><<<hb_grid(nS), HB_THREADS, smem, s>>>(
            P, H, T, (const ulonglong2*)dets, psi, nS, eps, 1, 0, nullptr, nullptr, (K*)keys,
            vals, nullptr, cursor_dev, (uint64_t)cap, 1);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int hb_pt2_append(nqs_problem* p, const HashS& H, const uint64_t* dets, const double* psi,
                  int64_t nS, double eps, void* keys, double* vals, int64_t cap,
                  unsigned long long* cursor_dev, cudaStream_t s) {
    HbTab T;
    NQS_TRY(hb_tables(p, &T));
    const int kbits = 2 * p->d.norb;
    if (kbits <= 32)
        return hb_pt2_append_k<uint32_t>(p, T, H, dets, psi, nS, eps, keys, vals, cap, cursor_dev,
                                         s);
    if (kbits <= 64)
        return hb_pt2_append_k<uint64_t>(p, T, H, dets, psi, nS, eps, keys, vals, cap, cursor_dev,
                                         s);
    return hb_pt2_append_k<Key128>(p, T, H, dets, psi, nS, eps, keys, vals, cap, cursor_dev, s);
}

extern "C" int nqs_hb_select(nqs_problem* p, const uint64_t* dets, const double* psi, int64_t nS,
                             double eps_hb, const nqs_opts* opts, nqs_detset* out,
                             nqs_stream_t stream) {
    if (!p || !dets || !psi || !out || nS <= 0 || !(eps_hb >= 0.0)) return NQS_ERR_ARG;
    if (((uintptr_t)dets) & 15) return NQS_ERR_ARG;
    if (nS >= ((int64_t)1 << 31)) return NQS_ERR_UNSUPPORTED;
    out->dets = nullptr;
    out->value = nullptr;
    out->index = nullptr;
    out->n = out->n_emitted = out->n_examined = 0;
    cudaStream_t s = (cudaStream_t)stream;
    nqs_opts def;
    if (!opts) {
        nqs_opts_default(&def);
        opts = &def;
    }
    HbTab T;
    NQS_TRY(hb_tables(p, &T));
    Scratch sc(p, s);
    if (opts->validate) NQS_TRY(validate_dets(p, sc, dets, nS, true, s));
    HashS H;
    NQS_TRY(hash_build(p, sc, dets, nS, &H, s));
    int st;
    const int kbits = 2 * p->d.norb;
    if (kbits <= 32) st = hb_run<uint32_t>(p, sc, H, T, dets, psi, nS, eps_hb, out, s);
    else if (kbits <= 64) st = hb_run<uint64_t>(p, sc, H, T, dets, psi, nS, eps_hb, out, s);
    else st = hb_run<Key128>(p, sc, H, T, dets, psi, nS, eps_hb, out, s);
    if (st < 0) nqs_detset_free(out);
    return st;
}

extern "C" int nqs_detset_free(nqs_detset* d) {
    if (!d) return NQS_OK;
    cudaFree(d->dets);
    cudaFree(d->value);
    cudaFree(d->index);
    d->dets = nullptr;
    d->value = nullptr;
    d->index = nullptr;
    d->n = 0;
    return NQS_OK;
}

// Device-side Slater-Condon machinery: per-det occupation lists, decoding of the canonical
// excitation index, excitation signs, matrix elements and the diagonal element.
//
// Canonical excitation order of one det (class offsets in ProblemDev):
//   class 0  alpha singles       i in occ_a asc, a in vir_a asc
//   class 1  beta singles        same for beta
//   class 2  alpha-alpha doubles hole pair (i<j) lexicographic, then particle pair (a<b)
//   class 3  beta-beta doubles
//   class 4  alpha-beta doubles  (i_a, a_a) single index major, (j_b, b_b) minor, b fastest
// The matrix-element summation order below is the library's canonical order; it makes H_SS
// symmetric bit for bit (the same terms are added in the same order from either side).
#pragma once
#include "nqs_internal.cuh"

#define FULL_MASK 0xffffffffu

// per-warp occupation lists of the det being processed
struct DetCtx {
    uint8_t occA[64];
    uint8_t virA[64];
    uint8_t occB[64];
    uint8_t virB[64];
};

// pair tables (shared by all warps of a CTA): entry = lo | hi << 8, lo < hi, lexicographic
struct PairTables {
    const uint16_t* occA;
    const uint16_t* virA;
    const uint16_t* occB;
    const uint16_t* virB;
};

__host__ __device__ __forceinline__ int64_t choose2(int64_t n) { return n * (n - 1) / 2; }

// shared-memory bytes needed for the pair tables of a problem (16-byte rounded)
__host__ __device__ __forceinline__ size_t pair_table_bytes(const ProblemDev& P) {
    size_t n = choose2(P.na) + choose2(P.ma) + choose2(P.nb) + choose2(P.mb);
    return (n * sizeof(uint16_t) + 15) & ~(size_t)15;
}

// fill the pair tables cooperatively (whole CTA), then __syncthreads()
__device__ __forceinline__ PairTables setup_pair_tables(const ProblemDev& P, uint16_t* base) {
    PairTables T;
    T.occA = base;
    T.virA = T.occA + choose2(P.na);
    T.occB = T.virA + choose2(P.ma);
    T.virB = T.occB + choose2(P.nb);
    int sizes[4] = {P.na, P.ma, P.nb, P.mb};
    uint16_t* outs[4] = {(uint16_t*)T.occA, (uint16_t*)T.virA, (uint16_t*)T.occB,
                         (uint16_t*)T.virB};
    for (int t = 0; t < 4; ++t) {
        int n = sizes[t];
        int total = (int)choose2(n);
        for (int k = threadIdx.x; k < total; k += blockDim.x) {
            // invert k = lo*(2n-lo-1)/2 + (hi-lo-1) by walking rows (n <= 64)
            int lo = 0, rem = k;
            while (rem >= n - 1 - lo) {
                rem -= n - 1 - lo;
                ++lo;
            }
            int hi = lo + 1 + rem;
            outs[t][k] = (uint16_t)(lo | (hi << 8));
        }
    }
    __syncthreads();
    return T;
}

// lane-parallel construction of the occupation lists of det (A, B); ends with __syncwarp
__device__ __forceinline__ void fill_ctx(const ProblemDev& P, uint64_t A, uint64_t B, DetCtx* c,
                                         int lane) {
    for (int p = lane; p < P.norb; p += 32) {
        uint64_t below = (p == 0) ? 0ull : ((1ull << p) - 1ull);
        int ka = __popcll(A & below), kb = __popcll(B & below);
        if ((A >> p) & 1ull) c->occA[ka] = (uint8_t)p;
        else c->virA[p - ka] = (uint8_t)p;
        if ((B >> p) & 1ull) c->occB[kb] = (uint8_t)p;
        else c->virB[p - kb] = (uint8_t)p;
    }
    __syncwarp();
}

struct Exc {
    uint64_t a2, b2;  // the excited det
    int cls;          // 0..4
    int i, a, j, b;   // holes i(, j) and particles a(, b); j, b unused for singles
    int sign;         // +1 / -1
};

// decode canonical index e (< P.nexc) of det (A, B)
__device__ __forceinline__ void decode_exc(const ProblemDev& P, const PairTables& T,
                                           const DetCtx& c, uint64_t A, uint64_t B, uint32_t e,
                                           Exc& x) {
    const uint32_t o1 = (uint32_t)P.sA, o2 = o1 + (uint32_t)P.sB, o3 = o2 + (uint32_t)P.dAA,
                   o4 = o3 + (uint32_t)P.dBB;
    if (e < o2) {
        bool alpha = e < o1;
        uint32_t l = alpha ? e : e - o1;
        uint32_t m = alpha ? P.ma : P.mb;
        uint32_t xo = l / m, yv = l - xo * m;
        int i = alpha ? c.occA[xo] : c.occB[xo];
        int a = alpha ? c.virA[yv] : c.virB[yv];
        uint64_t w = alpha ? A : B;
        uint64_t w2 = w ^ (1ull << i) ^ (1ull << a);
        x.cls = alpha ? 0 : 1;
        x.i = i;
        x.a = a;
        x.j = -1;
        x.b = -1;
        x.sign = exc_sign(w, i, a);
        x.a2 = alpha ? w2 : A;
        x.b2 = alpha ? B : w2;
    } else if (e < o4) {
        bool alpha = e < o3;
        uint32_t l = alpha ? e - o2 : e - o3;
        uint32_t Q = (uint32_t)(alpha ? choose2(P.ma) : choose2(P.mb));
        uint32_t pi = l / Q, qi = l - pi * Q;
        uint16_t po = alpha ? T.occA[pi] : T.occB[pi];
        uint16_t pv = alpha ? T.virA[qi] : T.virB[qi];
        const uint8_t* occ = alpha ? c.occA : c.occB;
        const uint8_t* vir = alpha ? c.virA : c.virB;
        int i = occ[po & 0xff], j = occ[po >> 8];
        int a = vir[pv & 0xff], b = vir[pv >> 8];
        uint64_t w = alpha ? A : B;
        int s1 = exc_sign(w, i, a);
        uint64_t w1 = w ^ (1ull << i) ^ (1ull << a);
        int s2 = exc_sign(w1, j, b);
        uint64_t w2 = w1 ^ (1ull << j) ^ (1ull << b);
        x.cls = alpha ? 2 : 3;
        x.i = i;
        x.j = j;
        x.a = a;
        x.b = b;
        x.sign = s1 * s2;
        x.a2 = alpha ? w2 : A;
        x.b2 = alpha ? B : w2;
    } else {
        uint32_t l = e - o4;
        uint32_t sB = (uint32_t)P.sB;
        uint32_t la = l / sB, lb = l - la * sB;
        uint32_t xa = la / P.ma, ya = la - xa * P.ma;
        uint32_t xb = lb / P.mb, yb = lb - xb * P.mb;
        int i = c.occA[xa], a = c.virA[ya], j = c.occB[xb], b = c.virB[yb];
        x.cls = 4;
        x.i = i;
        x.a = a;
        x.j = j;
        x.b = b;
        x.sign = exc_sign(A, i, a) * exc_sign(B, j, b);
        x.a2 = A ^ (1ull << i) ^ (1ull << a);
        x.b2 = B ^ (1ull << j) ^ (1ull << b);
    }
}

// only the excited det (cheaper than decode_exc when the element is not needed)
__device__ __forceinline__ void decode_key(const ProblemDev& P, const PairTables& T,
                                           const DetCtx& c, uint64_t A, uint64_t B, uint32_t e,
                                           uint64_t& a2, uint64_t& b2) {
    const uint32_t o1 = (uint32_t)P.sA, o2 = o1 + (uint32_t)P.sB, o3 = o2 + (uint32_t)P.dAA,
                   o4 = o3 + (uint32_t)P.dBB;
    if (e < o2) {
        bool alpha = e < o1;
        uint32_t l = alpha ? e : e - o1;
        uint32_t m = alpha ? P.ma : P.mb;
        uint32_t xo = l / m, yv = l - xo * m;
        int i = alpha ? c.occA[xo] : c.occB[xo];
        int a = alpha ? c.virA[yv] : c.virB[yv];
        uint64_t f = (1ull << i) ^ (1ull << a);
        a2 = alpha ? A ^ f : A;
        b2 = alpha ? B : B ^ f;
    } else if (e < o4) {
        bool alpha = e < o3;
        uint32_t l = alpha ? e - o2 : e - o3;
        uint32_t Q = (uint32_t)(alpha ? choose2(P.ma) : choose2(P.mb));
        uint32_t pi = l / Q, qi = l - pi * Q;
        uint16_t po = alpha ? T.occA[pi] : T.occB[pi];
        uint16_t pv = alpha ? T.virA[qi] : T.virB[qi];
        const uint8_t* occ = alpha ? c.occA : c.occB;
        const uint8_t* vir = alpha ? c.virA : c.virB;
        uint64_t f = (1ull << occ[po & 0xff]) ^ (1ull << occ[po >> 8]) ^ (1ull << vir[pv & 0xff]) ^
                     (1ull << vir[pv >> 8]);
        a2 = alpha ? A ^ f : A;
        b2 = alpha ? B : B ^ f;
    } else {
        uint32_t l = e - o4;
        uint32_t sB = (uint32_t)P.sB;
        uint32_t la = l / sB, lb = l - la * sB;
        uint32_t xa = la / P.ma, ya = la - xa * P.ma;
        uint32_t xb = lb / P.mb, yb = lb - xb * P.mb;
        a2 = A ^ (1ull << c.occA[xa]) ^ (1ull << c.virA[ya]);
        b2 = B ^ (1ull << c.occB[xb]) ^ (1ull << c.virB[yb]);
    }
}

// Incremental enumeration of excited keys for a lane whose canonical index grows by 32 between
// calls (a warp walking the connected set in rounds of 32): singles decode directly; same-spin
// doubles keep their hole-pair / particle-pair positions and alpha-beta doubles their positions
// in the occupied and virtual lists, and step them by 32 without dividing.
struct EnumPos {
    int cls;             // class of the lane's current index (-1: not located yet)
    int pi, qi;          // same-spin doubles: hole-pair and particle-pair positions
    int xa, ya, xb, yb;  // alpha-beta doubles: positions in the occupied / virtual lists
    int d_hi, d_lo;      // a step of 32 in the current class: 32 = d_hi * (inner size) + d_lo
};

__device__ __forceinline__ void ab_locate(const ProblemDev& P, uint32_t l, EnumPos& q) {
    const uint32_t sB = (uint32_t)P.sB;
    const uint32_t la = l / sB, lb = l - la * sB;
    q.xa = (int)(la / (uint32_t)P.ma);
    q.ya = (int)(la - (uint32_t)q.xa * (uint32_t)P.ma);
    q.xb = (int)(lb / (uint32_t)P.mb);
    q.yb = (int)(lb - (uint32_t)q.xb * (uint32_t)P.mb);
    q.d_hi = 32 / P.mb;
    q.d_lo = 32 - q.d_hi * P.mb;
    q.cls = 4;
}

// (xa, ya, xb, yb) of the index 32 further on: add 32 = d_hi * mb + d_lo to (xb, yb), then
// carry whole beta-hole rounds into the alpha positions
__device__ __forceinline__ void ab_advance32(const ProblemDev& P, EnumPos& q) {
    q.yb += q.d_lo;
    q.xb += q.d_hi;
    if (q.yb >= P.mb) {
        q.yb -= P.mb;
        ++q.xb;
    }
    while (q.xb >= P.nb) {
        q.xb -= P.nb;
        if (++q.ya == P.ma) {
            q.ya = 0;
            ++q.xa;
        }
    }
}

// same-spin doubles: position of canonical offset l (first call in the class), or 32 further on
__device__ __forceinline__ void ss_step(uint32_t l, int cls, int Q, EnumPos& q) {
    if (q.cls != cls) {
        q.pi = (int)(l / (uint32_t)Q);
        q.qi = (int)(l - (uint32_t)q.pi * (uint32_t)Q);
        q.d_hi = 32 / Q;
        q.d_lo = 32 - q.d_hi * Q;
        q.cls = cls;
    } else {
        q.qi += q.d_lo;
        q.pi += q.d_hi;
        if (q.qi >= Q) {
            q.qi -= Q;
            ++q.pi;
        }
    }
}

// the excited det of canonical index e (this lane's next index: e grows by 32 between calls).
// Singles decode directly; same-spin and alpha-beta doubles step their positions by 32.
__device__ __forceinline__ void step_key(const ProblemDev& P, const PairTables& T,
                                          const DetCtx& c, uint64_t A, uint64_t B, uint32_t e,
                                          uint32_t o2, uint32_t o3, uint32_t o4, EnumPos& q,
                                          uint64_t& a2, uint64_t& b2) {
    if (e < o2) {
        decode_key(P, T, c, A, B, e, a2, b2);
        return;
    }
    if (e < o4) {
        const bool alpha = e < o3;
        const int Q = (int)(alpha ? choose2(P.ma) : choose2(P.mb));
        ss_step(e - (alpha ? o2 : o3), alpha ? 2 : 3, Q, q);
        const uint16_t po = alpha ? T.occA[q.pi] : T.occB[q.pi];
        const uint16_t pv = alpha ? T.virA[q.qi] : T.virB[q.qi];
        const uint8_t* occ = alpha ? c.occA : c.occB;
        const uint8_t* vir = alpha ? c.virA : c.virB;
        const uint64_t f = (1ull << occ[po & 0xff]) ^ (1ull << occ[po >> 8]) ^
                           (1ull << vir[pv & 0xff]) ^ (1ull << vir[pv >> 8]);
        a2 = alpha ? A ^ f : A;
        b2 = alpha ? B : B ^ f;
        return;
    }
    if (q.cls != 4) ab_locate(P, e - o4, q);
    else ab_advance32(P, q);
    a2 = A ^ (1ull << c.occA[q.xa]) ^ (1ull << c.virA[q.ya]);
    b2 = B ^ (1ull << c.occB[q.xb]) ^ (1ull << c.virB[q.yb]);
}

// the full excitation of canonical index e, with the same incremental positions as step_key
// (the same values as decode_exc)
__device__ __forceinline__ void step_exc(const ProblemDev& P, const PairTables& T,
                                         const DetCtx& c, uint64_t A, uint64_t B, uint32_t e,
                                         uint32_t o2, uint32_t o3, uint32_t o4, EnumPos& q,
                                         Exc& x) {
    if (e < o2) {
        decode_exc(P, T, c, A, B, e, x);
        return;
    }
    if (e < o4) {
        const bool alpha = e < o3;
        const int Q = (int)(alpha ? choose2(P.ma) : choose2(P.mb));
        ss_step(e - (alpha ? o2 : o3), alpha ? 2 : 3, Q, q);
        const uint16_t po = alpha ? T.occA[q.pi] : T.occB[q.pi];
        const uint16_t pv = alpha ? T.virA[q.qi] : T.virB[q.qi];
        const uint8_t* occ = alpha ? c.occA : c.occB;
        const uint8_t* vir = alpha ? c.virA : c.virB;
        const int i = occ[po & 0xff], j = occ[po >> 8];
        const int a = vir[pv & 0xff], b = vir[pv >> 8];
        const uint64_t w = alpha ? A : B;
        const int s1 = exc_sign(w, i, a);
        const uint64_t w1 = w ^ (1ull << i) ^ (1ull << a);
        const int s2 = exc_sign(w1, j, b);
        const uint64_t w2 = w1 ^ (1ull << j) ^ (1ull << b);
        x.cls = alpha ? 2 : 3;
        x.i = i;
        x.j = j;
        x.a = a;
        x.b = b;
        x.sign = s1 * s2;
        x.a2 = alpha ? w2 : A;
        x.b2 = alpha ? B : w2;
        return;
    }
    if (q.cls != 4) ab_locate(P, e - o4, q);
    else ab_advance32(P, q);
    const int i = c.occA[q.xa], a = c.virA[q.ya], j = c.occB[q.xb], b = c.virB[q.yb];
    x.cls = 4;
    x.i = i;
    x.a = a;
    x.j = j;
    x.b = b;
    x.sign = exc_sign(A, i, a) * exc_sign(B, j, b);
    x.a2 = A ^ (1ull << i) ^ (1ull << a);
    x.b2 = B ^ (1ull << j) ^ (1ull << b);
}

// Alpha-beta doubles from per-configuration tables (the emission kernels): the beta single of
// index lb = xb * mb + yb as its excited string and its ERI column offset j * norb + b with the
// sign of the beta move in bit 31; the alpha single's string, ERI row offset
// (i * norb + a) * norb^2 and sign stay in registers while the alpha index stays. Element and
// key are those of decode_exc / exc_element bit for bit: eri[(((i n + a) n + j) n + b)] with the
// product of the two single signs.
struct AbTab {
    uint64_t* bmask;  // [sB]
    uint32_t* bco;    // [sB]
};
__host__ __device__ __forceinline__ size_t ab_tab_bytes(const ProblemDev& P) {
    return ((size_t)P.sB * 12 + 15) & ~(size_t)15;
}
__device__ __forceinline__ AbTab ab_tab_at(uint8_t* base, const ProblemDev& P) {
    AbTab t;
    t.bmask = (uint64_t*)base;
    t.bco = (uint32_t*)(base + (size_t)P.sB * 8);
    return t;
}
// lane-parallel fill for configuration (., B) with occupation lists c; ends with __syncwarp
__device__ __forceinline__ void fill_ab_tab(const ProblemDev& P, const DetCtx& c, uint64_t B,
                                            AbTab t, int lane) {
    const int n = P.norb;
    for (int lb = lane; lb < P.sB; lb += 32) {
        const int xb = lb / P.mb, yb = lb - xb * P.mb;
        const int j = c.occB[xb], b = c.virB[yb];
        t.bmask[lb] = B ^ (1ull << j) ^ (1ull << b);
        t.bco[lb] = (uint32_t)(j * n + b) | (exc_sign(B, j, b) < 0 ? 0x80000000u : 0u);
    }
    __syncwarp();
}
struct AbState {
    int on;            // located yet
    int xa, ya, lb;    // alpha hole / particle positions, beta single index
    uint64_t a2;       // the alpha string
    uint32_t ro, sa;   // ERI row offset, alpha sign in bit 31
};
__device__ __forceinline__ void ab_load_alpha(const ProblemDev& P, const DetCtx& c, uint64_t A,
                                              AbState& s) {
    const int n = P.norb, i = c.occA[s.xa], a = c.virA[s.ya];
    s.a2 = A ^ (1ull << i) ^ (1ull << a);
    s.ro = (uint32_t)((i * n + a) * n * n);
    s.sa = exc_sign(A, i, a) < 0 ? 0x80000000u : 0u;
}
// the alpha-beta excitation of canonical offset l = e - o4 (first call) or 32 further on
__device__ __forceinline__ void ab_fast_step(const ProblemDev& P, const DetCtx& c, uint64_t A,
                                             uint32_t l, AbState& s) {
    if (!s.on) {
        const uint32_t sB = (uint32_t)P.sB;
        const uint32_t la = l / sB;
        s.lb = (int)(l - la * sB);
        s.xa = (int)(la / (uint32_t)P.ma);
        s.ya = (int)(la - (uint32_t)s.xa * (uint32_t)P.ma);
        s.on = 1;
        ab_load_alpha(P, c, A, s);
        return;
    }
    s.lb += 32;
    if (s.lb >= P.sB) {
        do {
            s.lb -= P.sB;
            if (++s.ya == P.ma) {
                s.ya = 0;
                ++s.xa;
            }
        } while (s.lb >= P.sB);
        ab_load_alpha(P, c, A, s);
    }
}
// H_x'x (signed) of the current alpha-beta excitation and its beta string
__device__ __forceinline__ double ab_fast_element(const ProblemDev& P, const AbTab& t,
                                                  const AbState& s, uint64_t& b2) {
    b2 = t.bmask[s.lb];
    const uint32_t co = t.bco[s.lb];
    const double v = __ldg(&P.eri[s.ro + (co & 0x7fffffffu)]);
    return __longlong_as_double(__double_as_longlong(v) ^
                                ((long long)((s.sa ^ co) >> 31) << 63));
}

__device__ __forceinline__ double eri_at(const ProblemDev& P, int p, int q, int r, int s) {
    const int n = P.norb;
    return __ldg(&P.eri[(((size_t)p * n + q) * n + r) * n + s]);
}

// <x'|H|x> for the decoded excitation x of det with occupation lists c.
//   single i->a of spin s: h_ia + sum_{j in occ_a, j != i (if s=a)} t_a(j)
//                               + sum_{j in occ_b, j != i (if s=b)} t_b(j),
//     t(j) = (ia|jj) - (ij|ja) for j of spin s, (ia|jj) otherwise (ascending j, alpha first);
//   same-spin double: (ia|jb) - (ib|ja); alpha-beta double: (ia|jb); times the sign.
__device__ __forceinline__ double exc_element(const ProblemDev& P, const DetCtx& c, const Exc& x) {
    double v;
    const int n = P.norb;
    if (x.cls <= 1) {
        const size_t base = ((size_t)x.i * n + x.a) * n;
        v = __ldg(&P.h[x.i * n + x.a]);
        const bool alpha = x.cls == 0;
        for (int k = 0; k < P.na; ++k) {
            int j = c.occA[k];
            if (alpha) {
                if (j == x.i) continue;
                v = v + __ldg(&P.TD[base + j]);
            } else {
                v = v + __ldg(&P.TJ[base + j]);
            }
        }
        for (int k = 0; k < P.nb; ++k) {
            int j = c.occB[k];
            if (!alpha) {
                if (j == x.i) continue;
                v = v + __ldg(&P.TD[base + j]);
            } else {
                v = v + __ldg(&P.TJ[base + j]);
            }
        }
    } else if (x.cls <= 3) {
        // (ib|ja) read as (ja|ib): equal bit for bit under the eightfold symmetry
        v = eri_at(P, x.i, x.a, x.j, x.b) - eri_at(P, x.j, x.a, x.i, x.b);
    } else {
        v = eri_at(P, x.i, x.a, x.j, x.b);
    }
    // the sign as a flip of the sign bit (the same value as -v, without an FP64 instruction)
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(x.sign < 0) << 63));
}

// The element of a single (x.cls <= 1) in fixed point, without its sign: the integer sum of the
// same terms as exc_element, each table entry rounded once to the grid 2^-P.sfx_e, so it is
// exact and differs from exc_element's FP64 sum by at most 49 half-units of the grid plus that
// sum's own rounding (at most 48 ulps of hoff_max). The sums over the occupied orbitals j of the
// configuration (wA, wB) come from the byte tables, one entry per byte of each string; the
// same-spin sum there includes j = i, whose term is subtracted (integer sums: exact in any
// grouping).
__device__ __forceinline__ long long single_element_fx(const ProblemDev& P, uint64_t wA,
                                                       uint64_t wB, const Exc& x) {
    const int n = P.norb, nb = P.nbytes;
    const size_t ia = (size_t)x.i * n + x.a;
    const bool alpha = x.cls == 0;
    const uint64_t ws = alpha ? wA : wB, wo = alpha ? wB : wA;  // same spin, other spin
    const long long* same = P.SDt + ia * nb * 256;
    const long long* other = P.SJt + ia * nb * 256;
    long long v = __ldg(&P.hfx_off[ia]) - __ldg(&P.TDfx[ia * n + x.i]);
    for (int k = 0; k < nb; ++k) {
        v += __ldg(&same[k * 256 + (int)((ws >> (8 * k)) & 255ull)]);
        v += __ldg(&other[k * 256 + (int)((wo >> (8 * k)) & 255ull)]);
    }
    return v;
}

// H_xx: sum_{occ} h_ii + sum_{i<j same spin} [J_ij - K_ij] + sum_{i alpha, j beta} J_ij, in the
// order alpha h, beta h, alpha pairs, beta pairs, alpha-beta pairs (one running sum).
__device__ __forceinline__ double diag_element_impl(const ProblemDev& P, uint64_t a, uint64_t b) {
    const int n = P.norb;
    double e = 0.0;
    for (uint64_t w = a; w; w &= w - 1) {
        int i = __ffsll((long long)w) - 1;
        e = e + __ldg(&P.h[i * n + i]);
    }
    for (uint64_t w = b; w; w &= w - 1) {
        int i = __ffsll((long long)w) - 1;
        e = e + __ldg(&P.h[i * n + i]);
    }
    for (uint64_t wi = a; wi; wi &= wi - 1) {
        int i = __ffsll((long long)wi) - 1;
        for (uint64_t wj = wi & (wi - 1); wj; wj &= wj - 1) {
            int j = __ffsll((long long)wj) - 1;
            double t = __ldg(&P.J[i * n + j]) - __ldg(&P.K[i * n + j]);
            e = e + t;
        }
    }
    for (uint64_t wi = b; wi; wi &= wi - 1) {
        int i = __ffsll((long long)wi) - 1;
        for (uint64_t wj = wi & (wi - 1); wj; wj &= wj - 1) {
            int j = __ffsll((long long)wj) - 1;
            double t = __ldg(&P.J[i * n + j]) - __ldg(&P.K[i * n + j]);
            e = e + t;
        }
    }
    for (uint64_t wi = a; wi; wi &= wi - 1) {
        int i = __ffsll((long long)wi) - 1;
        for (uint64_t wj = b; wj; wj &= wj - 1) {
            int j = __ffsll((long long)wj) - 1;
            e = e + __ldg(&P.J[i * n + j]);
        }
    }
    return e;
}

// H_xx with the one-body diagonal hd[p] = h_pp and the J/K tables in shared memory; the same
// terms in the same order as diag_element_impl (bit-identical result)
__device__ __forceinline__ double diag_element_smem(int n, const double* hd, const double* J,
                                                    const double* K, uint64_t a, uint64_t b) {
    double e = 0.0;
    for (uint64_t w = a; w; w &= w - 1) e = e + hd[__ffsll((long long)w) - 1];
    for (uint64_t w = b; w; w &= w - 1) e = e + hd[__ffsll((long long)w) - 1];
    for (uint64_t wi = a; wi; wi &= wi - 1) {
        const int i = __ffsll((long long)wi) - 1;
        for (uint64_t wj = wi & (wi - 1); wj; wj &= wj - 1) {
            const int j = __ffsll((long long)wj) - 1;
            const double t = J[i * n + j] - K[i * n + j];
            e = e + t;
        }
    }
    for (uint64_t wi = b; wi; wi &= wi - 1) {
        const int i = __ffsll((long long)wi) - 1;
        for (uint64_t wj = wi & (wi - 1); wj; wj &= wj - 1) {
            const int j = __ffsll((long long)wj) - 1;
            const double t = J[i * n + j] - K[i * n + j];
            e = e + t;
        }
    }
    for (uint64_t wi = a; wi; wi &= wi - 1) {
        const int i = __ffsll((long long)wi) - 1;
        for (uint64_t wj = b; wj; wj &= wj - 1) e = e + J[i * n + __ffsll((long long)wj) - 1];
    }
    return e;
}

// H_xx accumulated exactly in 64-bit fixed point (tables in shared memory), converted once to
// FP64: integer adds instead of FP64 adds (FP64 issues at a small fraction of the FP32/INT32
// rate on this GPU). Same terms as diag_element_impl; the sum itself is exact, so the only
// difference from an FP64 sum is the one rounding of each table entry (~2^-52 relative).
__device__ __forceinline__ double diag_element_fixed(int n, const long long* hf,
                                                     const long long* jk, const long long* jf,
                                                     double dscale, uint64_t a, uint64_t b) {
    long long e = 0;
    for (uint64_t w = a; w; w &= w - 1) e += hf[__ffsll((long long)w) - 1];
    for (uint64_t w = b; w; w &= w - 1) e += hf[__ffsll((long long)w) - 1];
    for (uint64_t wi = a; wi; wi &= wi - 1) {
        const long long* row = jk + (__ffsll((long long)wi) - 1) * n;
        for (uint64_t wj = wi & (wi - 1); wj; wj &= wj - 1) e += row[__ffsll((long long)wj) - 1];
    }
    for (uint64_t wi = b; wi; wi &= wi - 1) {
        const long long* row = jk + (__ffsll((long long)wi) - 1) * n;
        for (uint64_t wj = wi & (wi - 1); wj; wj &= wj - 1) e += row[__ffsll((long long)wj) - 1];
    }
    for (uint64_t wi = a; wi; wi &= wi - 1) {
        const long long* row = jf + (__ffsll((long long)wi) - 1) * n;
        for (uint64_t wj = b; wj; wj &= wj - 1) e += row[__ffsll((long long)wj) - 1];
    }
    return (double)e * dscale;
}

// H_xx from the byte tables: F(a) + F(b) + G(a, b) with F(w) = sum_k Dt[k][w_k] +
// sum_{k<l} Xt[kl][w_k][w_l] and G = sum_{k,l} Yt[k][l][a_k][b_l]; the same exact fixed-point
// sum as diag_element_fixed, in a handful of (L2-resident) table reads.
__device__ __forceinline__ double diag_element_bytes(const ProblemDev& P, uint64_t a, uint64_t b) {
    const int nb = P.nbytes;
    long long e = 0;
    int pair = 0;
    for (int k = 0; k < nb; ++k) {
        const unsigned ak = (unsigned)(a >> (8 * k)) & 255u, bk = (unsigned)(b >> (8 * k)) & 255u;
        e += __ldg(&P.Dt[k * 256 + ak]) + __ldg(&P.Dt[k * 256 + bk]);
        for (int l = k + 1; l < nb; ++l, ++pair) {
            const unsigned al = (unsigned)(a >> (8 * l)) & 255u,
                           bl = (unsigned)(b >> (8 * l)) & 255u;
            const long long* X = P.Xt + (size_t)pair * 65536;
            e += __ldg(&X[ak * 256 + al]) + __ldg(&X[bk * 256 + bl]);
        }
        for (int l = 0; l < nb; ++l) {
            const unsigned bl = (unsigned)(b >> (8 * l)) & 255u;
            e += __ldg(&P.Yt[((size_t)(k * nb + l)) * 65536 + ak * 256 + bl]);
        }
    }
    return (double)e * P.dscale;
}

// cooperative load of the fixed-point diagonal tables into shared memory, then __syncthreads()
__device__ __forceinline__ void load_fixed_tables(const ProblemDev& P, long long* dst) {
    const int m = P.norb + 2 * P.norb * P.norb;
    for (int t = threadIdx.x; t < m; t += blockDim.x) dst[t] = P.hfx[t];
    __syncthreads();
}

// cooperative load of h_pp, J and K into shared memory (whole block), then __syncthreads()
__device__ __forceinline__ void load_diag_tables(const ProblemDev& P, double* hd, double* J,
                                                 double* K) {
    const int n = P.norb;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        J[t] = P.J[t];
        K[t] = P.K[t];
        if (t < n) hd[t] = P.h[t * n + t];
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

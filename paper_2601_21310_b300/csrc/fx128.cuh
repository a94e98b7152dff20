// Exact 128-bit fixed-point accumulation of FP64 terms (PT2 run sums).
//
// c(x') = sum_y H_x'y psi_y (Eq. pt2_correction) is summed as integers: each FP64 term v is
// rounded once to the grid 2^-F (round half away from zero) and held as a two's-complement
// 128-bit integer; additions are then exact and associative, so the sum of a run does not
// depend on the order in which its terms arrive, and it is converted to FP64 once (round to
// nearest even). F is chosen per call from a bound B on |v| times the longest possible run
// (F = 125 - ceil(log2(run_max * B))), so no partial sum can overflow and a term's rounding
// error is at most 2^-(F+1) = 2^-126 * run_max * B: far below FP64's own resolution of any
// term that can move the energy. All of this is integer arithmetic (no FP64 pipe).
#pragma once

#include <stdint.h>

struct Fx128 {
    uint64_t lo, hi;  // value = (hi:lo as a signed 128-bit integer) * 2^-F
};

__device__ __forceinline__ Fx128 fx_zero() { return Fx128{0ull, 0ull}; }

__device__ __forceinline__ Fx128 fx_add(Fx128 a, Fx128 b) {
    Fx128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

__device__ __forceinline__ Fx128 fx_neg(Fx128 a) {
    Fx128 r;
    r.lo = ~a.lo + 1ull;
    r.hi = ~a.hi + (r.lo == 0ull ? 1ull : 0ull);
    return r;
}

// v (finite FP64) -> round(v * 2^F); the caller's F keeps |v| * 2^F below 2^126
__device__ __forceinline__ Fx128 fx_from_double(double v, int F) {
    const uint64_t bits = (uint64_t)__double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7ff);
    uint64_t m = bits & ((1ull << 52) - 1ull);
    int ex;  // |v| = m * 2^ex
    if (e == 0) {
        ex = -1074;
    } else {
        m |= 1ull << 52;
        ex = e - 1075;
    }
    const int sh = ex + F;
    Fx128 r;
    if (m == 0ull) {
        r = fx_zero();
    } else if (sh >= 0) {  // exact left shift (sh <= 73 by the choice of F)
        if (sh == 0) {
            r.lo = m;
            r.hi = 0ull;
        } else if (sh < 64) {
            r.lo = m << sh;
            r.hi = m >> (64 - sh);
        } else {
            r.lo = 0ull;
            r.hi = m << (sh - 64);
        }
    } else {  // right shift with rounding half away from zero on the magnitude
        const int rs = -sh;
        if (rs > 54) {
            r = fx_zero();
        } else {
            r.lo = (m + (1ull << (rs - 1))) >> rs;
            r.hi = 0ull;
        }
    }
    return (bits >> 63) ? fx_neg(r) : r;
}

// round-to-nearest-even FP64 value of x * 2^-F
__device__ __forceinline__ double fx_to_double(Fx128 x, int F) {
    const bool neg = (int64_t)x.hi < 0;
    if (neg) x = fx_neg(x);
    if (x.hi == 0ull && x.lo == 0ull) return 0.0;
    const int lz = x.hi ? __clzll((long long)x.hi) : 64 + __clzll((long long)x.lo);
    // the 64 bits below the leading one (inclusive), with every lower bit folded into bit 0
    uint64_t top, rest;
    if (lz == 0) {
        top = x.hi;
        rest = x.lo;
    } else if (lz < 64) {
        top = (x.hi << lz) | (x.lo >> (64 - lz));
        rest = x.lo << lz;
    } else {
        top = x.lo << (lz - 64);
        rest = 0ull;
    }
    top |= rest ? 1ull : 0ull;
    // top * 2^(64 - lz) = x, so x * 2^-F = top * 2^(64 - lz - F)
    const double d = ldexp(__ull2double_rn(top), 64 - lz - F);
    return neg ? -d : d;
}

__device__ __forceinline__ Fx128 fx_shfl_up(Fx128 v, int d) {
    return Fx128{__shfl_up_sync(0xffffffffu, v.lo, d), __shfl_up_sync(0xffffffffu, v.hi, d)};
}
__device__ __forceinline__ Fx128 fx_shfl(Fx128 v, int src) {
    return Fx128{__shfl_sync(0xffffffffu, v.lo, src), __shfl_sync(0xffffffffu, v.hi, src)};
}

// grid exponent F for terms bounded by |v| <= vmax in runs of at most run_max terms
__device__ __forceinline__ int fx_scale(double vmax, double run_max) {
    const double b = vmax * run_max;
    if (!(b > 0.0)) return 100;
    int k;
    frexp(b, &k);  // b < 2^k
    return 125 - k;
}

// ------------------------------------------------------------------------------------------
// Accumulation into a hash table of configurations (PT2 over a connected space too large to
// sort at once): a slot holds the key (a, b) and an Fx128 sum; keys are claimed with a 128-bit
// compare-and-swap and sums added with 64-bit atomics (the low word's carry passed to the high
// word), so every slot ends with the exact sum of its terms in any order of arrival.
// ------------------------------------------------------------------------------------------
struct __align__(32) FxSlot {
    unsigned long long a, b;    // key; a = b = ~0 marks an empty slot
    unsigned long long lo, hi;  // Fx128 sum
};

#define FX_EMPTY 0xffffffffffffffffull

// 128-bit compare-and-swap of the slot's key: returns the key found (the empty key when this
// thread claimed the slot)
__device__ __forceinline__ void fx_cas_key(FxSlot* s, unsigned long long a, unsigned long long b,
                                           unsigned long long& oa, unsigned long long& ob) {
    asm volatile(
        "{\n\t.reg .b128 cmp, val, old;\n\t"
        "mov.b128 cmp, {%2, %3};\n\t"
        "mov.b128 val, {%4, %5};\n\t"
        "atom.global.cas.b128 old, [%6], cmp, val;\n\t"
        "mov.b128 {%0, %1}, old;\n\t}"
        : "=l"(oa), "=l"(ob)
        : "l"(FX_EMPTY), "l"(FX_EMPTY), "l"(a), "l"(b), "l"(s)
        : "memory");
}

__device__ __forceinline__ void fx_atomic_add(FxSlot* s, Fx128 v) {
    const unsigned long long old = atomicAdd(&s->lo, v.lo);
    const unsigned long long carry = (old + v.lo < old) ? 1ull : 0ull;
    const unsigned long long h = v.hi + carry;
    if (h) atomicAdd(&s->hi, h);
}

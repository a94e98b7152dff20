// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/nqs.h"

#define NQS_MAX_NORB 64

// ------------------------------------------------------------------------------------------
// error plumbing: every CUDA call is checked; a failure records a message and returns a code
// ------------------------------------------------------------------------------------------
void nqs_record_error(const char* what, cudaError_t e, const char* file, int line);
void nqs_record_message(const char* msg);

#define NQS_CK(call)                                                            \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            nqs_record_error(#call, e_, __FILE__, __LINE__);                    \
            return (e_ == cudaErrorMemoryAllocation) ? NQS_ERR_OOM : NQS_ERR_CUDA; \
        }                                                                       \
    } while (0)

// every kernel launch is followed by NQS_CK_LAUNCH, which also counts it (nqs_launch_count)
void nqs_note_launch();
#define NQS_CK_LAUNCH()              \
    do {                             \
        nqs_note_launch();           \
        NQS_CK(cudaGetLastError());  \
    } while (0)

#define NQS_TRY(expr)            \
    do {                         \
        int s_ = (expr);         \
        if (s_ < 0) return s_;   \
    } while (0)

// ------------------------------------------------------------------------------------------
// problem handle
// ------------------------------------------------------------------------------------------
struct ProblemDev {
    int norb, na, nb, ma, mb;
    int64_t sA, sB, dAA, dBB, dAB;  // class sizes of the canonical excitation list
    int64_t nexc;                   // excitations per det
    const double* h;                // [norb][norb]
    const double* eri;              // [norb]^4
    const double* J;                // J[p][q] = (pp|qq)
    const double* K;                // K[p][q] = (pq|qp)
    const double* TJ;               // TJ[(i*norb+a)*norb+j] = (ia|jj)
    const double* TD;               // TD[(i*norb+a)*norb+j] = (ia|jj) - (ij|ja), rounded once
    // fixed-point copies for exact integer accumulation of H_xx (value = int * dscale):
    // hfx[p] = h_pp, JKfx[p][q] = J_pq - K_pq (same spin), Jfx[p][q] = J_pq (opposite spin)
    const long long* hfx;
    const long long* JKfx;
    const long long* Jfx;
    double dscale;
    // byte tables of the same sums (diag_element_bytes): nbytes = ceil(norb / 8);
    //   Dt[k][u]        = sum over bits i of byte u at byte k of h_ii + sum_{i<j} (J-K)_ij
    //   Xt[kl][u][v]    = sum_{i in u at k, j in v at l} (J-K)_ij      for byte pairs k < l
    //   Yt[k][l][u][v]  = sum_{i in u at k, j in v at l} J_ij          for all k, l
    const long long* Dt;
    const long long* Xt;
    const long long* Yt;
    int nbytes;
    // bound on |<x'|H|y>| over every off-diagonal pair (singles: |h_ia| + sum_j (2 |(ia|jj)| +
    // |(ij|ja)|); doubles: 2 max |(pq|rs)|): the range of the PT2 fixed-point run sums
    double hoff_max;
    // single-excitation elements in exact fixed point (value = int * 2^-sfx_e): the same terms
    // as TJ / TD / h rounded once each, for the screened PT2 emission (hb.cu); every partial sum
    // of one element stays below 2^62 (sfx_e from hoff_max)
    const long long* TJfx;
    const long long* TDfx;
    const long long* hfx_off;  // h_pq
    int sfx_e;
    // byte tables of those terms per single: SDt[i][a][k][u] = sum of TDfx[i][a][j] over the
    // orbitals j = 8k + bit of the set bits of byte value u (j < norb), SJt the same of TJfx;
    // an element's sum over an occupied set is then one entry per byte of its string
    const long long* SDt;
    const long long* SJt;
};

struct nqs_problem {
    ProblemDev d;
    int device;
    double ecore;
    double *h, *eri, *J, *K, *TJ, *TD;
    long long* fx;  // hfx | JKfx | Jfx
    long long* bt;  // Dt | Xt | Yt
    long long* sfx; // TJfx | TDfx | hfx_off
    long long* sbt; // SDt | SJt
    cudaMemPool_t pool;  // library-owned stream-ordered pool for per-call scratch
    int* err_word;       // device: set by a kernel whose bounded wait timed out
    double* hb_val;      // heat-bath integral tables (hb.cu), built on first use
    uint16_t* hb_code;
    size_t scratch_limit;  // 0 = none; else scratch requests beyond it fail with NQS_ERR_OOM
};

// read and clear the problem's device error word (synchronises the stream)
int check_err_word(nqs_problem* p, cudaStream_t s);

struct nqs_net {
    nqs_problem* prob;
    int H1, H2, nin, nout, dtype;
    const void* p[7];    // W1, b1, W2, b2, W3, b3, Phi0 (caller-owned device pointers)
};

// stream-ordered scratch from the problem's pool
int nqs_scratch_alloc(nqs_problem* p, void** ptr, size_t bytes, cudaStream_t s);
void nqs_scratch_free(nqs_problem* p, void* ptr, cudaStream_t s);

// RAII holder for scratch so that every early return frees what it took. With an arena (a
// caller-supplied device region), get() hands out 256-byte aligned slices of it instead and
// nothing is allocated or freed.
struct Scratch {
    nqs_problem* p;
    cudaStream_t s;
    void* ptrs[64];
    int n = 0;
    uint8_t* arena = nullptr;
    size_t arena_size = 0, arena_used = 0;
    Scratch(nqs_problem* p_, cudaStream_t s_) : p(p_), s(s_) {}
    Scratch(void* arena_, size_t size_, cudaStream_t s_)
        : p(nullptr), s(s_), arena((uint8_t*)arena_), arena_size(size_) {}
    ~Scratch() { release(); }
    // return every block taken so far (stream-ordered); the holder can be used again
    void release() {
        for (int i = n - 1; i >= 0; --i) nqs_scratch_free(p, ptrs[i], s);
        n = 0;
    }
    template <class T>
    int get(T** out, size_t count) {
        void* v = nullptr;
        if (count == 0) count = 1;
        if (arena) {
            size_t off = (arena_used + 255) & ~(size_t)255;
            if (off + count * sizeof(T) > arena_size) return NQS_ERR_OOM;
            arena_used = off + count * sizeof(T);
            *out = (T*)(arena + off);
            return NQS_OK;
        }
        int st = nqs_scratch_alloc(p, &v, count * sizeof(T), s);
        if (st != NQS_OK) return st;
        if (n == 64) { nqs_scratch_free(p, v, s); return NQS_ERR_OOM; }
        ptrs[n++] = v;
        *out = (T*)v;
        return NQS_OK;
    }
};

// ------------------------------------------------------------------------------------------
// device helpers: bit strings
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t bits_between(int p, int q) {
    int lo = min(p, q), hi = max(p, q);
    uint64_t below_hi = (hi >= 64) ? ~0ull : ((1ull << hi) - 1ull);
    uint64_t upto_lo = (lo + 1 >= 64) ? ~0ull : ((1ull << (lo + 1)) - 1ull);
    return below_hi & ~upto_lo;
}
// (-1)^(occupied orbitals of w strictly between i and a), as +1 / -1
__device__ __forceinline__ int exc_sign(uint64_t w, int i, int a) {
    return (__popcll(w & bits_between(i, a)) & 1) ? -1 : 1;
}

// SplitMix64 output finaliser (Steele, Lea, Flood, OOPSLA 2014); bucket and hash function
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t det_hash(uint64_t a, uint64_t b) {
    return mix64(mix64(a) ^ b);
}
// PT2 bucket of a configuration among B < 2^32: the high 32 bits of det_hash scaled to [0, B)
// (one multiply; a 64-bit remainder by a variable B costs a long instruction sequence per
// excitation)
__host__ __device__ __forceinline__ uint32_t det_bucket(uint64_t a, uint64_t b, uint64_t B) {
    return (uint32_t)(((det_hash(a, b) >> 32) * B) >> 32);
}

// ------------------------------------------------------------------------------------------
// hash table of S: open addressing, linear probing, capacity a power of two >= 16|S| (8|S|
// above 2^22 configurations, 4|S| above 2^26). Each slot holds the configuration's position in
// S and a 2-byte fingerprint (16 bits of the hash, low bit forced to 1; 0 = empty): a probe
// reads the fingerprints (32 slots per 64 bytes; 32 MB for 16 M slots, so they stay in L2) and
// only on a match reads the position and compares the key in S itself. Most probes of the method
// miss, and a miss then never reads a key; at these load factors most misses end at the first
// slot.
// ------------------------------------------------------------------------------------------
struct HashS {
    const ulonglong2* set;  // the hashed configurations {a, b}, in their own order
    const int32_t* idx;     // [cap] position in set of the slot's configuration
    const uint16_t* fp;     // [cap] fingerprint, 0 = empty slot
    uint64_t mask;          // cap - 1
};

// Hash of a configuration for this table (independent of the bucket hash det_hash, which is
// part of the PT2 interface): two odd-constant multiplies, xor, one xorshift; the slot comes
// from bits 24.. and the fingerprint from bits 0..15. Half the work of det_hash with the same
// probe-length statistics on the method's sets.
__host__ __device__ __forceinline__ uint64_t s_hash(uint64_t a, uint64_t b) {
    uint64_t h = (a * 0x9E3779B97F4A7C15ull) ^ (b * 0xC2B2AE3D27D4EB4Full);
    return h ^ (h >> 31);
}
__host__ __device__ __forceinline__ uint64_t hash_slot(uint64_t h, uint64_t mask) {
    return (h >> 24) & mask;
}
__host__ __device__ __forceinline__ uint16_t hash_fingerprint(uint64_t h) {
    return (uint16_t)(h | 1ull);
}

// lookup with the hash h = s_hash(a, b) already formed
__device__ __forceinline__ int32_t hash_lookup_h(const HashS& H, uint64_t a, uint64_t b,
                                                 uint64_t h) {
    uint64_t slot = hash_slot(h, H.mask);
    const uint16_t f = hash_fingerprint(h);
    for (uint64_t it = 0; it <= H.mask; ++it) {
        const uint16_t v = __ldg(&H.fp[slot]);
        if (v == 0) return -1;
        if (v == f) {  // the key is compared in the set itself (L2-resident, unlike a copy
                       // of the keys per slot)
            const int32_t j = __ldg(&H.idx[slot]);
            const ulonglong2 k = __ldg(&H.set[j]);
            if (k.x == a && k.y == b) return j;
        }
        slot = (slot + 1) & H.mask;
    }
    return -1;
}

__device__ __forceinline__ int32_t hash_lookup(const HashS& H, uint64_t a, uint64_t b) {
    return hash_lookup_h(H, a, b, s_hash(a, b));
}

// position of (a, b) when the caller knows it is in the set (a hit of the count pass): the probe
// sequence up to the first empty slot holds its slot, so a single fingerprint match there is
// that slot and no key needs to be read; several matches fall back to comparing keys
__device__ __forceinline__ int32_t hash_lookup_member(const HashS& H, uint64_t a, uint64_t b) {
    const uint64_t h = s_hash(a, b);
    uint64_t slot = hash_slot(h, H.mask);
    const uint16_t f = hash_fingerprint(h);
    uint64_t first = 0;
    int matches = 0;
    for (uint64_t it = 0; it <= H.mask; ++it) {
        const uint16_t v = __ldg(&H.fp[slot]);
        if (v == 0) break;
        if (v == f) {
            if (matches == 0) first = slot;
            ++matches;
        }
        slot = (slot + 1) & H.mask;
    }
    if (matches == 1) return __ldg(&H.idx[first]);
    return hash_lookup_h(H, a, b, h);
}

// the H_SS enumeration kernels (connect.cu) and their launch shape
#define CONN_THREADS 256
#define CONN_WARPS (CONN_THREADS / 32)
__global__ void k_conn_count(ProblemDev P, HashS H, const ulonglong2* __restrict__ S, int64_t nS,
                             int64_t* rowcnt, uint32_t* __restrict__ bits);
__global__ void k_conn_fill(ProblemDev P, HashS H, const ulonglong2* __restrict__ S, int64_t nS,
                            const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                            double* __restrict__ val, const uint32_t* __restrict__ bits);
size_t conn_smem_bytes(const ProblemDev& P);
// the H_SS count pass over `rows` against the sorted unique set Rset (hashed in H): indices of
// Rset by alpha and beta string, then the indexed count kernel (connect.cu)
int conn_count_indexed(nqs_problem* p, Scratch& sc, const HashS& H, const uint64_t* rows,
                       int64_t nrows, const uint64_t* Rset, int64_t nR, int64_t* rowcnt,
                       uint32_t* bits, cudaStream_t s);
unsigned conn_grid_size(int64_t nS);

// slots_per_det > 0 fixes the capacity to the next power of two >= slots_per_det * nS (the
// allocation-free path, whose scratch is bounded); 0 takes the default sparse table
int hash_build(nqs_problem* p, Scratch& sc, const uint64_t* dets, int64_t nS, HashS* out,
               cudaStream_t s, int slots_per_det = 0);
// screened PT2 emission pass (hb.cu): counts per det when cnt != null, else the (key, H psi)
// pairs at offs; keys are uint32 / uint64 / Key128 by 2 norb
int hb_pt2_pass(nqs_problem* p, const HashS& H, const uint64_t* dets, const double* psi,
                int64_t nS, double eps, uint64_t B, uint64_t bucket, int64_t* cnt,
                const int64_t* offs, void* keys, double* vals, cudaStream_t s);
// the same emissions for all of C\S in one traversal, appended in timing order to keys / vals
// [cap]; *cursor_dev receives the number of pairs (> cap: too small, nothing past cap written)
int hb_pt2_append(nqs_problem* p, const HashS& H, const uint64_t* dets, const double* psi,
                  int64_t nS, double eps, void* keys, double* vals, int64_t cap,
                  unsigned long long* cursor_dev, cudaStream_t s);
int validate_dets(nqs_problem* p, Scratch& sc, const uint64_t* dets, int64_t nS, bool sorted,
                  cudaStream_t s);

// ------------------------------------------------------------------------------------------
// PT2 sort keys: the determinant (a, b) packed as the 2 norb-bit number (a << norb) | b, in a
// uint32 (2 norb <= 32), a uint64 (<= 64) or two words (<= 128); numeric order = (a, b) order.
// ------------------------------------------------------------------------------------------
struct Key128 {
    uint64_t lo, hi;
};
__host__ __device__ __forceinline__ bool operator!=(const Key128& x, const Key128& y) {
    return x.lo != y.lo || x.hi != y.hi;
}
template <class K>
__device__ __forceinline__ K key_zero() { return (K)0; }
template <>
__device__ __forceinline__ Key128 key_zero<Key128>() { return Key128{0ull, 0ull}; }
template <class K>
__device__ __forceinline__ uint32_t key_digit(const K& k, int s) { return (uint32_t)(k >> s) & 255u; }
__device__ __forceinline__ uint32_t key_digit(const Key128& k, int s) {
    return (uint32_t)(s < 64 ? (k.lo >> s) : (k.hi >> (s - 64))) & 255u;
}
template <class K>
__device__ __forceinline__ K key_make(uint64_t a, uint64_t b, int norb) {
    return (K)((a << norb) | b);
}
template <>
__device__ __forceinline__ Key128 key_make<Key128>(uint64_t a, uint64_t b, int norb) {
    Key128 k;
    k.lo = b | (norb < 64 ? (a << norb) : 0ull);
    k.hi = norb == 0 ? 0ull : (a >> (64 - norb));
    return k;
}
template <class K>
__device__ __forceinline__ void key_split(const K& k, int norb, uint64_t& a, uint64_t& b) {
    const uint64_t v = (uint64_t)k;
    a = v >> norb;
    b = v & ((1ull << norb) - 1ull);
}
__device__ __forceinline__ void key_split(const Key128& k, int norb, uint64_t& a, uint64_t& b) {
    const uint64_t m = norb >= 64 ? ~0ull : ((1ull << norb) - 1ull);
    b = k.lo & m;
    a = ((k.lo >> norb) | (k.hi << (64 - norb))) & m;
}
template <class K>
__device__ __forceinline__ K key_shfl_up(const K& k, int d) {
    return __shfl_up_sync(0xffffffffu, k, d);
}
__device__ __forceinline__ Key128 key_shfl_up(const Key128& k, int d) {
    return Key128{__shfl_up_sync(0xffffffffu, k.lo, d), __shfl_up_sync(0xffffffffu, k.hi, d)};
}
template <class K>
__device__ __forceinline__ K key_shfl(const K& k, int src) {
    return __shfl_sync(0xffffffffu, k, src);
}
__device__ __forceinline__ Key128 key_shfl(const Key128& k, int src) {
    return Key128{__shfl_sync(0xffffffffu, k.lo, src), __shfl_sync(0xffffffffu, k.hi, src)};
}

// ------------------------------------------------------------------------------------------
// primitives (primitives.cu)
// ------------------------------------------------------------------------------------------
// exclusive prefix sum of n values; total (device, may be null) receives the sum
int scan_exclusive_i64(nqs_problem* p, Scratch& sc, const int64_t* in, int64_t* out, int64_t n,
                       int64_t* total, cudaStream_t s);
int scan_exclusive_u32(nqs_problem* p, Scratch& sc, const uint32_t* in, uint32_t* out, int64_t n,
                       cudaStream_t s);
// the same for FP64 in a fixed tile order (deterministic; rounding differs from a serial sum)
int scan_exclusive_f64(nqs_problem* p, Scratch& sc, const double* in, double* out, int64_t n,
                       double* total, cudaStream_t s);
// y = H x for a device CSR (one warp per row, fixed summation order)
int csr_spmv(const nqs_csr* csr, const double* x, double* y, cudaStream_t s);
// the same without each row's first entry (the diagonal of H_SS): the off-diagonal part
int csr_spmv_offdiag(const nqs_csr* csr, const double* x, double* y, cudaStream_t s);
// compensated (Neumaier) sum of n FP64 values into *out (device); deterministic
int ksum_f64(nqs_problem* p, Scratch& sc, const double* x, int64_t n, double* out,
             cudaStream_t s);
// compensated dot products: out[0] = sum x*y, out[1] = sum y*y
int kdot2_f64(nqs_problem* p, Scratch& sc, const double* x, const double* y, int64_t n,
              double* out, cudaStream_t s);
// max of n FP64 values (ignoring entries whose mask byte is 0)
int max_f64_masked(nqs_problem* p, Scratch& sc, const double* x, const int8_t* mask, int64_t n,
                   double* out, cudaStream_t s);
// stable LSD radix sort of (u64 key, f64 value) pairs on the low `bits` key bits.
// Result ends in (keys, vals); (keys_alt, vals_alt) are scratch of the same size.
// The pointers are swapped in place so that (keys, vals) name the sorted result on return.
int radix_sort_pairs(nqs_problem* p, Scratch& sc, uint64_t*& keys, double*& vals,
                     uint64_t*& keys_alt, double*& vals_alt, int64_t n, int bits, cudaStream_t s);
int radix_sort_pairs32(nqs_problem* p, Scratch& sc, uint32_t*& keys, double*& vals,
                       uint32_t*& keys_alt, double*& vals_alt, int64_t n, int bits,
                       cudaStream_t s);
int radix_sort_pairs128(nqs_problem* p, Scratch& sc, Key128*& keys, double*& vals,
                        Key128*& keys_alt, double*& vals_alt, int64_t n, int bits,
                        cudaStream_t s);

inline unsigned grid_for(int64_t n, int block, int cap = 148 * 32) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

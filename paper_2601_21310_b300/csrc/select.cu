// Subspace selection of the outer loop, Sec. 2.4.2 (Algorithm 1 step 3: V <- Selector(T, K,
// key = |psi|)), with the three protocols the paper lists: Top-K, cumulative mass and absolute
// threshold.
//
// Ranking: configurations of T by log|psi| descending, ties by ascending key. Two stable LSD
// radix sorts give it: first by the 2 norb-bit key (which also exposes duplicates), then by an
// order-preserving 64-bit image of -log|psi| carrying the key-sorted positions; stability makes
// equal amplitudes keep key order. The kept prefix length c is
//   Top-K   min(K, n);
//   mass    1 + the first rank whose inclusive sum of w = exp(2 (log|psi| - max)) reaches
//           gamma * D (D = compensated sum of w); n if none does;
//   thresh  the number of ranks with w / D > eps (a prefix: w is non-increasing along ranks).
// The kept positions are flagged in T order and compacted in key order, so the output set is
// ascending by key, ready to serve as the next S.
#include <math.h>

#include "excite.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

// FP64 -> uint64 whose ascending order is the descending order of the value (-0 as +0)
__device__ __forceinline__ uint64_t desc_image(double x) {
    x = x + 0.0;
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const uint64_t asc = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    return ~asc;
}

template <class K>
__global__ void k_sel_keys(const ulonglong2* __restrict__ T, int64_t n, int norb,
                           K* __restrict__ keys, int64_t* __restrict__ pos) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const ulonglong2 x = T[i];
        keys[i] = key_make<K>(x.x, x.y, norb);
        pos[i] = i;
    }
}

// flag[0] |= 1 for a duplicate key, flag[0] |= 2 for a NaN or +inf log|psi|; builds the rank keys
template <class K>
__global__ void k_sel_rank_keys(const K* __restrict__ keys, const int64_t* __restrict__ kpos,
                                const double* __restrict__ logabs, int64_t n,
                                uint64_t* __restrict__ rk, int64_t* __restrict__ rpos,
                                int* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i > 0 && !(keys[i] != keys[i - 1])) atomicOr(flag, 1);
        const int64_t q = kpos[i];
        const double l = logabs[q];
        if (l != l || l == INFINITY) atomicOr(flag, 2);
        rk[i] = desc_image(l);
        rpos[i] = q;
    }
}

// w[r] = exp(2 (log|psi| of rank r - log|psi| of rank 0)); rank 0 holds the maximum
__global__ void k_sel_weights(const int64_t* __restrict__ rpos, const double* __restrict__ logabs,
                              int64_t n, double* __restrict__ w) {
    const double lmax = logabs[rpos[0]];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        w[i] = exp(2.0 * (logabs[rpos[i]] - lmax));
}

// mass: c = 1 + min { r : excl[r] + w[r] >= gamma * D }   (c initialised to n)
__global__ void k_sel_mass(const double* __restrict__ excl, const double* __restrict__ w,
                           int64_t n, const double* __restrict__ D, double gamma,
                           unsigned long long* __restrict__ c) {
    const double target = gamma * D[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (excl[i] + w[i] >= target) atomicMin(c, (unsigned long long)(i + 1));
}

// threshold: c = #{ r : w[r] / D > eps }   (c initialised to 0)
__global__ void k_sel_thresh(const double* __restrict__ w, int64_t n,
                             const double* __restrict__ D, double eps,
                             unsigned long long* __restrict__ c) {
    const double d = D[0];
    unsigned long long k = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        k += (w[i] / d > eps) ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) k += __shfl_down_sync(FULL_MASK, k, o);
    if ((threadIdx.x & 31) == 0 && k) atomicAdd(c, k);
}

__global__ void k_sel_set(unsigned long long* c, unsigned long long v) { *c = v; }

// sel[rpos[r]] = 1 for the first c ranks
__global__ void k_sel_mark(const int64_t* __restrict__ rpos, const unsigned long long* c,
                           uint32_t* __restrict__ sel) {
    const int64_t cc = (int64_t)c[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cc;
         i += (int64_t)gridDim.x * blockDim.x)
        sel[rpos[i]] = 1u;
}

// f[i] = sel[kpos[i]] in key order
__global__ void k_sel_flags(const int64_t* __restrict__ kpos, const uint32_t* __restrict__ sel,
                            int64_t n, uint32_t* __restrict__ f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] = sel[kpos[i]];
}

__global__ void k_sel_out(const int64_t* __restrict__ kpos, const uint32_t* __restrict__ f,
                          const uint32_t* __restrict__ at, int64_t n,
                          const ulonglong2* __restrict__ T, const double* __restrict__ logabs,
                          ulonglong2* __restrict__ od, double* __restrict__ ov,
                          int64_t* __restrict__ oi) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!f[i]) continue;
        const int64_t q = kpos[i], u = at[i];
        od[u] = T[q];
        ov[u] = logabs[q];
        oi[u] = q;
    }
}

template <class K>
static int sort_by_key(nqs_problem* p, Scratch& sc, K*& keys, int64_t*& pos, K*& keys2,
                       int64_t*& pos2, int64_t n, int bits, cudaStream_t s) {
    double*& v = (double*&)pos;
    double*& v2 = (double*&)pos2;
    if (sizeof(K) == 4)
        return radix_sort_pairs32(p, sc, (uint32_t*&)keys, v, (uint32_t*&)keys2, v2, n, bits, s);
    if (sizeof(K) == 8)
        return radix_sort_pairs(p, sc, (uint64_t*&)keys, v, (uint64_t*&)keys2, v2, n, bits, s);
    return radix_sort_pairs128(p, sc, (Key128*&)keys, v, (Key128*&)keys2, v2, n, bits, s);
}

template <class K>
static int select_run(nqs_problem* p, Scratch& sc, const uint64_t* T, const double* logabs,
                      int64_t n, int mode, int64_t Kkeep, double param, int validate,
                      nqs_detset* out, cudaStream_t s) {
    const int norb = p->d.norb;
    const unsigned g = grid_for(n, 256);
    K *keys, *keys2;
    int64_t *kpos, *kpos2, *rpos, *rpos2;
    uint64_t *rk, *rk2;
    int* flag;
    unsigned long long* c_dev;
    NQS_TRY(sc.get(&keys, n));
    NQS_TRY(sc.get(&keys2, n));
    NQS_TRY(sc.get(&kpos, n));
    NQS_TRY(sc.get(&kpos2, n));
    NQS_TRY(sc.get(&rk, n));
    NQS_TRY(sc.get(&rk2, n));
    NQS_TRY(sc.get(&rpos, n));
    NQS_TRY(sc.get(&rpos2, n));
    NQS_TRY(sc.get(&flag, 1));
    NQS_TRY(sc.get(&c_dev, 1));
    NQS_CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
    ProfScope prof_(PROF_SELECT, s);
    k_sel_keys<K><<<g, 256, 0, s>>>((const ulonglong2*)T, n, norb, keys, kpos);
    NQS_CK_LAUNCH();
    NQS_TRY(sort_by_key<K>(p, sc, keys, kpos, keys2, kpos2, n, 2 * norb, s));
    k_sel_rank_keys<K><<<g, 256, 0, s>>>(keys, kpos, logabs, n, rk, rpos, flag);
    NQS_CK_LAUNCH();
    int hflag = 0;
    NQS_CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    if (hflag & 2) {
        nqs_record_message("nqs_select: log|psi| holds NaN or +inf");
        return NQS_ERR_ARG;
    }
    if ((hflag & 1) && validate) {
        nqs_record_message("nqs_select: T holds a configuration twice");
        return NQS_ERR_UNSORTED;
    }
    NQS_TRY(radix_sort_pairs(p, sc, rk, (double*&)rpos, rk2, (double*&)rpos2, n, 64, s));
    // kept prefix length
    if (mode == NQS_SELECT_TOPK) {
        const unsigned long long c = (unsigned long long)(Kkeep < n ? (Kkeep > 0 ? Kkeep : 0) : n);
        k_sel_set<<<1, 1, 0, s>>>(c_dev, c);
        NQS_CK_LAUNCH();
    } else {
        double *w, *excl, *D;
        NQS_TRY(sc.get(&w, n));
        NQS_TRY(sc.get(&D, 1));
        k_sel_weights<<<g, 256, 0, s>>>(rpos, logabs, n, w);
        NQS_CK_LAUNCH();
        NQS_TRY(ksum_f64(p, sc, w, n, D, s));
        if (mode == NQS_SELECT_MASS) {
            NQS_TRY(sc.get(&excl, n));
            NQS_TRY(scan_exclusive_f64(p, sc, w, excl, n, (double*)nullptr, s));
            k_sel_set<<<1, 1, 0, s>>>(c_dev, (unsigned long long)n);
            NQS_CK_LAUNCH();
            k_sel_mass<<<g, 256, 0, s>>>(excl, w, n, D, param, c_dev);
        } else {
            NQS_CK(cudaMemsetAsync(c_dev, 0, sizeof(unsigned long long), s));
            k_sel_thresh<<<g, 256, 0, s>>>(w, n, D, param, c_dev);
        }
        NQS_CK_LAUNCH();
    }
    // flag the kept positions, compact in key order
    uint32_t *sel, *f, *at;
    NQS_TRY(sc.get(&sel, n));
    NQS_TRY(sc.get(&f, n));
    NQS_TRY(sc.get(&at, n));
    NQS_CK(cudaMemsetAsync(sel, 0, n * sizeof(uint32_t), s));
    k_sel_mark<<<g, 256, 0, s>>>(rpos, c_dev, sel);
    NQS_CK_LAUNCH();
    k_sel_flags<<<g, 256, 0, s>>>(kpos, sel, n, f);
    NQS_CK_LAUNCH();
    NQS_TRY(scan_exclusive_u32(p, sc, f, at, n, s));
    unsigned long long c = 0;
    NQS_CK(cudaMemcpyAsync(&c, c_dev, sizeof c, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    if (c == 0) return NQS_OK;
    if (cudaMalloc(&out->dets, c * 2 * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&out->value, c * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&out->index, c * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        return NQS_ERR_OOM;
    }
    out->n = (int64_t)c;
    k_sel_out<<<g, 256, 0, s>>>(kpos, f, at, n, (const ulonglong2*)T, logabs,
                                (ulonglong2*)out->dets, out->value, out->index);
    NQS_CK_LAUNCH();
    NQS_CK(cudaStreamSynchronize(s));
    return NQS_OK;
}

extern "C" int nqs_select(nqs_problem* p, const uint64_t* T, const double* logabs, int64_t n,
                          int mode, int64_t K, double param, const nqs_opts* opts,
                          nqs_detset* out, nqs_stream_t stream) {
    if (!p || !T || !logabs || !out || n <= 0) return NQS_ERR_ARG;
    if (((uintptr_t)T) & 15) return NQS_ERR_ARG;
    if (mode != NQS_SELECT_TOPK && mode != NQS_SELECT_MASS && mode != NQS_SELECT_THRESHOLD)
        return NQS_ERR_ARG;
    if (mode == NQS_SELECT_MASS && !(param >= 0.0 && param <= 1.0)) return NQS_ERR_ARG;
    if (mode == NQS_SELECT_THRESHOLD && !(param >= 0.0)) return NQS_ERR_ARG;
    if (n >= ((int64_t)1 << 31)) return NQS_ERR_UNSUPPORTED;
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
    Scratch sc(p, s);
    int st;
    const int kbits = 2 * p->d.norb;
    if (kbits <= 32)
        st = select_run<uint32_t>(p, sc, T, logabs, n, mode, K, param, opts->validate, out, s);
    else if (kbits <= 64)
        st = select_run<uint64_t>(p, sc, T, logabs, n, mode, K, param, opts->validate, out, s);
    else
        st = select_run<Key128>(p, sc, T, logabs, n, mode, K, param, opts->validate, out, s);
    if (st < 0) nqs_detset_free(out);
    return st;
}

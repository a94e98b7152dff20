// Problem handle (integrals on the device), scratch pool, validation of S, the hash table of S
// and the diagonal element H_xx.
#include <stdlib.h>
#include <string.h>

#include <math.h>

#include <mutex>
#include <vector>

#include "excite.cuh"
#include "nqs_internal.cuh"

static thread_local char g_last_error[512];

void nqs_record_error(const char* what, cudaError_t e, const char* file, int line) {
    snprintf(g_last_error, sizeof g_last_error, "%s failed: %s (%s:%d)", what,
             cudaGetErrorString(e), file, line);
}

void nqs_record_message(const char* msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

extern "C" const char* nqs_last_error(void) { return g_last_error; }

extern "C" const char* nqs_status_string(int status) {
    switch (status) {
        case NQS_OK: return "ok";
        case NQS_WARN_SINGULAR: return "warning: an occupied block is exactly singular";
        case NQS_ERR_ARG: return "invalid argument";
        case NQS_ERR_UNSORTED: return "determinants not sorted ascending / not unique";
        case NQS_ERR_POPCOUNT: return "determinant with the wrong electron count";
        case NQS_ERR_NORB: return "orbital count unsupported";
        case NQS_ERR_OOM: return "device allocation failed";
        case NQS_ERR_CUDA: return "CUDA error";
        case NQS_ERR_TIMEOUT: return "device wait timed out";
        case NQS_ERR_UNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}

extern "C" const char* nqs_version(void) { return "nqs-b300 0.1 (sm_103a)"; }

extern "C" void nqs_opts_default(nqs_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = NQS_FP64;
    o->buckets = 1;
    o->chunk = 0;
    o->validate = 1;
    o->internal_pt2 = 1;
}

// ------------------------------------------------------------------------------------------
// scratch: a library-owned memory pool, so repeated calls reuse memory without cudaMalloc
// ------------------------------------------------------------------------------------------
int nqs_scratch_alloc(nqs_problem* p, void** ptr, size_t bytes, cudaStream_t s) {
    if (p->scratch_limit) {
        uint64_t used = 0;
        NQS_CK(cudaMemPoolGetAttribute(p->pool, cudaMemPoolAttrUsedMemCurrent, &used));
        if (used + bytes > p->scratch_limit) {
            nqs_record_message("scratch request beyond the problem's scratch limit");
            return NQS_ERR_OOM;
        }
    }
    cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, p->pool, s);
    if (e != cudaSuccess) {
        nqs_record_error("cudaMallocFromPoolAsync", e, __FILE__, __LINE__);
        cudaGetLastError();
        return NQS_ERR_OOM;
    }
    return NQS_OK;
}

void nqs_scratch_free(nqs_problem* p, void* ptr, cudaStream_t s) {
    if (ptr) cudaFreeAsync(ptr, s);
}

// ------------------------------------------------------------------------------------------
// problem create / destroy
// ------------------------------------------------------------------------------------------
// the single-excitation tables in fixed point: v * 2^e rounded to the nearest integer
__global__ void k_fx_tables(int64_t n3, int n, const double* TJ, const double* TD, const double* h,
                            int e, long long* out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 2 * n3 + (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double v = t < n3 ? TJ[t] : (t < 2 * n3 ? TD[t - n3] : h[t - 2 * n3]);
        out[t] = __double2ll_rn(ldexp(v, e));
    }
}

// entry t of SDt | SJt: the sum of the fixed-point single terms over the orbitals of one byte
__global__ void k_single_byte_tables(int n, int nb, const long long* TDfx, const long long* TJfx,
                                     long long* out) {
    const int64_t per = (int64_t)n * n * nb * 256;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 2 * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const long long* X = t < per ? TDfx : TJfx;
        const int64_t r = t < per ? t : t - per;
        const int u = (int)(r % 256), k = (int)((r / 256) % nb);
        const int64_t ia = r / (256 * (int64_t)nb);  // i * n + a
        long long v = 0;
        for (int bit = 0; bit < 8; ++bit) {
            const int j = 8 * k + bit;
            if (((u >> bit) & 1) && j < n) v += X[ia * n + j];
        }
        out[t] = v;
    }
}

__global__ void k_tables(int n, const double* eri, double* J, double* K, double* TJ, double* TD) {
    int64_t total = (int64_t)n * n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(t % n), a = (int)((t / n) % n), i = (int)(t / ((int64_t)n * n));
        TJ[t] = eri[(((size_t)i * n + a) * n + j) * n + j];   // (ia|jj)
        // (ia|jj) - (ij|ja): the same-spin term of a single's element, rounded once here
        TD[t] = __dsub_rn(TJ[t], eri[(((size_t)i * n + j) * n + j) * n + a]);
        if (a == 0) {
            J[i * n + j] = eri[(((size_t)i * n + i) * n + j) * n + j];  // (ii|jj)
            K[i * n + j] = eri[(((size_t)i * n + j) * n + j) * n + i];  // (ij|ji)
        }
    }
}

// entry t of the byte tables (layout in ProblemDev); sums of fixed-point terms, exact
__global__ void k_byte_tables(ProblemDev d, size_t nD, size_t nX, size_t nY) {
    const int n = d.norb, nb = d.nbytes;
    long long* out = (long long*)d.Dt;  // the three tables are contiguous
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nD + nX + nY;
         t += (size_t)gridDim.x * blockDim.x) {
        long long v = 0;
        if (t < nD) {
            const int k = (int)(t / 256), u = (int)(t % 256);
            for (int i = 0; i < 8; ++i) {
                if (!((u >> i) & 1) || 8 * k + i >= n) continue;
                const int pi = 8 * k + i;
                v += d.hfx[pi];
                for (int j = i + 1; j < 8; ++j)
                    if (((u >> j) & 1) && 8 * k + j < n) v += d.JKfx[pi * n + 8 * k + j];
            }
        } else {
            const bool same = t < nD + nX;
            const size_t r = same ? t - nD : t - nD - nX;
            const size_t pair = r / 65536;
            const int u = (int)((r % 65536) / 256), w = (int)(r % 256);
            int k, l;
            if (same) {  // pair index over k < l, lexicographic
                int rem = (int)pair;
                k = 0;
                while (rem >= nb - 1 - k) {
                    rem -= nb - 1 - k;
                    ++k;
                }
                l = k + 1 + rem;
            } else {
                k = (int)(pair / nb);
                l = (int)(pair % nb);
            }
            const long long* tab = same ? d.JKfx : d.Jfx;
            for (int i = 0; i < 8; ++i) {
                if (!((u >> i) & 1) || 8 * k + i >= n) continue;
                for (int j = 0; j < 8; ++j)
                    if (((w >> j) & 1) && 8 * l + j < n) v += tab[(8 * k + i) * n + 8 * l + j];
            }
        }
        out[t] = v;
    }
}

extern "C" int nqs_problem_create(int norb, int nalpha, int nbeta, const double* h,
                                  const double* eri, double ecore, nqs_problem** out) {
    if (!out || !h || !eri) return NQS_ERR_ARG;
    *out = nullptr;
    if (norb < 1 || norb > NQS_MAX_NORB) return NQS_ERR_NORB;
    if (nalpha <= 0 || nbeta <= 0 || nalpha >= norb || nbeta >= norb) return NQS_ERR_ARG;
    nqs_problem* p = (nqs_problem*)calloc(1, sizeof(nqs_problem));
    if (!p) return NQS_ERR_OOM;
    p->ecore = ecore;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        free(p);
        return NQS_ERR_CUDA;
    }
    size_t n2 = (size_t)norb * norb, n3 = n2 * norb, n4 = n3 * norb;
    auto fail = [&](int code) {
        nqs_problem_destroy(p);
        return code;
    };
    if (cudaMalloc(&p->h, n2 * 8) != cudaSuccess || cudaMalloc(&p->eri, n4 * 8) != cudaSuccess ||
        cudaMalloc(&p->J, n2 * 8) != cudaSuccess || cudaMalloc(&p->K, n2 * 8) != cudaSuccess ||
        cudaMalloc(&p->TJ, n3 * 8) != cudaSuccess || cudaMalloc(&p->TD, n3 * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(NQS_ERR_OOM);
    }
    if (cudaMemcpy(p->h, h, n2 * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->eri, eri, n4 * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(NQS_ERR_CUDA);
    k_tables<<<grid_for((int64_t)n3, 256), 256>>>(norb, p->eri, p->J, p->K, p->TJ, p->TD);
    nqs_note_launch();
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return fail(NQS_ERR_CUDA);

    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = p->device;
    if (cudaMemPoolCreate(&p->pool, &props) != cudaSuccess) {
        p->pool = nullptr;
        return fail(NQS_ERR_CUDA);
    }
    uint64_t thresh = ~0ull;  // keep freed scratch in the pool between calls
    cudaMemPoolSetAttribute(p->pool, cudaMemPoolAttrReleaseThreshold, &thresh);
    if (cudaMalloc(&p->err_word, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->err_word, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(NQS_ERR_OOM);
    }

    ProblemDev& d = p->d;
    d.norb = norb;
    d.na = nalpha;
    d.nb = nbeta;
    d.ma = norb - nalpha;
    d.mb = norb - nbeta;
    d.sA = (int64_t)d.na * d.ma;
    d.sB = (int64_t)d.nb * d.mb;
    d.dAA = choose2(d.na) * choose2(d.ma);
    d.dBB = choose2(d.nb) * choose2(d.mb);
    d.dAB = d.sA * d.sB;
    d.nexc = d.sA + d.sB + d.dAA + d.dBB + d.dAB;
    d.h = p->h;
    d.eri = p->eri;
    d.J = p->J;
    d.K = p->K;
    d.TJ = p->TJ;
    d.TD = p->TD;
    if (d.nexc >= ((int64_t)1 << 31)) return fail(NQS_ERR_NORB);
    // Fixed-point tables for the diagonal: every partial sum of H_xx is bounded by
    // bound = sum_p |h_pp| + sum_{p<q} |J_pq - K_pq| * 2 + sum_{p,q} |J_pq|, so with
    // scale 2^e, e = 61 - ceil(log2(bound)), no int64 partial sum can overflow and each term
    // is rounded once (relative error ~2^-e * number of terms).
    {
        const int n = norb;
        std::vector<double> Jh(n * n), Kh(n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                Jh[i * n + j] = eri[(((size_t)i * n + i) * n + j) * n + j];
                Kh[i * n + j] = eri[(((size_t)i * n + j) * n + j) * n + i];
            }
        double bound = 1.0;
        for (int i = 0; i < n; ++i) bound += fabs(h[i * n + i]);
        for (int i = 0; i < n * n; ++i) bound += 2.0 * fabs(Jh[i] - Kh[i]) + fabs(Jh[i]);
        const int e = 61 - (int)ceil(log2(bound));
        std::vector<long long> fx(n + 2 * n * n);
        for (int i = 0; i < n; ++i) fx[i] = llrint(ldexp(h[i * n + i], e));
        for (int i = 0; i < n * n; ++i) {
            fx[n + i] = llrint(ldexp(Jh[i] - Kh[i], e));
            fx[n + n * n + i] = llrint(ldexp(Jh[i], e));
        }
        if (cudaMalloc(&p->fx, fx.size() * sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(NQS_ERR_OOM);
        }
        if (cudaMemcpy(p->fx, fx.data(), fx.size() * sizeof(long long),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(NQS_ERR_CUDA);
        d.hfx = p->fx;
        d.JKfx = p->fx + n;
        d.Jfx = p->fx + n + n * n;
        d.dscale = ldexp(1.0, -e);
        double hmax = 0.0, emax = 0.0;
        for (size_t q = 0; q < (size_t)n * n * n * n; ++q) emax = fmax(emax, fabs(eri[q]));
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < n; ++a) {
                if (a == i) continue;
                double f = fabs(h[i * n + a]);
                for (int j = 0; j < n; ++j)
                    f += 2.0 * fabs(eri[(((size_t)i * n + a) * n + j) * n + j]) +
                         fabs(eri[(((size_t)i * n + j) * n + j) * n + a]);
                hmax = fmax(hmax, f);
            }
        d.hoff_max = fmax(hmax, 2.0 * emax) * (1.0 + 1e-12);
        // fixed-point single tables: every partial sum of an element is bounded by hoff_max
        d.sfx_e = 62 - (int)ceil(log2(d.hoff_max > 0.0 ? d.hoff_max : 1.0));
        const int64_t n3 = (int64_t)n * n * n;
        if (cudaMalloc(&p->sfx, (2 * n3 + (int64_t)n * n) * sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(NQS_ERR_OOM);
        }
        k_fx_tables<<<grid_for(2 * n3 + (int64_t)n * n, 256), 256>>>(n3, n, p->TJ, p->TD, p->h,
                                                                   d.sfx_e, p->sfx);
        nqs_note_launch();
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
            return fail(NQS_ERR_CUDA);
        d.TJfx = p->sfx;
        d.TDfx = p->sfx + n3;
        d.hfx_off = p->sfx + 2 * n3;
        // byte tables
        const int nb = (n + 7) / 8;
        const int64_t nsb = (int64_t)n * n * nb * 256;
        if (cudaMalloc(&p->sbt, 2 * nsb * sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(NQS_ERR_OOM);
        }
        k_single_byte_tables<<<grid_for(2 * nsb, 256), 256>>>(n, nb, d.TDfx, d.TJfx, p->sbt);
        nqs_note_launch();
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
            return fail(NQS_ERR_CUDA);
        d.SDt = p->sbt;
        d.SJt = p->sbt + nsb;
        const size_t nD = (size_t)nb * 256, nX = (size_t)nb * (nb - 1) / 2 * 65536,
                     nY = (size_t)nb * nb * 65536;
        if (cudaMalloc(&p->bt, (nD + nX + nY) * sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(NQS_ERR_OOM);
        }
        d.Dt = p->bt;
        d.Xt = p->bt + nD;
        d.Yt = p->bt + nD + nX;
        d.nbytes = nb;
        k_byte_tables<<<grid_for((int64_t)(nD + nX + nY), 256), 256>>>(d, nD, nX, nY);
        nqs_note_launch();
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
            return fail(NQS_ERR_CUDA);
    }
    *out = p;
    return NQS_OK;
}

extern "C" int nqs_problem_destroy(nqs_problem* p) {
    if (!p) return NQS_OK;
    cudaDeviceSynchronize();
    cudaFree(p->h);
    cudaFree(p->eri);
    cudaFree(p->J);
    cudaFree(p->K);
    cudaFree(p->TJ);
    cudaFree(p->TD);
    cudaFree(p->err_word);
    cudaFree(p->fx);
    cudaFree(p->bt);
    cudaFree(p->sfx);
    cudaFree(p->sbt);
    cudaFree(p->hb_val);
    cudaFree(p->hb_code);
    if (p->pool) cudaMemPoolDestroy(p->pool);
    free(p);
    return NQS_OK;
}

extern "C" int nqs_set_scratch_limit(nqs_problem* p, int64_t bytes) {
    if (!p || bytes < 0) return NQS_ERR_ARG;
    p->scratch_limit = (size_t)bytes;
    return NQS_OK;
}

extern "C" int nqs_pool_usage(nqs_problem* p, int64_t* used, int64_t* reserved) {
    if (!p || !used || !reserved) return NQS_ERR_ARG;
    uint64_t u = 0, r = 0;
    NQS_CK(cudaMemPoolGetAttribute(p->pool, cudaMemPoolAttrUsedMemCurrent, &u));
    NQS_CK(cudaMemPoolGetAttribute(p->pool, cudaMemPoolAttrReservedMemCurrent, &r));
    *used = (int64_t)u;
    *reserved = (int64_t)r;
    return NQS_OK;
}

int check_err_word(nqs_problem* p, cudaStream_t s) {
    int h = 0;
    NQS_CK(cudaMemcpyAsync(&h, p->err_word, sizeof h, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    if (h) {
        NQS_CK(cudaMemsetAsync(p->err_word, 0, sizeof(int), s));
        nqs_record_message("a tensor-core pipeline wait timed out; results are invalid");
        return NQS_ERR_TIMEOUT;
    }
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// validation: sorted strictly ascending (optional) and right popcounts
// ------------------------------------------------------------------------------------------
__global__ void k_validate(const ulonglong2* S, int64_t n, int na, int nb, int check_sorted,
                           uint64_t norb_mask, int* flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        ulonglong2 x = S[i];
        if (__popcll(x.x) != na || __popcll(x.y) != nb || (x.x & ~norb_mask) || (x.y & ~norb_mask))
            atomicOr(&flags[0], 1);
        if (check_sorted && i > 0) {
            ulonglong2 y = S[i - 1];
            bool ok = (y.x < x.x) || (y.x == x.x && y.y < x.y);
            if (!ok) atomicOr(&flags[1], 1);
        }
    }
}

int validate_dets(nqs_problem* p, Scratch& sc, const uint64_t* dets, int64_t nS, bool sorted,
                  cudaStream_t s) {
    int* flags;
    NQS_TRY(sc.get(&flags, 2));
    NQS_CK(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
    uint64_t mask = p->d.norb == 64 ? ~0ull : ((1ull << p->d.norb) - 1ull);
    k_validate<<<grid_for(nS, 256), 256, 0, s>>>((const ulonglong2*)dets, nS, p->d.na, p->d.nb,
                                                 sorted ? 1 : 0, mask, flags);
    NQS_CK_LAUNCH();
    int h[2];
    NQS_CK(cudaMemcpyAsync(h, flags, sizeof h, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    if (h[0]) return NQS_ERR_POPCOUNT;
    if (h[1]) return NQS_ERR_UNSORTED;
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// hash table of S
// ------------------------------------------------------------------------------------------
__global__ void k_hash_clear(int32_t* idx, uint16_t* fp, uint64_t cap) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap;
         i += (uint64_t)gridDim.x * blockDim.x) {
        idx[i] = -1;
        fp[i] = 0;
    }
}

__global__ void k_hash_insert(const ulonglong2* S, int64_t n, int32_t* idx, uint64_t mask) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        ulonglong2 x = S[i];
        uint64_t slot = hash_slot(s_hash(x.x, x.y), mask);
        for (uint64_t it = 0; it <= mask; ++it) {  // capacity > n: an empty slot exists
            if (atomicCAS(&idx[slot], -1, (int32_t)i) == -1) break;
            slot = (slot + 1) & mask;
        }
    }
}

__global__ void k_hash_fp(const ulonglong2* S, const int32_t* idx, uint16_t* fp, uint64_t cap) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap;
         i += (uint64_t)gridDim.x * blockDim.x) {
        int32_t k = idx[i];
        if (k >= 0) {
            const ulonglong2 x = S[k];
            fp[i] = hash_fingerprint(s_hash(x.x, x.y));
        }
    }
}

int hash_build(nqs_problem* p, Scratch& sc, const uint64_t* dets, int64_t nS, HashS* out,
               cudaStream_t s, int slots_per_det) {
    // load factor <= 1/16 up to 2^22 configurations, 1/8 up to 2^26, else 1/4: a warp's probe
    // loop runs as long as its longest probe sequence, so short runs of occupied slots matter
    // more than memory (the 2-byte fingerprints of 2^26 slots take 128 MiB, about the L2 size)
    const uint64_t load = slots_per_det > 0 ? (uint64_t)slots_per_det
                          : nS <= ((int64_t)1 << 22) ? 16
                          : (nS <= ((int64_t)1 << 26) ? 8 : 4);
    uint64_t cap = 1024;
    while (cap < load * (uint64_t)nS) cap <<= 1;
    int32_t* idx;
    uint16_t* fp;
    NQS_TRY(sc.get(&idx, cap));
    NQS_TRY(sc.get(&fp, cap));
    k_hash_clear<<<grid_for(cap, 256), 256, 0, s>>>(idx, fp, cap);
    NQS_CK_LAUNCH();
    k_hash_insert<<<grid_for(nS, 256), 256, 0, s>>>((const ulonglong2*)dets, nS, idx, cap - 1);
    NQS_CK_LAUNCH();
    k_hash_fp<<<grid_for(cap, 256), 256, 0, s>>>((const ulonglong2*)dets, idx, fp, cap);
    NQS_CK_LAUNCH();
    out->set = (const ulonglong2*)dets;
    out->idx = idx;
    out->fp = fp;
    out->mask = cap - 1;
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// diagonal elements
// ------------------------------------------------------------------------------------------
__global__ void k_diag(ProblemDev P, const ulonglong2* dets, int64_t n, double* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        ulonglong2 x = dets[i];
        out[i] = diag_element_impl(P, x.x, x.y);
    }
}

extern "C" int nqs_diag(nqs_problem* p, const uint64_t* dets, int64_t n, double* out,
                        nqs_stream_t stream) {
    if (!p || (n > 0 && (!dets || !out)) || n < 0) return NQS_ERR_ARG;
    if (n == 0) return NQS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_diag<<<grid_for(n, 128), 128, 0, s>>>(p->d, (const ulonglong2*)dets, n, out);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

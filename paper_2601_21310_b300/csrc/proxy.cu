// Proxy-mode Hamiltonian, Eq. (proxy_hamiltonian) of Sec. 2.4.1, as a CSR over T = V + P:
//   (H~)_xy = H_xy when x or y lies in V, H_xx on the diagonal, 0 between distinct members of P.
// E_proxy (Eq. proxy_energy) and its gradient (Eq. proxy_gradient) are then the Rayleigh
// quotient and the gradient that nqs_energy_grad computes over T with this matrix.
//
// Rows of V: the H_SS enumeration of connect.cu with the hash table of all of T (columns are
// positions in T). Rows of P: the diagonal, then the transpose of the V rows' entries whose
// column lies in P: those entries are flagged, compacted, and radix-sorted by their P column
// (stable, so each P row lists its V columns in ascending order); H is symmetric bit for bit, so
// the transposed value is the element itself.
#include <string.h>

#include "excite.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

__global__ void k_proxy_flags(const int32_t* __restrict__ col, int64_t nnz, int32_t nV,
                              uint32_t* __restrict__ f) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        f[k] = col[k] >= nV ? 1u : 0u;
}

// keys = P index of the column, payload = entry position (as the 8 bytes of the sort's value)
__global__ void k_proxy_emit(const int32_t* __restrict__ col, int64_t nnz, int32_t nV,
                             const uint32_t* __restrict__ f, const uint32_t* __restrict__ at,
                             uint32_t* __restrict__ keys, int64_t* __restrict__ pos,
                             int* __restrict__ cntP) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (!f[k]) continue;
        const uint32_t q = (uint32_t)(col[k] - nV);
        keys[at[k]] = q;
        pos[at[k]] = k;
        atomicAdd(&cntP[q], 1);
    }
}

// row lengths over T: V rows from their CSR, P rows 1 + number of V neighbours
__global__ void k_proxy_rowlen(const int64_t* __restrict__ rpV, int64_t nV, const int* __restrict__ cntP,
                               int64_t nP, int64_t* __restrict__ len) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nV + nP;
         r += (int64_t)gridDim.x * blockDim.x)
        len[r] = r < nV ? rpV[r + 1] - rpV[r] : 1 + (int64_t)cntP[r - nV];
}

// flag[0] = 1 when a configuration of T does not find itself in the hash table (it occurs twice)
__global__ void k_proxy_unique(HashS H, const ulonglong2* __restrict__ T, int64_t nT,
                               int* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nT;
         i += (int64_t)gridDim.x * blockDim.x) {
        const ulonglong2 x = T[i];
        if (hash_lookup(H, x.x, x.y) != (int32_t)i) atomicOr(flag, 1);
    }
}

__global__ void k_i32_to_i64(const int* __restrict__ a, int64_t n, int64_t* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void k_proxy_copy_v(const int32_t* __restrict__ colV, const double* __restrict__ valV,
                               int64_t nnzV, int32_t* __restrict__ col, double* __restrict__ val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnzV;
         k += (int64_t)gridDim.x * blockDim.x) {
        col[k] = colV[k];
        val[k] = valV[k];
    }
}

// P rows: the diagonal first
__global__ void k_proxy_diag_p(ProblemDev P, const ulonglong2* __restrict__ T, int64_t nV,
                               int64_t nP, const int64_t* __restrict__ row_ptr,
                               int32_t* __restrict__ col, double* __restrict__ val) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nP;
         q += (int64_t)gridDim.x * blockDim.x) {
        const ulonglong2 x = T[nV + q];
        const int64_t at = row_ptr[nV + q];
        col[at] = (int32_t)(nV + q);
        val[at] = diag_element_impl(P, x.x, x.y);
    }
}

// sorted entry t (P index key, V-CSR position k): its V row (the column in T) by binary search
// in the V row pointers, written after the diagonal of its P row in sorted order
__global__ void k_proxy_fill_p(const uint32_t* __restrict__ keys, const int64_t* __restrict__ pos,
                               int64_t n, const int64_t* __restrict__ offP,
                               const int64_t* __restrict__ rpV, int64_t nV,
                               const double* __restrict__ valV, const int64_t* __restrict__ row_ptr,
                               int32_t* __restrict__ col, double* __restrict__ val) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q = keys[t];
        const int64_t k = pos[t];
        int64_t lo = 0, hi = nV;  // largest r with rpV[r] <= k
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (rpV[mid] <= k) lo = mid;
            else hi = mid;
        }
        const int64_t at = row_ptr[nV + q] + 1 + (t - offP[q]);
        col[at] = (int32_t)lo;
        val[at] = valV[k];
    }
}

extern "C" int nqs_proxy_hamiltonian(nqs_problem* p, const uint64_t* T, int64_t nV, int64_t nT,
                                     const nqs_opts* opts, nqs_csr* out, nqs_stream_t stream) {
    if (!p || !T || !out || nV <= 0 || nT < nV) return NQS_ERR_ARG;
    if (nT >= ((int64_t)1 << 31)) return NQS_ERR_UNSUPPORTED;
    if (((uintptr_t)T) & 15) return NQS_ERR_ARG;
    memset(out, 0, sizeof *out);
    cudaStream_t s = (cudaStream_t)stream;
    nqs_opts def;
    if (!opts) {
        nqs_opts_default(&def);
        opts = &def;
    }
    const int64_t nP = nT - nV;
    Scratch sc(p, s);
    if (opts->validate) {
        NQS_TRY(validate_dets(p, sc, T, nV, true, s));
        if (nP > 0) NQS_TRY(validate_dets(p, sc, T + 2 * nV, nP, true, s));
    }
    HashS H;
    NQS_TRY(hash_build(p, sc, T, nT, &H, s));
    if (opts->validate) {  // V and P disjoint: every configuration finds its own position
        int* flag;
        NQS_TRY(sc.get(&flag, 1));
        NQS_CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
        k_proxy_unique<<<grid_for(nT, 256), 256, 0, s>>>(H, (const ulonglong2*)T, nT, flag);
        NQS_CK_LAUNCH();
        int hf = 0;
        NQS_CK(cudaMemcpyAsync(&hf, flag, sizeof hf, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        if (hf) {
            nqs_record_message("nqs_proxy_hamiltonian: a configuration occurs in both V and P");
            return NQS_ERR_UNSORTED;
        }
    }
    const size_t smem = conn_smem_bytes(p->d);
    if (smem > 48 * 1024) {
        NQS_CK(cudaFuncSetAttribute(k_conn_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
        NQS_CK(cudaFuncSetAttribute(k_conn_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    }
    // rows of V: every connection inside T, one probe of the hash of T per excitation. The
    // indexed pass of nqs_connections (scans of alpha and beta runs) is slower here: T is much
    // larger than V, so the runs it would scan are long (measured at 16 and 30 orbitals)
    int64_t *rowcnt, *rpV;
    uint32_t* bits;
    NQS_TRY(sc.get(&rowcnt, nV));
    NQS_TRY(sc.get(&rpV, nV + 1));
    NQS_TRY(sc.get(&bits, (size_t)nV * ((p->d.nexc + 31) / 32)));
    {
        ProfScope prof_(PROF_CONN_COUNT, s);
        k_conn_count<<<conn_grid_size(nV), CONN_THREADS, smem, s>>>(p->d, H, (const ulonglong2*)T,
                                                                     nV, rowcnt, bits);
    }
    NQS_CK_LAUNCH();
    NQS_TRY(scan_exclusive_i64(p, sc, rowcnt, rpV, nV, rpV + nV, s));
    int64_t nnzV = 0;
    NQS_CK(cudaMemcpyAsync(&nnzV, rpV + nV, sizeof nnzV, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    if (nnzV >= ((int64_t)1 << 32)) {
        nqs_record_message("nqs_proxy_hamiltonian: 2^32 or more nonzeros in the rows of V");
        return NQS_ERR_UNSUPPORTED;
    }
    int32_t* colV;
    double* valV;
    NQS_TRY(sc.get(&colV, nnzV));
    NQS_TRY(sc.get(&valV, nnzV));
    {
        ProfScope prof_(PROF_CONN_FILL, s);
        k_conn_fill<<<conn_grid_size(nV), CONN_THREADS, smem, s>>>(
            p->d, H, (const ulonglong2*)T, nV, rpV, colV, valV, bits);
    }
    NQS_CK_LAUNCH();
    // V -> P entries, transposed into the rows of P
    uint32_t *f, *at, *keys, *keys2;
    int64_t *pos, *pos2, *offP, *len;
    int* cntP;
    NQS_TRY(sc.get(&f, nnzV));
    NQS_TRY(sc.get(&at, nnzV));
    NQS_TRY(sc.get(&cntP, nP));
    NQS_TRY(sc.get(&offP, nP + 1));
    NQS_CK(cudaMemsetAsync(cntP, 0, (nP > 0 ? nP : 1) * sizeof(int), s));
    const unsigned g = grid_for(nnzV, 256);
    k_proxy_flags<<<g, 256, 0, s>>>(colV, nnzV, (int32_t)nV, f);
    NQS_CK_LAUNCH();
    NQS_TRY(scan_exclusive_u32(p, sc, f, at, nnzV, s));
    uint32_t last_at = 0, last_f = 0;
    if (nnzV > 0) {
        NQS_CK(cudaMemcpyAsync(&last_at, at + nnzV - 1, 4, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaMemcpyAsync(&last_f, f + nnzV - 1, 4, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
    }
    const int64_t nVP = (int64_t)last_at + last_f;
    NQS_TRY(sc.get(&keys, nVP));
    NQS_TRY(sc.get(&keys2, nVP));
    NQS_TRY(sc.get(&pos, nVP));
    NQS_TRY(sc.get(&pos2, nVP));
    k_proxy_emit<<<g, 256, 0, s>>>(colV, nnzV, (int32_t)nV, f, at, keys, pos, cntP);
    NQS_CK_LAUNCH();
    if (nVP > 1) {
        int bits_p = 1;
        while (bits_p < 32 && ((int64_t)1 << bits_p) < nP) ++bits_p;
        NQS_TRY(radix_sort_pairs32(p, sc, keys, (double*&)pos, keys2, (double*&)pos2, nVP,
                                   bits_p, s));
    }
    // row pointers over T
    NQS_TRY(sc.get(&len, nT));
    k_proxy_rowlen<<<grid_for(nT, 256), 256, 0, s>>>(rpV, nV, cntP, nP, len);
    NQS_CK_LAUNCH();
    // the matrix comes from the problem's stream-ordered pool: no device-wide synchronisation
    // to allocate it, and nqs_csr_free_async returns it in stream order
    int64_t* row_ptr = nullptr;
    NQS_TRY(nqs_scratch_alloc(p, (void**)&row_ptr, (nT + 1) * sizeof(int64_t), s));
    auto fail = [&](int code) {
        nqs_scratch_free(p, row_ptr, s);
        return code;
    };
    int st = scan_exclusive_i64(p, sc, len, row_ptr, nT, row_ptr + nT, s);
    if (st < 0) return fail(st);
    int64_t* cnt64;
    st = sc.get(&cnt64, nP);
    if (st < 0) return fail(st);
    if (nP > 0) {
        // offsets of each P column's run in the sorted entries: exclusive scan of cntP
        k_i32_to_i64<<<grid_for(nP, 256), 256, 0, s>>>(cntP, nP, cnt64);
        nqs_note_launch();
        st = scan_exclusive_i64(p, sc, cnt64, offP, nP, offP + nP, s);
        if (st < 0) return fail(st);
    }
    int64_t nnz = 0;
    if (cudaMemcpyAsync(&nnz, row_ptr + nT, sizeof nnz, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(NQS_ERR_CUDA);
    int32_t* col = nullptr;
    double* val = nullptr;
    if (nqs_scratch_alloc(p, (void**)&col, (nnz > 0 ? nnz : 1) * sizeof(int32_t), s) != NQS_OK ||
        nqs_scratch_alloc(p, (void**)&val, (nnz > 0 ? nnz : 1) * sizeof(double), s) != NQS_OK) {
        nqs_scratch_free(p, col, s);
        return fail(NQS_ERR_OOM);
    }
    k_proxy_copy_v<<<grid_for(nnzV, 256), 256, 0, s>>>(colV, valV, nnzV, col, val);
    nqs_note_launch();
    if (nP > 0) {
        k_proxy_diag_p<<<grid_for(nP, 256), 256, 0, s>>>(p->d, (const ulonglong2*)T, nV, nP,
                                                         row_ptr, col, val);
        nqs_note_launch();
    }
    if (nVP > 0) {
        k_proxy_fill_p<<<grid_for(nVP, 256), 256, 0, s>>>(keys, pos, nVP, offP, rpV, nV, valV,
                                                          row_ptr, col, val);
        nqs_note_launch();
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        nqs_scratch_free(p, col, s);
        nqs_scratch_free(p, val, s);
        nqs_record_error("nqs_proxy_hamiltonian", e, __FILE__, __LINE__);
        return fail(NQS_ERR_CUDA);
    }
    out->row_ptr = row_ptr;
    out->col = col;
    out->val = val;
    out->nnz = nnz;
    out->n_rows = nT;
    return NQS_OK;
}

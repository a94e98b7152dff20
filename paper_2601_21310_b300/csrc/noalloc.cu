// nqs_connections_noalloc: the H_SS build for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or a stream-ordered allocator at all: code that runs
// inside a host that owns every device allocation (a framework with its own arena that gives
// the library none) or an embedded solver that runs on a fixed device budget. For them this
// entry point does the same work as
// nqs_connections with all inputs and outputs passed in and its scratch (the hash table of S,
// the per-row counts, the scan partials and the validation flags) in one file-scope device
// array of fixed size, NQS_NOALLOC_SCRATCH_BYTES. Every GPU that loads this library holds that
// array until the process exits.
//
// The host cannot use the array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device, with that device current, looks the address up
// with cudaGetSymbolAddress and caches it. The cache assumes the device's primary context
// lives until the process exits (a cudaDeviceReset would leave a stale address behind). The call synchronises its stream: it reads the number
// of nonzeros back to the host before writing the columns.
// All calls share the array and it keeps the previous call's contents: everything that must
// start from zero is cleared on every call, and calls whose work overlaps on the GPU (two
// streams, two host threads) race on it and must be serialised by the caller.
#include <string.h>

#include <mutex>

#include "excite.cuh"
#include "nqs_internal.cuh"

#define NQS_NOALLOC_MAX_DETS 65536
#define NQS_NOALLOC_SCRATCH_BYTES (8u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[NQS_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];  // per device ordinal

static int noalloc_scratch_address(void** out) {
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return NQS_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            nqs_record_error("cudaGetSymbolAddress(g_noalloc_scratch)", e, __FILE__, __LINE__);
            return NQS_ERR_CUDA;
        }
        g_noalloc_addr[dev] = ptr;
    }
    *out = g_noalloc_addr[dev];
    return NQS_OK;
}

extern "C" int nqs_connections_noalloc(nqs_problem* p, const uint64_t* dets, int64_t nS,
                                       int validate, int64_t* row_ptr, int32_t* col,
                                       double* val, int64_t capacity, int64_t* nnz,
                                       int64_t* n_enumerated, nqs_stream_t stream) {
    if (!p || !dets || !row_ptr || !nnz || nS <= 0 || capacity < 0) return NQS_ERR_ARG;
    if (((uintptr_t)dets) & 15) return NQS_ERR_ARG;
    if (nS > NQS_NOALLOC_MAX_DETS) {
        nqs_record_message("nqs_connections_noalloc: nS exceeds the static scratch limit of 65536 "
                           "determinants; use nqs_connections");
        return NQS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void* arena = nullptr;
    NQS_TRY(noalloc_scratch_address(&arena));
    Scratch sc(arena, NQS_NOALLOC_SCRATCH_BYTES, s);
    if (validate) NQS_TRY(validate_dets(p, sc, dets, nS, true, s));
    HashS H;
    NQS_TRY(hash_build(p, sc, dets, nS, &H, s, 4));  // load factor 1/4 within the static scratch
    size_t smem = conn_smem_bytes(p->d);
    if (smem > 48 * 1024) {
        NQS_CK(cudaFuncSetAttribute(k_conn_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
        NQS_CK(cudaFuncSetAttribute(k_conn_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    }
    int64_t* rowcnt;
    NQS_TRY(sc.get(&rowcnt, nS));
    k_conn_count<<<conn_grid_size(nS), CONN_THREADS, smem, s>>>(p->d, H, (const ulonglong2*)dets,
                                                                nS, rowcnt, nullptr);
    NQS_CK_LAUNCH();
    NQS_TRY(scan_exclusive_i64(p, sc, rowcnt, row_ptr, nS, row_ptr + nS, s));
    int64_t total = 0;
    NQS_CK(cudaMemcpyAsync(&total, row_ptr + nS, sizeof total, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    *nnz = total;
    if (n_enumerated) *n_enumerated = nS * p->d.nexc;
    if (total > capacity || (total > 0 && (!col || !val))) {
        nqs_record_message("nqs_connections_noalloc: col/val capacity smaller than nnz; *nnz holds "
                           "the size needed");
        return NQS_ERR_ARG;
    }
    k_conn_fill<<<conn_grid_size(nS), CONN_THREADS, smem, s>>>(p->d, H, (const ulonglong2*)dets,
                                                               nS, row_ptr, col, val, nullptr);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

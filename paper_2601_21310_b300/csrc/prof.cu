// Per-kernel CUDA-event timing registry (see prof.cuh).
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "nqs_internal.cuh"
#include "prof.cuh"

bool g_prof_on = false;
static std::atomic<long long> g_launches{0};

void nqs_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" int64_t nqs_launch_count(void) { return (int64_t)g_launches.load(); }

static const char* kNames[PROF_N] = {"conn_count", "conn_fill", "pt2_count", "pt2_emit",
                                     "rs_hist",    "rs_scatter", "seg_reduce", "gemm",
                                     "lu",         "spmv",      "layer1",    "unique_terms",
                                     "heads",      "scan",      "hb_select",
                                     "select"};

struct EvPair {
    cudaEvent_t a, b;
};
static std::mutex g_mu;
static std::vector<EvPair> g_open[PROF_N];
static std::vector<EvPair> g_done[PROF_N];
static std::vector<cudaEvent_t> g_free;

static cudaEvent_t get_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(int id, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    EvPair p;
    p.a = get_event();
    p.b = nullptr;
    cudaEventRecord(p.a, s);
    g_open[id].push_back(p);
}

void prof_end(int id, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_open[id].empty()) return;
    EvPair p = g_open[id].back();
    g_open[id].pop_back();
    p.b = get_event();
    cudaEventRecord(p.b, s);
    g_done[id].push_back(p);
}

extern "C" int nqs_profile_enable(int on) {
    g_prof_on = on != 0;
    return NQS_OK;
}

extern "C" int nqs_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < PROF_N; ++i) {
        for (auto& p : g_done[i]) {
            g_free.push_back(p.a);
            g_free.push_back(p.b);
        }
        g_done[i].clear();
    }
    return NQS_OK;
}

extern "C" int nqs_profile_read(const char* name, double* total_ms, int64_t* launches) {
    if (!name || !total_ms || !launches) return NQS_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < PROF_N; ++i) {
        if (strcmp(name, kNames[i]) != 0) continue;
        double t = 0;
        for (auto& p : g_done[i]) {
            if (cudaEventSynchronize(p.b) != cudaSuccess) return NQS_ERR_CUDA;
            float ms = 0;
            if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) return NQS_ERR_CUDA;
            t += ms;
        }
        *total_ms = t;
        *launches = (int64_t)g_done[i].size();
        return NQS_OK;
    }
    return NQS_ERR_ARG;
}

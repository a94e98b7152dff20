// Optional per-kernel timing with CUDA events recorded on the launching stream. Off by
// default; when on, every instrumented launch is bracketed by two events and the elapsed
// times are summed per kernel name when read back.
#pragma once
#include <cuda_runtime.h>

enum ProfId {
    PROF_CONN_COUNT = 0,
    PROF_CONN_FILL,
    PROF_PT2_COUNT,
    PROF_PT2_EMIT,
    PROF_RS_HIST,
    PROF_RS_SCATTER,
    PROF_SEG_REDUCE,
    PROF_GEMM,
    PROF_LU,
    PROF_SPMV,
    PROF_LAYER1,
    PROF_UNIQUE,
    PROF_HEADS,
    PROF_SCAN,
    PROF_HB_SELECT,
    PROF_SELECT,
    PROF_N
};

extern bool g_prof_on;
void prof_begin(int id, cudaStream_t s);
void prof_end(int id, cudaStream_t s);

struct ProfScope {
    int id;
    cudaStream_t s;
    ProfScope(int id_, cudaStream_t s_) : id(id_), s(s_) {
        if (g_prof_on) prof_begin(id, s);
    }
    ~ProfScope() {
        if (g_prof_on) prof_end(id, s);
    }
};

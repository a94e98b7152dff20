// Batched E_S + gradient over many independent problems (uneven orbital counts and |S|).
//
// The batch fans the problems out over a pool of side streams (largest |S| first, round
// robin), each problem running its whole energy/gradient pipeline on its stream, and joins
// them back to the caller's stream. nqs_batch_capture records that fork/join once into a CUDA
// graph (stream-ordered scratch allocations become graph memory nodes; nothing synchronises
// the host), so a step is then one graph launch. GEMM tile widths are taken from the
// autotuner's table, filled by an eager run with tuning enabled before capture.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "nqs_internal.cuh"

struct nqs_batch {
    int n;
    std::vector<nqs_problem*> prob;
    std::vector<nqs_net*> net;
    std::vector<nqs_csr> csr;
    std::vector<const uint64_t*> dets;
    std::vector<int64_t> nS;
    std::vector<double*> out;
    std::vector<void*> grad;
    std::vector<int> order;  // problems by decreasing |S|
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" int nqs_batch_destroy(nqs_batch* b) {
    if (!b) return NQS_OK;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto s : b->side) cudaStreamDestroy(s);
    delete b;
    return NQS_OK;
}

extern "C" int nqs_batch_create(int n, nqs_problem* const* problems, nqs_net* const* nets,
                                const nqs_csr* csrs, const uint64_t* const* dets,
                                const int64_t* nS, double* const* outs, void* const* grads,
                                int nstreams, nqs_batch** out) {
    if (!out || n <= 0 || !problems || !nets || !csrs || !dets || !nS || !outs || !grads)
        return NQS_ERR_ARG;
    if (nstreams < 1) nstreams = 1;
    if (nstreams > n) nstreams = n;
    nqs_batch* b = new nqs_batch();
    b->n = n;
    for (int i = 0; i < n; ++i) {
        if (!problems[i] || !nets[i] || !dets[i] || nS[i] <= 0 || !outs[i] ||
            nets[i]->prob != problems[i] || csrs[i].n_rows != nS[i]) {
            delete b;
            return NQS_ERR_ARG;
        }
        b->prob.push_back(problems[i]);
        b->net.push_back(nets[i]);
        b->csr.push_back(csrs[i]);
        b->dets.push_back(dets[i]);
        b->nS.push_back(nS[i]);
        b->out.push_back(outs[i]);
        b->grad.push_back(grads[i]);
    }
    b->order.resize(n);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return b->nS[x] > b->nS[y]; });
    auto fail = [&](int code) {
        nqs_batch_destroy(b);
        return code;
    };
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(NQS_ERR_CUDA);
    for (int k = 0; k < nstreams; ++k) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return fail(NQS_ERR_CUDA);
        b->side.push_back(s);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(NQS_ERR_CUDA);
        b->join.push_back(e);
    }
    *out = b;
    return NQS_OK;
}

// fork to the side streams, one energy/gradient pipeline per problem, join back
extern "C" int nqs_batch_run(nqs_batch* b, nqs_stream_t stream) {
    if (!b) return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    NQS_CK(cudaEventRecord(b->fork, s));
    const int ns = (int)b->side.size();
    for (int k = 0; k < ns; ++k) NQS_CK(cudaStreamWaitEvent(b->side[k], b->fork, 0));
    for (int t = 0; t < b->n; ++t) {
        const int i = b->order[t];
        nqs_opts o;
        nqs_opts_default(&o);
        o.precision = b->net[i]->dtype;
        o.validate = 0;
        NQS_TRY(nqs_energy_grad(b->prob[i], b->net[i], &b->csr[i], b->dets[i], b->nS[i], b->out[i],
                                b->grad[i], nullptr, &o, (nqs_stream_t)b->side[t % ns]));
    }
    for (int k = 0; k < ns; ++k) {
        NQS_CK(cudaEventRecord(b->join[k], b->side[k]));
        NQS_CK(cudaStreamWaitEvent(s, b->join[k], 0));
    }
    return NQS_OK;
}

extern "C" int nqs_batch_capture(nqs_batch* b, nqs_stream_t stream) {
    if (!b || !stream) return NQS_ERR_ARG;  // the legacy default stream cannot be captured
    cudaStream_t s = (cudaStream_t)stream;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    NQS_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    int st = nqs_batch_run(b, stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st < 0) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        nqs_record_error("cudaStreamEndCapture", e, __FILE__, __LINE__);
        return NQS_ERR_CUDA;
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        nqs_record_error("cudaGraphInstantiate", e, __FILE__, __LINE__);
        b->exec = nullptr;
        return NQS_ERR_CUDA;
    }
    return NQS_OK;
}

extern "C" int nqs_batch_launch(nqs_batch* b, nqs_stream_t stream) {
    if (!b || !b->exec) return NQS_ERR_ARG;
    NQS_CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return NQS_OK;
}

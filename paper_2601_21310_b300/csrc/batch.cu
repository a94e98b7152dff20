// Batched E_S + gradient over many independent problems (uneven orbital counts and |S|).
//
// Two modes.
//   NQS_BATCH_GROUPED (the default when every problem qualifies): the pipeline runs stage by
//     stage, each stage one launch over all problems: the input bits and weight copies, the
//     three forward layers as grouped persistent tcgen05 GEMMs over a (problem, tile) work list,
//     the LU factorisations (one launch per block size), the energy stage (max log|psi|, psi~,
//     SpMV, compensated N and D, E, adjoint weights), the adjoint into dPhi, and the backward
//     layers and weight gradients as grouped GEMMs. A step is about twenty launches whatever the
//     number of problems; the workspace and every GEMM descriptor are built once, and each GEMM
//     stage's tile width is picked by the autotuner (timed on first use) or by the width rule.
//   NQS_BATCH_STREAMS: the problems fan out over a pool of side streams (largest |S| first,
//     round robin), each running its whole nqs_energy_grad pipeline, and join back.
// nqs_batch_capture records one run into a CUDA graph, so a step is then one graph launch.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <vector>

#include "ansatz.cuh"
#include "ksum.cuh"
#include "nqs_internal.cuh"

// grouped mode: workspace, descriptors and GEMM sets
struct GroupedState {
    void* ws = nullptr;
    GProb* dP = nullptr;
    std::vector<GProb> hP;
    GDims dims;
    double2* kpart = nullptr;
    int64_t* tile_off = nullptr;  // prefix of the problems' dPhi transpose tiles
    int64_t tiles = 0;
    bool with_grad = false;
    std::vector<int> lu_n;
    std::vector<GLuJob*> lu_jobs;
    std::vector<int> lu_count;
    TcGroupSet* sets[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int bn[6] = {0, 0, 0, 0, 0, 0};
    ~GroupedState() {
        cudaFree(ws);
        cudaFree(dP);
        cudaFree(kpart);
        cudaFree(tile_off);
        for (auto j : lu_jobs) cudaFree(j);
        for (auto t : sets) tc_group_set_destroy(t);
    }
};

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
    int mode = NQS_BATCH_STREAMS;
    GroupedState* g = nullptr;
};

// every problem in the mixed form with tensor-core shapes, one micro-batch, FP32 register LU,
// and gradients for all problems or for none
static bool grouped_eligible(const nqs_batch* b) {
    const bool any_grad = b->grad[0] != nullptr;
    for (int i = 0; i < b->n; ++i) {
        const nqs_net* net = b->net[i];
        const ProblemDev& P = b->prob[i]->d;
        if (net->dtype != NQS_MIXED || net->H1 % 8 || net->H2 % 8) return false;
        if (b->nS[i] > ((int64_t)1 << 20) || P.na > 12 || P.nb > 12) return false;
        if ((b->grad[i] != nullptr) != any_grad) return false;
        if (b->prob[i]->device != b->prob[0]->device) return false;
    }
    return true;
}

extern "C" int nqs_batch_destroy(nqs_batch* b) {
    if (!b) return NQS_OK;
    cudaDeviceSynchronize();
    delete b->g;
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
    b->mode = grouped_eligible(b) ? NQS_BATCH_GROUPED : NQS_BATCH_STREAMS;
    *out = b;
    return NQS_OK;
}

extern "C" int nqs_batch_set_mode(nqs_batch* b, int mode) {
    if (!b || (mode != NQS_BATCH_STREAMS && mode != NQS_BATCH_GROUPED)) return NQS_ERR_ARG;
    if (mode == NQS_BATCH_GROUPED && !grouped_eligible(b)) return NQS_ERR_UNSUPPORTED;
    if (mode != b->mode && b->exec) {  // a recorded graph belongs to the other mode
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    b->mode = mode;
    return NQS_OK;
}

extern "C" int nqs_batch_get_mode(const nqs_batch* b) { return b ? b->mode : NQS_ERR_ARG; }

// ------------------------------------------------------------------------------------------
// grouped mode
// ------------------------------------------------------------------------------------------
static int64_t r8(int64_t v) { return (v + 7) & ~(int64_t)7; }

// time one launch of a grouped GEMM set on stream s (one warm-up, two timed)
static int time_set(const TcGroupSet* set, cudaStream_t s, float* ms) {
    cudaEvent_t e0, e1;
    NQS_CK(cudaEventCreate(&e0));
    NQS_CK(cudaEventCreate(&e1));
    int st = tc_group_set_launch(set, s);
    if (st == NQS_OK) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2 && st == NQS_OK; ++r) st = tc_group_set_launch(set, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            st = NQS_ERR_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// one grouped GEMM set per stage: with tuning on, the fastest of the tile widths 64/128/256
// (timed here, outside any capture); otherwise the width rule of the single GEMM for the
// stage's widest output
static int build_set(const std::vector<TcGemm>& gs, cudaStream_t s, TcGroupSet** out, int* bn) {
    int maxN = 0;
    for (const auto& g : gs) maxN = g.N > maxN ? g.N : maxN;
    const int rule = maxN <= 64 ? 64 : (maxN <= 128 ? 128 : 256);
    if (!tc_autotune_on()) {
        *bn = rule;
        return tc_group_set_create(gs.data(), (int)gs.size(), rule, out);
    }
    TcGroupSet* best = nullptr;
    float best_ms = 1e30f;
    int best_bn = rule;
    for (int w : {64, 128, 256}) {
        if (w >= 2 * ((maxN + 63) / 64 * 64)) continue;
        TcGroupSet* t = nullptr;
        NQS_TRY(tc_group_set_create(gs.data(), (int)gs.size(), w, &t));
        float ms = 0;
        const int st = time_set(t, s, &ms);
        if (st < 0) {
            tc_group_set_destroy(t);
            tc_group_set_destroy(best);
            return st;
        }
        if (ms < best_ms) {
            tc_group_set_destroy(best);
            best = t;
            best_ms = ms;
            best_bn = w;
        } else {
            tc_group_set_destroy(t);
        }
    }
    *out = best;
    *bn = best_bn;
    return NQS_OK;
}

static int grouped_prepare(nqs_batch* b, cudaStream_t s) {
    if (b->g) return NQS_OK;
    GroupedState* G = new GroupedState();
    auto fail = [&](int code) {
        delete G;
        return code;
    };
    const int n = b->n;
    G->with_grad = b->grad[0] != nullptr;
    G->hP.resize(n);
    // workspace sizes, 256-byte aligned slices of one allocation
    size_t total = 0;
    auto take = [&](size_t bytes) {
        const size_t off = total;
        total += (bytes + 255) & ~(size_t)255;
        return off;
    };
    struct Off {
        size_t X, XT, W1p, H1a, H1T, H2a, H2T, W2T, W3T, dPhi, dPhiT, dZ2, dZ2T, dZ1T, Phi, Aa, Ab,
            la2, logabs, psi, v, w, ex2, sg2, sign, sing;
    };
    std::vector<Off> off(n);
    GDims d;
    memset(&d, 0, sizeof d);
    d.np = n;
    for (int i = 0; i < n; ++i) {
        const nqs_net* net = b->net[i];
        const ProblemDev& P = b->prob[i]->d;
        GProb& q = G->hP[i];
        memset(&q, 0, sizeof q);
        q.dets = (const ulonglong2*)b->dets[i];
        q.M = b->nS[i];
        q.norb = P.norb;
        q.na = P.na;
        q.nb = P.nb;
        q.nin = net->nin;
        q.nout = net->nout;
        q.H1 = net->H1;
        q.H2 = net->H2;
        q.ldX = (int)r8(net->nin);
        q.ldM = r8(q.M);
        q.ldP = r8(net->nout);
        q.W1 = (const __nv_bfloat16*)net->p[0];
        q.b1 = (const float*)net->p[1];
        q.W2 = (const __nv_bfloat16*)net->p[2];
        q.b2 = (const float*)net->p[3];
        q.W3 = (const __nv_bfloat16*)net->p[4];
        q.b3 = (const float*)net->p[5];
        q.phi0 = (const float*)net->p[6];
        q.rp = b->csr[i].row_ptr;
        q.col = b->csr[i].col;
        q.val = b->csr[i].val;
        q.out = b->out[i];
        q.grad = (float*)b->grad[i];
        const int64_t M = q.M;
        Off& o = off[i];
        o.X = take(M * q.ldX * 2);
        o.XT = take((size_t)q.nin * q.ldM * 2);
        o.W1p = take((size_t)q.H1 * q.ldX * 2);
        o.H1a = take(M * q.H1 * 2);
        o.H1T = take((size_t)q.H1 * q.ldM * 2);
        o.H2a = take(M * q.H2 * 2);
        o.H2T = take((size_t)q.H2 * q.ldM * 2);
        o.W2T = take((size_t)q.H1 * q.H2 * 2);
        o.W3T = take((size_t)q.H2 * q.ldP * 2);
        o.dPhi = take(M * q.ldP * 2);
        o.dPhiT = take((size_t)q.nout * q.ldM * 2);
        o.dZ2 = take(M * q.H2 * 2);
        o.dZ2T = take((size_t)q.H2 * q.ldM * 2);
        o.dZ1T = take((size_t)q.H1 * q.ldM * 2);
        o.Phi = take(M * q.nout * 4);
        o.Aa = take(M * q.na * q.na * 4);
        o.Ab = take(M * q.nb * q.nb * 4);
        o.la2 = take(2 * M * 8);
        o.logabs = take(M * 8);
        o.psi = take(M * 8);
        o.v = take(M * 8);
        o.w = take(M * 8);
        o.ex2 = take(2 * M * 4);
        o.sg2 = take(2 * M);
        o.sign = take(M);
        o.sing = take(4);
        d.maxM = std::max<int64_t>(d.maxM, M);
        d.maxMX = std::max<int64_t>(d.maxMX, M * (q.ldX / 8));
        d.max_nin = std::max(d.max_nin, q.nin);
        d.max_nout = std::max(d.max_nout, q.nout);
        d.max_H = std::max(d.max_H, std::max(q.H1, q.H2));
    }
    G->dims = d;
    if (cudaMalloc(&G->ws, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(NQS_ERR_OOM);
    }
    uint8_t* base = (uint8_t*)G->ws;
    for (int i = 0; i < n; ++i) {
        GProb& q = G->hP[i];
        const Off& o = off[i];
        q.X = (__nv_bfloat16*)(base + o.X);
        q.XT = (__nv_bfloat16*)(base + o.XT);
        q.W1p = (__nv_bfloat16*)(base + o.W1p);
        q.H1a = (__nv_bfloat16*)(base + o.H1a);
        q.H1T = (__nv_bfloat16*)(base + o.H1T);
        q.H2a = (__nv_bfloat16*)(base + o.H2a);
        q.H2T = (__nv_bfloat16*)(base + o.H2T);
        q.W2T = (__nv_bfloat16*)(base + o.W2T);
        q.W3T = (__nv_bfloat16*)(base + o.W3T);
        q.dPhi = (__nv_bfloat16*)(base + o.dPhi);
        q.dPhiT = (__nv_bfloat16*)(base + o.dPhiT);
        q.dZ2 = (__nv_bfloat16*)(base + o.dZ2);
        q.dZ2T = (__nv_bfloat16*)(base + o.dZ2T);
        q.dZ1T = (__nv_bfloat16*)(base + o.dZ1T);
        q.Phi = (float*)(base + o.Phi);
        q.Ainv_a = (float*)(base + o.Aa);
        q.Ainv_b = (float*)(base + o.Ab);
        q.la2 = (double*)(base + o.la2);
        q.logabs = (double*)(base + o.logabs);
        q.psi = (double*)(base + o.psi);
        q.v = (double*)(base + o.v);
        q.w = (double*)(base + o.w);
        q.ex2 = (int*)(base + o.ex2);
        q.sg2 = (int8_t*)(base + o.sg2);
        q.sign = (int8_t*)(base + o.sign);
        q.singular = (int*)(base + o.sing);
    }
    // padding columns of X^T / H^T beyond M and of dPhi beyond nout are read as zeros
    if (cudaMemsetAsync(G->ws, 0, total, s) != cudaSuccess) return fail(NQS_ERR_CUDA);
    if (cudaMalloc(&G->dP, sizeof(GProb) * n) != cudaSuccess ||
        cudaMalloc(&G->kpart, sizeof(double2) * 2 * KR_BLOCKS * n) != cudaSuccess) {
        cudaGetLastError();
        return fail(NQS_ERR_OOM);
    }
    if (cudaMemcpy(G->dP, G->hP.data(), sizeof(GProb) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(NQS_ERR_CUDA);
    {
        std::vector<int64_t> toff(n + 1, 0);
        for (int i = 0; i < n; ++i)
            toff[i + 1] = toff[i] + ((G->hP[i].M + 31) / 32) * ((G->hP[i].nout + 31) / 32);
        G->tiles = toff[n];
        if (cudaMalloc(&G->tile_off, sizeof(int64_t) * (n + 1)) != cudaSuccess) {
            cudaGetLastError();
            return fail(NQS_ERR_OOM);
        }
        if (cudaMemcpy(G->tile_off, toff.data(), sizeof(int64_t) * (n + 1),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(NQS_ERR_CUDA);
    }
    // LU jobs by block size (both spins)
    std::map<int, std::vector<GLuJob>> byn;
    for (int i = 0; i < n; ++i) {
        const GProb& q = G->hP[i];
        for (int spin = 0; spin < 2; ++spin) {
            GLuJob j;
            j.dets = q.dets;
            j.M = q.M;
            j.norb = q.norb;
            j.nel = q.na + q.nb;
            j.spin = spin;
            j.Phi = q.Phi;
            j.la = q.la2 + spin * q.M;
            j.ex = q.ex2 + spin * q.M;
            j.sg = q.sg2 + spin * q.M;
            j.Ainv = G->with_grad ? (spin == 0 ? q.Ainv_a : q.Ainv_b) : nullptr;
            j.singular = q.singular;
            byn[spin == 0 ? q.na : q.nb].push_back(j);
        }
    }
    for (auto& kv : byn) {
        GLuJob* dj = nullptr;
        if (cudaMalloc(&dj, sizeof(GLuJob) * kv.second.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(NQS_ERR_OOM);
        }
        G->lu_jobs.push_back(dj);
        if (cudaMemcpy(dj, kv.second.data(), sizeof(GLuJob) * kv.second.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(NQS_ERR_CUDA);
        G->lu_n.push_back(kv.first);
        G->lu_count.push_back((int)kv.second.size());
    }
    // the GEMM stages
    std::vector<TcGemm> st[6];
    int* err = b->prob[0]->err_word;
    for (int i = 0; i < n; ++i) {
        const GProb& q = G->hP[i];
        TcGemm g;
        memset(&g, 0, sizeof g);
        g.err = err;
        g.M = (int)q.M;
        // layer 1: H1 = tanh(X W1p^T + b1), with H1^T
        g.A = q.X; g.lda = q.ldX; g.B = q.W1p; g.ldb = q.ldX; g.N = q.H1; g.K = q.ldX;
        g.epi = EPI_BIAS_TANH; g.bias = q.b1; g.C = q.H1a; g.ldc = q.H1; g.c_bf16 = 1;
        g.CT = q.H1T; g.ldct = q.ldM;
        st[0].push_back(g);
        // layer 2: H2 = tanh(H1 W2^T + b2), with H2^T
        g.A = q.H1a; g.lda = q.H1; g.B = q.W2; g.ldb = q.H1; g.N = q.H2; g.K = q.H1;
        g.bias = q.b2; g.C = q.H2a; g.ldc = q.H2; g.CT = q.H2T;
        st[1].push_back(g);
        // layer 3: Phi = Phi0 + H2 W3^T + b3
        memset(&g, 0, sizeof g);
        g.err = err;
        g.M = (int)q.M;
        g.A = q.H2a; g.lda = q.H2; g.B = q.W3; g.ldb = q.H2; g.N = q.nout; g.K = q.H2;
        g.epi = EPI_BIAS_PHI0; g.bias = q.b3; g.phi0 = q.phi0; g.C = q.Phi; g.ldc = q.nout;
        st[2].push_back(g);
        if (!G->with_grad) continue;
        // dZ2 = (dPhi W3) (1 - H2^2), row-major and transposed
        memset(&g, 0, sizeof g);
        g.err = err;
        g.M = (int)q.M;
        g.A = q.dPhi; g.lda = q.ldP; g.B = q.W3T; g.ldb = q.ldP; g.N = q.H2; g.K = q.nout;
        g.epi = EPI_TANH_BWD; g.aux = q.H2a; g.ld_aux = q.H2; g.C = q.dZ2; g.ldc = q.H2;
        g.c_bf16 = 1; g.CT = q.dZ2T; g.ldct = q.ldM;
        st[3].push_back(g);
        // dZ1^T = ((dZ2 W2) (1 - H1^2))^T
        memset(&g, 0, sizeof g);
        g.err = err;
        g.M = (int)q.M;
        g.A = q.dZ2; g.lda = q.H2; g.B = q.W2T; g.ldb = q.H2; g.N = q.H1; g.K = q.H2;
        g.epi = EPI_TANH_BWD; g.aux = q.H1a; g.ld_aux = q.H1; g.CT = q.dZ1T; g.ldct = q.ldM;
        st[4].push_back(g);
        // weight gradients (K = |S|): dW3 = dPhi^T H2, dW2 = dZ2^T H1, dW1 = dZ1^T X
        float* gW1 = q.grad;
        float* gW2 = gW1 + (size_t)q.H1 * q.nin + q.H1;
        float* gW3 = gW2 + (size_t)q.H2 * q.H1 + q.H2;
        auto wg = [&](const __nv_bfloat16* At, int rows, const __nv_bfloat16* Bt, int cols,
                      float* o) {
            TcGemm w;
            memset(&w, 0, sizeof w);
            w.err = err;
            w.A = At; w.lda = q.ldM; w.B = Bt; w.ldb = q.ldM; w.M = rows; w.N = cols;
            w.K = (int)q.M; w.epi = EPI_STORE; w.C = o; w.ldc = cols;
            st[5].push_back(w);
        };
        wg(q.dPhiT, q.nout, q.H2T, q.H2, gW3);
        wg(q.dZ2T, q.H2, q.H1T, q.H1, gW2);
        wg(q.dZ1T, q.H1, q.XT, q.nin, gW1);
    }
    for (int k = 0; k < 6; ++k) {
        if (st[k].empty()) continue;
        const int r = build_set(st[k], s, &G->sets[k], &G->bn[k]);
        if (r < 0) return fail(r);
    }
    b->g = G;
    return NQS_OK;
}

static int grouped_run(nqs_batch* b, cudaStream_t s) {
    GroupedState* G = b->g;
    const GDims& d = G->dims;
    NQS_TRY(g_bits_prep(G->dP, d, s));
    for (int k = 0; k < 3; ++k) NQS_TRY(tc_group_set_launch(G->sets[k], s));
    for (size_t t = 0; t < G->lu_n.size(); ++t)
        NQS_TRY(g_lu(G->lu_jobs[t], G->lu_count[t], G->lu_n[t], d.maxM, s));
    NQS_TRY(g_combine(G->dP, d, s));
    NQS_TRY(g_energy(G->dP, d, G->kpart, s));
    if (!G->with_grad) return NQS_OK;
    NQS_TRY(g_adjoint(G->dP, d, s));
    NQS_TRY(g_transpose_dphi(G->dP, d, G->tile_off, G->tiles, s));
    for (int k = 3; k < 6; ++k) NQS_TRY(tc_group_set_launch(G->sets[k], s));
    NQS_TRY(g_bias_grads(G->dP, d, s));
    return NQS_OK;
}

// fork to the side streams, one energy/gradient pipeline per problem, join back; or the
// grouped pipeline
extern "C" int nqs_batch_run(nqs_batch* b, nqs_stream_t stream) {
    if (!b) return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (b->mode == NQS_BATCH_GROUPED) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        NQS_CK(cudaStreamIsCapturing(s, &cap));
        if (!b->g && cap != cudaStreamCaptureStatusNone) return NQS_ERR_ARG;  // prepare first
        NQS_TRY(grouped_prepare(b, s));
        return grouped_run(b, s);
    }
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
    if (b->mode == NQS_BATCH_GROUPED) NQS_TRY(grouped_prepare(b, s));  // outside the capture
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

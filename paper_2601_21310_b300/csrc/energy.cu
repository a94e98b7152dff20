// E_S and its gradient (Eqs. variational_energy, variational_gradient; Algorithm 1 step 2),
// the device SpMV v = H_SS psi (the paper's host-resident SciPy SpMV, moved on-device), the
// amplitude entry point and the network handle.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ansatz.cuh"
#include "excite.cuh"
#include "ksum.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

// y = H x, one warp per row, FP64. Lanes stride the row with four independent partial sums
// (the loads of four strides in flight per lane: the gathers x[col] are dependent loads), which
// are added in a fixed order and then reduced by a shuffle tree: the result is deterministic.
// OFFDIAG skips each row's first entry (the diagonal, first in every row of H_SS).
template <bool OFFDIAG>
__device__ __forceinline__ void spmv_rows(const int64_t* __restrict__ rp,
                                          const int32_t* __restrict__ col,
                                          const double* __restrict__ val,
                                          const double* __restrict__ x, int64_t n,
                                          double* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t k1 = rp[r + 1];
        int64_t k = rp[r] + (OFFDIAG ? 1 : 0) + lane;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (; k + 96 < k1; k += 128) {
            const int32_t c0 = __ldg(col + k), c1 = __ldg(col + k + 32), c2 = __ldg(col + k + 64),
                          c3 = __ldg(col + k + 96);
            const double v0 = __ldg(val + k), v1 = __ldg(val + k + 32), v2 = __ldg(val + k + 64),
                         v3 = __ldg(val + k + 96);
            s0 = fma(v0, __ldg(x + c0), s0);
            s1 = fma(v1, __ldg(x + c1), s1);
            s2 = fma(v2, __ldg(x + c2), s2);
            s3 = fma(v3, __ldg(x + c3), s3);
        }
        for (; k < k1; k += 32) s0 = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s0);
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
        if (lane == 0) y[r] = s;
    }
}

template <bool OFFDIAG>
__global__ void __launch_bounds__(256) k_spmv(const int64_t* __restrict__ rp,
                                              const int32_t* __restrict__ col,
                                              const double* __restrict__ val,
                                              const double* __restrict__ x, int64_t n,
                                              double* __restrict__ y) {
    spmv_rows<OFFDIAG>(rp, col, val, x, n, y);
}

// psi~ = sign * exp(log|psi| - max log|psi|)
__global__ void k_scaled_psi(const double* __restrict__ logabs, const int8_t* __restrict__ sign,
                             const double* __restrict__ maxlog, int64_t n,
                             double* __restrict__ psi) {
    const double M = *maxlog;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        psi[i] = sign[i] == 0 ? 0.0 : (double)sign[i] * exp(logabs[i] - M);
}

__global__ void k_energy(double* out) { out[0] = out[1] / out[2]; }

// w_x = (2/D) (v_x - E psi~_x) psi~_x
__global__ void k_adjoint_weight(const double* __restrict__ v, const double* __restrict__ psi,
                                 const double* __restrict__ ev, int64_t n, double* __restrict__ w) {
    const double E = ev[0], D = ev[2];
    const double c = __ddiv_rn(2.0, D);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        w[i] = __dmul_rn(__dmul_rn(c, __dsub_rn(v[i], __dmul_rn(E, psi[i]))), psi[i]);
}

// Asymmetric mode on the proxy CSR over T = V + P: per row, the sum over every entry (H_VT psi
// for rows of V; H_PV psi_V for rows of P, whose leading diagonal is skipped) and the sum over
// the columns inside V. One warp per row, lanes stride the row, then a shuffle tree.
__global__ void k_asym_spmv(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const double* __restrict__ x,
                            int64_t n, int64_t nV, double* __restrict__ v_all,
                            double* __restrict__ v_in) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        double sa = 0.0, si = 0.0;
        const int64_t k0 = rp[r] + (r >= nV ? 1 : 0);
        for (int64_t k = k0 + lane; k < rp[r + 1]; k += 32) {
            const double t = __dmul_rn(val[k], x[col[k]]);
            sa = __dadd_rn(sa, t);
            if (col[k] < nV) si = __dadd_rn(si, t);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(FULL_MASK, sa, o);
            si += __shfl_xor_sync(FULL_MASK, si, o);
        }
        if (lane == 0) {
            v_all[r] = sa;
            v_in[r] = si;
        }
    }
}

// w_z = c_z psi~_z with the coefficients of the estimator (exact = 0) or of the exact gradient
__global__ void k_asym_weight(const double* __restrict__ v_all, const double* __restrict__ v_in,
                              const double* __restrict__ psi, const double* __restrict__ ev,
                              int64_t n, int64_t nV, int exact, double* __restrict__ w) {
    const double E = ev[0], D = ev[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double c;
        if (i < nV)
            c = exact ? __ddiv_rn(__dsub_rn(__dadd_rn(v_all[i], v_in[i]),
                                            __dmul_rn(__dmul_rn(2.0, E), psi[i])),
                                  D)
                      : __ddiv_rn(__dmul_rn(2.0, __dsub_rn(v_all[i], __dmul_rn(E, psi[i]))), D);
        else
            c = exact ? __ddiv_rn(v_all[i], D) : 0.0;
        w[i] = __dmul_rn(c, psi[i]);
    }
}

int csr_spmv(const nqs_csr* csr, const double* x, double* y, cudaStream_t s) {
    int64_t n = csr->n_rows;
    {
        ProfScope prof_(PROF_SPMV, s);
        k_spmv<false><<<grid_for(n * 32, 256, 148 * 64), 256, 0, s>>>(csr->row_ptr, csr->col,
                                                                      csr->val, x, n, y);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int csr_spmv_offdiag(const nqs_csr* csr, const double* x, double* y, cudaStream_t s) {
    int64_t n = csr->n_rows;
    {
        ProfScope prof_(PROF_SPMV, s);
        k_spmv<true><<<grid_for(n * 32, 256, 148 * 64), 256, 0, s>>>(csr->row_ptr, csr->col,
                                                                     csr->val, x, n, y);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

extern "C" int nqs_energy_from_psi(const nqs_csr* csr, const double* psi, int64_t nS, double* out,
                                   double* v, nqs_stream_t stream) {
    if (!csr || !psi || !out || nS <= 0 || csr->n_rows != nS) return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // no problem handle here: scratch comes from the device's default stream-ordered pool
    nqs_problem host;
    memset(&host, 0, sizeof host);
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    NQS_CK(cudaDeviceGetDefaultMemPool(&host.pool, dev));
    Scratch sc(&host, s);
    double* vv = v;
    if (!vv) NQS_TRY(sc.get(&vv, nS));
    NQS_TRY(csr_spmv(csr, psi, vv, s));
    NQS_TRY(kdot2_f64(&host, sc, vv, psi, nS, out + 1, s));
    k_energy<<<1, 1, 0, s>>>(out);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// network handle
// ------------------------------------------------------------------------------------------
extern "C" int nqs_net_create(nqs_problem* p, int H1, int H2, int dtype,
                              const void* const* params, nqs_net** out) {
    if (!p || !params || !out || H1 <= 0 || H2 <= 0) return NQS_ERR_ARG;
    if (dtype != NQS_FP64 && dtype != NQS_MIXED) return NQS_ERR_ARG;
    for (int i = 0; i < 7; ++i)
        if (!params[i]) return NQS_ERR_ARG;
    nqs_net* n = (nqs_net*)calloc(1, sizeof(nqs_net));
    if (!n) return NQS_ERR_OOM;
    n->prob = p;
    n->H1 = H1;
    n->H2 = H2;
    n->nin = 2 * p->d.norb;
    n->nout = p->d.norb * (p->d.na + p->d.nb);
    n->dtype = dtype;
    for (int i = 0; i < 7; ++i) n->p[i] = params[i];
    *out = n;
    return NQS_OK;
}

extern "C" int nqs_net_destroy(nqs_net* n) {
    free(n);
    return NQS_OK;
}

extern "C" int64_t nqs_net_num_params(const nqs_net* n) {
    if (!n) return 0;
    return (int64_t)n->H1 * n->nin + n->H1 + (int64_t)n->H2 * n->H1 + n->H2 +
           (int64_t)n->nout * n->H2 + n->nout;
}

static int check_common(nqs_problem* p, nqs_net* net, const uint64_t* dets, int64_t nS,
                        const nqs_opts* opts) {
    if (!p || !net || !dets || nS <= 0 || net->prob != p) return NQS_ERR_ARG;
    if (((uintptr_t)dets) & 15) return NQS_ERR_ARG;
    if (nS >= ((int64_t)1 << 31)) return NQS_ERR_UNSUPPORTED;
    if (opts && opts->precision != net->dtype) return NQS_ERR_ARG;
    return NQS_OK;
}

__global__ void k_add_f32(float* __restrict__ a, const float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}
__global__ void k_add_f64(double* __restrict__ a, const double* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

// micro-batch size of the amplitude and energy paths: 2^opts->batch_log2 (0: 2^20)
static int64_t micro_batch(const nqs_opts* opts) {
    const int lg = (opts && opts->batch_log2 > 0 && opts->batch_log2 < 31) ? opts->batch_log2 : 20;
    return (int64_t)1 << lg;
}

// Forward over n configurations. One micro-batch: activations are kept in f for the backward
// (when keep). More: amplitudes only, batch by batch (the backward recomputes them).
static int forward_batched(nqs_net* net, Scratch& sc, const uint64_t* dets, int64_t n,
                           int64_t mb, bool keep, Fwd& f, double* logabs, int8_t* sign,
                           cudaStream_t s) {
    if (n <= mb) return net_forward(net, sc, dets, n, f, keep, logabs, sign, s);
    for (int64_t c0 = 0; c0 < n; c0 += mb) {
        const int64_t m = n - c0 < mb ? n - c0 : mb;
        Scratch bs(net->prob, s);
        Fwd fb;
        NQS_TRY(net_forward(net, bs, dets + 2 * c0, m, fb, false, logabs + c0, sign + c0, s));
    }
    return NQS_OK;
}

// grad = sum over the n configurations of w_x d log|psi_x| / d theta (weights as in
// net_backward). One micro-batch: from the activations in f. More: per batch, the forward is
// recomputed with activations kept, the batch's gradient formed and added (Sec. 3.2:
// gradients accumulated over fixed-size micro-batches, so memory is bounded by the batch).
static int backward_batched(nqs_net* net, Scratch& sc, const uint64_t* dets, int64_t n,
                            int64_t mb, const Fwd& f, const double* w, void* grad,
                            cudaStream_t s) {
    if (n <= mb) return net_backward(net, sc, dets, f, w, grad, s);
    const int64_t np = nqs_net_num_params(net);
    const bool mixed = net->dtype == NQS_MIXED;
    void* part = nullptr;
    if (mixed) NQS_TRY(sc.get((float**)&part, np));
    else NQS_TRY(sc.get((double**)&part, np));
    double* la;
    int8_t* sg;
    NQS_TRY(sc.get(&la, mb));
    NQS_TRY(sc.get(&sg, mb));
    for (int64_t c0 = 0; c0 < n; c0 += mb) {
        const int64_t m = n - c0 < mb ? n - c0 : mb;
        Scratch bs(net->prob, s);
        Fwd fb;
        NQS_TRY(net_forward(net, bs, dets + 2 * c0, m, fb, true, la, sg, s));
        NQS_TRY(net_backward(net, bs, dets + 2 * c0, fb, w + c0, c0 == 0 ? grad : part, s));
        if (c0 > 0) {
            if (mixed) k_add_f32<<<grid_for(np, 256), 256, 0, s>>>((float*)grad, (const float*)part, np);
            else k_add_f64<<<grid_for(np, 256), 256, 0, s>>>((double*)grad, (const double*)part, np);
            NQS_CK_LAUNCH();
        }
    }
    return NQS_OK;
}


extern "C" int nqs_amplitudes(nqs_problem* p, nqs_net* net, const uint64_t* dets, int64_t nS,
                              double* logabs, int8_t* sign, const nqs_opts* opts,
                              nqs_stream_t stream) {
    NQS_TRY(check_common(p, net, dets, nS, opts));
    if (!logabs || !sign) return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (opts && opts->validate) {
        Scratch sv(p, s);
        NQS_TRY(validate_dets(p, sv, dets, nS, false, s));
    }
    // micro-batches bound the activation memory for large target sets (Sec. 3.3); each
    // configuration's amplitude is independent of the others, so the batching is invisible
    int sing_any = 0;
    const int64_t mb = micro_batch(opts);
    for (int64_t c0 = 0; c0 < nS; c0 += mb) {
        const int64_t m = nS - c0 < mb ? nS - c0 : mb;
        Scratch sc(p, s);
        Fwd f;
        NQS_TRY(net_forward(net, sc, dets + 2 * c0, m, f, false, logabs + c0, sign + c0, s));
        int sing = 0;
        NQS_CK(cudaMemcpyAsync(&sing, f.singular, sizeof sing, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        sing_any |= sing;
    }
    NQS_TRY(check_err_word(p, s));
    return sing_any ? NQS_WARN_SINGULAR : NQS_OK;
}

extern "C" int nqs_energy_grad(nqs_problem* p, nqs_net* net, const nqs_csr* csr,
                               const uint64_t* dets, int64_t nS, double* out, void* grad,
                               double* psi_out, const nqs_opts* opts, nqs_stream_t stream) {
    NQS_TRY(check_common(p, net, dets, nS, opts));
    if (!csr || !out || csr->n_rows != nS) return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(p, s);
    if (opts && opts->validate) NQS_TRY(validate_dets(p, sc, dets, nS, true, s));
    double *logabs, *psi, *v;
    int8_t* sign;
    NQS_TRY(sc.get(&logabs, nS));
    NQS_TRY(sc.get(&sign, nS));
    NQS_TRY(sc.get(&v, nS));
    psi = psi_out;
    if (!psi) NQS_TRY(sc.get(&psi, nS));
    Fwd f;
    const int64_t mb = micro_batch(opts);
    NQS_TRY(forward_batched(net, sc, dets, nS, mb, grad != nullptr, f, logabs, sign, s));
    NQS_TRY(max_f64_masked(p, sc, logabs, sign, nS, out + 3, s));
    k_scaled_psi<<<grid_for(nS, 256), 256, 0, s>>>(logabs, sign, out + 3, nS, psi);
    NQS_CK_LAUNCH();
    NQS_TRY(csr_spmv(csr, psi, v, s));
    NQS_TRY(kdot2_f64(p, sc, v, psi, nS, out + 1, s));
    k_energy<<<1, 1, 0, s>>>(out);
    NQS_CK_LAUNCH();
    if (grad) {
        double* w;
        NQS_TRY(sc.get(&w, nS));
        k_adjoint_weight<<<grid_for(nS, 256), 256, 0, s>>>(v, psi, out, nS, w);
        NQS_CK_LAUNCH();
        NQS_TRY(backward_batched(net, sc, dets, nS, mb, f, w, grad, s));
    }
    // with validation on, synchronise and report a timed-out tensor-core wait
    if (opts && opts->validate) NQS_TRY(check_err_word(p, s));
    return NQS_OK;
}

// Asymmetric mode (Sec. 2.4.1, Eqs. asymmetric_energy, asymmetric_gradient) on T = V + P with
// the proxy CSR over T: E_asym = sum_V psi (H_VT psi) / sum_V psi^2, and the gradient as the
// log-derivative estimator (exact = 0) or the derivative of E_asym (exact = 1).
extern "C" int nqs_asym_energy_grad(nqs_problem* p, nqs_net* net, const nqs_csr* csr,
                                    const uint64_t* T, int64_t nT, int64_t nV, int exact,
                                    double* out, void* grad, double* psi_out,
                                    const nqs_opts* opts, nqs_stream_t stream) {
    NQS_TRY(check_common(p, net, T, nT, opts));
    if (!csr || !out || csr->n_rows != nT || nV <= 0 || nV > nT) return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(p, s);
    double *logabs, *psi, *v_all, *v_in;
    int8_t* sign;
    NQS_TRY(sc.get(&logabs, nT));
    NQS_TRY(sc.get(&sign, nT));
    NQS_TRY(sc.get(&v_all, nT));
    NQS_TRY(sc.get(&v_in, nT));
    psi = psi_out;
    if (!psi) NQS_TRY(sc.get(&psi, nT));
    Fwd f;
    const int64_t mb = micro_batch(opts);
    NQS_TRY(forward_batched(net, sc, T, nT, mb, grad != nullptr, f, logabs, sign, s));
    NQS_TRY(max_f64_masked(p, sc, logabs, sign, nT, out + 3, s));
    k_scaled_psi<<<grid_for(nT, 256), 256, 0, s>>>(logabs, sign, out + 3, nT, psi);
    NQS_CK_LAUNCH();
    {
        ProfScope prof_(PROF_SPMV, s);
        k_asym_spmv<<<grid_for(nT * 32, 256, 148 * 64), 256, 0, s>>>(
            csr->row_ptr, csr->col, csr->val, psi, nT, nV, v_all, v_in);
    }
    NQS_CK_LAUNCH();
    NQS_TRY(kdot2_f64(p, sc, v_all, psi, nV, out + 1, s));  // N and D over V
    k_energy<<<1, 1, 0, s>>>(out);
    NQS_CK_LAUNCH();
    if (grad) {
        double* w;
        NQS_TRY(sc.get(&w, nT));
        k_asym_weight<<<grid_for(nT, 256), 256, 0, s>>>(v_all, v_in, psi, out, nT, nV,
                                                        exact ? 1 : 0, w);
        NQS_CK_LAUNCH();
        NQS_TRY(backward_batched(net, sc, T, nT, mb, f, w, grad, s));
    }
    if (opts && opts->validate) NQS_TRY(check_err_word(p, s));
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// Batched problems: the energy stage over all problems, one launch per step (blockIdx.y =
// problem), with the arithmetic of the single-problem path: max log|psi| (over psi != 0),
// psi~ = sign exp(log|psi| - max), v = H_SS psi~ (spmv_rows), N = psi~.v and D = psi~.psi~ as
// in kdot2_f64 (KR_BLOCKS partial sums per problem, then one block), E = N / D and the adjoint
// weights w = (2/D)(v - E psi~) psi~.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_g_maxlog(const GProb* __restrict__ Pv) {
    const GProb& P = Pv[blockIdx.y];
    __shared__ double sm[256];
    double m = -INFINITY;
    for (int64_t i = threadIdx.x; i < P.M; i += 256)
        if (P.sign[i] != 0) m = fmax(m, P.logabs[i]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) P.out[3] = sm[0];
}

__global__ void k_g_scaled_psi(const GProb* __restrict__ Pv) {
    const GProb& P = Pv[blockIdx.y];
    const double M = P.out[3];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.M;
         i += (int64_t)gridDim.x * blockDim.x)
        P.psi[i] = P.sign[i] == 0 ? 0.0 : (double)P.sign[i] * exp(P.logabs[i] - M);
}

__global__ void __launch_bounds__(256) k_g_spmv(const GProb* __restrict__ Pv) {
    const GProb& P = Pv[blockIdx.y];
    spmv_rows<false>(P.rp, P.col, P.val, P.psi, P.M, P.v);
}

// blockIdx.z = 0: partial sums of v psi~, 1: of psi~ psi~ (KR_BLOCKS blocks per problem)
__global__ void __launch_bounds__(KR_THREADS) k_g_dot(const GProb* __restrict__ Pv,
                                                       double2* __restrict__ part) {
    const GProb& P = Pv[blockIdx.y];
    const int mode = blockIdx.z;
    KS k{0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * KR_THREADS + threadIdx.x; i < P.M;
         i += (int64_t)KR_BLOCKS * KR_THREADS) {
        const double v = mode == 0 ? __dmul_rn(P.v[i], P.psi[i]) : __dmul_rn(P.psi[i], P.psi[i]);
        k = ks_add(k, v);
    }
    KS r = block_ks(k);
    if (threadIdx.x == 0)
        part[((int64_t)blockIdx.y * 2 + mode) * KR_BLOCKS + blockIdx.x] = make_double2(r.s, r.c);
}

// one block per (problem, mode): N, D; then E = N / D (one thread)
__global__ void __launch_bounds__(KR_THREADS) k_g_dot_final(const GProb* __restrict__ Pv,
                                                             const double2* __restrict__ part) {
    const GProb& P = Pv[blockIdx.x];
    const int mode = blockIdx.y;
    const double2* pp = part + ((int64_t)blockIdx.x * 2 + mode) * KR_BLOCKS;
    KS k{0.0, 0.0};
    for (int i = threadIdx.x; i < KR_BLOCKS; i += KR_THREADS) k = ks_merge(k, KS{pp[i].x, pp[i].y});
    KS r = block_ks(k);
    if (threadIdx.x == 0) P.out[1 + mode] = r.s + r.c;
}

__global__ void k_g_weights(const GProb* __restrict__ Pv) {
    const GProb& P = Pv[blockIdx.y];
    const double N = P.out[1], D = P.out[2];
    const double E = N / D;
    if (blockIdx.x == 0 && threadIdx.x == 0) P.out[0] = E;
    if (!P.grad) return;
    const double c = __ddiv_rn(2.0, D);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.M;
         i += (int64_t)gridDim.x * blockDim.x)
        P.w[i] = __dmul_rn(__dmul_rn(c, __dsub_rn(P.v[i], __dmul_rn(E, P.psi[i]))), P.psi[i]);
}

int g_energy(const GProb* P, const GDims& d, double2* part, cudaStream_t s) {
    k_g_maxlog<<<dim3(1, d.np), 256, 0, s>>>(P);
    NQS_CK_LAUNCH();
    k_g_scaled_psi<<<dim3(grid_for(d.maxM, 256, 256), d.np), 256, 0, s>>>(P);
    NQS_CK_LAUNCH();
    {
        ProfScope prof_(PROF_SPMV, s);
        k_g_spmv<<<dim3(grid_for(d.maxM * 32, 256, 1024), d.np), 256, 0, s>>>(P);
    }
    NQS_CK_LAUNCH();
    k_g_dot<<<dim3(KR_BLOCKS, d.np, 2), KR_THREADS, 0, s>>>(P, part);
    NQS_CK_LAUNCH();
    k_g_dot_final<<<dim3(d.np, 2), KR_THREADS, 0, s>>>(P, part);
    NQS_CK_LAUNCH();
    k_g_weights<<<dim3(grid_for(d.maxM, 256, 256), d.np), 256, 0, s>>>(P);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

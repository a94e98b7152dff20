// Post-hoc diagonalisation diagnostic E_diag = lambda_min(H_VV) (Sec. 3.5, the subspace
// diagonalisation of the Supporting Information): Lanczos on the CSR of H_VV with full
// reorthogonalisation (classical Gram-Schmidt, applied twice per step) on the device, and the
// lowest eigenvalue of the Lanczos tridiagonal matrix by Sturm-sequence bisection on the host.
//
// Per step: w = H q_j (the library's warp-per-row SpMV); alpha_j = q_j . w; w -= Q^T (Q w) twice over all
// basis vectors so far (the first pass also removes alpha_j q_j and beta_{j-1} q_{j-1});
// beta_j = |w|; q_{j+1} = w / beta_j. Dot products use the library's fixed-order compensated
// reductions, so a run is deterministic. The basis is kept: iters x n FP64.
#include <math.h>
#include <string.h>

#include <vector>

#include "excite.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

// h[i] = Q[i] . w for i < m: one CTA per basis vector, fixed-order block reduction
__global__ void __launch_bounds__(256) k_lz_proj(const double* __restrict__ Q, int64_t n, int m,
                                                 const double* __restrict__ w,
                                                 double* __restrict__ h) {
    __shared__ double part[8];
    const double* q = Q + (size_t)blockIdx.x * n;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(q[i], w[i], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += part[k];
        h[blockIdx.x] = t;
    }
    (void)m;
}

// w[i] -= sum_k h[k] Q[k][i]
__global__ void k_lz_sub(const double* __restrict__ Q, int64_t n, int m,
                         const double* __restrict__ h, double* __restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int k = 0; k < m; ++k) s = fma(-h[k], Q[(size_t)k * n + i], s);
        w[i] = s;
    }
}

__global__ void k_lz_scale(const double* __restrict__ w, int64_t n, const double* __restrict__ nrm2,
                           double* __restrict__ q) {
    const double inv = 1.0 / sqrt(nrm2[0]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        q[i] = w[i] * inv;
}

// the default start vector: deterministic values in [0.5, 1.5) from a SplitMix64 of the index
__global__ void k_lz_start(int64_t n, double* __restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        w[i] = 0.5 + (double)(mix64((uint64_t)i + 0x9e3779b97f4a7c15ull) >> 11) * 0x1.0p-53;
}

// number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm sequence)
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int cnt = 0;
    double d = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        const double off = i == 0 ? 0.0 : b[i - 1] * b[i - 1];
        d = (a[i] - x) - (i == 0 ? 0.0 : off / d);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// lowest eigenvalue of the tridiagonal by bisection inside the Gershgorin interval
static double tridiag_min(const std::vector<double>& a, const std::vector<double>& b) {
    double lo = INFINITY, hi = -INFINITY;
    for (size_t i = 0; i < a.size(); ++i) {
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(1.0, fabs(lo)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, mid) >= 1) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

extern "C" int nqs_lanczos_min(const nqs_csr* csr, int max_iters, double tol, const double* start,
                               double* eigval, int* iters_done, nqs_stream_t stream) {
    if (!csr || !eigval || max_iters < 1 || csr->n_rows <= 0 || !(tol >= 0.0)) return NQS_ERR_ARG;
    const int64_t n = csr->n_rows;
    const int m_max = (int)(max_iters < n ? max_iters : n);
    cudaStream_t s = (cudaStream_t)stream;
    nqs_problem host;
    memset(&host, 0, sizeof host);
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    NQS_CK(cudaDeviceGetDefaultMemPool(&host.pool, dev));
    Scratch sc(&host, s);
    double *Q, *w, *h, *dots;
    NQS_TRY(sc.get(&Q, (size_t)(m_max + 1) * n));
    NQS_TRY(sc.get(&w, n));
    NQS_TRY(sc.get(&h, m_max + 1));
    NQS_TRY(sc.get(&dots, 2));
    const unsigned g = grid_for(n, 256);
    if (start) NQS_CK(cudaMemcpyAsync(w, start, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else {
        k_lz_start<<<g, 256, 0, s>>>(n, w);
        NQS_CK_LAUNCH();
    }
    NQS_TRY(kdot2_f64(&host, sc, w, w, n, dots, s));
    k_lz_scale<<<g, 256, 0, s>>>(w, n, dots + 1, Q);
    NQS_CK_LAUNCH();
    std::vector<double> a, b;
    double prev = INFINITY, lam = 0.0;
    int m = 0;
    for (m = 0; m < m_max; ++m) {
        double* q = Q + (size_t)m * n;
        NQS_TRY(csr_spmv(csr, q, w, s));
        Scratch st(&host, s);  // per-step reduction scratch
        NQS_TRY(kdot2_f64(&host, st, q, w, n, dots, s));  // dots[0] = alpha_m
        double hd[2];
        NQS_CK(cudaMemcpyAsync(hd, dots, sizeof hd, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        a.push_back(hd[0]);
        for (int pass = 0; pass < 2; ++pass) {  // w -= Q Q^T w over q_0..q_m
            k_lz_proj<<<m + 1, 256, 0, s>>>(Q, n, m + 1, w, h);
            NQS_CK_LAUNCH();
            k_lz_sub<<<g, 256, 0, s>>>(Q, n, m + 1, h, w);
            NQS_CK_LAUNCH();
        }
        NQS_TRY(kdot2_f64(&host, st, w, w, n, dots, s));
        NQS_CK(cudaMemcpyAsync(hd, dots, sizeof hd, cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
        const double beta = sqrt(hd[1]);
        lam = tridiag_min(a, b);
        const bool converged = fabs(lam - prev) <= tol * fmax(1.0, fabs(lam));
        prev = lam;
        if (converged || beta <= 1e-14 * fmax(1.0, fabs(lam)) || m + 1 == m_max) {
            ++m;
            break;
        }
        b.push_back(beta);
        k_lz_scale<<<g, 256, 0, s>>>(w, n, dots + 1, Q + (size_t)(m + 1) * n);
        NQS_CK_LAUNCH();
    }
    *eigval = lam;
    if (iters_done) *iters_done = m;
    return NQS_OK;
}

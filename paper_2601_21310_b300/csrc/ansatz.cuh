// Backflow network and determinant kernels (shared declarations between ansatz.cu,
// gemm_tc.cu and energy.cu).
#pragma once
#include "nqs_internal.cuh"

// epilogues of the dense layers
enum { EPI_STORE = 0, EPI_BIAS_TANH = 1, EPI_BIAS_PHI0 = 2, EPI_TANH_BWD = 3 };

struct GemmArgs {
    int M, N, K;
    const void* A;
    int64_t a_m, a_k;  // A(m, k) = A[m * a_m + k * a_k]
    const void* B;
    int64_t b_n, b_k;  // B(n, k) = B[n * b_n + k * b_k]
    void* C;
    int64_t ldc;       // C[m * ldc + n]
    int epi;
    const void* bias;  // [N] (accumulator type)
    const void* aux;   // EPI_BIAS_PHI0: Phi0 [N] (accumulator type); EPI_TANH_BWD: h [M][ld_aux]
    int64_t ld_aux;
};

// dtype-dispatched dense layer: C = epi(A B^T). FP64 form: all double. Mixed form: A, B bf16,
// FP32 accumulation, bias/Phi0 float, output bf16 (activations) or float (Phi, gradients).
int gemm_f64(const GemmArgs& g, cudaStream_t s);
int gemm_bf16_simt(const GemmArgs& g, bool out_bf16, cudaStream_t s);

// tcgen05 path (gemm_tc.cu): C[m][n] = epi(sum_k A[m][k] B[n][k]), A [M][lda] and B [N][ldb]
// bfloat16 with k contiguous (lda, ldb multiples of 8); with a_mn (b_mn) set, A (B) is stored
// with m (n) contiguous instead, A[m][k] at A[k * lda + m] (the row-major activations of a
// weight gradient, read without a transposed copy). Optional row-major C (bf16 or float) and
// transposed bf16 copy CT[n][m]. EPI_STORE with float C may split K across CTAs.
struct TcGemm {
    const __nv_bfloat16* A;
    int64_t lda;
    const __nv_bfloat16* B;
    int64_t ldb;
    int M, N, K;
    int epi;
    void* C;
    int64_t ldc;
    int c_bf16;
    __nv_bfloat16* CT;
    int64_t ldct;
    const float* bias;
    const float* phi0;
    const __nv_bfloat16* aux;
    int64_t ld_aux;
    int* err;
    int a_mn, b_mn;
};
int gemm_bf16_tcgen05(const TcGemm& g, Scratch& sc, cudaStream_t s);

// Grouped form for many independent GEMMs of different shapes (one per batched problem): the
// descriptors (tensor maps, epilogue arguments, split-K partial buffers) are built once for
// fixed operand addresses; each launch runs every group's tiles in one persistent kernel with
// tile width BN (64, 128 or 256), then one grouped split-K reduction.
struct TcGroupSet;
int tc_group_set_create(const TcGemm* gs, int n, int BN, TcGroupSet** out);
int tc_group_set_launch(const TcGroupSet* set, cudaStream_t s);
int tc_group_set_units(const TcGroupSet* set);
void tc_group_set_destroy(TcGroupSet* set);
int tc_autotune_on();  // nqs_set_autotune state

// forward intermediates kept for the backward
struct Fwd {
    int64_t M;
    void* X;        // [M][nin] 0/1 (input type), only for the weight gradient of layer 1
    void* H1;       // [M][H1]
    void* H2;       // [M][H2]
    void* Phi;      // [M][nout] (double or float)
    void* Ainv_a;   // [M][na][na] (double or float), inverse of the alpha occupied block
    void* Ainv_b;   // [M][nb][nb]
    double* logabs; // [M]
    int8_t* sign;   // [M]
    int* singular;  // device flag
    // mixed form on tensor cores: X is [M][ldX] bf16 (nin padded to 8 with zero columns);
    // the weight gradients read X, H1 and H2 row-major as MN-major GEMM operands
    bool tc;
    int64_t ldX;
    int* err;       // tensor-core pipeline error word
};

int net_forward(nqs_net* net, Scratch& sc, const uint64_t* dets, int64_t M, Fwd& f,
                bool keep_for_backward, double* logabs, int8_t* sign, cudaStream_t s);
// w: device [M] adjoint weights w_x = dE/dpsi~_x * psi~_x; grad: device (double or float)
int net_backward(nqs_net* net, Scratch& sc, const uint64_t* dets, const Fwd& f, const double* w,
                 void* grad, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Batched problems, one launch per pipeline stage over all of them (batch.cu drives these).
// One descriptor per problem in device memory; a grouped kernel takes the problem from
// blockIdx.y (blockIdx.z for per-problem job lists) and strides over that problem's rows.
// Mixed form only (BF16 network on the tensor cores, FP32 LU up to 12 x 12 blocks).
// ------------------------------------------------------------------------------------------
struct GProb {
    const ulonglong2* dets;
    int64_t M;                 // |S|
    int norb, na, nb, nin, nout, H1, H2, ldX;
    int64_t ldM, ldP;          // M and nout rounded up to 8
    const __nv_bfloat16 *W1, *W2, *W3;           // caller's weights
    const float *b1, *b2, *b3, *phi0;             // caller's biases and Phi0
    const int64_t* rp;         // H_SS of the problem (library CSR)
    const int32_t* col;
    const double* val;
    double* out;               // caller's [4] = {E, N, D, max log|psi|}
    float* grad;               // caller's gradient (W1, b1, W2, b2, W3, b3) or null
    // workspace
    __nv_bfloat16 *X, *XT, *W1p, *H1a, *H1T, *H2a, *H2T, *W2T, *W3T, *dPhi, *dPhiT, *dZ2, *dZ2T,
        *dZ1T;
    float *Phi, *Ainv_a, *Ainv_b;
    double *la2, *logabs, *psi, *v, *w;
    int* ex2;
    int8_t *sg2, *sign;
    int* singular;
};

// register-LU job of one spin block of one problem (problems grouped by block size n)
struct GLuJob {
    const ulonglong2* dets;
    int64_t M;
    int norb, nel, spin;
    const float* Phi;
    double* la;
    int* ex;
    int8_t* sg;
    float* Ainv;
    int* singular;
};

// launch extents over the problems: the largest of each size
struct GDims {
    int np;
    int64_t maxM, maxMX;  // rows; rows x (ldX / 8)
    int max_nin, max_nout, max_H;
};

int g_bits_prep(const GProb* P, const GDims& d, cudaStream_t s);
int g_lu(const GLuJob* jobs, int njobs, int n, int64_t maxM, cudaStream_t s);
int g_combine(const GProb* P, const GDims& d, cudaStream_t s);
int g_adjoint(const GProb* P, const GDims& d, cudaStream_t s);
// tile_off: device [np + 1] prefix of each problem's 32 x 32 tiles of dPhi (tiles in all)
int g_transpose_dphi(const GProb* P, const GDims& d, const int64_t* tile_off, int64_t tiles,
                     cudaStream_t s);
int g_bias_grads(const GProb* P, const GDims& d, cudaStream_t s);
// energy.cu: max log|psi|, scaled psi, SpMV, compensated N and D (part: device
// [np][2][256] partial sums), E and the adjoint weights
int g_energy(const GProb* P, const GDims& d, double2* part, cudaStream_t s);

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
// bfloat16 with k contiguous (lda, ldb multiples of 8). Optional row-major C (bf16 or float)
// and transposed bf16 copy CT[n][m]. EPI_STORE with float C may split K across CTAs.
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
};
int gemm_bf16_tcgen05(const TcGemm& g, Scratch& sc, cudaStream_t s);

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
    // mixed form on tensor cores: transposed copies ([H][ldM], ldM = M rounded up to 8)
    bool tc;
    int64_t ldM;
    void* H1T;
    void* H2T;
    void* XT;       // [nin][ldM]
    int* err;       // tensor-core pipeline error word
};

int net_forward(nqs_net* net, Scratch& sc, const uint64_t* dets, int64_t M, Fwd& f,
                bool keep_for_backward, double* logabs, int8_t* sign, cudaStream_t s);
// w: device [M] adjoint weights w_x = dE/dpsi~_x * psi~_x; grad: device (double or float)
int net_backward(nqs_net* net, Scratch& sc, const uint64_t* dets, const Fwd& f, const double* w,
                 void* grad, cudaStream_t s);

// Neural-backflow amplitude (Sec. 2.2; Eqs. effective_orbital_matrix, occupied_submatrix,
// backflow_amplitude) and its hand-written adjoint (Eq. variational_gradient via Jacobi's
// formula d det A / dA = det A * A^{-T}).
//
//   layer 1: z1 = W1 x + b1 over the 0/1 input -> a gather-sum of the occupied columns of W1
//   layer 2: z2 = W2 h1 + b2, h2 = tanh z2        (dense GEMM)
//   layer 3: Phi = Phi0 + (W3 h2 + b3)            (dense GEMM, epilogue adds b3 then Phi0)
//   psi = det Phi[occ_a, 0:na] * det Phi[occ_b, na:na+nb]: warp-per-block LU with partial
//   pivoting (FP64 form: double; mixed form: float) with log|det| summed in FP64, and the
//   block inverse kept for the adjoint.
#include <math.h>
#include <string.h>

#include "ansatz.cuh"
#include "excite.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

template <class T>
struct Cvt;
template <>
struct Cvt<double> {
    __device__ static double to_acc(double x) { return x; }
    __device__ static double from(double x) { return x; }
};
template <>
struct Cvt<float> {
    __device__ static float to_acc(float x) { return x; }
    __device__ static float from(float x) { return x; }
};
template <>
struct Cvt<__nv_bfloat16> {
    __device__ static float to_acc(__nv_bfloat16 x) { return __bfloat162float(x); }
    __device__ static __nv_bfloat16 from(float x) { return __float2bfloat16_rn(x); }
};

__device__ __forceinline__ double act_tanh(double z) { return tanh(z); }
__device__ __forceinline__ float act_tanh(float z) { return tanhf(z); }

// ------------------------------------------------------------------------------------------
// layer 1: gather-sum over occupied inputs (alpha bit p -> column p, beta bit p -> norb + p),
// summed in ascending column order, then + b1, tanh.
// ------------------------------------------------------------------------------------------
template <class TW, class TAcc, class TH>
__global__ void k_layer1(const ulonglong2* __restrict__ dets, int64_t M, int norb, int H1,
                         const TW* __restrict__ W1, const TAcc* __restrict__ b1,
                         TH* __restrict__ H, TH* __restrict__ X) {
    const int nin = 2 * norb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M * H1;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = t / H1;
        int i = (int)(t - m * H1);
        ulonglong2 x = dets[m];
        const TW* w = W1 + (int64_t)i * nin;
        TAcc z = TAcc(0);
        for (uint64_t v = x.x; v; v &= v - 1) z += Cvt<TW>::to_acc(w[__ffsll((long long)v) - 1]);
        for (uint64_t v = x.y; v; v &= v - 1)
            z += Cvt<TW>::to_acc(w[norb + __ffsll((long long)v) - 1]);
        z = z + b1[i];
        H[t] = Cvt<TH>::from(act_tanh(z));
        if (X && i < nin) {
            uint64_t word = i < norb ? x.x : x.y;
            int bit = i < norb ? i : i - norb;
            X[m * nin + i] = Cvt<TH>::from((TAcc)((word >> bit) & 1ull));
        }
    }
}

// X for layers narrower than the input (H1 < 2 norb): a separate fill
template <class TH, class TAcc>
__global__ void k_bits(const ulonglong2* __restrict__ dets, int64_t M, int norb, TH* X) {
    const int nin = 2 * norb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M * nin;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = t / nin;
        int i = (int)(t - m * nin);
        ulonglong2 x = dets[m];
        uint64_t word = i < norb ? x.x : x.y;
        int bit = i < norb ? i : i - norb;
        X[t] = Cvt<TH>::from((TAcc)((word >> bit) & 1ull));
    }
}

// ------------------------------------------------------------------------------------------
// generic SIMT GEMM C = epi(A B^T) with arbitrary element strides: the FP64 form, and the
// reference mixed path (BF16 inputs, FP32 accumulation). 64x64 tile, 16-deep k slices.
// ------------------------------------------------------------------------------------------
#define GB_M 64
#define GB_N 64
#define GB_K 16

template <class TIn, class TAcc, class TOut>
__global__ void __launch_bounds__(256) k_gemm_simt(GemmArgs g) {
    __shared__ TAcc As[GB_K][GB_M + 1];
    __shared__ TAcc Bs[GB_K][GB_N + 1];
    const TIn* A = (const TIn*)g.A;
    const TIn* B = (const TIn*)g.B;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * GB_M, n0 = (int64_t)blockIdx.x * GB_N;
    TAcc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = TAcc(0);
    const bool a_kfast = g.a_k == 1, b_kfast = g.b_k == 1;
    for (int k0 = 0; k0 < g.K; k0 += GB_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = tid + 256 * q;
            int r, kk;
            if (a_kfast) {
                r = e / GB_K;
                kk = e % GB_K;
            } else {
                kk = e / GB_M;
                r = e % GB_M;
            }
            int64_t gm = m0 + r;
            int gk = k0 + kk;
            As[kk][r] = (gm < g.M && gk < g.K) ? Cvt<TIn>::to_acc(A[gm * g.a_m + gk * g.a_k])
                                               : TAcc(0);
            if (b_kfast) {
                r = e / GB_K;
                kk = e % GB_K;
            } else {
                kk = e / GB_N;
                r = e % GB_N;
            }
            int64_t gn = n0 + r;
            gk = k0 + kk;
            Bs[kk][r] = (gn < g.N && gk < g.K) ? Cvt<TIn>::to_acc(B[gn * g.b_n + gk * g.b_k])
                                               : TAcc(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            TAcc a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
    TOut* C = (TOut*)g.C;
    const TAcc* bias = (const TAcc*)g.bias;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            TAcc v = acc[i][j];
            if (g.epi == EPI_BIAS_TANH) {
                TAcc z = v + bias[n];
                v = act_tanh(z);
            } else if (g.epi == EPI_BIAS_PHI0) {
                TAcc z = v + bias[n];
                v = ((const TAcc*)g.aux)[n] + z;
            } else if (g.epi == EPI_TANH_BWD) {
                TAcc h = Cvt<TIn>::to_acc(((const TIn*)g.aux)[m * g.ld_aux + n]);
                v = v * (TAcc(1) - h * h);
            }
            C[m * g.ldc + n] = Cvt<TOut>::from(v);
        }
    }
}

int gemm_f64(const GemmArgs& g, cudaStream_t s) {
    dim3 grid((g.N + GB_N - 1) / GB_N, (unsigned)((g.M + GB_M - 1) / GB_M));
    {
        ProfScope prof_(PROF_GEMM, s);
        k_gemm_simt<double, double, double><<<grid, 256, 0, s>>>(g);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int gemm_bf16_simt(const GemmArgs& g, bool out_bf16, cudaStream_t s) {
    dim3 grid((g.N + GB_N - 1) / GB_N, (unsigned)((g.M + GB_M - 1) / GB_M));
    {
        ProfScope prof_(PROF_GEMM, s);
        if (out_bf16) k_gemm_simt<__nv_bfloat16, float, __nv_bfloat16><<<grid, 256, 0, s>>>(g);
        else k_gemm_simt<__nv_bfloat16, float, float><<<grid, 256, 0, s>>>(g);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// mixed-form GEMMs with strided operands (widths that are not multiples of 8, which the
// tensor-memory-access unit cannot address): BF16 inputs, FP32 accumulation on the CUDA cores
static int gemm_mixed(const GemmArgs& g, bool out_bf16, cudaStream_t s) {
    return gemm_bf16_simt(g, out_bf16, s);
}

// |det| accumulated as m * 2^e with m in [0.5, 1): one FP64 multiply per pivot and no log in
// the factorisation kernels (FP64 issues slowly on this part): they store (m, e) per block and
// k_combine takes one log per configuration, log(m_a m_b) + (e_a + e_b) ln 2. The split of a
// positive normal double into mantissa and exponent is done on its bit pattern.
struct LogDet {
    double m = 1.0;
    int e = 0;
    __device__ __forceinline__ void mul(double v) {  // v > 0, finite
        const double x = m * v;
        if (!(x >= 2.2250738585072014e-308)) {  // subnormal product: the library split
            int k;
            m = frexp(x, &k);
            e += k;
            return;
        }
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        e += (int)((b >> 52) & 0x7ffull) - 1022;
        m = __longlong_as_double((long long)((b & ~(0x7ffull << 52)) | (1022ull << 52)));
    }
};

// ------------------------------------------------------------------------------------------
// batched LU: one warp per (det, spin block); the block sits in shared memory. Task t covers
// det t/2, spin t%2; it writes |det| of its block as (mantissa, exponent) to la2/ex2[spin*M + m],
// the sign to sg2[spin*M + m] and the block inverse to Ainv (if requested). Pivot: largest |a_ik|, lowest row on ties.
// ------------------------------------------------------------------------------------------
#define LU_WARPS 4

template <class T>
__global__ void __launch_bounds__(LU_WARPS * 32) k_lu(const ulonglong2* __restrict__ dets,
                                                      int64_t M, int norb, int na, int nb,
                                                      const T* __restrict__ Phi,
                                                      double* __restrict__ la2,
                                                      int* __restrict__ ex2,
                                                      int8_t* __restrict__ sg2, T* Ainv_a,
                                                      T* Ainv_b, int* singular) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nmax = na > nb ? na : nb, ld = nmax + 1;
    T* A = (T*)smem_raw + (size_t)warp * 2 * nmax * ld;
    T* Xs = A + nmax * ld;
    __shared__ int perm_s[LU_WARPS][64];
    __shared__ uint8_t occ_s[LU_WARPS][64];
    const int nel = na + nb;
    for (int64_t task = (int64_t)blockIdx.x * LU_WARPS + warp; task < 2 * M;
         task += (int64_t)gridDim.x * LU_WARPS) {
        const int64_t m = task >> 1;
        const int spin = (int)(task & 1);
        const int n = spin == 0 ? na : nb;
        const int col0 = spin == 0 ? 0 : na;
        ulonglong2 x = dets[m];
        uint64_t w = spin == 0 ? x.x : x.y;
        for (int p = lane; p < norb; p += 32) {
            if ((w >> p) & 1ull) {
                uint64_t below = p == 0 ? 0ull : ((1ull << p) - 1ull);
                occ_s[warp][__popcll(w & below)] = (uint8_t)p;
            }
        }
        __syncwarp();
        const T* phi = Phi + m * (int64_t)norb * nel;
        for (int t = lane; t < n * n; t += 32) {
            int r = t / n, c = t - r * n;
            A[r * ld + c] = phi[(int64_t)occ_s[warp][r] * nel + col0 + c];
        }
        for (int t = lane; t < n; t += 32) perm_s[warp][t] = t;
        __syncwarp();
        int sgn = 1;
        LogDet det_acc;
        bool sing = false;
        for (int k = 0; k < n; ++k) {
            T best = T(-1);
            int bi = n;
            for (int i = k + lane; i < n; i += 32) {
                T v = fabs(A[i * ld + k]);
                if (v > best) {
                    best = v;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                T ob = __shfl_xor_sync(FULL_MASK, best, o);
                int oi = __shfl_xor_sync(FULL_MASK, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (bi != k) {
                for (int c = lane; c < n; c += 32) {
                    T t = A[k * ld + c];
                    A[k * ld + c] = A[bi * ld + c];
                    A[bi * ld + c] = t;
                }
                if (lane == 0) {
                    int t = perm_s[warp][k];
                    perm_s[warp][k] = perm_s[warp][bi];
                    perm_s[warp][bi] = t;
                }
                sgn = -sgn;
            }
            __syncwarp();
            T piv = A[k * ld + k];
            if (piv == T(0)) {
                sing = true;
                break;
            }
            if (piv < T(0)) sgn = -sgn;
            det_acc.mul(fabs((double)piv));
            for (int i = k + 1 + lane; i < n; i += 32) {
                T l = A[i * ld + k] / piv;
                A[i * ld + k] = l;
                for (int j = k + 1; j < n; ++j) A[i * ld + j] -= l * A[k * ld + j];
            }
            __syncwarp();
        }
        T* Ainv = spin == 0 ? Ainv_a : Ainv_b;
        if (lane == 0) {
            la2[spin * M + m] = sing ? 0.0 : det_acc.m;
            ex2[spin * M + m] = sing ? 0 : det_acc.e;
            sg2[spin * M + m] = (int8_t)(sing ? 0 : sgn);
            if (sing && singular) atomicOr(singular, 1);
        }
        if (Ainv) {
            if (sing) {
                for (int t = lane; t < n * n; t += 32) Ainv[m * n * n + t] = T(0);
            } else {
                // column c of the inverse: solve L U y = P^T e_c (lane c)
                for (int c = lane; c < n; c += 32) {
                    for (int i = 0; i < n; ++i) {
                        T v = perm_s[warp][i] == c ? T(1) : T(0);
                        for (int j = 0; j < i; ++j) v -= A[i * ld + j] * Xs[j * ld + c];
                        Xs[i * ld + c] = v;
                    }
                    for (int i = n - 1; i >= 0; --i) {
                        T v = Xs[i * ld + c];
                        for (int j = i + 1; j < n; ++j) v -= A[i * ld + j] * Xs[j * ld + c];
                        Xs[i * ld + c] = v / A[i * ld + i];
                    }
                }
                __syncwarp();
                for (int t = lane; t < n * n; t += 32) {
                    int r = t / n, c = t - r * n;
                    Ainv[m * n * n + t] = Xs[r * ld + c];
                }
            }
        }
        __syncwarp();
    }
}

// log|psi| = log(m_a m_b) + (e_a + e_b) ln 2 from the two blocks' (mantissa, exponent) pairs
__global__ void k_combine(int64_t M, const double* __restrict__ la2, const int* __restrict__ ex2,
                          const int8_t* __restrict__ sg2, double* __restrict__ logabs,
                          int8_t* __restrict__ sign) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        int s = sg2[m] * sg2[M + m];
        sign[m] = (int8_t)s;
        logabs[m] = s == 0 ? -INFINITY
                           : log(la2[m] * la2[M + m]) + (double)(ex2[m] + ex2[M + m]) * M_LN2;
    }
}

// Small blocks: one thread per (det, spin block), the block in registers (N known at compile
// time, so every register index is static; the pivot row is swapped with predicated moves).
// Same partial pivoting as the warp kernel (largest |a_ik|, lowest row on ties), |det| in FP64
// as (mantissa, exponent), and the inverse solved column by column from the factors.
template <class T, int N>
__device__ __forceinline__ void lu_reg_rows(const ulonglong2* __restrict__ dets, int64_t M,
                                            int norb, int nel, int spin,
                                            const T* __restrict__ Phi,
                                            double* __restrict__ la_out, int* __restrict__ ex_out,
                                            int8_t* __restrict__ sg_out, T* __restrict__ Ainv,
                                            int* singular) {
    const int col0 = spin == 0 ? 0 : nel - N;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const ulonglong2 x = dets[m];
        uint64_t w = spin == 0 ? x.x : x.y;
        const T* phi = Phi + m * (int64_t)norb * nel + col0;
        T A[N][N];
        int perm[N];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            const int p = __ffsll((long long)w) - 1;
            w &= w - 1;
#pragma unroll
            for (int c = 0; c < N; ++c) A[r][c] = phi[(int64_t)p * nel + c];
            perm[r] = r;
        }
        int sgn = 1;
        LogDet det_acc;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            T best = fabs(A[k][k]);
            int pv = k;
#pragma unroll
            for (int i = k + 1; i < N; ++i)
                if (fabs(A[i][k]) > best) {
                    best = fabs(A[i][k]);
                    pv = i;
                }
            if (pv != k) {
                sgn = -sgn;
#pragma unroll
                for (int i = k + 1; i < N; ++i)
                    if (i == pv) {
#pragma unroll
                        for (int c = 0; c < N; ++c) {
                            const T t = A[k][c];
                            A[k][c] = A[i][c];
                            A[i][c] = t;
                        }
                        const int t = perm[k];
                        perm[k] = perm[i];
                        perm[i] = t;
                    }
            }
            const T piv = A[k][k];
            if (piv == T(0)) ok = false;
            if (ok) {
                if (piv < T(0)) sgn = -sgn;
                det_acc.mul(fabs((double)piv));
#pragma unroll
                for (int i = k + 1; i < N; ++i) {
                    const T l = A[i][k] / piv;
                    A[i][k] = l;
#pragma unroll
                    for (int j = k + 1; j < N; ++j) A[i][j] -= l * A[k][j];
                }
            }
        }
        la_out[m] = ok ? det_acc.m : 0.0;
        ex_out[m] = ok ? det_acc.e : 0;
        sg_out[m] = (int8_t)(ok ? sgn : 0);
        if (!ok && singular) atomicOr(singular, 1);
        if (Ainv) {
            T* out = Ainv + m * (int64_t)N * N;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                T y[N];
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    T v = perm[i] == c ? T(1) : T(0);
#pragma unroll
                    for (int j = 0; j < i; ++j) v -= A[i][j] * y[j];
                    y[i] = v;
                }
#pragma unroll
                for (int i = N - 1; i >= 0; --i) {
                    T v = y[i];
#pragma unroll
                    for (int j = i + 1; j < N; ++j) v -= A[i][j] * y[j];
                    y[i] = ok ? v / A[i][i] : T(0);
                }
#pragma unroll
                for (int i = 0; i < N; ++i) out[i * N + c] = y[i];
            }
        }
    }
}

template <class T, int N>
__global__ void __launch_bounds__(128) k_lu_reg(const ulonglong2* __restrict__ dets, int64_t M,
                                                int norb, int nel, int spin,
                                                const T* __restrict__ Phi,
                                                double* __restrict__ la_out,
                                                int* __restrict__ ex_out,
                                                int8_t* __restrict__ sg_out, T* __restrict__ Ainv,
                                                int* singular) {
    lu_reg_rows<T, N>(dets, M, norb, nel, spin, Phi, la_out, ex_out, sg_out, Ainv, singular);
}

// the same over many problems' blocks of one size: blockIdx.y = job
template <int N>
__global__ void __launch_bounds__(128) k_g_lu(const GLuJob* __restrict__ jobs) {
    const GLuJob J = jobs[blockIdx.y];
    lu_reg_rows<float, N>(J.dets, J.M, J.norb, J.nel, J.spin, J.Phi, J.la, J.ex, J.sg, J.Ainv,
                          J.singular);
}

template <class T, int N>
static int launch_lu_reg_n(const uint64_t* dets, int64_t M, int norb, int nel, int spin,
                           const T* Phi, double* la, int* ex, int8_t* sg, T* Ainv, int* singular,
                           cudaStream_t s) {
    k_lu_reg<T, N><<<grid_for(M, 128, 148 * 32), 128, 0, s>>>(
        (const ulonglong2*)dets, M, norb, nel, spin, Phi, la, ex, sg, Ainv, singular);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// dispatch on the block size; returns NQS_ERR_UNSUPPORTED above the register limit
template <class T>
static int launch_lu_reg(const uint64_t* dets, int64_t M, int norb, int nel, int spin, int n,
                         const T* Phi, double* la, int* ex, int8_t* sg, T* Ainv, int* singular,
                         cudaStream_t s) {
    const int nmax = sizeof(T) == 8 ? 7 : 12;
    if (n > nmax) return NQS_ERR_UNSUPPORTED;
    switch (n) {
#define NQS_LU_CASE(K)                                                                     \
    case K:                                                                                \
        return launch_lu_reg_n<T, (K <= (sizeof(T) == 8 ? 7 : 12) ? K : 1)>(               \
            dets, M, norb, nel, spin, Phi, la, ex, sg, Ainv, singular, s);
        NQS_LU_CASE(1) NQS_LU_CASE(2) NQS_LU_CASE(3) NQS_LU_CASE(4) NQS_LU_CASE(5)
        NQS_LU_CASE(6) NQS_LU_CASE(7) NQS_LU_CASE(8) NQS_LU_CASE(9) NQS_LU_CASE(10)
        NQS_LU_CASE(11) NQS_LU_CASE(12)
#undef NQS_LU_CASE
        default: return NQS_ERR_UNSUPPORTED;
    }
}

// Mixed-form blocks of 25..32 rows: one warp per (configuration, spin block), lane i holds row i
// of the block in registers (N is a template parameter, so every register index is static).
// Partial pivoting as in the other kernels (largest |a_ik|; on ties the row that would sit
// lowest after the row exchanges so far, tracked per lane as its current position): a warp
// max-reduction over |a_ik| of the rows not yet used, then a min-reduction over the positions
// of the maxima. Rows are not moved; the lane that pivots step k holds row k of U and row k of
// the multipliers of L. The pivot row reaches the other lanes by shuffles. The factors are then
// stored in pivot order in shared memory and lane c solves L U x = P e_c for column c of the
// inverse, reading the factors as 16-byte broadcasts. |det| = product of the pivots, reduced
// over the lanes in FP64 as mantissa x 2^exponent.
#define LU_LANE_WARPS 4
template <int N>
__global__ void __launch_bounds__(LU_LANE_WARPS * 32) k_lu_lane(
    const ulonglong2* __restrict__ dets, int64_t M, int norb, int nel, int spin,
    const float* __restrict__ Phi, double* __restrict__ la_out, int* __restrict__ ex_out,
    int8_t* __restrict__ sg_out, float* __restrict__ Ainv, int* singular) {
    constexpr int LD = (N + 3) & ~3;  // factor rows padded to 16 bytes
    __shared__ __align__(16) float lu_s[LU_LANE_WARPS][N][LD];
    __shared__ float dinv_s[LU_LANE_WARPS][N];
    __shared__ uint8_t occ_s[LU_LANE_WARPS][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col0 = spin == 0 ? 0 : nel - N;
    const bool vec = ((nel | col0) & 3) == 0 && (N & 3) == 0;
    float(*LU)[LD] = lu_s[warp];
    for (int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; m < M;
         m += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const ulonglong2 x = dets[m];
        const uint64_t w = spin == 0 ? x.x : x.y;
        for (int p = lane; p < norb; p += 32) {
            const uint64_t below = p == 0 ? 0ull : ((1ull << p) - 1ull);
            if ((w >> p) & 1ull) occ_s[warp][__popcll(w & below)] = (uint8_t)p;
        }
        __syncwarp();
        float r[N];
        if (lane < N) {
            const float* row = Phi + m * (int64_t)norb * nel + (int64_t)occ_s[warp][lane] * nel + col0;
            if (vec) {
#pragma unroll
                for (int c = 0; c < N; c += 4) {
                    const float4 v = *(const float4*)(row + c);
                    r[c] = v.x;
                    r[c + 1] = v.y;
                    r[c + 2] = v.z;
                    r[c + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int c = 0; c < N; ++c) r[c] = row[c];
            }
        } else {
#pragma unroll
            for (int c = 0; c < N; ++c) r[c] = 0.f;
        }
        bool used = lane >= N;
        int pos = lane, step = 0, sgn = 1;
        float piv_own = 1.f, dinv_own = 1.f;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (!ok) continue;  // warp-uniform
            const unsigned key = used ? 0u : __float_as_uint(fabsf(r[k]));
            const unsigned mx = __reduce_max_sync(FULL_MASK, key);
            if (mx == 0u) {  // no nonzero pivot left: singular block
                ok = false;
                continue;
            }
            const unsigned cand = key == mx ? (unsigned)pos : 0xffffffffu;
            const unsigned pmin = __reduce_min_sync(FULL_MASK, cand);
            const int p = __ffs(__ballot_sync(FULL_MASK, cand == pmin)) - 1;
            const float piv = __shfl_sync(FULL_MASK, r[k], p);
            if ((int)pmin != k) {  // the equivalent row exchange of positions k and pmin
                sgn = -sgn;
                if (pos == k) pos = (int)pmin;
            }
            if (piv < 0.f) sgn = -sgn;
            const float rp = 1.0f / piv;
            if (lane == p) {
                used = true;
                pos = k;
                step = k;
                piv_own = fabsf(piv);
                dinv_own = rp;
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {  // full range: the guard is static once unrolled
                if (j > k) {
                    const float u = __shfl_sync(FULL_MASK, r[j], p);
                    if (!used) r[j] = fmaf(-(r[k] * rp), u, r[j]);
                }
            }
            if (!used) r[k] *= rp;
        }
        // |det| over the lanes: mantissa in [0.5, 1) and exponent of each pivot, a product tree
        int e_own = 0;
        const double m_own = lane < N && ok ? (double)frexpf(piv_own, &e_own) : 1.0;
        double mt = m_own;
        int et = lane < N && ok ? e_own : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mt *= __shfl_xor_sync(FULL_MASK, mt, o);
            et += __shfl_xor_sync(FULL_MASK, et, o);
        }
        if (lane == 0) {
            la_out[m] = ok ? mt : 0.0;
            ex_out[m] = ok ? et : 0;
            sg_out[m] = (int8_t)(ok ? sgn : 0);
            if (!ok && singular) atomicOr(singular, 1);
        }
        if (Ainv) {
            float* out = Ainv + m * (int64_t)N * N;
            if (!ok) {
                for (int t = lane; t < N * N; t += 32) out[t] = 0.f;
            } else {
                if (lane < N) {
#pragma unroll
                    for (int c = 0; c < LD; c += 4)
                        *(float4*)&LU[step][c] = make_float4(r[c], c + 1 < N ? r[c + 1] : 0.f,
                                                             c + 2 < N ? r[c + 2] : 0.f,
                                                             c + 3 < N ? r[c + 3] : 0.f);
                    dinv_s[warp][step] = dinv_own;
                }
                __syncwarp();
                if (lane < N) {
                    // forward: y = L^{-1} e_step, L unit lower triangular
                    float y[N];
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                        float v = i == step ? 1.f : 0.f;
#pragma unroll
                        for (int c = 0; c < ((i + 3) & ~3); c += 4) {
                            const float4 l4 = *(const float4*)&LU[i][c];
                            if (c < i) v = fmaf(-l4.x, y[c], v);
                            if (c + 1 < i) v = fmaf(-l4.y, y[c + 1], v);
                            if (c + 2 < i) v = fmaf(-l4.z, y[c + 2], v);
                            if (c + 3 < i) v = fmaf(-l4.w, y[c + 3], v);
                        }
                        y[i] = v;
                    }
                    // backward: x = U^{-1} y
#pragma unroll
                    for (int i = N - 1; i >= 0; --i) {
                        float v = y[i];
#pragma unroll
                        for (int c = (i + 1) & ~3; c < N; c += 4) {
                            const float4 u4 = *(const float4*)&LU[i][c];
                            if (c > i) v = fmaf(-u4.x, y[c], v);
                            if (c + 1 > i && c + 1 < N) v = fmaf(-u4.y, y[c + 1], v);
                            if (c + 2 > i && c + 2 < N) v = fmaf(-u4.z, y[c + 2], v);
                            if (c + 3 > i && c + 3 < N) v = fmaf(-u4.w, y[c + 3], v);
                        }
                        y[i] = v * dinv_s[warp][i];
                    }
#pragma unroll
                    for (int i = 0; i < N; ++i) out[i * N + lane] = y[i];
                }
            }
        }
        __syncwarp();
    }
}

// Mixed-form blocks of 13..24 rows, four blocks per warp: the eight lanes of group g (lanes
// 8g .. 8g + 7) factor the block of configuration 4w + g, lane l holding rows l, l + 8, l + 16
// of it in registers. The pivot rule, the row-exchange sign and the arithmetic (the multiplier
// a_ik * (1 / a_kk) rounded, then one FMA per entry) are those of k_lu_lane. The pivot search
// reduces one 64-bit key per lane over the group (|a_ik| bits, then the complement of the row's
// position, so that ties go to the lowest position); the pivot row reaches the group through
// shared memory (16-byte stores by its owner, 16-byte broadcast loads by every lane), so each
// shared-memory access serves four blocks where k_lu_lane spends one shuffle per entry and
// block, and no lane idles (k_lu_lane leaves 32 - n lanes without a row). Inverse: each lane
// solves the columns of its own rows, the solves sharing every factor load.
#define LU_GRP_WARPS 4
template <int N>
__global__ void __launch_bounds__(LU_GRP_WARPS * 32) k_lu_grp(
    const ulonglong2* __restrict__ dets, int64_t M, int norb, int nel, int spin,
    const float* __restrict__ Phi, double* __restrict__ la_out, int* __restrict__ ex_out,
    int8_t* __restrict__ sg_out, float* __restrict__ Ainv, int* singular) {
    constexpr int R = (N + 7) / 8;     // rows per lane
    constexpr int LD = (N + 3) & ~3;  // factor rows padded to 16 bytes
    __shared__ __align__(16) float fac_s[LU_GRP_WARPS][4][N][LD];
    __shared__ __align__(16) float prow_s[LU_GRP_WARPS][4][LD];
    __shared__ float dinv_s[LU_GRP_WARPS][4][N];
    __shared__ uint8_t occ_s[LU_GRP_WARPS][4][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 3, l = lane & 7;
    const int col0 = spin == 0 ? 0 : nel - N;
    const bool vec = ((nel | col0) & 3) == 0 && (N & 3) == 0;
    float(*F)[LD] = fac_s[warp][g];
    float* prow = prow_s[warp][g];
    float* dinv = dinv_s[warp][g];
    uint8_t* occ = occ_s[warp][g];
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t mw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; mw * 4 < M;
         mw += wstride) {
        const int64_t m = mw * 4 + g;
        const bool mv = m < M;
        uint64_t wb = 0;
        if (mv) {
            const ulonglong2 x = dets[m];
            wb = spin == 0 ? x.x : x.y;
        }
        for (int p = l; p < norb; p += 8) {
            const uint64_t below = p == 0 ? 0ull : ((1ull << p) - 1ull);
            if ((wb >> p) & 1ull) occ[__popcll(wb & below)] = (uint8_t)p;
        }
        __syncwarp();
        float r[R][N];
        bool used[R];
        int pos[R], step[R];
        float piv_own[R], dinv_own[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int i = l + 8 * t;
            const bool live = mv && i < N;
            used[t] = !live;  // rows past the block (and groups past M) never pivot
            pos[t] = i;
            step[t] = 0;
            piv_own[t] = 1.f;
            dinv_own[t] = 1.f;
            if (live) {
                const float* row =
                    Phi + m * (int64_t)norb * nel + (int64_t)occ[i] * nel + col0;
                if (vec) {
#pragma unroll
                    for (int c = 0; c < N; c += 4) {
                        const float4 v = *(const float4*)(row + c);
                        r[t][c] = v.x;
                        r[t][c + 1] = v.y;
                        r[t][c + 2] = v.z;
                        r[t][c + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < N; ++c) r[t][c] = row[c];
                }
            } else {
#pragma unroll
                for (int c = 0; c < N; ++c) r[t][c] = 0.f;
            }
        }
        int sgn = 1;
        bool ok = mv;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            unsigned long long best = 0ull;
#pragma unroll
            for (int t = 0; t < R; ++t)
                if (!used[t]) {
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(fabsf(r[t][k])) << 32) |
                        (unsigned long long)(~(unsigned)pos[t]);
                    best = key > best ? key : best;
                }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(FULL_MASK, best, o, 8);
                best = other > best ? other : best;
            }
            if ((best >> 32) == 0ull) ok = false;  // no nonzero pivot left: singular block
            const int pmin = (int)(~(unsigned)best);
            int tstar = -1;
#pragma unroll
            for (int t = 0; t < R; ++t)
                if (ok && !used[t] && pos[t] == pmin) tstar = t;
            __syncwarp();  // the previous step's reads of prow are done
#pragma unroll
            for (int t = 0; t < R; ++t)
                if (t == tstar) {
#pragma unroll
                    for (int c = k & ~3; c < LD; c += 4)
                        *(float4*)&prow[c] =
                            make_float4(c < N ? r[t][c] : 0.f, c + 1 < N ? r[t][c + 1] : 0.f,
                                        c + 2 < N ? r[t][c + 2] : 0.f,
                                        c + 3 < N ? r[t][c + 3] : 0.f);
                }
            __syncwarp();
            if (ok) {
                const float piv = prow[k];
                if (pmin != k) {  // the equivalent row exchange of positions k and pmin
                    sgn = -sgn;
#pragma unroll
                    for (int t = 0; t < R; ++t)
                        if (pos[t] == k) pos[t] = pmin;
                }
                if (piv < 0.f) sgn = -sgn;
                const float rp = 1.0f / piv;
#pragma unroll
                for (int t = 0; t < R; ++t)
                    if (t == tstar) {
                        used[t] = true;
                        pos[t] = k;
                        step[t] = k;
                        piv_own[t] = fabsf(piv);
                        dinv_own[t] = rp;
                    }
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    if (used[t]) continue;
                    const float f = r[t][k] * rp;
#pragma unroll
                    for (int c = (k + 1) & ~3; c < N; c += 4) {
                        const float4 u4 = *(const float4*)&prow[c];
                        if (c > k) r[t][c] = fmaf(-f, u4.x, r[t][c]);
                        if (c + 1 > k && c + 1 < N) r[t][c + 1] = fmaf(-f, u4.y, r[t][c + 1]);
                        if (c + 2 > k && c + 2 < N) r[t][c + 2] = fmaf(-f, u4.z, r[t][c + 2]);
                        if (c + 3 > k && c + 3 < N) r[t][c + 3] = fmaf(-f, u4.w, r[t][c + 3]);
                    }
                    r[t][k] = f;
                }
            }
        }
        // |det| over the group: mantissa in [0.5, 1) and exponent of each pivot, a product tree
        double mt = 1.0;
        int et = 0;
#pragma unroll
        for (int t = 0; t < R; ++t)
            if (ok && l + 8 * t < N) {
                int e = 0;
                mt *= (double)frexpf(piv_own[t], &e);
                et += e;
            }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            mt *= __shfl_xor_sync(FULL_MASK, mt, o, 8);
            et += __shfl_xor_sync(FULL_MASK, et, o, 8);
        }
        if (l == 0 && mv) {
            la_out[m] = ok ? mt : 0.0;
            ex_out[m] = ok ? et : 0;
            sg_out[m] = (int8_t)(ok ? sgn : 0);
            if (!ok && singular) atomicOr(singular, 1);
        }
        if (Ainv) {
            float* out = Ainv + m * (int64_t)N * N;
            if (ok) {
#pragma unroll
                for (int t = 0; t < R; ++t)
                    if (l + 8 * t < N) {
#pragma unroll
                        for (int c = 0; c < LD; c += 4)
                            *(float4*)&F[step[t]][c] = make_float4(
                                r[t][c], c + 1 < N ? r[t][c + 1] : 0.f,
                                c + 2 < N ? r[t][c + 2] : 0.f, c + 3 < N ? r[t][c + 3] : 0.f);
                        dinv[step[t]] = dinv_own[t];
                    }
            } else if (mv) {
                for (int q = l; q < N * N; q += 8) out[q] = 0.f;
            }
            __syncwarp();
            if (ok) {
                // lane l, row t: y = L^{-1} e_step, then x = U^{-1} y: column l + 8t of the
                // inverse (the unit vector of that row's pivot step)
                float y[R][N];
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    float v[R];
#pragma unroll
                    for (int t = 0; t < R; ++t) v[t] = i == step[t] ? 1.f : 0.f;
#pragma unroll
                    for (int c = 0; c < ((i + 3) & ~3); c += 4) {
                        const float4 l4 = *(const float4*)&F[i][c];
#pragma unroll
                        for (int t = 0; t < R; ++t) {
                            if (c < i) v[t] = fmaf(-l4.x, y[t][c], v[t]);
                            if (c + 1 < i) v[t] = fmaf(-l4.y, y[t][c + 1], v[t]);
                            if (c + 2 < i) v[t] = fmaf(-l4.z, y[t][c + 2], v[t]);
                            if (c + 3 < i) v[t] = fmaf(-l4.w, y[t][c + 3], v[t]);
                        }
                    }
#pragma unroll
                    for (int t = 0; t < R; ++t) y[t][i] = v[t];
                }
#pragma unroll
                for (int i = N - 1; i >= 0; --i) {
                    float v[R];
#pragma unroll
                    for (int t = 0; t < R; ++t) v[t] = y[t][i];
#pragma unroll
                    for (int c = (i + 1) & ~3; c < N; c += 4) {
                        const float4 u4 = *(const float4*)&F[i][c];
#pragma unroll
                        for (int t = 0; t < R; ++t) {
                            if (c > i) v[t] = fmaf(-u4.x, y[t][c], v[t]);
                            if (c + 1 > i && c + 1 < N) v[t] = fmaf(-u4.y, y[t][c + 1], v[t]);
                            if (c + 2 > i && c + 2 < N) v[t] = fmaf(-u4.z, y[t][c + 2], v[t]);
                            if (c + 3 > i && c + 3 < N) v[t] = fmaf(-u4.w, y[t][c + 3], v[t]);
                        }
                    }
                    const float di = dinv[i];
#pragma unroll
                    for (int t = 0; t < R; ++t) y[t][i] = v[t] * di;
                }
#pragma unroll
                for (int t = 0; t < R; ++t)
                    if (l + 8 * t < N) {
#pragma unroll
                        for (int i = 0; i < N; ++i) out[i * N + l + 8 * t] = y[t][i];
                    }
            }
        }
        __syncwarp();  // occ, F and dinv are rewritten by the next configuration
    }
}

template <int N>
static int launch_lu_grp_n(const uint64_t* dets, int64_t M, int norb, int nel, int spin,
                           const float* Phi, double* la, int* ex, int8_t* sg, float* Ainv,
                           int* singular, cudaStream_t s) {
    const int64_t warps = (M + 3) / 4;
    k_lu_grp<N><<<grid_for(warps * 32, LU_GRP_WARPS * 32, 148 * 32), LU_GRP_WARPS * 32, 0, s>>>(
        (const ulonglong2*)dets, M, norb, nel, spin, Phi, la, ex, sg, Ainv, singular);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

template <int N>
static int launch_lu_lane_n(const uint64_t* dets, int64_t M, int norb, int nel, int spin,
                            const float* Phi, double* la, int* ex, int8_t* sg, float* Ainv,
                            int* singular, cudaStream_t s) {
    k_lu_lane<N><<<grid_for(M * 32, LU_LANE_WARPS * 32, 148 * 32), LU_LANE_WARPS * 32, 0, s>>>(
        (const ulonglong2*)dets, M, norb, nel, spin, Phi, la, ex, sg, Ainv, singular);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

static int launch_lu_lane(const uint64_t* dets, int64_t M, int norb, int nel, int spin, int n,
                          const float* Phi, double* la, int* ex, int8_t* sg, float* Ainv,
                          int* singular, cudaStream_t s) {
    switch (n) {
#define NQS_GRP_CASE(K)                                                                       \
    case K:                                                                                   \
        return launch_lu_grp_n<K>(dets, M, norb, nel, spin, Phi, la, ex, sg, Ainv, singular, s);
#define NQS_LANE_CASE(K)                                                                      \
    case K:                                                                                   \
        return launch_lu_lane_n<K>(dets, M, norb, nel, spin, Phi, la, ex, sg, Ainv, singular, s);
        NQS_GRP_CASE(13) NQS_GRP_CASE(14) NQS_GRP_CASE(15) NQS_GRP_CASE(16)
        NQS_GRP_CASE(17) NQS_GRP_CASE(18) NQS_GRP_CASE(19) NQS_GRP_CASE(20)
        NQS_GRP_CASE(21) NQS_GRP_CASE(22) NQS_GRP_CASE(23) NQS_GRP_CASE(24)
        NQS_LANE_CASE(25) NQS_LANE_CASE(26) NQS_LANE_CASE(27) NQS_LANE_CASE(28)
        NQS_LANE_CASE(29) NQS_LANE_CASE(30) NQS_LANE_CASE(31) NQS_LANE_CASE(32)
#undef NQS_LANE_CASE
#undef NQS_GRP_CASE
        default: return NQS_ERR_UNSUPPORTED;
    }
}

template <class T>
static int launch_lu(nqs_net* net, const uint64_t* dets, int64_t M, const T* Phi, double* la2,
                     int* ex2, int8_t* sg2, T* Ainv_a, T* Ainv_b, int* singular,
                     cudaStream_t s) {
    const ProblemDev& P = net->prob->d;
    const int nel = P.na + P.nb;
    if (P.na <= (sizeof(T) == 8 ? 7 : 12) && P.nb <= (sizeof(T) == 8 ? 7 : 12)) {
        ProfScope prof_(PROF_LU, s);
        NQS_TRY(launch_lu_reg<T>(dets, M, P.norb, nel, 0, P.na, Phi, la2, ex2, sg2, Ainv_a,
                                 singular, s));
        NQS_TRY(launch_lu_reg<T>(dets, M, P.norb, nel, 1, P.nb, Phi, la2 + M, ex2 + M, sg2 + M,
                                 Ainv_b, singular, s));
        return NQS_OK;
    }
    if constexpr (sizeof(T) == 4) {
        if (P.na <= 32 && P.nb <= 32) {  // FP32: register kernels per block
            ProfScope prof_(PROF_LU, s);
            for (int spin = 0; spin < 2; ++spin) {
                const int n = spin == 0 ? P.na : P.nb;
                T* inv = spin == 0 ? Ainv_a : Ainv_b;
                if (n <= 12)
                    NQS_TRY(launch_lu_reg<T>(dets, M, P.norb, nel, spin, n, Phi, la2 + spin * M,
                                             ex2 + spin * M, sg2 + spin * M, inv, singular, s));
                else
                    NQS_TRY(launch_lu_lane(dets, M, P.norb, nel, spin, n, Phi, la2 + spin * M,
                                           ex2 + spin * M, sg2 + spin * M, inv, singular, s));
            }
            return NQS_OK;
        }
    }
    int nmax = P.na > P.nb ? P.na : P.nb;
    size_t smem = (size_t)LU_WARPS * 2 * nmax * (nmax + 1) * sizeof(T);
    if (smem > 48 * 1024)
        NQS_CK(cudaFuncSetAttribute(k_lu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    unsigned grid = grid_for(2 * M, LU_WARPS, 148 * 64);
    {
        ProfScope prof_(PROF_LU, s);
        k_lu<T><<<grid, LU_WARPS * 32, smem, s>>>((const ulonglong2*)dets, M, P.norb, P.na, P.nb, Phi,
                                                  la2, ex2, sg2, Ainv_a, Ainv_b, singular);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// forward: layer 1 gather, layers 2 and 3 as GEMMs, then the two LU factorisations
// ------------------------------------------------------------------------------------------
static bool tc_shapes_ok(const nqs_net* net) {
    return net->dtype == NQS_MIXED && net->H1 % 8 == 0 && net->H2 % 8 == 0;
}
static int forward_mixed_tc(nqs_net* net, Scratch& sc, const uint64_t* dets, int64_t M, Fwd& f,
                            bool keep, double* logabs, int8_t* sign, cudaStream_t s);
static int backward_mixed_tc(nqs_net* net, Scratch& sc, const uint64_t* dets, const Fwd& f,
                             const double* w, void* grad, cudaStream_t s);

int net_forward(nqs_net* net, Scratch& sc, const uint64_t* dets, int64_t M, Fwd& f,
                bool keep, double* logabs, int8_t* sign, cudaStream_t s) {
    if (tc_shapes_ok(net)) return forward_mixed_tc(net, sc, dets, M, f, keep, logabs, sign, s);
    const ProblemDev& P = net->prob->d;
    const bool mixed = net->dtype == NQS_MIXED;
    const int H1 = net->H1, H2 = net->H2, nin = net->nin, nout = net->nout;
    const size_t esz = mixed ? 2 : 8;  // activation element size
    const size_t psz = mixed ? 4 : 8;  // Phi / LU element size
    memset(&f, 0, sizeof f);
    f.M = M;
    f.logabs = logabs;
    f.sign = sign;
    NQS_TRY(sc.get((uint8_t**)&f.H1, M * H1 * esz));
    NQS_TRY(sc.get((uint8_t**)&f.H2, M * H2 * esz));
    NQS_TRY(sc.get((uint8_t**)&f.Phi, M * nout * psz));
    if (keep) {
        NQS_TRY(sc.get((uint8_t**)&f.X, M * nin * esz));
        NQS_TRY(sc.get((uint8_t**)&f.Ainv_a, M * P.na * P.na * psz));
        NQS_TRY(sc.get((uint8_t**)&f.Ainv_b, M * P.nb * P.nb * psz));
    }
    NQS_TRY(sc.get(&f.singular, 1));
    NQS_CK(cudaMemsetAsync(f.singular, 0, sizeof(int), s));
    const ulonglong2* D2 = (const ulonglong2*)dets;
    unsigned g1 = grid_for(M * H1, 256, 148 * 64);
    if (mixed) {
        k_layer1<__nv_bfloat16, float, __nv_bfloat16><<<g1, 256, 0, s>>>(
            D2, M, P.norb, H1, (const __nv_bfloat16*)net->p[0], (const float*)net->p[1],
            (__nv_bfloat16*)f.H1, nullptr);
        NQS_CK_LAUNCH();
        if (keep) {
            k_bits<__nv_bfloat16, float><<<grid_for(M * nin, 256), 256, 0, s>>>(
                D2, M, P.norb, (__nv_bfloat16*)f.X);
            NQS_CK_LAUNCH();
        }
    } else {
        k_layer1<double, double, double><<<g1, 256, 0, s>>>(D2, M, P.norb, H1,
                                                            (const double*)net->p[0],
                                                            (const double*)net->p[1],
                                                            (double*)f.H1, nullptr);
        NQS_CK_LAUNCH();
        if (keep) {
            k_bits<double, double><<<grid_for(M * nin, 256), 256, 0, s>>>(D2, M, P.norb,
                                                                         (double*)f.X);
            NQS_CK_LAUNCH();
        }
    }
    GemmArgs g{};
    g.M = (int)M;
    g.N = H2;
    g.K = H1;
    g.A = f.H1;
    g.a_m = H1;
    g.a_k = 1;
    g.B = net->p[2];
    g.b_n = H1;
    g.b_k = 1;
    g.C = f.H2;
    g.ldc = H2;
    g.epi = EPI_BIAS_TANH;
    g.bias = net->p[3];
    NQS_TRY(mixed ? gemm_mixed(g, true, s) : gemm_f64(g, s));
    g.N = nout;
    g.K = H2;
    g.A = f.H2;
    g.a_m = H2;
    g.B = net->p[4];
    g.b_n = H2;
    g.C = f.Phi;
    g.ldc = nout;
    g.epi = EPI_BIAS_PHI0;
    g.bias = net->p[5];
    g.aux = net->p[6];
    NQS_TRY(mixed ? gemm_mixed(g, false, s) : gemm_f64(g, s));
    double* la2;
    int* ex2;
    int8_t* sg2;
    NQS_TRY(sc.get(&la2, 2 * M));
    NQS_TRY(sc.get(&ex2, 2 * M));
    NQS_TRY(sc.get(&sg2, 2 * M));
    if (mixed)
        NQS_TRY(launch_lu<float>(net, dets, M, (const float*)f.Phi, la2, ex2, sg2,
                                 (float*)f.Ainv_a, (float*)f.Ainv_b, f.singular, s));
    else
        NQS_TRY(launch_lu<double>(net, dets, M, (const double*)f.Phi, la2, ex2, sg2,
                                  (double*)f.Ainv_a, (double*)f.Ainv_b, f.singular, s));
    k_combine<<<grid_for(M, 256), 256, 0, s>>>(M, la2, ex2, sg2, logabs, sign);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// backward (hand-written adjoint)
//   dPhi(x)[occ_s[j]][col0_s + k] = w_x (A_s^{-1})[k][j]     (Jacobi's formula)
//   dW3 = dPhi^T H2, db3 = colsum dPhi, dZ2 = (dPhi W3) * (1 - H2^2)
//   dW2 = dZ2^T H1,  db2 = colsum dZ2,  dZ1 = (dZ2 W2) * (1 - H1^2)
//   dW1 = dZ1^T X,   db1 = colsum dZ1
// ------------------------------------------------------------------------------------------
template <class TG>
__device__ __forceinline__ TG grad_from_double(double g);
template <>
__device__ __forceinline__ double grad_from_double<double>(double g) { return g; }
template <>
__device__ __forceinline__ __nv_bfloat16 grad_from_double<__nv_bfloat16>(double g) {
    return __float2bfloat16_rn((float)g);
}

template <class T, class TG>
__global__ void __launch_bounds__(256) k_adjoint(const ulonglong2* __restrict__ dets, int64_t M,
                                                 int norb, int na, int nb,
                                                 const double* __restrict__ w,
                                                 const T* __restrict__ Ainv_a,
                                                 const T* __restrict__ Ainv_b,
                                                 TG* __restrict__ dPhi, int64_t ldp) {
    // One warp per configuration: its occupied orbitals are listed in shared memory, then the
    // lanes write dPhi[occ_j][col0 + k] = w * (A^-1)_kj of each spin block, a block row (k
    // contiguous) per group of lanes. dPhi is zero elsewhere (cleared by the caller). The
    // product is formed in T (FP32 in the mixed form, whose dPhi is bf16; FP64 otherwise).
    __shared__ uint8_t occ_s[8][2][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nel = na + nb;
    for (int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; m < M;
         m += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const ulonglong2 x = dets[m];
        for (int p = lane; p < norb; p += 32) {
            const uint64_t below = p == 0 ? 0ull : ((1ull << p) - 1ull);
            if ((x.x >> p) & 1ull) occ_s[warp][0][__popcll(x.x & below)] = (uint8_t)p;
            if ((x.y >> p) & 1ull) occ_s[warp][1][__popcll(x.y & below)] = (uint8_t)p;
        }
        __syncwarp();
        const T wm = (T)w[m];
        for (int spin = 0; spin < 2; ++spin) {
            const int n = spin == 0 ? na : nb, col0 = spin == 0 ? 0 : na;
            const T* inv = spin == 0 ? Ainv_a + m * na * na : Ainv_b + m * nb * nb;
            for (int r = lane; r < n * n; r += 32) {
                const int j = r / n, k = r - j * n;
                const T g = wm * inv[k * n + j];
                dPhi[m * ldp + (int64_t)occ_s[warp][spin][j] * nel + col0 + k] =
                    grad_from_double<TG>((double)g);
            }
        }
        __syncwarp();
    }
}

// column sums of X [M][N] into out[N], split over row chunks then combined (deterministic)
template <class TIn, class TAcc>
__global__ void k_colsum_part(const TIn* __restrict__ X, int64_t M, int N, int64_t rows_per,
                              TAcc* __restrict__ part) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int64_t r0 = (int64_t)blockIdx.y * rows_per, r1 = r0 + rows_per < M ? r0 + rows_per : M;
    TAcc s = TAcc(0);
    for (int64_t r = r0; r < r1; ++r) s += Cvt<TIn>::to_acc(X[r * N + n]);
    part[(int64_t)blockIdx.y * N + n] = s;
}
template <class TAcc>
__global__ void k_colsum_final(const TAcc* __restrict__ part, int splits, int N,
                               TAcc* __restrict__ out) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    TAcc s = TAcc(0);
    for (int k = 0; k < splits; ++k) s += part[(int64_t)k * N + n];
    out[n] = s;
}

template <class TIn, class TAcc>
static int colsum(Scratch& sc, const void* X, int64_t M, int N, void* out, cudaStream_t s) {
    int splits = (int)((M + 1023) / 1024);
    if (splits > 256) splits = 256;
    if (splits < 1) splits = 1;
    int64_t rows_per = (M + splits - 1) / splits;
    TAcc* part;
    NQS_TRY(sc.get(&part, (size_t)splits * N));
    dim3 grid((N + 127) / 128, splits);
    k_colsum_part<TIn, TAcc><<<grid, 128, 0, s>>>((const TIn*)X, M, N, rows_per, part);
    NQS_CK_LAUNCH();
    k_colsum_final<TAcc><<<(N + 127) / 128, 128, 0, s>>>(part, splits, N, (TAcc*)out);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int net_backward(nqs_net* net, Scratch& sc, const uint64_t* dets, const Fwd& f, const double* w,
                 void* grad, cudaStream_t s) {
    if (f.tc) return backward_mixed_tc(net, sc, dets, f, w, grad, s);
    const ProblemDev& P = net->prob->d;
    const bool mixed = net->dtype == NQS_MIXED;
    const int64_t M = f.M;
    const int H1 = net->H1, H2 = net->H2, nin = net->nin, nout = net->nout;
    const size_t esz = mixed ? 2 : 8, gsz = mixed ? 4 : 8;
    uint8_t* G = (uint8_t*)grad;
    uint8_t* gW1 = G;
    uint8_t* gb1 = gW1 + (size_t)H1 * nin * gsz;
    uint8_t* gW2 = gb1 + (size_t)H1 * gsz;
    uint8_t* gb2 = gW2 + (size_t)H2 * H1 * gsz;
    uint8_t* gW3 = gb2 + (size_t)H2 * gsz;
    uint8_t* gb3 = gW3 + (size_t)nout * H2 * gsz;
    void *dPhi, *dZ2, *dZ1;
    NQS_TRY(sc.get((uint8_t**)&dPhi, M * nout * esz));
    NQS_TRY(sc.get((uint8_t**)&dZ2, M * H2 * esz));
    NQS_TRY(sc.get((uint8_t**)&dZ1, M * H1 * esz));
    NQS_CK(cudaMemsetAsync(dPhi, 0, M * nout * esz, s));
    const ulonglong2* D2 = (const ulonglong2*)dets;
    if (mixed)
        k_adjoint<float, __nv_bfloat16><<<grid_for(M * 32, 256, 148 * 64), 256, 0, s>>>(
            D2, M, P.norb, P.na, P.nb, w, (const float*)f.Ainv_a, (const float*)f.Ainv_b,
            (__nv_bfloat16*)dPhi, nout);
    else
        k_adjoint<double, double><<<grid_for(M * 32, 256, 148 * 64), 256, 0, s>>>(
            D2, M, P.norb, P.na, P.nb, w, (const double*)f.Ainv_a, (const double*)f.Ainv_b,
            (double*)dPhi, nout);
    NQS_CK_LAUNCH();
    auto gemm = [&](const GemmArgs& g, bool out_act) -> int {
        return mixed ? gemm_mixed(g, out_act, s) : gemm_f64(g, s);
    };
    GemmArgs g{};
    // dW3[o][k] = sum_m dPhi[m][o] H2[m][k]
    g.M = nout; g.N = H2; g.K = (int)M;
    g.A = dPhi; g.a_m = 1; g.a_k = nout;
    g.B = f.H2; g.b_n = 1; g.b_k = H2;
    g.C = gW3; g.ldc = H2; g.epi = EPI_STORE;
    NQS_TRY(gemm(g, false));
    // dZ2[m][k] = (sum_o dPhi[m][o] W3[o][k]) (1 - H2^2)
    g = GemmArgs{};
    g.M = (int)M; g.N = H2; g.K = nout;
    g.A = dPhi; g.a_m = nout; g.a_k = 1;
    g.B = net->p[4]; g.b_n = 1; g.b_k = H2;
    g.C = dZ2; g.ldc = H2; g.epi = EPI_TANH_BWD; g.aux = f.H2; g.ld_aux = H2;
    NQS_TRY(gemm(g, true));
    // dW2[i][k] = sum_m dZ2[m][i] H1[m][k]
    g = GemmArgs{};
    g.M = H2; g.N = H1; g.K = (int)M;
    g.A = dZ2; g.a_m = 1; g.a_k = H2;
    g.B = f.H1; g.b_n = 1; g.b_k = H1;
    g.C = gW2; g.ldc = H1; g.epi = EPI_STORE;
    NQS_TRY(gemm(g, false));
    // dZ1[m][k] = (sum_i dZ2[m][i] W2[i][k]) (1 - H1^2)
    g = GemmArgs{};
    g.M = (int)M; g.N = H1; g.K = H2;
    g.A = dZ2; g.a_m = H2; g.a_k = 1;
    g.B = net->p[2]; g.b_n = 1; g.b_k = H1;
    g.C = dZ1; g.ldc = H1; g.epi = EPI_TANH_BWD; g.aux = f.H1; g.ld_aux = H1;
    NQS_TRY(gemm(g, true));
    // dW1[i][k] = sum_m dZ1[m][i] X[m][k]
    g = GemmArgs{};
    g.M = H1; g.N = nin; g.K = (int)M;
    g.A = dZ1; g.a_m = 1; g.a_k = H1;
    g.B = f.X; g.b_n = 1; g.b_k = nin;
    g.C = gW1; g.ldc = nin; g.epi = EPI_STORE;
    NQS_TRY(gemm(g, false));
    if (mixed) {
        NQS_TRY((colsum<__nv_bfloat16, float>(sc, dPhi, M, nout, gb3, s)));
        NQS_TRY((colsum<__nv_bfloat16, float>(sc, dZ2, M, H2, gb2, s)));
        NQS_TRY((colsum<__nv_bfloat16, float>(sc, dZ1, M, H1, gb1, s)));
    } else {
        NQS_TRY((colsum<double, double>(sc, dPhi, M, nout, gb3, s)));
        NQS_TRY((colsum<double, double>(sc, dZ2, M, H2, gb2, s)));
        NQS_TRY((colsum<double, double>(sc, dZ1, M, H1, gb1, s)));
    }
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// mixed form on tensor cores (tcgen05): the layer GEMMs take K-major operands; the weight
// gradients (K = |S|) read the row-major activations and adjoints as MN-major operands, so no
// transposed copy of an [|S|][H] matrix is made. The transposes below are of the weights.
// ------------------------------------------------------------------------------------------
// dst[c][r] = src[r][c] for r < R, c < Cn: 64 x 64 tiles through shared memory. Each thread
// moves 8 consecutive elements (16 bytes) on the global side when the row is whole and aligned
// (vec), else element by element; the shared tile's row stride of 66 elements (33 words) keeps
// the column reads of the write-out to 2-way bank conflicts.
#define TR_T 64
#define TR_LD 66
__global__ void __launch_bounds__(256) k_transpose_bf16(const __nv_bfloat16* __restrict__ src,
                                                        int64_t R, int64_t Cn, int64_t lds,
                                                        __nv_bfloat16* __restrict__ dst,
                                                        int64_t ldd, int vec) {
    __shared__ __align__(16) unsigned short tile[TR_T][TR_LD];
    const int64_t r0 = (int64_t)blockIdx.y * TR_T, c0 = (int64_t)blockIdx.x * TR_T;
    const unsigned short* S = (const unsigned short*)src;
    unsigned short* D = (unsigned short*)dst;
    for (int t = threadIdx.x; t < TR_T * 8; t += 256) {
        const int rr = t >> 3, c8 = (t & 7) * 8;
        const int64_t r = r0 + rr, c = c0 + c8;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (r < R) {
            if (vec && c + 8 <= Cn) {
                const uint4 v = __ldcs((const uint4*)(S + r * lds + c));
                w[0] = v.x;
                w[1] = v.y;
                w[2] = v.z;
                w[3] = v.w;
            } else {
                for (int j = 0; j < 8; ++j)
                    if (c + j < Cn) w[j >> 1] |= (uint32_t)S[r * lds + c + j] << (16 * (j & 1));
            }
        }
        uint32_t* row = (uint32_t*)&tile[rr][c8];  // 4-byte aligned: TR_LD and c8 are even
        row[0] = w[0];
        row[1] = w[1];
        row[2] = w[2];
        row[3] = w[3];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < TR_T * 8; t += 256) {
        const int cc = t >> 3, r8 = (t & 7) * 8;
        const int64_t c = c0 + cc, r = r0 + r8;
        if (c >= Cn) continue;
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            w[k] = (uint32_t)tile[r8 + 2 * k][cc] | ((uint32_t)tile[r8 + 2 * k + 1][cc] << 16);
        if (vec && r + 8 <= R) {
            *(uint4*)(D + c * ldd + r) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            for (int j = 0; j < 8; ++j)
                if (r + j < R) D[c * ldd + r + j] = (unsigned short)(w[j >> 1] >> (16 * (j & 1)));
        }
    }
}

static int transpose_bf16(const void* src, int64_t R, int64_t Cn, int64_t lds, void* dst,
                          int64_t ldd, cudaStream_t s) {
    dim3 grid((unsigned)((Cn + TR_T - 1) / TR_T), (unsigned)((R + TR_T - 1) / TR_T));
    // 16-byte global accesses when both matrices' rows start on 16-byte boundaries
    const int vec = (((uintptr_t)src | (uintptr_t)dst) & 15) == 0 && (lds & 7) == 0 &&
                    (ldd & 7) == 0;
    k_transpose_bf16<<<grid, 256, 0, s>>>((const __nv_bfloat16*)src, R, Cn, lds,
                                          (__nv_bfloat16*)dst, ldd, vec);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// X[m][c] = input bit c of det m as bf16 0/1 (alpha bits 0..norb-1, then beta), zero for
// nin <= c < ldX; one thread per 8 columns (one 16-byte store)
__global__ void k_bits_rows(const ulonglong2* __restrict__ dets, int64_t M, int norb, int ldX,
                            __nv_bfloat16* __restrict__ X) {
    const int nin = 2 * norb, per = ldX / 8;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = t / per;
        const int c0 = (int)(t - m * per) * 8;
        const ulonglong2 x = dets[m];
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t v = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = c0 + 2 * k + h;
                uint32_t bit = 0;
                if (c < norb) bit = (uint32_t)(x.x >> c) & 1u;
                else if (c < nin) bit = (uint32_t)(x.y >> (c - norb)) & 1u;
                v |= (bit ? 0x3F80u : 0u) << (16 * h);  // bf16 1.0 = 0x3F80
            }
            w[k] = v;
        }
        *(uint4*)(X + m * ldX + c0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// W1 [H1][nin] -> [H1][ldX] with zero columns nin..ldX-1 (16-byte row pitch for TMA)
__global__ void k_pad_cols_bf16(const __nv_bfloat16* __restrict__ W, int R, int nin, int ldX,
                                __nv_bfloat16* __restrict__ Wp) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)R * ldX;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / ldX), c = (int)(t - (int64_t)r * ldX);
        Wp[t] = c < nin ? W[(int64_t)r * nin + c] : __float2bfloat16_rn(0.f);
    }
}

// chunk length of the bias-gradient row sums of the batched problems (k_g_bias_grads)
#define ROWSUM_CHUNK 16384

// out[n] = sum over the M rows of X [M][ld] (bf16) of column n, FP32 with compensated
// (Kahan) additions, fixed order: a row is covered by tpr = ceil(N / 8) threads rounded up to
// a warp (thread t: columns 8t .. 8t + 7, one 16-byte load per row), a 256-thread block holds
// 256 / tpr such groups, and group q of block b sums rows [(b G + q) R, (b G + q + 1) R) in row
// order (R = COLSUM_ROWS, G groups a block); then one warp per column adds the groups'
// partial sums: lane l of the column's warp the partials l, l + 32, ... in order, then the 32
// lane sums by a fixed shuffle tree. The compensation keeps the error near one rounding of the
// result whatever |S|, so the order of the terms does not show at the level of FP32.
#define COLSUM_ROWS 1024
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__global__ void __launch_bounds__(256) k_colsum_bf16_part(const __nv_bfloat16* __restrict__ X,
                                                          int64_t M, int N, int64_t ld, int tpr,
                                                          float2* __restrict__ part) {
    const int groups = 256 / tpr;
    const int q = threadIdx.x / tpr, tt = threadIdx.x - q * tpr;
    if (q >= groups) return;
    const int64_t pidx = (int64_t)blockIdx.x * groups + q;
    const int64_t r0 = pidx * COLSUM_ROWS;
    const int64_t r1 = r0 + COLSUM_ROWS < M ? r0 + COLSUM_ROWS : M;
    for (int c8 = 8 * tt; c8 < N; c8 += 8 * tpr) {
        float acc[8], cmp[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] = cmp[t] = 0.f;
#pragma unroll 4
        for (int64_t r = r0; r < r1; ++r) {
            const uint4 pk = *(const uint4*)(X + r * ld + c8);
            const __nv_bfloat162* h2 = (const __nv_bfloat162*)&pk;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float2 f = __bfloat1622float2(h2[t]);
                kahan_add(acc[2 * t], cmp[2 * t], f.x);
                kahan_add(acc[2 * t + 1], cmp[2 * t + 1], f.y);
            }
        }
        float2* out = part + pidx * N;
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (c8 + t < N) out[c8 + t] = make_float2(acc[t], cmp[t]);
    }
}

__global__ void k_colsum_bf16_final(const float2* __restrict__ part, int N, int64_t nparts,
                                    float* __restrict__ out) {
    const int n = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= N) return;  // warp-uniform
    float t = 0.f, c = 0.f;
    for (int64_t b = lane; b < nparts; b += 32) {
        const float2 p = part[b * N + n];
        kahan_add(t, c, p.x);
        kahan_add(t, c, -p.y);  // the group's own compensation (its sum's missing part, negated)
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ot = __shfl_xor_sync(FULL_MASK, t, o), oc = __shfl_xor_sync(FULL_MASK, c, o);
        kahan_add(t, c, ot);
        kahan_add(t, c, -oc);
    }
    if (lane == 0) out[n] = t;
}

// ld: a multiple of 8 with room for N rounded up to 8 (the padding columns are read, not used)
static int colsum_bf16(Scratch& sc, const void* X, int64_t M, int N, int64_t ld, float* out,
                       cudaStream_t s) {
    if (ld % 8 || ld < ((N + 7) & ~7) || ((uintptr_t)X & 15) || N <= 0) return NQS_ERR_ARG;
    int tpr = ((N + 7) / 8 + 31) & ~31;
    if (tpr > 256) tpr = 256;
    const int groups = 256 / tpr;
    const int64_t nparts = (M + COLSUM_ROWS - 1) / COLSUM_ROWS;
    const int64_t nblocks = (nparts + groups - 1) / groups;
    float2* part;
    NQS_TRY(sc.get(&part, (size_t)nblocks * groups * N));
    k_colsum_bf16_part<<<(unsigned)nblocks, 256, 0, s>>>((const __nv_bfloat16*)X, M, N, ld, tpr,
                                                         part);
    NQS_CK_LAUNCH();
    k_colsum_bf16_final<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(part, N, nparts, out);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

static int forward_mixed_tc(nqs_net* net, Scratch& sc, const uint64_t* dets, int64_t M, Fwd& f,
                            bool keep, double* logabs, int8_t* sign, cudaStream_t s) {
    const ProblemDev& P = net->prob->d;
    const int H1 = net->H1, H2 = net->H2, nin = net->nin, nout = net->nout;
    memset(&f, 0, sizeof f);
    f.M = M;
    f.tc = true;
    f.logabs = logabs;
    f.sign = sign;
    f.err = net->prob->err_word;
    NQS_TRY(sc.get((__nv_bfloat16**)&f.H1, M * H1));
    NQS_TRY(sc.get((__nv_bfloat16**)&f.H2, M * H2));
    NQS_TRY(sc.get((float**)&f.Phi, M * nout));
    if (keep) {
        NQS_TRY(sc.get((float**)&f.Ainv_a, M * P.na * P.na));
        NQS_TRY(sc.get((float**)&f.Ainv_b, M * P.nb * P.nb));
    }
    NQS_TRY(sc.get(&f.singular, 1));
    NQS_CK(cudaMemsetAsync(f.singular, 0, sizeof(int), s));
    const ulonglong2* D2 = (const ulonglong2*)dets;
    // layer 1 on the tensor cores: H1 = tanh(X W1^T + b1) with X the 0/1 input matrix (exact
    // in bf16), K = nin padded to a 16-byte row pitch with zero columns on both operands
    const int ldX = (nin + 7) & ~7;
    __nv_bfloat16 *X, *W1p;
    NQS_TRY(sc.get(&X, (size_t)M * ldX));
    NQS_TRY(sc.get(&W1p, (size_t)H1 * ldX));
    {
        ProfScope prof_(PROF_LAYER1, s);
        k_bits_rows<<<grid_for(M * (ldX / 8), 256), 256, 0, s>>>(D2, M, P.norb, ldX, X);
    }
    NQS_CK_LAUNCH();
    k_pad_cols_bf16<<<grid_for((int64_t)H1 * ldX, 256), 256, 0, s>>>(
        (const __nv_bfloat16*)net->p[0], H1, nin, ldX, W1p);
    NQS_CK_LAUNCH();
    f.X = X;
    f.ldX = ldX;
    TcGemm g;
    memset(&g, 0, sizeof g);
    g.err = f.err;
    g.A = X;
    g.lda = ldX;
    g.B = W1p;
    g.ldb = ldX;
    g.M = (int)M;
    g.N = H1;
    g.K = ldX;
    g.epi = EPI_BIAS_TANH;
    g.bias = (const float*)net->p[1];
    g.C = f.H1;
    g.ldc = H1;
    g.c_bf16 = 1;
    NQS_TRY(gemm_bf16_tcgen05(g, sc, s));
    memset(&g, 0, sizeof g);
    g.err = f.err;
    // layer 2: H2 = tanh(H1 W2^T + b2)
    g.A = (const __nv_bfloat16*)f.H1;
    g.lda = H1;
    g.B = (const __nv_bfloat16*)net->p[2];
    g.ldb = H1;
    g.M = (int)M;
    g.N = H2;
    g.K = H1;
    g.epi = EPI_BIAS_TANH;
    g.bias = (const float*)net->p[3];
    g.C = f.H2;
    g.ldc = H2;
    g.c_bf16 = 1;
    NQS_TRY(gemm_bf16_tcgen05(g, sc, s));
    // layer 3: Phi = Phi0 + (H2 W3^T + b3)
    memset(&g, 0, sizeof g);
    g.err = f.err;
    g.A = (const __nv_bfloat16*)f.H2;
    g.lda = H2;
    g.B = (const __nv_bfloat16*)net->p[4];
    g.ldb = H2;
    g.M = (int)M;
    g.N = nout;
    g.K = H2;
    g.epi = EPI_BIAS_PHI0;
    g.bias = (const float*)net->p[5];
    g.phi0 = (const float*)net->p[6];
    g.C = f.Phi;
    g.ldc = nout;
    NQS_TRY(gemm_bf16_tcgen05(g, sc, s));
    double* la2;
    int* ex2;
    int8_t* sg2;
    NQS_TRY(sc.get(&la2, 2 * M));
    NQS_TRY(sc.get(&ex2, 2 * M));
    NQS_TRY(sc.get(&sg2, 2 * M));
    NQS_TRY(launch_lu<float>(net, dets, M, (const float*)f.Phi, la2, ex2, sg2,
                             (float*)f.Ainv_a, (float*)f.Ainv_b, f.singular, s));
    k_combine<<<grid_for(M, 256), 256, 0, s>>>(M, la2, ex2, sg2, logabs, sign);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// dPhi of the mixed form written whole rows at a time: each warp clears a shared-memory copy
// of its configuration's row ([norb][nel] bf16, ldp entries), places w_m (A^-1)_kj at
// [occ_j][col0 + k] of each spin block (the values of k_adjoint), and writes the row out with
// 16-byte stores. No separate clearing pass; the global stores are whole rows.
__global__ void __launch_bounds__(256) k_adjoint_rows(const ulonglong2* __restrict__ dets,
                                                      int64_t M, int norb, int na, int nb,
                                                      const double* __restrict__ w,
                                                      const float* __restrict__ Ainv_a,
                                                      const float* __restrict__ Ainv_b,
                                                      __nv_bfloat16* __restrict__ dPhi,
                                                      int64_t ldp) {
    extern __shared__ __align__(16) uint8_t adj_smem[];
    __shared__ uint8_t occ_s[8][2][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nel = na + nb;
    const int nvec = (int)(ldp / 8);  // 16-byte pieces of a row (ldp is a multiple of 8)
    uint4* rowv = (uint4*)adj_smem + (int64_t)warp * nvec;
    __nv_bfloat16* row = (__nv_bfloat16*)rowv;
    for (int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; m < M;
         m += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const ulonglong2 x = dets[m];
        for (int v = lane; v < nvec; v += 32) rowv[v] = make_uint4(0u, 0u, 0u, 0u);
        for (int p = lane; p < norb; p += 32) {
            const uint64_t below = p == 0 ? 0ull : ((1ull << p) - 1ull);
            if ((x.x >> p) & 1ull) occ_s[warp][0][__popcll(x.x & below)] = (uint8_t)p;
            if ((x.y >> p) & 1ull) occ_s[warp][1][__popcll(x.y & below)] = (uint8_t)p;
        }
        __syncwarp();
        const float wm = (float)w[m];
        for (int spin = 0; spin < 2; ++spin) {
            const int n = spin == 0 ? na : nb, col0 = spin == 0 ? 0 : na;
            const float* inv = spin == 0 ? Ainv_a + m * na * na : Ainv_b + m * nb * nb;
            for (int r = lane; r < n * n; r += 32) {
                const int j = r / n, k = r - j * n;
                const float g = wm * inv[k * n + j];
                row[occ_s[warp][spin][j] * nel + col0 + k] = __float2bfloat16_rn(g);
            }
        }
        __syncwarp();
        uint4* out = (uint4*)(dPhi + m * ldp);
        for (int v = lane; v < nvec; v += 32) out[v] = rowv[v];
        __syncwarp();
    }
}

static int backward_mixed_tc(nqs_net* net, Scratch& sc, const uint64_t* dets, const Fwd& f,
                             const double* w, void* grad, cudaStream_t s) {
    const ProblemDev& P = net->prob->d;
    const int64_t M = f.M;
    const int H1 = net->H1, H2 = net->H2, nin = net->nin, nout = net->nout;
    const int64_t ldP = (nout + 7) & ~7;
    float* G = (float*)grad;
    float* gW1 = G;
    float* gb1 = gW1 + (size_t)H1 * nin;
    float* gW2 = gb1 + H1;
    float* gb2 = gW2 + (size_t)H2 * H1;
    float* gW3 = gb2 + H2;
    float* gb3 = gW3 + (size_t)nout * H2;
    __nv_bfloat16 *dPhi, *W3T, *W2T, *dZ2, *dZ1;
    NQS_TRY(sc.get(&dPhi, M * ldP));
    NQS_TRY(sc.get(&W3T, (size_t)H2 * ldP));
    NQS_TRY(sc.get(&W2T, (size_t)H1 * H2));
    NQS_TRY(sc.get(&dZ2, M * H2));
    NQS_TRY(sc.get(&dZ1, M * H1));
    const size_t adj_smem = (size_t)8 * ldP * 2;  // one dPhi row per warp
    if (adj_smem <= 48 * 1024) {
        k_adjoint_rows<<<grid_for(M * 32, 256, 148 * 64), 256, adj_smem, s>>>(
            (const ulonglong2*)dets, M, P.norb, P.na, P.nb, w, (const float*)f.Ainv_a,
            (const float*)f.Ainv_b, dPhi, ldP);
    } else {
        NQS_CK(cudaMemsetAsync(dPhi, 0, M * ldP * 2, s));
        k_adjoint<float, __nv_bfloat16><<<grid_for(M * 32, 256, 148 * 64), 256, 0, s>>>(
            (const ulonglong2*)dets, M, P.norb, P.na, P.nb, w, (const float*)f.Ainv_a,
            (const float*)f.Ainv_b, dPhi, ldP);
    }
    NQS_CK_LAUNCH();
    NQS_TRY(transpose_bf16(net->p[4], nout, H2, H2, W3T, ldP, s));  // W3 [nout][H2] -> [H2][nout]
    NQS_TRY(transpose_bf16(net->p[2], H2, H1, H1, W2T, H2, s));     // W2 [H2][H1] -> [H1][H2]
    TcGemm g;
    // dZ2 = (dPhi W3) * (1 - H2^2)
    memset(&g, 0, sizeof g);
    g.err = f.err;
    g.A = dPhi;
    g.lda = ldP;
    g.B = W3T;
    g.ldb = ldP;
    g.M = (int)M;
    g.N = H2;
    g.K = nout;
    g.epi = EPI_TANH_BWD;
    g.aux = (const __nv_bfloat16*)f.H2;
    g.ld_aux = H2;
    g.C = dZ2;
    g.ldc = H2;
    g.c_bf16 = 1;
    NQS_TRY(gemm_bf16_tcgen05(g, sc, s));
    // dZ1 = (dZ2 W2) * (1 - H1^2)
    memset(&g, 0, sizeof g);
    g.err = f.err;
    g.A = dZ2;
    g.lda = H2;
    g.B = W2T;
    g.ldb = H2;
    g.M = (int)M;
    g.N = H1;
    g.K = H2;
    g.epi = EPI_TANH_BWD;
    g.aux = (const __nv_bfloat16*)f.H1;
    g.ld_aux = H1;
    g.C = dZ1;
    g.ldc = H1;
    g.c_bf16 = 1;
    NQS_TRY(gemm_bf16_tcgen05(g, sc, s));
    // weight gradients dW = dZ^T H: reductions over |S| (K = M) with both operands read
    // row-major ([M][ld], MN-major), split across CTAs
    auto wgrad = [&](const __nv_bfloat16* dZ, int64_t ldz, int rows, const __nv_bfloat16* Hm,
                     int64_t ldh, int cols, float* out) -> int {
        TcGemm q;
        memset(&q, 0, sizeof q);
        q.err = f.err;
        q.A = dZ;
        q.lda = ldz;
        q.a_mn = 1;
        q.B = Hm;
        q.ldb = ldh;
        q.b_mn = 1;
        q.M = rows;
        q.N = cols;
        q.K = (int)M;
        q.epi = EPI_STORE;
        q.C = out;
        q.ldc = cols;
        return gemm_bf16_tcgen05(q, sc, s);
    };
    NQS_TRY(wgrad(dPhi, ldP, nout, (const __nv_bfloat16*)f.H2, H2, H2, gW3));
    NQS_TRY(wgrad(dZ2, H2, H2, (const __nv_bfloat16*)f.H1, H1, H1, gW2));
    NQS_TRY(wgrad(dZ1, H1, H1, (const __nv_bfloat16*)f.X, f.ldX, nin, gW1));
    NQS_TRY(colsum_bf16(sc, dPhi, M, nout, ldP, gb3, s));
    NQS_TRY(colsum_bf16(sc, dZ2, M, H2, H2, gb2, s));
    NQS_TRY(colsum_bf16(sc, dZ1, M, H1, H1, gb1, s));
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// Batched problems: one launch per stage over all problems (blockIdx.y = problem). The
// arithmetic of each stage is that of the single-problem kernels above.
// ------------------------------------------------------------------------------------------
// X [M][ldX] (bf16 0/1, zero pad columns) and its transpose XT [nin][ldM]; W1p = W1 padded to
// ldX columns; W2T = W2^T [H1][H2]; W3T = W3^T [H2][ldP] (blockIdx.z: 0 bits, 1 W1p, 2 W2T,
// 3 W3T)
__global__ void k_g_bits_prep(const GProb* __restrict__ Pv) {
    const GProb& P = Pv[blockIdx.y];
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const uint16_t one = 0x3F80u;  // bf16 1.0
    if (blockIdx.z == 0) {
        const int per = P.ldX / 8;
        for (int64_t t = t0; t < P.M * per; t += step) {
            const int64_t m = t / per;
            const int c0 = (int)(t - m * per) * 8;
            const ulonglong2 x = P.dets[m];
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t v = 0;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = c0 + 2 * k + h;
                    uint32_t bit = 0;
                    if (c < P.norb) bit = (uint32_t)(x.x >> c) & 1u;
                    else if (c < P.nin) bit = (uint32_t)(x.y >> (c - P.norb)) & 1u;
                    v |= (bit ? (uint32_t)one : 0u) << (16 * h);
                    if (c < P.nin) ((uint16_t*)P.XT)[(int64_t)c * P.ldM + m] = bit ? one : 0;
                }
                w[k] = v;
            }
            *(uint4*)(P.X + m * P.ldX + c0) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else if (blockIdx.z == 1) {
        for (int64_t t = t0; t < (int64_t)P.H1 * P.ldX; t += step) {
            const int r = (int)(t / P.ldX), c = (int)(t - (int64_t)r * P.ldX);
            P.W1p[t] = c < P.nin ? P.W1[(int64_t)r * P.nin + c] : __float2bfloat16_rn(0.f);
        }
    } else if (blockIdx.z == 2) {
        for (int64_t t = t0; t < (int64_t)P.H1 * P.H2; t += step) {
            const int r = (int)(t / P.H2), c = (int)(t - (int64_t)r * P.H2);  // W2T[r][c]
            P.W2T[t] = P.W2[(int64_t)c * P.H1 + r];
        }
    } else {
        for (int64_t t = t0; t < (int64_t)P.H2 * P.ldP; t += step) {
            const int r = (int)(t / P.ldP), c = (int)(t - (int64_t)r * P.ldP);  // W3T[r][c]
            if (c < P.nout) P.W3T[t] = P.W3[(int64_t)c * P.H2 + r];
        }
    }
}

int g_bits_prep(const GProb* P, const GDims& d, cudaStream_t s) {
    const int64_t work = d.maxMX > (int64_t)d.max_H * d.max_H ? d.maxMX : (int64_t)d.max_H * d.max_H;
    k_g_bits_prep<<<dim3(grid_for(work, 256, 256), d.np, 4), 256, 0, s>>>(P);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

template <int N>
static int g_lu_n(const GLuJob* jobs, int njobs, int64_t maxM, cudaStream_t s) {
    k_g_lu<N><<<dim3(grid_for(maxM, 128, 256), njobs), 128, 0, s>>>(jobs);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int g_lu(const GLuJob* jobs, int njobs, int n, int64_t maxM, cudaStream_t s) {
    ProfScope prof_(PROF_LU, s);
    switch (n) {
#define NQS_GLU(K) \
    case K: return g_lu_n<K>(jobs, njobs, maxM, s);
        NQS_GLU(1) NQS_GLU(2) NQS_GLU(3) NQS_GLU(4) NQS_GLU(5) NQS_GLU(6) NQS_GLU(7) NQS_GLU(8)
        NQS_GLU(9) NQS_GLU(10) NQS_GLU(11) NQS_GLU(12)
#undef NQS_GLU
        default: return NQS_ERR_UNSUPPORTED;
    }
}

__global__ void k_g_combine(const GProb* __restrict__ Pv) {
    const GProb& P = Pv[blockIdx.y];
    const int64_t M = P.M;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const int sg = P.sg2[m] * P.sg2[M + m];
        P.sign[m] = (int8_t)sg;
        P.logabs[m] = sg == 0 ? -INFINITY
                              : log(P.la2[m] * P.la2[M + m]) +
                                    (double)(P.ex2[m] + P.ex2[M + m]) * M_LN2;
    }
}

int g_combine(const GProb* P, const GDims& d, cudaStream_t s) {
    k_g_combine<<<dim3(grid_for(d.maxM, 256, 256), d.np), 256, 0, s>>>(P);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// dPhi rows: zero, then w_m (A^-1)_kj at [occ_j][col0 + k] of each spin block (as k_adjoint)
__global__ void __launch_bounds__(256) k_g_adjoint(const GProb* __restrict__ Pv) {
    const GProb& P = Pv[blockIdx.y];
    __shared__ uint8_t occ_s[8][2][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nel = P.na + P.nb;
    for (int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; m < P.M;
         m += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const ulonglong2 x = P.dets[m];
        __nv_bfloat16* row = P.dPhi + m * P.ldP;
        for (int c = lane; c < P.ldP; c += 32) row[c] = __float2bfloat16_rn(0.f);
        for (int p = lane; p < P.norb; p += 32) {
            const uint64_t below = p == 0 ? 0ull : ((1ull << p) - 1ull);
            if ((x.x >> p) & 1ull) occ_s[warp][0][__popcll(x.x & below)] = (uint8_t)p;
            if ((x.y >> p) & 1ull) occ_s[warp][1][__popcll(x.y & below)] = (uint8_t)p;
        }
        __syncwarp();
        const float wm = (float)P.w[m];
        for (int spin = 0; spin < 2; ++spin) {
            const int n = spin == 0 ? P.na : P.nb, col0 = spin == 0 ? 0 : P.na;
            const float* inv = spin == 0 ? P.Ainv_a + m * n * n : P.Ainv_b + m * n * n;
            for (int r = lane; r < n * n; r += 32) {
                const int j = r / n, k = r - j * n;
                const float g = wm * inv[k * n + j];
                row[(int64_t)occ_s[warp][spin][j] * nel + col0 + k] = __float2bfloat16_rn(g);
            }
        }
        __syncwarp();
    }
}

int g_adjoint(const GProb* P, const GDims& d, cudaStream_t s) {
    k_g_adjoint<<<dim3(grid_for(d.maxM * 32, 256, 512), d.np), 256, 0, s>>>(P);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// dPhiT [nout][ldM] = dPhi^T, 32 x 32 tiles through shared memory, one block per tile over the
// work list of every problem's tiles (tile_off: prefix of ceil(M/32) ceil(nout/32) per problem)
__global__ void k_g_transpose_dphi(const GProb* __restrict__ Pv, const int64_t* __restrict__ tile_off,
                                   int np) {
    __shared__ unsigned short tile[32][33];
    const int64_t t = blockIdx.x;
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const GProb& P = Pv[lo];
    const int64_t local = t - tile_off[lo];
    const int64_t tc = (P.nout + 31) / 32;
    const int64_t r0 = (local / tc) * 32, c0 = (local % tc) * 32;
    const unsigned short* S = (const unsigned short*)P.dPhi;
    unsigned short* D = (unsigned short*)P.dPhiT;
    const int64_t R = P.M, Cn = P.nout;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < R && c < Cn) ? S[r * P.ldP + c] : (unsigned short)0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (c < Cn && r < R) D[c * P.ldM + r] = tile[threadIdx.x][i];
    }
}

int g_transpose_dphi(const GProb* P, const GDims& d, const int64_t* tile_off, int64_t tiles,
                     cudaStream_t s) {
    k_g_transpose_dphi<<<(unsigned)tiles, dim3(32, 8), 0, s>>>(P, tile_off, d.np);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// bias gradients: the row sums of dPhiT (db3), dZ2T (db2) and dZ1T (db1) over the first M
// columns, FP32 in a fixed order (chunks of ROWSUM_CHUNK entries reduced by a fixed tree, the
// chunk sums added in order). blockIdx.x = row, blockIdx.y = problem, blockIdx.z = which matrix.
__global__ void __launch_bounds__(256) k_g_bias_grads(const GProb* __restrict__ Pv) {
    const GProb& P = Pv[blockIdx.y];
    if (!P.grad) return;
    const int which = blockIdx.z;
    const int R = which == 0 ? P.nout : (which == 1 ? P.H2 : P.H1);
    const int r = blockIdx.x;
    if (r >= R) return;
    const __nv_bfloat16* X = which == 0 ? P.dPhiT : (which == 1 ? P.dZ2T : P.dZ1T);
    float* gb1 = P.grad + (size_t)P.H1 * P.nin;
    float* gb2 = gb1 + P.H1 + (size_t)P.H2 * P.H1;
    float* gb3 = gb2 + P.H2 + (size_t)P.nout * P.H2;
    float* out = which == 0 ? gb3 : (which == 1 ? gb2 : gb1);
    __shared__ float red[8];
    const __nv_bfloat16* row = X + (int64_t)r * P.ldM;
    const int64_t M = P.M, ld = P.ldM;
    float total = 0.f;
    for (int64_t c0 = 0; c0 < M; c0 += ROWSUM_CHUNK) {
        const int64_t c1 = c0 + ROWSUM_CHUNK < M ? c0 + ROWSUM_CHUNK : M;
        float acc = 0.f;
        if ((ld % 8) == 0) {
            const int64_t v1 = c0 + ((c1 - c0) & ~(int64_t)7);
            for (int64_t i = c0 + 8 * threadIdx.x; i < v1; i += 8 * 256) {
                const uint4 pk = *(const uint4*)(row + i);
                const __nv_bfloat162* h2 = (const __nv_bfloat162*)&pk;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float2 f = __bfloat1622float2(h2[t]);
                    acc += f.x + f.y;
                }
            }
            for (int64_t i = v1 + threadIdx.x; i < c1; i += 256) acc += __bfloat162float(row[i]);
        } else {
            for (int64_t i = c0 + threadIdx.x; i < c1; i += 256) acc += __bfloat162float(row[i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int k = 0; k < 8; ++k) t += red[k];
            total += t;
        }
    }
    if (threadIdx.x == 0) out[r] = total;
}

int g_bias_grads(const GProb* P, const GDims& d, cudaStream_t s) {
    const int R = d.max_nout > d.max_H ? d.max_nout : d.max_H;
    k_g_bias_grads<<<dim3((unsigned)R, d.np, 3), 256, 0, s>>>(P);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

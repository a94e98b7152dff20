// BF16 tensor-core GEMM for the dense backflow layers on sm_103a (5th-generation tensor cores):
//   C[m][n] = epilogue( sum_k A[m][k] * B[n][k] ),  A, B bfloat16, each operand K-major
//   (k contiguous) or MN-major (m or n contiguous: the row-major activations a weight gradient
//   reduces over), FP32 accumulation in tensor memory.
//
// Two kernels. k_gemm_tc (below) runs 64- and 128-column tiles on single SMs; k_gemm_tc_pair
// runs 256-column tiles on clusters of two SMs sharing one M = 256 MMA stream (cta_group::2),
// each SM staging its own rows of A and half of B; its roles are those described here.
//
// Persistent kernel, one CTA per SM, work units (128 x BN output tiles, times the K splits)
// dealt round-robin; ten warps:
//   warp 0 / lane 0  TMA producer: 128x64 (A) and BNx64 (B) tiles, 128-byte swizzle, into a
//                    shared-memory ring of up to 8 stages guarded by mbarriers (full / empty);
//   warp 1 / lane 0  MMA issuer: tcgen05.mma.cta_group::1.kind::f16 (M=128, N=BN, K=16) x 4 per
//                    stage into one of two TMEM accumulators; tcgen05.commit frees the stage
//                    and, after the last stage of a tile, hands the accumulator over;
//   warps 2..9       epilogue: tcgen05.ld (32 lanes x 32 columns per load; warp w reads TMEM
//                    lanes 32 (w % 4).. = tile rows, and one half of the columns), fused bias /
//                    tanh / Phi0 / tanh' epilogues, row-major and (optionally) transposed
//                    stores, then frees the accumulator. The epilogue of one tile overlaps the
//                    main loop of the next.
// Split-K writes FP32 partials that a second kernel sums in a fixed order.
// Every mbarrier wait is bounded (about 2 s of clock); a timeout raises a CTA-wide abort flag
// that ends every role's loop, the producer still waits for its copies in flight, the error
// word is set and the tensor memory is released.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "ansatz.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

#define TC_EPI_WARPS 8
#define TC_THREADS (32 * (2 + TC_EPI_WARPS))
#define TC_BK 64  // bf16 elements per 128-byte swizzle row

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024u >> 4) << 32;           // stride byte offset
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // swizzle: 128 B
    return d;
}

// shared-memory matrix descriptor: MN-major operand, 128-byte swizzle; the tile is a row of
// 64-element (128-byte) MN atoms 8 KB apart (leading byte offset), each 64 k-rows of 128 bytes
// with 8-row groups 1024 B apart (stride byte offset)
__device__ __forceinline__ uint64_t sdesc_sw128_mn(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(8192u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both operands K-major (bits 15 / 16
// select MN-major A / B)
template <int BN>
__device__ __forceinline__ uint32_t idesc_bf16() {
    return (1u << 4)            // D format: F32
           | (1u << 7)          // A format: BF16
           | (1u << 10)         // B format: BF16
           | ((uint32_t)(BN >> 3) << 17)   // N / 8
           | ((uint32_t)(128 >> 4) << 24); // M / 16
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// the same load without the wait: the registers are valid only after tmem_wait_ld(r), whose
// read-write operands keep every use of r behind the wait
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]),
                   "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]),
                   "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

struct TcArgs {
    int M, N, K;
    int epi;                 // EPI_* (ansatz.cuh)
    void* C;                 // [M][ldc] (bf16 if c_bf16 else float), may be null
    int64_t ldc;
    int c_bf16;
    __nv_bfloat16* CT;       // [N][ldct] transposed bf16 copy, may be null
    int64_t ldct;
    const float* bias;       // [N]
    const float* phi0;       // [N]
    const __nv_bfloat16* aux;  // [M][ld_aux] activation for tanh'
    int64_t ld_aux;
    float* partial;          // split-K partials [splits][M][N]
    int splits;
    int tma_c, tma_ct, tma_p;  // stores go through the tensor maps below (else direct)
    int* err;
    int a_mn, b_mn;          // MN-major operands (TcGemm)
};

// The operand copies of k-block kb into one stage: K-major, one box of 64 k x rows; MN-major,
// boxes of 64 (m or n) x 64 k-rows, 8 KB apart. `bar` is a shared::cluster address; pair
// selects the .cta_group::2 form (the barrier may sit in the other CTA of the pair).
__device__ __forceinline__ void tma_load_any(bool pair, void* dst, const CUtensorMap* map,
                                             uint32_t bar, int x, int y) {
    if (pair)
        asm volatile(
            "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::"
            "bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
            "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
            "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
            : "memory");
}
__device__ __forceinline__ void load_operand(bool pair, bool mn, uint8_t* dst,
                                             const CUtensorMap* map, uint32_t bar, int kb,
                                             int row0, int rows) {
    if (!mn) {
        tma_load_any(pair, dst, map, bar, kb * TC_BK, row0);
    } else {
        for (int j = 0; j < rows / 64; ++j)
            tma_load_any(pair, dst + j * 8192, map, bar, row0 + 64 * j, kb * TC_BK);
    }
}
// descriptor of the operand at saddr and its advance per K = 16 step
__device__ __forceinline__ uint64_t operand_desc(bool mn, uint32_t saddr) {
    return mn ? sdesc_sw128_mn(saddr) : sdesc_sw128(saddr);
}
__device__ __forceinline__ uint64_t operand_step(bool mn) {
    return mn ? (uint64_t)(2048u >> 4) : (uint64_t)2;  // 16 k-rows of 128 B, or 32 B in the row
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
            (uint64_t)map),
        "r"(smem_u32(src)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y,
                                             int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            (uint64_t)map),
        "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read0() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// The epilogue of 32 accumulator columns [nb, nb + 32) of the 32 tile rows of one warp, staged
// in the warp's 4 KB shared-memory buffer and written by TMA stores (the hardware clips rows
// >= M and columns >= N): the row-major output (bf16 or FP32), the transposed bf16 copy, or the
// FP32 split-K partial. Row-contiguous operands of the epilogue (tanh' activations) are read
// with 16-byte loads.
template <class U>
__device__ __forceinline__ void epilogue32_tma(const TcArgs& a, const U& w, int row, bool row_ok,
                                               int nb, int rowbase, const uint32_t (&r)[32],
                                               uint8_t* stage, const CUtensorMap* mapC,
                                               const CUtensorMap* mapCT, const CUtensorMap* mapP) {
    const int lane = threadIdx.x & 31;
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
    if (a.splits <= 1 && row_ok) {
        if (a.epi == EPI_BIAS_TANH) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (nb + j < a.N) v[j] = tanhf(v[j] + a.bias[nb + j]);
        } else if (a.epi == EPI_BIAS_PHI0) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (nb + j < a.N) {
                    const float z = v[j] + a.bias[nb + j];
                    v[j] = a.phi0[nb + j] + z;
                }
        } else if (a.epi == EPI_TANH_BWD) {
            const __nv_bfloat16* hrow = a.aux + (size_t)row * a.ld_aux + nb;
            if (nb + 32 <= a.N && (a.ld_aux % 8) == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 pk = *(const uint4*)(hrow + 8 * q);
                    const __nv_bfloat162* h2 = (const __nv_bfloat162*)&pk;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float2 hf = __bfloat1622float2(h2[t]);
                        v[8 * q + 2 * t] *= 1.0f - hf.x * hf.x;
                        v[8 * q + 2 * t + 1] *= 1.0f - hf.y * hf.y;
                    }
                }
            } else {
                for (int j = 0; j < 32; ++j)
                    if (nb + j < a.N) {
                        const float h = __bfloat162float(hrow[j]);
                        v[j] *= 1.0f - h * h;
                    }
            }
        }
    }
    const bool f32 = a.splits > 1 || !a.c_bf16;
    const bool do_c = a.splits > 1 || a.C;
    // the stores issued from this buffer by the previous chunk must have read it; waiting only
    // now lets that read overlap this chunk's accumulator load and epilogue arithmetic
    if (lane == 0) bulk_wait_read0();
    __syncwarp();
    // The staging rows are written in the layout of the store map's swizzle (128-byte swizzle
    // for 128-byte FP32 rows, 64-byte swizzle for 64-byte bf16 rows: the 16-byte chunk index is
    // XORed with address bits 7.. of the row), so the 16-byte stores of the eight lanes of a
    // quarter-warp fall in eight different bank groups instead of one or two.
    if (do_c) {
        if (f32) {
            float4* dst = (float4*)(stage + lane * 128);
            const int sw = lane & 7;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                dst[q ^ sw] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
            uint4* dst = (uint4*)(stage + lane * 64);
            const int sw = (lane >> 1) & 3;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 pk;
                uint32_t* wd = (uint32_t*)&pk;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(v[q * 8 + 2 * t], v[q * 8 + 2 * t + 1]);
                    wd[t] = *(uint32_t*)&h2;
                }
                dst[q ^ sw] = pk;
            }
        }
    }
    uint16_t* stT = (uint16_t*)(stage + 2048);
    if (a.CT) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            __nv_bfloat16 hv = __float2bfloat16_rn(v[j]);
            stT[j * 32 + lane] = *(uint16_t*)&hv;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
        if (a.splits > 1) tma_store_3d(mapP, stage, nb, rowbase, w.z);
        else if (a.C) tma_store_2d(mapC, stage, nb, rowbase);
        if (a.CT) tma_store_2d(mapCT, stT, rowbase, nb);
        bulk_commit();
    }
    __syncwarp();
}

// The epilogue of 32 accumulator columns [nb, nb + 32) of one tile row: fused bias / tanh /
// Phi0 / tanh' and row-major (optionally transposed) stores, or the FP32 split-K partial.
template <class U>
__device__ __forceinline__ void epilogue32(const TcArgs& a, const U& w, int row, bool row_ok,
                                           int nb, const uint32_t (&r)[32]) {
    if (a.splits > 1) {
        float* P = a.partial + (size_t)w.z * a.M * a.N;
        if (row_ok)
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (nb + j < a.N) P[(size_t)row * a.N + nb + j] = __uint_as_float(r[j]);
        return;
    }
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int n = nb + j;
        float x = __uint_as_float(r[j]);
        if (n < a.N && row_ok) {
            if (a.epi == EPI_BIAS_TANH) {
                x = tanhf(x + a.bias[n]);
            } else if (a.epi == EPI_BIAS_PHI0) {
                float z = x + a.bias[n];
                x = a.phi0[n] + z;
            } else if (a.epi == EPI_TANH_BWD) {
                float h = __bfloat162float(a.aux[(size_t)row * a.ld_aux + n]);
                x = x * (1.0f - h * h);
            }
        }
        v[j] = x;
    }
    if (row_ok && a.C) {
        if (a.c_bf16) {
            __nv_bfloat16* C = (__nv_bfloat16*)a.C + (size_t)row * a.ldc;
            if (nb + 32 <= a.N && (a.ldc % 8) == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint4 pk;
                    uint32_t* wd = (uint32_t*)&pk;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[q * 8 + 2 * t],
                                                                  v[q * 8 + 2 * t + 1]);
                        wd[t] = *(uint32_t*)&h2;
                    }
                    *(uint4*)(C + nb + q * 8) = pk;
                }
            } else {
                for (int j = 0; j < 32; ++j)
                    if (nb + j < a.N) C[nb + j] = __float2bfloat16_rn(v[j]);
            }
        } else {
            float* C = (float*)a.C + (size_t)row * a.ldc;
            if (nb + 32 <= a.N && (a.ldc % 4) == 0) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *(float4*)(C + nb + q * 4) =
                        make_float4(v[q * 4], v[q * 4 + 1], v[q * 4 + 2], v[q * 4 + 3]);
            } else {
                for (int j = 0; j < 32; ++j)
                    if (nb + j < a.N) C[nb + j] = v[j];
            }
        }
    }
    if (row_ok && a.CT) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (nb + j < a.N) a.CT[(size_t)(nb + j) * a.ldct + row] = __float2bfloat16_rn(v[j]);
    }
}

template <int BN>
struct TcSmem {
    static constexpr int A_BYTES = 128 * TC_BK * 2;
    static constexpr int B_BYTES = BN * TC_BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = (200 * 1024) / STAGE < 8 ? (200 * 1024) / STAGE : 8;
    static constexpr int EPI = TC_EPI_WARPS * 4096;  // per-warp epilogue staging
    static constexpr int BYTES = STAGES * STAGE + EPI + 1024 /*align*/ + 256 /*barriers*/;
};

// shared memory of one CTA (227 KB opt-in limit); barriers: full and empty per stage, two
// accumulator-full and two accumulator-empty, then the TMEM address slot and the abort flag
static_assert(TcSmem<64>::BYTES <= 232448 && TcSmem<128>::BYTES <= 232448 &&
                  TcSmem<256>::BYTES <= 232448,
              "single-SM GEMM shared memory");
static_assert((2 * TcSmem<64>::STAGES + 4) * 8 + 8 <= 256, "single-SM GEMM barrier block");

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait that also gives up as soon as another role of the CTA has aborted; `limit` SM
// clocks (about 2 s by default)
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort,
                                             long long limit = 4000000000ll) {
    const uint32_t addr = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            return false;
        }
    }
}

// One work unit = (split z, row tile, column tile); units are dealt round-robin to the
// persistent CTAs, column tile fastest so that CTAs running together share the A rows in L2.
struct Unit {
    int m0, n0, kb0, nk, z;
};
__device__ __forceinline__ Unit unit_of(int u, const TcArgs& a, int BN) {
    const int ntn = (a.N + BN - 1) / BN, ntm = (a.M + 127) / 128;
    const int tiles = ntn * ntm;
    const int z = u / tiles, t = u - z * tiles;
    const int nkb = (a.K + TC_BK - 1) / TC_BK;
    const int per = (nkb + a.splits - 1) / a.splits;
    Unit r;
    r.z = z;
    r.m0 = (t / ntn) * 128;
    r.n0 = (t % ntn) * BN;
    r.kb0 = z * per;
    r.nk = max(0, min(nkb, r.kb0 + per) - r.kb0);
    return r;
}

// Persistent, warp-specialised: warp 0 lane 0 issues TMA, warp 1 lane 0 issues tcgen05.mma into
// one of two TMEM accumulators (2 x BN columns), warps 2..9 drain the other accumulator
// through the epilogue meanwhile (warp w reads TMEM lanes 32 (w % 4).., half (w - 2) / 4 of the
// columns). Barriers: full/empty per shared-memory stage, tfull/tempty per accumulator.
template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmCT,
              const __grid_constant__ CUtensorMap tmP, TcArgs a) {
    using L = TcSmem<BN>;
    constexpr int ST = L::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* epi_stage = smem + ST * L::STAGE;
    uint64_t* full = (uint64_t*)(smem + ST * L::STAGE + L::EPI);
    uint64_t* empty = full + ST;
    uint64_t* tfull = empty + ST;
    uint64_t* tempty = tfull + 2;
    uint32_t* tslot = (uint32_t*)(tempty + 2);
    volatile int* abort = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int units = ((a.N + BN - 1) / BN) * ((a.M + 127) / 128) * a.splits;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], TC_EPI_WARPS);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(tslot)),
            "r"((uint32_t)(2 * BN)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        uint32_t it = 0;
        for (int u = blockIdx.x; u < units && !*abort; u += gridDim.x) {
            const Unit w = unit_of(u, a, BN);
            for (int i = 0; i < w.nk; ++i, ++it) {
                const int s = it % ST;
                const uint32_t ph = (it / ST) & 1u;
                if (it >= (uint32_t)ST && !mbar_wait_ab(&empty[s], ph ^ 1u, abort)) break;
                uint8_t* st = smem + s * L::STAGE;
                mbar_expect_tx(&full[s], (uint32_t)L::STAGE);
                const uint32_t fb = smem_u32(&full[s]);
                load_operand(false, a.a_mn, st, &tmA, fb, w.kb0 + i, w.m0, 128);
                load_operand(false, a.b_mn, st + L::A_BYTES, &tmB, fb, w.kb0 + i, w.n0, BN);
            }
        }
        // never leave with copies in flight: wait (bounded) for the last load of each stage
        const uint32_t last = it;
        for (uint32_t j = last > (uint32_t)ST ? last - ST : 0; j < last; ++j) {
            volatile int no_abort = 0;
            mbar_wait_ab(&full[j % ST], (j / ST) & 1u, &no_abort);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc =
            idesc_bf16<BN>() | ((uint32_t)a.a_mn << 15) | ((uint32_t)a.b_mn << 16);
        const uint64_t sa = operand_step(a.a_mn), sb = operand_step(a.b_mn);
        uint32_t it = 0, j = 0;
        for (int u = blockIdx.x; u < units && !*abort; u += gridDim.x, ++j) {
            const Unit w = unit_of(u, a, BN);
            const uint32_t b = j & 1u, use = j >> 1;
            if (use > 0 && !mbar_wait_ab(&tempty[b], (use - 1) & 1u, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + b * BN;
            bool ok = true;
            for (int i = 0; i < w.nk; ++i, ++it) {
                const int s = it % ST;
                if (!mbar_wait_ab(&full[s], (it / ST) & 1u, abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint8_t* st = smem + s * L::STAGE;
                const uint64_t da = operand_desc(a.a_mn, smem_u32(st));
                const uint64_t db = operand_desc(a.b_mn, smem_u32(st + L::A_BYTES));
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk)
                    umma(acc, da + sa * kk, db + sb * kk, idesc, (i | kk) != 0 ? 1u : 0u);
                umma_commit(&empty[s]);
            }
            if (!ok) break;
            umma_commit(&tfull[b]);
        }
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3, half = (warp - 2) >> 2;
        const int c_lo = half * (BN / 2), c_hi = c_lo + BN / 2;
        uint32_t j = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++j) {
            const Unit w = unit_of(u, a, BN);
            const uint32_t b = j & 1u, use = j >> 1;
            if (!mbar_wait_ab(&tfull[b], use & 1u, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = w.m0 + q * 32 + lane;
            const bool row_ok = row < a.M;
#pragma unroll 1
            for (int c = c_lo; c < c_hi; c += 32) {
                uint32_t r[32];
                if (w.nk > 0) {
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * BN + (uint32_t)c, r);
                } else {
#pragma unroll
                    for (int t = 0; t < 32; ++t) r[t] = 0u;
                }
                if (a.tma_c)
                    epilogue32_tma(a, w, row, row_ok, w.n0 + c, w.m0 + q * 32, r,
                                   epi_stage + (warp - 2) * 4096, &tmC, &tmCT, &tmP);
                else
                    epilogue32(a, w, row, row_ok, w.n0 + c, r);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        if (a.tma_c && lane == 0) bulk_wait0();  // every store of this warp has landed
    }
    if (*abort && a.err) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)(2 * BN)));
}

// ------------------------------------------------------------------------------------------
// Paired form (tcgen05 cta_group::2): a cluster of two CTAs on two SMs computes a 256 x BN
// output tile with one MMA stream of M = 256 issued by the even CTA. Each CTA stages its own
// 128 rows of A and one half (BN/2 rows) of B, so an SM moves A + B/2 per k-block instead of
// A + B, and its tensor memory receives the accumulator rows of its own A rows (all BN
// columns), which its epilogue warps drain exactly as in k_gemm_tc.
// Barriers: the even CTA's full[s] counts the transaction bytes of both CTAs' copies (the odd
// CTA's copies signal it through the .cta_group::2 form of the load); the MMA's commits
// arrive on empty[s] and tfull[b] of both CTAs (multicast); the epilogue warps of both CTAs
// arrive on the even CTA's tempty[b]. A timeout in either CTA raises the abort flag of both.
// ------------------------------------------------------------------------------------------
template <int BN>
struct TcSmem2 {
    static constexpr int A_BYTES = 128 * TC_BK * 2;
    static constexpr int B_BYTES = (BN / 2) * TC_BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    // one 4 KB staging buffer per epilogue warp: a second one would cost a pipeline stage at
    // BN = 256, and the deeper operand pipeline is worth more (1354 against 1193 TFLOP/s on
    // 2^20 x 2016 x 1024 with 6 stages and one buffer, against 5 stages and two)
    static constexpr int EPI = TC_EPI_WARPS * 4096;
    static constexpr int ROOM = 232448 - 1024 /*align*/ - 256 /*barriers*/ - EPI;
    static constexpr int STAGES = ROOM / STAGE < 8 ? ROOM / STAGE : 8;
    static constexpr int BYTES = STAGES * STAGE + EPI + 1024 + 256;
};

// as TcSmem, plus the drain barrier of the MMA issuer
static_assert(TcSmem2<256>::BYTES <= 232448, "paired GEMM shared memory");
static_assert((2 * TcSmem2<256>::STAGES + 5) * 8 + 8 <= 256, "paired GEMM barrier block");

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_idx() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// address of the same shared-memory variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t smem_in_cta(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
                 : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

// bounded wait as mbar_wait_ab; acquire at cluster scope (arrivals from the other CTA), and a
// timeout also raises the other CTA's abort flag
__device__ __forceinline__ bool mbar_wait_pair(uint64_t* bar, uint32_t parity, volatile int* abort,
                                               uint32_t peer_abort) {
    const uint32_t addr = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort) return false;
        if (clock64() - t0 > 4000000000ll) {
            *abort = 1;
            st_cluster_u32(peer_abort, 1u);
            return false;
        }
    }
}

template <int BN>
__device__ __forceinline__ uint32_t idesc_bf16_m256() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(256 >> 4) << 24);
}

__device__ __forceinline__ void umma_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// commit of the MMAs issued so far, arriving on the barrier at this offset in the CTAs of mask
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(smem_u32(bar)),
        "h"(mask)
        : "memory");
}

// one work unit of the paired form: (split z, 256-row tile, BN-column tile)
__device__ __forceinline__ Unit unit_of_pair(int u, const TcArgs& a, int BN) {
    const int ntn = (a.N + BN - 1) / BN, ntm = (a.M + 255) / 256;
    const int tiles = ntn * ntm;
    const int z = u / tiles, t = u - z * tiles;
    const int nkb = (a.K + TC_BK - 1) / TC_BK;
    const int per = (nkb + a.splits - 1) / a.splits;
    Unit r;
    r.z = z;
    r.m0 = (t / ntn) * 256;
    r.n0 = (t % ntn) * BN;
    r.kb0 = z * per;
    r.nk = max(0, min(nkb, r.kb0 + per) - r.kb0);
    return r;
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC,
                   const __grid_constant__ CUtensorMap tmCT,
                   const __grid_constant__ CUtensorMap tmP, TcArgs a) {
    using L = TcSmem2<BN>;
    constexpr int ST = L::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* epi_stage = smem + ST * L::STAGE;
    uint64_t* full = (uint64_t*)(smem + ST * L::STAGE + L::EPI);
    uint64_t* empty = full + ST;
    uint64_t* tfull = empty + ST;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tslot = (uint32_t*)(drain + 1);
    volatile int* abort = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const int cid = (int)cluster_idx(), ncl = (int)cluster_count();
    const int units = ((a.N + BN - 1) / BN) * ((a.M + 255) / 256) * a.splits;
    const uint32_t peer_abort = smem_in_cta((const void*)abort, rank ^ 1u);

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * TC_EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(tslot)),
            "r"((uint32_t)(2 * BN)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // both CTAs' barriers are initialised before any copy or arrival may reach them
    cluster_sync_all();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        uint32_t it = 0;
        for (int u = cid; u < units && !*abort; u += ncl) {
            const Unit w = unit_of_pair(u, a, BN);
            for (int i = 0; i < w.nk; ++i, ++it) {
                const int s = it % ST;
                const uint32_t ph = (it / ST) & 1u;
                if (it >= (uint32_t)ST && !mbar_wait_pair(&empty[s], ph ^ 1u, abort, peer_abort))
                    break;
                uint8_t* st = smem + s * L::STAGE;
                if (rank == 0) mbar_expect_tx(&full[s], 2u * (uint32_t)L::STAGE);
                const uint32_t fb = smem_in_cta(&full[s], 0u);
                load_operand(true, a.a_mn, st, &tmA, fb, w.kb0 + i, w.m0 + (int)rank * 128, 128);
                load_operand(true, a.b_mn, st + L::A_BYTES, &tmB, fb, w.kb0 + i,
                             w.n0 + (int)rank * (BN / 2), BN / 2);
            }
        }
        // the even CTA's full barriers count both CTAs' copies: waiting (bounded) for the last
        // load of each stage there covers the copies in flight of the pair
        if (rank == 0) {
            const uint32_t last = it;
            for (uint32_t j = last > (uint32_t)ST ? last - ST : 0; j < last; ++j) {
                volatile int no_abort = 0;
                mbar_wait_ab(&full[j % ST], (j / ST) & 1u, &no_abort);
            }
        }
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // ---------------- MMA issuer (even CTA) ----------------
        const uint32_t idesc =
            idesc_bf16_m256<BN>() | ((uint32_t)a.a_mn << 15) | ((uint32_t)a.b_mn << 16);
        const uint64_t sa = operand_step(a.a_mn), sb = operand_step(a.b_mn);
        uint32_t it = 0, j = 0;
        for (int u = cid; u < units && !*abort; u += ncl, ++j) {
            const Unit w = unit_of_pair(u, a, BN);
            const uint32_t b = j & 1u, use = j >> 1;
            if (use > 0 && !mbar_wait_pair(&tempty[b], (use - 1) & 1u, abort, peer_abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + b * BN;
            bool ok = true;
            for (int i = 0; i < w.nk; ++i, ++it) {
                const int s = it % ST;
                if (!mbar_wait_pair(&full[s], (it / ST) & 1u, abort, peer_abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint8_t* st = smem + s * L::STAGE;
                const uint64_t da = operand_desc(a.a_mn, smem_u32(st));
                const uint64_t db = operand_desc(a.b_mn, smem_u32(st + L::A_BYTES));
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk)
                    umma_pair(acc, da + sa * kk, db + sb * kk, idesc, (i | kk) != 0 ? 1u : 0u);
                umma_commit_pair(&empty[s], (uint16_t)3);
            }
            if (!ok) break;
            umma_commit_pair(&tfull[b], (uint16_t)3);
        }
        // every MMA issued has completed (it reads the other CTA's shared memory) before the
        // pair may leave
        umma_commit_pair(drain, (uint16_t)1);
        volatile int no_abort = 0;
        mbar_wait_ab(drain, 0u, &no_abort);
    } else if (warp >= 2) {
        // ---------------- epilogue (both CTAs, own accumulator rows) ----------------
        const int q = warp & 3, half = (warp - 2) >> 2;
        const int c_lo = half * (BN / 2), c_hi = c_lo + BN / 2;
        const uint32_t tempty0 = smem_in_cta(&tempty[0], 0u);
        uint32_t j = 0;
        for (int u = cid; u < units; u += ncl, ++j) {
            Unit w = unit_of_pair(u, a, BN);
            w.m0 += (int)rank * 128;
            const uint32_t b = j & 1u, use = j >> 1;
            if (!mbar_wait_pair(&tfull[b], use & 1u, abort, peer_abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = w.m0 + q * 32 + lane;
            const bool row_ok = row < a.M;
            uint8_t* stage = epi_stage + (warp - 2) * 4096;
            auto drain = [&](int c, const uint32_t (&r)[32]) {
                if (a.tma_c)
                    epilogue32_tma(a, w, row, row_ok, w.n0 + c, w.m0 + q * 32, r, stage, &tmC,
                                   &tmCT, &tmP);
                else
                    epilogue32(a, w, row, row_ok, w.n0 + c, r);
            };
            auto release = [&]() {  // every accumulator load of this warp has completed
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(tempty0 + b * 8u);
            };
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + b * BN;
            if (w.nk > 0) {
                // the load of the next 32 columns is in flight while this block is staged and
                // stored; the accumulator is released as soon as its last load has completed
                uint32_t ra[32], rb[32];
                tmem_ld32_async(tbase + (uint32_t)c_lo, ra);
#pragma unroll 1
                for (int c = c_lo; c < c_hi; c += 64) {
                    tmem_wait_ld(ra);
                    if (c + 32 < c_hi) tmem_ld32_async(tbase + (uint32_t)(c + 32), rb);
                    else release();
                    drain(c, ra);
                    if (c + 32 < c_hi) {
                        tmem_wait_ld(rb);
                        if (c + 64 < c_hi) tmem_ld32_async(tbase + (uint32_t)(c + 64), ra);
                        else release();
                        drain(c + 32, rb);
                    }
                }
            } else {
                uint32_t r[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) r[t] = 0u;
                release();
#pragma unroll 1
                for (int c = c_lo; c < c_hi; c += 32) drain(c, r);
            }
        }
        if (a.tma_c && lane == 0) bulk_wait0();
    }
    if (*abort && a.err) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // no CTA of the pair leaves (or releases tensor memory) while the other may still touch its
    // shared memory or the pair's accumulators
    cluster_sync_all();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)(2 * BN)));
    cluster_sync_all();
}

// ------------------------------------------------------------------------------------------
// Grouped form: one persistent launch over the (group, split, row tile, column tile) work list
// of many independent GEMMs of different shapes (the batched problems of one pipeline stage).
// Each group's tensor maps and epilogue arguments live in device memory; unit u belongs to the
// group whose [unit0, unit0 + units) holds it (binary search over the groups). The roles and
// the pipeline are those of k_gemm_tc; a role that meets a new group first makes the group's
// tensor maps visible to the tensor-map proxy (they were written by a host copy).
// ------------------------------------------------------------------------------------------
struct __align__(128) TcGroupDev {
    CUtensorMap tmA, tmB, tmC, tmCT, tmP;
    TcArgs a;
    int unit0, units;
};

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"((uint64_t)m)
                 : "memory");
}

__device__ __forceinline__ int group_of(const TcGroupDev* __restrict__ G, int ng, int u) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (G[mid].unit0 <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc_g(const TcGroupDev* __restrict__ G, int ng, int units) {
    using L = TcSmem<BN>;
    constexpr int ST = L::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* epi_stage = smem + ST * L::STAGE;
    uint64_t* full = (uint64_t*)(smem + ST * L::STAGE + L::EPI);
    uint64_t* empty = full + ST;
    uint64_t* tfull = empty + ST;
    uint64_t* tempty = tfull + 2;
    uint32_t* tslot = (uint32_t*)(tempty + 2);
    volatile int* abort = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], TC_EPI_WARPS);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(tslot)),
            "r"((uint32_t)(2 * BN)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        uint32_t it = 0;
        int gcur = -1;
        for (int u = blockIdx.x; u < units && !*abort; u += gridDim.x) {
            const int g = group_of(G, ng, u);
            if (g != gcur) {
                gcur = g;
                tmap_acquire(&G[g].tmA);
                tmap_acquire(&G[g].tmB);
            }
            const Unit w = unit_of(u - G[g].unit0, G[g].a, BN);
            for (int i = 0; i < w.nk; ++i, ++it) {
                const int s = it % ST;
                const uint32_t ph = (it / ST) & 1u;
                if (it >= (uint32_t)ST && !mbar_wait_ab(&empty[s], ph ^ 1u, abort)) break;
                uint8_t* st = smem + s * L::STAGE;
                mbar_expect_tx(&full[s], (uint32_t)L::STAGE);
                tma_load_2d(st, &G[g].tmA, &full[s], (w.kb0 + i) * TC_BK, w.m0);
                tma_load_2d(st + L::A_BYTES, &G[g].tmB, &full[s], (w.kb0 + i) * TC_BK, w.n0);
            }
        }
        // never leave with copies in flight: wait (bounded) for the last load of each stage
        const uint32_t last = it;
        for (uint32_t j = last > (uint32_t)ST ? last - ST : 0; j < last; ++j) {
            volatile int no_abort = 0;
            mbar_wait_ab(&full[j % ST], (j / ST) & 1u, &no_abort);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = idesc_bf16<BN>();
        uint32_t it = 0, j = 0;
        for (int u = blockIdx.x; u < units && !*abort; u += gridDim.x, ++j) {
            const int g = group_of(G, ng, u);
            const Unit w = unit_of(u - G[g].unit0, G[g].a, BN);
            const uint32_t b = j & 1u, use = j >> 1;
            if (use > 0 && !mbar_wait_ab(&tempty[b], (use - 1) & 1u, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + b * BN;
            bool ok = true;
            for (int i = 0; i < w.nk; ++i, ++it) {
                const int s = it % ST;
                if (!mbar_wait_ab(&full[s], (it / ST) & 1u, abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint8_t* st = smem + s * L::STAGE;
                const uint64_t da = sdesc_sw128(smem_u32(st));
                const uint64_t db = sdesc_sw128(smem_u32(st + L::A_BYTES));
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk)
                    umma(acc, da + 2 * kk, db + 2 * kk, idesc, (i | kk) != 0 ? 1u : 0u);
                umma_commit(&empty[s]);
            }
            if (!ok) break;
            umma_commit(&tfull[b]);
        }
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3, half = (warp - 2) >> 2;
        const int c_lo = half * (BN / 2), c_hi = c_lo + BN / 2;
        uint32_t j = 0;
        int gcur = -1;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++j) {
            const int g = group_of(G, ng, u);
            const TcArgs& a = G[g].a;  // read in place (L1): fewer live registers
            if (g != gcur) {
                // stores of the previous group's buffers have landed before its maps change
                if (gcur >= 0 && lane == 0) bulk_wait0();
                gcur = g;
                if (lane == 0) {
                    tmap_acquire(&G[g].tmC);
                    tmap_acquire(&G[g].tmCT);
                    tmap_acquire(&G[g].tmP);
                }
                __syncwarp();
            }
            const Unit w = unit_of(u - G[g].unit0, a, BN);
            const uint32_t b = j & 1u, use = j >> 1;
            if (!mbar_wait_ab(&tfull[b], use & 1u, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = w.m0 + q * 32 + lane;
            const bool row_ok = row < a.M;
#pragma unroll 1
            for (int c = c_lo; c < c_hi; c += 32) {
                uint32_t r[32];
                if (w.nk > 0 && w.n0 + c < a.N) {
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * BN + (uint32_t)c, r);
                } else {
#pragma unroll
                    for (int t = 0; t < 32; ++t) r[t] = 0u;
                }
                if (w.n0 + c >= a.N) continue;  // a column block past this group's N
                if (a.tma_c)
                    epilogue32_tma(a, w, row, row_ok, w.n0 + c, w.m0 + q * 32, r,
                                   epi_stage + (warp - 2) * 4096, &G[g].tmC, &G[g].tmCT,
                                   &G[g].tmP);
                else
                    epilogue32(a, w, row, row_ok, w.n0 + c, r);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        if (lane == 0) bulk_wait0();  // every store of this warp has landed
    }
    if (*abort && G[0].a.err) atomicExch(G[0].a.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)(2 * BN)));
}

// split-K sums of many groups: blockIdx.y = job
struct SplitJob {
    const float* P;
    float* C;
    int64_t ldc;
    int splits, M, N;
};
__global__ void k_splitk_reduce_g(const SplitJob* __restrict__ jobs) {
    const SplitJob J = jobs[blockIdx.y];
    const int64_t total = (int64_t)J.M * J.N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < J.splits; ++z) s += J.P[(size_t)z * total + t];
        const int64_t m = t / J.N, n = t - m * J.N;
        J.C[m * J.ldc + n] = s;
    }
}

// C[m][n] = sum over splits of P[z][m][n] (fixed order)
__global__ void k_splitk_reduce(const float* __restrict__ P, int splits, int M, int N,
                                float* __restrict__ C, int64_t ldc) {
    const int64_t total = (int64_t)M * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += P[(size_t)z * total + t];
        const int64_t m = t / N, n = t - m * N;
        C[m * ldc + n] = s;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encoder() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode ? NQS_OK : NQS_ERR_CUDA;
}

// 2-D bf16 tensor map over [rows][ld] (k contiguous) with a box of box_rows x 64
int make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld,
             int box_rows) {
    NQS_TRY(get_encoder());
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {TC_BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box,
                          es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        nqs_record_message("cuTensorMapEncodeTiled rejected a GEMM operand");
        return NQS_ERR_CUDA;
    }
    return NQS_OK;
}

// store map with a 32 x 32 box and the given swizzle of the shared-memory side: dims innermost
// first, strides in bytes of the outer dims; false when the layout cannot take TMA (alignment) —
// the caller then stores directly
bool make_store_map(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esize, int rank,
                    const cuuint64_t* dims, const cuuint64_t* strides,
                    CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE) {
    if (get_encoder() != NQS_OK || ((uintptr_t)base & 15)) return false;
    for (int i = 0; i < rank - 1; ++i)
        if (strides[i] % 16) return false;
    cuuint32_t box[3] = {32, 32, 1};
    cuuint32_t es[3] = {1, 1, 1};
    (void)esize;
    CUresult r = g_encode(m, dt, rank, (void*)base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 148;
    }
    return n;
}

template <int BN>
int launch_tc(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc,
              const CUtensorMap& tct, const CUtensorMap& tp, const TcArgs& a, cudaStream_t s) {
    const int smem = TcSmem<BN>::BYTES;
    NQS_CK(cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int units = ((a.N + BN - 1) / BN) * ((a.M + 127) / 128) * a.splits;
    const int grid = units < num_sms() ? units : num_sms();
    {
        ProfScope prof_(PROF_GEMM, s);
        k_gemm_tc<BN><<<grid, TC_THREADS, smem, s>>>(ta, tb, tc, tct, tp, a);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// The paired form: clusters of two CTAs, as many clusters as can be resident at once (the SMs
// of a GPC pair up; an odd SM left over in a GPC stays idle), at most one per 256 x BN unit.
template <int BN>
int launch_tc_pair(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc,
                   const CUtensorMap& tct, const CUtensorMap& tp, const TcArgs& a,
                   cudaStream_t s) {
    const int smem = TcSmem2<BN>::BYTES;
    NQS_CK(cudaFuncSetAttribute(k_gemm_tc_pair<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // resident clusters, per device and tile width (one template instance each); concurrent
    // first calls may both query, and store the same value
    static std::atomic<int> cache[64];
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return NQS_ERR_UNSUPPORTED;
    int max_clusters = cache[dev].load(std::memory_order_relaxed);
    if (max_clusters == 0) {
        cfg.gridDim = dim3(2 * (num_sms() / 2), 1, 1);
        int n = 0;
        NQS_CK(cudaOccupancyMaxActiveClusters(&n, k_gemm_tc_pair<BN>, &cfg));
        if (n <= 0) return NQS_ERR_UNSUPPORTED;
        max_clusters = n;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    const int units = ((a.N + BN - 1) / BN) * ((a.M + 255) / 256) * a.splits;
    const int clusters = units < max_clusters ? units : max_clusters;
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    {
        ProfScope prof_(PROF_GEMM, s);
        NQS_CK(cudaLaunchKernelEx(&cfg, k_gemm_tc_pair<BN>, ta, tb, tc, tct, tp, a));
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

}  // namespace

// the tile width a shape gets without tuning
static int heuristic_bn_shape(int N) { return N <= 64 ? 64 : (N <= 128 ? 128 : 256); }

// K splits of a plain FP32-output GEMM: enough units to fill the GPU, and no unit longer than
// TC_MAX_UNIT_KB k-blocks. The CTAs that work on one split read the same K window of A and B and
// share it in L2 only while they stay close in K; over long ranges they drift apart and the
// operands come from DRAM again (the weight gradients over 2^20 configurations: the step's
// GEMMs took 28.4 ms with units of 4096 k-blocks, 26.5 ms with at most 512; one wave of
// longer units, 148 / tiles splits, measured 28.4 ms on three boxes and 24.5 ms on one).
#define TC_MAX_UNIT_KB 512
static int single_bn_for(const TcGemm& g);  // the tile width the single GEMM runs g with

static int tc_split_count(int tiles, int nkb) {
    int splits = 1;
    while (tiles * splits < 148 && splits * 2 <= nkb && splits < 64) splits *= 2;
    while (nkb / splits > TC_MAX_UNIT_KB && splits * 2 <= nkb && splits < 64) splits *= 2;
    return splits;
}

// launch with a given tile width
static bool g_pair = true;  // nqs_set_gemm_pairing

static int gemm_tc_run(const TcGemm& g, Scratch& sc, cudaStream_t s, int BN) {
    // 256-column tiles run in the paired (two-SM) form
    const bool pair = g_pair && BN == 256;
    CUtensorMap ta, tb;
    // K-major: boxes of 64 k x (128 or the B tile's) rows; MN-major: boxes of 64 x 64 k-rows
    if (g.a_mn) NQS_TRY(make_map(&ta, g.A, g.K, g.M, g.lda, 64));
    else NQS_TRY(make_map(&ta, g.A, g.M, g.K, g.lda, 128));
    if (g.b_mn) NQS_TRY(make_map(&tb, g.B, g.K, g.N, g.ldb, 64));
    else NQS_TRY(make_map(&tb, g.B, g.N, g.K, g.ldb, pair ? BN / 2 : BN));
    TcArgs a;
    memset(&a, 0, sizeof a);
    a.M = g.M;
    a.N = g.N;
    a.K = g.K;
    a.epi = g.epi;
    a.C = g.C;
    a.ldc = g.ldc;
    a.c_bf16 = g.c_bf16;
    a.CT = g.CT;
    a.ldct = g.ldct;
    a.bias = g.bias;
    a.phi0 = g.phi0;
    a.aux = g.aux;
    a.ld_aux = g.ld_aux;
    a.err = g.err;
    a.a_mn = g.a_mn ? 1 : 0;
    a.b_mn = g.b_mn ? 1 : 0;
    // split K when the output has too few tiles to fill the GPU
    const int tiles = ((g.N + BN - 1) / BN) * ((g.M + 127) / 128);
    const int nkb = (g.K + TC_BK - 1) / TC_BK;
    int splits = 1;
    if (g.epi == EPI_STORE && !g.CT && !g.c_bf16) splits = tc_split_count(tiles, nkb);
    if (splits > 1) {
        NQS_TRY(sc.get(&a.partial, (size_t)splits * g.M * g.N));
        // ceil split so that no split is empty
        const int per = (nkb + splits - 1) / splits;
        splits = (nkb + per - 1) / per;
    }
    a.splits = splits;
    // epilogue stores through TMA when every output the GEMM writes has a TMA-able layout
    CUtensorMap tc, tct, tp;
    memset(&tc, 0, sizeof tc);
    memset(&tct, 0, sizeof tct);
    memset(&tp, 0, sizeof tp);
    bool tma = true;
    if (splits > 1) {
        const cuuint64_t dims[3] = {(cuuint64_t)g.N, (cuuint64_t)g.M, (cuuint64_t)splits};
        const cuuint64_t str[2] = {(cuuint64_t)g.N * 4, (cuuint64_t)g.M * g.N * 4};
        tma = make_store_map(&tp, a.partial, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 3, dims, str,
                             CU_TENSOR_MAP_SWIZZLE_128B);
    } else {
        if (g.C) {
            const cuuint64_t dims[2] = {(cuuint64_t)g.N, (cuuint64_t)g.M};
            const cuuint64_t str[1] = {(cuuint64_t)g.ldc * (g.c_bf16 ? 2 : 4)};
            tma = make_store_map(&tc, g.C,
                                 g.c_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                 g.c_bf16 ? 2 : 4, 2, dims, str,
                                 g.c_bf16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
        }
        if (tma && g.CT) {
            tma = g.C == nullptr || g.c_bf16;  // one 4 KB staging buffer: bf16 C + bf16 CT
            const cuuint64_t dims[2] = {(cuuint64_t)g.M, (cuuint64_t)g.N};
            const cuuint64_t str[1] = {(cuuint64_t)g.ldct * 2};
            tma = tma && make_store_map(&tct, g.CT, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2, dims,
                                        str);
        }
    }
    a.tma_c = tma ? 1 : 0;
    int st = pair ? launch_tc_pair<256>(ta, tb, tc, tct, tp, a, s)
                  : (BN == 64 ? launch_tc<64>(ta, tb, tc, tct, tp, a, s)
                              : (BN == 128 ? launch_tc<128>(ta, tb, tc, tct, tp, a, s)
                                           : launch_tc<256>(ta, tb, tc, tct, tp, a, s)));
    NQS_TRY(st);
    if (splits > 1) {
        k_splitk_reduce<<<grid_for((int64_t)g.M * g.N, 256), 256, 0, s>>>(
            a.partial, splits, g.M, g.N, (float*)g.C, g.ldc);
        NQS_CK_LAUNCH();
    }
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// grouped GEMM sets (batched problems): descriptors built once, one launch per use
// ------------------------------------------------------------------------------------------
struct TcGroupSet {
    TcGroupDev* dev = nullptr;
    int ng = 0, units = 0, BN = 0;
    std::vector<float*> partials;
    SplitJob* jobs = nullptr;
    int njobs = 0;
    int64_t max_mn = 0;
};

void tc_group_set_destroy(TcGroupSet* set) {
    if (!set) return;
    cudaFree(set->dev);
    cudaFree(set->jobs);
    for (float* q : set->partials) cudaFree(q);
    delete set;
}

int tc_group_set_create(const TcGemm* gs, int n, int BN, TcGroupSet** out) {
    if (!gs || n <= 0 || !out || (BN != 64 && BN != 128 && BN != 256)) return NQS_ERR_ARG;
    TcGroupSet* set = new TcGroupSet();
    set->BN = BN;
    auto fail = [&](int code) {
        tc_group_set_destroy(set);
        return code;
    };
    std::vector<TcGroupDev> host(n);
    std::vector<SplitJob> jobs;
    int unit0 = 0;
    for (int i = 0; i < n; ++i) {
        const TcGemm& g = gs[i];
        if (g.M <= 0 || g.N <= 0 || g.K <= 0) return fail(NQS_ERR_ARG);
        if (g.a_mn || g.b_mn) return fail(NQS_ERR_UNSUPPORTED);  // K-major operands only
        if ((g.lda * 2) % 16 || (g.ldb * 2) % 16 || ((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15))
            return fail(NQS_ERR_UNSUPPORTED);
        TcGroupDev& d = host[i];
        memset(&d, 0, sizeof d);
        int st = make_map(&d.tmA, g.A, g.M, g.K, g.lda, 128);
        if (st == NQS_OK) st = make_map(&d.tmB, g.B, g.N, g.K, g.ldb, BN);
        if (st != NQS_OK) return fail(st);
        TcArgs& a = d.a;
        a.M = g.M;
        a.N = g.N;
        a.K = g.K;
        a.epi = g.epi;
        a.C = g.C;
        a.ldc = g.ldc;
        a.c_bf16 = g.c_bf16;
        a.CT = g.CT;
        a.ldct = g.ldct;
        a.bias = g.bias;
        a.phi0 = g.phi0;
        a.aux = g.aux;
        a.ld_aux = g.ld_aux;
        a.err = g.err;
        // K splits as the single GEMM chooses them for this shape, with the tile width it uses
        // (tuned or not), so both give the same partial sums
        const int bref = single_bn_for(g);
        const int tiles_ref = ((g.N + bref - 1) / bref) * ((g.M + 127) / 128);
        const int nkb = (g.K + TC_BK - 1) / TC_BK;
        int splits = 1;
        if (g.epi == EPI_STORE && !g.CT && !g.c_bf16) splits = tc_split_count(tiles_ref, nkb);
        if (splits > 1) {
            const int per = (nkb + splits - 1) / splits;
            splits = (nkb + per - 1) / per;
        }
        a.splits = splits;
        bool tma = true;
        if (splits > 1) {
            float* P = nullptr;
            if (cudaMalloc(&P, (size_t)splits * g.M * g.N * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                return fail(NQS_ERR_OOM);
            }
            set->partials.push_back(P);
            a.partial = P;
            const cuuint64_t dims[3] = {(cuuint64_t)g.N, (cuuint64_t)g.M, (cuuint64_t)splits};
            const cuuint64_t str[2] = {(cuuint64_t)g.N * 4, (cuuint64_t)g.M * g.N * 4};
            tma = make_store_map(&d.tmP, P, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 3, dims, str,
                                 CU_TENSOR_MAP_SWIZZLE_128B);
            jobs.push_back(SplitJob{P, (float*)g.C, g.ldc, splits, g.M, g.N});
            const int64_t mn = (int64_t)g.M * g.N;
            if (mn > set->max_mn) set->max_mn = mn;
        } else {
            if (g.C) {
                const cuuint64_t dims[2] = {(cuuint64_t)g.N, (cuuint64_t)g.M};
                const cuuint64_t str[1] = {(cuuint64_t)g.ldc * (g.c_bf16 ? 2 : 4)};
                tma = make_store_map(&d.tmC, g.C,
                                     g.c_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                     g.c_bf16 ? 2 : 4, 2, dims, str,
                                     g.c_bf16 ? CU_TENSOR_MAP_SWIZZLE_64B
                                              : CU_TENSOR_MAP_SWIZZLE_128B);
            }
            if (tma && g.CT) {
                tma = g.C == nullptr || g.c_bf16;
                const cuuint64_t dims[2] = {(cuuint64_t)g.M, (cuuint64_t)g.N};
                const cuuint64_t str[1] = {(cuuint64_t)g.ldct * 2};
                tma = tma && make_store_map(&d.tmCT, g.CT, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 2,
                                            dims, str);
            }
        }
        a.tma_c = tma ? 1 : 0;
        d.unit0 = unit0;
        d.units = ((g.N + BN - 1) / BN) * ((g.M + 127) / 128) * splits;
        unit0 += d.units;
    }
    set->ng = n;
    set->units = unit0;
    if (cudaMalloc(&set->dev, sizeof(TcGroupDev) * n) != cudaSuccess ||
        cudaMemcpy(set->dev, host.data(), sizeof(TcGroupDev) * n, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaGetLastError();
        return fail(NQS_ERR_OOM);
    }
    if (!jobs.empty()) {
        set->njobs = (int)jobs.size();
        if (cudaMalloc(&set->jobs, sizeof(SplitJob) * jobs.size()) != cudaSuccess ||
            cudaMemcpy(set->jobs, jobs.data(), sizeof(SplitJob) * jobs.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return fail(NQS_ERR_OOM);
        }
    }
    *out = set;
    return NQS_OK;
}

template <int BN>
static int launch_tc_g(const TcGroupSet* set, cudaStream_t s) {
    const int smem = TcSmem<BN>::BYTES;
    NQS_CK(cudaFuncSetAttribute(k_gemm_tc_g<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem));
    const int grid = set->units < num_sms() ? set->units : num_sms();
    {
        ProfScope prof_(PROF_GEMM, s);
        k_gemm_tc_g<BN><<<grid, TC_THREADS, smem, s>>>(set->dev, set->ng, set->units);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int tc_group_set_launch(const TcGroupSet* set, cudaStream_t s) {
    if (!set || set->units <= 0) return NQS_ERR_ARG;
    const int st = set->BN == 64    ? launch_tc_g<64>(set, s)
                   : set->BN == 128 ? launch_tc_g<128>(set, s)
                                    : launch_tc_g<256>(set, s);
    NQS_TRY(st);
    if (set->njobs > 0) {
        k_splitk_reduce_g<<<dim3(grid_for(set->max_mn, 256, 64), set->njobs), 256, 0, s>>>(
            set->jobs);
        NQS_CK_LAUNCH();
    }
    return NQS_OK;
}

int tc_group_set_units(const TcGroupSet* set) { return set ? set->units : 0; }

// ------------------------------------------------------------------------------------------
// tile-width autotuner: when enabled, the first GEMM of each (M, N, K, epilogue, output kind)
// shape is timed with BN = 64, 128 and 256 (CUDA events on the launching stream, one warm-up
// and two timed runs each) and the fastest width is remembered for the process. Tuning never
// runs inside stream capture; untuned shapes use the heuristic below.
// ------------------------------------------------------------------------------------------
namespace {
struct TuneKey {
    int M, N, K, epi, kind;
    bool operator<(const TuneKey& o) const {
        if (M != o.M) return M < o.M;
        if (N != o.N) return N < o.N;
        if (K != o.K) return K < o.K;
        if (epi != o.epi) return epi < o.epi;
        return kind < o.kind;
    }
};
std::map<TuneKey, int> g_tuned;
std::mutex g_tune_mu;
bool g_autotune = false;

int heuristic_bn(int N) { return heuristic_bn_shape(N); }
}  // namespace

static int single_bn_for(const TcGemm& g) {
    const TuneKey key{g.M, g.N, g.K, g.epi,
                      (g.c_bf16 ? 1 : 0) | (g.CT ? 2 : 0) | (g.a_mn ? 4 : 0) | (g.b_mn ? 8 : 0)};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    return it != g_tuned.end() ? it->second : heuristic_bn_shape(g.N);
}

int tc_autotune_on() { return g_autotune ? 1 : 0; }

extern "C" int nqs_set_gemm_pairing(int on) {
    g_pair = on != 0;
    return NQS_OK;
}

extern "C" int nqs_set_autotune(int on) {
    g_autotune = on != 0;
    return NQS_OK;
}

extern "C" int nqs_autotune_entries(int* M, int* N, int* K, int* bn, int capacity) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    int i = 0;
    for (const auto& kv : g_tuned) {
        if (i < capacity && M && N && K && bn) {
            M[i] = kv.first.M;
            N[i] = kv.first.N;
            K[i] = kv.first.K;
            bn[i] = kv.second;
        }
        ++i;
    }
    return i;
}

int gemm_bf16_tcgen05(const TcGemm& g, Scratch& sc, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return NQS_ERR_ARG;
    if ((g.lda * 2) % 16 || (g.ldb * 2) % 16 || ((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15))
        return NQS_ERR_UNSUPPORTED;
    const TuneKey key{g.M, g.N, g.K, g.epi,
                      (g.c_bf16 ? 1 : 0) | (g.CT ? 2 : 0) | (g.a_mn ? 4 : 0) | (g.b_mn ? 8 : 0)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return gemm_tc_run(g, sc, s, it->second);
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NQS_CK(cudaStreamIsCapturing(s, &cap));
    if (!g_autotune || cap != cudaStreamCaptureStatusNone)
        return gemm_tc_run(g, sc, s, heuristic_bn(g.N));
    cudaEvent_t e0, e1;
    NQS_CK(cudaEventCreate(&e0));
    NQS_CK(cudaEventCreate(&e1));
    int best = heuristic_bn(g.N);
    float best_ms = 1e30f;
    for (int bn : {64, 128, 256}) {
        if (bn >= 2 * ((g.N + 63) / 64 * 64)) continue;  // tile at least twice as wide as N
        NQS_TRY(gemm_tc_run(g, sc, s, bn));
        NQS_CK(cudaEventRecord(e0, s));
        for (int r = 0; r < 2; ++r) NQS_TRY(gemm_tc_run(g, sc, s, bn));
        NQS_CK(cudaEventRecord(e1, s));
        NQS_CK(cudaEventSynchronize(e1));
        float ms = 0;
        NQS_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
            best_ms = ms;
            best = bn;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = best;
    }
    return gemm_tc_run(g, sc, s, best);
}


// ------------------------------------------------------------------------------------------
// C ABI: plain library GEMM C = A B^T (bf16 in, FP32 out), the same kernel the network uses
// ------------------------------------------------------------------------------------------
extern "C" int nqs_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N,
                             int K, float* C, int64_t ldc, int* err_flag, nqs_stream_t stream) {
    return nqs_gemm_bf16_ex(A, lda, 0, B, ldb, 0, M, N, K, C, ldc, err_flag, stream);
}

extern "C" int nqs_gemm_bf16_ex(const void* A, int64_t lda, int a_mn, const void* B, int64_t ldb,
                                int b_mn, int M, int N, int K, float* C, int64_t ldc,
                                int* err_flag, nqs_stream_t stream) {
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0) return NQS_ERR_ARG;
    if ((a_mn && lda < M) || (!a_mn && lda < K) || (b_mn && ldb < N) || (!b_mn && ldb < K))
        return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    nqs_problem host;
    memset(&host, 0, sizeof host);
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    NQS_CK(cudaDeviceGetDefaultMemPool(&host.pool, dev));
    Scratch sc(&host, s);
    TcGemm g;
    memset(&g, 0, sizeof g);
    g.A = (const __nv_bfloat16*)A;
    g.lda = lda;
    g.B = (const __nv_bfloat16*)B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = EPI_STORE;
    g.C = C;
    g.ldc = ldc;
    g.err = err_flag;
    g.a_mn = a_mn ? 1 : 0;
    g.b_mn = b_mn ? 1 : 0;
    return gemm_bf16_tcgen05(g, sc, s);
}

// ------------------------------------------------------------------------------------------
// Failure-detection check: one thread waits, with the pipeline's bounded mbarrier wait, on a
// barrier that expects one arrival that never comes. The wait gives up after `limit` clocks
// and reports through the problem's error word, as a timed-out GEMM pipeline does.
// ------------------------------------------------------------------------------------------
__global__ void k_wait_probe(long long limit, int* err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_ab(&bar, 0u, (volatile int*)&abort_flag, limit))
        atomicExch(err, 1);
    __syncthreads();
}

extern "C" int nqs_wait_probe(nqs_problem* p, int64_t limit_cycles, nqs_stream_t stream) {
    if (!p || limit_cycles < 1 || limit_cycles > 4000000000ll) return NQS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_wait_probe<<<1, 32, 0, s>>>((long long)limit_cycles, p->err_word);
    NQS_CK_LAUNCH();
    return check_err_word(p, s);
}

// Device primitives: exclusive scans, compensated FP64 reductions, masked max and a stable
// LSD radix sort of (u64 key, f64 value) pairs. All are deterministic for a given input size.
#include "excite.cuh"
#include "nqs_internal.cuh"
#include "prof.cuh"

// ------------------------------------------------------------------------------------------
// exclusive scan: tiles of 256 threads x 8 items, three phases (tile sums, scan of the sums,
// tile scans plus offsets), recursive on the tile sums.
// ------------------------------------------------------------------------------------------
#define SC_THREADS 256
#define SC_ITEMS 8
#define SC_TILE (SC_THREADS * SC_ITEMS)

template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (SC_THREADS / 32) ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(FULL_MASK, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (SC_THREADS / 32)) warp_tot[lane] = wi - w;
        if (lane == (SC_THREADS / 32) - 1) *total = wi;
    }
    __syncthreads();
    T r = warp_tot[warp] + incl - v;
    __syncthreads();
    return r;
}

// a thread's SC_ITEMS consecutive elements: 16-byte loads when the whole run is in range and
// the array is 16-byte aligned (vec), else element by element
template <class T>
__device__ __forceinline__ void sc_load(const T* in, int64_t base, int64_t n, bool vec,
                                        T (&v)[SC_ITEMS]) {
    if (vec && base + SC_ITEMS <= n) {
        const uint4* q = (const uint4*)(in + base);
#pragma unroll
        for (int k = 0; k < (int)(SC_ITEMS * sizeof(T) / 16); ++k) {
            const uint4 w = q[k];
            T* d = (T*)&w;
#pragma unroll
            for (int j = 0; j < (int)(16 / sizeof(T)); ++j) v[k * (16 / sizeof(T)) + j] = d[j];
        }
    } else {
#pragma unroll
        for (int k = 0; k < SC_ITEMS; ++k) v[k] = (base + k < n) ? in[base + k] : T(0);
    }
}

template <class T>
__global__ void __launch_bounds__(SC_THREADS) k_tile_sum(const T* in, int64_t n, T* sums) {
    __shared__ T warp_tot[SC_THREADS / 32];
    __shared__ T total;
    int64_t base = (int64_t)blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
    const bool vec = (((uintptr_t)in) & 15) == 0;
    T v[SC_ITEMS];
    sc_load<T>(in, base, n, vec, v);
    T s = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) s += v[k];
    block_exclusive_scan<T>(s, warp_tot, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <class T>
__global__ void __launch_bounds__(SC_THREADS) k_tile_scan(const T* in, T* out, int64_t n,
                                                          const T* offs, T* grand) {
    __shared__ T warp_tot[SC_THREADS / 32];
    __shared__ T total;
    int64_t base = (int64_t)blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
    const bool vec = ((((uintptr_t)in) | ((uintptr_t)out)) & 15) == 0;
    T v[SC_ITEMS];
    sc_load<T>(in, base, n, vec, v);
    T s = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) s += v[k];
    T ex = block_exclusive_scan<T>(s, warp_tot, &total);
    T off = offs ? offs[blockIdx.x] : T(0);
    T run = off + ex;
    __align__(16) T o[SC_ITEMS];
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        o[k] = run;
        run += v[k];
    }
    if (vec && base + SC_ITEMS <= n) {
        uint4* q = (uint4*)(out + base);
#pragma unroll
        for (int k = 0; k < (int)(SC_ITEMS * sizeof(T) / 16); ++k) q[k] = ((const uint4*)o)[k];
    } else {
#pragma unroll
        for (int k = 0; k < SC_ITEMS; ++k)
            if (base + k < n) out[base + k] = o[k];
    }
    if (grand && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *grand = off + total;
}

template <class T>
static int scan_exclusive(nqs_problem* p, Scratch& sc, const T* in, T* out, int64_t n, T* total,
                          cudaStream_t s) {
    if (n <= 0) {
        if (total) NQS_CK(cudaMemsetAsync(total, 0, sizeof(T), s));
        return NQS_OK;
    }
    int64_t tiles = (n + SC_TILE - 1) / SC_TILE;
    if (tiles == 1) {
        k_tile_scan<T><<<1, SC_THREADS, 0, s>>>(in, out, n, nullptr, total);
        NQS_CK_LAUNCH();
        return NQS_OK;
    }
    T* sums;
    NQS_TRY(sc.get(&sums, tiles));
    {
        ProfScope prof_(PROF_SCAN, s);
        k_tile_sum<T><<<(unsigned)tiles, SC_THREADS, 0, s>>>(in, n, sums);
    }
    NQS_CK_LAUNCH();
    NQS_TRY(scan_exclusive<T>(p, sc, sums, sums, tiles, (T*)nullptr, s));
    {
        ProfScope prof_(PROF_SCAN, s);
        k_tile_scan<T><<<(unsigned)tiles, SC_THREADS, 0, s>>>(in, out, n, sums, total);
    }
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int scan_exclusive_i64(nqs_problem* p, Scratch& sc, const int64_t* in, int64_t* out, int64_t n,
                       int64_t* total, cudaStream_t s) {
    return scan_exclusive<int64_t>(p, sc, in, out, n, total, s);
}
int scan_exclusive_u32(nqs_problem* p, Scratch& sc, const uint32_t* in, uint32_t* out, int64_t n,
                       cudaStream_t s) {
    return scan_exclusive<uint32_t>(p, sc, in, out, n, (uint32_t*)nullptr, s);
}
int scan_exclusive_f64(nqs_problem* p, Scratch& sc, const double* in, double* out, int64_t n,
                       double* total, cudaStream_t s) {
    return scan_exclusive<double>(p, sc, in, out, n, total, s);
}

// ------------------------------------------------------------------------------------------
// compensated (Neumaier) reductions: fixed grid, fixed tree -> deterministic
// ------------------------------------------------------------------------------------------
#include "ksum.cuh"

// mode 0: sum x; mode 1: sum x*y; mode 2: sum y*y
template <int MODE>
__global__ void __launch_bounds__(KR_THREADS) k_ksum(const double* x, const double* y, int64_t n,
                                                      double2* part) {
    KS k{0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * KR_THREADS + threadIdx.x; i < n;
         i += (int64_t)KR_BLOCKS * KR_THREADS) {
        double v = MODE == 0 ? x[i] : (MODE == 1 ? __dmul_rn(x[i], y[i]) : __dmul_rn(y[i], y[i]));
        k = ks_add(k, v);
    }
    KS r = block_ks(k);
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(r.s, r.c);
}

__global__ void __launch_bounds__(KR_THREADS) k_ksum_final(const double2* part, int nparts,
                                                            double* out) {
    KS k{0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += KR_THREADS) k = ks_merge(k, KS{part[i].x, part[i].y});
    KS r = block_ks(k);
    if (threadIdx.x == 0) *out = r.s + r.c;
}

int ksum_f64(nqs_problem* p, Scratch& sc, const double* x, int64_t n, double* out,
             cudaStream_t s) {
    double2* part;
    NQS_TRY(sc.get(&part, KR_BLOCKS));
    k_ksum<0><<<KR_BLOCKS, KR_THREADS, 0, s>>>(x, nullptr, n, part);
    NQS_CK_LAUNCH();
    k_ksum_final<<<1, KR_THREADS, 0, s>>>(part, KR_BLOCKS, out);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

int kdot2_f64(nqs_problem* p, Scratch& sc, const double* x, const double* y, int64_t n,
              double* out, cudaStream_t s) {
    double2* part;
    NQS_TRY(sc.get(&part, 2 * KR_BLOCKS));
    k_ksum<1><<<KR_BLOCKS, KR_THREADS, 0, s>>>(x, y, n, part);
    NQS_CK_LAUNCH();
    k_ksum<2><<<KR_BLOCKS, KR_THREADS, 0, s>>>(x, y, n, part + KR_BLOCKS);
    NQS_CK_LAUNCH();
    k_ksum_final<<<1, KR_THREADS, 0, s>>>(part, KR_BLOCKS, out);
    NQS_CK_LAUNCH();
    k_ksum_final<<<1, KR_THREADS, 0, s>>>(part + KR_BLOCKS, KR_BLOCKS, out + 1);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

__global__ void __launch_bounds__(KR_THREADS) k_max_masked(const double* x, const int8_t* mask,
                                                            int64_t n, double* part, int final_) {
    __shared__ double sm[KR_THREADS];
    double m = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * KR_THREADS + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * KR_THREADS)
        if (!mask || mask[i] != 0) m = fmax(m, x[i]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = KR_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

int max_f64_masked(nqs_problem* p, Scratch& sc, const double* x, const int8_t* mask, int64_t n,
                   double* out, cudaStream_t s) {
    double* part;
    NQS_TRY(sc.get(&part, KR_BLOCKS));
    k_max_masked<<<KR_BLOCKS, KR_THREADS, 0, s>>>(x, mask, n, part, 0);
    NQS_CK_LAUNCH();
    k_max_masked<<<1, KR_THREADS, 0, s>>>(part, nullptr, KR_BLOCKS, out, 1);
    NQS_CK_LAUNCH();
    return NQS_OK;
}

// ------------------------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits, keys of 32 or 64 bits with FP64 values. Per pass:
//   k_rs_hist     per-tile digit histograms (digit-major, tile-minor counts);
//   one exclusive scan over the counts -> global offset of (digit, tile);
//   k_rs_scatter  each warp ranks its keys with __match_any_sync (elements in ascending index
//                 order: warp, item, lane), the tile is staged in shared memory in digit order
//                 (values loaded straight into place), then written out so that consecutive
//                 threads store consecutive elements of each digit run (coalesced writes).
// Equal digits keep their input order (stable). No inter-block waiting of any kind.
// ------------------------------------------------------------------------------------------
#define RS_THREADS 256
#define RS_WARPS (RS_THREADS / 32)
// items per thread: 16 for 4/8-byte keys, 8 for 16-byte keys (tile staging must fit in smem)
template <class K>
struct RsCfg {
    static constexpr int ITEMS = sizeof(K) > 8 ? 8 : 16;
    static constexpr int TILE = RS_THREADS * ITEMS;
};

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K* __restrict__ keys, int64_t n,
                                                         int shift, uint32_t* __restrict__ counts,
                                                         int64_t T) {
    constexpr int RS_ITEMS = RsCfg<K>::ITEMS;
    constexpr int RS_TILE = RsCfg<K>::TILE;
    // one private sub-histogram per warp keeps shared-atomic contention inside a warp
    __shared__ uint32_t hist[RS_WARPS][256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    K key[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t i = base + k * RS_THREADS + threadIdx.x;
        key[k] = i < n ? keys[i] : key_zero<K>();
    }
    uint32_t* h = hist[threadIdx.x >> 5];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t i = base + k * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[key_digit(key[k], shift)], 1u);
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) c += hist[w][threadIdx.x];
    counts[(int64_t)threadIdx.x * T + blockIdx.x] = c;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Tile staging: one thread issues bulk asynchronous copies (global -> shared, completion
// counted in bytes on an mbarrier) for the tile's keys and values, so the whole tile is in
// flight at once; ranks are then computed from shared memory, a permutation is built in digit
// order, and the tile is written out digit run by digit run (coalesced). The wait on the
// mbarrier is bounded; on timeout the error word is set and the tile is left unwritten.
template <class K>
__global__ void __launch_bounds__(RS_THREADS, 3) k_rs_scatter(const K* __restrict__ kin,
                                                            const double* __restrict__ vin,
                                                            K* __restrict__ kout,
                                                            double* __restrict__ vout, int64_t n,
                                                            int shift,
                                                            const uint32_t* __restrict__ offs,
                                                            int64_t T, int* err) {
    constexpr int RS_ITEMS = RsCfg<K>::ITEMS;
    constexpr int RS_TILE = RsCfg<K>::TILE;
    extern __shared__ __align__(16) uint8_t rs_smem[];
    double* sv = (double*)rs_smem;             // [RS_TILE] values, input order
    K* sk = (K*)(sv + RS_TILE);                // [RS_TILE] keys, input order
    uint16_t* perm = (uint16_t*)(sk + RS_TILE);  // [RS_TILE] input index at each sorted slot
    __shared__ uint32_t whist[RS_WARPS][256];
    __shared__ uint32_t gdelta[256];  // global position of digit d's run minus its tile start
    __shared__ uint32_t warp_tot[RS_THREADS / 32];
    __shared__ uint32_t total;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int ok_s;
    const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
    const int tn = (int)((n - tbase) < RS_TILE ? (n - tbase) : RS_TILE);
    const bool bulk = tn == RS_TILE;  // full tiles are 16-byte aligned multiples of 16 bytes
    if (threadIdx.x == 0) {
        ok_s = 1;
        if (bulk) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            const uint32_t kb = RS_TILE * sizeof(K), vb = RS_TILE * sizeof(double);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                             smem_addr(&bar)),
                         "r"(kb + vb)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                "[%3];" ::"r"(smem_addr(sk)),
                "l"(kin + tbase), "r"(kb), "r"(smem_addr(&bar))
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                "[%3];" ::"r"(smem_addr(sv)),
                "l"(vin + tbase), "r"(vb), "r"(smem_addr(&bar))
                : "memory");
        }
    }
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&whist[0][0])[i] = 0;
    // this tile's global offset of digit threadIdx.x (read while the tile is in flight)
    const uint32_t goff = offs[(int64_t)threadIdx.x * T + blockIdx.x];
    if (!bulk) {
        for (int i = threadIdx.x; i < tn; i += RS_THREADS) {
            sk[i] = kin[tbase + i];
            sv[i] = vin[tbase + i];
        }
    }
    __syncthreads();
    if (bulk) {
        const long long t0 = clock64();
        while (true) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(smem_addr(&bar))
                : "memory");
            if (done) break;
            if (clock64() - t0 > 4000000000ll) {
                ok_s = 0;
                break;
            }
        }
    }
    __syncthreads();
    if (!ok_s) {
        if (threadIdx.x == 0 && err) atomicExch(err, 1);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wb = warp * (RS_ITEMS * 32);
    // Ranking. The digits and the match masks of all items are independent of the running
    // per-warp counts, so they are formed first (independent shared loads and matches in
    // flight together); only the count update below is a chain, item by item (elements in
    // ascending index order: warp, item, lane). Digit 256 marks a slot past the tile's end.
    uint32_t dg[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int li = wb + k * 32 + lane;
        dg[k] = li < tn ? key_digit(sk[li], shift) : 256u;
    }
    uint32_t rank[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) rank[k] = __match_any_sync(FULL_MASK, dg[k]);
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const unsigned peers = rank[k];
        const bool v = dg[k] < 256u;
        const uint32_t old = v ? whist[warp][dg[k]] : 0u;
        __syncwarp();
        if (v && lane == __ffs(peers) - 1) whist[warp][dg[k]] = old + __popc(peers);
        __syncwarp();
        rank[k] = ((old + __popc(peers & lt)) << 9) | dg[k];  // rank in warp, digit
    }
    __syncthreads();
    // thread d: the tile's count of digit d, the warps' exclusive prefixes over it, the start of
    // digit d's run in the tile; each warp's slot base for digit d is folded into whist
    uint32_t cnt = 0;
    uint32_t wpre[RS_WARPS];
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
        wpre[w] = cnt;
        cnt += whist[w][threadIdx.x];
    }
    const uint32_t dstart = block_exclusive_scan<uint32_t>(cnt, warp_tot, &total);
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) whist[w][threadIdx.x] = dstart + wpre[w];
    gdelta[threadIdx.x] = goff - dstart;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const uint32_t d = rank[k] & 511u;
        if (d < 256u) perm[whist[warp][d] + (rank[k] >> 9)] = (uint16_t)(wb + k * 32 + lane);
    }
    __syncthreads();
    // write-out in sorted-slot order: consecutive threads store consecutive elements of each
    // digit run; slot i of digit d goes to gdelta[d] + i (unsigned wrap-around is exact)
    if (bulk) {
#pragma unroll
        for (int k = 0; k < RS_ITEMS; ++k) {
            const int i = k * RS_THREADS + threadIdx.x;
            const int j = perm[i];
            const K kk = sk[j];
            const uint32_t gp = gdelta[key_digit(kk, shift)] + (uint32_t)i;
            kout[gp] = kk;
            vout[gp] = sv[j];
        }
    } else {
        for (int i = threadIdx.x; i < tn; i += RS_THREADS) {
            const int j = perm[i];
            const K kk = sk[j];
            const uint32_t gp = gdelta[key_digit(kk, shift)] + (uint32_t)i;
            kout[gp] = kk;
            vout[gp] = sv[j];
        }
    }
}

template <class K>
static int radix_sort_impl(nqs_problem* p, Scratch& sc, K*& keys, double*& vals, K*& keys_alt,
                           double*& vals_alt, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1) return NQS_OK;
    if (n >= (int64_t)1 << 32) return NQS_ERR_UNSUPPORTED;
    constexpr int RS_TILE = RsCfg<K>::TILE;
    int64_t T = (n + RS_TILE - 1) / RS_TILE;
    uint32_t* counts;
    NQS_TRY(sc.get(&counts, 256 * T));
    const int smem = RS_TILE * (int)(sizeof(double) + sizeof(K) + sizeof(uint16_t));
    NQS_CK(cudaFuncSetAttribute(k_rs_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem));
    for (int shift = 0; shift < bits; shift += 8) {
        {
            ProfScope prof_(PROF_RS_HIST, s);
            k_rs_hist<K><<<(unsigned)T, RS_THREADS, 0, s>>>(keys, n, shift, counts, T);
        }
        NQS_CK_LAUNCH();
        NQS_TRY(scan_exclusive_u32(p, sc, counts, counts, 256 * T, s));
        {
            ProfScope prof_(PROF_RS_SCATTER, s);
            k_rs_scatter<K><<<(unsigned)T, RS_THREADS, smem, s>>>(keys, vals, keys_alt, vals_alt, n,
                                                                  shift, counts, T, p->err_word);
        }
        NQS_CK_LAUNCH();
        K* tk = keys;
        keys = keys_alt;
        keys_alt = tk;
        double* tv = vals;
        vals = vals_alt;
        vals_alt = tv;
    }
    return NQS_OK;
}

int radix_sort_pairs(nqs_problem* p, Scratch& sc, uint64_t*& keys, double*& vals,
                     uint64_t*& keys_alt, double*& vals_alt, int64_t n, int bits, cudaStream_t s) {
    return radix_sort_impl<uint64_t>(p, sc, keys, vals, keys_alt, vals_alt, n, bits, s);
}

int radix_sort_pairs32(nqs_problem* p, Scratch& sc, uint32_t*& keys, double*& vals,
                       uint32_t*& keys_alt, double*& vals_alt, int64_t n, int bits,
                       cudaStream_t s) {
    return radix_sort_impl<uint32_t>(p, sc, keys, vals, keys_alt, vals_alt, n, bits, s);
}

int radix_sort_pairs128(nqs_problem* p, Scratch& sc, Key128*& keys, double*& vals,
                        Key128*& keys_alt, double*& vals_alt, int64_t n, int bits,
                        cudaStream_t s) {
    return radix_sort_impl<Key128>(p, sc, keys, vals, keys_alt, vals_alt, n, bits, s);
}

// Neumaier-compensated FP64 sums (deterministic: fixed partition and fixed trees), shared by
// the reductions of primitives.cu and the batched energy stage of energy.cu.
#pragma once

struct KS {
    double s, c;
};
__device__ __forceinline__ KS ks_add(KS k, double x) {
    double t = __dadd_rn(k.s, x);
    if (fabs(k.s) >= fabs(x)) k.c = __dadd_rn(k.c, __dadd_rn(__dsub_rn(k.s, t), x));
    else k.c = __dadd_rn(k.c, __dadd_rn(__dsub_rn(x, t), k.s));
    k.s = t;
    return k;
}
__device__ __forceinline__ KS ks_merge(KS a, KS b) {
    KS r = ks_add(a, b.s);
    r.c = __dadd_rn(r.c, b.c);
    return r;
}

#define KR_THREADS 256
#define KR_BLOCKS 256

__device__ __forceinline__ KS block_ks(KS v) {
    __shared__ double ss[KR_THREADS], cc[KR_THREADS];
    ss[threadIdx.x] = v.s;
    cc[threadIdx.x] = v.c;
    __syncthreads();
    for (int o = KR_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            KS a{ss[threadIdx.x], cc[threadIdx.x]}, b{ss[threadIdx.x + o], cc[threadIdx.x + o]};
            KS r = ks_merge(a, b);
            ss[threadIdx.x] = r.s;
            cc[threadIdx.x] = r.c;
        }
        __syncthreads();
    }
    KS r{ss[0], cc[0]};
    __syncthreads();
    return r;
}


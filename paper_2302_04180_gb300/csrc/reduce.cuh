// Reducers used by every kernel that carries dot products:
//  ExactR<K, Q>  the reproducible exact dot (exact_acc.cuh), K dots at once;
//  PlainR<K>     the comparator: binary64 fma accumulation per thread, warp
//                and block trees, then atomicAdd across blocks, whose order
//                changes from run to run (the paper's non-reproducible
//                "original", Sec. 3.2 / Sec. 4.1).
// Both end with the same last-block protocol, so solver tails are shared.
#pragma once

#include "exact_acc.cuh"

namespace rbs {

template <int K_, int Q>
struct ExactR {
    static constexpr int K = K_;
    Win<Q> win[K];
    uint32_t flags[K];
    unsigned long long (*sacc)[NL];
    uint32_t *sflags;

    __device__ __forceinline__ void init() {
        __shared__ unsigned long long s_acc[K][NL];
        __shared__ uint32_t s_flags[K];
        sacc = s_acc;
        sflags = s_flags;
#pragma unroll
        for (int k = 0; k < K; k++) {
            win[k].init();
            flags[k] = 0u;
        }
        sacc_zero<K>(sacc, sflags);
    }
    __device__ __forceinline__ void add(int k, double x, double y) {
        exact_add<Q>(win[k], flags[k], sacc[k], x, y);
    }
    __device__ __forceinline__ void add_sq(int k, double x) {
        exact_add<Q, true>(win[k], flags[k], sacc[k], x, x);
    }
    // true in the last block, with vals[0..K-1] rounded (shared memory).
    // SCRATCH: the per-warp scratch size the kernel already uses, so that the
    // flush staging shares it.
    template <int SCRATCH = FLUSH_SCRATCH>
    __device__ __forceinline__ bool finish(DotScratch *g, double *vals) {
        return exact_finish<K, Q, SCRATCH>(win, flags, sacc, sflags, g, vals);
    }
};

// ExactR with a second (low) window per dot: for standalone dots, whose
// operands may span far more exponents than the solver's vectors.
template <int K_, int Q>
struct ExactR2 {
    static constexpr int K = K_;
    Win<Q> win[K], low[K];
    uint32_t flags[K];
    unsigned long long (*sacc)[NL];
    uint32_t *sflags;

    __device__ __forceinline__ void init() {
        __shared__ unsigned long long s_acc[K][NL];
        __shared__ uint32_t s_flags[K];
        sacc = s_acc;
        sflags = s_flags;
#pragma unroll
        for (int k = 0; k < K; k++) {
            win[k].init();
            low[k].init();
            flags[k] = 0u;
        }
        sacc_zero<K>(sacc, sflags);
    }
    __device__ __forceinline__ void add(int k, double x, double y) {
        exact_add2<Q>(win[k], low[k], flags[k], sacc[k], x, y);
    }
    template <int SCRATCH = FLUSH_SCRATCH>
    __device__ __forceinline__ void flush_low() {
#pragma unroll
        for (int k = 0; k < K; k++) warp_flush<Q, SCRATCH>(low[k], sacc[k]);
    }
    template <int SCRATCH = FLUSH_SCRATCH>
    __device__ __forceinline__ bool finish(DotScratch *g, double *vals) {
        flush_low<SCRATCH>();
        return exact_finish<K, Q, SCRATCH>(win, flags, sacc, sflags, g, vals);
    }
};

template <int K_>
struct PlainR {
    static constexpr int K = K_;
    double s[K];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < K; k++) s[k] = 0.0;
    }
    __device__ __forceinline__ void add(int k, double x, double y) { s[k] = fma(x, y, s[k]); }
    __device__ __forceinline__ void add_sq(int k, double x) { s[k] = fma(x, x, s[k]); }
    template <int SCRATCH = 0>
    __device__ __forceinline__ bool finish(DotScratch *g, double *vals) {
        __shared__ double s_part[K][32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < K; k++) {
            double v = s[k];
            for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
            if (lane == 0) s_part[k][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < K) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = __dadd_rn(t, s_part[threadIdx.x][w]);
            atomicAdd((double *)&g->limbs[threadIdx.x][0], t);
        }
        __threadfence();
        __syncthreads();
        __shared__ bool s_last;
        if (threadIdx.x == 0) s_last = (atomicAdd(&g->ticket, 1u) == gridDim.x - 1);
        __syncthreads();
        if (!s_last) return false;
        __threadfence();
        if (threadIdx.x < K)
            vals[threadIdx.x] = __longlong_as_double((long long)atomicExch(&g->limbs[threadIdx.x][0], 0ull));
        if (threadIdx.x == 0) g->ticket = 0u;
        __syncthreads();
        return true;
    }
};

}  // namespace rbs

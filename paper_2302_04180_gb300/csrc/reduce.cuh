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
    // coop = false after a timed-out staged copy (ERR_TIMEOUT): per-lane flushes
    template <int SCRATCH = FLUSH_SCRATCH, int WARPS = MAX_WARPS>
    __device__ __forceinline__ bool finish(DotScratch *g, double *vals, unsigned nblk = 0u, bool coop = true) {
        return exact_finish<K, Q, SCRATCH, WARPS>(win, flags, sacc, sflags, g, vals, false, nullptr, nullptr, nblk,
                                                  coop);
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
    __device__ __forceinline__ bool finish_export(DotScratch *g, double *vals, long long *limbs, int32_t *fl) {
        flush_low();
        return exact_finish<K, Q>(win, flags, sacc, sflags, g, vals, true, limbs, fl);
    }
};

// Exact reducer for standalone dots of one or two outputs, with the
// per-thread window in shared memory instead of registers: 64-bit carry-save
// digits, W per sign (positive and negative products kept apart, so a product
// adds its five words to five digits picked by address -- no word selects, no
// two's complement). Layout [K][sign][digit][thread], so the lanes of a warp
// touch consecutive words. The window covers W - 4 = 9 placements (288 bits
// of exponent); the product that anchors it lands at placement ANCHOR, with
// 3 placements of headroom above and 5 below (measured best across condition
// numbers 1 to 1e48). A product above it flushes and re-anchors it, one below
// it goes straight into the block accumulator. Digits stay below 2^52 (at most
// 2^20 products per thread per launch, 2^32 each). Blocks of at most 256
// threads.
template <int K_>
struct ExactS {
    static constexpr int K = K_;
    static constexpr int W = 13;
    static constexpr int ANCHOR = 5;  // placement of the product that (re)anchors the window
    static constexpr int NT = 256;
    long long *win;
    int a[K];
    uint32_t flags[K];
    unsigned long long (*sacc)[NL];
    uint32_t *sflags;

    __device__ __forceinline__ void init() {
        __shared__ long long s_win[K * 2 * W * NT];
        __shared__ unsigned long long s_acc[K][NL];
        __shared__ uint32_t s_flags[K];
        win = s_win;
        sacc = s_acc;
        sflags = s_flags;
#pragma unroll
        for (int k = 0; k < K; k++) {
            a[k] = WIN_EMPTY;
            flags[k] = 0u;
#pragma unroll
            for (int j = 0; j < 2 * W; j++) win[(k * 2 * W + j) * NT + threadIdx.x] = 0;
        }
        sacc_zero<K>(sacc, sflags);
    }
    // this thread's window k into the block accumulator, digits back to zero
    __device__ __forceinline__ void flush(int k) {
        if (a[k] < 0) return;
        long long *pp = win + (k * 2 * W) * NT + threadIdx.x, *pn = pp + W * NT;
#pragma unroll
        for (int j = 0; j < W; j++) {
            const long long d = pp[j * NT] - pn[j * NT];
            pp[j * NT] = 0;
            pn[j * NT] = 0;
            if (d) sacc_add(&sacc[k][a[k] + j], d);
        }
    }
    __device__ __forceinline__ void add(int k, double x, double y) {
        uint32_t u[5], m;
        int L;
        if (!prod_exact(x, y, flags[k], u, L, m)) return;
        int q = L - a[k];
        if ((unsigned)q > (unsigned)(W - 5)) {
            if (q < 0) {  // below the window (never for an empty one: its anchor is far below)
                smem_deposit(sacc[k], u, L, m);
                return;
            }
            flush(k);
            a[k] = L - ANCHOR < 0 ? 0 : L - ANCHOR;
            q = L - a[k];
        }
        long long *p = win + ((k * 2 + (int)(m & 1u)) * W + q) * NT + threadIdx.x;
#pragma unroll
        for (int j = 0; j < 5; j++) p[j * NT] += (long long)u[j];
    }
    // Warp-cooperative flush of every lane's window k at the end of the kernel
    // (all 32 lanes call it; the digits are left as they are). The lanes'
    // windows usually sit on the same limbs, so per-lane atomics would collide
    // 32 ways. When every non-empty window has the same anchor, each digit is
    // summed over the warp with shuffles (each lane reads its own digits:
    // conflict-free) and lane j adds digit j's sum with one atomic. Otherwise,
    // with anchors at most 32 - W limbs apart, lane j sums every lane's digit
    // of limb lo + j from shared memory; wider spreads flush per lane.
    __device__ __forceinline__ void flush_warp(int k) {
        const unsigned FULL = 0xffffffffu;
        const int lane = threadIdx.x & 31;
        const bool has = a[k] >= 0;
        const int lo = (int)__reduce_min_sync(FULL, (unsigned)(has ? a[k] : 0x7fffffff));
        const int hi = (int)__reduce_max_sync(FULL, (unsigned)(has ? a[k] : 0));
        if (lo == 0x7fffffff) return;
        if (lo == hi) {
            const long long *pp = win + (k * 2 * W) * NT + threadIdx.x, *pn = pp + W * NT;
            long long mine = 0;
#pragma unroll
            for (int j = 0; j < W; j++) {
                long long d = has ? pp[j * NT] - pn[j * NT] : 0;  // |d| < 2^52: the warp sum < 2^57
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(FULL, d, o);
                if (lane == j) mine = d;
            }
            if (lane < W && mine && lo + lane < NL) sacc_add(&sacc[k][lo + lane], mine);
            a[k] = WIN_EMPTY;
            return;
        }
        if (hi - lo > 32 - W) {
            flush(k);
            return;
        }
        const long long *w0 = win + (k * 2 * W) * NT + (threadIdx.x & ~31);
        long long sum = 0;
        for (int l = 0; l < 32; l++) {
            const int al = __shfl_sync(FULL, a[k], l);
            const int j = lo + lane - al;
            if (al >= 0 && j >= 0 && j < W) sum += w0[j * NT + l] - w0[(W + j) * NT + l];
        }
        if (sum && lo + lane < NL) sacc_add(&sacc[k][lo + lane], sum);
        a[k] = WIN_EMPTY;
    }
    template <int SCRATCH = 0>
    __device__ __forceinline__ bool finish(DotScratch *g, double *vals) {
#pragma unroll
        for (int k = 0; k < K; k++) flush_warp(k);
        return block_grid_finish<K>(flags, sacc, sflags, g, vals);
    }
    __device__ __forceinline__ bool finish_export(DotScratch *g, double *vals, long long *limbs, int32_t *fl) {
#pragma unroll
        for (int k = 0; k < K; k++) flush_warp(k);
        return block_grid_finish<K>(flags, sacc, sflags, g, vals, true, limbs, fl);
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
    template <int SCRATCH = 0, int WARPS = MAX_WARPS>
    __device__ __forceinline__ bool finish(DotScratch *g, double *vals, unsigned nblk = 0u, bool coop = true) {
        (void)coop;  // its partials live in their own shared array
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
        if (threadIdx.x == 0) s_last = (atomicAdd(&g->ticket, 1u) == (nblk ? nblk : gridDim.x) - 1);
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

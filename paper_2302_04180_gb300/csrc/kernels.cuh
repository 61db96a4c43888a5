// Kernel-side helpers shared by the translation units: CSR view, the
// fma-ordered row product, pair-wise vector traversal.
#pragma once

#include <cuda_pipeline.h>

#include "reduce.cuh"

namespace rbs {

struct CSRView {
    int64_t n, nnz;
    const int64_t *rowptr;
    const int32_t *col;
    const double *val;
};

// One CSR row in stored order, starting from +0.0, each step one fma rounded
// to nearest even (Sec. 4.1 SpMV with the fma rule of Sec. 3.3). Every index
// is checked; a bad one is skipped and reported through `bad`.
__device__ __forceinline__ double spmv_row(const CSRView &A, int64_t i, const double *__restrict__ x,
                                           bool &bad) {
    const int64_t b = A.rowptr[i], e = A.rowptr[i + 1];
    double acc = 0.0;
    if (b < 0 || e < b || e > A.nnz) {
        bad = true;
        return acc;
    }
    for (int64_t k = b; k < e; k++) {
        const int32_t c = A.col[k];
        if ((uint64_t)(int64_t)c >= (uint64_t)A.n) {
            bad = true;
            continue;
        }
        acc = fma(A.val[k], __ldg(x + c), acc);
    }
    return acc;
}

// Warp-staged SpMV: each warp walks chunks of 32 consecutive rows. A chunk's
// contiguous nonzero span (col, val) is copied into the warp's shared memory
// with coalesced asynchronous copies, then every lane runs its own row: it
// issues the x gathers of up to 8 entries at once, then the fma chain in stored
// order. The walk is software-pipelined three chunks deep: the row pointers of
// chunk c+2 are loading and the operands of chunk c+1 are copying (second
// buffer) while chunk c computes. The arithmetic is exactly spmv_row's; only
// the memory schedule differs. Spans longer than SPMV_CAP (or malformed row
// pointers) take the per-lane path. fn(row, y_row) runs in the owning lane.
// All 32 lanes of every warp must enter; blocks have at most MAX_WARPS warps.
constexpr int SPMV_CAP = 256;
constexpr int SPMV_BUF = SPMV_CAP * (sizeof(int32_t) + sizeof(double));  // 3 KB per buffer

struct SpmvChunk {
    long long B;  // first nonzero of the chunk
    int span;     // nonzeros in the chunk
    bool staged;  // operands are in shared memory
};

// Prepare chunk rb (row pointers b, e of this lane's row already loaded):
// decide whether it can be staged and issue its copies into buffer `buf`.
// Always commits one copy group, so group counting stays uniform.
__device__ __forceinline__ SpmvChunk spmv_prepare(const CSRView &A, int64_t rb, long long b, long long e,
                                                  unsigned char *buf) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    SpmvChunk c{0, 0, false};
    if (rb < A.n) {
        const bool live = rb + lane < A.n;
        const int last = (int)((A.n - 1 - rb) < 31 ? (A.n - 1 - rb) : 31);
        const long long B = __shfl_sync(FULL, b, 0);
        const long long E = __shfl_sync(FULL, e, last);
        const bool ok = !live || (b >= B && e >= b && e <= E);
        const long long span = E - B;
        c.B = B;
        c.span = (int)(span > 0 && span <= SPMV_CAP ? span : 0);
        c.staged = __all_sync(FULL, ok) && B >= 0 && E <= A.nnz && span >= 0 && span <= SPMV_CAP;
        if (c.staged) {
            int32_t *scol = reinterpret_cast<int32_t *>(buf);
            double *sval = reinterpret_cast<double *>(buf + SPMV_CAP * sizeof(int32_t));
            for (int t = lane; t < c.span; t += 32) {
                __pipeline_memcpy_async(scol + t, A.col + B + t, sizeof(int32_t));
                __pipeline_memcpy_async(sval + t, A.val + B + t, sizeof(double));
            }
        }
    }
    __pipeline_commit();
    return c;
}

template <class F>
__device__ __forceinline__ void spmv_warp_rows(const CSRView &A, const double *__restrict__ x, bool &bad,
                                               F &&fn) {
    static_assert(2 * SPMV_BUF <= WARP_SCRATCH, "warp scratch");
    const int lane = threadIdx.x & 31;
    const int64_t step = (int64_t)gridDim.x * (blockDim.x >> 5) * 32;
    int64_t rb = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    unsigned char *bufs = warp_scratch();
    auto rowptrs = [&](int64_t r0, long long &b, long long &e) {
        const int64_t r = r0 + lane;
        b = 0;
        e = 0;
        if (r0 < A.n && r < A.n) {
            b = A.rowptr[r];
            e = A.rowptr[r + 1];
        }
    };
    long long b0, e0, b1, e1, b2, e2;
    rowptrs(rb, b0, e0);
    SpmvChunk c0 = spmv_prepare(A, rb, b0, e0, bufs);
    rowptrs(rb + step, b1, e1);
    int cur = 0;
    for (; rb < A.n; rb += step) {
        const SpmvChunk c1 = spmv_prepare(A, rb + step, b1, e1, bufs + (cur ^ 1) * SPMV_BUF);
        rowptrs(rb + 2 * step, b2, e2);
        __pipeline_wait_prior(1);  // chunk rb's copies have landed
        __syncwarp();
        const int64_t r = rb + lane;
        if (r < A.n) {
            double acc = 0.0;
            if (c0.staged) {
                const int32_t *scol = reinterpret_cast<const int32_t *>(bufs + cur * SPMV_BUF);
                const double *sval =
                    reinterpret_cast<const double *>(bufs + cur * SPMV_BUF + SPMV_CAP * sizeof(int32_t));
                const int lo = (int)(b0 - c0.B), hi = (int)(e0 - c0.B);
                for (int k0 = lo; k0 < hi; k0 += 8) {
                    // all gathers first (up to 8 in flight), then the chain in
                    // stored order; values and indices are re-read from shared
                    // memory so only the gathered x stay in registers
                    double xv[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        xv[j] = 0.0;
                        if (k0 + j < hi) {
                            const int32_t cidx = scol[k0 + j];
                            if ((uint64_t)(int64_t)cidx < (uint64_t)A.n) xv[j] = __ldg(x + cidx);
                            else bad = true;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (k0 + j < hi && (uint64_t)(int64_t)scol[k0 + j] < (uint64_t)A.n)
                            acc = fma(sval[k0 + j], xv[j], acc);
                }
            } else {
                acc = spmv_row(A, r, x, bad);
            }
            fn(r, acc);
        }
        __syncwarp();  // buffer `cur` is refilled two chunks later
        c0 = c1;
        b0 = b1;
        e0 = e1;
        b1 = b2;
        e1 = e2;
        cur ^= 1;
    }
    __pipeline_wait_prior(0);
    __syncwarp();
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// Row traversal of y = A x with epilogue fn(row, y_row): mode 0 warp-staged,
// mode 1 one thread per row. Same bits either way.
template <class F>
__device__ __forceinline__ void spmv_each(const CSRView &A, const double *__restrict__ x, int mode, bool &bad,
                                          F &&fn) {
    if (mode == 0) {
        spmv_warp_rows(A, x, bad, fn);
    } else {
        for (int64_t i = gtid(); i < A.n; i += gstride()) fn(i, spmv_row(A, i, x, bad));
    }
}

__device__ __forceinline__ double2 ld2(const double *p, int64_t i) {
    return *reinterpret_cast<const double2 *>(p + i);
}
__device__ __forceinline__ void st2(double *p, int64_t i, double2 v) {
    *reinterpret_cast<double2 *>(p + i) = v;
}

// Visit element pairs (2j, 2j+1) with 16-byte accesses, then the odd tail
// element in one thread. f(i, pair) handles element i (and i+1 if pair).
template <class F>
__device__ __forceinline__ void for_pairs(int64_t n, F &&f) {
    const int64_t n2 = n >> 1;
    for (int64_t j = gtid(); j < n2; j += gstride()) f(2 * j, true);
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) f(n - 1, false);
}

}  // namespace rbs

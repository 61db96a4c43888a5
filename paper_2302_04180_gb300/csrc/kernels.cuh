// Kernel-side helpers shared by the translation units: CSR view, the
// fma-ordered row product, pair-wise vector traversal.
#pragma once

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

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

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

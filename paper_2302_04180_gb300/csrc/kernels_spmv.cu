// Standalone SpMV kernels (short rows warp-staged, long rows register-staged,
// one thread per row), Jacobi and the CSR structure check.
#include <mutex>

#include "kernels.cuh"
#include "launch.h"

namespace rbs {

// y = A x (Sec. 4.1), warp-staged rows (mode 0) or one thread per row (mode
// 1) in a grid-stride loop. CHECKED: every index is range-checked (the
// standalone product); without it the solver has validated the structure at
// set-up. With a solver state, the kernel is a no-op once the solver stopped.
template <bool CHECKED, int CAP>
__global__ void __launch_bounds__(256, 3)
    k_spmv(CSRView A, const double *__restrict__ x, double *__restrict__ y, const SolverState *st, unsigned *err,
           int mode) {
    if (st && st->done) return;
    unsigned eb = 0u;
    spmv_each<CHECKED, CAP>(A, x, nullptr, mode, eb, [&](int64_t i, double v, double) { y[i] = v; });
    if (eb) atomicOr(err, eb);
}

// y = A x for long rows (mode 3): register-staged chunks (spmv_rows_reg) in
// 4-warp blocks, three resident per SM.
template <bool CHECKED>
__global__ void __launch_bounds__(SPMV_REG_WARPS * 32, 3)
    k_spmv_reg(CSRView A, const double *__restrict__ x, double *__restrict__ y, const SolverState *st,
               unsigned *err, int mode) {
    if (st && st->done) return;
    unsigned eb = 0u;
    spmv_rows_reg<CHECKED, SPMV_CAP_LONG, false>(
        A, 0, A.n, (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), (int64_t)gridDim.x * (blockDim.x >> 5),
        x, nullptr, true, (mode & SPMV_TEST_STALL) != 0, eb, [&](int64_t i, double v, double) { y[i] = v; });
    if (eb) atomicOr(err, eb);
}

static CSRView view(const CSRArgs &A) { return CSRView{A.n, A.nnz, A.rowptr, A.col, A.val}; }

static void spmv_carveout(int c) {
    static std::mutex mu;
    static int applied[64];
    static bool init = false;
    std::lock_guard<std::mutex> lk(mu);
    if (!init) {
        for (int i = 0; i < 64; i++) applied[i] = -2;
        init = true;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && applied[dev] != c) {
        cudaFuncSetAttribute(k_spmv<true, SPMV_CAP_SHORT>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
        cudaFuncSetAttribute(k_spmv<false, SPMV_CAP_SHORT>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
        // the long-row kernel needs all of it, whatever the knob says
        cudaFuncSetAttribute(k_spmv_reg<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_spmv_reg<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaGetLastError();
        applied[dev] = c;
    }
}

// Resident blocks per SM of the SpMV kernel of `mode` at this block size (the
// long-row kernel: at its own block of SPMV_REG_WARPS warps).
int spmv_blocks_per_sm(int block, int carveout, int mode) {
    spmv_carveout(carveout);
    int nb = 0;
    const cudaError_t e = mode == SPMV_MODE_LONG
                              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_reg<true>, SPMV_REG_WARPS * 32, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv<true, SPMV_CAP_SHORT>, block, 0);
    if (e != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

// The long-row kernel runs its own launch shape: blocks of SPMV_REG_WARPS
// warps, all of them resident (cfg's grid and block are not used).
static Cfg spmv_reg_cfg(int64_t n, int carveout) {
    static std::mutex mu;
    static int sms[64], bps[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int nsm, nb;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!sms[dev]) {
            int v = 0;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
                cudaGetLastError();
                v = 1;
            }
            bps[dev] = spmv_blocks_per_sm(SPMV_REG_WARPS * 32, carveout, SPMV_MODE_LONG);
            sms[dev] = v;
        }
        nsm = sms[dev];
        nb = bps[dev];
    }
    Cfg c;
    c.block = SPMV_REG_WARPS * 32;
    const int64_t need = (n + c.block - 1) / c.block, cap = (int64_t)nsm * nb;
    c.grid = (int)(need < 1 ? 1 : (need < cap ? need : cap));
    return c;
}

cudaError_t launch_spmv(const CSRArgs &A, const double *x, double *y, const SolverState *st,
                        unsigned *err, Cfg cfg, cudaStream_t s) {
    spmv_carveout(cfg.carveout);
    if ((cfg.mode & SPMV_MODE_MASK) == SPMV_MODE_LONG) {
        const Cfg r = spmv_reg_cfg(A.n, cfg.carveout);
        if (st) k_spmv_reg<false><<<r.grid, r.block, 0, s>>>(view(A), x, y, st, err, cfg.mode);
        else k_spmv_reg<true><<<r.grid, r.block, 0, s>>>(view(A), x, y, st, err, cfg.mode);
    } else if (st) {
        k_spmv<false, SPMV_CAP_SHORT><<<cfg.grid, cfg.block, 0, s>>>(view(A), x, y, st, err, cfg.mode);
    } else {
        k_spmv<true, SPMV_CAP_SHORT><<<cfg.grid, cfg.block, 0, s>>>(view(A), x, y, st, err, cfg.mode);
    }
    return cudaGetLastError();
}

// invd_i = RN(1 / d_i) with d the given diagonal or the first stored (i, i)
// entry (Sec. 4, Jacobi M = diag(A)); a zero, NaN or missing entry sets err bit 2.
__global__ void __launch_bounds__(256) k_jacobi_invd(CSRView A, const double *diag, double *invd, unsigned *err) {
    bool bad = false, idx_bad = false;
    for (int64_t i = gtid(); i < A.n; i += gstride()) {
        double d = 0.0;
        bool found = false;
        if (diag) {
            d = diag[i];
            found = true;
        } else {
            const int64_t b = A.rowptr[i], e = A.rowptr[i + 1];
            if (b < 0 || e < b || e > A.nnz) {
                idx_bad = true;
            } else {
                for (int64_t k = b; k < e; k++)
                    if ((int64_t)A.col[k] == i) {
                        d = A.val[k];
                        found = true;
                        break;
                    }
            }
        }
        if (!found || d == 0.0 || d != d) {
            bad = true;
            invd[i] = 0.0;
        } else {
            invd[i] = __ddiv_rn(1.0, d);
        }
    }
    if (bad) atomicOr(err, 2u);
    if (idx_bad) atomicOr(err, 1u);
}

cudaError_t launch_jacobi_invd(const CSRArgs &A, const double *diag, double *invd, unsigned *err, Cfg cfg,
                               cudaStream_t s) {
    k_jacobi_invd<<<cfg.grid, cfg.block, 0, s>>>(view(A), diag, invd, err);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_jacobi_apply(int64_t n, const double *invd, const double *p,
                                                     double *phat) {
    for (int64_t i = gtid(); i < n; i += gstride()) phat[i] = __dmul_rn(p[i], invd[i]);
}

cudaError_t launch_jacobi_apply(int64_t n, const double *invd, const double *p, double *phat, Cfg cfg,
                                cudaStream_t s) {
    k_jacobi_apply<<<cfg.grid, cfg.block, 0, s>>>(n, invd, p, phat);
    return cudaGetLastError();
}

// CSR structure check: rowptr[0] == 0, non-decreasing, rowptr[n] == nnz,
// 0 <= col < n. Sets err bit 1 on any violation.
__global__ void __launch_bounds__(256) k_csr_check(CSRView A, unsigned *err) {
    bool bad = false;
    if (gtid() == 0 && (A.rowptr[0] != 0 || A.rowptr[A.n] != A.nnz)) bad = true;
    for (int64_t i = gtid(); i < A.n; i += gstride())
        if (A.rowptr[i + 1] < A.rowptr[i]) bad = true;
    for (int64_t k = gtid(); k < A.nnz; k += gstride())
        if ((uint64_t)(int64_t)A.col[k] >= (uint64_t)A.n) bad = true;
    if (bad) atomicOr(err, 1u);
}

cudaError_t launch_csr_check(const CSRArgs &A, unsigned *err, Cfg cfg, cudaStream_t s) {
    k_csr_check<<<cfg.grid, cfg.block, 0, s>>>(view(A), err);
    return cudaGetLastError();
}

}  // namespace rbs

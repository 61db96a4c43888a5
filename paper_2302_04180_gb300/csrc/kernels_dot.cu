// Standalone kernels: exact dot (single and multi-output), long-accumulator
// export and rounding, fma-ordered SpMV, Jacobi, CSR validation.
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "kernels.cuh"
#include "launch.h"

namespace rbs {

template <int K>
struct DotArgs {
    const double *x[K];
    const double *y[K];
};

// K exact dots over the same length (Sec. 2 exdot; Sec. 4.1/4.2 merged
// reductions). Aligned operands go through 16-byte loads, two pairs deep (long
// dots of one or two outputs: the next two pairs in flight while these add).
// SMEM: one or two outputs keep their windows in shared memory (ExactS: fewer
// integer operations per product, dearer to clear and flush per thread); long
// dots take it, short ones and more outputs keep register windows (ExactR2).
template <int K, int Q, bool SMEM>
using ExdotRed = typename std::conditional<(SMEM && K <= 2), ExactS<K>, ExactR2<K, Q>>::type;
constexpr int64_t EXDOT_SMEM_MIN_N = 1LL << 23;  // measured crossover on GB300

template <int K, int Q, bool EXPORT, bool SMEM>
__global__ void __launch_bounds__(256) k_exdot(DotArgs<K> a, int64_t n, bool aligned, DotScratch *g,
                                              double *out, long long *limbs, int32_t *flags_out) {
    ExdotRed<K, Q, SMEM> red;
    red.init();
    if (aligned && SMEM && K <= 2) {
        // long dots (shared-memory windows): the next iteration's four pairs
        // load while this one's are added, so that the stream does not stop
        // for the products (2^27: 427 -> 400 us; the register-window reducer
        // of shorter dots measured slower this way and keeps the loop below)
        const int64_t n2 = n >> 1, st = gstride();
        int64_t j = gtid();
        if (j + st < n2) {
            double2 xa[K], ya[K], xb[K], yb[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                xa[k] = __ldcs(reinterpret_cast<const double2 *>(a.x[k]) + j);
                ya[k] = __ldcs(reinterpret_cast<const double2 *>(a.y[k]) + j);
                xb[k] = __ldcs(reinterpret_cast<const double2 *>(a.x[k]) + j + st);
                yb[k] = __ldcs(reinterpret_cast<const double2 *>(a.y[k]) + j + st);
            }
            for (;;) {
                const int64_t jn = j + 2 * st;
                const bool more = jn + st < n2;
                double2 xc[K], yc[K], xd[K], yd[K];
                if (more) {
#pragma unroll
                    for (int k = 0; k < K; k++) {
                        xc[k] = __ldcs(reinterpret_cast<const double2 *>(a.x[k]) + jn);
                        yc[k] = __ldcs(reinterpret_cast<const double2 *>(a.y[k]) + jn);
                        xd[k] = __ldcs(reinterpret_cast<const double2 *>(a.x[k]) + jn + st);
                        yd[k] = __ldcs(reinterpret_cast<const double2 *>(a.y[k]) + jn + st);
                    }
                }
#pragma unroll
                for (int k = 0; k < K; k++) {
                    red.add(k, xa[k].x, ya[k].x);
                    red.add(k, xa[k].y, ya[k].y);
                    red.add(k, xb[k].x, yb[k].x);
                    red.add(k, xb[k].y, yb[k].y);
                }
                j = jn;
                if (!more) break;
#pragma unroll
                for (int k = 0; k < K; k++) {
                    xa[k] = xc[k];
                    ya[k] = yc[k];
                    xb[k] = xd[k];
                    yb[k] = yd[k];
                }
            }
        }
        if (j < n2) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                const double2 xv = __ldcs(reinterpret_cast<const double2 *>(a.x[k]) + j);
                const double2 yv = __ldcs(reinterpret_cast<const double2 *>(a.y[k]) + j);
                red.add(k, xv.x, yv.x);
                red.add(k, xv.y, yv.y);
            }
        }
        if ((n & 1) && gtid() == 0) {
#pragma unroll
            for (int k = 0; k < K; k++) red.add(k, a.x[k][n - 1], a.y[k][n - 1]);
        }
    } else if (aligned) {
        const int64_t n2 = n >> 1, st = gstride();
        int64_t j = gtid();
        for (; j + st < n2; j += 2 * st) {
            double2 xa[K], ya[K], xb[K], yb[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                xa[k] = __ldcs(reinterpret_cast<const double2 *>(a.x[k]) + j);
                ya[k] = __ldcs(reinterpret_cast<const double2 *>(a.y[k]) + j);
                xb[k] = __ldcs(reinterpret_cast<const double2 *>(a.x[k]) + j + st);
                yb[k] = __ldcs(reinterpret_cast<const double2 *>(a.y[k]) + j + st);
            }
#pragma unroll
            for (int k = 0; k < K; k++) {
                red.add(k, xa[k].x, ya[k].x);
                red.add(k, xa[k].y, ya[k].y);
                red.add(k, xb[k].x, yb[k].x);
                red.add(k, xb[k].y, yb[k].y);
            }
        }
        if (j < n2) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                const double2 xv = __ldcs(reinterpret_cast<const double2 *>(a.x[k]) + j);
                const double2 yv = __ldcs(reinterpret_cast<const double2 *>(a.y[k]) + j);
                red.add(k, xv.x, yv.x);
                red.add(k, xv.y, yv.y);
            }
        }
        if ((n & 1) && gtid() == 0) {
#pragma unroll
            for (int k = 0; k < K; k++) red.add(k, a.x[k][n - 1], a.y[k][n - 1]);
        }
    } else {
        for (int64_t i = gtid(); i < n; i += gstride()) {
#pragma unroll
            for (int k = 0; k < K; k++) red.add(k, a.x[k][i], a.y[k][i]);
        }
    }
    __shared__ double vals[K];
    if (EXPORT) {
        red.finish_export(g, vals, limbs, flags_out);
    } else {
        if (red.finish(g, vals) && threadIdx.x < K) out[threadIdx.x] = vals[threadIdx.x];
    }
}

template <int K, int Q>
static cudaError_t exdot_k(const double *const *xs, const double *const *ys, int64_t n, DotScratch *g,
                           double *out, Cfg cfg, cudaStream_t s) {
    DotArgs<K> a;
    bool aligned = true;
    for (int k = 0; k < K; k++) {
        a.x[k] = xs[k];
        a.y[k] = ys[k];
        aligned = aligned && ((uintptr_t)xs[k] % 16 == 0) && ((uintptr_t)ys[k] % 16 == 0);
    }
    if (K <= 2 && n >= EXDOT_SMEM_MIN_N)
        k_exdot<K, Q, false, true><<<cfg.grid, cfg.block, 0, s>>>(a, n, aligned, g, out, nullptr, nullptr);
    else
        k_exdot<K, Q, false, false><<<cfg.grid, cfg.block, 0, s>>>(a, n, aligned, g, out, nullptr, nullptr);
    return cudaGetLastError();
}

template <int Q>
static cudaError_t exdot_q(int k, const double *const *xs, const double *const *ys, int64_t n,
                           DotScratch *g, double *out, Cfg cfg, cudaStream_t s) {
    switch (k) {
        case 1: return exdot_k<1, Q>(xs, ys, n, g, out, cfg, s);
        case 2: return exdot_k<2, Q>(xs, ys, n, g, out, cfg, s);
        case 3: return exdot_k<3, Q>(xs, ys, n, g, out, cfg, s);
        case 4: return exdot_k<4, Q>(xs, ys, n, g, out, cfg, s);
        case 5: return exdot_k<5, Q>(xs, ys, n, g, out, cfg, s);
        case 6: return exdot_k<6, Q>(xs, ys, n, g, out, cfg, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int Q, bool SMEM>
static int exdot_occ_q(int k, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (k) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_exdot<1, Q, false, SMEM>, block, 0); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_exdot<2, Q, false, SMEM>, block, 0); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_exdot<3, Q, false, false>, block, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_exdot<4, Q, false, false>, block, 0); break;
        case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_exdot<5, Q, false, false>, block, 0); break;
        case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_exdot<6, Q, false, false>, block, 0); break;
        default: break;
    }
    if (e != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

// Cached per device and kernel variant: the query costs a few microseconds of
// host time, which a short dot would otherwise pay on every call.
int exdot_blocks_per_sm(int k, int window, int block, int64_t n) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, bool>, int> cache;
    const bool smem = k <= 2 && n >= EXDOT_SMEM_MIN_N;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    const auto key = std::make_tuple(dev, k, window, block, smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        const auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int nb;
    if (window == 2) nb = smem ? exdot_occ_q<2, true>(k, block) : exdot_occ_q<2, false>(k, block);
    else if (window == 1) nb = smem ? exdot_occ_q<1, true>(k, block) : exdot_occ_q<1, false>(k, block);
    else nb = smem ? exdot_occ_q<4, true>(k, block) : exdot_occ_q<4, false>(k, block);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = nb;
    return nb;
}

cudaError_t launch_exdot(int k, const double *const *xs, const double *const *ys, int64_t n,
                         DotScratch *g, double *out, int window, Cfg cfg, cudaStream_t s) {
    if (window == 2) return exdot_q<2>(k, xs, ys, n, g, out, cfg, s);
    if (window == 1) return exdot_q<1>(k, xs, ys, n, g, out, cfg, s);
    return exdot_q<4>(k, xs, ys, n, g, out, cfg, s);
}

cudaError_t launch_exdot_partial(const double *x, const double *y, int64_t n, DotScratch *g,
                                 int64_t *limbs, int32_t *flags, int window, Cfg cfg, cudaStream_t s) {
    (void)window;
    DotArgs<1> a;
    a.x[0] = x;
    a.y[0] = y;
    const bool aligned = ((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0);
    if (n >= EXDOT_SMEM_MIN_N)
        k_exdot<1, 4, true, true><<<cfg.grid, cfg.block, 0, s>>>(a, n, aligned, g, nullptr, (long long *)limbs,
                                                              flags);
    else
        k_exdot<1, 4, true, false><<<cfg.grid, cfg.block, 0, s>>>(a, n, aligned, g, nullptr, (long long *)limbs,
                                                               flags);
    return cudaGetLastError();
}

__global__ void k_round_limbs(const int64_t *limbs, const int32_t *flags, double *out) {
    __shared__ long long G[NL];
    for (int j = threadIdx.x; j < NL; j += blockDim.x) G[j] = (long long)limbs[j];
    __syncthreads();
    if (threadIdx.x == 0) *out = round_limbs_thread(G, (uint32_t)*flags);
}

cudaError_t launch_round_limbs(const int64_t *limbs, const int32_t *flags, double *out, cudaStream_t s) {
    k_round_limbs<<<1, 160, 0, s>>>(limbs, flags, out);
    return cudaGetLastError();
}

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

// ---- allocation-free exact dot ---------------------------------------------------
//
// rbs_exdot_noalloc runs the same exact-dot kernel as rbs_exdot_multi, but keeps
// its only scratch -- the cross-block long accumulators, flags and ticket --
// in the file-scope device array below instead of the per-stream workspace, so
// it never allocates device or pinned host memory. It serves callers that
// cannot allocate at the point of the call: code running while a CUDA graph is
// being captured (a cudaMalloc is not a capturable step), latency-critical
// loops that cannot afford the implicit device synchronisation of an
// allocation, and applications whose own memory pool owns the device memory.
//
// The array is 8 KiB and holds at most RBS_NOALLOC_MAX_DOTS accumulators.
// Every GPU that loads this library keeps the array until the process exits.
// All calls on a device share it, so calls that overlap on the GPU (for
// example on two streams at once) race and must be ordered by the caller.
namespace rbs {
namespace {

constexpr size_t NOALLOC_BYTES = 8192;
static_assert(sizeof(DotScratch) <= NOALLOC_BYTES, "scratch array too small");
static_assert(RBS_NOALLOC_MAX_DOTS == KMAX, "accumulator count");

static __device__ __align__(256) unsigned char noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex noalloc_mu;
void *noalloc_ptr[NOALLOC_MAX_DEVICES];
int noalloc_sms[NOALLOC_MAX_DEVICES];

// Set-up, once per device, with that device current: the array's device
// address (in host code its name is only a host-side stand-in), a one-time
// clear, and the SM count for the launch shape.
int noalloc_setup(int dev, void **ptr, int *sms) {
    std::lock_guard<std::mutex> lk(noalloc_mu);
    if (!noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
        if (e != cudaSuccess) return set_error(RBS_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return set_error(RBS_ECUDA, "cudaDeviceGetAttribute failed");
        e = cudaMemset(p, 0, NOALLOC_BYTES);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return set_error(RBS_ECUDA, "clearing the no-alloc scratch failed");
        noalloc_sms[dev] = n;
        noalloc_ptr[dev] = p;
    }
    *ptr = noalloc_ptr[dev];
    *sms = noalloc_sms[dev];
    return RBS_OK;
}

bool device_resident(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace rbs

extern "C" int rbs_exdot_noalloc(int k, const double *const *xs, const double *const *ys, int64_t n,
                                 double *out, void *stream) {
    using namespace rbs;
    if (k < 1 || k > RBS_NOALLOC_MAX_DOTS)
        return set_error(RBS_EINVAL, "rbs_exdot_noalloc: k must be 1..RBS_NOALLOC_MAX_DOTS (6), the "
                                     "accumulators its fixed scratch array holds");
    if (n < 0 || !xs || !ys || !out) return set_error(RBS_EINVAL, "rbs_exdot_noalloc: bad argument");
    if (!device_resident(out)) return set_error(RBS_EINVAL, "rbs_exdot_noalloc: out must be device memory");
    for (int j = 0; j < k; j++)
        if (n > 0 && (!xs[j] || !ys[j] || !device_resident(xs[j]) || !device_resident(ys[j])))
            return set_error(RBS_EINVAL, "rbs_exdot_noalloc: operands must be device memory");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(RBS_ECUDA, "rbs_exdot_noalloc: no usable current device");
    void *p = nullptr;
    int sms = 0;
    int rc = noalloc_setup(dev, &p, &sms);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the shared array keeps the last call's contents: clear it first
    if (cudaMemsetAsync(p, 0, sizeof(DotScratch), s) != cudaSuccess)
        return set_error(RBS_ECUDA, "rbs_exdot_noalloc: cudaMemsetAsync failed");
    if (n == 0) {
        if (cudaMemsetAsync(out, 0, k * sizeof(double), s) != cudaSuccess)
            return set_error(RBS_ECUDA, "rbs_exdot_noalloc: cudaMemsetAsync failed");
        return RBS_OK;
    }
    Cfg c;
    c.block = 256;
    int64_t g = (n + 2LL * c.block - 1) / (2LL * c.block);
    const int64_t cap = (int64_t)sms * exdot_blocks_per_sm(k, 4, c.block, n);  // whole waves
    g = g < 1 ? 1 : (g < cap ? g : cap);
    const int64_t minimum = (n + ((int64_t)c.block << 20) - 1) / ((int64_t)c.block << 20);
    if (g < minimum) g = minimum;
    c.grid = (int)(g > 0x7fffffff ? 0x7fffffff : g);
    cudaError_t e = exdot_q<4>(k, xs, ys, n, reinterpret_cast<DotScratch *>(p), out, c, s);
    if (e != cudaSuccess) return set_error(RBS_ECUDA, "rbs_exdot_noalloc: kernel launch failed");
    return RBS_OK;
}

// ---- lightweight FPE-8 dot (Sec. 3.2) -----------------------------------------------
//
// The paper's lightweight variant: each thread keeps a floating-point
// expansion of at most eight binary64 terms. A product enters as TwoProd's
// r + s (Alg. 2) and each part is added with a cascade of TwoSums (Alg. 1)
// that stops as soon as the carried error is zero (early exit). Where the
// paper rounds the final expansion with NearSum, the terms here go into the
// exact integer accumulator and are rounded once: the same correctly rounded
// value. When a thread would need a ninth term, a TwoProd may be inexact
// (|x*y| below 2^-969, where its error can underflow) or a value is not
// finite, the kernel reports that information could be lost -- the paper's
// warning -- and the entry point falls back to the exact dot.
namespace rbs {

__device__ __forceinline__ void fpe_two_sum(double a, double b, double &r, double &s) {
    r = __dadd_rn(a, b);
    const double z = __dsub_rn(r, a);
    s = __dadd_rn(__dsub_rn(a, __dsub_rn(r, z)), __dsub_rn(b, z));
}

// c += x exactly while at most 8 terms are needed; false if a ninth is needed.
__device__ __forceinline__ bool fpe_add(double (&c)[8], double x) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
        if (x == 0.0) return true;
        double r, s;
        fpe_two_sum(c[k], x, r, s);
        c[k] = r;
        x = s;
    }
    return x == 0.0;
}

__global__ void __launch_bounds__(256) k_fpe_dot(const double *__restrict__ x, const double *__restrict__ y,
                                                 int64_t n, DotScratch *g, double *out, unsigned *lost) {
    ExactR<1, 4> red;
    red.init();
    double c[8];
#pragma unroll
    for (int k = 0; k < 8; k++) c[k] = 0.0;
    bool ok = true;
    for (int64_t i = gtid(); i < n; i += gstride()) {
        const double a = x[i], b = y[i];
        const double r = __dmul_rn(a, b);
        const double s = fma(a, b, -r);
        const double ar = fabs(r);
        if (!finite_d(r) || (ar < 0x1p-969 && (r != 0.0 || (a != 0.0 && b != 0.0)))) {
            ok = false;
            continue;
        }
        ok = fpe_add(c, r) && ok;
        ok = fpe_add(c, s) && ok;
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
        if (!finite_d(c[k])) ok = false;
        else red.add(0, c[k], 1.0);
    }
    if (!ok) atomicOr(lost, 1u);
    __shared__ double vals[1];
    if (red.finish(g, vals) && threadIdx.x == 0) *out = vals[0];
}

int fpe_blocks_per_sm(int block) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fpe_dot, block, 0) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

cudaError_t launch_fpe_dot(const double *x, const double *y, int64_t n, DotScratch *g, double *out,
                           unsigned *lost, Cfg cfg, cudaStream_t s) {
    k_fpe_dot<<<cfg.grid, cfg.block, 0, s>>>(x, y, n, g, out, lost);
    return cudaGetLastError();
}

}  // namespace rbs

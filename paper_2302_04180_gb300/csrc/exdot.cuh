// The standalone exact-dot kernel templates (Sec. 2 exdot; Sec. 4.1/4.2
// merged reductions), their launchers and occupancy queries, per window size
// Q. Each window size is instantiated in one translation unit only
// (kernels_dot.cu: Q = 4, the default; kernels_exdot_w1.cu / _w2.cu: Q = 1, 2),
// so that the three compile in parallel.
#pragma once

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
inline cudaError_t exdot_k(const double *const *xs, const double *const *ys, int64_t n, DotScratch *g,
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
inline cudaError_t exdot_q(int k, const double *const *xs, const double *const *ys, int64_t n,
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
inline int exdot_occ_q(int k, int block) {
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

}  // namespace rbs

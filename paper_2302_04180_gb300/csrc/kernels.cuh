// Kernel-side helpers shared by the translation units: CSR view, the
// fma-ordered row product, pair-wise vector traversal.
#pragma once

#include <cuda_pipeline.h>

#include "launch.h"
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
template <bool L2X = false>
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
        acc = fma(A.val[k], L2X ? __ldcg(x + c) : __ldg(x + c), acc);
    }
    return acc;
}

// Error bits that kernels OR into the workspace error word.
constexpr unsigned ERR_INDEX = 1u;    // an out-of-range CSR index or row pointer
// a bounded wait on an asynchronous copy expired; the kernel's exact windows
// must then be flushed with finish(..., coop = false), which does not use the
// staging buffers as scratch
constexpr unsigned ERR_TIMEOUT = 4u;

// Warp-staged SpMV: each warp walks chunks of 32 consecutive rows. A chunk's
// contiguous nonzero span (col, val), and the chunk's slice of an optional
// companion vector z that the epilogue reads, are copied into the warp's shared
// memory; then every lane runs its own row: it issues the x gathers of up to 8
// entries at once, then the fma chain in stored order. The walk is software-
// pipelined three chunks deep: the row pointers of chunk c+2 are loading and
// the operands of chunk c+1 are copying (second buffer) while chunk c computes.
// (A third buffer measured slower on GB300: the shared memory it takes comes
// out of the L1 that serves the x gathers.)
//
// Copies: a full chunk whose arrays start on 16-byte boundaries is fetched by
// one lane with three bulk asynchronous copies (the span rounded out to whole
// 16-byte units, never past the end of the arrays) that complete on the
// buffer's mbarrier; any other chunk by per-lane 16-byte (or, unaligned,
// element) asynchronous copies. Spans longer than CAP (or, when CHECKED,
// malformed row pointers) take the per-lane unstaged path. With CHECKED every
// index is range-checked and a bad one reported (ERR_INDEX); without it the
// caller has validated the structure (rowptr monotone from 0 to nnz, columns
// in [0, n)). The arithmetic is exactly spmv_row's; only the memory schedule
// differs. fn(row, y_row, z_row) runs in the owning lane (z_row = 0 without z).
// All 32 lanes of every warp must enter; blocks have at most MAX_WARPS warps.
// Kernels that also flush exact windows name SpmvLayout<CAP>::SCRATCH so that
// the flush reuses the same shared buffer.
// Staging layout of one chunk buffer for spans of at most CAP nonzeros: the
// z slice (32 doubles), then val (CAP + 2 for the 16-byte rounding), then col
// (CAP + 8); two buffers per warp. CAP 224 holds 32 rows of a 7-point stencil
// (three 256-thread blocks per SM); CAP 1024 holds 32 rows of up to 32
// nonzeros, e.g. the 27-point stencil (one block per SM).
template <int CAP>
struct SpmvLayout {
    static constexpr int VAL_OFF = 32 * 8;
    static constexpr int COL_OFF = VAL_OFF + (CAP + 2) * 8;
    static constexpr int BUF = (COL_OFF + (CAP + 8) * 4 + 15) / 16 * 16;
    static constexpr int SCRATCH = 2 * BUF;  // per warp
    static_assert(COL_OFF % 16 == 0 && BUF >= COL_OFF + (CAP + 8) * 4, "16-byte units");
    static_assert(SCRATCH >= FLUSH_SCRATCH, "the flush reuses the staging buffers");
};
constexpr int SPMV_CAP_SHORT = 224, SPMV_CAP_LONG = 1024;
constexpr long long SPMV_WAIT_LIMIT = 1LL << 17;  // polls of at most ~10 us: ~1.3 s before ERR_TIMEOUT

// Test mode of the bounded wait (bit SPMV_TEST_STALL of the SpMV mode, a
// kernel argument): the issuing lane announces a chunk's bulk copies on the
// mbarrier without issuing them, and the wait gives up after
// SPMV_TEST_WAIT_LIMIT polls, so that the timeout path runs.
constexpr long long SPMV_TEST_WAIT_LIMIT = 64;  // (SPMV_MODE_MASK, SPMV_TEST_STALL: launch.h)

enum : int { CHUNK_UNSTAGED = 0, CHUNK_LANES = 1, CHUNK_BULK = 2 };

struct SpmvChunk {
    long long B;  // first nonzero of the chunk
    int how;      // CHUNK_*
};

// First val / col element a staged chunk holds: the span rounded down to a
// 16-byte unit for wide copies.
__device__ __forceinline__ long long spmv_va(long long B, bool wide) { return wide ? (B & ~1LL) : B; }
__device__ __forceinline__ long long spmv_ca(long long B, bool wide) { return wide ? (B & ~3LL) : B; }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// One 16-byte asynchronous copy of which the first `src_bytes` are read from
// global memory (the rest of the 16 shared bytes are zero-filled).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, unsigned src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

// mbarrier and bulk-copy primitives (one arrival per phase: the issuing lane's).
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// One bounded poll: returns once the phase of `parity` has completed or after
// at most about 10 us of suspension.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(10000u)
        : "memory");
    return ok != 0u;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Prepare chunk rb (row pointers b, e of this lane's row already loaded):
// decide how it is staged and issue its copies into buffer `buf` (mbarrier
// `bar` for bulk copies). Always commits one cp.async group, so group counting
// stays uniform.
template <bool CHECKED, int CAP>
__device__ __forceinline__ SpmvChunk spmv_prepare(const CSRView &A, int64_t r_end, const double *z, bool wide,
                                                  bool bulk_ok, bool z_bulk, bool skip_bulk, int64_t rb, long long b,
                                                  long long e, unsigned char *buf, unsigned long long *bar) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    SpmvChunk c{0, CHUNK_UNSTAGED};
    if (rb < r_end) {
        const bool live = rb + lane < r_end;
        const int last = (int)((r_end - 1 - rb) < 31 ? (r_end - 1 - rb) : 31);
        const long long B = __shfl_sync(FULL, b, 0);
        const long long E = __shfl_sync(FULL, e, last);
        const long long span = E - B;
        c.B = B;
        using L = SpmvLayout<CAP>;
        bool ok = span >= 0 && span <= CAP;
        if (CHECKED) ok = __all_sync(FULL, !live || (b >= B && e >= b && e <= E)) && ok && B >= 0 && E <= A.nnz;
        if (ok) {
            double *sval = reinterpret_cast<double *>(buf + L::VAL_OFF);
            int32_t *scol = reinterpret_cast<int32_t *>(buf + L::COL_OFF);
            const long long va = spmv_va(B, wide), ca = spmv_ca(B, wide);
            const long long ve = (E + 1) & ~1LL, ce = (E + 3) & ~3LL;
            if (bulk_ok && last == 31 && ve <= A.nnz && ce <= A.nnz) {
                c.how = CHUNK_BULK;
                if (lane == 0) {
                    const unsigned vbytes = (unsigned)(ve - va) * 8u, cbytes = (unsigned)(ce - ca) * 4u;
                    const unsigned zbytes = z && z_bulk ? 256u : 0u;
                    // earlier generic-proxy reads of this buffer happen before
                    // the bulk copies overwrite it
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    mbar_arrive_expect_tx(bar, vbytes + cbytes + zbytes);
                    if (!skip_bulk) {
                        if (vbytes) bulk_copy_g2s(sval, A.val + va, vbytes, bar);
                        if (cbytes) bulk_copy_g2s(scol, A.col + ca, cbytes, bar);
                        if (zbytes) bulk_copy_g2s(buf, z + rb, 256u, bar);
                    }
                }
                // a z written earlier in the same kernel is copied by the lanes
                // (generic proxy), so that the earlier writes are seen
                if (z && !z_bulk && live)
                    __pipeline_memcpy_async(reinterpret_cast<double *>(buf) + lane, z + rb + lane, 8);
            } else {
                c.how = CHUNK_LANES;
                if (wide) {
                    // 2 vals / 4 cols per unit; the last unit of an array reads
                    // only the elements that exist
                    const int nv = (int)((ve - va) >> 1), nc = (int)((ce - ca) >> 2);
                    for (int u = lane; u < nv; u += 32) {
                        const long long k = va + 2 * u;
                        cp_async16(sval + 2 * u, A.val + k, A.nnz - k >= 2 ? 16u : 8u);
                    }
                    for (int u = lane; u < nc; u += 32) {
                        const long long k = ca + 4 * u;
                        const long long left = A.nnz - k;
                        cp_async16(scol + 4 * u, A.col + k, left >= 4 ? 16u : (unsigned)left * 4u);
                    }
                } else {
                    for (int t = lane; t < (int)span; t += 32) {
                        __pipeline_memcpy_async(scol + t, A.col + B + t, sizeof(int32_t));
                        __pipeline_memcpy_async(sval + t, A.val + B + t, sizeof(double));
                    }
                }
                if (z && live)
                    __pipeline_memcpy_async(reinterpret_cast<double *>(buf) + lane, z + rb + lane, 8);
            }
        }
    }
    __pipeline_commit();
    return c;
}

// Rows [r_begin, r_end) in chunks of 32, chunk k taken by warp k mod nwarps
// (this warp is number `warp` of nwarps). L2X: x is read through L2 only
// (ld.global.cg), for an x that other blocks write in the same kernel; z_bulk:
// z may be fetched by the bulk copy (it is not written in the same kernel).
template <bool CHECKED, int CAP, bool L2X, class F>
__device__ __forceinline__ void spmv_rows(const CSRView &A, int64_t r_begin, int64_t r_end, int64_t warp,
                                          int64_t nwarps, const double *__restrict__ x,
                                          const double *__restrict__ z, bool z_bulk, bool test_stall,
                                          unsigned &err, F &&fn) {
    __shared__ __align__(8) unsigned long long s_bar[MAX_WARPS][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t step = nwarps * 32;
    int64_t rb = r_begin + warp * 32;
    // valid columns are [0, ncol): with CHECKED the largest column of a row is
    // tested once, and every gather stays in range
    const unsigned ncol = A.n < 0x80000000LL ? (unsigned)A.n : 0x80000000u;
    const bool wide = ((reinterpret_cast<uintptr_t>(A.col) | reinterpret_cast<uintptr_t>(A.val)) & 15) == 0;
    const bool bulk_ok = wide && (!z_bulk || (reinterpret_cast<uintptr_t>(z) & 15) == 0);
    using L = SpmvLayout<CAP>;
    unsigned char *bufs = warp_scratch<L::SCRATCH>();
    unsigned long long *bars = s_bar[wid];
    if (lane == 0) {
        mbar_init(bars);
        mbar_init(bars + 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncwarp();
    unsigned parity = 0u;  // bit k: phase of buffer k's barrier to wait for
    const long long wait_limit = test_stall ? SPMV_TEST_WAIT_LIMIT : SPMV_WAIT_LIMIT;
    const bool skip_bulk = test_stall;
    auto rowptrs = [&](int64_t r0, long long &b, long long &e) {
        const int64_t r = r0 + lane;
        b = 0;
        e = 0;
        if (r0 < r_end && r < r_end) {
            b = A.rowptr[r];
            e = A.rowptr[r + 1];
        }
    };
    long long b0, e0, b1, e1, b2, e2;
    rowptrs(rb, b0, e0);
    SpmvChunk c0 = spmv_prepare<CHECKED, CAP>(A, r_end, z, wide, bulk_ok, z_bulk, skip_bulk, rb, b0, e0, bufs, bars);
    rowptrs(rb + step, b1, e1);
    int cur = 0;
    SpmvChunk c1{0, CHUNK_UNSTAGED};
    for (; rb < r_end; rb += step) {
        c1 = spmv_prepare<CHECKED, CAP>(A, r_end, z, wide, bulk_ok, z_bulk, skip_bulk, rb + step, b1, e1,
                                        bufs + (cur ^ 1) * L::BUF, bars + (cur ^ 1));
        rowptrs(rb + 2 * step, b2, e2);
        if (c0.how == CHUNK_BULK) {
            long long spins = 0;
            while (!mbar_try_wait(bars + cur, (parity >> cur) & 1u))
                if (++spins > wait_limit) break;
            // the whole warp leaves together if any lane's wait ran out
            if (__any_sync(0xffffffffu, spins > wait_limit)) goto stalled;
            parity ^= 1u << cur;
        }
        __pipeline_wait_prior(1);  // chunk rb's per-lane copies have landed
        __syncwarp();
        const int64_t r = rb + lane;
        if (r < r_end) {
            double acc = 0.0, zr = 0.0;
            if (c0.how != CHUNK_UNSTAGED) {
                const unsigned char *buf = bufs + cur * L::BUF;
                const int32_t *scol =
                    reinterpret_cast<const int32_t *>(buf + L::COL_OFF) + (b0 - spmv_ca(c0.B, wide));
                const double *sval =
                    reinterpret_cast<const double *>(buf + L::VAL_OFF) + (b0 - spmv_va(c0.B, wide));
                const int len = (int)(e0 - b0);
                unsigned cmax = 0u;
                for (int k0 = 0; k0 < len; k0 += 8) {
                    // all gathers first (up to 8 in flight), then the chain in
                    // stored order
                    double xv[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        xv[j] = 0.0;
                        if (k0 + j < len) {
                            const unsigned cidx = (unsigned)scol[k0 + j];
                            if (CHECKED) {
                                // a bad column is reported and its gather clamped
                                // into range (the call fails; the value is moot)
                                cmax = max(cmax, cidx);
                                xv[j] = L2X ? __ldcg(x + min(cidx, ncol - 1u)) : __ldg(x + min(cidx, ncol - 1u));
                            } else {
                                xv[j] = L2X ? __ldcg(x + cidx) : __ldg(x + cidx);
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (k0 + j < len) acc = fma(sval[k0 + j], xv[j], acc);
                }
                if (CHECKED && len > 0 && cmax >= ncol) err |= ERR_INDEX;
                if (z) zr = reinterpret_cast<const double *>(buf)[lane];
            } else {
                bool bad = false;
                acc = spmv_row<L2X>(A, r, x, bad);
                if (bad) err |= ERR_INDEX;
                if (z) zr = z[r];
            }
            fn(r, acc, zr);
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
    // a bulk chunk prepared past the end is never waited for: there is none,
    // since prepare stages nothing for rb >= r_end
    __syncwarp();
    return;
stalled:
    // A wait ran out (ERR_TIMEOUT): stage nothing more (a late copy could still
    // land in the buffers) and read this and every later row from global memory.
    // The call fails and its results are undefined; the kernel's exact windows
    // are then flushed without the staging buffers as scratch (see ERR_TIMEOUT).
    err |= ERR_TIMEOUT;
    for (; rb < r_end; rb += step) {
        const int64_t r = rb + lane;
        if (r < r_end) {
            bool bad = false;
            const double acc = spmv_row<L2X>(A, r, x, bad);
            if (bad) err |= ERR_INDEX;
            fn(r, acc, z ? z[r] : 0.0);
        }
    }
    __pipeline_wait_prior(0);
    // Bulk copies issued into the two buffers before the stall may still be in
    // flight: wait for them (again bounded) so that none lands in this CTA's
    // shared memory after the kernel ends. (The test stall issues none.)
    if (!skip_bulk && lane == 0) {
        const bool pend[2] = {c0.how == CHUNK_BULK, c1.how == CHUNK_BULK};
        const int bufid[2] = {cur, cur ^ 1};
        for (int k = 0; k < 2; k++) {
            if (!pend[k]) continue;
            long long spins = 0;
            while (!mbar_try_wait(bars + bufid[k], (parity >> bufid[k]) & 1u) && ++spins <= wait_limit) {
            }
        }
    }
    __syncwarp();
}

// Long rows through registers (rows of up to SPMV_REG_LEN nonzeros, e.g. the
// 27-point stencil). The row product is a chain of dependent fmas, and on this
// GPU one warp's chain already keeps an SM sub-partition's FP64 unit busy: the
// kernel is bound by that unit once a chain is ready on every sub-partition at
// all times. spmv_rows holds two staging buffers per warp for the whole of a
// chunk's chain, which leaves room for 8 warps per SM; here each warp has ONE
// buffer, and moves the chunk into registers as soon as it lands: every lane
// gathers its row's x entries (all at once) and loads its row's values, after
// which the buffer is refilled with the next chunk while the chain runs from
// registers. Three 4-warp blocks fit per SM. Chunks with a longer row, or not
// staged, are computed as in spmv_rows before the refill. Staging, the bounded
// waits, the index checks and the timeout fallback are those of spmv_rows; the
// arithmetic is exactly spmv_row's.
constexpr int SPMV_REG_LEN = 28;  // (SPMV_REG_WARPS, the warps per block of its kernels: launch.h)
template <bool CHECKED, int CAP, bool L2X, class F>
__device__ __forceinline__ void spmv_rows_reg(const CSRView &A, int64_t r_begin, int64_t r_end, int64_t warp,
                                              int64_t nwarps, const double *__restrict__ x,
                                              const double *__restrict__ z, bool z_bulk, bool test_stall,
                                              unsigned &err, F &&fn) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int G = SPMV_REG_LEN;
    __shared__ __align__(8) unsigned long long s_bar[SPMV_REG_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t step = nwarps * 32;
    int64_t rb = r_begin + warp * 32;
    const unsigned ncol = A.n < 0x80000000LL ? (unsigned)A.n : 0x80000000u;
    const bool wide = ((reinterpret_cast<uintptr_t>(A.col) | reinterpret_cast<uintptr_t>(A.val)) & 15) == 0;
    const bool bulk_ok = wide && (!z_bulk || (reinterpret_cast<uintptr_t>(z) & 15) == 0);
    using L = SpmvLayout<CAP>;
    unsigned char *buf = warp_scratch<L::BUF, SPMV_REG_WARPS>();
    unsigned long long *bar = s_bar + wid;
    if (lane == 0) {
        mbar_init(bar);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncwarp();
    unsigned parity = 0u;
    const long long wait_limit = test_stall ? SPMV_TEST_WAIT_LIMIT : SPMV_WAIT_LIMIT;
    const bool skip_bulk = test_stall;
    auto rowptrs = [&](int64_t r0, long long &b, long long &e) {
        const int64_t r = r0 + lane;
        b = 0;
        e = 0;
        if (r0 < r_end && r < r_end) {
            b = A.rowptr[r];
            e = A.rowptr[r + 1];
        }
    };
    long long b0, e0, b1, e1, b2, e2;
    rowptrs(rb, b0, e0);
    SpmvChunk c0 = spmv_prepare<CHECKED, CAP>(A, r_end, z, wide, bulk_ok, z_bulk, skip_bulk, rb, b0, e0, buf, bar);
    rowptrs(rb + step, b1, e1);
    for (; rb < r_end; rb += step) {
        if (c0.how == CHUNK_BULK) {
            long long spins = 0;
            while (!mbar_try_wait(bar, parity))
                if (++spins > wait_limit) break;
            if (__any_sync(FULL, spins > wait_limit)) goto stalled;
            parity ^= 1u;
        }
        __pipeline_wait_prior(0);  // chunk rb's per-lane copies have landed
        __syncwarp();
        {
            const int64_t r = rb + lane;
            const bool live = r < r_end;
            const int len = live ? (int)(e0 - b0) : 0;
            const bool reg = c0.how != CHUNK_UNSTAGED && __all_sync(FULL, len <= G);
            const int lmax = (int)__reduce_max_sync(FULL, (unsigned)(len > 0 ? len : 0));
            double acc = 0.0, zr = 0.0;
            double xv[G], vv[G];
            if (reg) {
                if (live && len > 0) {
                    const int32_t *scol =
                        reinterpret_cast<const int32_t *>(buf + L::COL_OFF) + (b0 - spmv_ca(c0.B, wide));
                    const double *sval =
                        reinterpret_cast<const double *>(buf + L::VAL_OFF) + (b0 - spmv_va(c0.B, wide));
                    unsigned cmax = 0u;
                    // every gather of the row in flight at once (entries past the
                    // row's end repeat its last one and are not used)
#pragma unroll
                    for (int j = 0; j < G; j++) {
                        const int k = j < len ? j : len - 1;
                        const unsigned cidx = (unsigned)scol[k];
                        if (CHECKED) {
                            cmax = max(cmax, cidx);
                            xv[j] = L2X ? __ldcg(x + min(cidx, ncol - 1u)) : __ldg(x + min(cidx, ncol - 1u));
                        } else {
                            xv[j] = L2X ? __ldcg(x + cidx) : __ldg(x + cidx);
                        }
                        vv[j] = sval[k];
                    }
                    if (CHECKED && cmax >= ncol) err |= ERR_INDEX;
                }
                if (z && live) zr = reinterpret_cast<const double *>(buf)[lane];
            } else if (live) {
                if (c0.how != CHUNK_UNSTAGED) {
                    const int32_t *scol =
                        reinterpret_cast<const int32_t *>(buf + L::COL_OFF) + (b0 - spmv_ca(c0.B, wide));
                    const double *sval =
                        reinterpret_cast<const double *>(buf + L::VAL_OFF) + (b0 - spmv_va(c0.B, wide));
                    unsigned cmax = 0u;
                    for (int k = 0; k < len; k++) {
                        const unsigned cidx = (unsigned)scol[k];
                        if (CHECKED) cmax = max(cmax, cidx);
                        const unsigned c = CHECKED ? min(cidx, ncol - 1u) : cidx;
                        acc = fma(sval[k], L2X ? __ldcg(x + c) : __ldg(x + c), acc);
                    }
                    if (CHECKED && len > 0 && cmax >= ncol) err |= ERR_INDEX;
                    if (z) zr = reinterpret_cast<const double *>(buf)[lane];
                } else {
                    bool bad = false;
                    acc = spmv_row<L2X>(A, r, x, bad);
                    if (bad) err |= ERR_INDEX;
                    if (z) zr = z[r];
                }
            }
            __syncwarp();  // every lane is done with the buffer: refill it
            c0 = spmv_prepare<CHECKED, CAP>(A, r_end, z, wide, bulk_ok, z_bulk, skip_bulk, rb + step, b1, e1, buf,
                                            bar);
            rowptrs(rb + 2 * step, b2, e2);
            if (reg && live) {
                // the chain in stored order, cut at the warp's longest row in
                // groups of 4 (a warp-uniform branch)
#pragma unroll
                for (int g = 0; g < G; g += 4) {
                    if (g >= lmax) break;
#pragma unroll
                    for (int j = g; j < g + 4; j++)
                        if (j < len) acc = fma(vv[j], xv[j], acc);
                }
            }
            if (live) fn(r, acc, zr);
        }
        b0 = b1;
        e0 = e1;
        b1 = b2;
        e1 = e2;
    }
    __pipeline_wait_prior(0);
    __syncwarp();
    return;
stalled:
    // A wait ran out (ERR_TIMEOUT): as in spmv_rows, stage nothing more and
    // read this and every later row from global memory, then wait (bounded)
    // for the copy still in flight into the buffer.
    err |= ERR_TIMEOUT;
    for (; rb < r_end; rb += step) {
        const int64_t r = rb + lane;
        if (r < r_end) {
            bool bad = false;
            const double acc = spmv_row<L2X>(A, r, x, bad);
            if (bad) err |= ERR_INDEX;
            fn(r, acc, z ? z[r] : 0.0);
        }
    }
    __pipeline_wait_prior(0);
    if (!skip_bulk && lane == 0) {
        long long spins = 0;
        while (!mbar_try_wait(bar, parity) && ++spins <= wait_limit) {
        }
    }
    __syncwarp();
}

// The whole matrix over the grid: every warp of every block.
template <bool CHECKED, int CAP, class F>
__device__ __forceinline__ void spmv_warp_rows(const CSRView &A, const double *__restrict__ x,
                                               const double *__restrict__ z, bool test_stall, unsigned &err,
                                               F &&fn) {
    spmv_rows<CHECKED, CAP, false>(A, 0, A.n, (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                                   (int64_t)gridDim.x * (blockDim.x >> 5), x, z, true, test_stall, err, fn);
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// Row traversal of y = A x with epilogue fn(row, y_row, z_row): mode 1 one
// thread per row, any other mode warp-staged with spans of up to CAP nonzeros.
// Same bits either way. z may be null. Error bits (ERR_*) accumulate in err.
template <bool CHECKED, int CAP, class F>
__device__ __forceinline__ void spmv_each(const CSRView &A, const double *__restrict__ x,
                                          const double *__restrict__ z, int mode, unsigned &err, F &&fn) {
    if ((mode & SPMV_MODE_MASK) != 1) {
        spmv_warp_rows<CHECKED, CAP>(A, x, z, (mode & SPMV_TEST_STALL) != 0, err, fn);
    } else {
        bool bad = false;
        for (int64_t i = gtid(); i < A.n; i += gstride()) fn(i, spmv_row(A, i, x, bad), z ? z[i] : 0.0);
        if (bad) err |= ERR_INDEX;
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

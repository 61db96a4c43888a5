// Exact dot-product accumulation on sm_103a (Sec. 2 "ExBLAS"; Sec. 3.2).
//
// The paper's exdot keeps every bit of every product (TwoProd, Alg. 2) in
// floating-point expansions and a Kulisch long accumulator, and rounds once.
// On GB300 the binary64 pipe issues under two operations per SM per clock, so
// this design keeps the exact work off it entirely:
//
//  * each product x*y is formed exactly as a 106-bit integer (four 32x32->64
//    integer multiply-adds on the 53-bit significands) at bit position
//    pos = e_x + e_y - 2, the accumulator's bit 0 weighing 2^-2148 (the lowest
//    bit of a product of two subnormals). This is TwoProd's exact r + s, in
//    integer form, with no underflow or overflow exception;
//  * each thread adds its products into a 256-bit two's complement register
//    window anchored at a 32-bit limb `a`; a product lands at limb offset
//    q = (pos >> 5) - a in [0, Q) with a funnel shift and a log-shifter of
//    word selects, then one 8-word add with carry;
//  * products above the window flush it and re-anchor it; products below it
//    are added straight into the block's shared-memory long accumulator
//    (RBS_LIMBS signed 64-bit limbs, limb j weighing 2^(32 j - 2148), carry-save
//    with 31 spare bits, the paper's "carry-safe bits" of Sec. 3.2);
//  * at the end each window is added into the shared accumulator, the block
//    accumulator is partially normalised and added into a global one with
//    integer atomics (exact, so order does not matter), and the last block
//    normalises, rounds once to nearest even and resets the scratch.
//
// The value is therefore the exact sum rounded once, whatever the grid, block
// size, window size or schedule.
#pragma once

#include "common.cuh"

namespace rbs {

// ---- the register window ----------------------------------------------------

// Anchor of an empty window: far below every limb, so that no product ever
// matches the in-window test (q = L - a >= Q) and the first one anchors it.
constexpr int WIN_EMPTY = -(1 << 30);

template <int Q>
struct Win {
    uint32_t w[8];
    int a;  // anchor limb, WIN_EMPTY when empty

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < 8; k++) w[k] = 0u;
        a = WIN_EMPTY;
    }
};

// w += v + c over 8 words with carry (c in {0, 1}).
__device__ __forceinline__ void add8_carry(uint32_t (&w)[8], const uint32_t (&v)[8], uint32_t c) {
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %8, 0xffffffff;\n\t"
        "addc.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %11;\n\t"
        "addc.cc.u32 %3, %3, %12;\n\t"
        "addc.cc.u32 %4, %4, %13;\n\t"
        "addc.cc.u32 %5, %5, %14;\n\t"
        "addc.cc.u32 %6, %6, %15;\n\t"
        "addc.u32 %7, %7, %16;\n\t}"
        : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(w[4]), "+r"(w[5]), "+r"(w[6]),
          "+r"(w[7])
        : "r"(c), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
          "r"(v[7]));
}

// The 106-bit product p (4 words) shifted left by r in [0, 31]: 5 words.
__device__ __forceinline__ void shift5(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3, uint32_t r,
                                       uint32_t (&u)[5]) {
    u[0] = p0 << r;
    u[1] = __funnelshift_l(p0, p1, r);
    u[2] = __funnelshift_l(p1, p2, r);
    u[3] = __funnelshift_l(p2, p3, r);
    u[4] = __funnelshift_l(p3, 0u, r);
}

// Place the 5-word shifted product at word offset q (log-shifter of word
// selects) and add it, negated when m = ~0: the placed 8-word value is
// complemented word by word (the product's words are XORed with m before
// placement and every fill word is m) and 1 is carried in, which is its
// two's complement negation.
template <int Q, bool SIGNED>
__device__ __forceinline__ void win_place_add(Win<Q> &W, const uint32_t (&u)[5], int q, uint32_t m) {
    uint32_t x[5], v[8];
#pragma unroll
    for (int k = 0; k < 5; k++) x[k] = SIGNED ? (u[k] ^ m) : u[k];
    const uint32_t f = SIGNED ? m : 0u;
    if (Q == 1) {
        v[0] = x[0]; v[1] = x[1]; v[2] = x[2]; v[3] = x[3]; v[4] = x[4];
        v[5] = f; v[6] = f; v[7] = f;
    } else {
        const bool b1 = (q & 1) != 0;
        uint32_t t[6];
        t[0] = b1 ? f : x[0];
        t[1] = b1 ? x[0] : x[1];
        t[2] = b1 ? x[1] : x[2];
        t[3] = b1 ? x[2] : x[3];
        t[4] = b1 ? x[3] : x[4];
        t[5] = b1 ? x[4] : f;
        if (Q == 2) {
#pragma unroll
            for (int k = 0; k < 6; k++) v[k] = t[k];
            v[6] = f; v[7] = f;
        } else {
            const bool b2 = (q & 2) != 0;
            v[0] = b2 ? f : t[0];
            v[1] = b2 ? f : t[1];
            v[2] = b2 ? t[0] : t[2];
            v[3] = b2 ? t[1] : t[3];
            v[4] = b2 ? t[2] : t[4];
            v[5] = b2 ? t[3] : t[5];
            v[6] = b2 ? t[4] : f;
            v[7] = b2 ? t[5] : f;
        }
    }
    add8_carry(W.w, v, SIGNED ? (m & 1u) : 0u);
}

// win_place_add for windows anchored top-aligned (products of the anchor's
// limb land at q = Q - 1): with Q = 4 the placements q = 2, 3 take the first
// select level only and a branch picks the word layout, so the common case of
// products within two limbs skips the second level (a branch that is uniform
// across the warp on well-scaled data; divergent warps run both layouts, which
// costs about what the second select level does).
template <int Q>
__device__ __forceinline__ void win_place_add_top(Win<Q> &W, const uint32_t (&u)[5], int q, uint32_t m) {
    if (Q != 4) {
        win_place_add<Q, true>(W, u, q, m);
        return;
    }
    uint32_t x[5], t[6], v[8];
#pragma unroll
    for (int k = 0; k < 5; k++) x[k] = u[k] ^ m;
    const bool b1 = (q & 1) != 0;
    t[0] = b1 ? m : x[0];
    t[1] = b1 ? x[0] : x[1];
    t[2] = b1 ? x[1] : x[2];
    t[3] = b1 ? x[2] : x[3];
    t[4] = b1 ? x[3] : x[4];
    t[5] = b1 ? x[4] : m;
    if (q & 2) {
        v[0] = m;
        v[1] = m;
#pragma unroll
        for (int k = 0; k < 6; k++) v[k + 2] = t[k];
    } else {
#pragma unroll
        for (int k = 0; k < 6; k++) v[k] = t[k];
        v[6] = m;
        v[7] = m;
    }
    add8_carry(W.w, v, m & 1u);
}

// Add a signed 64-bit value to a limb of a block accumulator in shared memory
// with two 32-bit atomics: the low word's add returns the old low word, which
// gives that add's carry into the high word. Measured on GB300 with four lanes
// per address and every warp of the block on the same addresses (the pattern of
// products that miss their register windows): 64-bit shared atomic adds run at
// about 0.26 per SM per clock, 32-bit ones at about 7.4. The limb is the same
// modular sum either way: each add carries exactly what its own low-word step
// overflowed, in whatever order the low-word atomics are served. Every shared
// accumulator update goes through here, so the two widths never mix on a limb.
__device__ __forceinline__ void sacc_add(unsigned long long *p, long long v) {
    unsigned *w = reinterpret_cast<unsigned *>(p);
    const unsigned lo = (unsigned)v, hi = (unsigned)((unsigned long long)v >> 32);
    const unsigned old = atomicAdd(w, lo);
    const unsigned h = hi + ((unsigned)(old + lo) < old ? 1u : 0u);
    if (h) atomicAdd(w + 1, h);
}

// Add the window into the block accumulator as carry-save limbs: words 0..6
// unsigned, word 7 the signed top of the two's complement value.
template <int Q>
__device__ __forceinline__ void win_flush(Win<Q> &W, unsigned long long *sacc) {
    if (W.a < 0) return;
#pragma unroll
    for (int k = 0; k < 7; k++)
        if (W.w[k]) sacc_add(&sacc[W.a + k], (long long)W.w[k]);
    if (W.w[7]) sacc_add(&sacc[W.a + 7], (long long)(int32_t)W.w[7]);
#pragma unroll
    for (int k = 0; k < 8; k++) W.w[k] = 0u;
    W.a = WIN_EMPTY;
}

// Product straight into the block accumulator (rare path).
__device__ __forceinline__ void smem_deposit(unsigned long long *sacc, const uint32_t (&u)[5], int L,
                                             uint32_t m) {
#pragma unroll
    for (int k = 0; k < 5; k++) {
        if (u[k]) {
            const long long v = (long long)u[k];
            sacc_add(&sacc[L + k], m ? -v : v);
        }
    }
}

// Non-finite operand handling (reading of the paper's silence; see rbs.h).
static __device__ __noinline__ uint32_t special_flags(uint32_t xh, uint32_t xl, uint32_t yh, uint32_t yl) {
    const uint32_t ex = (xh >> 20) & 0x7ffu, ey = (yh >> 20) & 0x7ffu;
    const bool xnan = ex == 0x7ffu && ((xh & 0xfffffu) | xl) != 0u;
    const bool ynan = ey == 0x7ffu && ((yh & 0xfffffu) | yl) != 0u;
    if (xnan || ynan) return F_NAN;
    const bool xzero = ((xh & 0x7fffffffu) | xl) == 0u;
    const bool yzero = ((yh & 0x7fffffffu) | yl) == 0u;
    if (xzero || yzero) return F_NAN;  // inf * 0
    return ((xh ^ yh) & 0x80000000u) ? F_NINF : F_PINF;
}

// Exact accumulation of x*y into window W / block accumulator sacc. With
// SQUARE the product is x*x: it cannot be negative, so no sign handling.
template <int Q, bool SQUARE = false>
__device__ __forceinline__ void exact_add(Win<Q> &W, uint32_t &flags, unsigned long long *sacc, double x,
                                          double y) {
    const uint32_t xh = (uint32_t)__double2hiint(x), xl = (uint32_t)__double2loint(x);
    const uint32_t yh = SQUARE ? xh : (uint32_t)__double2hiint(y);
    const uint32_t yl = SQUARE ? xl : (uint32_t)__double2loint(y);
    const uint32_t ex = (xh >> 20) & 0x7ffu, ey = SQUARE ? ex : (yh >> 20) & 0x7ffu;
    if (ex == 0x7ffu || ey == 0x7ffu) {
        flags |= special_flags(xh, xl, yh, yl);
        return;
    }
    const uint32_t A1 = (xh & 0xfffffu) | (ex ? 0x100000u : 0u);
    const uint32_t B1 = SQUARE ? A1 : ((yh & 0xfffffu) | (ey ? 0x100000u : 0u));
    if ((A1 | xl) == 0u || (B1 | yl) == 0u) return;  // a zero product adds nothing
    const int pos = (int)max(ex, 1u) + (int)max(ey, 1u) - 2;
    // 106-bit significand product (A1:xl) * (B1:yl)
    const unsigned long long m00 = (unsigned long long)xl * yl;
    const unsigned long long m01 = (unsigned long long)xl * B1 + (m00 >> 32);
    const unsigned long long m10 = (unsigned long long)A1 * yl + (uint32_t)m01;
    const unsigned long long m11 =
        (unsigned long long)A1 * B1 + (unsigned long long)((uint32_t)(m01 >> 32) + (uint32_t)(m10 >> 32));
    const uint32_t p0 = (uint32_t)m00, p1 = (uint32_t)m10, p2 = (uint32_t)m11, p3 = (uint32_t)(m11 >> 32);
    const uint32_t m = SQUARE ? 0u : (uint32_t)((int32_t)(xh ^ yh) >> 31);
    const int L = pos >> 5;
    uint32_t u[5];
    shift5(p0, p1, p2, p3, (uint32_t)pos & 31u, u);
    int q = L - W.a;
    if ((unsigned)q < (unsigned)Q) {
        win_place_add<Q, !SQUARE>(W, u, q, m);
        return;
    }
    if (W.a < 0 || q >= Q) {
        // empty, or above the window: flush and re-anchor with the product at
        // offset Q-2 (or 0), leaving room for somewhat larger products
        win_flush<Q>(W, sacc);
        int a = L - (Q >= 2 ? Q - 2 : 0);
        a = a < 0 ? 0 : a;
        W.a = a;
        win_place_add<Q, !SQUARE>(W, u, L - a, m);
        return;
    }
    smem_deposit(sacc, u, L, m);
}

// The exact product x*y as five 32-bit words u (the 106-bit significand
// product shifted left by pos & 31) at limb L = pos >> 5, sign mask m (0 or
// ~0). Returns false, adding nothing, for a zero product; a non-finite operand
// sets its flag and also returns false.
__device__ __forceinline__ bool prod_exact(double x, double y, uint32_t &flags, uint32_t (&u)[5], int &L,
                                           uint32_t &m) {
    const uint32_t xh = (uint32_t)__double2hiint(x), xl = (uint32_t)__double2loint(x);
    const uint32_t yh = (uint32_t)__double2hiint(y), yl = (uint32_t)__double2loint(y);
    const uint32_t exm = xh & 0x7ff00000u, eym = yh & 0x7ff00000u;  // biased exponents << 20
    uint32_t A1, B1;
    int pos;
    if (exm - 0x00100000u < 0x7fe00000u && eym - 0x00100000u < 0x7fe00000u) {
        A1 = (xh & 0xfffffu) | 0x100000u;
        B1 = (yh & 0xfffffu) | 0x100000u;
        pos = (int)((exm >> 20) + (eym >> 20)) - 2;
    } else {
        const uint32_t ex = exm >> 20, ey = eym >> 20;
        if (ex == 0x7ffu || ey == 0x7ffu) {
            flags |= special_flags(xh, xl, yh, yl);
            return false;
        }
        A1 = (xh & 0xfffffu) | (ex ? 0x100000u : 0u);
        B1 = (yh & 0xfffffu) | (ey ? 0x100000u : 0u);
        if ((A1 | xl) == 0u || (B1 | yl) == 0u) return false;
        pos = (int)max(ex, 1u) + (int)max(ey, 1u) - 2;
    }
    const unsigned long long m00 = (unsigned long long)xl * yl;
    const unsigned long long m01 = (unsigned long long)xl * B1 + (m00 >> 32);
    const unsigned long long m10 = (unsigned long long)A1 * yl + (uint32_t)m01;
    const unsigned long long m11 =
        (unsigned long long)A1 * B1 + (unsigned long long)((uint32_t)(m01 >> 32) + (uint32_t)(m10 >> 32));
    m = (uint32_t)((int32_t)(xh ^ yh) >> 31);
    L = pos >> 5;
    shift5((uint32_t)m00, (uint32_t)m10, (uint32_t)m11, (uint32_t)(m11 >> 32), (uint32_t)pos & 31u, u);
    return true;
}

// Two windows per thread: H takes the product if it fits; a product above H
// re-anchors H at it and the old H becomes the low window L; a product below H
// goes to L (anchoring or re-anchoring it when it is empty or lies between L and
// H); only products below both go to shared memory. Wide-exponent sums (the
// ill-conditioned dots) then rarely touch shared memory.
template <int Q>
__device__ __forceinline__ void exact_add2(Win<Q> &H, Win<Q> &Lw, uint32_t &flags, unsigned long long *sacc,
                                           double x, double y) {
    const uint32_t xh = (uint32_t)__double2hiint(x), xl = (uint32_t)__double2loint(x);
    const uint32_t yh = (uint32_t)__double2hiint(y), yl = (uint32_t)__double2loint(y);
    const uint32_t exm = xh & 0x7ff00000u, eym = yh & 0x7ff00000u;  // biased exponents << 20
    uint32_t A1, B1;
    int pos;
    if (exm - 0x00100000u < 0x7fe00000u && eym - 0x00100000u < 0x7fe00000u) {
        // both operands normal (the common case): implicit bit set, no zero
        A1 = (xh & 0xfffffu) | 0x100000u;
        B1 = (yh & 0xfffffu) | 0x100000u;
        pos = (int)((exm >> 20) + (eym >> 20)) - 2;
    } else {
        const uint32_t ex = exm >> 20, ey = eym >> 20;
        if (ex == 0x7ffu || ey == 0x7ffu) {
            flags |= special_flags(xh, xl, yh, yl);
            return;
        }
        A1 = (xh & 0xfffffu) | (ex ? 0x100000u : 0u);
        B1 = (yh & 0xfffffu) | (ey ? 0x100000u : 0u);
        if ((A1 | xl) == 0u || (B1 | yl) == 0u) return;
        pos = (int)max(ex, 1u) + (int)max(ey, 1u) - 2;
    }
    const unsigned long long m00 = (unsigned long long)xl * yl;
    const unsigned long long m01 = (unsigned long long)xl * B1 + (m00 >> 32);
    const unsigned long long m10 = (unsigned long long)A1 * yl + (uint32_t)m01;
    const unsigned long long m11 =
        (unsigned long long)A1 * B1 + (unsigned long long)((uint32_t)(m01 >> 32) + (uint32_t)(m10 >> 32));
    const uint32_t p0 = (uint32_t)m00, p1 = (uint32_t)m10, p2 = (uint32_t)m11, p3 = (uint32_t)(m11 >> 32);
    const uint32_t m = (uint32_t)((int32_t)(xh ^ yh) >> 31);
    const int L = pos >> 5;
    uint32_t u[5];
    shift5(p0, p1, p2, p3, (uint32_t)pos & 31u, u);
    const int q = L - H.a;
    if ((unsigned)q < (unsigned)Q) {
        win_place_add_top<Q>(H, u, q, m);
        return;
    }
    const int back = Q - 1;  // top-aligned: the anchoring product at q = Q - 1
    if (q >= Q) {
        if (H.a != WIN_EMPTY) {
            win_flush<Q>(Lw, sacc);
            Lw = H;
        }
#pragma unroll
        for (int k = 0; k < 8; k++) H.w[k] = 0u;
        H.a = L - back < 0 ? 0 : L - back;
        win_place_add_top<Q>(H, u, L - H.a, m);
        return;
    }
    const int ql = L - Lw.a;
    if ((unsigned)ql < (unsigned)Q) {
        win_place_add_top<Q>(Lw, u, ql, m);
        return;
    }
    if (ql >= Q) {
        win_flush<Q>(Lw, sacc);
        Lw.a = L - back < 0 ? 0 : L - back;
        win_place_add_top<Q>(Lw, u, L - Lw.a, m);
        return;
    }
    smem_deposit(sacc, u, L, m);
}

// Warp-cooperative flush of every lane's window (all 32 lanes call it). The
// lanes' windows usually sit on the same few limbs, so per-lane atomics would
// collide 32 ways. Instead each lane stages its 8 carry-save limbs (words 0..6
// unsigned, word 7 signed) in shared memory, lane j sums the warp's
// contributions to limb base + j (at most 32 x 2^32 in magnitude), and one
// conflict-free atomic per limb lands in the block accumulator. Windows spread
// over more than 32 limbs fall back to per-lane atomics.
constexpr int MAX_WARPS = 8;                        // every kernel here runs blocks of at most 256 threads
constexpr int FLUSH_SCRATCH = 32 * 8 * 8 + 32 * 4;  // bytes of the warp_flush staging

// Each warp's private slice of one shared buffer of BYTES per warp, for blocks
// of at most WARPS warps. Phases of a kernel that stage data per warp (SpMV
// operands, then the window flush) reuse it by naming the same BYTES; a warp
// only ever touches its own slice, so no block barrier is needed between them.
template <int BYTES, int WARPS = MAX_WARPS>
__device__ __forceinline__ unsigned char *warp_scratch() {
    static_assert(BYTES % 16 == 0, "16-byte aligned slices");
    __shared__ __align__(16) unsigned char buf[WARPS * BYTES];
    return buf + (threadIdx.x >> 5) * BYTES;
}

template <int Q, int SCRATCH = FLUSH_SCRATCH, int WARPS = MAX_WARPS>
__device__ __forceinline__ void warp_flush(Win<Q> &W, unsigned long long *sacc) {
    static_assert(SCRATCH >= FLUSH_SCRATCH, "flush staging");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool has = W.a >= 0;
    const int lo = __reduce_min_sync(FULL, (unsigned)(has ? W.a : 0x7fffffff));
    const int hi = (int)__reduce_max_sync(FULL, (unsigned)(has ? W.a : 0));
    if (lo == 0x7fffffff) return;  // no lane holds a window
    if (hi - lo > 24) {
        win_flush<Q>(W, sacc);
        return;
    }
    __syncwarp();
    long long(*st)[8] = reinterpret_cast<long long(*)[8]>(warp_scratch<SCRATCH, WARPS>());  // 2 KB
    int *off = reinterpret_cast<int *>(warp_scratch<SCRATCH, WARPS>() + 32 * 8 * 8);        // 128 B
#pragma unroll
    for (int k = 0; k < 7; k++) st[lane][k] = has ? (long long)W.w[k] : 0ll;
    st[lane][7] = has ? (long long)(int32_t)W.w[7] : 0ll;
    off[lane] = has ? W.a - lo : 0;
    __syncwarp();
    long long sum = 0;
#pragma unroll 8
    for (int l = 0; l < 32; l++) {
        const int k = lane - off[l];
        if (k >= 0 && k < 8) sum += st[l][k];
    }
    __syncwarp();
    if (sum && lo + lane < NL) sacc_add(&sacc[lo + lane], sum);
#pragma unroll
    for (int k = 0; k < 8; k++) W.w[k] = 0u;
    W.a = WIN_EMPTY;
}

// ---- block- and grid-level reduction ------------------------------------------

// Zero the block accumulators (K of them). All threads call it; ends in a barrier.
template <int K>
__device__ __forceinline__ void sacc_zero(unsigned long long (*sacc)[NL], uint32_t *sflags) {
    for (int j = threadIdx.x; j < K * NL; j += blockDim.x) (&sacc[0][0])[j] = 0ull;
    if (threadIdx.x < K) sflags[threadIdx.x] = 0u;
    __syncthreads();
}

// Partially normalise a carry-save limb array value by value:
// out_j = lo32(L_j) + (L_{j-1} >> 32); the top limb keeps its full value.
__device__ __forceinline__ long long partial_norm(const unsigned long long *L, int j) {
    const long long cur = (long long)L[j];
    const long long below = j > 0 ? ((long long)L[j - 1] >> 32) : 0;
    if (j == NL - 1) return cur + below;
    return (long long)(cur & 0xffffffffll) + below;
}

// Round an exact value given as carry-save signed limbs (|limb| < 2^62) once
// to nearest even, given its lowest and highest nonzero limbs lo and hi (lo =
// -1 or lo > hi: the value is zero). G is modified (normalised in place). One
// thread.
static __device__ __noinline__ double round_limbs_span(long long *G, uint32_t flags, int lo, int hi) {
    if (flags & F_NAN) return qnan();
    if ((flags & F_PINF) && (flags & F_NINF)) return qnan();
    if (flags & F_PINF) return __longlong_as_double(0x7ff0000000000000ll);
    if (flags & F_NINF) return __longlong_as_double((long long)0xfff0000000000000ull);
    if (lo < 0 || lo > hi) return 0.0;
    // carry propagation from lo up; two limbs past hi the carry is 0 or -1
    int top = hi + 2 < NL - 1 ? hi + 2 : NL - 1;
    long long c = 0;
    for (int j = lo; j <= top; j++) {
        const long long t = G[j] + c;
        G[j] = t & 0xffffffffll;
        c = t >> 32;
    }
    const bool neg = c < 0;
    if (neg) {  // magnitude = two's complement negation of words lo..top
        unsigned long long cy = 1;
        for (int j = lo; j <= top; j++) {
            const unsigned long long t = (unsigned long long)(~(uint32_t)G[j]) + cy;
            G[j] = (long long)(t & 0xffffffffull);
            cy = t >> 32;
        }
    }
    int tw = -1;
    for (int j = top; j >= lo; j--)
        if (G[j] != 0) {
            tw = j;
            break;
        }
    if (tw < 0) return 0.0;
    const int h = 32 * tw + 31 - __clz((uint32_t)G[tw]);  // top set bit
    const int lsb = h - 52 > 1074 ? h - 52 : 1074;         // bit 1074 weighs 2^-1074
    const int len = h - lsb + 1;
    auto word = [&](int j) -> unsigned long long {
        return (j >= lo && j <= top) ? (unsigned long long)(uint32_t)G[j] : 0ull;
    };
    const int w0 = lsb >> 5, s = lsb & 31;
    const unsigned long long lo64 = word(w0) | (word(w0 + 1) << 32);
    unsigned long long mant = lo64 >> s;
    if (s) mant |= word(w0 + 2) << (64 - s);
    mant &= (len >= 64) ? ~0ull : ((1ull << len) - 1ull);
    int round_bit = 0, sticky = 0;
    if (lsb >= 1) {
        const int rb = lsb - 1;
        round_bit = (int)((word(rb >> 5) >> (rb & 31)) & 1ull);
        const int sw = rb >> 5, sb = rb & 31;
        if (sb && (word(sw) & ((1ull << sb) - 1ull))) sticky = 1;
        for (int j = lo; j < sw && !sticky; j++)
            if (word(j)) sticky = 1;
    }
    if (round_bit && (sticky || (mant & 1ull))) mant += 1ull;
    // value = mant * 2^(lsb - 2148); as binary64 bits: ((lsb - 1074) << 52) + mant
    unsigned long long bits = ((unsigned long long)(lsb - 1074) << 52) + mant;
    if (lsb - 1074 >= 2047 || bits >= 0x7ff0000000000000ull) bits = 0x7ff0000000000000ull;
    if (neg) bits |= 0x8000000000000000ull;
    return __longlong_as_double((long long)bits);
}

// round_limbs_span after a scan of all NL limbs for the nonzero span.
static __device__ __noinline__ double round_limbs_thread(long long *G, uint32_t flags) {
    int lo = -1, hi = -1;
    for (int j = 0; j < NL; j++)
        if (G[j] != 0) {
            if (lo < 0) lo = j;
            hi = j;
        }
    return round_limbs_span(G, flags, lo, hi);
}

// Block- and grid-level finish of K exact reductions, once every thread's own
// accumulators are in the block accumulators sacc (flags[k]: this thread's
// non-finite flags). Every thread of each of the nblk blocks that share the
// reduction (the whole grid unless given) calls it. Returns true in the block
// that finishes last; there the rounded values are in vals[0..K-1] (shared
// memory) after a barrier, or, with export_limbs, the partially normalised
// limbs of the first reduction are in limbs_out.
template <int K>
__device__ __forceinline__ bool block_grid_finish(const uint32_t (&flags)[K], unsigned long long (*sacc)[NL],
                                                  uint32_t *sflags, DotScratch *g, double *vals,
                                                  bool export_limbs = false, long long *limbs_out = nullptr,
                                                  int32_t *flags_out = nullptr, unsigned nblk = 0u) {
    // nonzero limb span of each reduction, found while the last block reads
    // the limbs back (so that its rounding need not scan all NL of them)
    __shared__ int s_span[K][2];
    if (threadIdx.x < K) {
        s_span[threadIdx.x][0] = NL;
        s_span[threadIdx.x][1] = -1;
    }
#pragma unroll
    for (int k = 0; k < K; k++)
        if (flags[k]) atomicOr(&sflags[k], flags[k]);
    __syncthreads();
    for (int idx = threadIdx.x; idx < K * NL; idx += blockDim.x) {
        const int k = idx / NL, j = idx - k * NL;
        const long long v = partial_norm(sacc[k], j);
        if (v) atomicAdd(&g->limbs[k][j], (unsigned long long)v);
    }
    if (threadIdx.x < K && sflags[threadIdx.x]) atomicOr(&g->flags[threadIdx.x], sflags[threadIdx.x]);
    __threadfence();
    __syncthreads();
    __shared__ bool s_last;
    if (threadIdx.x == 0) s_last = (atomicAdd(&g->ticket, 1u) == (nblk ? nblk : gridDim.x) - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // read back (and clear) the global accumulators into shared memory
    for (int idx = threadIdx.x; idx < K * NL; idx += blockDim.x) {
        const int k = idx / NL, j = idx - k * NL;
        const unsigned long long v = atomicExch(&g->limbs[k][j], 0ull);
        sacc[k][j] = v;
        if (v) {
            atomicMin(&s_span[k][0], j);
            atomicMax(&s_span[k][1], j);
        }
    }
    if (threadIdx.x < K) sflags[threadIdx.x] = atomicExch(&g->flags[threadIdx.x], 0u);
    if (threadIdx.x == 0) g->ticket = 0u;
    __syncthreads();
    if (export_limbs) {
        for (int idx = threadIdx.x; idx < NL; idx += blockDim.x)
            limbs_out[idx] = partial_norm(sacc[0], idx);
        if (threadIdx.x == 0) *flags_out = (int32_t)sflags[0];
        return true;
    }
    if (threadIdx.x < K)
        vals[threadIdx.x] = round_limbs_span((long long *)sacc[threadIdx.x], sflags[threadIdx.x],
                                             s_span[threadIdx.x][0], s_span[threadIdx.x][1]);
    __syncthreads();
    return true;
}

// Grid-level finish of K exact reductions held in register windows: flush the
// windows into the block accumulators, then block_grid_finish (nblk: blocks
// that share the reduction, 0 for the whole grid). SCRATCH, WARPS: the
// per-warp shared buffer the kernel already uses (warp_scratch), which the
// flush reuses.
// coop = false: flush every lane's window with its own atomics, without the
// warp's shared scratch (whose bytes a timed-out asynchronous copy may still
// overwrite).
template <int K, int Q, int SCRATCH = FLUSH_SCRATCH, int WARPS = MAX_WARPS>
__device__ __forceinline__ bool exact_finish(Win<Q> (&win)[K], uint32_t (&flags)[K],
                                             unsigned long long (*sacc)[NL], uint32_t *sflags,
                                             DotScratch *g, double *vals, bool export_limbs = false,
                                             long long *limbs_out = nullptr, int32_t *flags_out = nullptr,
                                             unsigned nblk = 0u, bool coop = true) {
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (coop) warp_flush<Q, SCRATCH, WARPS>(win[k], sacc[k]);
        else win_flush<Q>(win[k], sacc[k]);
    }
    return block_grid_finish<K>(flags, sacc, sflags, g, vals, export_limbs, limbs_out, flags_out, nblk);
}

}  // namespace rbs

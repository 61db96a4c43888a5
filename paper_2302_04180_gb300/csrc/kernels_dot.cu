// Standalone kernels: exact dot (single and multi-output; window size Q = 4
// here, Q = 1 and 2 in kernels_exdot_w1.cu / _w2.cu), long-accumulator export
// and rounding, the allocation-free exact dot, the FPE-8 dot.
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "exdot.cuh"

namespace rbs {

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
    if (window == 2) nb = exdot_occ_w2(k, block, smem);
    else if (window == 1) nb = exdot_occ_w1(k, block, smem);
    else nb = smem ? exdot_occ_q<4, true>(k, block) : exdot_occ_q<4, false>(k, block);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = nb;
    return nb;
}

cudaError_t launch_exdot(int k, const double *const *xs, const double *const *ys, int64_t n,
                         DotScratch *g, double *out, int window, Cfg cfg, cudaStream_t s) {
    if (window == 2) return launch_exdot_w2(k, xs, ys, n, g, out, cfg, s);
    if (window == 1) return launch_exdot_w1(k, xs, ys, n, g, out, cfg, s);
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

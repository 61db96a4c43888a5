// Shared definitions of the GB300 library: device state, scratch layouts,
// launch helpers. Compiled for sm_103a only, with -fmad=false so that no
// a*b+c in this code is contracted; every fused step is an explicit fma()
// (the contraction rule of Sec. 3.3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rbs.h"

namespace rbs {

constexpr int NL = RBS_LIMBS;  // 136 limbs of 32-bit weight steps: 2^-2148 .. 2^2204
constexpr int KMAX = 6;        // most dots fused into one pass (Fig. 4 S16 + tau)

// Flags of non-finite products (OR-reduced beside the limbs).
constexpr uint32_t F_NAN = 1u, F_PINF = 2u, F_NINF = 4u;

// Scratch of the cross-block exact reduction: all zero at rest; the last block
// of every reduction reads it back with atomicExch(.., 0), so it is zero again
// when the kernel ends.
struct DotScratch {
    unsigned long long limbs[KMAX][NL];
    unsigned int flags[KMAX];
    unsigned int ticket;
    unsigned int err;  // sticky workspace error word (bad CSR index seen)
};

// Solver scalars, resident on the device for the whole solve. Kernels read
// them at launch; the last block of each reduction writes them.
struct SolverState {
    double tol, tau_max, tau0, rho0;
    double rho, alpha, omega, beta, tau;
    double mu0, alpha0;
    double rec[RBS_HIST_W];  // record of the iteration in progress
    int32_t iter, maxit, done, status, converged, variant, hist_cap, loops;
};

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000ll); }

__device__ __forceinline__ bool finite_d(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

}  // namespace rbs

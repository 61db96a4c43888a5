// The standalone exact dot with 2-limb register windows (the "exdot.window"
// knob = 2): its own translation unit, compiled in parallel with the others.
#include "exdot.cuh"

namespace rbs {

cudaError_t launch_exdot_w2(int k, const double *const *xs, const double *const *ys, int64_t n, DotScratch *g,
                             double *out, Cfg cfg, cudaStream_t s) {
    return exdot_q<2>(k, xs, ys, n, g, out, cfg, s);
}

int exdot_occ_w2(int k, int block, bool smem) {
    return smem ? exdot_occ_q<2, true>(k, block) : exdot_occ_q<2, false>(k, block);
}

}  // namespace rbs

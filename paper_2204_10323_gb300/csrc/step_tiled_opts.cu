// step_tiled_opts.cu -- the temporal-blocking kernels (step_tiled.cuh) with the
// scheme options of Eq. 3: theta-weighted numerator discharges (mode bit 0)
// and the vector norm in the friction term (bit 1).  A translation unit of its
// own, so that the build compiles it beside the one for Eq. 3 as printed.
#include "step_tiled.cuh"

namespace flood {

cudaError_t launch_step_tiled_opts(const StepArgs<float> &a, int mode, cudaStream_t st)
{
    switch (mode) {
    case 1: return launch_tiled_mode<1>(a, st);
    case 2: return launch_tiled_mode<2>(a, st);
    case 3: return launch_tiled_mode<3>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_tiled_ensemble_opts(const StepArgs<float> *table, const int *base, int n, int total_items,
                                            int k_steps, int s0, int want_hmax, int *next_item, int mode,
                                            cudaStream_t st)
{
    switch (mode) {
    case 1: return launch_tiled_ensemble_mode<1>(table, base, n, total_items, k_steps, s0, want_hmax, next_item, st);
    case 2: return launch_tiled_ensemble_mode<2>(table, base, n, total_items, k_steps, s0, want_hmax, next_item, st);
    case 3: return launch_tiled_ensemble_mode<3>(table, base, n, total_items, k_steps, s0, want_hmax, next_item, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace flood

// Walk kernel instantiations with the level-1 codebook in FP32, and their dispatch
// (compiled apart from lc_search.cu so the instantiations build in parallel).
#include "lc_walk.cuh"

namespace lc {

// Dispatch on (sub-space width variant, codebook element type, full walk).  The full walk
// exists for the uniform splits (variants 1-3) and, in FP32, for any split.
cudaError_t walk_config_f32(int variant, int M1, bool fq, const WalkArgs &wa, size_t per_warp, int sms, int want,
                            int *wpc, int *grid, size_t *smem)
{
    if (fq) {
        switch (variant) {
        case 1: return launch_walk<16, 6, float, true>(wa, per_warp, sms, want, wpc, grid, smem);
        case 2: return launch_walk<32, 3, float, true>(wa, per_warp, sms, want, wpc, grid, smem);
        case 3: return launch_walk<64, 2, float, true>(wa, per_warp, sms, want, wpc, grid, smem);
        default:
            {
                if (M1 == 16) return launch_walk<16, 0, float, true>(wa, per_warp, sms, want, wpc, grid, smem);
                if (M1 == 32) return launch_walk<32, 0, float, true>(wa, per_warp, sms, want, wpc, grid, smem);
                return launch_walk<64, 0, float, true>(wa, per_warp, sms, want, wpc, grid, smem);
            }
            return cudaErrorInvalidValue;
        }
    }
    switch (variant) {
    case 1: return launch_walk<16, 6, float, false>(wa, per_warp, sms, want, wpc, grid, smem);
    case 2: return launch_walk<32, 3, float, false>(wa, per_warp, sms, want, wpc, grid, smem);
    case 3: return launch_walk<64, 2, float, false>(wa, per_warp, sms, want, wpc, grid, smem);
    default:
        if (M1 == 16) return launch_walk<16, 0, float, false>(wa, per_warp, sms, want, wpc, grid, smem);
        if (M1 == 32) return launch_walk<32, 0, float, false>(wa, per_warp, sms, want, wpc, grid, smem);
        return launch_walk<64, 0, float, false>(wa, per_warp, sms, want, wpc, grid, smem);
    }
}

// The walk instantiation a plan launches (for finding its node in a captured graph).
const void *walk_fn_f32(int variant, int M1, bool fq)
{
    if (fq) {
        switch (variant) {
        case 1: return (const void *)walk_kernel<16, 6, float, true>;
        case 2: return (const void *)walk_kernel<32, 3, float, true>;
        case 3: return (const void *)walk_kernel<64, 2, float, true>;
        default:
            {
                if (M1 == 16) return (const void *)walk_kernel<16, 0, float, true>;
                if (M1 == 32) return (const void *)walk_kernel<32, 0, float, true>;
                return (const void *)walk_kernel<64, 0, float, true>;
            }
            return nullptr;
        }
    }
    switch (variant) {
    case 1: return (const void *)walk_kernel<16, 6, float, false>;
    case 2: return (const void *)walk_kernel<32, 3, float, false>;
    case 3: return (const void *)walk_kernel<64, 2, float, false>;
    default:
        if (M1 == 16) return (const void *)walk_kernel<16, 0, float, false>;
        if (M1 == 32) return (const void *)walk_kernel<32, 0, float, false>;
        return (const void *)walk_kernel<64, 0, float, false>;
    }
}

cudaError_t walk_run_f32(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                         cudaStream_t st)
{
    if (fq) {
        switch (variant) {
        case 1: return run_walk<16, 6, float, true>(wa, smem, wpc, grid, st);
        case 2: return run_walk<32, 3, float, true>(wa, smem, wpc, grid, st);
        case 3: return run_walk<64, 2, float, true>(wa, smem, wpc, grid, st);
        default:
            {
                if (M1 == 16) return run_walk<16, 0, float, true>(wa, smem, wpc, grid, st);
                if (M1 == 32) return run_walk<32, 0, float, true>(wa, smem, wpc, grid, st);
                return run_walk<64, 0, float, true>(wa, smem, wpc, grid, st);
            }
            return cudaErrorInvalidValue;
        }
    }
    switch (variant) {
    case 1: return run_walk<16, 6, float, false>(wa, smem, wpc, grid, st);
    case 2: return run_walk<32, 3, float, false>(wa, smem, wpc, grid, st);
    case 3: return run_walk<64, 2, float, false>(wa, smem, wpc, grid, st);
    default:
        if (M1 == 16) return run_walk<16, 0, float, false>(wa, smem, wpc, grid, st);
        if (M1 == 32) return run_walk<32, 0, float, false>(wa, smem, wpc, grid, st);
        return run_walk<64, 0, float, false>(wa, smem, wpc, grid, st);
    }
}


}  // namespace lc

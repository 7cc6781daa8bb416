// Walk kernel instantiations with the level-1 codebook in FP16, and their dispatch
// (compiled apart from lc_search.cu so the instantiations build in parallel).
#include "lc_walk.cuh"

namespace lc {

// Dispatch on (sub-space width variant, codebook element type, full walk).  The full walk
// exists for the uniform splits (variants 1-3); in FP16 only for those.
cudaError_t walk_config_f16(int variant, int M1, bool fq, const WalkArgs &wa, size_t per_warp, int sms, int want,
                            int *wpc, int *grid, size_t *smem)
{
    if (fq) {
        switch (variant) {
        case 1: return launch_walk<16, 6, __half, true>(wa, per_warp, sms, want, wpc, grid, smem);
        case 2: return launch_walk<32, 3, __half, true>(wa, per_warp, sms, want, wpc, grid, smem);
        case 3: return launch_walk<64, 2, __half, true>(wa, per_warp, sms, want, wpc, grid, smem);
        default:
            return cudaErrorInvalidValue;
        }
    }
    switch (variant) {
    case 1: return launch_walk<16, 6, __half, false>(wa, per_warp, sms, want, wpc, grid, smem);
    case 2: return launch_walk<32, 3, __half, false>(wa, per_warp, sms, want, wpc, grid, smem);
    case 3: return launch_walk<64, 2, __half, false>(wa, per_warp, sms, want, wpc, grid, smem);
    default:
        if (M1 == 16) return launch_walk<16, 0, __half, false>(wa, per_warp, sms, want, wpc, grid, smem);
        if (M1 == 32) return launch_walk<32, 0, __half, false>(wa, per_warp, sms, want, wpc, grid, smem);
        return launch_walk<64, 0, __half, false>(wa, per_warp, sms, want, wpc, grid, smem);
    }
}

// The walk instantiation a plan launches (for finding its node in a captured graph).
const void *walk_fn_f16(int variant, int M1, bool fq)
{
    if (fq) {
        switch (variant) {
        case 1: return (const void *)walk_kernel<16, 6, __half, true>;
        case 2: return (const void *)walk_kernel<32, 3, __half, true>;
        case 3: return (const void *)walk_kernel<64, 2, __half, true>;
        default:
            return nullptr;
        }
    }
    switch (variant) {
    case 1: return (const void *)walk_kernel<16, 6, __half, false>;
    case 2: return (const void *)walk_kernel<32, 3, __half, false>;
    case 3: return (const void *)walk_kernel<64, 2, __half, false>;
    default:
        if (M1 == 16) return (const void *)walk_kernel<16, 0, __half, false>;
        if (M1 == 32) return (const void *)walk_kernel<32, 0, __half, false>;
        return (const void *)walk_kernel<64, 0, __half, false>;
    }
}

cudaError_t walk_run_f16(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                         cudaStream_t st)
{
    if (fq) {
        switch (variant) {
        case 1: return run_walk<16, 6, __half, true>(wa, smem, wpc, grid, st);
        case 2: return run_walk<32, 3, __half, true>(wa, smem, wpc, grid, st);
        case 3: return run_walk<64, 2, __half, true>(wa, smem, wpc, grid, st);
        default:
            return cudaErrorInvalidValue;
        }
    }
    switch (variant) {
    case 1: return run_walk<16, 6, __half, false>(wa, smem, wpc, grid, st);
    case 2: return run_walk<32, 3, __half, false>(wa, smem, wpc, grid, st);
    case 3: return run_walk<64, 2, __half, false>(wa, smem, wpc, grid, st);
    default:
        if (M1 == 16) return run_walk<16, 0, __half, false>(wa, smem, wpc, grid, st);
        if (M1 == 32) return run_walk<32, 0, __half, false>(wa, smem, wpc, grid, st);
        return run_walk<64, 0, __half, false>(wa, smem, wpc, grid, st);
    }
}


}  // namespace lc

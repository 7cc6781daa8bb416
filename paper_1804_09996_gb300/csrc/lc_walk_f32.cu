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

// The same dispatch as above for a generic launcher f(WalkShape<M1, D1, FQ>).
template <typename F>
static cudaError_t by_shape(int variant, int M1, bool fq, F &&f)
{
    if (fq) {
        switch (variant) {
        case 1: return f(WalkShape<16, 6, true>{});
        case 2: return f(WalkShape<32, 3, true>{});
        case 3: return f(WalkShape<64, 2, true>{});
        default: return M1 == 16 ? f(WalkShape<16, 0, true>{}) : M1 == 32 ? f(WalkShape<32, 0, true>{})
                                           : f(WalkShape<64, 0, true>{});
        }
    }
    switch (variant) {
    case 1: return f(WalkShape<16, 6, false>{});
    case 2: return f(WalkShape<32, 3, false>{});
    case 3: return f(WalkShape<64, 2, false>{});
    default: return M1 == 16 ? f(WalkShape<16, 0, false>{}) : M1 == 32 ? f(WalkShape<32, 0, false>{})
                                                             : f(WalkShape<64, 0, false>{});
    }
}

cudaError_t descent_config_f32(int variant, int M1, bool fq, const WalkArgs &wa, int sms, int *wpc, int *grid,
                               size_t *smem)
{
    return by_shape(variant, M1, fq, [&](auto t) {
        using T = decltype(t);
        return launch_descent<T::M1, T::D1, float, T::FQ>(wa, sms, wpc, grid, smem);
    });
}

cudaError_t descent_run_f32(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                            cudaStream_t st)
{
    return by_shape(variant, M1, fq, [&](auto t) {
        using T = decltype(t);
        return run_descent<T::M1, T::D1, float, T::FQ>(wa, smem, wpc, grid, st);
    });
}

}  // namespace lc

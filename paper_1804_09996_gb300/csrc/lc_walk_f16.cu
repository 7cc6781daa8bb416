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

// The same dispatch as above for a generic launcher f(WalkShape<M1, D1, FQ>).
template <typename F>
static cudaError_t by_shape(int variant, int M1, bool fq, F &&f)
{
    if (fq) {
        switch (variant) {
        case 1: return f(WalkShape<16, 6, true>{});
        case 2: return f(WalkShape<32, 3, true>{});
        case 3: return f(WalkShape<64, 2, true>{});
        default: return cudaErrorInvalidValue;
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

cudaError_t descent_config_f16(int variant, int M1, bool fq, const WalkArgs &wa, int sms, int *wpc, int *grid,
                               size_t *smem)
{
    return by_shape(variant, M1, fq, [&](auto t) {
        using T = decltype(t);
        return launch_descent<T::M1, T::D1, __half, T::FQ>(wa, sms, wpc, grid, smem);
    });
}

cudaError_t descent_run_f16(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                            cudaStream_t st)
{
    return by_shape(variant, M1, fq, [&](auto t) {
        using T = decltype(t);
        return run_descent<T::M1, T::D1, __half, T::FQ>(wa, smem, wpc, grid, st);
    });
}

cudaError_t walk_config_tab(const WalkArgs &wa, size_t per_warp, int sms, int want, int *wpc, int *grid, size_t *smem)
{
    return launch_walk<32, 3, __half, false, true>(wa, per_warp, sms, want, wpc, grid, smem);
}

cudaError_t walk_run_tab(const WalkArgs &wa, size_t smem, int wpc, int grid, cudaStream_t st)
{
    return run_walk<32, 3, __half, false, true>(wa, smem, wpc, grid, st);
}

const void *walk_fn_tab() { return (const void *)walk_kernel<32, 3, __half, false, true>; }

cudaError_t descent_config_tab(const WalkArgs &wa, int sms, int *wpc, int *grid, size_t *smem)
{
    return launch_descent<32, 3, __half, false, true>(wa, sms, wpc, grid, smem);
}

cudaError_t descent_run_tab(const WalkArgs &wa, size_t smem, int wpc, int grid, cudaStream_t st)
{
    return run_descent<32, 3, __half, false, true>(wa, smem, wpc, grid, st);
}

}  // namespace lc

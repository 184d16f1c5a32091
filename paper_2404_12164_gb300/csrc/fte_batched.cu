// Ensemble variants of the step kernel (many parameter sets in one launch):
// per-set tallies either in shared memory (all sets' bins per block) or merged
// per warp into FP64 accumulators in global memory, at 128 or 256 threads per
// block, for the cell or the pair record layout (compile-time, as for the
// single-set kernels).  The step arithmetic is the single-set kernel's (fte_step.cuh).
#include "fte_step.cuh"

namespace fte {

template <int MODE, int NT, int LAY>
static const void* pick(int kperp, int dtype)
{
    if (dtype == FTE_BF16)
        return kperp ? (const void*)advance_kernel<true, FTE_BF16, MODE, NT, LAY>
                     : (const void*)advance_kernel<false, FTE_BF16, MODE, NT, LAY>;
    if (dtype == FTE_F16)
        return kperp ? (const void*)advance_kernel<true, FTE_F16, MODE, NT, LAY>
                     : (const void*)advance_kernel<false, FTE_F16, MODE, NT, LAY>;
    return kperp ? (const void*)advance_kernel<true, FTE_F32, MODE, NT, LAY>
                 : (const void*)advance_kernel<false, FTE_F32, MODE, NT, LAY>;
}

template <int MODE, int NT>
static const void* pick_layout(int kperp, int dtype, int pair)
{
    return pair ? pick<MODE, NT, kLayPair>(kperp, dtype) : pick<MODE, NT, kLayCell>(kperp, dtype);
}

const void* advance_fn_batched(int kperp, int dtype, int mode, int nt, int pair)
{
    if (mode == kModeShared) {
        if (nt == 128) return pick_layout<kModeShared, 128>(kperp, dtype, pair);
        if (nt == 256) return pick_layout<kModeShared, 256>(kperp, dtype, pair);
    } else if (mode == kModeGlobal) {
        if (nt == 128) return pick_layout<kModeGlobal, 128>(kperp, dtype, pair);
        if (nt == 256) return pick_layout<kModeGlobal, 256>(kperp, dtype, pair);
    }
    return nullptr;
}

cudaError_t launch_advance_batched(const AdvanceArgs& a, const BatchArgs& b, int kperp, int mode, int nt,
                                   int blocks, size_t smem, cudaStream_t s)
{
    const void* fn = advance_fn_batched(kperp, a.g.dtype, mode, nt, a.g.pair);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&a, (void*)&b};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(nt), args, smem, s);
}

}  // namespace fte

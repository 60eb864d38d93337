// pd_fft.cu -- TBT part of K u by FFT (placeholder until the tile kernel lands).
#include "pd_internal.cuh"

namespace pd {
int fft_prepare(pd_grid *) { return PD_OK; }
int launch_fft_tile(pd_grid *, bool, const MatvecArgs &, cudaStream_t)
{
    return fail(PD_ERR_INVALID, "FFT method not built");
}
}  // namespace pd

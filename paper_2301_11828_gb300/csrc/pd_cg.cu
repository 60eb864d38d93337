// pd_cg.cu -- conjugate gradients (placeholder).
#include "pd_internal.cuh"

extern "C" int pd_cg_solve(pd_grid *, const double *, double *, double, int, uint32_t, pd_cg_stats *, void *)
{
    return pd::fail(PD_ERR_INVALID, "CG not built");
}

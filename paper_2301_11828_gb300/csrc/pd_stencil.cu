// pd_stencil.cu -- dispatch of the shared-memory tiled neighbour-sum kernels
// (pd_stencil2d.cu, pd_direct2d.cu, pd_stencil3d.cu) and the coefficient lookup
// the host uses to pack their parameter tables.
#include <vector>

#include "pd_stencil.cuh"

namespace pd {

void coef_of(const pd_grid *g, int ox, int oy, int oz, bool unit, double *c)
{
    const int nc = ncoef(g->dim);
    int k = -1;
    for (int i = 0; i < g->nnb; ++i)
        if (g->off[3 * i] == ox && g->off[3 * i + 1] == oy && g->off[3 * i + 2] == oz) {
            k = i;
            break;
        }
    const double s = unit ? 1.0 : g->E;
    for (int i = 0; i < nc; ++i) c[i] = (k >= 0) ? g->coef1[(size_t)nc * k + i] * s : 0.0;
}

int launch_stencil(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s)
{
    if (a.batch < 1 || a.batch > 65535) return fail(PD_ERR_INVALID, "batch must be in [1, 65535]");
    if (g->dim == 2) {
        if (a.use_E || a.use_mu) return run_direct2d(g, f64, a, s);
        if (!g->no_tma && !a.no_tma && tma_stencil_eligible(g, a, f64)) {
            if (g->stencil_tile_rows == 0 && walk_stencil_eligible(g, a)) return run_tbt2d_walk(g, a, s);
            return run_tbt2d_tma(g, a, s);
        }
        return run_tbt2d(g, f64, a, s);
    }
    return run_tbt3d(g, f64, a, s);
}

int stencil_blocks(pd_grid *g, bool f64, bool direct)
{
    const int M = g->M;
    if (g->dim == 2) {
        const int R = direct ? (f64 ? 2 : 4) : (f64 ? (M <= 4 ? 4 : 2) : 8);
        const int TY = kGY2 * R;
        return (int)(((g->n[0] + kTX2 - 1) / kTX2) * ((g->n[1] + TY - 1) / TY));
    }
    const int R = 4;   // the smaller of the 3D forms' z-rows per thread (the most CTAs)
    return (int)(((g->n[0] + kTX3 - 1) / kTX3) * ((g->n[1] + kTY3 - 1) / kTY3) * ((g->n[2] + R - 1) / R));
}

}  // namespace pd

// pd_cg.cuh -- device state shared by the CG driver (pd_cg.cu) and the
// persistent inner loop (pd_cg_persist.cu).
#pragma once
#include <cstdint>

#include "pd_internal.cuh"

namespace pd {

// Scalars of one CG solve, kept on the device between launches.
struct CgScal {
    double rr;            // r.r of the current iterate
    double pq;            // p.q, written by the fused matvec dot
    double rr_new;        // r.r after the update (last block)
    double tol2;          // inner loop stops when rr <= tol2
    double beta;          // beta of the next direction p = r + beta p_old
    double aux;           // scratch for the host-driven reductions
    int done;
    int iters;
    unsigned int retire[4];
    int pbuf;             // persistent loop: which of the two direction buffers holds p_old
};

// Two-level grid barrier / all-reduce of the persistent loop (zero-initialised;
// every counter returns to zero after each use).  Counters sit on their own
// 128-byte lines.
struct __align__(128) CgBarGroup {
    unsigned int count;
    unsigned int pad[31];
};
struct __align__(128) CgBar {
    CgBarGroup grp[32];
    unsigned int top;
    unsigned int pad0[31];
    unsigned int gen;
    unsigned int pad1[31];
    double gsum[32][2];
    double total[2];
};

// True when the FP32 inner loop of the mixed CG runs as one persistent
// cooperative kernel on this grid: 2D, constant modulus, no broken bonds, TMA
// eligible, stencil method, cooperative launch supported, and every tile in one
// wave of resident CTAs (beyond that, graph-replayed launches are as fast).
bool cg_persist_eligible(const pd_grid *g);

// Grid size (CTAs) the persistent kernel is launched with on this grid.
int cg_persist_ctas(const pd_grid *g);

// Vectors of the persistent loop (FP32, [2][N] each, 16-byte aligned).
// hi + lo += v with the rounding error of the add kept in lo (two-sum of Knuth).
// The FP32 solution increment is accumulated this way: each rounding of a
// plain FP32 sum would be amplified by K up to its condition number and open a
// gap between the recursive residual and b - K x as large as the residual on
// fine grids.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v)
{
    const float s = hi + v, bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

struct CgVecs {
    float *x, *xlo, *r, *q;   // x + xlo: the FP32 increment as an unevaluated sum
    float *p[2];   // direction, double-buffered: tiles read p_old from one while CTAs write p to the other
};

// Runs inner iterations of the FP32 CG until r.r <= sc->tol2 or `budget`
// iterations (state in sc: rr, beta, pbuf = index of p_old, iters, done).
// part holds >= 2 * cg_persist_ctas(g) doubles, gbar a zero-initialised
// barrier, tile_flags one byte per 64 x 32 tile (1 = the tile has a
// constrained node).
int cg_persist_run(pd_grid *g, const CgVecs &v, CgScal *sc, CgBar *gbar, double *part, const uint8_t *tile_flags,
                   int budget, cudaStream_t s);

// The graph-replayed form of the same loop on 2D TMA-eligible grids (any size):
// per iteration cg_dirmv_run (direction p = r + beta p_old formed from the TMA
// boxes, q = P K P p, p.q into sc->pq) then the update kernel of pd_cg.cu.
bool cg_dirmv_eligible(const pd_grid *g);
int cg_dirmv_run(pd_grid *g, const CgVecs &v, CgScal *sc, double *partial, const uint8_t *tile_flags, cudaStream_t s);

// tile_flags[t] = 1 when tile t (64 x 32 outputs, row-major over tiles) holds a
// constrained node.
int cg_persist_tile_flags(pd_grid *g, uint8_t *tile_flags, cudaStream_t s);
int cg_persist_ntiles(const pd_grid *g);

}  // namespace pd

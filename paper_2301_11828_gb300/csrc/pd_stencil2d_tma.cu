// pd_stencil2d_tma.cu -- FP32 2D stencil (TBT form, Sec. 3.2-3.4) for sm_103a:
// persistent CTAs, TMA-fed multi-buffered halo tiles, packed FP32x2 math.
//
// Same operator as pd_stencil2d.cu:
//     (K u)_p = Kd_p u_p - sum_{o in half} c(o) (u~_{p+o} + u~_{p-o}),
// with u~ zero outside the grid.  Differences in how it is computed:
//   * The halo box of a tile (both components) is fetched by one
//     cp.async.bulk.tensor (TMA) per tile into shared memory.  The tensor
//     map's out-of-bounds fill supplies the zero padding outside the grid, so
//     no thread tests bounds on the way in.  While a CTA computes one tile the
//     TMA engine already loads its next kStages - 1 tiles into the other
//     buffers (enough bytes in flight per SM to cover HBM latency); an mbarrier
//     per buffer with an expected byte count signals arrival.  Every wait has an
//     iteration limit; on expiry the kernel records an error code and returns.
//   * The x start of the box is rounded down to a 16-byte boundary (TMA rule)
//     and the box is widened to cover the halo.
//   * Buffers are released per warp: each warp arrives on the buffer's "empty"
//     mbarrier when it has read its columns, and thread 0 waits on that
//     barrier (bounded) before loading the buffer again.  Warps of a CTA drift
//     up to kStages - 1 tiles apart instead of meeting at a block barrier
//     after every tile (edge outputs take longer than interior ones).  When
//     the input has to be projected (all threads rewrite the box), and for
//     M > 3 (two CTAs per SM), the CTA runs in lockstep with block barriers.
//   * For each offset pair the two components are handled as one packed
//     FP32x2 value s = (s_x, s_y): the accumulators a1 += (cxx, cyy) * s and
//     a2 += (cxy, cxy) * s give (K u) after the final swap
//     a_x = a1.x + a2.y, a_y = a1.y + a2.x -- one packed add and two packed
//     fused multiply-adds per pair instead of six scalar instructions.
//   * With projection, only the tiles that hold a constrained output (or, for
//     the input, a constrained node within the halo) take the masking paths;
//     per-tile flags are computed once per grid (the constraints are fixed).
// k_tbt2d_tma is the pair form (PD_PAIR_FORM, kept for comparison): its terms
// cancel on smooth fields.  The default FP32 product is k_tbt2d_acc (below):
// the same pipeline, with the sums taken as differences of nearby values.
// Used for FP32 grids whose row length is a multiple of 4 floats (TMA stride
// rule); other grids use the plain kernel.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "pd_stencil.cuh"
#include "pd_tma2d.cuh"

namespace pd {

namespace {

using namespace tma2d;

constexpr int kStages = 3;               // halo tiles in flight or in use per CTA

// Three CTAs per SM (three halo tiles in flight each) up to M = 4 (M = 3 in
// the difference form); register growth beyond that leaves two.
template <int M, bool DIFF>
__global__ void __launch_bounds__(kThreads, (M <= 3 || (M == 4 && !DIFF) ? 3 : 2))
k_tbt2d_tma(const __grid_constant__ CUtensorMap map, const float *__restrict__ u, float *__restrict__ out, int nx,
            int ny, int64_t N, int tiles_x, int tiles_y, int ntiles, const uint8_t *__restrict__ cons,
            int project_in, int project_out, const uint8_t *__restrict__ tflags, const float *__restrict__ kd,
            float scale, PackTab<M> tab,
            double *dot_partial, double *dot_out, unsigned int *retire, int *err)
{
    constexpr int XL = x_lead<M>(), BX = box_x<M>(), BY = box_y<M>(), WL = kRt + 2 * M;
    constexpr int PLANE = BX * BY;
    constexpr uint32_t kBytes = 2u * PLANE * sizeof(float);
    constexpr int NP = PackTab<M>::kPairs;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *const sbase = reinterpret_cast<float *>(smem_raw);   // buffer k at sbase + 2 * PLANE * k
    __shared__ __align__(8) uint64_t bars[kStages];    // full: the tile has landed
    __shared__ __align__(8) uint64_t empty[kStages];   // every warp has read the buffer
    __shared__ int s_abort;
    // Edge-class diagonal table (Kd by clipped face distances), kept in shared
    // memory when small so that edge outputs do not wait on global loads.
    constexpr int KDS = (M <= 3) ? 3 * (M + 1) * (M + 1) * (M + 1) * (M + 1) : 1;
    __shared__ float s_kd[KDS];
    if (M <= 3)
        for (int i = threadIdx.x; i < KDS; i += kThreads) s_kd[i] = __ldg(kd + i);

    if (threadIdx.x == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&bars[k], 1);
            mbar_init(&empty[k], kThreads / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();
    // lockstep (block barriers): when the box is rewritten by all threads, and for M > 3, where
    // two CTAs per SM leave too few warps to cover warp 0 waiting for the slowest one
    // (measured: M = 6 ran 15 % slower with per-warp release, M = 3 4 % faster)
    const bool lockstep = project_in != 0 || M > 3;
    const int lane = threadIdx.x & 31;

    const int tx = threadIdx.x % kTXt, ty = threadIdx.x / kTXt;
    // Tile t lies in tile row r = t / tiles_x; the columns of each row are
    // rotated by r so that a persistent CTA, which takes every gridDim.x-th
    // tile, meets left/right edge tiles (slower epilogue) as often as the others.
    auto tile_coords = [&](int t, int &x0, int &y0, int &b) {
        const int r = t / tiles_x;
        x0 = ((t - r * tiles_x + r) % tiles_x) * kTXt;
        y0 = (r % tiles_y) * kTYt;
        b = r / tiles_y;
    };
    auto issue = [&](int t, int which) {
        int x0, y0, b;
        tile_coords(t, x0, y0, b);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[which], kBytes);
        tma_load_3d(sbase + 2 * PLANE * which, &map, x0 - XL, y0 - M, 2 * b, &bars[which]);
    };

    // The CTA's k-th tile is blockIdx.x + k * gridDim.x; it lands in buffer k % kStages,
    // whose barrier completes its (k / kStages)-th phase.  kStages - 1 loads run ahead.
    int it = 0, n_issued = 0;   // n_issued: loads issued so far (thread 0 only)
    if (threadIdx.x == 0)
        for (int k = 0; k < kStages - 1; ++k) {
            const int64_t tk = blockIdx.x + (int64_t)k * gridDim.x;
            if (tk < ntiles) {
                issue((int)tk, k);
                ++n_issued;
            }
        }
    double dot_blk_total = 0.0;   // per-thread, summed over this CTA's tiles (dot needs one batch)
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int cur = it % kStages;
        if (threadIdx.x == 0) {
            // the next load goes to buffer (it - 1) % kStages, free once every warp has
            // released its use it - 1 (lockstep: the block barrier that ended it - 1)
            const int64_t tn = t + (int64_t)(kStages - 1) * gridDim.x;
            if (tn < ntiles) {
                const int prev = (it + kStages - 1) % kStages;
                if (lockstep || it == 0 || mbar_wait(&empty[prev], ((it - 1) / kStages) & 1)) {
                    issue((int)tn, prev);
                    ++n_issued;
                } else {
                    atomicExch(err, 1);   // the warps waiting for that tile give up in turn
                    s_abort = 1;
                }
            }
        }
        const bool ok = mbar_wait(&bars[cur], (it / kStages) & 1);
        if (lockstep) {
            if (!ok) {
                atomicExch(err, 1);
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) break;
        } else if (__any_sync(0xffffffffu, !ok)) {   // warp-uniform decision
            if (lane == 0) {
                atomicExch(err, 1);
                s_abort = 1;
            }
            break;
        }
        int x0, y0, b;
        tile_coords(t, x0, y0, b);
        float *sx = sbase + 2 * PLANE * cur, *sy = sx + PLANE;
        // projection where this tile needs it (uniform over the CTA; nothing to decide
        // when the launch projects nothing)
        bool pin = false, pout = false;
        if (project_in | project_out) {
            const uint8_t tf = tflags ? __ldg(tflags + (y0 / kTYt) * tiles_x + x0 / kTXt) : 3;
            pin = project_in && (tf & 2);
            pout = project_out && (tf & 1);
        }
        if (pin) {
            for (int e = threadIdx.x; e < PLANE; e += kThreads) {
                const int gx = x0 - XL + e % BX, gy = y0 - M + e / BX;
                if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                    const uint8_t m = __ldg(cons + (int64_t)gy * nx + gx);
                    if (m & 1) sx[e] = 0.f;
                    if (m & 2) sy[e] = 0.f;
                }
            }
            __syncthreads();
        }

        // The tile body is instantiated twice: tiles whose every output keeps a
        // full horizon inside the grid (and need no projection or dot) take a
        // copy without the edge table, bounds tests and projection, so the
        // compiler schedules the common case without the rare paths.
        auto tile_body = [&](auto EDGE) {
            constexpr bool edge = decltype(EDGE)::value;
            u64 a1[kRt], a2[kRt], w0[WL];
            tile_pairs<M, DIFF>(sx + (ty * kRt) * BX + tx + XL, sy + (ty * kRt) * BX + tx + XL, tab, a1, a2, w0);

            float *ob = out + (int64_t)b * 2 * N;
            const int gx = x0 + tx;
            // outputs whose horizon stays inside the grid: interior Kd (none in the
            // difference form), no tests
            auto interior_epilogue = [&]() {
                const float kxx = tab.v[4 * NP], kxy = tab.v[4 * NP + 1], kyy = tab.v[4 * NP + 2];
                float *o0 = ob + (int64_t)(y0 + ty * kRt) * nx + gx;
#pragma unroll
                for (int r = 0; r < kRt; ++r) {
                    const float2 x1 = upk(a1[r]), x2 = upk(a2[r]);
                    float fx, fy;
                    if constexpr (DIFF) {
                        fx = -(x1.x + x2.y);
                        fy = -(x1.y + x2.x);
                    } else {
                        const float2 up = upk(w0[r + M]);
                        fx = __fmaf_rn(kxx, up.x, __fmaf_rn(kxy, up.y, -(x1.x + x2.y)));
                        fy = __fmaf_rn(kxy, up.x, __fmaf_rn(kyy, up.y, -(x1.y + x2.x)));
                    }
                    o0[(int64_t)r * nx] = fx * scale;
                    o0[(int64_t)r * nx + N] = fy * scale;
                }
            };
            if constexpr (!edge) {
                interior_epilogue();
            } else {
                // General epilogue.  Every branch below is uniform over the tile or
                // the warp, so tiles and warps that need no edge handling do not
                // execute it, predicated off or otherwise.
                const bool full = (x0 + kTXt <= nx) && (y0 + kTYt <= ny);   // no bounds test needed
                const bool lane_xe = (gx < M) || (gx >= nx - M);
                const bool warp_xe = __any_sync(0xffffffffu, lane_xe);     // warp holds an x-edge output
                const int gy0 = y0 + ty * kRt;
                const bool warp_ye = (gy0 < M) || (gy0 + kRt > ny - M);     // warp holds a y-edge row
                if (full && !warp_xe && !warp_ye && !pout && !dot_partial) {
                    interior_epilogue();   // this warp's outputs are all interior
                    return;
                }
                // Edge class of output (gx, gy): clipped face distances, lane part xc
                // once per tile, row part per output row (warp-uniform).
                const int xc = min(gx, M) * (M + 1) + min(nx - 1 - gx, M);
                float *o0 = ob + (int64_t)gy0 * nx + gx;
                const uint8_t *m0 = cons + (int64_t)gy0 * nx + gx;
                float dot = 0.f;
#pragma unroll
                for (int r = 0; r < kRt; ++r) {
                    const int gy = gy0 + r;
                    if (!full && !(gx < nx && gy < ny)) continue;
                    const float2 up = upk(w0[r + M]);
                    const float2 x1 = upk(a1[r]), x2 = upk(a2[r]);
                    const float ax = x1.x + x2.y, ay = x1.y + x2.x;
                    const int cls = xc * ((M + 1) * (M + 1)) + min(gy, M) * (M + 1) + min(ny - 1 - gy, M);
                    float kxx, kxy, kyy;
                    if constexpr (M <= 3) {
                        kxx = s_kd[3 * cls];
                        kxy = s_kd[3 * cls + 1];
                        kyy = s_kd[3 * cls + 2];
                    } else {
                        kxx = __ldg(kd + 3 * cls);
                        kxy = __ldg(kd + 3 * cls + 1);
                        kyy = __ldg(kd + 3 * cls + 2);
                    }
                    if constexpr (DIFF) {   // the sums already hold -Kd_int u_p
                        kxx -= tab.v[4 * NP];
                        kxy -= tab.v[4 * NP + 1];
                        kyy -= tab.v[4 * NP + 2];
                    }
                    float fx = __fmaf_rn(kxx, up.x, __fmaf_rn(kxy, up.y, -ax));
                    float fy = __fmaf_rn(kxy, up.x, __fmaf_rn(kyy, up.y, -ay));
                    if (pout) {
                        const uint8_t m = __ldg(m0 + (int64_t)r * nx);
                        if (m & 1) fx = 0.f;
                        if (m & 2) fy = 0.f;
                    }
                    fx *= scale;
                    fy *= scale;
                    o0[(int64_t)r * nx] = fx;
                    o0[(int64_t)r * nx + N] = fy;
                    if (dot_partial) dot = __fmaf_rn(up.x, fx, __fmaf_rn(up.y, fy, dot));
                }
                if (dot_partial) dot_blk_total += (double)dot;
            }
        };
        const bool interior = (x0 >= M) && (x0 + kTXt <= nx - M) && (y0 >= M) && (y0 + kTYt <= ny - M);
        if (interior && !pout && !dot_partial)
            tile_body(std::false_type{});
        else
            tile_body(std::true_type{});
        if (lockstep) {
            __syncthreads();   // all reads of buf[cur] done before it is refilled
        } else {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[cur]);   // this warp's reads of buf[cur] are done
        }
    }
    __syncthreads();   // every warp has left the loop (and s_abort is visible)
    if (s_abort) {
        // let the copies still in flight land (bounded waits) before the CTA exits
        if (threadIdx.x == 0)
            for (int k = it; k < n_issued; ++k) mbar_wait(&bars[k % kStages], (k / kStages) & 1);
        return;
    }
    if (dot_partial) {
        // single-field launches only (batch == 1): one partial per CTA
        __shared__ double red[kThreads / 32];
        const double s = block_sum(dot_blk_total, red);
        grid_finish(s, gridDim.x, blockIdx.x, dot_partial, dot_out, retire, red);
    }
}

// Unsigned division by a divisor fixed per launch, by multiplication and shifts
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, the unsigned N-bit algorithm): the tile walk
// decomposes tile numbers without the ~20-instruction integer division.
struct FastDiv {
    uint32_t d, m, s1, s2;
};
inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 0 ? l - 1 : 0;
    return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f)
{
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Accurate FP32 product (the default for FP32 2D grids): the same persistent
// TMA pipeline, with the pair sums evaluated as differences (tile_eg for warps
// whose outputs all have their whole horizon inside the grid, tile_diff with
// out-of-grid terms dropped elsewhere), so that K u = -a with no diagonal term
// to cancel against.  The coefficients carry -scale.  Tiles of 64 columns by
// 8 GY rows (GY = 2, 4 or 8 warps' worth of rows; 64 x 64 the default at M <= 3,
// measured 2 % faster than 64 x 32 there and slower at M = 4).  Two CTAs per SM
// up to M = 4 with 64 x 32 or 64 x 16 tiles (about 120 registers); one with
// 64 x 64 tiles (512 threads) and beyond M = 4, where the shared differences of
// the interior form need up to 250 registers (measured faster than two CTAs
// with spills, or the plain difference form).
constexpr int kAccStages = 3;   // halo tiles in flight or in use per CTA
template <int M, int GY>
__global__ void __launch_bounds__(64 * GY, (M <= 4 && GY <= 4 ? 2 : 1))
k_tbt2d_acc(const __grid_constant__ CUtensorMap map, float *__restrict__ out, int nx, int ny, int64_t N,
            int ybuf0, int ty0, int yend, int tiles_x, int tiles_y, FastDiv div_tx, FastDiv div_ty, int ntiles,
            const uint8_t *__restrict__ cons,
            int project_in, int project_out, const uint8_t *__restrict__ tflags, AccTab<M> tab,
            double *dot_partial, double *dot_out, unsigned int *retire, int *err)
{
    constexpr int TH = 64 * GY, TYt = GY * kRt;   // threads; tile rows
    constexpr int XL = x_lead<M>(), BX = box_x<M>(), BY = TYt + 2 * M;
    constexpr int PLANE = BX * BY;
    constexpr uint32_t kBytes = 2u * PLANE * sizeof(float);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *const sbase = reinterpret_cast<float *>(smem_raw);   // buffer k at sbase + 2 * PLANE * k
    __shared__ __align__(8) uint64_t bars[kAccStages];    // full: the tile has landed
    __shared__ __align__(8) uint64_t empty[kAccStages];   // every warp has read the buffer
    __shared__ int s_abort;

    if (threadIdx.x == 0) {
        for (int k = 0; k < kAccStages; ++k) {
            mbar_init(&bars[k], 1);
            mbar_init(&empty[k], TH / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();
    const bool lockstep = project_in != 0 || M > 3;
    const int lane = threadIdx.x & 31;
    const int tx = threadIdx.x % kTXt, ty = threadIdx.x / kTXt;
    // Tile t: tile row R = t / tiles_x (field b = R / tiles_y, row ty0 + R % tiles_y of
    // the grid's tiling); the columns of a row are rotated by R so that a persistent
    // CTA meets edge tiles as often as the others.  Rows are grid rows throughout;
    // the input buffer starts at grid row ybuf0 and the output at grid row 32 ty0,
    // and outputs are stored up to grid row yend (the whole grid: 0, 0, ny).
    auto tile_coords = [&](int t, int &x0, int &y0, int &b) {
        const uint32_t R = fdiv((uint32_t)t, div_tx);
        uint32_t c = (uint32_t)t - R * (uint32_t)tiles_x + R;
        c -= fdiv(c, div_tx) * (uint32_t)tiles_x;
        const uint32_t bq = fdiv(R, div_ty);
        x0 = (int)c * kTXt;
        y0 = ty0 * kTYt + (int)(R - bq * (uint32_t)tiles_y) * TYt;
        b = (int)bq;
    };
    auto issue = [&](int t, int which) {
        int x0, y0, b;
        tile_coords(t, x0, y0, b);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[which], kBytes);
        tma_load_3d(sbase + 2 * PLANE * which, &map, x0 - XL, y0 - M - ybuf0, 2 * b, &bars[which]);
    };

    int it = 0, n_issued = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kAccStages - 1; ++k) {
            const int64_t tk = blockIdx.x + (int64_t)k * gridDim.x;
            if (tk < ntiles) {
                issue((int)tk, k);
                ++n_issued;
            }
        }
    double dot_blk_total = 0.0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int cur = it % kAccStages;
        if (threadIdx.x == 0) {
            const int64_t tn = t + (int64_t)(kAccStages - 1) * gridDim.x;
            if (tn < ntiles) {
                const int prev = (it + kAccStages - 1) % kAccStages;
                if (lockstep || it == 0 || mbar_wait(&empty[prev], ((it - 1) / kAccStages) & 1)) {
                    issue((int)tn, prev);
                    ++n_issued;
                } else {
                    atomicExch(err, 1);
                    s_abort = 1;
                }
            }
        }
        const bool ok = mbar_wait(&bars[cur], (it / kAccStages) & 1);
        if (lockstep) {
            if (!ok) {
                atomicExch(err, 1);
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) break;
        } else if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) {
                atomicExch(err, 1);
                s_abort = 1;
            }
            break;
        }
        int x0, y0, b;
        tile_coords(t, x0, y0, b);
        float *sx = sbase + 2 * PLANE * cur, *sy = sx + PLANE;
        bool pin = false, pout = false;
        if (project_in | project_out) {
            // the flags are per 64 x 32 tile of the grid: a taller tile takes the union
            uint8_t tf = tflags ? 0 : 3;
            if (tflags)
                for (int k = 0; k < (TYt + kTYt - 1) / kTYt && y0 + k * kTYt < ny; ++k)
                    tf |= __ldg(tflags + (y0 / kTYt + k) * tiles_x + x0 / kTXt);
            pin = project_in && (tf & 2);
            pout = project_out && (tf & 1);
        }
        if (pin) {
            for (int e = threadIdx.x; e < PLANE; e += TH) {
                const int gx = x0 - XL + e % BX, gy = y0 - M + e / BX;
                if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                    const uint8_t m = __ldg(cons + (int64_t)gy * nx + gx);
                    if (m & 1) sx[e] = 0.f;
                    if (m & 2) sy[e] = 0.f;
                }
            }
            __syncthreads();
        }
        const int gx = x0 + tx, gy0 = y0 + ty * kRt;
        const float *colx = sx + (ty * kRt) * BX + tx + XL, *coly = sy + (ty * kRt) * BX + tx + XL;
        // every output of this warp keeps its whole horizon inside the grid
        const bool tile_in = (x0 >= M) && (x0 + kTXt <= nx - M) && (y0 >= M) && (y0 + TYt <= ny - M);
        const bool warp_in = tile_in || (__all_sync(0xffffffffu, gx >= M && gx < nx - M) && gy0 >= M &&
                                         gy0 + kRt <= ny - M);
        u64 a1[kRt], a2[kRt];
        if (warp_in)
            tile_eg<M>(colx, coly, tab, a1, a2);
        else
            tile_diff<M, true>(colx, coly, tab, a1, a2, gx, nx, gy0 - M, ny);

        float *o0 = out + (int64_t)b * 2 * N + (int64_t)(gy0 - ty0 * kTYt) * nx + gx;
        const bool full = (x0 + kTXt <= nx) && (y0 + TYt <= yend);
        if (full && !pout && !dot_partial) {
#pragma unroll
            for (int r = 0; r < kRt; ++r) {
                const float2 x1 = upk(a1[r]), x2 = upk(a2[r]);
                o0[(int64_t)r * nx] = x1.x + x2.y;
                o0[(int64_t)r * nx + N] = x1.y + x2.x;
            }
        } else {
            const uint8_t *m0 = cons + (int64_t)gy0 * nx + gx;
            float dot = 0.f;
#pragma unroll
            for (int r = 0; r < kRt; ++r) {
                const int gy = gy0 + r;
                if (!full && !(gx < nx && gy < yend)) continue;
                const float2 x1 = upk(a1[r]), x2 = upk(a2[r]);
                float fx = x1.x + x2.y, fy = x1.y + x2.x;
                if (pout) {
                    const uint8_t m = __ldg(m0 + (int64_t)r * nx);
                    if (m & 1) fx = 0.f;
                    if (m & 2) fy = 0.f;
                }
                o0[(int64_t)r * nx] = fx;
                o0[(int64_t)r * nx + N] = fy;
                if (dot_partial)
                    dot = __fmaf_rn(colx[(r + M) * BX], fx, __fmaf_rn(coly[(r + M) * BX], fy, dot));
            }
            if (dot_partial) dot_blk_total += (double)dot;
        }
        if (lockstep) {
            __syncthreads();
        } else {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[cur]);
        }
    }
    __syncthreads();
    if (s_abort) {
        if (threadIdx.x == 0)
            for (int k = it; k < n_issued; ++k) mbar_wait(&bars[k % kAccStages], (k / kAccStages) & 1);
        return;
    }
    if (dot_partial) {
        __shared__ double red[TH / 32];
        const double s = block_sum(dot_blk_total, red);
        grid_finish(s, gridDim.x, blockIdx.x, dot_partial, dot_out, retire, red);
    }
}

// Per 64 x 32 tile: bit 0 when an output node is constrained, bit 1 when a node
// within M of the tile (the part of the halo box the stencil reads) is.
template <int M>
__global__ void k_tma_flags(const uint8_t *__restrict__ cons, int nx, int ny, int tiles_x, int ntiles,
                            uint8_t *__restrict__ flags)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int x0 = (t % tiles_x) * kTXt, y0 = (t / tiles_x) * kTYt;
    uint8_t out = 0, halo = 0;
    for (int y = max(0, y0 - M); y < min(ny, y0 + kTYt + M); ++y)
        for (int x = max(0, x0 - M); x < min(nx, x0 + kTXt + M); ++x) {
            const uint8_t c = cons[(int64_t)y * nx + x];
            halo |= c;
            if (y >= y0 && y < y0 + kTYt && x >= x0 && x < x0 + kTXt) out |= c;
        }
    flags[t] = (out ? 1 : 0) | (halo ? 2 : 0);
}

// ------------------------------------------------------------------ host side
template <int M, bool ACC, int GYA = kGY2>
int run(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    constexpr int BX = box_x<M>(), BY = box_y<M>();
    const int nx = (int)g->n[0], ny = (int)g->n[1];
    // row window (pd_matvec_rows): rows of the input buffer and of the output
    const int in_row0 = (int)a.in_row0, in_rows = a.in_rows < 0 ? ny : (int)a.in_rows;
    const int out_row0 = (int)a.out_row0, out_rows = a.out_rows < 0 ? ny : (int)a.out_rows;
    const bool window = in_rows != ny || out_rows != ny;
    if (window && (!ACC || out_row0 % kTYt != 0 || a.dot_partial))
        return fail(PD_ERR_INVALID, "row windows need the default FP32 form, tile-aligned rows, no fused dot");
    constexpr int GY = ACC ? GYA : kGY2, TH = 64 * GY, TYt = GY * kRt, BYa = TYt + 2 * M;
    CUtensorMap map;
    if (!make_map<M>(&map, a.u, nx, in_rows, a.batch, ACC ? BYa : BY))
        return fail(PD_ERR_CUDA, "tensor map encode failed");
    const size_t smem = ACC ? (size_t)kAccStages * 2 * BX * BYa * sizeof(float)
                            : (size_t)kStages * 2 * BX * BY * sizeof(float);
    void *kern;
    if constexpr (ACC)
        kern = (void *)k_tbt2d_acc<M, GY>;
    else
        kern = (void *)k_tbt2d_tma<M, false>;
    static int attr_done[64] = {0};   // per instantiation
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr_done[dev] = 1;
    }
    const int tiles_x = (nx + kTXt - 1) / kTXt, tiles_y = (out_rows + TYt - 1) / TYt;
    const int64_t nt = (int64_t)tiles_x * tiles_y * a.batch;
    if (nt > (1ll << 30)) return fail(PD_ERR_INVALID, "too many tiles");
    int occ = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TH, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (occ < 1) occ = 1;
    int blocks = (int)std::min<int64_t>(nt, (int64_t)occ * sms);
    if (a.dot_partial && a.batch != 1) return fail(PD_ERR_INVALID, "fused dot needs a single field");
    const uint8_t *tflags = nullptr;
    if (a.project) {   // the constraints are fixed per grid: the flags are computed once
        const int nts = tiles_x * ((ny + kTYt - 1) / kTYt);   // per tile of the whole grid
        if (g->tma_flags_M != M) {
            if (!g->d_tma_flags) PD_CUDA(cudaMalloc(&g->d_tma_flags, (size_t)nts));
            k_tma_flags<M><<<(nts + 127) / 128, 128, 0, s>>>(g->d_cons, nx, ny, tiles_x, nts, g->d_tma_flags);
            PD_CUDA(cudaGetLastError());
            g->tma_flags_M = M;
        }
        tflags = g->d_tma_flags;
    }
    const int pin = (a.project && !a.input_projected) ? 1 : 0, pout = a.project ? 1 : 0;
    if constexpr (ACC) {
        const FastDiv dtx = make_fastdiv((uint32_t)tiles_x), dty = make_fastdiv((uint32_t)tiles_y);
        k_tbt2d_acc<M, GY><<<blocks, TH, smem, s>>>(map, (float *)a.out, nx, ny, (int64_t)out_rows * nx, in_row0,
                                                      out_row0 / kTYt, out_row0 + out_rows, tiles_x, tiles_y, dtx,
                                                      dty, (int)nt, g->d_cons, pin, pout, tflags,
                                                      make_acc<M>(g, a.scale), a.dot_partial, a.dot_out, a.retire,
                                                      g->d_err);
    } else {
        k_tbt2d_tma<M, false><<<blocks, kThreads, smem, s>>>(map, (const float *)a.u, (float *)a.out, nx, ny, g->N,
                                                             tiles_x, tiles_y, (int)nt, g->d_cons, pin, pout, tflags,
                                                             g->d_kd32, (float)a.scale, make_pack<M>(g),
                                                             a.dot_partial, a.dot_out, a.retire, g->d_err);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace

namespace tma2d {
EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}
}  // namespace tma2d

bool tma_stencil_eligible(const pd_grid *g, const MatvecArgs &a, bool f64)
{
    if (f64 || g->dim != 2 || a.use_E || a.use_mu) return false;
    if (g->n[0] % 4 != 0) return false;                       // row stride must be a multiple of 16 bytes
    if (((uintptr_t)a.u & 15) != 0) return false;             // 16-byte aligned base
    return tma2d::encode_fn() != nullptr;
}

int run_tbt2d_tma(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
#define PD_TMA_CASE(m) \
    case m:                                                                                  \
        if (a.pair_form) return run<m, false>(g, a, s);                                      \
        if (m <= 4 && g->stencil_tile_rows == 16) return run<m, true, (m <= 4 ? 2 : kGY2)>(g, a, s); \
        if (m <= 3 && g->stencil_tile_rows == 64) return run<m, true, (m <= 3 ? 8 : kGY2)>(g, a, s); \
        return run<m, true>(g, a, s);
    switch (g->M) {
        PD_TMA_CASE(1)
        PD_TMA_CASE(2)
        PD_TMA_CASE(3)
        PD_TMA_CASE(4)
        PD_TMA_CASE(5)
        PD_TMA_CASE(6)
        PD_TMA_CASE(7)
        PD_TMA_CASE(8)
    }
#undef PD_TMA_CASE
    return fail(PD_ERR_INVALID, "horizon M not compiled for 2D");
}

}  // namespace pd

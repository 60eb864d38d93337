// pd_batch.cu -- many independent static solves (Eq. mat:e2 on plates of
// uneven size and horizon) advanced together: one launch per CG stage serves
// every plate, and the inner iterations run as a captured CUDA graph.
//
// Layout: the vectors of all plates are concatenated (plate i at element
// offset off_i); per plate a descriptor holds its extents, horizon, constraint
// mask, diagonal-block table and coefficient pairs.
//   * Tile kernel: a persistent grid walks the list of 64 x 32 output tiles of
//     all plates (TBT pair form of pd_stencil2d.cu with the plate's own
//     horizon), writing K p and one partial of p.Kp per tile.
//   * Chunk kernels: the concatenated vectors are cut into chunks of at most
//     4096 elements that never straddle two plates; per-plate scalars are
//     re-summed from the tile or chunk partials of that plate in a fixed order
//     (deterministic), partials of r.r are double-buffered by iteration parity.
//   * Converged plates drop out: their tiles and chunks return at once.
//   * Plates are grouped by size (a group's FP32 vectors fit L2); groups are
//     independent and advance concurrently, each on its own stream with its own
//     graph, the host serving whichever group's last step has finished.
// The refinement outer loop (FP64 residual, FP32 inner CG, FP64 update) is
// the one of PD_CG_MIXED: each pass ends after a tenfold drop of the FP32
// residual, and the next pass keeps the search direction (reliable updates).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "pd_reduce.cuh"
#include "pd_stencil.cuh"

namespace pd {
namespace {

constexpr int kMaxBM = 4;               // horizons compiled for batches
constexpr int kMaxPairs = 24;           // count_offsets(2, 4) / 2
constexpr int kChunk = 4096;
constexpr int kBT = 256;
constexpr int kTX = 64, kR = 8, kTY = 32;   // FP32 tile
constexpr int kR64 = 4, kTY64 = 16;         // FP64 tile
constexpr int64_t kGroupNodes = 2 << 20;    // nodes per group: 4 FP32 vectors of 2 components = 64 MB

struct PlateDesc {
    int nx, ny, M, tiles_x, tiles_y, tile_base, chunk_base, nchunks;
    int64_t N, off;                     // nodes, element offset of component 0 in the concatenated vectors
    const uint8_t *cons;
    const float *kd32;
    const double *kd64;
    float c32[3 * (kMaxPairs + 1)];     // pairs in kernel order, then the interior Kd
    double c64[3 * (kMaxPairs + 1)];
};

// Contiguous tile and chunk ranges of one group (device memory; each group's
// captured graph points at its own copy).
struct BatchRange {
    int tile_begin32, tile_end32, tile_begin64, tile_end64, chunk_begin, chunk_end;
};

struct BatchScal {
    double tol2;     // inner stop on r.r (r normalised to |r| = 1 at the start)
    double inv_rn;   // 1 / |r64|
    double rn;       // |r64|
    double pscale;   // inner start: p = r + pscale p_old (0: new direction)
    double beta;     // beta of the iteration the inner loop stopped at
    int done;        // inner loop finished (or plate finished)
    int iters;
};

__device__ __forceinline__ int plate_of_tile(const PlateDesc *d, int np, int t)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].tile_base <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One tile of K p for plate desc (TBT form, horizon M, R rows per thread).  FP32
// sums the differences (u~_{p+o} - u_p) + (u~_{p-o} - u_p) (error relative to
// |K p| for smooth directions, then K p = (Kd_p - Kd_int) p_p - sum), FP64 the
// pairs u~_{p+o} + u~_{p-o} (K p = Kd_p p_p - sum).
template <typename T, int M, int R>
__device__ __forceinline__ T tile_body(const PlateDesc &d, const T *coef, const T *__restrict__ in, T *__restrict__ out,
                                       int x0, int y0, T *s_x, T *s_y)
{
    constexpr int TYt = kGY2 * R, SX = kTX + 2 * M, SY = TYt + 2 * M, WL = R + 2 * M;
    constexpr int NP = count_offsets(2, M) / 2;
    const int nx = d.nx, ny = d.ny;
    const int64_t N = d.N;
    const T *ub = in + d.off;
    T *ob = out + d.off;
    for (int t = threadIdx.x; t < SX * SY; t += kBT) {
        const int r = t / SX, c = t - r * SX;
        const int gx = x0 - M + c, gy = y0 - M + r;
        T vx = T(0), vy = T(0);
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
            const int64_t p = (int64_t)gy * nx + gx;
            vx = ub[p];
            vy = ub[N + p];
        }
        s_x[t] = vx;
        s_y[t] = vy;
    }
    __syncthreads();
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const T *colx = s_x + (ty * R) * SX + tx + M;
    const T *coly = s_y + (ty * R) * SX + tx + M;
    constexpr bool DIFF = sizeof(T) == 4;
    T ax[R], ay[R], ctx[R], cty[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ax[r] = T(0);
        ay[r] = T(0);
        ctx[r] = DIFF ? colx[(r + M) * SX] : T(0);   // the outputs' own values
        cty[r] = DIFF ? coly[(r + M) * SX] : T(0);
    }
    static_for<1, M + 1>([&](auto OX) {
        constexpr int ox = decltype(OX)::value;
        constexpr int My = isqrt_c(M * M - ox * ox);
        T px[WL], py[WL], mx[WL], my[WL];
#pragma unroll
        for (int i = 0; i < WL; ++i) {
            px[i] = colx[i * SX + ox];
            py[i] = coly[i * SX + ox];
            mx[i] = colx[i * SX - ox];
            my[i] = coly[i * SX - ox];
        }
        static_for<-My, My + 1>([&](auto OY) {
            constexpr int oy = decltype(OY)::value;
            constexpr int pi = pair_index2(M, ox, oy);
            const T cxx = coef[3 * pi], cxy = coef[3 * pi + 1], cyy = coef[3 * pi + 2];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T sx = DIFF ? (px[r + M + oy] - ctx[r]) + (mx[r + M - oy] - ctx[r])
                                  : px[r + M + oy] + mx[r + M - oy];
                if constexpr (oy == 0) {
                    ax[r] = dfma(cxx, sx, ax[r]);   // axis pair: c_xy = c_yy = 0 exactly
                } else {
                    const T sy = DIFF ? (py[r + M + oy] - cty[r]) + (my[r + M - oy] - cty[r])
                                      : py[r + M + oy] + my[r + M - oy];
                    ax[r] = dfma(cxx, sx, dfma(cxy, sy, ax[r]));
                    ay[r] = dfma(cxy, sx, dfma(cyy, sy, ay[r]));
                }
            }
        });
    });
    T cx[WL], cy[WL];
#pragma unroll
    for (int i = 0; i < WL; ++i) {
        cx[i] = colx[i * SX];
        cy[i] = coly[i * SX];
    }
    static_for<1, M + 1>([&](auto OY) {
        constexpr int oy = decltype(OY)::value;
        constexpr int pi = pair_index2(M, 0, oy);
        const T cyy = coef[3 * pi + 2];   // axis pair: c_xx = c_xy = 0 exactly
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T sy = DIFF ? (cy[r + M + oy] - cy[r + M]) + (cy[r + M - oy] - cy[r + M])
                              : cy[r + M + oy] + cy[r + M - oy];
            ay[r] = dfma(cyy, sy, ay[r]);
        }
    });
    const T *kd = (sizeof(T) == 4) ? (const T *)d.kd32 : (const T *)d.kd64;
    T dot = T(0);
    const int gx = x0 + tx;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gy = y0 + ty * R + r;
        if (gx < nx && gy < ny) {
            const int64_t p = (int64_t)gy * nx + gx;
            const T upx = cx[r + M], upy = cy[r + M];
            T kxx = coef[3 * NP], kxy = coef[3 * NP + 1], kyy = coef[3 * NP + 2];
            const int a0 = min(gx, M), a1 = min(nx - 1 - gx, M), b0 = min(gy, M), b1 = min(ny - 1 - gy, M);
            if (a0 != M || a1 != M || b0 != M || b1 != M) {
                const int cls = ((a0 * (M + 1) + a1) * (M + 1) + b0) * (M + 1) + b1;
                kxx = kd[3 * cls] - (DIFF ? kxx : T(0));
                kxy = kd[3 * cls + 1] - (DIFF ? kxy : T(0));
                kyy = kd[3 * cls + 2] - (DIFF ? kyy : T(0));
            } else if (DIFF) {   // full horizon: the difference sums are the whole product
                kxx = kxy = kyy = T(0);
            }
            T fx = dfma(kxx, upx, dfma(kxy, upy, -ax[r]));
            T fy = dfma(kxy, upx, dfma(kyy, upy, -ay[r]));
            const uint8_t m = d.cons ? d.cons[p] : 0;
            if (m & 1) fx = T(0);
            if (m & 2) fy = T(0);
            ob[p] = fx;
            ob[N + p] = fy;
            dot = dfma(upx, fx, dfma(upy, fy, dot));
        }
    }
    return dot;
}

// Persistent tile kernel over every plate: out = P K P in (inputs kept projected
// by the solver), partial[t] = in.out over tile t.  Plates with scal.done skip.
template <typename T>
__global__ void __launch_bounds__(kBT)
k_batch_matvec(const PlateDesc *__restrict__ desc, int np, int ntiles, const T *__restrict__ in, T *__restrict__ out,
               double *partial, const BatchScal *__restrict__ scal, const BatchRange *__restrict__ range)
{
    constexpr int R = sizeof(T) == 4 ? kR : kR64;
    constexpr int SXmax = kTX + 2 * kMaxBM, SYmax = kGY2 * R + 2 * kMaxBM;
    __shared__ T s_x[SXmax * SYmax], s_y[SXmax * SYmax];
    __shared__ T coef[3 * (kMaxPairs + 1)];
    __shared__ double red[kBT / 32];
    int t0 = 0, t1 = ntiles;
    if (range) {
        t0 = (sizeof(T) == 4) ? range->tile_begin32 : range->tile_begin64;
        t1 = (sizeof(T) == 4) ? range->tile_end32 : range->tile_end64;
    }
    for (int t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
        const int pl = plate_of_tile(desc, np, t);
        const PlateDesc &d = desc[pl];
        if (scal && scal[pl].done) continue;   // uniform over the CTA
        const int lt = t - d.tile_base;
        const int x0 = (lt % d.tiles_x) * kTX, y0 = (lt / d.tiles_x) * (kGY2 * R);
        for (int i = threadIdx.x; i < 3 * (kMaxPairs + 1); i += kBT)
            coef[i] = (sizeof(T) == 4) ? (T)d.c32[i] : (T)d.c64[i];
        __syncthreads();
        T dot = T(0);
        switch (d.M) {
            case 1: dot = tile_body<T, 1, R>(d, coef, in, out, x0, y0, s_x, s_y); break;
            case 2: dot = tile_body<T, 2, R>(d, coef, in, out, x0, y0, s_x, s_y); break;
            case 3: dot = tile_body<T, 3, R>(d, coef, in, out, x0, y0, s_x, s_y); break;
            default: dot = tile_body<T, 4, R>(d, coef, in, out, x0, y0, s_x, s_y); break;
        }
        const double s = block_sum(dot, red);
        if (threadIdx.x == 0 && partial) partial[t] = s;
        __syncthreads();
    }
}

// Sum of a[0..n) by one warp: lane-strided partial sums, then a butterfly
// (fixed order, so every caller gets the same bits); the total is in all lanes.
__device__ __forceinline__ double warp_sum(const double *__restrict__ a, int n)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += a[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// x += alpha p, r -= alpha q over the chunk; alpha = rr / pq re-summed per plate.
__global__ void __launch_bounds__(kBT)
k_batch_update(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, const BatchRange *__restrict__ range, float *x, float *xlo, float *r,
               const float *__restrict__ p, const float *__restrict__ q, const double *__restrict__ tile_part,
               const double *__restrict__ rr_prev, double *rr_cur, const BatchScal *__restrict__ scal)
{
    __shared__ double red[kBT / 32];
    __shared__ double s_alpha;
    const int c0 = range ? range->chunk_begin : 0, c1 = range ? range->chunk_end : nch;
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const int pl = cplate[c];
        const PlateDesc &d = desc[pl];
        if (scal[pl].done) continue;
        if (threadIdx.x < 32) {
            const double pq = warp_sum(tile_part + d.tile_base, d.tiles_x * d.tiles_y);
            const double rr = warp_sum(rr_prev + d.chunk_base, d.nchunks);
            if (threadIdx.x == 0) s_alpha = (pq != 0.0) ? rr / pq : 0.0;
        }
        __syncthreads();
        const float a = (float)s_alpha;
        const int64_t L = 2 * d.N;
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + L);
        float acc = 0.f;
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) {
            // the increment as a compensated sum x + xlo (two-sum of Knuth): rounding of a
            // plain FP32 sum, amplified by K, would open a gap to the recursive residual
            const float dx = a * p[i], xh = x[i], sum = xh + dx, bp = sum - xh;
            x[i] = sum;
            xlo[i] += (xh - (sum - bp)) + (dx - bp);
            const float ri = r[i] - a * q[i];
            r[i] = ri;
            acc += ri * ri;
        }
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) rr_cur[c] = s;
        __syncthreads();
    }
}

// p = r + beta p; beta = rr_cur / rr_prev; plates below their tolerance are marked done.
__global__ void __launch_bounds__(kBT)
k_batch_pupdate(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, const BatchRange *__restrict__ range, float *p,
                const float *__restrict__ r, const double *__restrict__ rr_prev, const double *__restrict__ rr_cur,
                BatchScal *scal)
{
    __shared__ double s_beta;
    __shared__ int s_stop;
    const int c0 = range ? range->chunk_begin : 0, c1 = range ? range->chunk_end : nch;
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const int pl = cplate[c];
        const PlateDesc &d = desc[pl];
        if (scal[pl].done) continue;
        if (threadIdx.x < 32) {
            const double rn = warp_sum(rr_cur + d.chunk_base, d.nchunks);
            const double ro = warp_sum(rr_prev + d.chunk_base, d.nchunks);
            if (threadIdx.x == 0) {
                s_beta = (ro > 0.0) ? rn / ro : 0.0;
                s_stop = !(rn > scal[pl].tol2);
                if (c == d.chunk_base) scal[pl].iters += 1;
            }
        }
        __syncthreads();
        if (s_stop) {
            // every chunk of the plate reaches the same decision; the flag is read by the next launch
            if (threadIdx.x == 0) {
                scal[pl].done = 1;
                if (c == d.chunk_base) scal[pl].beta = s_beta;   // for the next pass's kept direction
            }
            __syncthreads();
            continue;
        }
        const float beta = (float)s_beta;
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + 2 * d.N);
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) p[i] = r[i] + beta * p[i];
        __syncthreads();
    }
}

// r64 = P(b - Ku), chunk partials of r64.r64
__global__ void __launch_bounds__(kBT)
k_batch_resid(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, const BatchRange *__restrict__ range, double *r64,
              const double *__restrict__ b, const double *__restrict__ Ku, double *part,
              const BatchScal *__restrict__ scal)
{
    __shared__ double red[kBT / 32];
    const int c0 = range ? range->chunk_begin : 0, c1 = range ? range->chunk_end : nch;
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        if (scal && scal[cplate[c]].done) continue;
        const PlateDesc &d = desc[cplate[c]];
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + 2 * d.N);
        double acc = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) {
            const int64_t e = i - d.off;
            const int comp = (int)(e / d.N);
            const int64_t pnode = e - comp * d.N;
            const bool fixed = d.cons && ((d.cons[pnode] >> comp) & 1);
            const double v = fixed ? 0.0 : b[i] - Ku[i];
            r64[i] = v;
            acc += v * v;
        }
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) part[c] = s;
        __syncthreads();
    }
}

// inner start: r32 = r64 / |r64|, p = r32 + pscale p_old, x = 0; chunk partials of r32.r32
// into rr (the "previous" buffer of the first iteration).  pscale = beta_k |r_prev| / |r|
// keeps the search direction across a residual replacement (p_old was scaled by the
// previous pass's |r|), which is CG with reliable updates; 0 starts a new direction.
__global__ void __launch_bounds__(kBT)
k_batch_start(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, const BatchRange *__restrict__ range, float *r32, float *p32,
              float *x32, float *xlo32, const double *__restrict__ r64, double *rr, const BatchScal *__restrict__ scal)
{
    __shared__ double red[kBT / 32];
    const int c0 = range ? range->chunk_begin : 0, c1 = range ? range->chunk_end : nch;
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const int pl = cplate[c];
        if (scal[pl].done) continue;
        const PlateDesc &d = desc[pl];
        const double inv = scal[pl].inv_rn;
        const float ps = (float)scal[pl].pscale;
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + 2 * d.N);
        float acc = 0.f;
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) {
            const float v = (float)(r64[i] * inv);
            r32[i] = v;
            p32[i] = (ps != 0.f) ? v + ps * p32[i] : v;
            x32[i] = 0.f;
            xlo32[i] = 0.f;
            acc += v * v;
        }
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) rr[c] = s;
        __syncthreads();
    }
}

// zero the constrained components of u (the solution satisfies u = 0 on Omega_c)
__global__ void __launch_bounds__(kBT)
k_batch_project(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch,
                const BatchRange *__restrict__ range, double *u)
{
    const int c0 = range ? range->chunk_begin : 0, c1 = range ? range->chunk_end : nch;
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const PlateDesc &d = desc[cplate[c]];
        if (!d.cons) continue;
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + 2 * d.N);
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) {
            const int64_t e = i - d.off;
            const int comp = (int)(e / d.N);
            if ((d.cons[e - comp * d.N] >> comp) & 1) u[i] = 0.0;
        }
    }
}

// u += |r| x on plates that ran an inner solve this pass
__global__ void __launch_bounds__(kBT)
k_batch_correct(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, const BatchRange *__restrict__ range, double *u,
                const float *__restrict__ x32, const float *__restrict__ xlo32, const BatchScal *__restrict__ scal,
                const int *__restrict__ active)
{
    const int c0 = range ? range->chunk_begin : 0, c1 = range ? range->chunk_end : nch;
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const int pl = cplate[c];
        if (!active[pl]) continue;
        const PlateDesc &d = desc[pl];
        const double rn = scal[pl].rn;
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + 2 * d.N);
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) u[i] += rn * ((double)x32[i] + (double)xlo32[i]);
    }
}

}  // namespace
}  // namespace pd

using namespace pd;

struct pd_batch {
    std::vector<pd_grid *> grids;       // in solve order (ascending size)
    std::vector<int> order;             // solve position -> caller's index
    std::vector<std::pair<int, int>> groups;   // [begin, end) solve positions sharing one pass
    int np = 0, ntiles32 = 0, ntiles64 = 0, nch = 0;
    int64_t total = 0;                  // concatenated vector length
    std::vector<int64_t> offs;
    PlateDesc *d_desc32 = nullptr, *d_desc64 = nullptr;
    int *d_cplate = nullptr, *d_active = nullptr;
    BatchScal *d_scal = nullptr;
    BatchRange *d_range = nullptr;      // [groups] device copies of ranges
    std::vector<BatchRange> ranges;     // per group
    void *ws = nullptr;
    double *u64, *b64, *r64, *q64, *part_t, *rrA, *rrB, *part_c;
    float *r32, *p32, *q32, *x32, *xlo32;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> gstream;  // per group: its passes run concurrently with the others
    std::vector<cudaEvent_t> gevent;    // per group: completion of the last work the host waits for
    std::vector<cudaGraphExec_t> graph; // per group: 32 inner iterations
    void *h_pin = nullptr;              // pinned mailbox: BatchScal [np], active [np], part [nch]
    int blocks = 0;
};

extern "C" {

int pd_batch_create(pd_grid *const *grids, int count, pd_batch **out)
{
    if (!out || !grids || count < 1) return fail(PD_ERR_INVALID, "need count >= 1 grids");
    *out = nullptr;
    pd_batch *bt = new pd_batch();
    bt->np = count;
    bt->order.resize(count);
    for (int i = 0; i < count; ++i) bt->order[i] = i;
    for (int i = 0; i < count; ++i)
        if (!grids[i]) return fail(PD_ERR_INVALID, "NULL grid in batch");
    std::stable_sort(bt->order.begin(), bt->order.end(),
                     [&](int a, int b) { return grids[a]->N < grids[b]->N; });
    std::vector<PlateDesc> d32(count), d64(count);
    std::vector<int> cplate;
    int tb32 = 0, tb64 = 0;
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        pd_grid *g = grids[bt->order[i]];
        if (!g || g->dim != 2 || g->M > kMaxBM || g->has_E || g->sc) {
            delete bt;
            return fail(PD_ERR_INVALID, "batch plates must be 2D, horizon M <= 4, without a modulus field or surface correction");
        }
        bt->grids.push_back(g);
        PlateDesc d{};
        d.nx = (int)g->n[0];
        d.ny = (int)g->n[1];
        d.M = g->M;
        d.N = g->N;
        d.off = off;
        d.cons = g->has_cons ? g->d_cons : nullptr;
        d.kd32 = g->d_kd32;
        d.kd64 = g->d_kd64;
        const int M = g->M;
        double tot[3] = {0, 0, 0}, c[6];
        auto put = [&](int ox, int oy) {
            const int pi = pair_index2(M, ox, oy);
            coef_of(g, ox, oy, 0, false, c);
            for (int k = 0; k < 3; ++k) {
                d.c32[3 * pi + k] = (float)c[k];
                d.c64[3 * pi + k] = c[k];
                tot[k] += 2 * c[k];
            }
        };
        for (int ox = 1; ox <= M; ++ox) {
            const int My = isqrt_c(M * M - ox * ox);
            for (int oy = -My; oy <= My; ++oy) put(ox, oy);
        }
        for (int oy = 1; oy <= M; ++oy) put(0, oy);
        const int NP = count_offsets(2, M) / 2;
        for (int k = 0; k < 3; ++k) {
            d.c32[3 * NP + k] = (float)tot[k];
            d.c64[3 * NP + k] = tot[k];
        }
        d.tiles_x = (d.nx + kTX - 1) / kTX;
        d.chunk_base = (int)cplate.size();
        d.nchunks = (int)((2 * d.N + kChunk - 1) / kChunk);
        for (int k = 0; k < d.nchunks; ++k) cplate.push_back(i);
        PlateDesc e = d;
        d.tiles_y = (d.ny + kTY - 1) / kTY;
        d.tile_base = tb32;
        tb32 += d.tiles_x * d.tiles_y;
        e.tiles_y = (e.ny + kTY64 - 1) / kTY64;
        e.tile_base = tb64;
        tb64 += e.tiles_x * e.tiles_y;
        d32[i] = d;
        d64[i] = e;
        bt->offs.push_back(off);
        off += 2 * d.N;
    }
    bt->total = off;
    // groups of consecutive (similar-size) plates whose FP32 working set stays in L2
    {
        int64_t acc = 0;
        int begin = 0;
        for (int i = 0; i < count; ++i) {
            const int64_t n = bt->grids[i]->N;
            if (i > begin && acc + n > kGroupNodes) {
                bt->groups.push_back({begin, i});
                begin = i;
                acc = 0;
            }
            acc += n;
        }
        bt->groups.push_back({begin, count});
        for (const auto &gr : bt->groups) {
            const PlateDesc &f32 = d32[gr.first], &l32 = d32[gr.second - 1];
            const PlateDesc &f64 = d64[gr.first], &l64 = d64[gr.second - 1];
            BatchRange r;
            r.tile_begin32 = f32.tile_base;
            r.tile_end32 = l32.tile_base + l32.tiles_x * l32.tiles_y;
            r.tile_begin64 = f64.tile_base;
            r.tile_end64 = l64.tile_base + l64.tiles_x * l64.tiles_y;
            r.chunk_begin = f32.chunk_base;
            r.chunk_end = l32.chunk_base + l32.nchunks;
            bt->ranges.push_back(r);
        }
    }
    bt->ntiles32 = tb32;
    bt->ntiles64 = tb64;
    bt->nch = (int)cplate.size();
    auto bail = [&](int code, const char *msg) {
        pd_batch_destroy(bt);
        return fail(code, msg);
    };
    if (cudaMalloc(&bt->d_desc32, sizeof(PlateDesc) * count) != cudaSuccess ||
        cudaMalloc(&bt->d_desc64, sizeof(PlateDesc) * count) != cudaSuccess ||
        cudaMalloc(&bt->d_cplate, sizeof(int) * bt->nch) != cudaSuccess ||
        cudaMalloc(&bt->d_active, sizeof(int) * count) != cudaSuccess ||
        cudaMalloc(&bt->d_scal, sizeof(BatchScal) * count) != cudaSuccess ||
        cudaMalloc(&bt->d_range, sizeof(BatchRange) * bt->groups.size()) != cudaSuccess)
        return bail(PD_ERR_OOM, "batch descriptors");
    cudaMemcpy(bt->d_range, bt->ranges.data(), sizeof(BatchRange) * bt->groups.size(), cudaMemcpyHostToDevice);
    if (cudaMallocHost(&bt->h_pin, (sizeof(BatchScal) + sizeof(int)) * count + sizeof(double) * bt->nch + 64) !=
        cudaSuccess)
        return bail(PD_ERR_OOM, "batch mailbox");
    for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return bail(PD_ERR_CUDA, "group stream");
        bt->gstream.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return bail(PD_ERR_CUDA, "group event");
        bt->gevent.push_back(ev);
        bt->graph.push_back(nullptr);
    }
    cudaMemcpy(bt->d_desc32, d32.data(), sizeof(PlateDesc) * count, cudaMemcpyHostToDevice);
    cudaMemcpy(bt->d_desc64, d64.data(), sizeof(PlateDesc) * count, cudaMemcpyHostToDevice);
    cudaMemcpy(bt->d_cplate, cplate.data(), sizeof(int) * bt->nch, cudaMemcpyHostToDevice);
    const int64_t L = bt->total;
    const int64_t nt = std::max(bt->ntiles32, bt->ntiles64);
    const size_t need = sizeof(double) * (4 * (size_t)L + (size_t)nt + 3 * (size_t)bt->nch) +
                        sizeof(float) * 5 * (size_t)L + 17 * 256;
    if (cudaMalloc(&bt->ws, need) != cudaSuccess) return bail(PD_ERR_OOM, "batch workspace");
    char *c = (char *)bt->ws;
    auto take = [&](size_t n) { char *q = c; c += (n + 255) & ~(size_t)255; return q; };
    bt->u64 = (double *)take(sizeof(double) * L);
    bt->b64 = (double *)take(sizeof(double) * L);
    bt->r64 = (double *)take(sizeof(double) * L);
    bt->q64 = (double *)take(sizeof(double) * L);
    bt->part_t = (double *)take(sizeof(double) * nt);
    bt->rrA = (double *)take(sizeof(double) * bt->nch);
    bt->rrB = (double *)take(sizeof(double) * bt->nch);
    bt->part_c = (double *)take(sizeof(double) * bt->nch);
    bt->r32 = (float *)take(sizeof(float) * L);
    bt->p32 = (float *)take(sizeof(float) * L);
    bt->q32 = (float *)take(sizeof(float) * L);
    bt->x32 = (float *)take(sizeof(float) * L);
    bt->xlo32 = (float *)take(sizeof(float) * L);
    if (cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(PD_ERR_CUDA, "capture stream");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    bt->blocks = std::max(1, sms) * 4;
    *out = bt;
    return PD_OK;
}

int pd_batch_destroy(pd_batch *bt)
{
    if (!bt) return PD_OK;
    for (auto gr : bt->graph)
        if (gr) cudaGraphExecDestroy(gr);
    for (auto st : bt->gstream) cudaStreamDestroy(st);
    for (auto ev : bt->gevent) cudaEventDestroy(ev);
    if (bt->h_pin) cudaFreeHost(bt->h_pin);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    cudaFree(bt->d_desc32);
    cudaFree(bt->d_desc64);
    cudaFree(bt->d_cplate);
    cudaFree(bt->d_active);
    cudaFree(bt->d_scal);
    cudaFree(bt->d_range);
    cudaFree(bt->ws);
    delete bt;
    return PD_OK;
}

}  // extern "C"

namespace {

// Two inner iterations (even count keeps the parity of the r.r buffers aligned).
int batch_two_iterations(pd_batch *bt, const BatchRange *rg, cudaStream_t s)
{
    for (int k = 0; k < 2; ++k) {
        double *prev = (k == 0) ? bt->rrB : bt->rrA;
        double *cur = (k == 0) ? bt->rrA : bt->rrB;
        k_batch_matvec<float><<<bt->blocks, kBT, 0, s>>>(bt->d_desc32, bt->np, bt->ntiles32, bt->p32, bt->q32,
                                                         bt->part_t, bt->d_scal, rg);
        k_batch_update<<<bt->blocks, kBT, 0, s>>>(bt->d_desc32, bt->d_cplate, bt->nch, rg, bt->x32, bt->xlo32, bt->r32,
                                                  bt->p32, bt->q32, bt->part_t, prev, cur, bt->d_scal);
        k_batch_pupdate<<<bt->blocks, kBT, 0, s>>>(bt->d_desc32, bt->d_cplate, bt->nch, rg, bt->p32, bt->r32, prev, cur,
                                                   bt->d_scal);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace

extern "C" int pd_batch_cg_solve(pd_batch *bt, const double *const *b, double *const *u, double rtol, int max_iter,
                                 pd_cg_stats *stats, void *stream)
{
    if (!bt || !b || !u) return fail(PD_ERR_INVALID, "NULL argument");
    if (!(rtol > 0) || max_iter < 2) return fail(PD_ERR_INVALID, "rtol > 0 and max_iter >= 2 required");
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    const int np = bt->np;
    for (int i = 0; i < np; ++i) {
        const int ci = bt->order[i];
        if (!b[ci] || !u[ci]) return fail(PD_ERR_INVALID, "NULL plate vector");
        const size_t bytes = sizeof(double) * 2 * (size_t)bt->grids[i]->N;
        PD_CUDA(cudaMemcpyAsync(bt->b64 + bt->offs[i], b[ci], bytes, cudaMemcpyDeviceToDevice, s));
        PD_CUDA(cudaMemcpyAsync(bt->u64 + bt->offs[i], u[ci], bytes, cudaMemcpyDeviceToDevice, s));
    }
    k_batch_project<<<bt->blocks, kBT, 0, s>>>(bt->d_desc64, bt->d_cplate, bt->nch, nullptr, bt->u64);
    std::vector<double> part(bt->nch), bb(np, 0.0), rr(np, 0.0);
    std::vector<BatchScal> sc(np);
    std::vector<int> active(np, 0), outer(np, 0), iters(np, 0), fmv(np, 0), cpl(bt->nch);
    {
        int k = 0;
        for (int i = 0; i < np; ++i) {
            const int nc = (int)((2 * bt->grids[i]->N + kChunk - 1) / kChunk);
            for (int j = 0; j < nc; ++j) cpl[k++] = i;
        }
    }
    // |P b|^2 per plate (residual of u = 0)
    PD_CUDA(cudaMemsetAsync(bt->q64, 0, sizeof(double) * bt->total, s));
    k_batch_resid<<<bt->blocks, kBT, 0, s>>>(bt->d_desc64, bt->d_cplate, bt->nch, nullptr, bt->r64, bt->b64,
                                            bt->q64, bt->part_c, nullptr);
    PD_CUDA(cudaMemcpyAsync(part.data(), bt->part_c, sizeof(double) * bt->nch, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < bt->nch; ++c) bb[cpl[c]] += part[c];
    // Groups are independent (disjoint plates, tiles and chunks), so each advances
    // on its own stream as a small state machine and the host serves whichever
    // group's last step has finished.  Each group replays its own graph of 32
    // inner iterations (fixed pointers, including its device range).
    constexpr int kPairsPerGraph = 16;   // 32 iterations per replay
    constexpr double kRU = 0.1;          // a pass ends after a tenfold drop of the FP32 residual (or at the target)
    const int ng = (int)bt->groups.size();
    for (int gi = 0; gi < ng; ++gi) {
        if (bt->graph[gi]) continue;
        cudaGraph_t gr = nullptr;
        bool ok = cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        for (int k = 0; k < kPairsPerGraph && ok; ++k) ok = batch_two_iterations(bt, bt->d_range + gi, bt->cap) == PD_OK;
        ok = (cudaStreamEndCapture(bt->cap, &gr) == cudaSuccess) && ok;
        if (!ok || cudaGraphInstantiate(&bt->graph[gi], gr, 0) != cudaSuccess) bt->graph[gi] = nullptr;
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
    }
    BatchScal *h_sc = (BatchScal *)bt->h_pin;                 // [np]
    int *h_active = (int *)(h_sc + np);                        // [np]
    double *h_part = (double *)(((uintptr_t)(h_active + np) + 15) & ~(uintptr_t)15);   // [nch]
    std::vector<double> beta_last(np, 0.0), rn_prev(np, 0.0);
    std::vector<int> ran(np, 0);   // the plate ran an inner loop in its group's last pass
    enum Phase { kResid, kInner, kDone };
    struct Run {
        int first, last, cb, ce;   // plates [first, last), chunks [cb, ce)
        Phase phase = kResid;
        int pass = 0, group_iters = 0, issued = 0;
        bool converged = false;
    };
    std::vector<Run> run(ng);
    cudaEvent_t fork = nullptr;
    PD_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    PD_CUDA(cudaEventRecord(fork, s));   // inputs staged on the caller's stream
    // FP64 residual of a group's plates (its other work is done), its chunk sums to the host
    auto issue_resid = [&](int gi) -> int {
        Run &R = run[gi];
        cudaStream_t st = bt->gstream[gi];
        for (int i = R.first; i < R.last; ++i) h_sc[i] = BatchScal{};
        PD_CUDA(cudaMemcpyAsync(bt->d_scal + R.first, h_sc + R.first, sizeof(BatchScal) * (R.last - R.first),
                                cudaMemcpyHostToDevice, st));
        k_batch_matvec<double><<<bt->blocks, kBT, 0, st>>>(bt->d_desc64, np, bt->ntiles64, bt->u64, bt->q64, nullptr,
                                                          bt->d_scal, bt->d_range + gi);
        k_batch_resid<<<bt->blocks, kBT, 0, st>>>(bt->d_desc64, bt->d_cplate, bt->nch, bt->d_range + gi, bt->r64,
                                                  bt->b64, bt->q64, bt->part_c, bt->d_scal);
        PD_CUDA(cudaGetLastError());
        PD_CUDA(cudaMemcpyAsync(h_part + R.cb, bt->part_c + R.cb, sizeof(double) * (R.ce - R.cb),
                                cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaEventRecord(bt->gevent[gi], st));
        R.phase = kResid;
        return PD_OK;
    };
    auto issue_inner = [&](int gi) -> int {
        cudaStream_t st = bt->gstream[gi];
        if (bt->graph[gi]) {
            PD_CUDA(cudaGraphLaunch(bt->graph[gi], st));
        } else {
            for (int k = 0; k < kPairsPerGraph; ++k) {
                int rc = batch_two_iterations(bt, bt->d_range + gi, st);
                if (rc) return rc;
            }
        }
        run[gi].issued += 2 * kPairsPerGraph;
        PD_CUDA(cudaMemcpyAsync(h_sc + run[gi].first, bt->d_scal + run[gi].first,
                                sizeof(BatchScal) * (run[gi].last - run[gi].first), cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaEventRecord(bt->gevent[gi], st));
        run[gi].phase = kInner;
        return PD_OK;
    };
    for (int gi = 0; gi < ng; ++gi) {
        Run &R = run[gi];
        R.first = bt->groups[gi].first;
        R.last = bt->groups[gi].second;
        R.cb = bt->ranges[gi].chunk_begin;
        R.ce = bt->ranges[gi].chunk_end;
        PD_CUDA(cudaStreamWaitEvent(bt->gstream[gi], fork, 0));
        int rc = issue_resid(gi);
        if (rc) return rc;
    }
    int status = PD_OK;
    for (int left = ng; left > 0;) {
        bool progressed = false;
        for (int gi = 0; gi < ng; ++gi) {
            Run &R = run[gi];
            if (R.phase == kDone) continue;
            const cudaError_t q = cudaEventQuery(bt->gevent[gi]);
            if (q == cudaErrorNotReady) continue;
            PD_CUDA(q);
            progressed = true;
            cudaStream_t st = bt->gstream[gi];
            if (R.phase == kResid) {
                int n_active = 0;
                for (int i = R.first; i < R.last; ++i) rr[i] = 0.0;
                for (int c = R.cb; c < R.ce; ++c) rr[cpl[c]] += h_part[c];
                for (int i = R.first; i < R.last; ++i) {
                    const bool kept = ran[i] && std::isfinite(beta_last[i]) && rn_prev[i] > 0.0;
                    active[i] = 0;
                    h_sc[i] = BatchScal{};
                    h_sc[i].done = 1;
                    ++fmv[i];
                    const double bn = bb[i] > 0 ? std::sqrt(bb[i]) : 1.0;
                    const double rn = std::sqrt(rr[i]);
                    ran[i] = 0;
                    if (rn / bn <= rtol) continue;
                    active[i] = 1;
                    ran[i] = 1;
                    ++outer[i];
                    ++n_active;
                    const double need = 0.3 * rtol * bn / (rn > 0 ? rn : 1.0);
                    const double tau = std::min(0.5, std::max(kRU, need));
                    h_sc[i].tol2 = tau * tau;
                    h_sc[i].rn = rn;
                    h_sc[i].inv_rn = rn > 0 ? 1.0 / rn : 0.0;
                    h_sc[i].pscale = (kept && rn > 0) ? beta_last[i] * rn_prev[i] / rn : 0.0;
                    h_sc[i].done = 0;
                    rn_prev[i] = rn;
                }
                if (n_active == 0 || R.group_iters >= max_iter || R.pass >= 60) {
                    R.converged = (n_active == 0);
                    R.phase = kDone;
                    --left;
                    continue;
                }
                for (int i = R.first; i < R.last; ++i) h_active[i] = active[i];
                PD_CUDA(cudaMemcpyAsync(bt->d_scal + R.first, h_sc + R.first, sizeof(BatchScal) * (R.last - R.first),
                                        cudaMemcpyHostToDevice, st));
                PD_CUDA(cudaMemcpyAsync(bt->d_active + R.first, h_active + R.first, sizeof(int) * (R.last - R.first),
                                        cudaMemcpyHostToDevice, st));
                k_batch_start<<<bt->blocks, kBT, 0, st>>>(bt->d_desc32, bt->d_cplate, bt->nch, bt->d_range + gi,
                                                          bt->r32, bt->p32, bt->x32, bt->xlo32, bt->r64, bt->rrB,
                                                          bt->d_scal);
                PD_CUDA(cudaGetLastError());
                R.issued = 0;
                int rc = issue_inner(gi);
                if (rc) return rc;
            } else {   // kInner: one replay finished
                bool all = true;
                for (int i = R.first; i < R.last; ++i) all = all && h_sc[i].done;
                if (!all && R.group_iters + R.issued < max_iter) {
                    int rc = issue_inner(gi);
                    if (rc) return rc;
                    continue;
                }
                int mx = 0;
                for (int i = R.first; i < R.last; ++i) {
                    iters[i] += h_sc[i].iters;
                    mx = std::max(mx, h_sc[i].iters);
                    beta_last[i] = h_sc[i].beta;
                }
                R.group_iters += mx;
                ++R.pass;
                k_batch_correct<<<bt->blocks, kBT, 0, st>>>(bt->d_desc32, bt->d_cplate, bt->nch, bt->d_range + gi,
                                                            bt->u64, bt->x32, bt->xlo32, bt->d_scal, bt->d_active);
                PD_CUDA(cudaGetLastError());
                int rc = issue_resid(gi);
                if (rc) return rc;
            }
        }
        if (!progressed) std::this_thread::yield();
    }
    for (int gi = 0; gi < ng; ++gi) {   // join: the caller's stream waits for every group
        if (!run[gi].converged) status = PD_ERR_NOT_CONVERGED;
        PD_CUDA(cudaEventRecord(bt->gevent[gi], bt->gstream[gi]));
        PD_CUDA(cudaStreamWaitEvent(s, bt->gevent[gi], 0));
    }
    cudaEventDestroy(fork);
    for (int i = 0; i < np; ++i) {
        const size_t bytes = sizeof(double) * 2 * (size_t)bt->grids[i]->N;
        PD_CUDA(cudaMemcpyAsync(u[bt->order[i]], bt->u64 + bt->offs[i], bytes, cudaMemcpyDeviceToDevice, s));
    }
    PD_CUDA(cudaStreamSynchronize(s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) {
        for (int i = 0; i < np; ++i) {
            const double bn = bb[i] > 0 ? std::sqrt(bb[i]) : 1.0;
            pd_cg_stats &st = stats[bt->order[i]];
            st.iterations = iters[i];
            st.outer = outer[i];
            st.f64_matvecs = fmv[i];
            st.rel_residual = std::sqrt(rr[i]) / bn;
            st.seconds = secs;
        }
    }
    if (status != PD_OK) return fail(PD_ERR_NOT_CONVERGED, "batched CG reached its iteration cap");
    return PD_OK;
}

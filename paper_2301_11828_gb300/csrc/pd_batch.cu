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
// The refinement outer loop (FP64 residual, FP32 inner CG, FP64 update) is
// the one of PD_CG_MIXED.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
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

struct PlateDesc {
    int nx, ny, M, tiles_x, tiles_y, tile_base, chunk_base, nchunks;
    int64_t N, off;                     // nodes, element offset of component 0 in the concatenated vectors
    const uint8_t *cons;
    const float *kd32;
    const double *kd64;
    float c32[3 * (kMaxPairs + 1)];     // pairs in kernel order, then the interior Kd
    double c64[3 * (kMaxPairs + 1)];
};

struct BatchScal {
    double tol2;     // inner stop on r.r (r normalised to |r| = 1 at the start)
    double inv_rn;   // 1 / |r64|
    double rn;       // |r64|
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

// One tile of K p for plate desc (TBT pair form, horizon M, R rows per thread).
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
    T ax[R], ay[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { ax[r] = T(0); ay[r] = T(0); }
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
                const T sx = px[r + M + oy] + mx[r + M - oy];
                const T sy = py[r + M + oy] + my[r + M - oy];
                ax[r] = dfma(cxx, sx, dfma(cxy, sy, ax[r]));
                ay[r] = dfma(cxy, sx, dfma(cyy, sy, ay[r]));
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
        const T cxx = coef[3 * pi], cxy = coef[3 * pi + 1], cyy = coef[3 * pi + 2];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T sx = cx[r + M + oy] + cx[r + M - oy];
            const T sy = cy[r + M + oy] + cy[r + M - oy];
            ax[r] = dfma(cxx, sx, dfma(cxy, sy, ax[r]));
            ay[r] = dfma(cxy, sx, dfma(cyy, sy, ay[r]));
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
                kxx = kd[3 * cls];
                kxy = kd[3 * cls + 1];
                kyy = kd[3 * cls + 2];
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
               double *partial, const BatchScal *__restrict__ scal)
{
    constexpr int R = sizeof(T) == 4 ? kR : kR64;
    constexpr int SXmax = kTX + 2 * kMaxBM, SYmax = kGY2 * R + 2 * kMaxBM;
    __shared__ T s_x[SXmax * SYmax], s_y[SXmax * SYmax];
    __shared__ T coef[3 * (kMaxPairs + 1)];
    __shared__ double red[kBT / 32];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
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
        const double s = block_sum((double)dot, red);
        if (threadIdx.x == 0 && partial) partial[t] = s;
        __syncthreads();
    }
}

// x += alpha p, r -= alpha q over the chunk; alpha = rr / pq re-summed per plate.
__global__ void __launch_bounds__(kBT)
k_batch_update(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, float *x, float *r,
               const float *__restrict__ p, const float *__restrict__ q, const double *__restrict__ tile_part,
               const double *__restrict__ rr_prev, double *rr_cur, const BatchScal *__restrict__ scal)
{
    __shared__ double red[kBT / 32];
    __shared__ double s_alpha;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int pl = cplate[c];
        const PlateDesc &d = desc[pl];
        if (scal[pl].done) continue;
        if (threadIdx.x == 0) {
            double pq = 0.0, rr = 0.0;
            for (int t = 0; t < d.tiles_x * d.tiles_y; ++t) pq += tile_part[d.tile_base + t];
            for (int k = 0; k < d.nchunks; ++k) rr += rr_prev[d.chunk_base + k];
            s_alpha = (pq != 0.0) ? rr / pq : 0.0;
        }
        __syncthreads();
        const float a = (float)s_alpha;
        const int64_t L = 2 * d.N;
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + L);
        float acc = 0.f;
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) {
            x[i] += a * p[i];
            const float ri = r[i] - a * q[i];
            r[i] = ri;
            acc += ri * ri;
        }
        const double s = block_sum((double)acc, red);
        if (threadIdx.x == 0) rr_cur[c] = s;
        __syncthreads();
    }
}

// p = r + beta p; beta = rr_cur / rr_prev; plates below their tolerance are marked done.
__global__ void __launch_bounds__(kBT)
k_batch_pupdate(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, float *p,
                const float *__restrict__ r, const double *__restrict__ rr_prev, const double *__restrict__ rr_cur,
                BatchScal *scal)
{
    __shared__ double s_beta;
    __shared__ int s_stop;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int pl = cplate[c];
        const PlateDesc &d = desc[pl];
        if (scal[pl].done) continue;
        if (threadIdx.x == 0) {
            double rn = 0.0, ro = 0.0;
            for (int k = 0; k < d.nchunks; ++k) {
                rn += rr_cur[d.chunk_base + k];
                ro += rr_prev[d.chunk_base + k];
            }
            s_beta = (ro > 0.0) ? rn / ro : 0.0;
            s_stop = !(rn > scal[pl].tol2);
            if (c == d.chunk_base) {
                scal[pl].iters += 1;
            }
        }
        __syncthreads();
        if (s_stop) {
            // every chunk of the plate reaches the same decision; the flag is read by the next launch
            if (threadIdx.x == 0) scal[pl].done = 1;
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
k_batch_resid(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, double *r64,
              const double *__restrict__ b, const double *__restrict__ Ku, double *part)
{
    __shared__ double red[kBT / 32];
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
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

// inner start: r32 = r64 / |r64|, p = r32, x = 0; chunk partials of r32.r32 into rr (the
// "previous" buffer of the first iteration)
__global__ void __launch_bounds__(kBT)
k_batch_start(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, float *r32, float *p32,
              float *x32, const double *__restrict__ r64, double *rr, const BatchScal *__restrict__ scal)
{
    __shared__ double red[kBT / 32];
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int pl = cplate[c];
        const PlateDesc &d = desc[pl];
        const double inv = scal[pl].inv_rn;
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + 2 * d.N);
        float acc = 0.f;
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) {
            const float v = (float)(r64[i] * inv);
            r32[i] = v;
            p32[i] = v;
            x32[i] = 0.f;
            acc += v * v;
        }
        const double s = block_sum((double)acc, red);
        if (threadIdx.x == 0) rr[c] = s;
        __syncthreads();
    }
}

// zero the constrained components of u (the solution satisfies u = 0 on Omega_c)
__global__ void __launch_bounds__(kBT)
k_batch_project(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, double *u)
{
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
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
k_batch_correct(const PlateDesc *__restrict__ desc, const int *__restrict__ cplate, int nch, double *u,
                const float *__restrict__ x32, const BatchScal *__restrict__ scal, const int *__restrict__ active)
{
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int pl = cplate[c];
        if (!active[pl]) continue;
        const PlateDesc &d = desc[pl];
        const double rn = scal[pl].rn;
        const int64_t lo = d.off + (int64_t)(c - d.chunk_base) * kChunk;
        const int64_t hi = min(lo + (int64_t)kChunk, d.off + 2 * d.N);
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) u[i] += rn * (double)x32[i];
    }
}

}  // namespace
}  // namespace pd

using namespace pd;

struct pd_batch {
    std::vector<pd_grid *> grids;
    int np = 0, ntiles32 = 0, ntiles64 = 0, nch = 0;
    int64_t total = 0;                  // concatenated vector length
    std::vector<int64_t> offs;
    PlateDesc *d_desc32 = nullptr, *d_desc64 = nullptr;
    int *d_cplate = nullptr, *d_active = nullptr;
    BatchScal *d_scal = nullptr;
    void *ws = nullptr;
    double *u64, *b64, *r64, *q64, *part_t, *rrA, *rrB, *part_c;
    float *r32, *p32, *q32, *x32;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    int blocks = 0;
};

extern "C" {

int pd_batch_create(pd_grid *const *grids, int count, pd_batch **out)
{
    if (!out || !grids || count < 1) return fail(PD_ERR_INVALID, "need count >= 1 grids");
    *out = nullptr;
    pd_batch *bt = new pd_batch();
    bt->np = count;
    std::vector<PlateDesc> d32(count), d64(count);
    std::vector<int> cplate;
    int tb32 = 0, tb64 = 0;
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        pd_grid *g = grids[i];
        if (!g || g->dim != 2 || g->M > kMaxBM || g->has_E) {
            delete bt;
            return fail(PD_ERR_INVALID, "batch plates must be 2D, horizon M <= 4, without a modulus field");
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
        cudaMalloc(&bt->d_scal, sizeof(BatchScal) * count) != cudaSuccess)
        return bail(PD_ERR_OOM, "batch descriptors");
    cudaMemcpy(bt->d_desc32, d32.data(), sizeof(PlateDesc) * count, cudaMemcpyHostToDevice);
    cudaMemcpy(bt->d_desc64, d64.data(), sizeof(PlateDesc) * count, cudaMemcpyHostToDevice);
    cudaMemcpy(bt->d_cplate, cplate.data(), sizeof(int) * bt->nch, cudaMemcpyHostToDevice);
    const int64_t L = bt->total;
    const int64_t nt = std::max(bt->ntiles32, bt->ntiles64);
    const size_t need = sizeof(double) * (4 * (size_t)L + (size_t)nt + 3 * (size_t)bt->nch) +
                        sizeof(float) * 4 * (size_t)L + 16 * 256;
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
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    cudaFree(bt->d_desc32);
    cudaFree(bt->d_desc64);
    cudaFree(bt->d_cplate);
    cudaFree(bt->d_active);
    cudaFree(bt->d_scal);
    cudaFree(bt->ws);
    delete bt;
    return PD_OK;
}

}  // extern "C"

namespace {

// Two inner iterations (even count keeps the parity of the r.r buffers aligned).
int batch_two_iterations(pd_batch *bt, cudaStream_t s)
{
    for (int k = 0; k < 2; ++k) {
        double *prev = (k == 0) ? bt->rrB : bt->rrA;
        double *cur = (k == 0) ? bt->rrA : bt->rrB;
        k_batch_matvec<float><<<bt->blocks, kBT, 0, s>>>(bt->d_desc32, bt->np, bt->ntiles32, bt->p32, bt->q32,
                                                         bt->part_t, bt->d_scal);
        k_batch_update<<<bt->blocks, kBT, 0, s>>>(bt->d_desc32, bt->d_cplate, bt->nch, bt->x32, bt->r32, bt->p32,
                                                  bt->q32, bt->part_t, prev, cur, bt->d_scal);
        k_batch_pupdate<<<bt->blocks, kBT, 0, s>>>(bt->d_desc32, bt->d_cplate, bt->nch, bt->p32, bt->r32, prev, cur,
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
        if (!b[i] || !u[i]) return fail(PD_ERR_INVALID, "NULL plate vector");
        const size_t bytes = sizeof(double) * 2 * (size_t)bt->grids[i]->N;
        PD_CUDA(cudaMemcpyAsync(bt->b64 + bt->offs[i], b[i], bytes, cudaMemcpyDeviceToDevice, s));
        PD_CUDA(cudaMemcpyAsync(bt->u64 + bt->offs[i], u[i], bytes, cudaMemcpyDeviceToDevice, s));
    }
    k_batch_project<<<bt->blocks, kBT, 0, s>>>(bt->d_desc64, bt->d_cplate, bt->nch, bt->u64);
    std::vector<double> part(bt->nch), bb(np, 0.0), rr(np, 0.0);
    std::vector<BatchScal> sc(np);
    std::vector<int> active(np, 0), finished(np, 0), outer(np, 0), iters(np, 0);
    // |P b|^2 per plate (residual of u = 0)
    PD_CUDA(cudaMemsetAsync(bt->q64, 0, sizeof(double) * bt->total, s));
    k_batch_resid<<<bt->blocks, kBT, 0, s>>>(bt->d_desc64, bt->d_cplate, bt->nch, bt->r64, bt->b64, bt->q64,
                                            bt->part_c);
    PD_CUDA(cudaMemcpyAsync(part.data(), bt->part_c, sizeof(double) * bt->nch, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    std::vector<int> cpl(bt->nch);
    {
        int k = 0;
        for (int i = 0; i < np; ++i) {
            const int nc = (int)((2 * bt->grids[i]->N + kChunk - 1) / kChunk);
            for (int j = 0; j < nc; ++j) cpl[k++] = i;
        }
    }
    for (int c = 0; c < bt->nch; ++c) bb[cpl[c]] += part[c];
    int total_iters = 0, passes = 0, status = PD_ERR_NOT_CONVERGED;
    double worst = 0.0;
    for (passes = 0; passes < 60; ++passes) {
        // FP64 residual of every plate
        k_batch_matvec<double><<<bt->blocks, kBT, 0, s>>>(bt->d_desc64, np, bt->ntiles64, bt->u64, bt->q64, nullptr,
                                                          nullptr);
        k_batch_resid<<<bt->blocks, kBT, 0, s>>>(bt->d_desc64, bt->d_cplate, bt->nch, bt->r64, bt->b64, bt->q64,
                                                bt->part_c);
        PD_CUDA(cudaMemcpyAsync(part.data(), bt->part_c, sizeof(double) * bt->nch, cudaMemcpyDeviceToHost, s));
        PD_CUDA(cudaStreamSynchronize(s));
        std::fill(rr.begin(), rr.end(), 0.0);
        for (int c = 0; c < bt->nch; ++c) rr[cpl[c]] += part[c];
        int n_active = 0;
        worst = 0.0;
        for (int i = 0; i < np; ++i) {
            const double bn = bb[i] > 0 ? std::sqrt(bb[i]) : 1.0;
            const double rel = std::sqrt(rr[i]) / bn;
            worst = std::max(worst, rel);
            finished[i] = (rel <= rtol) ? 1 : 0;
            active[i] = !finished[i];
            const double rn = std::sqrt(rr[i]);
            const double need = 0.3 * rtol * bn / (rn > 0 ? rn : 1.0);
            const double tau = std::min(0.5, std::max(need, 2e-5));
            sc[i].tol2 = tau * tau;
            sc[i].rn = rn;
            sc[i].inv_rn = rn > 0 ? 1.0 / rn : 0.0;
            sc[i].done = finished[i];
            sc[i].iters = 0;
            if (active[i]) {
                ++n_active;
                ++outer[i];
            }
        }
        if (n_active == 0) {
            status = PD_OK;
            break;
        }
        if (total_iters >= max_iter) break;
        PD_CUDA(cudaMemcpyAsync(bt->d_scal, sc.data(), sizeof(BatchScal) * np, cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(bt->d_active, active.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
        k_batch_start<<<bt->blocks, kBT, 0, s>>>(bt->d_desc32, bt->d_cplate, bt->nch, bt->r32, bt->p32, bt->x32,
                                                bt->r64, bt->rrB, bt->d_scal);
        PD_CUDA(cudaGetLastError());
        // inner loop: chunks of iterations as one graph
        constexpr int kPairsPerGraph = 16;   // 32 iterations per replay
        if (!bt->graph) {
            cudaGraph_t gr = nullptr;
            bool ok = cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            for (int k = 0; k < kPairsPerGraph && ok; ++k) ok = batch_two_iterations(bt, bt->cap) == PD_OK;
            ok = (cudaStreamEndCapture(bt->cap, &gr) == cudaSuccess) && ok;
            if (!ok || cudaGraphInstantiate(&bt->graph, gr, 0) != cudaSuccess) bt->graph = nullptr;
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
        }
        int issued = 0;
        while (total_iters + issued < max_iter) {
            if (bt->graph) {
                PD_CUDA(cudaGraphLaunch(bt->graph, s));
            } else {
                for (int k = 0; k < kPairsPerGraph; ++k) {
                    int rc = batch_two_iterations(bt, s);
                    if (rc) return rc;
                }
            }
            issued += 2 * kPairsPerGraph;
            PD_CUDA(cudaMemcpyAsync(sc.data(), bt->d_scal, sizeof(BatchScal) * np, cudaMemcpyDeviceToHost, s));
            PD_CUDA(cudaStreamSynchronize(s));
            bool all = true;
            for (int i = 0; i < np; ++i) all = all && sc[i].done;
            if (all) break;
        }
        int mx = 0;
        for (int i = 0; i < np; ++i) {
            iters[i] += sc[i].iters;
            mx = std::max(mx, sc[i].iters);
        }
        total_iters += mx;
        k_batch_correct<<<bt->blocks, kBT, 0, s>>>(bt->d_desc32, bt->d_cplate, bt->nch, bt->u64, bt->x32, bt->d_scal,
                                                  bt->d_active);
        PD_CUDA(cudaGetLastError());
    }
    for (int i = 0; i < np; ++i) {
        const size_t bytes = sizeof(double) * 2 * (size_t)bt->grids[i]->N;
        PD_CUDA(cudaMemcpyAsync(u[i], bt->u64 + bt->offs[i], bytes, cudaMemcpyDeviceToDevice, s));
    }
    PD_CUDA(cudaStreamSynchronize(s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) {
        for (int i = 0; i < np; ++i) {
            const double bn = bb[i] > 0 ? std::sqrt(bb[i]) : 1.0;
            stats[i].iterations = iters[i];
            stats[i].outer = outer[i];
            stats[i].f64_matvecs = passes + 1;
            stats[i].rel_residual = std::sqrt(rr[i]) / bn;
            stats[i].seconds = secs;
        }
    }
    if (status != PD_OK) return fail(PD_ERR_NOT_CONVERGED, "batched CG reached its iteration cap");
    return PD_OK;
}

// pd_cg_persist.cu -- the FP32 inner loop of the mixed CG as one persistent,
// cooperatively launched kernel (2D grids on the TMA stencil path).
//
// One launch runs CG iterations until r.r <= tol2 or an iteration budget is
// used up.  Per iteration, with beta and r.r known to every CTA:
//   A. each CTA takes tiles t = blockIdx.x + k * gridDim.x; TMA brings the halo
//      boxes of r and p_old; the direction p = r + beta p_old is formed in
//      shared memory (so p is never a separate pass), its interior written to
//      the other direction buffer, and q = P K P p with p.q comes from the
//      stencil of the batched matvec (Sec. 3.2-3.4).
//   all-reduce of the per-CTA p.q partials.
//   B. alpha = r.r / p.q; x += alpha p, r -= alpha q and the r.r partials over
//      a grid-stride range of 16-byte packs.
//   all-reduce of the r.r partials; every CTA forms beta and tests convergence
//   from the same bits, so all CTAs leave the loop together.
// The two direction buffers alternate: tiles read p_old from one while other
// CTAs write p to the other.  Sums run in a fixed order, so a solve is
// deterministic.  Every wait is bounded; a CTA that gives up sets the device
// error word, which makes every other CTA return too.
//
// A grid-wide barrier costs several microseconds on this GPU (a chain of
// dependent L2 round trips across both dies) -- about what a kernel boundary
// costs -- so the persistent form pays off where the operator is cheap: the
// driver uses it when all tiles fit one wave of resident CTAs.  (Forms of CG
// with one reduction per iteration exist; in FP32 the pipelined recurrences of
// Ghysels and Vanroose stagnate near 1e-5 relative residual on these plates, and
// Chronopoulos-Gear saves one barrier but needs ~20 % more iterations and three
// halo arrays, which does not pay at these sizes.)
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "pd_cg.cuh"
#include "pd_reduce.cuh"
#include "pd_tma2d.cuh"

namespace pd {

namespace {

using namespace tma2d;

constexpr int kSpin = 1 << 22;   // grid-barrier poll limit (with a short sleep per poll)

// Sum over the 32 lanes of a warp by an xor butterfly: every lane ends with the
// same value (each step adds the same two numbers in every lane pair).
__device__ __forceinline__ double warp_allsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide all-reduce of two values and barrier for a cooperative launch of at
// most 1024 CTAs, two-level so that no counter sees more than 32 arrivals: CTA b
// posts its values in part[2b..2b+1] and arrives at the counter of group b / 32;
// the last arrival of a group sums the group's values in index order and
// arrives at the top counter; the last group sums the group sums in order,
// publishes the totals and advances the generation the other CTAs poll
// (bounded).  The result is the same bits in every CTA and for every arrival
// order.  v0, v1 must be valid in thread 0; false (in every thread) when a wait
// gave up or another CTA set the device error word.
__device__ __forceinline__ bool grid_allreduce2(double v0, double v1, CgBar *B, double *part, int *err, int *s_fail,
                                                double *s_val, double &o0, double &o1)
{
    __syncthreads();   // this CTA's global writes precede its arrival
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, G = gridDim.x, bid = blockIdx.x;
        const int grp = bid >> 5, g0 = grp << 5, gn = min(G - g0, 32), ngrp = (G + 31) >> 5;
        volatile unsigned int *vgen = &B->gen;
        unsigned int gen = 0;
        int last = 0;
        if (lane == 0) {
            gen = *vgen;
            part[2 * bid] = v0;
            part[2 * bid + 1] = v1;
            __threadfence();
            last = (atomicAdd(&B->grp[grp].count, 1u) == (unsigned int)(gn - 1));
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            const double s0 = warp_allsum(lane < gn ? __ldcg(part + 2 * (g0 + lane)) : 0.0);
            const double s1 = warp_allsum(lane < gn ? __ldcg(part + 2 * (g0 + lane) + 1) : 0.0);
            int top = 0;
            if (lane == 0) {
                B->grp[grp].count = 0u;
                B->gsum[grp][0] = s0;
                B->gsum[grp][1] = s1;
                __threadfence();
                top = (atomicAdd(&B->top, 1u) == (unsigned int)(ngrp - 1));
            }
            top = __shfl_sync(0xffffffffu, top, 0);
            if (top) {
                __threadfence();
                const double t0 = warp_allsum(lane < ngrp ? __ldcg(&B->gsum[lane][0]) : 0.0);
                const double t1 = warp_allsum(lane < ngrp ? __ldcg(&B->gsum[lane][1]) : 0.0);
                if (lane == 0) {
                    B->total[0] = t0;
                    B->total[1] = t1;
                    B->top = 0u;
                    __threadfence();
                    atomicAdd(&B->gen, 1u);
                }
            }
        }
        if (lane == 0) {
            bool ok = false;
            for (int i = 0; i < kSpin; ++i) {
                if (*vgen != gen) {
                    ok = true;
                    break;
                }
                if (*(volatile int *)err) break;
                __nanosleep(32);
            }
            __threadfence();
            if (ok) {
                s_val[0] = __ldcg(&B->total[0]);
                s_val[1] = __ldcg(&B->total[1]);
            } else {
                atomicCAS(err, 0, 2);
                *s_fail = 1;
            }
        }
    }
    __syncthreads();
    o0 = s_val[0];
    o1 = s_val[1];
    return *s_fail == 0;
}

// The direction and operator part of one CG iteration for the tiles t = first,
// first + stride, ...: TMA brings the halo boxes of r and p_old into sr / sp,
// p = r + beta p_old is formed in shared memory, its interior written to pn, and
// q = P K P p (with the per-thread partial of p.q added to dot) written to q.
// Shared by the persistent loop and the graph-replayed one.  False (in every
// thread) when a TMA wait gave up; the error word is then set.
template <int M>
__device__ __forceinline__ bool cg_dir_tiles(const CUtensorMap *map_r, const CUtensorMap *mp, float *sr, float *sp,
                                             float *pn, float *q, float b32, int nx, int ny, int64_t N, int tiles_x,
                                             int ntiles, int first, int stride, const uint8_t *__restrict__ cons,
                                             const uint8_t *__restrict__ tile_flags, const float *s_kd,
                                             const float *__restrict__ kd, const PackTab<M> &tab, uint64_t *bar_,
                                             uint32_t &phase, int *s_fail, int *err, double &dot_cta)
{
    constexpr int XL = x_lead<M>(), BX = box_x<M>(), WL = kRt + 2 * M;
    constexpr int PLANE = BX * box_y<M>();
    constexpr uint32_t kBytes = 2u * PLANE * sizeof(float);
    constexpr int NP = PackTab<M>::kPairs;
    const int tx = threadIdx.x % kTXt, ty = threadIdx.x / kTXt;
    uint64_t &bar = *bar_;
    const int G = stride;
    for (int t = first; t < ntiles; t += G) {
        const int x0 = (t % tiles_x) * kTXt, y0 = (t / tiles_x) * kTYt;
        if (threadIdx.x == 0) {
            // r and p_old were written through the generic proxy before this launch or the last grid barrier
            asm volatile("fence.proxy.async;" ::: "memory");
            mbar_expect_tx(&bar, 2 * kBytes);
            tma_load_3d(sr, map_r, x0 - XL, y0 - M, 0, &bar);
            tma_load_3d(sp, mp, x0 - XL, y0 - M, 0, &bar);
        }
        if (!mbar_wait(&bar, phase)) {
            atomicCAS(err, 0, 1);
            *s_fail = 1;
        }
        phase ^= 1u;
        __syncthreads();
        if (*s_fail) {
            if (threadIdx.x == 0) mbar_wait(&bar, phase ^ 1u);   // let the copies land (bounded)
            return false;
        }
        // p = r + beta p_old over the whole box (zero outside the grid stays zero)
        for (int e = threadIdx.x; e < PLANE; e += kThreads) {
            sp[e] = sr[e] + b32 * sp[e];
            sp[PLANE + e] = sr[PLANE + e] + b32 * sp[PLANE + e];
        }
        __syncthreads();

        u64 a1[kRt], a2[kRt], w0[WL];
        // difference form: FP32 error relative to |K p| for smooth directions too
        tile_pairs<M, true>(sp + (ty * kRt) * BX + tx + XL, sp + PLANE + (ty * kRt) * BX + tx + XL, tab, a1, a2,
                            w0);

        const int gx = x0 + tx, gy0 = y0 + ty * kRt;
        const int64_t o0 = (int64_t)gy0 * nx + gx;
        float dot = 0.f;
        const bool interior = (x0 >= M) && (x0 + kTXt <= nx - M) && (y0 >= M) && (y0 + kTYt <= ny - M);
        if (interior && !tile_flags[t]) {
#pragma unroll
            for (int r = 0; r < kRt; ++r) {
                const float2 up = upk(w0[r + M]);
                const float2 x1 = upk(a1[r]), x2 = upk(a2[r]);
                const float fx = -(x1.x + x2.y);
                const float fy = -(x1.y + x2.x);
                const int64_t p = o0 + (int64_t)r * nx;
                q[p] = fx;
                q[N + p] = fy;
                pn[p] = up.x;
                pn[N + p] = up.y;
                dot = __fmaf_rn(up.x, fx, __fmaf_rn(up.y, fy, dot));
            }
        } else {
            const int xc = min(gx, M) * (M + 1) + min(nx - 1 - gx, M);
#pragma unroll
            for (int r = 0; r < kRt; ++r) {
                const int gy = gy0 + r;
                if (gx >= nx || gy >= ny) continue;
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
                kxx -= tab.v[4 * NP];   // the difference-form sums already hold -Kd_int u_p
                kxy -= tab.v[4 * NP + 1];
                kyy -= tab.v[4 * NP + 2];
                float fx = __fmaf_rn(kxx, up.x, __fmaf_rn(kxy, up.y, -ax));
                float fy = __fmaf_rn(kxy, up.x, __fmaf_rn(kyy, up.y, -ay));
                const int64_t p = o0 + (int64_t)r * nx;
                if (cons) {
                    const uint8_t m = __ldg(cons + p);
                    if (m & 1) fx = 0.f;
                    if (m & 2) fy = 0.f;
                }
                q[p] = fx;
                q[N + p] = fy;
                pn[p] = up.x;
                pn[N + p] = up.y;
                dot = __fmaf_rn(up.x, fx, __fmaf_rn(up.y, fy, dot));
            }
        }
        dot_cta += (double)dot;
        __syncthreads();   // the boxes are read; the next tile may overwrite them
    }
    return true;
}

template <int M>
__global__ void __launch_bounds__(kThreads, (M <= 3 ? 3 : 2))
k_cg_persist(const __grid_constant__ CUtensorMap map_r, const __grid_constant__ CUtensorMap map_p0,
             const __grid_constant__ CUtensorMap map_p1, const __grid_constant__ CgVecs v, int nx, int ny, int64_t N,
             int tiles_x, int ntiles, const uint8_t *__restrict__ cons, const uint8_t *__restrict__ tile_flags,
             const float *__restrict__ kd, PackTab<M> tab, CgScal *sc, CgBar *gbar, double *part, int budget,
             int *err)
{
    constexpr int XL = x_lead<M>(), BX = box_x<M>(), BY = box_y<M>(), WL = kRt + 2 * M;
    constexpr int PLANE = BX * BY;
    constexpr uint32_t kBytes = 2u * PLANE * sizeof(float);   // one array, both components
    constexpr int NP = PackTab<M>::kPairs;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *const sr = reinterpret_cast<float *>(smem_raw);   // r box: x plane, y plane
    float *const sp = sr + 2 * PLANE;                        // p box: x plane, y plane
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_fail;
    __shared__ double red[kThreads / 32];
    __shared__ double s_val[2];
    constexpr int KDS = (M <= 3) ? 3 * (M + 1) * (M + 1) * (M + 1) * (M + 1) : 1;
    __shared__ float s_kd[KDS];
    if (M <= 3)
        for (int i = threadIdx.x; i < KDS; i += kThreads) s_kd[i] = __ldg(kd + i);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();

    // solve state: identical in every CTA
    double rr = sc->rr, beta = sc->beta;
    const double tol2 = sc->tol2;
    int pbuf = sc->pbuf, iters = sc->iters, done = sc->done;
    const int G = gridDim.x;
    const int tx = threadIdx.x % kTXt, ty = threadIdx.x / kTXt;
    const int64_t nv = (2 * N) / 4;   // N is a multiple of 4 on the TMA path
    const int64_t t0 = (int64_t)blockIdx.x * kThreads + threadIdx.x, stride = (int64_t)G * kThreads;
    uint32_t phase = 0;

    for (int k = 0; k < budget && !done; ++k) {
        const CUtensorMap *mp = pbuf ? &map_p1 : &map_p0;
        float *pn = v.p[pbuf ^ 1];   // this iteration's direction
        const float b32 = (float)beta;

        // ---- A. direction and operator over this CTA's tiles
        double dot_cta = 0.0;
        if (!cg_dir_tiles<M>(&map_r, mp, sr, sp, pn, v.q, b32, nx, ny, N, tiles_x, ntiles, blockIdx.x, G, cons,
                             tile_flags, s_kd, kd, tab, &bar, phase, &s_fail, err, dot_cta))
            return;
        double pq, unused;
        if (!grid_allreduce2(block_sum(dot_cta, red), 0.0, gbar, part, err, &s_fail, s_val, pq, unused)) return;

        // ---- B. x += alpha p, r -= alpha q, r.r
        const float a32 = (float)((pq != 0.0) ? rr / pq : 0.0);
        float acc = 0.f;
        for (int64_t j = t0; j < nv; j += stride) {
            float4 xv = reinterpret_cast<float4 *>(v.x)[j], rv = reinterpret_cast<float4 *>(v.r)[j];
            float4 xl = reinterpret_cast<float4 *>(v.xlo)[j];
            const float4 pv = __ldcg(reinterpret_cast<const float4 *>(pn) + j);
            const float4 qv = __ldcg(reinterpret_cast<const float4 *>(v.q) + j);
            two_sum_acc(xv.x, xl.x, a32 * pv.x);
            two_sum_acc(xv.y, xl.y, a32 * pv.y);
            two_sum_acc(xv.z, xl.z, a32 * pv.z);
            two_sum_acc(xv.w, xl.w, a32 * pv.w);
            rv.x -= a32 * qv.x;
            rv.y -= a32 * qv.y;
            rv.z -= a32 * qv.z;
            rv.w -= a32 * qv.w;
            acc += rv.x * rv.x;
            acc += rv.y * rv.y;
            acc += rv.z * rv.z;
            acc += rv.w * rv.w;
            reinterpret_cast<float4 *>(v.x)[j] = xv;
            reinterpret_cast<float4 *>(v.xlo)[j] = xl;
            reinterpret_cast<float4 *>(v.r)[j] = rv;
        }
        double rn;
        if (!grid_allreduce2(block_sum(acc, red), 0.0, gbar, part, err, &s_fail, s_val, rn, unused)) return;
        beta = (rr > 0.0) ? rn / rr : 0.0;
        rr = rn;
        ++iters;
        pbuf ^= 1;   // p of this iteration becomes p_old
        if (!(rn > tol2)) done = 1;   // also stops on NaN
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->rr = rr;
        sc->beta = beta;
        sc->iters = iters;
        sc->done = done;
        sc->pbuf = pbuf;
    }
}

// The direction and operator step of one graph-replayed CG iteration (the
// update that follows is k_cg_update2 in pd_cg.cu): reads beta and the index of
// p_old from sc, forms p and q = P K P p for every tile and reduces p.q into
// sc->pq (last block, fixed order).
template <int M>
__global__ void __launch_bounds__(kThreads, (M <= 3 ? 3 : 2))
k_cg_dirmv(const __grid_constant__ CUtensorMap map_r, const __grid_constant__ CUtensorMap map_p0,
           const __grid_constant__ CUtensorMap map_p1, const __grid_constant__ CgVecs v, int nx, int ny, int64_t N,
           int tiles_x, int ntiles, const uint8_t *__restrict__ cons, const uint8_t *__restrict__ tile_flags,
           const float *__restrict__ kd, PackTab<M> tab, CgScal *sc, double *partial, int *err)
{
    constexpr int BX = box_x<M>(), BY = box_y<M>();
    constexpr int PLANE = BX * BY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *const sr = reinterpret_cast<float *>(smem_raw);
    float *const sp = sr + 2 * PLANE;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_fail;
    __shared__ double red[kThreads / 32];
    constexpr int KDS = (M <= 3) ? 3 * (M + 1) * (M + 1) * (M + 1) * (M + 1) : 1;
    __shared__ float s_kd[KDS];
    if (sc->done) return;   // uniform: the solve converged earlier in this chunk
    if (M <= 3)
        for (int i = threadIdx.x; i < KDS; i += kThreads) s_kd[i] = __ldg(kd + i);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();
    const int pbuf = sc->pbuf;
    const CUtensorMap *mp = pbuf ? &map_p1 : &map_p0;
    uint32_t phase = 0;
    double dot_cta = 0.0;
    if (!cg_dir_tiles<M>(&map_r, mp, sr, sp, v.p[pbuf ^ 1], v.q, (float)sc->beta, nx, ny, N, tiles_x, ntiles,
                         blockIdx.x, gridDim.x, cons, tile_flags, s_kd, kd, tab, &bar, phase, &s_fail, err, dot_cta))
        return;
    const double s = block_sum(dot_cta, red);
    grid_finish(s, gridDim.x, blockIdx.x, partial, &sc->pq, &sc->retire[2], red);
}

// one thread per tile: does the tile's 64 x 32 output block hold a constrained node?
__global__ void k_tile_flags(const uint8_t *__restrict__ cons, int nx, int ny, int tiles_x, int ntiles,
                             uint8_t *__restrict__ flags)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int x0 = (t % tiles_x) * kTXt, y0 = (t / tiles_x) * kTYt;
    uint8_t any = 0;
    if (cons)
        for (int y = y0; y < min(y0 + kTYt, ny); ++y)
            for (int xx = x0; xx < min(x0 + kTXt, nx); ++xx) any |= cons[(int64_t)y * nx + xx];
    flags[t] = any ? 1 : 0;
}

template <int M>
int launch(pd_grid *g, const CgVecs &v, CgScal *sc, CgBar *gbar, double *part, const uint8_t *tile_flags, int budget,
           cudaStream_t s)
{
    constexpr int BX = box_x<M>(), BY = box_y<M>();
    int nx = (int)g->n[0], ny = (int)g->n[1];
    CUtensorMap mr, m0, m1;
    if (!make_map<M>(&mr, v.r, nx, ny, 1) || !make_map<M>(&m0, v.p[0], nx, ny, 1) ||
        !make_map<M>(&m1, v.p[1], nx, ny, 1))
        return fail(PD_ERR_CUDA, "tensor map encode failed");
    const size_t smem = 4ull * BX * BY * sizeof(float);
    auto kern = k_cg_persist<M>;
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int G = cg_persist_ctas(g);
    int tiles_x = (nx + kTXt - 1) / kTXt;
    int ntiles = cg_persist_ntiles(g);
    int64_t N = g->N;
    const uint8_t *cons = g->has_cons ? g->d_cons : nullptr;
    const float *kd = g->d_kd32;
    PackTab<M> tab = make_pack<M>(g);
    int *err = g->d_err;
    CgVecs vv = v;
    void *args[] = {(void *)&mr, (void *)&m0, (void *)&m1, (void *)&vv, (void *)&nx, (void *)&ny, (void *)&N,
                    (void *)&tiles_x, (void *)&ntiles, (void *)&cons, (void *)&tile_flags, (void *)&kd, (void *)&tab,
                    (void *)&sc, (void *)&gbar, (void *)&part, (void *)&budget, (void *)&err};
    PD_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(kThreads), args, smem, s));
    return PD_OK;
}

int resident_ctas(int M);

template <int M>
int launch_dirmv(pd_grid *g, const CgVecs &v, CgScal *sc, double *partial, const uint8_t *tile_flags, cudaStream_t s)
{
    constexpr int BX = box_x<M>(), BY = box_y<M>();
    const int nx = (int)g->n[0], ny = (int)g->n[1];
    CUtensorMap mr, m0, m1;
    if (!make_map<M>(&mr, v.r, nx, ny, 1) || !make_map<M>(&m0, v.p[0], nx, ny, 1) ||
        !make_map<M>(&m1, v.p[1], nx, ny, 1))
        return fail(PD_ERR_CUDA, "tensor map encode failed");
    const size_t smem = 4ull * BX * BY * sizeof(float);
    auto kern = k_cg_dirmv<M>;
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int tiles_x = (nx + kTXt - 1) / kTXt;
    const int ntiles = cg_persist_ntiles(g);
    const int G = std::max(1, std::min(ntiles, resident_ctas(M)));
    kern<<<G, kThreads, smem, s>>>(mr, m0, m1, v, nx, ny, g->N, tiles_x, ntiles, g->has_cons ? g->d_cons : nullptr,
                                   tile_flags, g->d_kd32, make_pack<M>(g), sc, partial, g->d_err);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <int M>
int occupancy_ctas()
{
    constexpr int BX = box_x<M>(), BY = box_y<M>();
    const size_t smem = 4ull * BX * BY * sizeof(float);
    auto kern = k_cg_persist<M>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem) != cudaSuccess) return 0;
    return occ * sms;
}

int resident_ctas(int M)
{
    switch (M) {
        case 1: return occupancy_ctas<1>();
        case 2: return occupancy_ctas<2>();
        case 3: return occupancy_ctas<3>();
        case 4: return occupancy_ctas<4>();
        case 5: return occupancy_ctas<5>();
        case 6: return occupancy_ctas<6>();
        case 7: return occupancy_ctas<7>();
        case 8: return occupancy_ctas<8>();
    }
    return 0;
}

}  // namespace

int cg_persist_ntiles(const pd_grid *g)
{
    return (int)(((g->n[0] + kTXt - 1) / kTXt) * ((g->n[1] + kTYt - 1) / kTYt));
}

int cg_persist_ctas(const pd_grid *g)
{
    const int res = resident_ctas(g->M);
    return std::max(1, std::min(res, cg_persist_ntiles(g)));
}

bool cg_persist_eligible(const pd_grid *g)
{
    if (g->dim != 2 || g->has_E || g->broken_total > 0 || g->no_tma || g->sc) return false;
    if (g->auto_choice[0] == 2) return false;   // the FFT method was chosen for FP32
    if (g->M < 1 || g->M > 8 || g->n[0] % 4 != 0) return false;
    if (encode_fn() == nullptr) return false;
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
    const int res = resident_ctas(g->M);
    return res > 0 && cg_persist_ntiles(g) <= res;
}

bool cg_dirmv_eligible(const pd_grid *g)
{
    if (g->dim != 2 || g->has_E || g->broken_total > 0 || g->no_tma || g->sc) return false;
    if (g->auto_choice[0] == 2) return false;   // the FFT method was chosen for FP32
    if (g->M < 1 || g->M > 8 || g->n[0] % 4 != 0) return false;
    return encode_fn() != nullptr && resident_ctas(g->M) > 0;
}

int cg_dirmv_run(pd_grid *g, const CgVecs &v, CgScal *sc, double *partial, const uint8_t *tile_flags, cudaStream_t s)
{
    switch (g->M) {
        case 1: return launch_dirmv<1>(g, v, sc, partial, tile_flags, s);
        case 2: return launch_dirmv<2>(g, v, sc, partial, tile_flags, s);
        case 3: return launch_dirmv<3>(g, v, sc, partial, tile_flags, s);
        case 4: return launch_dirmv<4>(g, v, sc, partial, tile_flags, s);
        case 5: return launch_dirmv<5>(g, v, sc, partial, tile_flags, s);
        case 6: return launch_dirmv<6>(g, v, sc, partial, tile_flags, s);
        case 7: return launch_dirmv<7>(g, v, sc, partial, tile_flags, s);
        case 8: return launch_dirmv<8>(g, v, sc, partial, tile_flags, s);
    }
    return fail(PD_ERR_INVALID, "horizon M not compiled for 2D");
}

int cg_persist_tile_flags(pd_grid *g, uint8_t *tile_flags, cudaStream_t s)
{
    const int nt = cg_persist_ntiles(g);
    const int tiles_x = (int)((g->n[0] + kTXt - 1) / kTXt);
    k_tile_flags<<<(nt + 127) / 128, 128, 0, s>>>(g->has_cons ? g->d_cons : nullptr, (int)g->n[0], (int)g->n[1],
                                                  tiles_x, nt, tile_flags);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int cg_persist_run(pd_grid *g, const CgVecs &v, CgScal *sc, CgBar *gbar, double *part, const uint8_t *tile_flags,
                   int budget, cudaStream_t s)
{
    if (budget < 1) return PD_OK;
    switch (g->M) {
        case 1: return launch<1>(g, v, sc, gbar, part, tile_flags, budget, s);
        case 2: return launch<2>(g, v, sc, gbar, part, tile_flags, budget, s);
        case 3: return launch<3>(g, v, sc, gbar, part, tile_flags, budget, s);
        case 4: return launch<4>(g, v, sc, gbar, part, tile_flags, budget, s);
        case 5: return launch<5>(g, v, sc, gbar, part, tile_flags, budget, s);
        case 6: return launch<6>(g, v, sc, gbar, part, tile_flags, budget, s);
        case 7: return launch<7>(g, v, sc, gbar, part, tile_flags, budget, s);
        case 8: return launch<8>(g, v, sc, gbar, part, tile_flags, budget, s);
    }
    return fail(PD_ERR_INVALID, "horizon M not compiled for 2D");
}

}  // namespace pd

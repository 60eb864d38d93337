// pd_cg.cu -- conjugate gradients on the projected stiffness P K P u = P b.
//
// The paper drives its static problem (Eq. mat:e2) with adaptive dynamic
// relaxation; this library pairs the same operator with CG, in two modes:
//
//  * PD_CG_F64: textbook CG with FP64 vectors and the FP64 operator.
//  * PD_CG_MIXED: CG with FP32 vectors and the FP32 operator (dot products
//    reduced in FP64), u kept in FP64, with reliable updates: each time the
//    FP32 residual has fallen tenfold, the FP32 increment is folded into u, the
//    true residual r = P(b - K u) is formed with the FP64 operator and replaces
//    the FP32 one while the search direction is kept.  This is FP64 iterative
//    refinement without the restarts, so the iteration count stays close to
//    that of FP64 CG.
//
// One inner iteration is three launches: (1) q = K p with p.q fused into the
// stencil epilogue, (2) alpha = rr / pq, x += alpha p, r -= alpha q, r.r
// reduced in the same kernel, whose last block also forms beta and the
// convergence flag, (3) p = r + beta p.  All scalars stay on the device; the
// host only looks at the flag between chunks of iterations, which are captured
// once into a CUDA graph and replayed.  Every kernel returns early once the
// flag is set, so iterations after convergence inside a chunk change nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>

#include "pd_cg.cuh"
#include "pd_internal.cuh"
#include "pd_reduce.cuh"

namespace pd {

namespace {

constexpr int kBlk = 256;
constexpr int kRedMax = 152 * 8;      // upper bound of the streaming kernels' grid (grid-stride)
constexpr int kChunk = 32;            // inner iterations per graph launch


// 16 bytes of T: the streaming kernels move whole packs with one vector load
// or store.  A kernel gets the number of packs `nv` it may treat that way (0
// when a pointer is not 16-byte aligned) and handles elements [nv * n, L) one
// by one.
template <typename T>
struct alignas(16) Pk {
    static constexpr int n = 16 / (int)sizeof(T);
    T v[n];
};

template <typename T>
__device__ __forceinline__ Pk<T> ldp(const T *a, int64_t j)
{
    return reinterpret_cast<const Pk<T> *>(a)[j];
}

template <typename T>
__device__ __forceinline__ void stp(T *a, int64_t j, const Pk<T> &v)
{
    reinterpret_cast<Pk<T> *>(a)[j] = v;
}

__host__ __device__ inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Deterministic grid reduction whose last block returns true in thread 0.
__device__ __forceinline__ bool grid_last(double block_value, double *partial, double *out, unsigned int *retire,
                                          double *red)
{
    __shared__ bool s_last;
    const int nb = gridDim.x, bid = blockIdx.x;
    if (threadIdx.x == 0) {
        partial[bid] = block_value;
        __threadfence();
        const unsigned int t = atomicAdd(retire, 1u);
        s_last = (t == (unsigned int)(nb - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += __ldcg(&partial[i]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        *out = s;
        *retire = 0u;
        return true;
    }
    return false;
}

// x += alpha p ; r -= alpha q ; rr_new = r.r ; last block: beta, rr, done, iters.
// FP32: x + xlo is a compensated sum (two_sum_acc); FP64: xlo unused.
template <typename T>
__global__ void __launch_bounds__(kBlk, 4)
k_cg_update(T *x, T *xlo, T *r, const T *__restrict__ p, const T *__restrict__ q, int64_t L, int64_t nv, CgScal *sc,
            double *partial)
{
    __shared__ double red[kBlk / 32];
    __shared__ int s_done;
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_alpha = (sc->pq != 0.0) ? sc->rr / sc->pq : 0.0;
    }
    __syncthreads();
    if (s_done) return;
    const T a = (T)s_alpha;
    T acc = T(0);
    const int64_t t0 = (int64_t)blockIdx.x * kBlk + threadIdx.x, st = (int64_t)gridDim.x * kBlk;
    constexpr bool comp = sizeof(T) == 4;
    for (int64_t j = t0; j < nv; j += st) {
        Pk<T> xv = ldp(x, j), rv = ldp(r, j);
        Pk<T> xl;
        if constexpr (comp) xl = ldp(xlo, j);
        const Pk<T> pv = ldp(p, j), qv = ldp(q, j);
#pragma unroll
        for (int e = 0; e < Pk<T>::n; ++e) {
            if constexpr (comp)
                two_sum_acc(xv.v[e], xl.v[e], a * pv.v[e]);
            else
                xv.v[e] += a * pv.v[e];
            rv.v[e] -= a * qv.v[e];
            acc += rv.v[e] * rv.v[e];
        }
        stp(x, j, xv);
        if constexpr (comp) stp(xlo, j, xl);
        stp(r, j, rv);
    }
    for (int64_t i = nv * Pk<T>::n + t0; i < L; i += st) {
        if constexpr (comp) {
            float xi = x[i], xli = xlo[i];
            two_sum_acc(xi, xli, a * p[i]);
            x[i] = xi;
            xlo[i] = xli;
        } else {
            x[i] = x[i] + a * p[i];
        }
        const T ri = r[i] - a * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    const double bs = block_sum(acc, red);
    if (grid_last(bs, partial, &sc->rr_new, &sc->retire[0], red)) {
        const double rn = sc->rr_new;
        sc->beta = (sc->rr > 0.0) ? rn / sc->rr : 0.0;
        sc->rr = rn;
        sc->iters += 1;
        if (!(rn > sc->tol2)) sc->done = 1;   // also stops on NaN
    }
}

// p = r + beta p
template <typename T>
__global__ void __launch_bounds__(kBlk)
k_cg_p(T *p, const T *__restrict__ r, int64_t L, int64_t nv, const CgScal *sc)
{
    if (sc->done) return;
    const T beta = (T)sc->beta;
    const int64_t t0 = (int64_t)blockIdx.x * kBlk + threadIdx.x, st = (int64_t)gridDim.x * kBlk;
    for (int64_t j = t0; j < nv; j += st) {
        Pk<T> pv = ldp(p, j);
        const Pk<T> rv = ldp(r, j);
#pragma unroll
        for (int e = 0; e < Pk<T>::n; ++e) pv.v[e] = rv.v[e] + beta * pv.v[e];
        stp(p, j, pv);
    }
    for (int64_t i = nv * Pk<T>::n + t0; i < L; i += st) p[i] = r[i] + beta * p[i];
}

// Update of the graph-replayed fused loop: p_new sits in direction buffer
// pbuf ^ 1 (written by the direction/operator kernel).  x += alpha p_new,
// r -= alpha q, r.r; the last block forms beta, tests convergence and makes
// p_new the next p_old.  Every block reads pbuf before the last block flips it.
__global__ void __launch_bounds__(kBlk, 4)
k_cg_update2(float *x, float *xlo, float *r, const float *p0, const float *p1, const float *__restrict__ q, int64_t L,
             int64_t nv, CgScal *sc, double *partial)
{
    __shared__ double red[kBlk / 32];
    __shared__ int s_done, s_pbuf;
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_pbuf = sc->pbuf;
        s_alpha = (sc->pq != 0.0) ? sc->rr / sc->pq : 0.0;
    }
    __syncthreads();
    if (s_done) return;
    const float *__restrict__ p = s_pbuf ? p0 : p1;
    const float a = (float)s_alpha;
    float acc = 0.f;
    const int64_t t0 = (int64_t)blockIdx.x * kBlk + threadIdx.x, st = (int64_t)gridDim.x * kBlk;
    for (int64_t j = t0; j < nv; j += st) {
        Pk<float> xv = ldp(x, j), xl = ldp(xlo, j), rv = ldp(r, j);
        const Pk<float> pv = ldp(p, j), qv = ldp(q, j);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            two_sum_acc(xv.v[e], xl.v[e], a * pv.v[e]);
            rv.v[e] -= a * qv.v[e];
            acc += rv.v[e] * rv.v[e];
        }
        stp(x, j, xv);
        stp(xlo, j, xl);
        stp(r, j, rv);
    }
    for (int64_t i = nv * 4 + t0; i < L; i += st) {
        float xi = x[i], xli = xlo[i];
        two_sum_acc(xi, xli, a * p[i]);
        const float ri = r[i] - a * q[i];
        x[i] = xi;
        xlo[i] = xli;
        r[i] = ri;
        acc += ri * ri;
    }
    const double bs = block_sum(acc, red);
    if (grid_last(bs, partial, &sc->rr_new, &sc->retire[0], red)) {
        const double rn = sc->rr_new;
        sc->beta = (sc->rr > 0.0) ? rn / sc->rr : 0.0;
        sc->rr = rn;
        sc->iters += 1;
        sc->pbuf ^= 1;
        if (!(rn > sc->tol2)) sc->done = 1;   // also stops on NaN
    }
}

// out = a . b (accumulated per thread in the kernel's precision, FP64 across threads)
template <typename T>
__global__ void __launch_bounds__(kBlk)
k_dot(const T *__restrict__ a, const T *__restrict__ b, int64_t L, int64_t nv, double *out, double *partial,
      unsigned int *retire)
{
    __shared__ double red[kBlk / 32];
    T acc = T(0);
    const int64_t t0 = (int64_t)blockIdx.x * kBlk + threadIdx.x, st = (int64_t)gridDim.x * kBlk;
    for (int64_t j = t0; j < nv; j += st) {
        const Pk<T> av = ldp(a, j), bv = ldp(b, j);
#pragma unroll
        for (int e = 0; e < Pk<T>::n; ++e) acc += av.v[e] * bv.v[e];
    }
    for (int64_t i = nv * Pk<T>::n + t0; i < L; i += st) acc += a[i] * b[i];
    const double bs = block_sum(acc, red);
    grid_last(bs, partial, out, retire, red);
}

// r = P(b - Ku) in FP64, and r.r  (Ku already projected by the matvec)
__global__ void __launch_bounds__(kBlk)
k_resid(double *r, const double *__restrict__ b, const double *__restrict__ Ku, const uint8_t *__restrict__ cons,
        int64_t N, int dim, double *out, double *partial, unsigned int *retire)
{
    __shared__ double red[kBlk / 32];
    double acc = 0.0;
    const int64_t L = (int64_t)dim * N;
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < L; i += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(i / N);
        const int64_t p = i - c * N;
        const bool fixed = cons && ((cons[p] >> c) & 1);
        const double v = fixed ? 0.0 : b[i] - Ku[i];
        r[i] = v;
        acc += v * v;
    }
    const double bs = block_sum(acc, red);
    grid_last(bs, partial, out, retire, red);
}

// Inner start (mixed): r32 = r64 * inv, p32 = r32, x32 = 0, sc->rr = r32.r32, done flag.
// nv counts packs of four floats (two packs of doubles each).
__global__ void __launch_bounds__(kBlk)
k_inner_start(float *r32, float *p32, float *x32, float *xlo32, const double *__restrict__ r64, int64_t L, int64_t nv,
              double inv, double tau2, CgScal *sc, double *partial)
{
    __shared__ double red[kBlk / 32];
    float acc = 0.f;
    const int64_t t0 = (int64_t)blockIdx.x * kBlk + threadIdx.x, st = (int64_t)gridDim.x * kBlk;
    for (int64_t j = t0; j < nv; j += st) {
        const Pk<double> a = ldp(r64, 2 * j), b = ldp(r64, 2 * j + 1);
        Pk<float> v;
        v.v[0] = (float)(a.v[0] * inv);
        v.v[1] = (float)(a.v[1] * inv);
        v.v[2] = (float)(b.v[0] * inv);
        v.v[3] = (float)(b.v[1] * inv);
        stp(r32, j, v);
        stp(p32, j, v);
        stp(x32, j, Pk<float>{});
        stp(xlo32, j, Pk<float>{});
#pragma unroll
        for (int e = 0; e < 4; ++e) acc += v.v[e] * v.v[e];
    }
    for (int64_t i = nv * 4 + t0; i < L; i += st) {
        const float v = (float)(r64[i] * inv);
        r32[i] = v;
        p32[i] = v;
        x32[i] = 0.f;
        xlo32[i] = 0.f;
        acc += v * v;
    }
    const double bs = block_sum(acc, red);
    if (grid_last(bs, partial, &sc->rr, &sc->retire[1], red)) {
        sc->tol2 = tau2 * sc->rr;
        sc->done = (sc->rr > sc->tol2) ? 0 : 1;
        sc->iters = 0;
        sc->beta = 0.0;   // persistent loop: p = r + 0 * p_old on its first iteration
        sc->pbuf = 0;
    }
}

// Plain start (FP64): p = r, sc->rr = rr (given on device in sc->aux), tol2, done.
__global__ void __launch_bounds__(kBlk)
k_plain_start(double *p, const double *__restrict__ r, int64_t L, double tol2, CgScal *sc)
{
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < L; i += (int64_t)gridDim.x * kBlk) p[i] = r[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->rr = sc->aux;
        sc->tol2 = tol2;
        sc->done = (sc->rr > tol2) ? 0 : 1;
        sc->iters = 0;
    }
}

// u += s * (x32 + xlo32), then both = 0 (a reliable update folds the FP32 increment into u).
__global__ void __launch_bounds__(kBlk)
k_correct_zero(double *u, float *x32, float *xlo32, double s, int64_t L, int64_t nv)
{
    const int64_t t0 = (int64_t)blockIdx.x * kBlk + threadIdx.x, st = (int64_t)gridDim.x * kBlk;
    for (int64_t j = t0; j < nv; j += st) {
        const Pk<float> x = ldp(x32, j), xl = ldp(xlo32, j);
        Pk<double> a = ldp(u, 2 * j), b = ldp(u, 2 * j + 1);
        a.v[0] += s * ((double)x.v[0] + (double)xl.v[0]);
        a.v[1] += s * ((double)x.v[1] + (double)xl.v[1]);
        b.v[0] += s * ((double)x.v[2] + (double)xl.v[2]);
        b.v[1] += s * ((double)x.v[3] + (double)xl.v[3]);
        stp(u, 2 * j, a);
        stp(u, 2 * j + 1, b);
        stp(x32, j, Pk<float>{});
        stp(xlo32, j, Pk<float>{});
    }
    for (int64_t i = nv * 4 + t0; i < L; i += st) {
        u[i] += s * ((double)x32[i] + (double)xlo32[i]);
        x32[i] = 0.f;
        xlo32[i] = 0.f;
    }
}

// r32 = r64 * inv: the true residual replaces the recursive one.  The inner loop
// stopped in the update of iteration k, so p still holds p_{k-1} and sc->beta
// holds beta_k; the new direction is p_k = r_true + beta_k p_{k-1}, i.e. the
// direction CG would have formed had its recursive residual been exact.  The
// persistent loop forms p itself from r and p_old (form_p = 0).
// sc->rr = r32.r32, sc->tol2 = tol2 (absolute), the inner loop is re-armed.
__global__ void __launch_bounds__(kBlk)
k_replace(float *r32, float *p32, const double *__restrict__ r64, int64_t L, int64_t nv, double inv, double tol2,
          CgScal *sc, double *partial, int form_p)
{
    __shared__ double red[kBlk / 32];
    const float beta = (float)sc->beta;
    float acc = 0.f;
    const int64_t t0 = (int64_t)blockIdx.x * kBlk + threadIdx.x, st = (int64_t)gridDim.x * kBlk;
    for (int64_t j = t0; j < nv; j += st) {
        const Pk<double> a = ldp(r64, 2 * j), b = ldp(r64, 2 * j + 1);
        Pk<float> v, pv = ldp(p32, j);
        v.v[0] = (float)(a.v[0] * inv);
        v.v[1] = (float)(a.v[1] * inv);
        v.v[2] = (float)(b.v[0] * inv);
        v.v[3] = (float)(b.v[1] * inv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            pv.v[e] = v.v[e] + beta * pv.v[e];
            acc += v.v[e] * v.v[e];
        }
        if (form_p) stp(p32, j, pv);
        stp(r32, j, v);
    }
    for (int64_t i = nv * 4 + t0; i < L; i += st) {
        const float v = (float)(r64[i] * inv);
        if (form_p) p32[i] = v + beta * p32[i];
        r32[i] = v;
        acc += v * v;
    }
    const double bs = block_sum(acc, red);
    if (grid_last(bs, partial, &sc->rr, &sc->retire[1], red)) {
        sc->tol2 = tol2;
        sc->done = (sc->rr > tol2) ? 0 : 1;
        sc->iters = 0;
    }
}

__global__ void __launch_bounds__(kBlk)
k_zero_constrained(double *u, const uint8_t *__restrict__ cons, int64_t N, int dim)
{
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < (int64_t)dim * N; i += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(i / N);
        if ((cons[i - c * N] >> c) & 1) u[i] = 0.0;
    }
}

// ------------------------------------------------------------------ workspace
struct CgWs {
    size_t bytes = 0;
    void *base = nullptr;
    double *r64, *q64, *p64;    // FP64 residual, operator output, direction
    float *r32, *p32, *q32, *x32, *xlo32;
    float *p32b;                // persistent loop: second direction buffer
    uint8_t *tile_flags;        // persistent loop: tiles holding a constrained node
    CgBar *gbar;                // persistent loop: grid barrier
    int64_t flags_stamp = -1;   // op_stamp the tile flags were computed for
    CgScal *sc;
    double *partial;            // >= max(red, stencil CTAs) doubles
    double *partial2;
    int red = 0;                // grid of the streaming kernels: resident CTAs on all SMs, <= kRedMax
    int red64 = 0;              // the same for the FP64 update
    cudaStream_t cap = nullptr; // capture stream
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};   // [0] FP32 inner, [1] FP64 plain, [2] FP32 fused
    const void *graph_key[3] = {nullptr, nullptr, nullptr};
    int64_t graph_stamp[3] = {-1, -1, -1};
};

int ensure_ws(pd_grid *g, CgWs *&w)
{
    const int64_t L = (int64_t)g->dim * g->N;
    const int nblk = std::max(stencil_blocks(g, true, g->has_E || g->broken_total > 0),
                              stencil_blocks(g, false, g->has_E || g->broken_total > 0));
    const size_t nparts = (size_t)std::max(nblk, kRedMax) + 64;
    const size_t ntile = (size_t)((g->n[0] + 63) / 64) * (size_t)((g->n[1] + 31) / 32) * (size_t)g->n[2];
    const size_t need = sizeof(double) * 3 * L + sizeof(float) * 6 * L + sizeof(CgScal) + 2 * sizeof(double) * nparts +
                        ntile + sizeof(CgBar) + 2560;
    w = (CgWs *)g->cg;
    if (w && w->bytes >= need) return PD_OK;
    if (!w) {
        w = new CgWs();
        g->cg = w;
        PD_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
        int dev = 0, sms = 0, occ = 0;
        PD_CUDA(cudaGetDevice(&dev));
        PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_update<float>, kBlk, 0));
        w->red = std::max(1, std::min(kRedMax, sms * std::max(occ, 1)));
        PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_update<double>, kBlk, 0));
        w->red64 = std::max(1, std::min(kRedMax, sms * std::max(occ, 1)));
    }
    if (w->base) cudaFree(w->base);
    for (int i = 0; i < 3; ++i)
        if (w->graph[i]) {
            cudaGraphExecDestroy(w->graph[i]);
            w->graph[i] = nullptr;
        }
    w->base = nullptr;
    w->bytes = 0;
    if (cudaMalloc(&w->base, need) != cudaSuccess) return fail(PD_ERR_OOM, "CG workspace");
    w->bytes = need;
    char *c = (char *)w->base;
    auto take = [&](size_t n) { char *q = c; c += (n + 255) & ~(size_t)255; return q; };
    w->r64 = (double *)take(sizeof(double) * L);
    w->q64 = (double *)take(sizeof(double) * L);
    w->p64 = (double *)take(sizeof(double) * L);
    w->r32 = (float *)take(sizeof(float) * L);
    w->p32 = (float *)take(sizeof(float) * L);
    w->q32 = (float *)take(sizeof(float) * L);
    w->x32 = (float *)take(sizeof(float) * L);
    w->xlo32 = (float *)take(sizeof(float) * L);
    w->p32b = (float *)take(sizeof(float) * L);
    w->tile_flags = (uint8_t *)take(ntile);
    w->gbar = (CgBar *)take(sizeof(CgBar));
    w->flags_stamp = -1;
    w->sc = (CgScal *)take(sizeof(CgScal));
    w->partial = (double *)take(sizeof(double) * nparts);
    w->partial2 = (double *)take(sizeof(double) * nparts);
    PD_CUDA(cudaMemset(w->sc, 0, sizeof(CgScal)));
    PD_CUDA(cudaMemset(w->gbar, 0, sizeof(CgBar)));
    return PD_OK;
}

CgVecs cg_vecs(CgWs *w)
{
    CgVecs v;
    v.x = w->x32;
    v.xlo = w->xlo32;
    v.r = w->r32;
    v.q = w->q32;
    v.p[0] = w->p32;
    v.p[1] = w->p32b;
    return v;
}

int ensure_tile_flags(pd_grid *g, CgWs *w, cudaStream_t s)
{
    if (w->flags_stamp == g->op_stamp) return PD_OK;
    int rc = cg_persist_tile_flags(g, w->tile_flags, s);
    if (rc == PD_OK) w->flags_stamp = g->op_stamp;
    return rc;
}

// One inner iteration on FP32 (mixed) or FP64 (plain) vectors.  With `fused`
// (FP32 on a TMA-eligible 2D grid) it is two launches: direction + operator
// (k_cg_dirmv) and the update; otherwise matvec, update and direction.
int iteration(pd_grid *g, CgWs *w, bool f64, double *x64, cudaStream_t s, bool fused = false)
{
    const int64_t L = (int64_t)g->dim * g->N;
    if (fused && !f64) {
        int rc = cg_dirmv_run(g, cg_vecs(w), w->sc, w->partial, w->tile_flags, s);
        if (rc) return rc;
        k_cg_update2<<<w->red, kBlk, 0, s>>>(w->x32, w->xlo32, w->r32, w->p32, w->p32b, w->q32, L, L / 4, w->sc,
                                             w->partial2);
        PD_CUDA(cudaGetLastError());
        return PD_OK;
    }
    const bool fuse = !(g->broken_total > 0 && !g->has_E) && !g->sc;
    // The inner FP32 products: the difference form in 2D (fewer iterations for 25 % more
    // stencil work); the pair form in 3D (ALU-bound there; the FP64 refinement corrects its
    // rounding).  Plain FP64 CG: the pair form (its rounding, a few 1e-12 relative at most,
    // is far below the solver's tolerance; the FP64 pipe bounds the product and the pair
    // form executes a fifth fewer FP64 operations than the difference form).
    const uint32_t acc = g->dim == 2 ? PD_ACCURATE : PD_PAIR_FORM;
    const uint32_t fl = (f64 ? PD_F64 | PD_PAIR_FORM : PD_F32 | acc) | PD_PROJECT | kInputProjected;
    void *p = f64 ? (void *)w->p64 : (void *)w->p32;
    void *q = f64 ? (void *)w->q64 : (void *)w->q32;
    int rc;
    if (fuse) {
        rc = matvec(g, 1, p, q, fl, s, w->partial, &w->sc->pq, &w->sc->retire[2]);
    } else {
        rc = matvec(g, 1, p, q, fl, s);
        if (rc == PD_OK) {
            if (f64)
                k_dot<double><<<w->red, kBlk, 0, s>>>(w->p64, w->q64, L, L / 2, &w->sc->pq, w->partial2,
                                                     &w->sc->retire[3]);
            else
                k_dot<float><<<w->red, kBlk, 0, s>>>(w->p32, w->q32, L, L / 4, &w->sc->pq, w->partial2,
                                                    &w->sc->retire[3]);
        }
    }
    if (rc) return rc;
    if (f64) {
        const int64_t nv = aligned16(x64) ? L / 2 : 0;
        k_cg_update<double><<<w->red64, kBlk, 0, s>>>(x64, nullptr, w->r64, w->p64, w->q64, L, nv, w->sc,
                                                      w->partial2);
        k_cg_p<double><<<w->red64, kBlk, 0, s>>>(w->p64, w->r64, L, L / 2, w->sc);
    } else {
        k_cg_update<float><<<w->red, kBlk, 0, s>>>(w->x32, w->xlo32, w->r32, w->p32, w->q32, L, L / 4, w->sc,
                                                   w->partial2);
        k_cg_p<float><<<w->red, kBlk, 0, s>>>(w->p32, w->r32, L, L / 4, w->sc);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// Runs inner iterations until the device flag is set or `budget` iterations
// were issued.  Chunks of kChunk iterations run as one captured graph.
int inner_loop(pd_grid *g, CgWs *w, bool f64, double *x64, int budget, cudaStream_t s, int *done_iters,
               bool fused = false)
{
    const int gi = f64 ? 1 : (fused ? 2 : 0);
    if (fused) {
        int rc0 = ensure_tile_flags(g, w, s);
        if (rc0) return rc0;
    }
    // one plain iteration first: sets kernel attributes outside any capture
    int issued = 0;
    int rc = iteration(g, w, f64, x64, s, fused);
    if (rc) return rc;
    ++issued;
    const void *key = x64;
    if (!w->graph[gi] || w->graph_key[gi] != key || w->graph_stamp[gi] != g->op_stamp) {
        if (w->graph[gi]) {
            cudaGraphExecDestroy(w->graph[gi]);
            w->graph[gi] = nullptr;
        }
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            for (int i = 0; i < kChunk && ok; ++i) ok = (iteration(g, w, f64, x64, w->cap, fused) == PD_OK);
            ok = (cudaStreamEndCapture(w->cap, &graph) == cudaSuccess) && ok;
        }
        if (ok && cudaGraphInstantiate(&w->graph[gi], graph, 0) != cudaSuccess) {
            w->graph[gi] = nullptr;
            ok = false;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        w->graph_key[gi] = key;
        w->graph_stamp[gi] = g->op_stamp;
    }
    volatile CgScal *hs = (volatile CgScal *)g->h_pinned;
    while (issued < budget) {
        const int n = std::min(kChunk, budget - issued);
        if (w->graph[gi] && n == kChunk) {
            PD_CUDA(cudaGraphLaunch(w->graph[gi], s));
        } else {
            for (int i = 0; i < n; ++i) {
                rc = iteration(g, w, f64, x64, s, fused);
                if (rc) return rc;
            }
        }
        issued += n;
        PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(CgScal), cudaMemcpyDeviceToHost, s));
        PD_CUDA(cudaStreamSynchronize(s));
        if (hs->done) break;
    }
    PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(CgScal), cudaMemcpyDeviceToHost, s));
    volatile int *herr = (volatile int *)((char *)g->h_pinned + 2048);
    PD_CUDA(cudaMemcpyAsync((void *)herr, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    if (*herr) {   // a kernel gave up a bounded wait: its reductions may not have retired
        PD_CUDA(cudaMemsetAsync(w->sc, 0, sizeof(CgScal), s));
        return fail(PD_ERR_TIMEOUT, "CG: a device wait gave up (error word set)");
    }
    *done_iters = hs->iters;
    return hs->done ? PD_OK : PD_ERR_NOT_CONVERGED;
}

// The FP32 inner loop as persistent cooperative launches (pd_cg_persist.cu):
// one launch runs until convergence or kPersistChunk iterations.
int inner_loop_persist(pd_grid *g, CgWs *w, int budget, cudaStream_t s, int *done_iters)
{
    constexpr int kPersistChunk = 8192;
    if (cg_persist_ctas(g) > 1024 || (size_t)2 * cg_persist_ctas(g) > (size_t)kRedMax + 64)
        return fail(PD_ERR_STATE, "persistent CG: too many CTAs for the partial buffer");
    int rc0 = ensure_tile_flags(g, w, s);
    if (rc0) return rc0;
    const CgVecs v = cg_vecs(w);
    volatile CgScal *hs = (volatile CgScal *)g->h_pinned;
    volatile int *herr = (volatile int *)((char *)g->h_pinned + 2048);
    int issued = 0;
    while (issued < budget) {
        const int n = std::min(kPersistChunk, budget - issued);
        int rc = cg_persist_run(g, v, w->sc, w->gbar, w->partial, w->tile_flags, n, s);
        if (rc) return rc;
        issued += n;
        PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(CgScal), cudaMemcpyDeviceToHost, s));
        PD_CUDA(cudaMemcpyAsync((void *)herr, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PD_CUDA(cudaStreamSynchronize(s));
        if (*herr) {
            PD_CUDA(cudaMemsetAsync(w->sc, 0, sizeof(CgScal), s));
            PD_CUDA(cudaMemsetAsync(w->gbar, 0, sizeof(CgBar), s));
            return fail(PD_ERR_TIMEOUT, "persistent CG: a device wait gave up (error word set)");
        }
        if (hs->done) break;
    }
    *done_iters = hs->iters;
    return hs->done ? PD_OK : PD_ERR_NOT_CONVERGED;
}

// r64 = P(b - K u) with the FP64 operator; returns |r|^2 on the host.
int true_residual(pd_grid *g, CgWs *w, const double *b, const double *u, cudaStream_t s, double *rr)
{
    const int64_t L = (int64_t)g->dim * g->N;
    int rc = matvec(g, 1, u, w->q64, PD_F64 | PD_PROJECT, s);
    if (rc) return rc;
    k_resid<<<w->red, kBlk, 0, s>>>(w->r64, b, w->q64, g->has_cons ? g->d_cons : nullptr, g->N, g->dim,
                                        &w->sc->aux, w->partial2, &w->sc->retire[3]);
    PD_CUDA(cudaGetLastError());
    PD_CUDA(cudaMemcpyAsync(g->h_pinned, &w->sc->aux, sizeof(double), cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    *rr = *(volatile double *)g->h_pinned;
    (void)L;
    return PD_OK;
}

}  // namespace

void cg_release(pd_grid *g)
{
    CgWs *w = (CgWs *)g->cg;
    if (!w) return;
    for (int i = 0; i < 3; ++i)
        if (w->graph[i]) cudaGraphExecDestroy(w->graph[i]);
    if (w->base) cudaFree(w->base);
    if (w->cap) cudaStreamDestroy(w->cap);
    delete w;
    g->cg = nullptr;
}

}  // namespace pd

using namespace pd;

extern "C" int pd_cg_solve(pd_grid *g, const double *b, double *u, double rtol, int max_iter, uint32_t mode,
                           pd_cg_stats *stats, void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!b || !u) return fail(PD_ERR_INVALID, "b and u must be device pointers");
    if (!(rtol > 0) || max_iter < 1) return fail(PD_ERR_INVALID, "rtol > 0 and max_iter >= 1 required");
    const bool graph_only = (mode & PD_CG_GRAPH) != 0;
    mode &= ~(uint32_t)PD_CG_GRAPH;
    if (mode != PD_CG_F64 && mode != PD_CG_MIXED) return fail(PD_ERR_INVALID, "mode must be PD_CG_F64 or PD_CG_MIXED");
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    CgWs *w = nullptr;
    int rc = ensure_ws(g, w);
    if (rc) return rc;
    const int64_t L = (int64_t)g->dim * g->N;
    const int blocks = w->red;
    if (g->has_cons) k_zero_constrained<<<blocks, kBlk, 0, s>>>(u, g->d_cons, g->N, g->dim);

    // |P b|^2
    double bb = 0.0;
    {
        PD_CUDA(cudaMemsetAsync(w->q64, 0, sizeof(double) * L, s));
        k_resid<<<blocks, kBlk, 0, s>>>(w->r64, b, w->q64, g->has_cons ? g->d_cons : nullptr, g->N, g->dim,
                                        &w->sc->aux, w->partial2, &w->sc->retire[3]);
        PD_CUDA(cudaMemcpyAsync(g->h_pinned, &w->sc->aux, sizeof(double), cudaMemcpyDeviceToHost, s));
        PD_CUDA(cudaStreamSynchronize(s));
        bb = *(volatile double *)g->h_pinned;
    }
    const double bnorm = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
    int total_iters = 0, outer = 0, f64mv = 0;
    bool used_persist = false;
    double rel = 0.0;
    int status = PD_ERR_NOT_CONVERGED;

    if (mode == PD_CG_F64) {
        for (int restart = 0; restart < 4; ++restart) {
            double rr;
            rc = true_residual(g, w, b, u, s, &rr);
            if (rc) return rc;
            ++f64mv;
            rel = std::sqrt(rr) / bnorm;
            if (rel <= rtol) { status = PD_OK; break; }
            if (total_iters >= max_iter) break;
            ++outer;
            *(volatile double *)g->h_pinned = rr;
            PD_CUDA(cudaMemcpyAsync(&w->sc->aux, g->h_pinned, sizeof(double), cudaMemcpyHostToDevice, s));
            k_plain_start<<<blocks, kBlk, 0, s>>>(w->p64, w->r64, L, rtol * rtol * bb * 0.25, w->sc);
            int it = 0;
            rc = inner_loop(g, w, true, u, max_iter - total_iters, s, &it);
            total_iters += it;
            f64mv += it;
            if (rc != PD_OK && rc != PD_ERR_NOT_CONVERGED) return rc;
        }
    } else {
        // FP32 CG with reliable updates: whenever the FP32 recursive residual has
        // dropped by kRU since the last update, the FP32 increment is added to u
        // in FP64, the true residual b - K u is formed with the FP64 operator and
        // replaces the FP32 residual; the search direction is kept, so the Krylov
        // history is not lost as it is by a restart.  FP32 vectors are scaled by
        // the initial residual norm s0 so they stay O(1).
        constexpr double kRU = 0.1;
        const bool persist = !graph_only && cg_persist_eligible(g);
        const bool fused = !persist && cg_dirmv_eligible(g);
        used_persist = persist;
        double rr;
        rc = true_residual(g, w, b, u, s, &rr);
        if (rc) return rc;
        ++f64mv;
        rel = std::sqrt(rr) / bnorm;
        const double s0 = std::sqrt(rr) > 0 ? std::sqrt(rr) : 1.0;
        const double tgt2 = (0.5 * rtol * bnorm / s0) * (0.5 * rtol * bnorm / s0);
        if (rel <= rtol) {
            status = PD_OK;
        } else {
            double rr_ref = rr / (s0 * s0);
            k_inner_start<<<blocks, kBlk, 0, s>>>(w->r32, w->p32, w->x32, w->xlo32, w->r64, L, L / 4, 1.0 / s0,
                                                  std::max(kRU * kRU, tgt2 / rr_ref), w->sc, w->partial2);

            for (int phase = 0; phase < 1000; ++phase) {
                ++outer;
                int it = 0;
                rc = persist ? inner_loop_persist(g, w, max_iter - total_iters, s, &it)
                             : inner_loop(g, w, false, nullptr, max_iter - total_iters, s, &it, fused);
                total_iters += it;
                if (rc != PD_OK && rc != PD_ERR_NOT_CONVERGED) return rc;
                k_correct_zero<<<blocks, kBlk, 0, s>>>(u, w->x32, w->xlo32, s0, L, aligned16(u) ? L / 4 : 0);
                PD_CUDA(cudaGetLastError());
                rc = true_residual(g, w, b, u, s, &rr);
                if (rc) return rc;
                ++f64mv;
                rel = std::sqrt(rr) / bnorm;
                if (rel <= rtol) { status = PD_OK; break; }
                if (total_iters >= max_iter || !std::isfinite(rel)) break;
                rr_ref = rr / (s0 * s0);
                k_replace<<<blocks, kBlk, 0, s>>>(w->r32, w->p32, w->r64, L, L / 4, 1.0 / s0,
                                                  std::max(kRU * kRU * rr_ref, tgt2),
                                                  w->sc, w->partial2, (persist || fused) ? 0 : 1);
                PD_CUDA(cudaGetLastError());

            }
        }
    }
    PD_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        stats->iterations = total_iters;
        stats->outer = outer;
        stats->f64_matvecs = f64mv;
        stats->rel_residual = rel;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->persistent = used_persist ? 1 : 0;
    }
    if (status != PD_OK) return fail(PD_ERR_NOT_CONVERGED, "CG reached its iteration cap");
    return PD_OK;
}

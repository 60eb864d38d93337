// pd_adr.cu -- the paper's quasi-static solver: adaptive dynamic relaxation
// with central-difference explicit integration (Sec. 2.3, Algorithm 1, CDEI).
//
// ADR turns K u = b into the damped fictitious dynamics D u'' + c D u' = f + b
// (f = -P K P u, D diagonal) and integrates it with Algorithm 1, dt = 1:
//     v^(1/2)   = D^-1 (f^0 + b) / 2
//     v^(n+1/2) = ((2 - c^n) v^(n-1/2) + 2 D^-1 (f^n + b)) / (2 + c^n)
//     u^(n+1)   = u^n + v^(n+1/2)
// The paper takes D and c from its reference [KM] (Kilic and Madenci):
//   D_i = 1/4 sum_j |K_ij| (Gershgorin; the interior row, the largest, serves
//   every node of a component; with the surface correction, the largest row
//   over the whole grid), and c^n = 2 sqrt(u^T K1 u / u^T u) with the
//   diagonal local stiffness K1_ii = -(f_i^n - f_i^(n-1)) / (D_i v_i^(n-1/2))
//   (0 where v_i = 0), c^n = 0 when the quotient is not positive.
// The iteration stops when |f^n + b| <= rtol |b| at u^n, before the update.
//
// Per iteration: the FP64 operator (any method of pd_matvec, with D^f for
// broken bonds), one reduction kernel (r.r, u^T K1 u, u^T u; its last block
// forms c and the convergence flag) and one update kernel; chunks of 32
// iterations replay as one CUDA graph and the host reads the flag between
// chunks.  The two force buffers swap roles every iteration (the product of
// one iteration is the previous force of the next), so nothing is copied; a
// chunk has an even number of iterations, so every replay starts on the same
// buffer.  Everything is FP64, as in the oracle; the update multiplies by the
// reciprocals of D and 2 + c instead of dividing element by element.
//
// PD_ADR_MIXED runs the same iteration on FP32 vectors with an FP64 base point
// that is refreshed at every tenfold drop of the residual (the "mixed
// precision" section below says how it keeps the FP64 iteration count).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>

#include "pd_internal.cuh"
#include "pd_reduce.cuh"

namespace pd {

namespace {

constexpr int kBlk = 256;
constexpr int kChunk = 32;

struct AdrScal {
    double rr;       // |f^n + b|^2 at the current iterate
    double num;      // u^T K1 u
    double den;      // u^T u
    double c;        // damping of the next update
    double tol2;     // stop when rr <= tol2
    int done;
    int iters;       // updates applied
    unsigned int retire;
};

struct AdrWs {
    size_t bytes = 0;
    void *base = nullptr;
    double *q[2], *v, *pb;        // P K P u at two consecutive iterates (alternating), velocity, P b
    AdrScal *sc;
    double *partial;              // [3][blocks]
    int blocks = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    const void *key = nullptr;
    int64_t stamp = -1;
    // mixed mode: FP32 correction d = u - u_base, velocity, K d at two iterates, base residual,
    // FP32 copy of the base (for the damping quotient only)
    size_t mbytes = 0;
    void *mbase = nullptr;
    float *d32, *dlo32, *v32, *q32, *w32, *rb32, *ub32;
    cudaGraphExec_t mgraph = nullptr;
    int64_t mstamp = -1;
};

struct Dens {
    double d[3];
    // component c without a dynamically indexed copy of the kernel parameter in local memory
    __host__ __device__ double at(int c) const { return c == 0 ? d[0] : (c == 1 ? d[1] : d[2]); }
};

__device__ __forceinline__ bool last_block(unsigned int *retire)
{
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(retire, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    return s_last;
}

// pb = P b and r.r at u^0 (q = P K P u^0 already).
__global__ void __launch_bounds__(kBlk)
k_adr_resid0(double *pb, const double *__restrict__ b, const double *__restrict__ q, const uint8_t *__restrict__ cons,
             int64_t N, int dim, AdrScal *sc, double *partial)
{
    __shared__ double red[kBlk / 32];
    double acc = 0.0;
    for (int c = 0; c < dim; ++c)
        for (int64_t p = (int64_t)blockIdx.x * kBlk + threadIdx.x; p < N; p += (int64_t)gridDim.x * kBlk) {
            const int64_t i = c * N + p;
            const bool fixed = cons && ((cons[p] >> c) & 1);
            const double bi = fixed ? 0.0 : b[i];
            pb[i] = bi;
            const double r = bi - q[i];
            acc += r * r;
        }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
    if (last_block(&sc->retire)) {
        double t = 0.0;
        for (int i = threadIdx.x; i < gridDim.x; i += kBlk) t += __ldcg(partial + i);
        t = block_sum(t, red);
        if (threadIdx.x == 0) {
            sc->rr = t;
            sc->retire = 0u;
        }
    }
}

// First half step: v = (f^0 + b) / (2 D), u += v.
__global__ void __launch_bounds__(kBlk)
k_adr_first(double *u, double *v, const double *__restrict__ q, const double *__restrict__ pb, int64_t N, int dim,
            Dens D)
{
    for (int c = 0; c < dim; ++c)
        for (int64_t p = (int64_t)blockIdx.x * kBlk + threadIdx.x; p < N; p += (int64_t)gridDim.x * kBlk) {
            const int64_t i = c * N + p;
            const double vi = (pb[i] - q[i]) / D.at(c) / 2.0;
            v[i] = vi;
            u[i] += vi;
        }
}

// r.r, u^T K1 u and u^T u at u^n; the last block forms c^n and the stop flag.
__global__ void __launch_bounds__(kBlk)
k_adr_reduce(const double *__restrict__ u, const double *__restrict__ v, const double *__restrict__ q,
             const double *__restrict__ q_old, const double *__restrict__ pb, int64_t N, int dim, Dens D, AdrScal *sc,
             double *partial)
{
    __shared__ double red[kBlk / 32];
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = sc->done;
    __syncthreads();
    if (s_done) return;
    double a_rr = 0.0, a_num = 0.0, a_den = 0.0;
    for (int c = 0; c < dim; ++c) {
        const double Dc = D.at(c);
        for (int64_t p = (int64_t)blockIdx.x * kBlk + threadIdx.x; p < N; p += (int64_t)gridDim.x * kBlk) {
            const int64_t i = c * N + p;
            const double qi = q[i];
            const double r = pb[i] - qi;
            a_rr += r * r;
            const double ui = u[i], vi = v[i];
            if (vi != 0.0) a_num += ui * ((qi - q_old[i]) / (Dc * vi)) * ui;   // -(f - f_old) = q - q_old
            a_den += ui * ui;
        }
    }
    const int nb = gridDim.x;
    const double s0 = block_sum(a_rr, red), s1 = block_sum(a_num, red), s2 = block_sum(a_den, red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s0;
        partial[nb + blockIdx.x] = s1;
        partial[2 * nb + blockIdx.x] = s2;
    }
    if (last_block(&sc->retire)) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int i = threadIdx.x; i < nb; i += kBlk) {
            t0 += __ldcg(partial + i);
            t1 += __ldcg(partial + nb + i);
            t2 += __ldcg(partial + 2 * nb + i);
        }
        t0 = block_sum(t0, red);
        t1 = block_sum(t1, red);
        t2 = block_sum(t2, red);
        if (threadIdx.x == 0) {
            sc->rr = t0;
            sc->num = t1;
            sc->den = t2;
            sc->c = (t1 > 0.0 && t2 > 0.0) ? 2.0 * sqrt(t1 / t2) : 0.0;
            if (!(t0 > sc->tol2)) sc->done = 1;   // also stops on NaN
            sc->retire = 0u;
        }
    }
}

// v = ((2 - c) v + 2 (f + b) / D) / (2 + c), u += v.  invD: 1 / D per component.
__global__ void __launch_bounds__(kBlk)
k_adr_update(double *u, double *v, const double *__restrict__ q, const double *__restrict__ pb, int64_t N, int dim,
             Dens invD, AdrScal *sc)
{
    __shared__ int s_done;
    __shared__ double s_c;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_c = sc->c;
        if (blockIdx.x == 0 && !s_done) sc->iters += 1;
    }
    __syncthreads();
    if (s_done) return;
    const double c = s_c, a = 2.0 - c, e = 1.0 / (2.0 + c);
    for (int cc = 0; cc < dim; ++cc) {
        const double g = 2.0 * invD.at(cc);
        for (int64_t p = (int64_t)blockIdx.x * kBlk + threadIdx.x; p < N; p += (int64_t)gridDim.x * kBlk) {
            const int64_t i = cc * N + p;
            const double vi = (a * v[i] + (pb[i] - q[i]) * g) * e;
            v[i] = vi;
            u[i] += vi;
        }
    }
}

__global__ void __launch_bounds__(kBlk)
k_adr_zero_constrained(double *u, const uint8_t *__restrict__ cons, int64_t N, int dim)
{
    for (int64_t p = (int64_t)blockIdx.x * kBlk + threadIdx.x; p < N; p += (int64_t)gridDim.x * kBlk)
        for (int c = 0; c < dim; ++c)
            if ((cons[p] >> c) & 1) u[c * N + p] = 0.0;
}

// ------------------------------------------------------------------ mixed precision
// The same iteration with the operator applied in FP32 to the correction
// d = u - u_base only: the residual is r = r_base - K d, where r_base is the
// FP64 residual at the base point (recomputed whenever the FP32 estimate has
// dropped tenfold).  The product of each iteration is w = K v^(n-1/2), the
// change of K d over the last step, accumulated into q = K d: the damping
// quotient needs exactly that change, and taking it as the difference of two
// FP32 products of d would leave only rounding noise where v is small.  d is
// kept as an unevaluated FP32 sum d + d_lo (compensated summation of the
// steps): otherwise the roundings of d, which K amplifies up to its condition
// number, open a gap between q and K d that on a 1024^2 grid is as large as the
// residual itself.  In exact arithmetic the iterates are those above.  The product is taken
// without projection (the fast interior path of the FP32 stencil);
// constrained components are masked here instead.

// Vector access for the mixed kernels: when N is a multiple of 4 every component
// plane starts on a 16-byte boundary (the workspace vectors are 256-byte
// aligned), so nodes are taken four at a time (float4, and uchar4 of the
// constraint bytes); otherwise one at a time.
template <typename F>
__device__ __forceinline__ void adrm_for_each(int64_t N, int dim, F &&f)
{
    const int64_t t0 = (int64_t)blockIdx.x * kBlk + threadIdx.x, st = (int64_t)gridDim.x * kBlk;
    if ((N & 3) == 0) {
        const int64_t nq = N >> 2;
        for (int c = 0; c < dim; ++c)
            for (int64_t j = t0; j < nq; j += st) f(c, j, true);
    } else {
        for (int c = 0; c < dim; ++c)
            for (int64_t p = t0; p < N; p += st) f(c, p, false);
    }
}

__device__ __forceinline__ float4 ld4(const float *a, int64_t i4) { return reinterpret_cast<const float4 *>(a)[i4]; }
__device__ __forceinline__ void st4(float *a, int64_t i4, float4 v) { reinterpret_cast<float4 *>(a)[i4] = v; }

// r.r (estimated), u^T K1 u, u^T u at iterate n with q^n = q^(n-1) + w, K1_ii = w_i / (D v_i),
// u = u_base + d; the last block forms c and the flag.
__global__ void __launch_bounds__(kBlk)
k_adrm_reduce(const float *__restrict__ d, const float *__restrict__ ub, const float *__restrict__ v,
              const float *__restrict__ q, const float *__restrict__ w, const float *__restrict__ rb,
              const uint8_t *__restrict__ cons, int64_t N, int dim, Dens D, AdrScal *sc, double *partial)
{
    __shared__ double red[kBlk / 32];
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = sc->done;
    __syncthreads();
    if (s_done) return;
    // u^T K1 u sums terms of both signs and of very different sizes (small velocities give
    // large quotients) that largely cancel: that sum is compensated (Neumaier: the rounding
    // error of every add is kept in n_lo), the positive ones are plain FP32.  The quotient
    // only steers the damping, so the fast FP32 divide serves.
    float a_rr = 0.f, a_den = 0.f, n_hi = 0.f, n_lo = 0.f;
    auto one = [&](bool fixed, float wi, float qi, float rbi, float ubi, float di, float vi, float Dc) {
        const float r = fixed ? 0.f : rbi - (qi + wi);
        a_rr = __fmaf_rn(r, r, a_rr);
        const float ui = ubi + di;
        // velocities below 1e-30 are taken as zero (keeps the quotient finite in FP32)
        if (!fixed && fabsf(vi) > 1e-30f) {
            const float x = ui * __fdividef(wi, Dc * vi) * ui;
            const float t = n_hi + x;
            n_lo += (fabsf(n_hi) >= fabsf(x)) ? (n_hi - t) + x : (x - t) + n_hi;
            n_hi = t;
        }
        a_den = __fmaf_rn(ui, ui, a_den);
    };
    adrm_for_each(N, dim, [&](int c, int64_t k, bool vec) {
        const float Dc = (float)D.at(c);
        if (vec) {
            const int64_t i4 = c * (N >> 2) + k;
            const float4 w4 = ld4(w, i4), q4 = ld4(q, i4), r4 = ld4(rb, i4), u4 = ld4(ub, i4), d4 = ld4(d, i4),
                         v4 = ld4(v, i4);
            const uchar4 m4 = cons ? reinterpret_cast<const uchar4 *>(cons)[k] : make_uchar4(0, 0, 0, 0);
            one((m4.x >> c) & 1, w4.x, q4.x, r4.x, u4.x, d4.x, v4.x, Dc);
            one((m4.y >> c) & 1, w4.y, q4.y, r4.y, u4.y, d4.y, v4.y, Dc);
            one((m4.z >> c) & 1, w4.z, q4.z, r4.z, u4.z, d4.z, v4.z, Dc);
            one((m4.w >> c) & 1, w4.w, q4.w, r4.w, u4.w, d4.w, v4.w, Dc);
        } else {
            const int64_t i = c * N + k;
            one(cons && ((cons[k] >> c) & 1), w[i], q[i], rb[i], ub[i], d[i], v[i], Dc);
        }
    });
    const int nb = gridDim.x;
    const double s0 = block_sum(a_rr, red), s1 = block_sum((double)n_hi + (double)n_lo, red),
                 s2 = block_sum(a_den, red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s0;
        partial[nb + blockIdx.x] = s1;
        partial[2 * nb + blockIdx.x] = s2;
    }
    if (last_block(&sc->retire)) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int i = threadIdx.x; i < nb; i += kBlk) {
            t0 += __ldcg(partial + i);
            t1 += __ldcg(partial + nb + i);
            t2 += __ldcg(partial + 2 * nb + i);
        }
        t0 = block_sum(t0, red);
        t1 = block_sum(t1, red);
        t2 = block_sum(t2, red);
        if (threadIdx.x == 0) {
            sc->rr = t0;
            sc->num = t1;
            sc->den = t2;
            sc->c = (t1 > 0.0 && t2 > 0.0 && isfinite(t1)) ? 2.0 * sqrt(t1 / t2) : 0.0;
            if (!(t0 > sc->tol2)) sc->done = 1;
            sc->retire = 0u;
        }
    }
}

// q += w; v = ((2 - c) v + 2 r / D) / (2 + c), d += v (compensated: the rounding
// error of each add goes to d_lo) on free components (constrained ones stay 0).
__global__ void __launch_bounds__(kBlk)
k_adrm_update(float *d, float *dlo, float *v, float *q, const float *__restrict__ w, const float *__restrict__ rb,
              const uint8_t *__restrict__ cons, int64_t N, int dim, Dens invD, AdrScal *sc)
{
    __shared__ int s_done;
    __shared__ double s_c;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_c = sc->c;
        if (blockIdx.x == 0 && !s_done) sc->iters += 1;
    }
    __syncthreads();
    if (s_done) return;
    const float a = (float)(2.0 - s_c), e = (float)(1.0 / (2.0 + s_c));
    // one node: returns false for a constrained component (left untouched: v = d = 0 there)
    auto one = [&](bool fixed, float &qi, float wi, float rbi, float &vi, float &di, float &dli, float g) {
        if (fixed) return;
        qi += wi;
        vi = (a * vi + (rbi - qi) * g) * e;
        const float dh = di, sum = dh + vi, bp = sum - dh;   // two-sum of Knuth
        di = sum;
        dli += (dh - (sum - bp)) + (vi - bp);
    };
    adrm_for_each(N, dim, [&](int cc, int64_t k, bool vec) {
        const float g = (float)(2.0 * invD.at(cc));
        if (vec) {
            const int64_t i4 = cc * (N >> 2) + k;
            const uchar4 m4 = cons ? reinterpret_cast<const uchar4 *>(cons)[k] : make_uchar4(0, 0, 0, 0);
            float4 q4 = ld4(q, i4), v4 = ld4(v, i4), d4 = ld4(d, i4), l4 = ld4(dlo, i4);
            const float4 w4 = ld4(w, i4), r4 = ld4(rb, i4);
            one((m4.x >> cc) & 1, q4.x, w4.x, r4.x, v4.x, d4.x, l4.x, g);
            one((m4.y >> cc) & 1, q4.y, w4.y, r4.y, v4.y, d4.y, l4.y, g);
            one((m4.z >> cc) & 1, q4.z, w4.z, r4.z, v4.z, d4.z, l4.z, g);
            one((m4.w >> cc) & 1, q4.w, w4.w, r4.w, v4.w, d4.w, l4.w, g);
            st4(q, i4, q4);
            st4(v, i4, v4);
            st4(d, i4, d4);
            st4(dlo, i4, l4);
        } else {
            const int64_t i = cc * N + k;
            one(cons && ((cons[k] >> cc) & 1), q[i], w[i], rb[i], v[i], d[i], dlo[i], g);
        }
    });
}

// First half step from the base: v = r_base / (2 D), d = v, and the FP32 copy of the base.
__global__ void __launch_bounds__(kBlk)
k_adrm_first(float *d, float *dlo, float *v, float *ub, const float *__restrict__ rb, const double *__restrict__ u,
             int64_t N, int dim, Dens invD)
{
    for (int c = 0; c < dim; ++c) {
        const float g = (float)(0.5 * invD.at(c));
        for (int64_t p = (int64_t)blockIdx.x * kBlk + threadIdx.x; p < N; p += (int64_t)gridDim.x * kBlk) {
            const int64_t i = c * N + p;
            const float vi = rb[i] * g;
            v[i] = vi;
            d[i] = vi;
            dlo[i] = 0.f;
            ub[i] = (float)u[i];
        }
    }
}

// u_base += d + d_lo in FP64, d = 0, refresh the FP32 copy of the base.
__global__ void __launch_bounds__(kBlk)
k_adrm_fold(double *u, float *d, float *dlo, float *ub, int64_t L)
{
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < L; i += (int64_t)gridDim.x * kBlk) {
        const double ui = u[i] + ((double)d[i] + (double)dlo[i]);
        u[i] = ui;
        d[i] = 0.f;
        dlo[i] = 0.f;
        ub[i] = (float)ui;
    }
}

// r_base = P b - P K P u (FP64 product already in q); its FP32 copy and |r|^2 (FP64).
__global__ void __launch_bounds__(kBlk)
k_adrm_true(float *rb, const double *__restrict__ pb, const double *__restrict__ q, int64_t L, AdrScal *sc,
            double *partial)
{
    __shared__ double red[kBlk / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < L; i += (int64_t)gridDim.x * kBlk) {
        const double r = pb[i] - q[i];
        rb[i] = (float)r;
        acc += r * r;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
    if (last_block(&sc->retire)) {
        double t = 0.0;
        for (int i = threadIdx.x; i < gridDim.x; i += kBlk) t += __ldcg(partial + i);
        t = block_sum(t, red);
        if (threadIdx.x == 0) {
            sc->rr = t;
            sc->retire = 0u;
        }
    }
}

int ensure_ws(pd_grid *g, AdrWs *&w)
{
    const int64_t L = (int64_t)g->dim * g->N;
    w = (AdrWs *)g->adr;
    if (!w) {
        w = new AdrWs();
        g->adr = w;
        PD_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
        int dev = 0, sms = 0;
        PD_CUDA(cudaGetDevice(&dev));
        PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        w->blocks = std::max(1, sms) * 4;
    }
    const size_t need = sizeof(double) * (4 * (size_t)L + 3 * (size_t)w->blocks) + sizeof(AdrScal) + 2048;
    if (w->bytes >= need) return PD_OK;
    if (w->graph) {
        cudaGraphExecDestroy(w->graph);
        w->graph = nullptr;
    }
    if (w->base) cudaFree(w->base);
    w->base = nullptr;
    w->bytes = 0;
    if (cudaMalloc(&w->base, need) != cudaSuccess) return fail(PD_ERR_OOM, "ADR workspace");
    w->bytes = need;
    char *c = (char *)w->base;
    auto take = [&](size_t n) { char *p = c; c += (n + 255) & ~(size_t)255; return p; };
    w->q[0] = (double *)take(sizeof(double) * L);
    w->q[1] = (double *)take(sizeof(double) * L);
    w->v = (double *)take(sizeof(double) * L);
    w->pb = (double *)take(sizeof(double) * L);
    w->partial = (double *)take(sizeof(double) * 3 * w->blocks);
    w->sc = (AdrScal *)take(sizeof(AdrScal));
    PD_CUDA(cudaMemset(w->sc, 0, sizeof(AdrScal)));
    return PD_OK;
}

// The density of [KM]: 1/4 of the absolute row sum of K for an interior node.
Dens density(const pd_grid *g)
{
    const int nc = g->dim == 2 ? 3 : 6;
    // index of the (a, b) entry in a coefficient row
    auto idx = [&](int a, int b) {
        if (g->dim == 2) {
            static const int m2[2][2] = {{0, 1}, {1, 2}};
            return m2[a][b];
        }
        static const int m3[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
        return m3[a][b];
    };
    Dens D{};
    for (int a = 0; a < g->dim; ++a) {
        double s = 0.0;
        for (int b = 0; b < g->dim; ++b) {
            double tot = 0.0, abs_sum = 0.0;
            for (int k = 0; k < g->nnb; ++k) {
                const double c = g->coef1[(size_t)k * nc + idx(a, b)] * g->E;
                tot += c;
                abs_sum += std::fabs(c);
            }
            s += std::fabs(tot) + abs_sum;
        }
        D.d[a] = 0.25 * s;
    }
    return D;
}

Dens recip(const Dens &D)
{
    Dens r{};
    for (int c = 0; c < 3; ++c) r.d[c] = D.d[c] != 0.0 ? 1.0 / D.d[c] : 0.0;
    return r;
}

// One iteration on the force buffer `cur` (the other holds the previous force).
// The FP64 product takes the pair form: its rounding (a few 1e-12 relative at most)
// is far below the solver's tolerance, and the FP64 pipe bounds the product.
int adr_iteration(pd_grid *g, AdrWs *w, double *u, const Dens &D, int cur, cudaStream_t s)
{
    double *q = w->q[cur], *q_old = w->q[cur ^ 1];
    int rc = matvec(g, 1, u, q, PD_F64 | PD_PAIR_FORM | PD_PROJECT | kInputProjected, s);
    if (rc) return rc;
    k_adr_reduce<<<w->blocks, kBlk, 0, s>>>(u, w->v, q, q_old, w->pb, g->N, g->dim, D, w->sc, w->partial);
    k_adr_update<<<w->blocks, kBlk, 0, s>>>(u, w->v, q, w->pb, g->N, g->dim, recip(D), w->sc);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int ensure_mixed(pd_grid *g, AdrWs *w)
{
    const size_t L = (size_t)g->dim * g->N;
    const size_t need = sizeof(float) * 7 * ((L + 63) & ~(size_t)63) + 1024;
    if (w->mbytes >= need) return PD_OK;
    if (w->mgraph) {
        cudaGraphExecDestroy(w->mgraph);
        w->mgraph = nullptr;
    }
    if (w->mbase) cudaFree(w->mbase);
    w->mbase = nullptr;
    w->mbytes = 0;
    if (cudaMalloc(&w->mbase, need) != cudaSuccess) return fail(PD_ERR_OOM, "ADR mixed workspace");
    w->mbytes = need;
    float *c = (float *)w->mbase;
    const size_t st = (L + 63) & ~(size_t)63;   // 256-byte aligned vectors (TMA needs 16)
    w->d32 = c;
    w->v32 = c + st;
    w->q32 = c + 2 * st;
    w->w32 = c + 3 * st;
    w->rb32 = c + 4 * st;
    w->ub32 = c + 5 * st;
    w->dlo32 = c + 6 * st;
    return PD_OK;
}

int adrm_iteration(pd_grid *g, AdrWs *w, const Dens &D, const Dens &invD, cudaStream_t s)
{
    const uint8_t *cons = g->has_cons ? g->d_cons : nullptr;
    int rc = matvec(g, 1, w->v32, w->w32, PD_F32 | PD_ACCURATE | kInputProjected, s);
    if (rc) return rc;
    k_adrm_reduce<<<w->blocks, kBlk, 0, s>>>(w->d32, w->ub32, w->v32, w->q32, w->w32, w->rb32, cons, g->N, g->dim,
                                             D, w->sc, w->partial);
    k_adrm_update<<<w->blocks, kBlk, 0, s>>>(w->d32, w->dlo32, w->v32, w->q32, w->w32, w->rb32, cons, g->N, g->dim,
                                             invD, w->sc);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace

void adr_release(pd_grid *g)
{
    AdrWs *w = (AdrWs *)g->adr;
    if (!w) return;
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->mgraph) cudaGraphExecDestroy(w->mgraph);
    if (w->mbase) cudaFree(w->mbase);
    if (w->base) cudaFree(w->base);
    if (w->cap) cudaStreamDestroy(w->cap);
    delete w;
    g->adr = nullptr;
}

}  // namespace pd

using namespace pd;

extern "C" int pd_adr_solve(pd_grid *g, const double *b, double *u, double rtol, int max_iter, uint32_t mode,
                            pd_cg_stats *stats, void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!b || !u) return fail(PD_ERR_INVALID, "b and u must be device pointers");
    if (!(rtol > 0) || max_iter < 1) return fail(PD_ERR_INVALID, "rtol > 0 and max_iter >= 1 required");
    if (mode != PD_ADR_F64 && mode != PD_ADR_MIXED) return fail(PD_ERR_INVALID, "mode must be PD_ADR_F64 or PD_ADR_MIXED");
    if (g->has_E) return fail(PD_ERR_INVALID, "ADR needs a constant modulus (no modulus field)");
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    AdrWs *w = nullptr;
    int rc = ensure_ws(g, w);
    if (rc) return rc;
    Dens D = density(g);
    if (g->sc) {   // corrected edge rows can outweigh the interior row: take the maximum over all rows
        double rm[3];
        rc = surface_row_abs_max(g, rm, s);
        if (rc) return rc;
        const bool interior = g->band_n < g->N;   // some row with a full, uncorrected horizon
        for (int c = 0; c < g->dim; ++c) D.d[c] = std::max(0.25 * rm[c], interior ? D.d[c] : 0.0);
    }
    const int blocks = w->blocks;
    if (g->has_cons) k_adr_zero_constrained<<<blocks, kBlk, 0, s>>>(u, g->d_cons, g->N, g->dim);
    // |P b|^2, and the residual at u^0
    volatile AdrScal *hs = (volatile AdrScal *)g->h_pinned;
    PD_CUDA(cudaMemsetAsync(w->q[0], 0, sizeof(double) * (size_t)g->dim * g->N, s));
    PD_CUDA(cudaMemsetAsync(w->sc, 0, sizeof(AdrScal), s));
    k_adr_resid0<<<blocks, kBlk, 0, s>>>(w->pb, b, w->q[0], g->has_cons ? g->d_cons : nullptr, g->N, g->dim, w->sc,
                                         w->partial);
    PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(AdrScal), cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    const double bb = hs->rr;
    const double bn = bb > 0 ? std::sqrt(bb) : 1.0;
    rc = matvec(g, 1, u, w->q[0], PD_F64 | PD_PROJECT | kInputProjected, s);
    if (rc) return rc;
    k_adr_resid0<<<blocks, kBlk, 0, s>>>(w->pb, b, w->q[0], g->has_cons ? g->d_cons : nullptr, g->N, g->dim, w->sc,
                                         w->partial);
    PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(AdrScal), cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    double rel = std::sqrt(hs->rr) / bn;
    int iters = 0, outer = 0, f64mv = 1;
    int status = PD_ERR_NOT_CONVERGED;
    if (rel <= rtol) {
        status = PD_OK;
    } else if (mode == PD_ADR_MIXED) {
        rc = ensure_mixed(g, w);
        if (rc) return rc;
        const Dens invD = recip(D);
        const int64_t L = (int64_t)g->dim * g->N;
        constexpr double kRU = 0.1;   // new FP64 base residual once the estimate has dropped tenfold
        const double floor2 = (0.5 * rtol * bn) * (0.5 * rtol * bn);
        k_adrm_true<<<blocks, kBlk, 0, s>>>(w->rb32, w->pb, w->q[0], L, w->sc, w->partial);
        k_adrm_first<<<blocks, kBlk, 0, s>>>(w->d32, w->dlo32, w->v32, w->ub32, w->rb32, u, g->N, g->dim,
                                                 invD);
        // K d^0 = 0: the first product K v^(1/2) then gives K d^1
        PD_CUDA(cudaMemsetAsync(w->q32, 0, sizeof(float) * (size_t)L, s));
        PD_CUDA(cudaGetLastError());
        double rr_b = hs->rr;
        AdrScal init{};
        init.iters = 1;
        init.tol2 = std::max(kRU * kRU * rr_b, floor2);
        *(AdrScal *)g->h_pinned = init;
        PD_CUDA(cudaMemcpyAsync(w->sc, g->h_pinned, sizeof(AdrScal), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaStreamSynchronize(s));
        if (!w->mgraph || w->mstamp != g->op_stamp) {   // chunks touch only the workspace
            if (w->mgraph) {
                cudaGraphExecDestroy(w->mgraph);
                w->mgraph = nullptr;
            }
            rc = adrm_iteration(g, w, D, invD, s);   // first use outside any capture (kernel attributes)
            if (rc) return rc;
            PD_CUDA(cudaMemsetAsync(w->q32, 0, sizeof(float) * (size_t)L, s));
            *(AdrScal *)g->h_pinned = init;
            PD_CUDA(cudaMemcpyAsync(w->sc, g->h_pinned, sizeof(AdrScal), cudaMemcpyHostToDevice, s));
            k_adrm_first<<<blocks, kBlk, 0, s>>>(w->d32, w->dlo32, w->v32, w->ub32, w->rb32, u, g->N, g->dim,
                                                 invD);
            PD_CUDA(cudaStreamSynchronize(s));
            cudaGraph_t graph = nullptr;
            bool ok = cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                for (int i = 0; i < kChunk && ok; ++i) ok = (adrm_iteration(g, w, D, invD, w->cap) == PD_OK);
                ok = (cudaStreamEndCapture(w->cap, &graph) == cudaSuccess) && ok;
            }
            if (ok && cudaGraphInstantiate(&w->mgraph, graph, 0) != cudaSuccess) w->mgraph = nullptr;
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            w->mstamp = g->op_stamp;
        }
        int dev_iters = 1;
        for (;;) {
            // one phase: FP32 iterations until the estimate reaches its target or the cap
            bool done = false;
            while (!done && dev_iters < max_iter) {
                const int n = std::min(kChunk, max_iter - dev_iters);   // at most one update per iteration
                if (w->mgraph && n == kChunk) {
                    PD_CUDA(cudaGraphLaunch(w->mgraph, s));
                } else {
                    for (int i = 0; i < n; ++i) {
                        rc = adrm_iteration(g, w, D, invD, s);
                        if (rc) return rc;
                    }
                }
                PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(AdrScal), cudaMemcpyDeviceToHost, s));
                PD_CUDA(cudaStreamSynchronize(s));
                done = hs->done != 0;
                dev_iters = hs->iters;
            }
            ++outer;
            // fold the correction into the FP64 base and take the true residual there
            k_adrm_fold<<<blocks, kBlk, 0, s>>>(u, w->d32, w->dlo32, w->ub32, L);
            rc = matvec(g, 1, u, w->q[0], PD_F64 | PD_PROJECT | kInputProjected, s);
            if (rc) return rc;
            k_adrm_true<<<blocks, kBlk, 0, s>>>(w->rb32, w->pb, w->q[0], L, w->sc, w->partial);
            PD_CUDA(cudaGetLastError());
            PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(AdrScal), cudaMemcpyDeviceToHost, s));
            PD_CUDA(cudaStreamSynchronize(s));
            ++f64mv;
            rr_b = hs->rr;
            rel = std::sqrt(rr_b) / bn;
            if (rel <= rtol) {
                status = PD_OK;
                break;
            }
            if (dev_iters >= max_iter || !std::isfinite(rel)) break;
            // in the new base the previous iterate sits at d = -v: q = K d there is -K v, so that the
            // next product K v brings q to K d = 0 at the base
            rc = matvec(g, 1, w->v32, w->q32, PD_F32 | PD_ACCURATE | kInputProjected, s, nullptr, nullptr, nullptr,
                        -1.0);
            if (rc) return rc;
            AdrScal next{};
            next.iters = dev_iters;
            next.tol2 = std::max(kRU * kRU * rr_b, floor2);
            next.rr = rr_b;
            *(AdrScal *)g->h_pinned = next;
            PD_CUDA(cudaMemcpyAsync(w->sc, g->h_pinned, sizeof(AdrScal), cudaMemcpyHostToDevice, s));
            PD_CUDA(cudaStreamSynchronize(s));
        }
        iters = dev_iters;
    } else {
        k_adr_first<<<blocks, kBlk, 0, s>>>(u, w->v, w->q[0], w->pb, g->N, g->dim, D);
        AdrScal init{};
        init.tol2 = rtol * rtol * bb;
        init.iters = 1;
        *(AdrScal *)g->h_pinned = init;
        PD_CUDA(cudaMemcpyAsync(w->sc, g->h_pinned, sizeof(AdrScal), cudaMemcpyHostToDevice, s));
        // one plain iteration (kernel attributes outside any capture), then graph chunks
        // the force of u^0 sits in q[0]; iteration k writes q[k & 1]
        int issued = 0;
        if (max_iter > 1) {
            rc = adr_iteration(g, w, u, D, 1, s);
            if (rc) return rc;
            ++issued;
        }
        if (!w->graph || w->key != u || w->stamp != g->op_stamp) {
            if (w->graph) {
                cudaGraphExecDestroy(w->graph);
                w->graph = nullptr;
            }
            cudaGraph_t graph = nullptr;
            bool ok = cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                for (int i = 0; i < kChunk && ok; ++i) ok = (adr_iteration(g, w, u, D, i & 1, w->cap) == PD_OK);
                ok = (cudaStreamEndCapture(w->cap, &graph) == cudaSuccess) && ok;
            }
            if (ok && cudaGraphInstantiate(&w->graph, graph, 0) != cudaSuccess) w->graph = nullptr;
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            w->key = u;
            w->stamp = g->op_stamp;
        }
        // the iteration that reaches max_iter updates only when it is below the cap
        const int budget = max_iter - 1;
        while (issued < budget) {
            const int n = std::min(kChunk, budget - issued);
            if (w->graph && n == kChunk) {
                PD_CUDA(cudaGraphLaunch(w->graph, s));
            } else {
                for (int i = 0; i < n; ++i) {
                    rc = adr_iteration(g, w, u, D, i & 1, s);
                    if (rc) return rc;
                }
            }
            issued += n;
            PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(AdrScal), cudaMemcpyDeviceToHost, s));
            PD_CUDA(cudaStreamSynchronize(s));
            if (hs->done) break;
        }
        PD_CUDA(cudaMemcpyAsync((void *)hs, w->sc, sizeof(AdrScal), cudaMemcpyDeviceToHost, s));
        PD_CUDA(cudaStreamSynchronize(s));
        iters = hs->iters;
        rel = std::sqrt(hs->rr) / bn;
        if (hs->done) status = PD_OK;
    }
    if (mode == PD_ADR_F64) f64mv = iters + 1;
    if (stats) {
        stats->iterations = iters;
        stats->outer = outer;
        stats->f64_matvecs = f64mv;
        stats->rel_residual = rel;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->persistent = 0;
    }
    if (status != PD_OK) return fail(PD_ERR_NOT_CONVERGED, "ADR reached its iteration cap");
    return PD_OK;
}

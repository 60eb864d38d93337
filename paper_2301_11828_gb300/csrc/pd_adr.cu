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
};

struct Dens {
    double d[3];
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
    const int64_t L = (int64_t)dim * N;
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < L; i += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(i / N);
        const bool fixed = cons && ((cons[i - c * N] >> c) & 1);
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
    const int64_t L = (int64_t)dim * N;
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < L; i += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(i / N);
        const double vi = (pb[i] - q[i]) / D.d[c] / 2.0;
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
    const int64_t L = (int64_t)dim * N;
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < L; i += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(i / N);
        const double r = pb[i] - q[i];
        a_rr += r * r;
        const double ui = u[i], vi = v[i];
        if (vi != 0.0) a_num += ui * ((q[i] - q_old[i]) / (D.d[c] * vi)) * ui;   // -(f - f_old) = q - q_old
        a_den += ui * ui;
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
    const int64_t L = (int64_t)dim * N;
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < L; i += (int64_t)gridDim.x * kBlk) {
        const int cc = (int)(i / N);
        const double vi = (a * v[i] + 2.0 * (pb[i] - q[i]) * invD.d[cc]) * e;
        v[i] = vi;
        u[i] += vi;
    }
}

__global__ void __launch_bounds__(kBlk)
k_adr_zero_constrained(double *u, const uint8_t *__restrict__ cons, int64_t N, int dim)
{
    for (int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x; i < (int64_t)dim * N; i += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(i / N);
        if ((cons[i - c * N] >> c) & 1) u[i] = 0.0;
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
int adr_iteration(pd_grid *g, AdrWs *w, double *u, const Dens &D, int cur, cudaStream_t s)
{
    double *q = w->q[cur], *q_old = w->q[cur ^ 1];
    int rc = matvec(g, 1, u, q, PD_F64 | PD_PROJECT | kInputProjected, s);
    if (rc) return rc;
    k_adr_reduce<<<w->blocks, kBlk, 0, s>>>(u, w->v, q, q_old, w->pb, g->N, g->dim, D, w->sc, w->partial);
    k_adr_update<<<w->blocks, kBlk, 0, s>>>(u, w->v, q, w->pb, g->N, g->dim, recip(D), w->sc);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace

void adr_release(pd_grid *g)
{
    AdrWs *w = (AdrWs *)g->adr;
    if (!w) return;
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->base) cudaFree(w->base);
    if (w->cap) cudaStreamDestroy(w->cap);
    delete w;
    g->adr = nullptr;
}

}  // namespace pd

using namespace pd;

extern "C" int pd_adr_solve(pd_grid *g, const double *b, double *u, double rtol, int max_iter, pd_cg_stats *stats,
                            void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!b || !u) return fail(PD_ERR_INVALID, "b and u must be device pointers");
    if (!(rtol > 0) || max_iter < 1) return fail(PD_ERR_INVALID, "rtol > 0 and max_iter >= 1 required");
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
    int iters = 0;
    int status = PD_ERR_NOT_CONVERGED;
    if (rel <= rtol) {
        status = PD_OK;
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
    if (stats) {
        stats->iterations = iters;
        stats->outer = 0;
        stats->f64_matvecs = iters + 1;
        stats->rel_residual = rel;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->persistent = 0;
    }
    if (status != PD_OK) return fail(PD_ERR_NOT_CONVERGED, "ADR reached its iteration cap");
    return PD_OK;
}

// pd_adjoint.cu -- reverse-mode sweep through velocity-Verlet segments
// (Algorithm 2 with a = (f + b)/rho, f = A(mu, E) u), for gradients of a loss of
// the final state with respect to the per-node modulus field.
//
// One forward step n -> n+1 (free components; constrained ones move with the
// prescribed velocity and do not depend on v or a):
//   F1  u_{n+1} = u_n + dt v_n + dt^2/2 a_n
//   F2  a_{n+1} = (A_{n+1} u_{n+1} + b) / rho       (A_{n+1} with the bond state mu_{n+1})
//   F3  v_{n+1} = v_n + dt/2 (a_n + a_{n+1})
// Reverse (adjoints ub, vb, ab of u_{n+1}, v_{n+1}, a_{n+1}):
//   F3: ab += dt/2 vb; ab_n = dt/2 vb; vb_n = vb                  (free components)
//   F2: ub += A_{n+1} ab / rho (A symmetric);
//       dL/dE_r += -1/(2 rho) sum_q (ab_q - ab_r)^T C1 (u_q - u_r)  (bond modulus (E_p + E_q)/2)
//   F1: vb_n += dt ub; ab_n += dt^2/2 ub                            (free components); ub_n = ub
// Constrained components of a are never used, so their adjoints are zero.
// Bond breaking is not differentiable: the sweep replays the bond state of every
// step from the mask at the start of the run and the recorded break steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "pd_internal.cuh"

namespace pd {
namespace {

constexpr int kBlk = 256;

int blocks_for(int64_t work)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + kBlk - 1) / kBlk, 152 * 16));
}

// mask_s = mask0 with every bond cleared whose recorded break step is in [1, s].
__global__ void __launch_bounds__(kBlk)
k_mask_at(uint32_t *out, const uint32_t *__restrict__ mask0, const int32_t *__restrict__ bstep, int64_t N, int nnb,
          int W, int32_t s)
{
    for (int64_t t = (int64_t)blockIdx.x * kBlk + threadIdx.x; t < (int64_t)W * N; t += (int64_t)gridDim.x * kBlk) {
        const int w = (int)(t / N);
        const int64_t p = t - (int64_t)w * N;
        uint32_t m = mask0[t];
        const int k0 = 32 * w, k1 = min(nnb, k0 + 32);
        for (int k = k0; k < k1; ++k) {
            const int32_t b = bstep[p * nnb + k];
            if (b > 0 && b <= s) m &= ~(1u << (k - k0));
        }
        out[t] = m;
    }
}

__global__ void __launch_bounds__(kBlk)
k_drift(double *u, const double *__restrict__ v, const double *__restrict__ a, const double *__restrict__ vp,
        const uint8_t *__restrict__ cons, int64_t N, int dim, double dt)
{
    const double h2 = 0.5 * dt * dt;
    for (int64_t t = (int64_t)blockIdx.x * kBlk + threadIdx.x; t < dim * N; t += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(t / N);
        const bool fixed = cons && ((cons[t - c * N] >> c) & 1);
        if (fixed) u[t] += dt * (vp ? vp[t] : 0.0);
        else u[t] += dt * v[t] + h2 * a[t];
    }
}

__global__ void __launch_bounds__(kBlk)
k_kick(double *v, double *a, const double *__restrict__ f, const double *__restrict__ b,
       const double *__restrict__ vp, const uint8_t *__restrict__ cons, int64_t N, int dim, double dt, double inv_rho,
       int first)
{
    for (int64_t t = (int64_t)blockIdx.x * kBlk + threadIdx.x; t < dim * N; t += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(t / N);
        const double an = (f[t] + (b ? b[t] : 0.0)) * inv_rho;
        if (!first) {
            const bool fixed = cons && ((cons[t - c * N] >> c) & 1);
            if (fixed) v[t] = vp ? vp[t] : 0.0;
            else v[t] += 0.5 * dt * (a[t] + an);
        }
        a[t] = an;
    }
}

// F3 reverse: ab += dt/2 vb (free), abn = dt/2 vb (free), vb kept on free / zeroed on constrained,
// ab zeroed on constrained components.
__global__ void __launch_bounds__(kBlk)
k_rev_kick(double *ab, double *abn, double *vb, const uint8_t *__restrict__ cons, int64_t N, int dim, double dt)
{
    for (int64_t t = (int64_t)blockIdx.x * kBlk + threadIdx.x; t < dim * N; t += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(t / N);
        const bool fixed = cons && ((cons[t - c * N] >> c) & 1);
        if (fixed) {
            ab[t] = 0.0;
            abn[t] = 0.0;
            vb[t] = 0.0;
        } else {
            const double hv = 0.5 * dt * vb[t];
            ab[t] += hv;
            abn[t] = hv;
        }
    }
}

// ub += t / rho  (t = A ab)
__global__ void __launch_bounds__(kBlk) k_axpy(double *y, const double *__restrict__ x, double s, int64_t L)
{
    for (int64_t t = (int64_t)blockIdx.x * kBlk + threadIdx.x; t < L; t += (int64_t)gridDim.x * kBlk) y[t] += s * x[t];
}

// F1 reverse: vb += dt ub, ab = abn + dt^2/2 ub (free components).
__global__ void __launch_bounds__(kBlk)
k_rev_drift(double *vb, double *ab, const double *__restrict__ abn, const double *__restrict__ ub,
            const uint8_t *__restrict__ cons, int64_t N, int dim, double dt)
{
    const double h2 = 0.5 * dt * dt;
    for (int64_t t = (int64_t)blockIdx.x * kBlk + threadIdx.x; t < dim * N; t += (int64_t)gridDim.x * kBlk) {
        const int c = (int)(t / N);
        const bool fixed = cons && ((cons[t - c * N] >> c) & 1);
        if (fixed) {
            ab[t] = 0.0;
        } else {
            vb[t] += dt * ub[t];
            ab[t] = abn[t] + h2 * ub[t];
        }
    }
}

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" int pd_step_adjoint(pd_grid *g, const double *u_start, const double *v_start, const double *b, int nsteps,
                               double dt, const double *v_prescribed, const uint32_t *mask0,
                               const int32_t *break_step, int32_t step_base, double *ubar, double *vbar, double *abar,
                               double *grad_E, void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!u_start || !v_start || !mask0 || !break_step || !ubar || !vbar || !abar)
        return fail(PD_ERR_INVALID, "NULL argument");
    if (nsteps < 0 || !(dt > 0) || step_base < 0) return fail(PD_ERR_INVALID, "nsteps >= 0, dt > 0, step_base >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t L = (int64_t)g->dim * g->N;
    const size_t mwords = (size_t)g->W * g->N;
    // workspace: nsteps + 1 displacement states, v, a, f, t, abn, one mask
    const size_t need = sizeof(double) * ((size_t)(nsteps + 1) * L + 5 * (size_t)L) + sizeof(uint32_t) * mwords + 4096;
    // kept by the grid between calls (a checkpointed sweep calls this once per segment)
    if (g->adj_ws_bytes < need) {
        cudaFree(g->adj_ws);
        g->adj_ws = nullptr;
        g->adj_ws_bytes = 0;
        if (cudaMalloc(&g->adj_ws, need) != cudaSuccess) return fail(PD_ERR_OOM, "adjoint workspace");
        g->adj_ws_bytes = need;
    }
    char *ws = (char *)g->adj_ws;
    double *U = (double *)ws;
    double *v = U + (size_t)(nsteps + 1) * L, *a = v + L, *f = a + L, *tv = f + L, *abn = tv + L;
    uint32_t *mk = (uint32_t *)(abn + L);
    uint32_t *saved_mask = g->d_mask;
    const uint8_t *cons = g->has_cons ? g->d_cons : nullptr;
    const int bl = blocks_for(L), blm = blocks_for((int64_t)mwords);
    const double inv_rho = 1.0 / g->rho;
    const uint32_t mflags = PD_F64 | PD_METHOD_STENCIL | kForceMu;
    const int64_t saved_broken = g->broken_total;
    int rc = PD_OK;
    auto use_mask_at = [&](int32_t step) {
        k_mask_at<<<blm, kBlk, 0, s>>>(mk, mask0, break_step, g->N, g->nnb, g->W, step);
        g->d_mask = mk;
    };
    auto bail = [&](int code) {
        g->d_mask = saved_mask;
        g->broken_total = saved_broken;
        return code;
    };
    g->broken_total = 1;   // the replayed masks may hold broken bonds: take the mask-aware paths
    // ---- replay the segment forward, storing u at every step
#define PD_ADJ_CUDA(call)                                                                          \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return bail(fail(PD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
    } while (0)
    PD_ADJ_CUDA(cudaMemcpyAsync(U, u_start, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    PD_ADJ_CUDA(cudaMemcpyAsync(v, v_start, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    use_mask_at(step_base);
    rc = matvec(g, 1, U, f, mflags, s, nullptr, nullptr, nullptr, -1.0);
    if (rc) return bail(rc);
    k_kick<<<bl, kBlk, 0, s>>>(v, a, f, b, v_prescribed, cons, g->N, g->dim, dt, inv_rho, 1);
    for (int st = 0; st < nsteps; ++st) {
        double *un = U + (size_t)(st + 1) * L;
        PD_ADJ_CUDA(cudaMemcpyAsync(un, U + (size_t)st * L, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
        k_drift<<<bl, kBlk, 0, s>>>(un, v, a, v_prescribed, cons, g->N, g->dim, dt);
        use_mask_at(step_base + st + 1);
        rc = matvec(g, 1, un, f, mflags, s, nullptr, nullptr, nullptr, -1.0);
        if (rc) return bail(rc);
        k_kick<<<bl, kBlk, 0, s>>>(v, a, f, b, v_prescribed, cons, g->N, g->dim, dt, inv_rho, 0);
    }
    // ---- reverse sweep
    for (int st = nsteps - 1; st >= 0; --st) {
        const double *un1 = U + (size_t)(st + 1) * L;   // u_{n+1}
        k_rev_kick<<<bl, kBlk, 0, s>>>(abar, abn, vbar, cons, g->N, g->dim, dt);
        use_mask_at(step_base + st + 1);
        rc = matvec(g, 1, abar, tv, mflags, s, nullptr, nullptr, nullptr, -1.0);   // A ab = -K ab
        if (rc) return bail(rc);
        k_axpy<<<bl, kBlk, 0, s>>>(ubar, tv, inv_rho, L);
        if (grad_E) {
            rc = launch_grad_modulus(g, un1, abar, -0.5 * inv_rho, grad_E, s);
            if (rc) return bail(rc);
        }
        k_rev_drift<<<bl, kBlk, 0, s>>>(vbar, abar, abn, ubar, cons, g->N, g->dim, dt);
    }
    if (step_base == 0) {
        // the start of the run: a_0 = (A_0 u_0 + b)/rho also depends on u_0 and E
        use_mask_at(0);
        k_rev_kick<<<bl, kBlk, 0, s>>>(abar, abn, tv, cons, g->N, g->dim, 0.0);   // zero ab on constrained components
        rc = matvec(g, 1, abar, tv, mflags, s, nullptr, nullptr, nullptr, -1.0);
        if (rc) return bail(rc);
        k_axpy<<<bl, kBlk, 0, s>>>(ubar, tv, inv_rho, L);
        if (grad_E) {
            rc = launch_grad_modulus(g, U, abar, -0.5 * inv_rho, grad_E, s);
            if (rc) return bail(rc);
        }
        PD_ADJ_CUDA(cudaMemsetAsync(abar, 0, sizeof(double) * L, s));
    }
    PD_ADJ_CUDA(cudaGetLastError());
    PD_ADJ_CUDA(cudaStreamSynchronize(s));
#undef PD_ADJ_CUDA
    return bail(PD_OK);
}

// pd_crack.cu -- broken bonds and the explicit dynamic loop.
//
//   * D^f gather (Eqs. df, tea:fr): for every node of Omega_br, one warp walks
//     the node's bond mask and removes the terms of its broken bonds from K u:
//         (K u)_p -= scale * sum_{q in v_p} c(q - p) (u_p - u_q).
//     The node list and its length live on the device, so the launch needs no
//     host round trip; an empty list costs one tiny launch.
//   * Breaking (Eqs. mu, fra:s1): one thread per node tests the bonds to nodes
//     with a larger index (offsets of the upper half of the canonical list), in
//     FP64 with explicitly rounded operations (no contraction), and clears the
//     bit at both ends.  Broken bonds never heal.
//   * Pre-notch: bonds whose segment meets a given segment, exact integers (in
//     3D the segment is extruded through z: bonds are tested by their x-y projection).
//   * Velocity-Verlet (Algorithm 2) with a = (f + b) / rho.
//   * Modulus gradient: bond sum of (lam_q - lam_r)^T C1 (u_q - u_r).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>
#include <chrono>
#include <mutex>
#include <string>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kBlk = 256;

__device__ __forceinline__ void node_coords(int64_t p, int nx, int ny, int &i, int &j, int &k)
{
    i = (int)(p % nx);
    j = (int)((p / nx) % ny);
    k = (int)(p / ((int64_t)nx * ny));
}

__device__ __forceinline__ void mark_broken_node(int64_t x, uint32_t *brflag, int32_t *brlist,
                                                 unsigned long long *count)
{
    if (atomicExch(&brflag[x], 1u) == 0u) {
        const unsigned long long idx = atomicAdd(&count[0], 1ull);
        brlist[idx] = (int32_t)x;
    }
}

// ------------------------------------------------------------------ D^f gather
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlk)
k_df_gather(const T *__restrict__ u, T *__restrict__ out, int64_t N, int nx, int ny, int nz, int nnb,
            const int32_t *__restrict__ brlist, const unsigned long long *__restrict__ count,
            const uint32_t *__restrict__ mask, const int32_t *__restrict__ off, const double *__restrict__ coef,
            const uint8_t *__restrict__ cons, int project, double scale, int64_t batch)
{
    const int64_t cnt = (int64_t)*count;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < cnt * batch; w += nwarps) {
        const int64_t b = w / cnt;
        const int64_t p = brlist[w - b * cnt];
        const T *ub = u + b * DIM * N;
        T *ob = out + b * DIM * N;
        int i, j, k;
        node_coords(p, nx, ny, i, j, k);
        const uint8_t cm = project ? cons[p] : 0;
        double up[DIM], acc[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            up[c] = ((cm >> c) & 1) ? 0.0 : (double)ub[c * N + p];
            acc[c] = 0.0;
        }
        for (int kk = lane; kk < nnb; kk += 32) {
            const uint32_t word = mask[(int64_t)(kk >> 5) * N + p];
            if ((word >> (kk & 31)) & 1u) continue;
            const int qi = i + off[3 * kk], qj = j + off[3 * kk + 1], qk = k + off[3 * kk + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            const int64_t q = ((int64_t)qk * ny + qj) * nx + qi;
            const uint8_t qm = project ? cons[q] : 0;
            double d[DIM];
#pragma unroll
            for (int c = 0; c < DIM; ++c) d[c] = up[c] - (((qm >> c) & 1) ? 0.0 : (double)ub[c * N + q]);
            if (DIM == 2) {
                const double *cf = coef + 3 * kk;
                acc[0] += cf[0] * d[0] + cf[1] * d[1];
                acc[1] += cf[1] * d[0] + cf[2] * d[DIM - 1];
            } else {
                const double *cf = coef + 6 * kk;
                acc[0] += cf[0] * d[0] + cf[1] * d[1] + cf[2] * d[DIM - 1];
                acc[1] += cf[1] * d[0] + cf[3] * d[1] + cf[4] * d[DIM - 1];
                acc[DIM - 1] += cf[2] * d[0] + cf[4] * d[1] + cf[5] * d[DIM - 1];
            }
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < DIM; ++c)
                if (!((cm >> c) & 1)) ob[c * N + p] = (T)((double)ob[c * N + p] - scale * acc[c]);
        }
    }
}

// ------------------------------------------------------------------ breaking
// Eq. fra:s1 is evaluated in a fixed operation order, each step rounded once:
//     X_c = xi_c + (u_q,c - u_p,c),  l2 = sum_c X_c X_c,  r2 = sum_c xi_c xi_c,
//     s = (sqrt(l2) - sqrt(r2)) / sqrt(r2),  broken iff s >= s0.
// For a fixed offset, s is a monotone non-decreasing function of l2 (a rounded
// square root, a rounded subtraction of a constant and a rounded division by a
// positive constant all are), so the test is exactly l2 >= T for the smallest
// double T that passes it.  k_break_thr finds T per offset by bisection over
// the bit patterns of the non-negative doubles, with the same rounded
// operations; k_break then needs no square root or division per bond.
// Offsets of the radius-ceil(m) disk beyond m (non-integer delta / h) are no
// bonds: their threshold is NaN, which no |xi + eta|^2 reaches.
template <int DIM>
__global__ void k_break_thr(int nnb, const int32_t *__restrict__ off, double h, double s0, double m2, double *thr)
{
    const int kk = nnb / 2 + blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= nnb) return;
    const int ox = off[3 * kk], oy = off[3 * kk + 1], oz = off[3 * kk + 2];
    if ((double)(ox * ox + oy * oy + oz * oz) > m2 + 1e-9) {
        thr[kk] = __longlong_as_double(0x7ff8000000000000ll);
        double *xi = thr + nnb;
        xi[3 * kk] = xi[3 * kk + 1] = xi[3 * kk + 2] = 0.0;
        return;
    }
    const double xi0 = __dmul_rn(h, (double)ox), xi1 = __dmul_rn(h, (double)oy), xi2 = __dmul_rn(h, (double)oz);
    double r2 = __dadd_rn(__dmul_rn(xi0, xi0), __dmul_rn(xi1, xi1));
    if (DIM == 3) r2 = __dadd_rn(r2, __dmul_rn(xi2, xi2));
    const double r = __dsqrt_rn(r2);
    double *xi = thr + nnb;   // xi_c = h o_c, rounded once, for k_break
    xi[3 * kk] = xi0;
    xi[3 * kk + 1] = xi1;
    xi[3 * kk + 2] = xi2;
    auto broken = [&](unsigned long long bits) {
        return __ddiv_rn(__dsub_rn(__dsqrt_rn(__longlong_as_double((long long)bits)), r), r) >= s0;
    };
    unsigned long long lo = 0ull, hi = 0x7ff0000000000000ull;   // +0 (not broken for s0 > 0), +inf (broken)
    if (broken(lo)) {
        thr[kk] = 0.0;
        return;
    }
    while (hi - lo > 1ull) {
        const unsigned long long mid = lo + (hi - lo) / 2;
        if (broken(mid)) hi = mid;
        else lo = mid;
    }
    thr[kk] = __longlong_as_double((long long)hi);
}

template <int DIM, typename TU>
__global__ void __launch_bounds__(kBlk)
k_break(const TU *__restrict__ u, int64_t N, int nx, int ny, int nz, int nnb, const int32_t *__restrict__ off,
        uint32_t *mask, double h, const double *__restrict__ thr, int32_t *break_step, int32_t step_id,
        uint32_t *brflag, int32_t *brlist, unsigned long long *count)
{
    unsigned long long newly = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        node_coords(p, nx, ny, i, j, k);
        double up[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int c = 0; c < DIM; ++c) up[c] = (double)u[c * N + p];
        for (int kk = nnb / 2; kk < nnb; ++kk) {
            uint32_t *wp = mask + (int64_t)(kk >> 5) * N + p;
            const uint32_t bit = 1u << (kk & 31);
            if (!(*wp & bit)) continue;
            const int ox = off[3 * kk], oy = off[3 * kk + 1], oz = off[3 * kk + 2];
            const int qi = i + ox, qj = j + oy, qk = k + oz;
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            const int64_t q = ((int64_t)qk * ny + qj) * nx + qi;
            // Eq. fra:s1 in a fixed operation order, each step rounded once (see k_break_thr).
            const double xi0 = __ldg(thr + nnb + 3 * kk), xi1 = __ldg(thr + nnb + 3 * kk + 1),
                         xi2 = __ldg(thr + nnb + 3 * kk + 2);
            const double X0 = __dadd_rn(xi0, __dsub_rn((double)u[q], up[0]));
            const double X1 = __dadd_rn(xi1, __dsub_rn((double)u[N + q], up[1]));
            double l2 = __dadd_rn(__dmul_rn(X0, X0), __dmul_rn(X1, X1));
            if (DIM == 3) {
                const double X2 = __dadd_rn(xi2, __dsub_rn((double)u[2 * N + q], up[2]));
                l2 = __dadd_rn(l2, __dmul_rn(X2, X2));
            }
            if (l2 >= thr[kk]) {
                atomicAnd(wp, ~bit);
                const int km = nnb - 1 - kk;
                atomicAnd(mask + (int64_t)(km >> 5) * N + q, ~(1u << (km & 31)));
                if (break_step) {
                    break_step[p * nnb + kk] = step_id;
                    break_step[q * nnb + km] = step_id;
                }
                ++newly;
                mark_broken_node(p, brflag, brlist, count);
                mark_broken_node(q, brflag, brlist, count);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) newly += __shfl_xor_sync(0xffffffffu, newly, o);
    if ((threadIdx.x & 31) == 0 && newly) {
        atomicAdd(&count[1], newly);
        atomicAdd(&count[2], newly);
    }
}

// ------------------------------------------------------------------ pre-notch segment
__device__ __forceinline__ int orient(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy)
{
    const int64_t v = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    return (v > 0) - (v < 0);
}

__device__ __forceinline__ bool within(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy)
{
    return cx >= min(ax, bx) && cx <= max(ax, bx) && cy >= min(ay, by) && cy <= max(ay, by);
}

__global__ void __launch_bounds__(kBlk)
k_segment(int64_t N, int nx, int ny, int nz, int nnb, const int32_t *__restrict__ off, double m2, uint32_t *mask,
          int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t den, uint32_t *brflag, int32_t *brlist,
          unsigned long long *count)
{
    unsigned long long newly = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        node_coords(p, nx, ny, i, j, k);
        const int64_t px = den * (2 * i + 1), py = den * (2 * j + 1);
        for (int kk = nnb / 2; kk < nnb; ++kk) {   // upper half: q > p
            const int ox = off[3 * kk], oy = off[3 * kk + 1], oz = off[3 * kk + 2];
            if ((double)(ox * ox + oy * oy + oz * oz) > m2 + 1e-9) continue;   // no bond (beyond delta)
            const int qi = i + ox, qj = j + oy, qk = k + oz;
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            const int64_t qx = den * (2 * qi + 1), qy = den * (2 * qj + 1);
            const int d1 = orient(ax, ay, bx, by, px, py), d2 = orient(ax, ay, bx, by, qx, qy);
            const int d3 = orient(px, py, qx, qy, ax, ay), d4 = orient(px, py, qx, qy, bx, by);
            bool meet = (d1 * d2 < 0 && d3 * d4 < 0) || (d1 == 0 && within(ax, ay, bx, by, px, py)) ||
                        (d2 == 0 && within(ax, ay, bx, by, qx, qy)) || (d3 == 0 && within(px, py, qx, qy, ax, ay)) ||
                        (d4 == 0 && within(px, py, qx, qy, bx, by));
            if (!meet) continue;
            const int64_t q = ((int64_t)qk * ny + qj) * nx + qi;
            uint32_t *wp = mask + (int64_t)(kk >> 5) * N + p;
            const uint32_t bit = 1u << (kk & 31);
            if (*wp & bit) {
                atomicAnd(wp, ~bit);
                const int km = nnb - 1 - kk;
                atomicAnd(mask + (int64_t)(km >> 5) * N + q, ~(1u << (km & 31)));
                ++newly;
                mark_broken_node(p, brflag, brlist, count);
                mark_broken_node(q, brflag, brlist, count);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) newly += __shfl_xor_sync(0xffffffffu, newly, o);
    if ((threadIdx.x & 31) == 0 && newly) {
        atomicAdd(&count[1], newly);
        atomicAdd(&count[2], newly);
    }
}

// ------------------------------------------------------------------ Omega_br rebuild from a mask
__global__ void __launch_bounds__(kBlk)
k_refresh(int64_t N, int nx, int ny, int nz, int nnb, const int32_t *__restrict__ off,
          const uint32_t *__restrict__ mask, uint32_t *brflag, int32_t *brlist, unsigned long long *count)
{
    unsigned long long bonds = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        node_coords(p, nx, ny, i, j, k);
        bool any = false;
        for (int kk = 0; kk < nnb; ++kk) {
            const int qi = i + off[3 * kk], qj = j + off[3 * kk + 1], qk = k + off[3 * kk + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            if ((mask[(int64_t)(kk >> 5) * N + p] >> (kk & 31)) & 1u) continue;
            any = true;
            if (kk >= nnb / 2) ++bonds;
        }
        if (any) mark_broken_node(p, brflag, brlist, count);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bonds += __shfl_xor_sync(0xffffffffu, bonds, o);
    if ((threadIdx.x & 31) == 0 && bonds) atomicAdd(&count[1], bonds);
}

// ------------------------------------------------------------------ modulus gradient
template <int DIM>
__global__ void __launch_bounds__(kBlk)
k_grad_modulus(const double *__restrict__ u, const double *__restrict__ lam, int64_t N, int nx, int ny, int nz,
               int nnb, const int32_t *__restrict__ off, const double *__restrict__ coef1,
               const uint32_t *__restrict__ mask, const double *__restrict__ nu_tab, int M, double scale,
               double *grad)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        node_coords(p, nx, ny, i, j, k);
        const double nu_p = nu_tab ? nu_tab[nu_class(i, j, k, nx, ny, nz, M, DIM)] : 1.0;
        double acc = 0.0;
        for (int kk = 0; kk < nnb; ++kk) {
            const int qi = i + off[3 * kk], qj = j + off[3 * kk + 1], qk = k + off[3 * kk + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            if (!((mask[(int64_t)(kk >> 5) * N + p] >> (kk & 31)) & 1u)) continue;
            const int64_t q = ((int64_t)qk * ny + qj) * nx + qi;
            double du[DIM], dl[DIM];
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                du[c] = u[c * N + q] - u[c * N + p];
                dl[c] = lam[c * N + q] - lam[c * N + p];
            }
            double t;
            if (DIM == 2) {
                const double *cf = coef1 + 3 * kk;
                t = dl[0] * (cf[0] * du[0] + cf[1] * du[1]) + dl[1] * (cf[1] * du[0] + cf[2] * du[DIM - 1]);
            } else {
                const double *cf = coef1 + 6 * kk;
                t = dl[0] * (cf[0] * du[0] + cf[1] * du[1] + cf[2] * du[DIM - 1]) +
                    dl[1] * (cf[1] * du[0] + cf[3] * du[1] + cf[4] * du[DIM - 1]) +
                    dl[DIM - 1] * (cf[2] * du[0] + cf[4] * du[1] + cf[5] * du[DIM - 1]);
            }
            // surface correction: the bond carries (nu_p + nu_q) / 2
            acc += nu_tab ? 0.5 * (nu_p + nu_tab[nu_class(qi, qj, qk, nx, ny, nz, M, DIM)]) * t : t;
        }
        grad[p] += scale * acc;
    }
}

// ------------------------------------------------------------------ Verlet
// Drift: u += dt v + dt^2/2 a on free components, u += dt vp on constrained ones.
__global__ void __launch_bounds__(kBlk)
k_drift(double *u, const double *__restrict__ v, const double *__restrict__ a, const double *__restrict__ vp,
        const uint8_t *__restrict__ cons, int64_t N, int dim, double dt)
{
    const double h2 = 0.5 * dt * dt;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < dim * N; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / N);
        const int64_t p = t - c * N;
        const bool fixed = cons && ((cons[p] >> c) & 1);
        if (fixed) u[t] += dt * (vp ? vp[t] : 0.0);
        else u[t] += dt * v[t] + h2 * a[t];
    }
}

// Kick: a_new = (f + b) / rho; v += dt/2 (a + a_new) on free components, v = vp on
// constrained ones; a = a_new.
__global__ void __launch_bounds__(kBlk)
k_kick(double *v, double *a, const double *__restrict__ f, const double *__restrict__ b,
       const double *__restrict__ vp, const uint8_t *__restrict__ cons, int64_t N, int dim, double dt,
       double inv_rho, int first)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < dim * N; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / N);
        const int64_t p = t - c * N;
        const double an = (f[t] + (b ? b[t] : 0.0)) * inv_rho;
        if (!first) {
            const bool fixed = cons && ((cons[p] >> c) & 1);
            if (fixed) v[t] = vp ? vp[t] : 0.0;
            else v[t] += 0.5 * dt * (a[t] + an);
        }
        a[t] = an;
    }
}

int grid_blocks(int64_t work)
{
    int64_t b = (work + kBlk - 1) / kBlk;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

int launch_df_gather(pd_grid *g, bool f64, const void *u, void *out, int64_t batch, bool project, double scale,
                     cudaStream_t s)
{
    const int blocks = 152 * 4;
    const int nx = (int)g->n[0], ny = (int)g->n[1], nz = (int)g->n[2];
#define PD_DF(T, D)                                                                                         \
    k_df_gather<T, D><<<blocks, kBlk, 0, s>>>((const T *)u, (T *)out, g->N, nx, ny, nz, g->nnb, g->d_brlist, \
                                               g->d_count, g->d_mask, g->d_off, g->d_coef, g->d_cons,       \
                                               project ? 1 : 0, scale, batch)
    if (g->dim == 2) {
        if (f64) PD_DF(double, 2); else PD_DF(float, 2);
    } else {
        if (f64) PD_DF(double, 3); else PD_DF(float, 3);
    }
#undef PD_DF
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int launch_break(pd_grid *g, const void *u, bool f64, int32_t *break_step, int32_t step_id, cudaStream_t s)
{
    if (!(g->s0 > 0.0)) return PD_OK;
    if (g->brk_thr_s0 != g->s0) {   // thresholds for this s0 (stream-ordered, no allocation)
        const int nh = g->nnb - g->nnb / 2;
        if (g->dim == 2)
            k_break_thr<2><<<(nh + 127) / 128, 128, 0, s>>>(g->nnb, g->d_off, g->h, g->s0, g->m * g->m,
                                                            g->d_brk_thr);
        else
            k_break_thr<3><<<(nh + 127) / 128, 128, 0, s>>>(g->nnb, g->d_off, g->h, g->s0, g->m * g->m,
                                                            g->d_brk_thr);
        PD_CUDA(cudaGetLastError());
        g->brk_thr_s0 = g->s0;
    }
    const int blocks = grid_blocks(g->N);
    const int nx = (int)g->n[0], ny = (int)g->n[1], nz = (int)g->n[2];
#define PD_BRK(D, TU)                                                                                          \
    k_break<D, TU><<<blocks, kBlk, 0, s>>>((const TU *)u, g->N, nx, ny, nz, g->nnb, g->d_off, g->d_mask, g->h, \
                                            g->d_brk_thr, break_step, step_id, g->d_brflag, g->d_brlist, g->d_count)
    if (g->dim == 2) {
        if (f64) PD_BRK(2, double); else PD_BRK(2, float);
    } else {
        if (f64) PD_BRK(3, double); else PD_BRK(3, float);
    }
#undef PD_BRK
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int launch_break_segment(pd_grid *g, const int64_t seg[4], int64_t den, cudaStream_t s)
{
    k_segment<<<grid_blocks(g->N), kBlk, 0, s>>>(g->N, (int)g->n[0], (int)g->n[1], (int)g->n[2], g->nnb, g->d_off,
                                                  g->m * g->m, g->d_mask,
                                                  2 * seg[0], 2 * seg[1], 2 * seg[2], 2 * seg[3], den, g->d_brflag,
                                                  g->d_brlist, g->d_count);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int refresh_broken_nodes(pd_grid *g, cudaStream_t s)
{
    PD_CUDA(cudaMemsetAsync(g->d_brflag, 0, sizeof(uint32_t) * (size_t)g->N, s));
    PD_CUDA(cudaMemsetAsync(g->d_count, 0, sizeof(unsigned long long) * 2, s));
    k_refresh<<<grid_blocks(g->N), kBlk, 0, s>>>(g->N, (int)g->n[0], (int)g->n[1], (int)g->n[2], g->nnb, g->d_off,
                                                  g->d_mask, g->d_brflag, g->d_brlist, g->d_count);
    PD_CUDA(cudaGetLastError());
    PD_CUDA(cudaMemcpyAsync(g->h_pinned, g->d_count, sizeof(unsigned long long) * 2, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    g->broken_total = (int64_t)g->h_pinned[1];
    ++g->op_stamp;
    return PD_OK;
}

int launch_grad_modulus(pd_grid *g, const double *u, const double *lam, double scale, double *grad, cudaStream_t s)
{
    const int nx = (int)g->n[0], ny = (int)g->n[1], nz = (int)g->n[2];
    if (g->dim == 2)
        k_grad_modulus<2><<<grid_blocks(g->N), kBlk, 0, s>>>(u, lam, g->N, nx, ny, nz, g->nnb, g->d_off, g->d_coef1,
                                                              g->d_mask, g->sc ? g->d_nu_tab : nullptr, g->M,
                                                              scale, grad);
    else
        k_grad_modulus<3><<<grid_blocks(g->N), kBlk, 0, s>>>(u, lam, g->N, nx, ny, nz, g->nnb, g->d_off, g->d_coef1,
                                                              g->d_mask, g->sc ? g->d_nu_tab : nullptr, g->M,
                                                              scale, grad);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pd

using namespace pd;

extern "C" int pd_step(pd_grid *g, double *u, double *v, const double *b, int nsteps, double dt,
                       const double *v_prescribed, int32_t *break_step, int32_t step_base, pd_step_stats *stats,
                       void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!u || !v) return fail(PD_ERR_INVALID, "u and v must be device pointers");
    if (nsteps < 0 || !(dt > 0)) return fail(PD_ERR_INVALID, "nsteps >= 0 and dt > 0 required");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t L = (int64_t)g->dim * g->N;
    const size_t need = sizeof(double) * 2 * (size_t)L;
    if (g->ws_bytes < need) {
        cudaFree(g->ws);
        g->ws = nullptr;
        g->ws_bytes = 0;
        if (cudaMalloc(&g->ws, need) != cudaSuccess) return fail(PD_ERR_OOM, "Verlet workspace");
        g->ws_bytes = need;
    }
    double *a = (double *)g->ws;
    double *f = a + L;
    const uint8_t *cons = g->has_cons ? g->d_cons : nullptr;
    const int blocks = grid_blocks(L);
    const uint32_t mflags = PD_F64 | PD_METHOD_STENCIL | kForceMu;
    PD_CUDA(cudaMemsetAsync(g->d_count + 2, 0, sizeof(unsigned long long), s));
    // f = A(mu) u = -K u at the incoming state, a = (f + b) / rho
    int rc = matvec(g, 1, u, f, mflags, s, nullptr, nullptr, nullptr, -1.0);
    if (rc) return rc;
    k_kick<<<blocks, kBlk, 0, s>>>(v, a, f, b, v_prescribed, cons, g->N, g->dim, dt, 1.0 / g->rho, 1);
    for (int st = 0; st < nsteps; ++st) {
        k_drift<<<blocks, kBlk, 0, s>>>(u, v, a, v_prescribed, cons, g->N, g->dim, dt);
        rc = launch_break(g, u, true, break_step, step_base + st + 1, s);
        if (rc) return rc;
        rc = matvec(g, 1, u, f, mflags, s, nullptr, nullptr, nullptr, -1.0);
        if (rc) return rc;
        k_kick<<<blocks, kBlk, 0, s>>>(v, a, f, b, v_prescribed, cons, g->N, g->dim, dt, 1.0 / g->rho, 0);
    }
    PD_CUDA(cudaGetLastError());
    PD_CUDA(cudaMemcpyAsync(g->h_pinned, g->d_count, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    g->broken_total = (int64_t)g->h_pinned[1];
    if (g->h_pinned[2]) ++g->op_stamp;
    if (stats) {
        stats->steps = nsteps;
        stats->newly_broken = (int64_t)g->h_pinned[2];
        stats->broken_total = g->broken_total;
    }
    return PD_OK;
}

// ---------------------------------------------------------------------------
// Stable step of the central-difference (Verlet) scheme of Algorithm 2: the
// undamped scheme u'' = -K u / rho is stable for dt < 2 / sqrt(lambda_max(K) / rho).
// lambda_max is bounded by the largest eigenvalue of the symbol of the
// full-horizon operator over the frequencies of a periodic grid of twice the
// extent (zero-extension only adds bond energy; broken bonds lower it; a
// modulus field scales it by at most its largest value), the unit-modulus
// symbol being K^1(k) = sum_{o in half} 2 c1(o) (1 - cos k.o) (2 x 2 or 3 x 3,
// real and symmetric since c1(o) = c1(-o)).
extern "C" int pd_stable_dt(pd_grid *g, double *dt)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!dt) return fail(PD_ERR_INVALID, "dt is NULL");
    const int d = g->dim, nc = ncoef(d);
    // the frequency grid: 2 n per axis in 2D; at most 2 x 48 per axis in 3D (the symbol
    // is a trigonometric polynomial of degree M, which that grid resolves finely)
    int64_t L[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) L[a] = d == 2 ? 2 * g->n[a] : std::min<int64_t>(2 * g->n[a], 96);
    std::vector<int> half;
    for (int k = 0; k < g->nnb; ++k) {   // one offset of each pair +-o: the first nonzero component positive
        const int32_t *o = &g->off[3 * k];
        const int f = o[2] != 0 ? o[2] : (o[1] != 0 ? o[1] : o[0]);
        if (f > 0) half.push_back(k);
    }
    const double two_pi = 6.283185307179586476925;
    double lam = 0.0;
    for (int64_t kz = 0; kz < L[2]; ++kz)
        for (int64_t ky = 0; ky < L[1]; ++ky)
            for (int64_t kx = 0; kx < L[0]; ++kx) {
                const double w[3] = {two_pi * kx / L[0], two_pi * ky / L[1], two_pi * kz / L[2]};
                double S[6] = {0, 0, 0, 0, 0, 0};
                for (int k : half) {
                    const int32_t *o = &g->off[3 * k];
                    const double f = 2.0 * (1.0 - std::cos(w[0] * o[0] + w[1] * o[1] + w[2] * o[2]));
                    for (int i = 0; i < nc; ++i) S[i] += f * g->coef1[(size_t)nc * k + i];
                }
                double m;
                if (d == 2) {   // xx, xy, yy
                    const double tr = 0.5 * (S[0] + S[2]), df = 0.5 * (S[0] - S[2]);
                    m = tr + std::sqrt(df * df + S[1] * S[1]);
                } else {        // xx, xy, xz, yy, yz, zz: largest eigenvalue of a symmetric 3 x 3
                    const double a = S[0], b = S[3], c = S[5], x = S[1], y = S[2], z = S[4];
                    const double q = (a + b + c) / 3.0;
                    const double p1 = x * x + y * y + z * z;
                    const double p2 = (a - q) * (a - q) + (b - q) * (b - q) + (c - q) * (c - q) + 2.0 * p1;
                    if (p2 <= 0.0) {
                        m = q;
                    } else {
                        const double p = std::sqrt(p2 / 6.0);
                        const double B00 = (a - q) / p, B11 = (b - q) / p, B22 = (c - q) / p;
                        const double B01 = x / p, B02 = y / p, B12 = z / p;
                        const double detB = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) +
                                            B02 * (B01 * B12 - B11 * B02);
                        const double r = std::max(-1.0, std::min(1.0, 0.5 * detB));
                        m = q + 2.0 * p * std::cos(std::acos(r) / 3.0);
                    }
                }
                lam = std::max(lam, m);
            }
    if (!(lam > 0)) return fail(PD_ERR_STATE, "the operator has no positive eigenvalue");
    *dt = 2.0 * std::sqrt(g->rho / (g->E_max * lam));
    return PD_OK;
}

// ---------------------------------------------------------------------------
// pd_step_noalloc: the velocity-Verlet loop of pd_step without any device
// allocation.  pd_step keeps its two work vectors (acceleration and force) in
// a buffer it cudaMallocs on first use; some callers cannot let a library do
// that (see pd.h).  This variant keeps the two vectors in the file-scope array
// below instead: 2^20 doubles (8 MiB), which every GPU that loads the library
// holds until the process exits, so dim * N may be at most 2^19
// (a 512 x 512 plate in 2D).
namespace pd {
namespace {

constexpr size_t kNoAllocDoubles = (size_t)1 << 20;
static __device__ __align__(256) double g_step_scratch[kNoAllocDoubles];

// The array's name is only a host-side stand-in in host code; its device
// address is looked up once per device with that device current.
std::mutex g_scratch_mu;
double *g_scratch_addr[64] = {};

// The grid's device must be current: the array is looked up, and the kernels
// run, on it.
int step_scratch(const pd_grid *g, double **out)
{
    int dev = -1;
    PD_CUDA(cudaGetDevice(&dev));
    if (dev != g->device)
        return fail(PD_ERR_INVALID, "pd_step_noalloc: the current device (" + std::to_string(dev) +
                                        ") is not the grid's (" + std::to_string(g->device) + ")");
    if (dev < 0 || dev >= 64) return fail(PD_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_step_scratch);
        if (e != cudaSuccess || !p)
            return fail(PD_ERR_CUDA, std::string("cudaGetSymbolAddress(step scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return PD_OK;
}

}  // namespace
}  // namespace pd

extern "C" int pd_step_noalloc(pd_grid *g, double *u, double *v, const double *b, int nsteps, double dt,
                               const double *v_prescribed, int32_t *break_step, int32_t step_base,
                               pd_step_stats *stats, void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!u || !v) return fail(PD_ERR_INVALID, "u and v must be device pointers");
    if (nsteps < 0 || !(dt > 0)) return fail(PD_ERR_INVALID, "nsteps >= 0 and dt > 0 required");
    const int64_t L = (int64_t)g->dim * g->N;
    if ((size_t)(2 * L) > kNoAllocDoubles)
        return fail(PD_ERR_INVALID, "pd_step_noalloc: dim * N = " + std::to_string(L) +
                                        " exceeds its fixed scratch (dim * N <= 524288); use pd_step");
    double *scratch = nullptr;
    int rc = step_scratch(g, &scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    double *a = scratch;       // both vectors are written in full before they are read
    double *f = scratch + L;
    const uint8_t *cons = g->has_cons ? g->d_cons : nullptr;
    const int blocks = grid_blocks(L);
    const uint32_t mflags = PD_F64 | PD_METHOD_STENCIL | kForceMu;
    PD_CUDA(cudaMemsetAsync(g->d_count + 2, 0, sizeof(unsigned long long), s));
    rc = matvec(g, 1, u, f, mflags, s, nullptr, nullptr, nullptr, -1.0);
    if (rc) return rc;
    k_kick<<<blocks, kBlk, 0, s>>>(v, a, f, b, v_prescribed, cons, g->N, g->dim, dt, 1.0 / g->rho, 1);
    for (int st = 0; st < nsteps; ++st) {
        k_drift<<<blocks, kBlk, 0, s>>>(u, v, a, v_prescribed, cons, g->N, g->dim, dt);
        rc = launch_break(g, u, true, break_step, step_base + st + 1, s);
        if (rc) return rc;
        rc = matvec(g, 1, u, f, mflags, s, nullptr, nullptr, nullptr, -1.0);
        if (rc) return rc;
        k_kick<<<blocks, kBlk, 0, s>>>(v, a, f, b, v_prescribed, cons, g->N, g->dim, dt, 1.0 / g->rho, 0);
    }
    PD_CUDA(cudaGetLastError());
    PD_CUDA(cudaMemcpyAsync(g->h_pinned, g->d_count, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    g->broken_total = (int64_t)g->h_pinned[1];
    if (g->h_pinned[2]) ++g->op_stamp;
    if (stats) {
        stats->steps = nsteps;
        stats->newly_broken = (int64_t)g->h_pinned[2];
        stats->broken_total = g->broken_total;
    }
    return PD_OK;
}

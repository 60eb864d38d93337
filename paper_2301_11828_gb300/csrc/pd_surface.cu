// pd_surface.cu -- surface correction on incomplete horizons (the remark on
// Omega_e in Sec. 3.3 and Eq. scr of Sec. 5.2).
//
// The paper scales the bonds of nodes whose horizon is cut by the boundary by
// a factor v_pq and takes the factor from its reference.  The reading used
// here is the volume method:
//     V_p  = sum over in-grid neighbours q of lambda(q - p)   (partial volume / h^d)
//     nu_p = V_full / V_p                                     (1 on a full horizon)
//     v_pq = (nu_p + nu_q) / 2                                (symmetric, so K stays SPD)
// and A_pq = v_pq A^_pq.  As the paper says, the factor breaks the Toeplitz
// structure, so the product is computed as the uncorrected one (TBT stencil or
// FFT plus D^e and D^f) followed by a direct correction over the edge band:
//     (K_sc u)_p = (K u)_p - sum_q mu_pq (v_pq - 1) C_pq (u_q - u_p).
// v_pq != 1 only when p or q has an incomplete horizon, i.e. only for nodes
// closer than 2M (grid units, along some axis) to a face; that band is a
// compacted node list built once.  nu depends only on the distances to the
// faces clipped at M, so it lives in a table of (M+1)^(2 dim) classes.
//
// One warp per band node: the lanes take the offsets, compute nu of the
// neighbour from its class, and reduce the three (or two) components.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kBlk = 256;

// out -= scale * sum_q mu (v - 1) C (u_q - u_p) on every band node; one field
// per grid row.  Arithmetic in C (the field's precision: FP64 is a slow pipe
// on this GPU and FP32 outputs need no more); coef: unit-modulus bond blocks
// in C, times Econst, or times (E_p + E_q) / 2 when E (per node) is given.
template <typename T, typename C, int DIM>
__global__ void __launch_bounds__(kBlk)
k_sc_gather(const T *__restrict__ u, T *__restrict__ out, int64_t N, int nx, int ny, int nz, int M, int nnb,
            const int32_t *__restrict__ band, int64_t nband, const int32_t *__restrict__ off,
            const C *__restrict__ coef, C Econst, const double *__restrict__ E, const C *__restrict__ nu_tab,
            const uint32_t *__restrict__ mask, int use_mu, const uint8_t *__restrict__ cons, int project,
            double scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const T *ub = u + (int64_t)blockIdx.y * DIM * N;   // one field per grid row
    T *ob = out + (int64_t)blockIdx.y * DIM * N;
    for (int64_t w = warp; w < nband; w += nwarps) {
        const int p = band[w];   // fewer than 2^31 nodes: 32-bit index arithmetic
        const int i = p % nx, j = (p / nx) % ny, k = p / (nx * ny);
        const C nu_p = nu_tab[nu_class(i, j, k, nx, ny, nz, M, DIM)];
        const C E_p = E ? (C)E[p] : C(0);
        const uint8_t cm = project ? cons[p] : 0;
        C up[DIM], acc[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            up[c] = ((cm >> c) & 1) ? C(0) : (C)ub[c * N + p];
            acc[c] = C(0);
        }
        for (int kk = lane; kk < nnb; kk += 32) {
            const int qi = i + off[3 * kk], qj = j + off[3 * kk + 1], qk = k + off[3 * kk + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            if (use_mu && !((mask[(int64_t)(kk >> 5) * N + p] >> (kk & 31)) & 1u)) continue;
            const C nu_q = nu_tab[nu_class(qi, qj, qk, nx, ny, nz, M, DIM)];
            C wgt = C(0.5) * (nu_p + nu_q) - C(1);
            if (wgt == C(0)) continue;
            const int q = (qk * ny + qj) * nx + qi;
            wgt *= E ? C(0.5) * (E_p + (C)E[q]) : Econst;
            const uint8_t qm = project ? cons[q] : 0;
            C d[DIM];
#pragma unroll
            for (int c = 0; c < DIM; ++c) d[c] = (((qm >> c) & 1) ? C(0) : (C)ub[c * N + q]) - up[c];
            if (DIM == 2) {
                const C *cf = coef + 3 * kk;
                acc[0] += wgt * (cf[0] * d[0] + cf[1] * d[1]);
                acc[1] += wgt * (cf[1] * d[0] + cf[2] * d[DIM - 1]);
            } else {
                const C *cf = coef + 6 * kk;
                acc[0] += wgt * (cf[0] * d[0] + cf[1] * d[1] + cf[2] * d[DIM - 1]);
                acc[1] += wgt * (cf[1] * d[0] + cf[3] * d[1] + cf[4] * d[DIM - 1]);
                acc[DIM - 1] += wgt * (cf[2] * d[0] + cf[4] * d[1] + cf[5] * d[DIM - 1]);
            }
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < DIM; ++c)
                if (!((cm >> c) & 1)) ob[c * N + p] = (T)((C)ob[c * N + p] - (C)scale * acc[c]);
        }
    }
}

// Largest absolute row sum of the corrected K over the band rows (bonds intact,
// no projection): per component a, sum_b |sum_q v C_ab| + sum_q sum_b |v C_ab|.
// The sums are non-negative, so their bit patterns order like the values and
// an integer atomicMax finds the maximum exactly.
template <int DIM>
__global__ void __launch_bounds__(kBlk)
k_sc_rowmax(int64_t N, int nx, int ny, int nz, int M, int nnb, const int32_t *__restrict__ band, int64_t nband,
            const int32_t *__restrict__ off, const double *__restrict__ coef, const double *__restrict__ nu_tab,
            unsigned long long *rowmax)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int NC = DIM == 2 ? 3 : 6;
    for (int64_t w = warp; w < nband; w += nwarps) {
        const int p = band[w];
        const int i = p % nx, j = (p / nx) % ny, k = p / (nx * ny);
        const double nu_p = nu_tab[nu_class(i, j, k, nx, ny, nz, M, DIM)];
        double diag[NC], offs[DIM];
#pragma unroll
        for (int c = 0; c < NC; ++c) diag[c] = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) offs[c] = 0.0;
        for (int kk = lane; kk < nnb; kk += 32) {
            const int qi = i + off[3 * kk], qj = j + off[3 * kk + 1], qk = k + off[3 * kk + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            const double v = 0.5 * (nu_p + nu_tab[nu_class(qi, qj, qk, nx, ny, nz, M, DIM)]);
            const double *cf = coef + NC * kk;
#pragma unroll
            for (int c = 0; c < NC; ++c) diag[c] += v * cf[c];
            if (DIM == 2) {
                offs[0] += fabs(v * cf[0]) + fabs(v * cf[1]);
                offs[1] += fabs(v * cf[1]) + fabs(v * cf[2]);
            } else {
                offs[0] += fabs(v * cf[0]) + fabs(v * cf[1]) + fabs(v * cf[2]);
                offs[1] += fabs(v * cf[1]) + fabs(v * cf[3]) + fabs(v * cf[4]);
                offs[DIM - 1] += fabs(v * cf[2]) + fabs(v * cf[4]) + fabs(v * cf[5]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int c = 0; c < NC; ++c) diag[c] += __shfl_xor_sync(0xffffffffu, diag[c], o);
#pragma unroll
            for (int c = 0; c < DIM; ++c) offs[c] += __shfl_xor_sync(0xffffffffu, offs[c], o);
        }
        if (lane == 0) {
            double r[DIM];
            if (DIM == 2) {
                r[0] = offs[0] + fabs(diag[0]) + fabs(diag[1]);
                r[1] = offs[1] + fabs(diag[1]) + fabs(diag[2]);
            } else {
                r[0] = offs[0] + fabs(diag[0]) + fabs(diag[1]) + fabs(diag[2]);
                r[1] = offs[1] + fabs(diag[1]) + fabs(diag[3]) + fabs(diag[4]);
                r[DIM - 1] = offs[DIM - 1] + fabs(diag[2]) + fabs(diag[4]) + fabs(diag[5]);
            }
#pragma unroll
            for (int c = 0; c < DIM; ++c) atomicMax(&rowmax[c], (unsigned long long)__double_as_longlong(r[c]));
        }
    }
}

}  // namespace

// Builds the nu class table and the band list (host, once), or drops them.
int surface_set(pd_grid *g, int mode)
{
    cudaFree(g->d_nu_tab);
    cudaFree(g->d_band);
    g->d_nu_tab = nullptr;
    g->d_band = nullptr;
    g->d_sc_rowmax = nullptr;
    g->d_sc_f32 = nullptr;
    g->band_n = 0;
    g->sc = 0;
    ++g->op_stamp;
    if (mode == PD_SC_NONE) return PD_OK;
    if (g->N > INT_MAX) return fail(PD_ERR_INVALID, "surface correction needs fewer than 2^31 nodes");
    const int M = g->M, dim = g->dim, B = M + 1;
    // lambda-weighted in-grid neighbour count per class of clipped face distances
    std::vector<double> lam(g->nnb);
    double full = 0.0;
    for (int k = 0; k < g->nnb; ++k) {
        const int32_t *o = &g->off[3 * k];
        lam[k] = lambda_of(o[0] * o[0] + o[1] * o[1] + o[2] * o[2], g->m);
        full += lam[k];
    }
    int ncls = 1;
    for (int a = 0; a < 2 * dim; ++a) ncls *= B;
    std::vector<double> tab(ncls);
    for (int c = 0; c < ncls; ++c) {
        int d[6] = {M, M, M, M, M, M};   // lo x, hi x, lo y, hi y, lo z, hi z
        int t = c;
        for (int a = 2 * dim - 1; a >= 0; --a) {
            d[a] = t % B;
            t /= B;
        }
        double V = 0.0;
        for (int k = 0; k < g->nnb; ++k) {
            const int32_t *o = &g->off[3 * k];
            bool in = (-o[0] <= d[0]) && (o[0] <= d[1]) && (-o[1] <= d[2]) && (o[1] <= d[3]);
            if (dim == 3) in = in && (-o[2] <= d[4]) && (o[2] <= d[5]);
            if (in) V += lam[k];
        }
        tab[c] = full / V;
    }
    // band: nodes closer than 2M to some face along some axis
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const int64_t W = 2 * (int64_t)M;
    std::vector<int32_t> band;
    auto near = [&](int64_t x, int64_t n) { return x < W || x >= n - W; };
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j) {
            const bool edge_row = near(j, ny) || (dim == 3 && near(k, nz));
            const int64_t base = (k * ny + j) * nx;
            if (edge_row) {
                for (int64_t i = 0; i < nx; ++i) band.push_back((int32_t)(base + i));
            } else {
                const int64_t lo_end = std::min(W, nx), hi_start = std::max(W, nx - W);
                for (int64_t i = 0; i < lo_end; ++i) band.push_back((int32_t)(base + i));
                for (int64_t i = hi_start; i < nx; ++i) band.push_back((int32_t)(base + i));
            }
        }
    // the table, three words of scratch for the row maximum, then FP32 copies of the
    // table and of the unit-modulus bond blocks for the FP32 gather
    const int nc = ncoef(dim);
    const size_t nf = tab.size() + (size_t)g->nnb * nc;
    PD_CUDA(cudaMalloc(&g->d_nu_tab, sizeof(double) * (tab.size() + 3) + sizeof(float) * nf));
    PD_CUDA(cudaMemcpy(g->d_nu_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
    g->d_sc_rowmax = (unsigned long long *)(g->d_nu_tab + tab.size());
    std::vector<float> f32(nf);
    for (size_t t = 0; t < tab.size(); ++t) f32[t] = (float)tab[t];
    for (size_t t = 0; t < (size_t)g->nnb * nc; ++t) f32[tab.size() + t] = (float)g->coef1[t];
    g->d_sc_f32 = (float *)(g->d_nu_tab + tab.size() + 3);
    g->sc_ncls = (int)tab.size();
    PD_CUDA(cudaMemcpy(g->d_sc_f32, f32.data(), sizeof(float) * nf, cudaMemcpyHostToDevice));
    if (!band.empty()) {
        PD_CUDA(cudaMalloc(&g->d_band, sizeof(int32_t) * band.size()));
        PD_CUDA(cudaMemcpy(g->d_band, band.data(), sizeof(int32_t) * band.size(), cudaMemcpyHostToDevice));
    }
    g->band_n = (int64_t)band.size();
    g->sc = mode;
    return PD_OK;
}

int launch_sc_gather(pd_grid *g, bool f64, const void *u, void *out, int64_t batch, bool project, bool use_mu,
                     double scale, cudaStream_t s)
{
    if (!g->sc || g->band_n == 0) return PD_OK;
    if (batch > 65535) return fail(PD_ERR_INVALID, "batch must be at most 65535");
    const int64_t per_field = std::max<int64_t>(1, std::min<int64_t>((g->band_n + 7) / 8, 152 * 8 / batch + 1));
    const dim3 blocks((unsigned)per_field, (unsigned)batch);   // 8 warps per block, one node per warp
    const int nx = (int)g->n[0], ny = (int)g->n[1], nz = (int)g->n[2];
    const double *E = g->has_E ? g->d_E : nullptr;
    const float *nu32 = g->d_sc_f32, *coef32 = g->d_sc_f32 + g->sc_ncls;
#define PD_SC(T, C, D, COEF, NU)                                                                                    \
    k_sc_gather<T, C, D><<<blocks, kBlk, 0, s>>>((const T *)u, (T *)out, g->N, nx, ny, nz, g->M, g->nnb, g->d_band,   \
                                                  g->band_n, g->d_off, COEF, (C)g->E, E, NU, g->d_mask,               \
                                                  use_mu ? 1 : 0, g->d_cons, project ? 1 : 0, scale)
    if (g->dim == 2) {
        if (f64) PD_SC(double, double, 2, g->d_coef1, g->d_nu_tab); else PD_SC(float, float, 2, coef32, nu32);
    } else {
        if (f64) PD_SC(double, double, 3, g->d_coef1, g->d_nu_tab); else PD_SC(float, float, 3, coef32, nu32);
    }
#undef PD_SC
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int surface_row_abs_max(pd_grid *g, double out[3], cudaStream_t s)
{
    out[0] = out[1] = out[2] = 0.0;
    if (!g->sc || g->band_n == 0) return PD_OK;
    unsigned long long *d = g->d_sc_rowmax;
    PD_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * 3, s));
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((g->band_n + 7) / 8, 152 * 8));
    const int nx = (int)g->n[0], ny = (int)g->n[1], nz = (int)g->n[2];
    if (g->dim == 2)
        k_sc_rowmax<2><<<blocks, kBlk, 0, s>>>(g->N, nx, ny, nz, g->M, g->nnb, g->d_band, g->band_n, g->d_off,
                                               g->d_coef, g->d_nu_tab, d);
    else
        k_sc_rowmax<3><<<blocks, kBlk, 0, s>>>(g->N, nx, ny, nz, g->M, g->nnb, g->d_band, g->band_n, g->d_off,
                                               g->d_coef, g->d_nu_tab, d);
    PD_CUDA(cudaGetLastError());
    unsigned long long h[3] = {0, 0, 0};
    PD_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < g->dim; ++c) {
        double v;
        std::memcpy(&v, &h[c], sizeof(v));
        out[c] = v;
    }
    return PD_OK;
}

}  // namespace pd

using namespace pd;

extern "C" int pd_set_surface_correction(pd_grid *g, int mode)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (mode != PD_SC_NONE && mode != PD_SC_VOLUME) return fail(PD_ERR_INVALID, "unknown surface-correction mode");
    cudaSetDevice(g->device);
    return surface_set(g, mode);
}

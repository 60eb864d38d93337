// pd_direct2d.cu -- 2D stencil, direct bond form with an inline bond mask and a
// per-node modulus (Eq. mat:f1 with the bond state mu of Eq. mu):
//     (K u)_p = sum_{o: p+o in grid, mu_p(o) = 1} w_pq c(o) (u_p - u_{p+o}),
// w_pq = (E_p + E_q)/2 with unit-modulus coefficients when a modulus field is
// set, else w_pq = 1 with the coefficients at the grid's modulus.  Used by the
// dynamic crack loop and by every operator application with a modulus field.
//
// The shared-memory box carries a third plane holding E/2 (or 1/2) inside the
// grid and 0 outside, so "q outside the grid" is "E_q == 0" (moduli are
// validated positive) and w_pq is one addition.  Each thread owns R consecutive
// y outputs of one column and reads their bond-mask words once.
//
// A bond's block is rank one, c(o) = kappa(o) o o^T (Eq. frb:e1), so an
// offset with both components nonzero applies it as kappa o (o . d) with
// d = u_p - u_q: one dot product with the integer offset and two FMAs, instead
// of the four products of the 2 x 2 block.
#include "pd_stencil.cuh"

namespace pd {

// Per offset in canonical order: (kappa ox, kappa oy) for offsets with both
// components nonzero, (c_xx, 0) for (ox, 0) and (0, c_yy) for (0, oy).
template <typename T, int M>
struct BondTab2 {
    static constexpr int kN = count_offsets(2, M);
    T v[kN * 2];
};

__device__ __forceinline__ bool nonzero_bits(double v) { return __double_as_longlong(v) != 0; }
__device__ __forceinline__ bool nonzero_bits(float v) { return __float_as_int(v) != 0; }

template <typename T, int M>
__global__ void __launch_bounds__(kThreads)
k_direct2d(const T *__restrict__ u, T *__restrict__ out, int nx, int ny, int64_t N,
           const uint8_t *__restrict__ cons, int project, const double *__restrict__ Ef,
           const uint32_t *__restrict__ mask, T scale, BondTab2<T, M> tab, double *dot_partial, double *dot_out,
           unsigned int *retire)
{
    constexpr int R = rows2d_direct<T, M>();
    constexpr int TX = kTX2, TY = kGY2 * R, SX = TX + 2 * M, SY = TY + 2 * M, WL = R + 2 * M;
    constexpr int NB = count_offsets(2, M);
    constexpr int W = (NB + 31) / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_x = reinterpret_cast<T *>(smem_raw);
    T *s_y = s_x + SX * SY;
    T *s_e = s_y + SX * SY;

    const int64_t b = blockIdx.z;
    const T *ub = u + b * 2 * N;
    T *ob = out + b * 2 * N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    for (int t = threadIdx.x; t < SX * SY; t += kThreads) {
        const int r = t / SX, c = t - r * SX;
        const int gx = x0 - M + c, gy = y0 - M + r;
        T vx = T(0), vy = T(0), ve = T(0);
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
            const int64_t p = (int64_t)gy * nx + gx;
            vx = __ldg(ub + p);
            vy = __ldg(ub + N + p);
            ve = Ef ? T(0.5) * (T)__ldg(Ef + p) : T(0.5);   // halved: exact
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) vx = T(0);
                if (m & 2) vy = T(0);
            }
        }
        s_x[t] = vx;
        s_y[t] = vy;
        s_e[t] = ve;
    }
    __syncthreads();

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int coff = (ty * R) * SX + tx + M;
    const int gx = x0 + tx;
    T upx[R], upy[R], ep[R], ax[R], ay[R];
    uint32_t mk[R][W];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        upx[r] = s_x[coff + (M + r) * SX];
        upy[r] = s_y[coff + (M + r) * SX];
        ep[r] = s_e[coff + (M + r) * SX];
        ax[r] = T(0);
        ay[r] = T(0);
        const int gy = y0 + ty * R + r;
        const bool in = (gx < nx && gy < ny);
#pragma unroll
        for (int w = 0; w < W; ++w)
            mk[r][w] = (mask && in) ? __ldg(mask + (int64_t)w * N + (int64_t)gy * nx + gx) : 0xffffffffu;
    }
    static_for<-M, M + 1>([&](auto OX) {
        constexpr int ox = decltype(OX)::value;
        constexpr int My = isqrt_c(M * M - ox * ox);
        T wx[WL], wy[WL], we[WL];
#pragma unroll
        for (int i = 0; i < WL; ++i) {
            wx[i] = s_x[coff + i * SX + ox];
            wy[i] = s_y[coff + i * SX + ox];
            we[i] = s_e[coff + i * SX + ox];
        }
        static_for<-My, My + 1>([&](auto OY) {
            constexpr int oy = decltype(OY)::value;
            if constexpr (ox != 0 || oy != 0) {
                constexpr int k = canon_index(2, M, ox, oy, 0);
                const T ka = tab.v[2 * k], kb = tab.v[2 * k + 1];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T eq = we[r + M + oy];
                    const bool on = ((mk[r][k >> 5] >> (k & 31)) & 1u) && nonzero_bits(eq);
                    const T wgt = on ? ep[r] + eq : T(0);   // (E_p + E_q)/2 from the halved planes
                    // c_xy and c_yy vanish for (ox, 0), c_xx and c_xy for (0, oy)
                    if constexpr (oy == 0) {
                        ax[r] = dfma(wgt, ka * (upx[r] - wx[r + M]), ax[r]);
                    } else if constexpr (ox == 0) {
                        ay[r] = dfma(wgt, kb * (upy[r] - wy[r + M + oy]), ay[r]);
                    } else {
                        const T dx = upx[r] - wx[r + M + oy];
                        const T dy = upy[r] - wy[r + M + oy];
                        const T t = wgt * dfma(T(oy), dy, T(ox) * dx);   // w_pq (o . d)
                        ax[r] = dfma(t, ka, ax[r]);
                        ay[r] = dfma(t, kb, ay[r]);
                    }
                }
            }
        });
    });
    T dot = T(0);   // per-thread partial in the kernel's precision; FP64 only across threads
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gy = y0 + ty * R + r;
        if (gx < nx && gy < ny) {
            const int64_t p = (int64_t)gy * nx + gx;
            T fx = ax[r], fy = ay[r];
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) fx = T(0);
                if (m & 2) fy = T(0);
            }
            fx *= scale;
            fy *= scale;
            ob[p] = fx;
            ob[N + p] = fy;
            dot = dfma(upx[r], fx, dfma(upy[r], fy, dot));
        }
    }
    if (dot_partial)
        finish_block_dot(dot, dot_partial, dot_out, retire, gridDim.x * gridDim.y,
                         blockIdx.x + gridDim.x * blockIdx.y, b);
}

namespace {

template <typename T, int M>
BondTab2<T, M> make_bond2(const pd_grid *g)
{
    BondTab2<T, M> t{};
    double c[6];
    for (int k = 0; k < g->nnb; ++k) {
        const int ox = g->off[3 * k], oy = g->off[3 * k + 1];
        coef_of(g, ox, oy, 0, g->has_E, c);
        if (ox != 0 && oy != 0) {   // c_xx = kappa ox^2: kappa ox = c_xx / ox, kappa oy = kappa ox * oy / ox
            const double kappa = c[0] / ((double)ox * ox);
            t.v[2 * k] = (T)(kappa * ox);
            t.v[2 * k + 1] = (T)(kappa * oy);
        } else {
            t.v[2 * k] = (T)c[0];
            t.v[2 * k + 1] = (T)c[2];
        }
    }
    return t;
}

template <typename T, int M>
int run(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    constexpr int R = rows2d_direct<T, M>();
    constexpr int TY = kGY2 * R;
    const size_t smem = sizeof(T) * 3 * (kTX2 + 2 * M) * (TY + 2 * M);
    auto kern = k_direct2d<T, M>;
    allow_smem(kern, smem);
    dim3 grid((unsigned)((g->n[0] + kTX2 - 1) / kTX2), (unsigned)((g->n[1] + TY - 1) / TY), (unsigned)a.batch);
    kern<<<grid, kThreads, smem, s>>>((const T *)a.u, (T *)a.out, (int)g->n[0], (int)g->n[1], g->N, g->d_cons,
                                      a.project ? 1 : 0, g->has_E ? g->d_E : nullptr,
                                      a.use_mu ? g->d_mask : nullptr, (T)a.scale, make_bond2<T, M>(g),
                                      a.dot_partial, a.dot_out, a.retire);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <typename T>
int run_t(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    switch (g->M) {
        case 1: return run<T, 1>(g, a, s);
        case 2: return run<T, 2>(g, a, s);
        case 3: return run<T, 3>(g, a, s);
        case 4: return run<T, 4>(g, a, s);
        case 5: return run<T, 5>(g, a, s);
        case 6: return run<T, 6>(g, a, s);
        case 7: return run<T, 7>(g, a, s);
        case 8: return run<T, 8>(g, a, s);
    }
    return fail(PD_ERR_INVALID, "horizon M not compiled for 2D");
}

}  // namespace

int run_direct2d(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s)
{
    return f64 ? run_t<double>(g, a, s) : run_t<float>(g, a, s);
}

}  // namespace pd

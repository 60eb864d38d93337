// pd_stencil2d.cu -- 2D stencil (Eq. mat:f1; the TBT structure of Sec. 3.2-3.4),
// FP64 and FP32 (the FP32 grids that the TMA-fed kernel does not take).
//
// The product is the in-grid bond sum taken as differences:
//     (K u)_p = -sum_{o in half} c(o) [m_{p+o} (u_{p+o} - u_p) + m_{p-o} (u_{p-o} - u_p)],
// m = 1 inside the grid and 0 outside.  It equals the TBT form
// Kd_p u_p - sum_o c(o) u~_{p+o} (the diagonal block Kd_p = sum of c(o) over the
// in-grid offsets, which folds in the edge self-term D^e of Eq. tea:sc), but
// has no diagonal term to cancel against, so that the rounding error stays
// relative to |K u| on smooth fields and on fields with a large constant part.
//
// Tiling: a CTA owns 64 x (4R) outputs; each of its 256 threads owns a column
// of R consecutive y outputs.  The (64 + 2M) x (4R + 2M) halo box of both
// components is staged in shared memory once; a thread walks its column offsets
// and, for each, applies every (ox, oy) pair to its R outputs.  Block entries
// that vanish by geometry (c_xy and c_yy of (ox, 0), c_xx and c_xy of (0, oy))
// are skipped at compile time.  PD_PAIR_FORM selects the pair form
// (k_tbt2d_pair, below).  The default FP64 product without a fused dot is the
// pair form on u minus the box's plane (k_tbt2d_pair<double, M, true>), which
// keeps the rounding relative to |K u| at less arithmetic than the difference
// form (PD_ACCURATE selects the latter in FP64).
//
// Row windows (pd_matvec_rows): the staged rows are those the input holds,
// [in_row0, in_end); rows of the grid outside them enter only outputs that the
// launch does not write.
#include "pd_stencil.cuh"

namespace pd {

constexpr int gcd_c(int a, int b) { return b == 0 ? (a < 0 ? -a : a) : gcd_c(b, a % b); }

// Pair blocks (xx, xy, yy) in pair_index2 order, then per k = 1..M the summed
// vertical block Cbar(k) = sum of c(o) over the pairs with |oy| = k (xx, yy).
template <typename T, int M>
struct PlainTab {
    static constexpr int kPairs = count_offsets(2, M) / 2;
    T v[3 * kPairs + 2 * M];
};

// Interior outputs (every neighbour inside the grid): the sums regrouped as in
// the FP32 TMA kernel's tile_eg -- per column offset ox the horizontal second
// differences E(i) = (u(x+ox,i) - u(x,i)) + (u(x-ox,i) - u(x,i)) and central
// differences G(i) = u(x+ox,i) - u(x-ox,i) of each window row, shared by the
// thread's R outputs; pairs (ox, k) and (ox, -k) together as
// cxx (E(r+k) + E(r-k)) + cxy (G(r+k) - G(r-k)) (x component; y alike); the
// vertical second differences of the own column once per k with Cbar(k).
template <typename T, int M, int R, int SX>
__device__ __forceinline__ void plain_eg(const T *colx, const T *coly, const PlainTab<T, M> &tab, T (&ax)[R],
                                         T (&ay)[R])
{
    constexpr int WL = R + 2 * M, NP = PlainTab<T, M>::kPairs;
    T wx[WL], wy[WL];
#pragma unroll
    for (int i = 0; i < WL; ++i) {
        wx[i] = colx[i * SX];
        wy[i] = coly[i * SX];
    }
    static_for<1, M + 1>([&](auto K) {
        constexpr int k = decltype(K)::value;
        const T cxx = tab.v[3 * NP + 2 * (k - 1)], cyy = tab.v[3 * NP + 2 * (k - 1) + 1];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = r + M;
            ax[r] = dfma(cxx, (wx[i + k] - wx[i]) + (wx[i - k] - wx[i]), ax[r]);
            ay[r] = dfma(cyy, (wy[i + k] - wy[i]) + (wy[i - k] - wy[i]), ay[r]);
        }
    });
    static_for<1, M + 1>([&](auto OX) {
        constexpr int ox = decltype(OX)::value;
        constexpr int My = isqrt_c(M * M - ox * ox);
        const T c0 = tab.v[3 * pair_index2(M, ox, 0)];
        T ex[WL], ey[WL], gx[WL], gy[WL];
#pragma unroll
        for (int i = M - My; i < R + M + My; ++i) {
            const T px = colx[i * SX + ox], mx = colx[i * SX - ox];
            ex[i] = (px - wx[i]) + (mx - wx[i]);
            if constexpr (My > 0) {
                const T py = coly[i * SX + ox], my = coly[i * SX - ox];
                ey[i] = (py - wy[i]) + (my - wy[i]);
                gx[i] = px - mx;
                gy[i] = py - my;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) ax[r] = dfma(c0, ex[r + M], ax[r]);   // axis pair (ox, 0)
        static_for<1, My + 1>([&](auto K) {
            constexpr int k = decltype(K)::value;
            constexpr int pi = pair_index2(M, ox, k);
            const T cxx = tab.v[3 * pi], cxy = tab.v[3 * pi + 1], cyy = tab.v[3 * pi + 2];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = r + M;
                ax[r] = dfma(cxx, ex[i + k] + ex[i - k], dfma(cxy, gy[i + k] - gy[i - k], ax[r]));
                ay[r] = dfma(cyy, ey[i + k] + ey[i - k], dfma(cxy, gx[i + k] - gx[i - k], ay[r]));
            }
        });
    });
}

template <typename T, int M>
__global__ void __launch_bounds__(kThreads)
k_tbt2d(const T *__restrict__ u, T *__restrict__ out, int nx, int ny, int64_t N,
        const uint8_t *__restrict__ cons, int project, T scale,
        PlainTab<T, M> tab, double *dot_partial, double *dot_out, unsigned int *retire,
        int in_row0, int in_end, int64_t Nin, int out_row0, int out_end)
{
    // Rows are grid rows; the input holds rows [in_row0, in_end) with plane size Nin, the
    // output rows [out_row0, out_end) with plane size N (the whole grid: 0, ny, N, 0, ny).
    constexpr int R = rows2d<T, M>();
    constexpr int TX = kTX2, TY = kGY2 * R, SX = TX + 2 * M, SY = TY + 2 * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_x = reinterpret_cast<T *>(smem_raw);
    T *s_y = s_x + SX * SY;

    const int64_t b = blockIdx.z;
    const T *ub = u + b * 2 * Nin - (int64_t)in_row0 * nx;   // indexed by grid node
    T *ob = out + b * 2 * N - (int64_t)out_row0 * nx;
    const int x0 = blockIdx.x * TX, y0 = out_row0 + blockIdx.y * TY;

    for (int t = threadIdx.x; t < SX * SY; t += kThreads) {
        const int r = t / SX, c = t - r * SX;
        const int gx = x0 - M + c, gy = y0 - M + r;
        T vx = T(0), vy = T(0);
        if (gx >= 0 && gx < nx && gy >= in_row0 && gy < in_end) {
            const int64_t p = (int64_t)gy * nx + gx;
            vx = __ldg(ub + p);
            vy = __ldg(ub + Nin + p);
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) vx = T(0);
                if (m & 2) vy = T(0);
            }
        }
        s_x[t] = vx;
        s_y[t] = vy;
    }
    __syncthreads();

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const T *colx = s_x + (ty * R) * SX + tx + M;   // (row0, col) of this thread's column
    const T *coly = s_y + (ty * R) * SX + tx + M;
    T ax[R], ay[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { ax[r] = T(0); ay[r] = T(0); }
    {
        const int gxt = x0 + tx, gyw = y0 + ty * R - M;   // grid column, grid row of window row 0
        T ux[R], uy[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            ux[r] = colx[(r + M) * SX];
            uy[r] = coly[(r + M) * SX];
        }
        // warps whose outputs all keep their horizon inside the grid take the shared
        // differences; the others the plain differences with out-of-grid terms dropped
        const bool warp_in = __all_sync(0xffffffffu, gxt >= M && gxt < nx - M) && gyw >= 0 && gyw + R + 2 * M <= ny;
        if (warp_in) plain_eg<T, M, R, SX>(colx, coly, tab, ax, ay);
        // Differences, terms with the neighbour outside the grid dropped.  The
        // staged value there is zero, so m (v - u_p) = v - m u_p (one FMA).
        if (!warp_in) static_for<0, M + 1>([&](auto OX) {
            constexpr int ox = decltype(OX)::value;
            constexpr int My = isqrt_c(M * M - ox * ox);
            const bool cp = gxt + ox < nx, cm = gxt - ox >= 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                static_for<-My, My + 1>([&](auto OY) {
                    constexpr int oy = decltype(OY)::value;
                    if constexpr (ox > 0 || oy > 0) {
                        constexpr int pi = pair_index2(M, ox, oy);
                        const int ip = r + M + oy, im = r + M - oy;
                        const T np = (cp && gyw + ip >= 0 && gyw + ip < ny) ? T(-1) : T(0);
                        const T nm = (cm && gyw + im >= 0 && gyw + im < ny) ? T(-1) : T(0);
                        const T sx = dfma(np, ux[r], colx[ip * SX + ox]) + dfma(nm, ux[r], colx[im * SX - ox]);
                        const T sy = dfma(np, uy[r], coly[ip * SX + ox]) + dfma(nm, uy[r], coly[im * SX - ox]);
                        const T cxx = tab.v[3 * pi], cyy = tab.v[3 * pi + 2];
                        if constexpr (oy == 0) {
                            ax[r] = dfma(cxx, sx, ax[r]);   // axis pair (ox, 0): c_xy = c_yy = 0
                        } else if constexpr (ox == 0) {
                            ay[r] = dfma(cyy, sy, ay[r]);   // axis pair (0, oy): c_xx = c_xy = 0
                        } else {
                            const T cxy = tab.v[3 * pi + 1];
                            ax[r] = dfma(cxx, sx, dfma(cxy, sy, ax[r]));
                            ay[r] = dfma(cxy, sx, dfma(cyy, sy, ay[r]));
                        }
                    }
                });
            }
        });
        T dot = T(0);
        const int gx = x0 + tx;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int gy = y0 + ty * R + r;
            if (gx < nx && gy < out_end) {
                const int64_t p = (int64_t)gy * nx + gx;
                T fx = -ax[r], fy = -ay[r];
                if (project) {
                    const uint8_t m = __ldg(cons + p);
                    if (m & 1) fx = T(0);
                    if (m & 2) fy = T(0);
                }
                fx *= scale;
                fy *= scale;
                ob[p] = fx;
                ob[N + p] = fy;
                dot = dfma(ux[r], fx, dfma(uy[r], fy, dot));
            }
        }
        if (dot_partial)
            finish_block_dot(dot, dot_partial, dot_out, retire, gridDim.x * gridDim.y,
                             blockIdx.x + gridDim.x * blockIdx.y, b);
    }
}


// The box's reference plane (k_tbt2d_pair<double, M, true>).  The pair form's
// rounding error is relative to the staged values, so a field with a large
// constant part or gradient loses digits of K u; the box's least-squares plane
// L is subtracted first, leaving the field's curvature part.  K maps a plane to
// zero at every node with a full horizon, and at a node near a face to
// -sum_b (Tx_ab gx_b + Ty_ab gy_b), Tx_ab = sum of c_ab(o) o_x over the in-grid
// offsets (Ty alike with o_y): the first-moment table of the node's edge class.
// L is quantised so that its value at every box node is exact in FP64:
// L = q (L0 + Gx (c - ar) + Gy (r - rr)) with q a power of two and integers
// below 2^53 -- the kernel then forms K (u - L) from exactly u - L (rounded
// once), and K u = K (u - L) + K L holds to rounding.
//
// Warp 0 fits the plane in FP32 to an 8 x 8 sample of the box's in-window
// rectangle [ca, cb) x [ra, rb) (box coordinates; fetch(c, r, vx, vy) reads a
// node; any plane serves, the fit only has to follow the field closely),
// quantises it in FP64 and writes the plane's row and column parts:
// lr[c][r] = q (L0 + Gy (r - rr)), lc[c][k] = q Gx (k - ar), whose sums are exact,
// and the per-node gradients g = (q Gx_x, q Gy_x, q Gx_y, q Gy_y).  The caller's
// next block barrier makes them visible to every thread.
template <int SX, int SY, typename F>
__device__ __forceinline__ void box_plane(F fetch, int ca, int cb, int ra, int rb,
                                          double (*lr)[SY], double (*lc)[SX], double *g)
{
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x, wx = cb - ca, wy = rb - ra;
    float mx = 0.f, my = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        mx += (float)(ca + (i * (wx - 1)) / 7);
        my += (float)(ra + (i * (wy - 1)) / 7);
    }
    mx *= 0.125f;
    my *= 0.125f;
    float sxx = 0.f, syy = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float dx = (float)(ca + (i * (wx - 1)) / 7) - mx, dy = (float)(ra + (i * (wy - 1)) / 7) - my;
        sxx = fmaf(dx, dx, sxx);
        syy = fmaf(dy, dy, syy);
    }
    float sm[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane & 7, j = (lane >> 3) + 4 * h;
        const int c = ca + (i * (wx - 1)) / 7, r = ra + (j * (wy - 1)) / 7;
        float vx, vy;
        fetch(c, r, vx, vy);
        const float dx = (float)c - mx, dy = (float)r - my;
        sm[0] += vx;
        sm[1] = fmaf(vx, dx, sm[1]);
        sm[2] = fmaf(vx, dy, sm[2]);
        sm[3] += vy;
        sm[4] = fmaf(vy, dx, sm[4]);
        sm[5] = fmaf(vy, dy, sm[5]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sm[k] += __shfl_xor_sync(0xffffffffu, sm[k], o);
    const float ix = sxx > 0.f ? 0.125f / sxx : 0.f, iy = syy > 0.f ? 0.125f / syy : 0.f;
    const int ar = ca + (wx - 1) / 2, rr = ra + (wy - 1) / 2;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const double gx = (double)(sm[3 * c + 1] * ix), gy = (double)(sm[3 * c + 2] * iy);
        const double l = (double)(sm[3 * c] * (1.f / 64.f) + (float)gx * ((float)ar - mx) + (float)gy * ((float)rr - my));
        const double bound = fabs(l) + 64.0 * (fabs(gx) + fabs(gy));
        double Q0 = 0.0, Gx = 0.0, Gy = 0.0;
        // q = 2^(k - 50) with bound < 2^k (from the exponent field), and 1/q exactly; box
        // offsets from (ar, rr) are below 80, so |L0| + 80 (|Gx| + |Gy|) < 2^53
        const long long eb = (__double_as_longlong(bound) >> 52) & 0x7ff;
        if (bound > 1e-280 && eb < 2000) {
            const double q = __longlong_as_double((eb - 49) << 52);
            const double iq = __longlong_as_double((2095 - eb) << 52);
            Q0 = q * rint(l * iq);
            Gx = q * rint(gx * iq);
            Gy = q * rint(gy * iq);
        }
        for (int k = lane; k < SX; k += 32) lc[c][k] = Gx * (double)(k - ar);
        for (int k = lane; k < SY; k += 32) lr[c][k] = fma(Gy, (double)(k - rr), Q0);
        if (lane == 0) {
            g[2 * c] = Gx;
            g[2 * c + 1] = Gy;
        }
    }
}

// The pair form  (K u)_p = Kd_p u_p - sum_{o in half} c(o) (u~_{p+o} + u~_{p-o})
// (u~ zero outside the grid, Kd_p the diagonal block over the in-grid offsets
// from the clipped-distance table, which folds in the edge self-term D^e of
// Eq. tea:sc).  Fewer operations than the difference form.  On u itself
// (PD_PAIR_FORM, PLANE false) its rounding error is relative to sum |c| |u|
// rather than |K u| (in FP64, on the full-horizon interior of smooth 1024^2
// fields, 1e-11 with a large constant part and 3e-10 with a large gradient):
// used where a solver's own tolerance is far above that, e.g.
// the FP64 CG and ADR iterations.  On u minus the box's plane (PLANE, FP64, no
// fused dot; box_plane) it is the default FP64 product.
template <typename T, int M, bool PLANE>
__global__ void __launch_bounds__(kThreads, (PLANE && M <= 4) ? 3 : 1)
k_tbt2d_pair(const T *__restrict__ u, T *__restrict__ out, int nx, int ny, int64_t N,
             const uint8_t *__restrict__ cons, int project, const T *__restrict__ kd, const T *__restrict__ kt,
             T scale, PairTab<T, 2, M> tab, double *dot_partial, double *dot_out, unsigned int *retire,
             int in_row0, int in_end, int64_t Nin, int out_row0, int out_end)
{
    static_assert(!PLANE || sizeof(T) == 8, "the box plane is formed in FP64");
    constexpr int R = rows2d<T, M>();
    constexpr int TX = kTX2, TY = kGY2 * R, SX = TX + 2 * M, SY = TY + 2 * M, WL = R + 2 * M;
    constexpr int NP = PairTab<T, 2, M>::kPairs;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_x = reinterpret_cast<T *>(smem_raw);
    T *s_y = s_x + SX * SY;

    const int64_t b = blockIdx.z;
    const T *ub = u + b * 2 * Nin - (int64_t)in_row0 * nx;   // indexed by grid node
    T *ob = out + b * 2 * N - (int64_t)out_row0 * nx;
    const int x0 = blockIdx.x * TX, y0 = out_row0 + blockIdx.y * TY;

    constexpr int PX = PLANE ? SX : 1, PY = PLANE ? SY : 1;
    __shared__ double s_lr[2][PY], s_lc[2][PX], s_g[4];
    if constexpr (PLANE) {
        // the plane from the box's in-window rectangle, before staging
        const int ca = max(0, M - x0), cb = min(SX, nx - x0 + M);
        const int ra = max(0, in_row0 - y0 + M), rb = min(SY, in_end - y0 + M);
        box_plane<SX, SY>([&](int c, int r, float &fx, float &fy) {
            const int64_t p = (int64_t)(y0 - M + r) * nx + (x0 - M + c);
            T vx = __ldg(ub + p), vy = __ldg(ub + Nin + p);
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) vx = T(0);
                if (m & 2) vy = T(0);
            }
            fx = (float)vx;
            fy = (float)vy;
        }, ca, cb, ra, rb, s_lr, s_lc, s_g);
        __syncthreads();
    }
    for (int t = threadIdx.x; t < SX * SY; t += kThreads) {
        const int r = t / SX, c = t - r * SX;
        const int gx = x0 - M + c, gy = y0 - M + r;
        T vx = T(0), vy = T(0);
        if (gx >= 0 && gx < nx && gy >= in_row0 && gy < in_end) {
            const int64_t p = (int64_t)gy * nx + gx;
            vx = __ldg(ub + p);
            vy = __ldg(ub + Nin + p);
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) vx = T(0);
                if (m & 2) vy = T(0);
            }
            if constexpr (PLANE) {
                vx -= s_lr[0][r] + s_lc[0][c];
                vy -= s_lr[1][r] + s_lc[1][c];
            }
        }
        s_x[t] = vx;
        s_y[t] = vy;
    }
    __syncthreads();
    [[maybe_unused]] T pg[4];   // the plane's per-node gradients (PLANE)
    if constexpr (PLANE) {
#pragma unroll
        for (int k = 0; k < 4; ++k) pg[k] = s_g[k];
    }

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const T *colx = s_x + (ty * R) * SX + tx + M;   // (row0, col) of this thread's column
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
            // rank-one block c(o) = kappa o o^T with o = g (ax_, ay_), g = gcd: the pair adds
            // (kappa g o) (ax_ sx + ay_ sy); the table holds kappa g o (the axis pair: c_xx)
            constexpr int gd = gcd_c(ox, oy), ax_ = ox / gd, ay_ = oy / gd;
            const T ka = tab.v[3 * pi], kb = tab.v[3 * pi + 1];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T sx = px[r + M + oy] + mx[r + M - oy];
                if constexpr (oy == 0) {
                    ax[r] = dfma(ka, sx, ax[r]);   // axis pair: c_xy = c_yy = 0 exactly
                } else {
                    const T sy = py[r + M + oy] + my[r + M - oy];
                    T d;
                    if constexpr (ax_ == 1) d = dfma(T(ay_), sy, sx);
                    else if constexpr (ay_ == 1 || ay_ == -1) d = dfma(T(ax_), sx, T(ay_) * sy);
                    else d = dfma(T(ay_), sy, T(ax_) * sx);
                    ax[r] = dfma(ka, d, ax[r]);
                    ay[r] = dfma(kb, d, ay[r]);
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
        const T cyy = tab.v[3 * pi + 2];   // axis pair: c_xx = c_xy = 0 exactly
#pragma unroll
        for (int r = 0; r < R; ++r) ay[r] = dfma(cyy, cy[r + M + oy] + cy[r + M - oy], ay[r]);
    });

    const int gx = x0 + tx;
    T fx[R], fy[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gy = y0 + ty * R + r;
        const T upx = cx[r + M], upy = cy[r + M];
        T kxx = tab.v[3 * NP], kxy = tab.v[3 * NP + 1], kyy = tab.v[3 * NP + 2];
        const int a0 = min(gx, M), a1 = min(nx - 1 - gx, M), b0 = min(gy, M), b1 = min(ny - 1 - gy, M);
        if ((a0 != M || a1 != M || b0 != M || b1 != M) && gx < nx && gy < out_end) {
            const int cls = ((a0 * (M + 1) + a1) * (M + 1) + b0) * (M + 1) + b1;
            kxx = __ldg(kd + 3 * cls);
            kxy = __ldg(kd + 3 * cls + 1);
            kyy = __ldg(kd + 3 * cls + 2);
        }
        fx[r] = dfma(kxx, upx, dfma(kxy, upy, -ax[r]));
        fy[r] = dfma(kxy, upx, dfma(kyy, upy, -ay[r]));
    }
    if constexpr (PLANE) {
        // K L at the nodes near a face, on the tiles that hold some (a block-uniform branch,
        // so that interior tiles do not execute it under a predicate)
        if (x0 < M || x0 + TX > nx - M || y0 < M || y0 + TY > ny - M) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int gy = y0 + ty * R + r;
                const int a0 = min(gx, M), a1 = min(nx - 1 - gx, M), b0 = min(gy, M), b1 = min(ny - 1 - gy, M);
                if ((a0 != M || a1 != M || b0 != M || b1 != M) && gx < nx && gy < out_end) {
                    const int cls = ((a0 * (M + 1) + a1) * (M + 1) + b0) * (M + 1) + b1;
                    const T *t6 = kt + 6 * cls;   // Tx_xx, Tx_xy, Tx_yy, Ty_xx, Ty_xy, Ty_yy
                    fx[r] -= __ldg(t6) * pg[0] + __ldg(t6 + 3) * pg[1] + __ldg(t6 + 1) * pg[2] + __ldg(t6 + 4) * pg[3];
                    fy[r] -= __ldg(t6 + 1) * pg[0] + __ldg(t6 + 4) * pg[1] + __ldg(t6 + 2) * pg[2] + __ldg(t6 + 5) * pg[3];
                }
            }
        }
    }

    T dot = T(0);   // per-thread partial in the kernel's precision; FP64 only across threads
    const bool scaled = scale != T(1);   // a product by one is exact: skipped
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gy = y0 + ty * R + r;
        if (gx < nx && gy < out_end) {
            const int64_t p = (int64_t)gy * nx + gx;
            T ox = fx[r], oy = fy[r];
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) ox = T(0);
                if (m & 2) oy = T(0);
            }
            if (scaled) {
                ox *= scale;
                oy *= scale;
            }
            ob[p] = ox;
            ob[N + p] = oy;
            dot = dfma(cx[r + M], ox, dfma(cy[r + M], oy, dot));
        }
    }
    if (dot_partial)
        finish_block_dot(dot, dot_partial, dot_out, retire, gridDim.x * gridDim.y,
                         blockIdx.x + gridDim.x * blockIdx.y, b);
}

namespace {

template <typename T, int M>
PlainTab<T, M> make_plain(const pd_grid *g)
{
    PlainTab<T, M> t{};
    constexpr int NP = PlainTab<T, M>::kPairs;
    double c[6], wb[M + 1][2] = {};
    auto put = [&](int ox, int oy) {
        const int pi = pair_index2(M, ox, oy);
        coef_of(g, ox, oy, 0, false, c);
        for (int i = 0; i < 3; ++i) t.v[3 * pi + i] = (T)c[i];
        const int k = oy < 0 ? -oy : oy;
        if (k > 0) {
            wb[k][0] += c[0];
            wb[k][1] += c[2];
        }
    };
    for (int ox = 1; ox <= M; ++ox) {
        const int My = isqrt_c(M * M - ox * ox);
        for (int oy = -My; oy <= My; ++oy) put(ox, oy);
    }
    for (int oy = 1; oy <= M; ++oy) put(0, oy);
    for (int k = 1; k <= M; ++k) {
        t.v[3 * NP + 2 * (k - 1)] = (T)wb[k][0];
        t.v[3 * NP + 2 * (k - 1) + 1] = (T)wb[k][1];
    }
    return t;
}

template <typename T, int M>
int run(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    constexpr int R = rows2d<T, M>();
    constexpr int TY = kGY2 * R;
    const size_t smem = sizeof(T) * 2 * (kTX2 + 2 * M) * (TY + 2 * M);
    auto kern = k_tbt2d<T, M>;
    allow_smem(kern, smem);
    const int64_t nx = g->n[0], ny = g->n[1];
    const int64_t in_rows = a.in_rows < 0 ? ny : a.in_rows, out_rows = a.out_rows < 0 ? ny : a.out_rows;
    if ((in_rows != ny || out_rows != ny) && a.dot_partial)
        return fail(PD_ERR_INVALID, "row windows take no fused dot");
    dim3 grid((unsigned)((nx + kTX2 - 1) / kTX2), (unsigned)((out_rows + TY - 1) / TY), (unsigned)a.batch);
    kern<<<grid, kThreads, smem, s>>>((const T *)a.u, (T *)a.out, (int)nx, (int)ny, out_rows * nx, g->d_cons,
                                      a.project ? 1 : 0, (T)a.scale, make_plain<T, M>(g), a.dot_partial,
                                      a.dot_out, a.retire, (int)a.in_row0, (int)(a.in_row0 + in_rows), in_rows * nx,
                                      (int)a.out_row0, (int)(a.out_row0 + out_rows));
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}


// The pair form's table: per pair (ox > 0, or ox = 0 < oy) kappa g (ox, oy) for pairs with
// both components nonzero (c(o) = kappa o o^T, g = gcd(ox, |oy|); k_tbt2d_pair applies it as
// kappa g o (o / g . s)), c_xx for (ox, 0) and c_yy (third slot) for (0, oy); then the
// interior diagonal Kd (sum of all c).
template <typename T, int M>
PairTab<T, 2, M> make_pairs2(const pd_grid *g)
{
    PairTab<T, 2, M> t{};
    double c[6], tot[3] = {0, 0, 0};
    auto put = [&](int ox, int oy) {
        const int pi = pair_index2(M, ox, oy);
        coef_of(g, ox, oy, 0, false, c);
        for (int i = 0; i < 3; ++i) {
            t.v[3 * pi + i] = (T)c[i];
            tot[i] += 2 * c[i];
        }
        if (ox != 0 && oy != 0) {
            const double kg = c[0] / ((double)ox * ox) * gcd_c(ox, oy);   // kappa g
            t.v[3 * pi] = (T)(kg * ox);
            t.v[3 * pi + 1] = (T)(kg * oy);
            t.v[3 * pi + 2] = T(0);
        }
    };
    for (int ox = 1; ox <= M; ++ox) {
        const int My = isqrt_c(M * M - ox * ox);
        for (int oy = -My; oy <= My; ++oy) put(ox, oy);
    }
    for (int oy = 1; oy <= M; ++oy) put(0, oy);
    constexpr int NP = PairTab<T, 2, M>::kPairs;
    for (int i = 0; i < 3; ++i) t.v[3 * NP + i] = (T)tot[i];
    return t;
}

template <typename T, int M, bool PLANE>
int run_pair(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    constexpr int R = rows2d<T, M>();
    constexpr int TY = kGY2 * R;
    const size_t smem = sizeof(T) * 2 * (kTX2 + 2 * M) * (TY + 2 * M);
    auto kern = k_tbt2d_pair<T, M, PLANE>;
    if (PLANE && a.dot_partial) return fail(PD_ERR_INVALID, "internal: the box plane takes no fused dot");
    allow_smem(kern, smem);
    const int64_t nx = g->n[0], ny = g->n[1];
    const int64_t in_rows = a.in_rows < 0 ? ny : a.in_rows, out_rows = a.out_rows < 0 ? ny : a.out_rows;
    if ((in_rows != ny || out_rows != ny) && a.dot_partial)
        return fail(PD_ERR_INVALID, "row windows take no fused dot");
    dim3 grid((unsigned)((nx + kTX2 - 1) / kTX2), (unsigned)((out_rows + TY - 1) / TY), (unsigned)a.batch);
    const T *kd = sizeof(T) == 4 ? (const T *)g->d_kd32 : (const T *)g->d_kd64;
    const T *kt = sizeof(T) == 4 ? (const T *)g->d_kt32 : (const T *)g->d_kt64;
    kern<<<grid, kThreads, smem, s>>>((const T *)a.u, (T *)a.out, (int)nx, (int)ny, out_rows * nx, g->d_cons,
                                      a.project ? 1 : 0, kd, kt, (T)a.scale, make_pairs2<T, M>(g), a.dot_partial,
                                      a.dot_out, a.retire, (int)a.in_row0, (int)(a.in_row0 + in_rows), in_rows * nx,
                                      (int)a.out_row0, (int)(a.out_row0 + out_rows));
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <typename T>
int run_t(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    if (a.pair_form) {
        switch (g->M) {
            case 1: return run_pair<T, 1, false>(g, a, s);
            case 2: return run_pair<T, 2, false>(g, a, s);
            case 3: return run_pair<T, 3, false>(g, a, s);
            case 4: return run_pair<T, 4, false>(g, a, s);
            case 5: return run_pair<T, 5, false>(g, a, s);
            case 6: return run_pair<T, 6, false>(g, a, s);
            case 7: return run_pair<T, 7, false>(g, a, s);
            case 8: return run_pair<T, 8, false>(g, a, s);
        }
        return fail(PD_ERR_INVALID, "horizon M not compiled for 2D");
    }
    if constexpr (sizeof(T) == 8) {
        // FP64 default: the pair form on u minus the box's plane; the difference form
        // with a fused dot or on request (PD_ACCURATE)
        if (!a.dot_partial && !a.accurate) {
            switch (g->M) {
                case 1: return run_pair<T, 1, true>(g, a, s);
                case 2: return run_pair<T, 2, true>(g, a, s);
                case 3: return run_pair<T, 3, true>(g, a, s);
                case 4: return run_pair<T, 4, true>(g, a, s);
                case 5: return run_pair<T, 5, true>(g, a, s);
                case 6: return run_pair<T, 6, true>(g, a, s);
                case 7: return run_pair<T, 7, true>(g, a, s);
                case 8: return run_pair<T, 8, true>(g, a, s);
            }
            return fail(PD_ERR_INVALID, "horizon M not compiled for 2D");
        }
    }
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

int run_tbt2d(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s)
{
    return f64 ? run_t<double>(g, a, s) : run_t<float>(g, a, s);
}

}  // namespace pd

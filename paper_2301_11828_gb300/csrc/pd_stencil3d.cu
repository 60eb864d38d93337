// pd_stencil3d.cu -- 3D stencil, TBTBT form (Sec. 4).
//
// Same operator as the 2D TBT form with 3x3 blocks (six unique reals per
// offset, Eq. mae:e1):  (K u)_p = Kd_p u_p - sum_{o != 0} c(o) u~_{p+o}, summed
// over offset pairs.  A CTA owns 32 x 8 x R outputs; a thread owns a z-column
// of R outputs.  The (32 + 2M) x (8 + 2M) x (R + 2M) halo box of the three
// components is staged in shared memory; for each (ox, oy) column pair the
// thread loads the z-windows of columns (x+ox, y+oy) and (x-ox, y-oy).
// DIFF (the FP32 default; PD_PAIR_FORM selects the pair form) sums
// (u_{p+o} - u_p) + (u_{p-o} - u_p) over the in-grid neighbours instead of
// u~_{p+o} + u~_{p-o} against Kd u_p: the FP32 error is then relative to |K u|
// on smooth fields too, and K u = -sum (no diagonal term to cancel against).
#include "pd_stencil.cuh"

namespace pd {

// acc[.][r] += c(o) s for one offset pair, s = u~_{p+o} + u~_{p-o}.  Entry c_ab
// carries the factor o_a o_b, so it vanishes exactly when o_a or o_b is zero;
// the flags (compile-time constants once the loops are unrolled) skip those
// entries and the sums they would need.  Kept terms run in the order
// c_xz, c_xy, c_xx / c_yz, c_yy, c_xy / c_zz, c_yz, c_xz.
template <typename T, int R>
__device__ __forceinline__ void pair3(T (&acc)[3][R], int r, bool nx_, bool ny_, bool nz_, T cxx, T cxy, T cxz,
                                      T cyy, T cyz, T czz, T s0, T s1, T s2)
{
    if (nx_) {
        T a = acc[0][r];
        if (nz_) a = dfma(cxz, s2, a);
        if (ny_) a = dfma(cxy, s1, a);
        acc[0][r] = dfma(cxx, s0, a);
    }
    if (ny_) {
        T a = acc[1][r];
        if (nz_) a = dfma(cyz, s2, a);
        a = dfma(cyy, s1, a);
        if (nx_) a = dfma(cxy, s0, a);
        acc[1][r] = a;
    }
    if (nz_) {
        T a = dfma(czz, s2, acc[2][r]);
        if (ny_) a = dfma(cyz, s1, a);
        if (nx_) a = dfma(cxz, s0, a);
        acc[2][r] = a;
    }
}

// Rank-one application of a pair's block (FP64 pair form): c(o) = kappa o o^T, so for an
// offset with two or three nonzero components acc += (kappa g o) d with d = (o / g) . s
// (g the gcd of the components): the reduced dot product takes one operation per nonzero
// component after the first (additions for components +-1), then one FMA per nonzero
// component, instead of the block's products.  k[] holds kappa g o.
constexpr int gcd3_c(int a, int b) { return b == 0 ? (a < 0 ? -a : a) : gcd3_c(b, a % b); }

template <int A, typename T> __device__ __forceinline__ T rk_first(T s)
{
    if constexpr (A == 1) return s;
    else if constexpr (A == -1) return -s;
    else return T(A) * s;
}
template <int A, typename T> __device__ __forceinline__ T rk_add(T s, T d)
{
    if constexpr (A == 1) return d + s;
    else if constexpr (A == -1) return d - s;
    else return dfma(T(A), s, d);
}

template <int OX, int OY, int OZ, typename T, int R>
__device__ __forceinline__ void pair3_rank1(T (&acc)[3][R], int r, const T *k, T s0, T s1, T s2)
{
    constexpr int g = gcd3_c(gcd3_c(OX, OY), OZ), ax = OX / g, ay = OY / g, az = OZ / g;
    T d;
    if constexpr (ax != 0) {
        d = rk_first<ax>(s0);
        if constexpr (ay != 0) d = rk_add<ay>(s1, d);
        if constexpr (az != 0) d = rk_add<az>(s2, d);
    } else {
        d = rk_first<ay>(s1);
        d = rk_add<az>(s2, d);
    }
    if constexpr (ax != 0) acc[0][r] = dfma(k[0], d, acc[0][r]);
    if constexpr (ay != 0) acc[1][r] = dfma(k[1], d, acc[1][r]);
    if constexpr (az != 0) acc[2][r] = dfma(k[2], d, acc[2][r]);
}

// Accurate (difference) form of the bond sum for one thread's z-column of R
// outputs.  For a column pair (ox, oy) let H+(i) = u(x+ox, y+oy, i) - u(x, y, i)
// and H-(i) = u(x-ox, y-oy, i) - u(x, y, i) (plane i of the window), and in the
// own column V_k(r) = u(r + k) - u(r).  The pair sum of offset (ox, oy, oz) is
//   s = H+(r + oz) + H-(r - oz) + V_oz(r) + V_-oz(r),
// so the windows of the column pair are turned into H+- once per plane and the
// vertical parts of every pair with |oz| = k are summed once per output:
//   Cbar(k) (V_k(r) + V_-k(r)),  Cbar(k) = c(0,0,k) + sum over column pairs of
//   c(ox,oy,k) + c(ox,oy,-k)  (diagonal: xz, yz flip sign with oz, xy cancel
//   between (ox, oy) and (-ox, oy)).
// Every operand is a difference of nearby values, so the FP32 error stays
// relative to |K u| on smooth fields.  MASK (some neighbour of the warp leaves the
// grid): H+- carry the lane's in-grid flags m+- of the two columns, and for the
// pairs (ox, oy, +-k) of one column pair the vertical parts combine to
//   S (m+ + m-) (A + B) + Q (m+ - m-) (A - B),
// A = v(r+k) V_k(r), B = v(r-k) V_-k(r) (v: the plane lies in the grid), S the
// xx/xy/yy/zz and Q the xz/yz entries of c(ox, oy, k): per-lane coefficients
// cb (xx, xy, yy, zz) and dq (xz, yz).  Out-of-grid planes are zero in the box,
// so their H vanish by themselves.  acc receives sum c(o) s (K u = -acc).
template <typename T, int M, bool MASK>
__device__ __forceinline__ void diff3_column(const T *base, const PairTab<T, 3, M> &tab, int gx, int gy, int nx,
                                             int ny, uint32_t zok, T (&acc)[3][rows3d<T, M, true>()])
{
    constexpr int R = rows3d<T, M, true>();
    constexpr int SX = kTX3 + 2 * M, SY = kTY3 + 2 * M, SZ = R + 2 * M;
    constexpr int PL = SX * SY * SZ;
    T w0[3][SZ];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < SZ; ++i) w0[c][i] = base[c * PL + i * SX * SY];
    // per-lane vertical coefficients (all flags 1 on interior warps)
    T cb[M][4], dq[M][2];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const T *cc = tab.v + 6 * pair_index3(M, 0, 0, k + 1);
        cb[k][0] = cb[k][1] = cb[k][2] = T(0);
        cb[k][3] = cc[5];
        dq[k][0] = dq[k][1] = T(0);
    }
    static_for<0, M + 1>([&](auto OYI) {
        constexpr int oy = M - decltype(OYI)::value;
        constexpr int Mx = isqrt_c(M * M - oy * oy);
        static_for<-Mx, Mx + 1>([&](auto OX) {
            constexpr int ox = decltype(OX)::value;
            if constexpr (oy > 0 || ox > 0) {
                constexpr int Mz = isqrt_c(M * M - ox * ox - oy * oy);
                T mp = T(1), mm = T(1);
                if constexpr (MASK) {
                    mp = (gx + ox >= 0 && gx + ox < nx && gy + oy < ny) ? T(1) : T(0);
                    mm = (gx - ox >= 0 && gx - ox < nx && gy - oy >= 0) ? T(1) : T(0);
                }
                static_for<1, Mz + 1>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    const T *cc = tab.v + 6 * pair_index3(M, ox, oy, k);   // xx, xy, xz, yy, yz, zz
                    const T sp = mp + mm, sq = mp - mm;
                    cb[k - 1][0] = dfma(sp, cc[0], cb[k - 1][0]);
                    cb[k - 1][1] = dfma(sp, cc[1], cb[k - 1][1]);
                    cb[k - 1][2] = dfma(sp, cc[3], cb[k - 1][2]);
                    cb[k - 1][3] = dfma(sp, cc[5], cb[k - 1][3]);
                    dq[k - 1][0] = dfma(sq, cc[2], dq[k - 1][0]);
                    dq[k - 1][1] = dfma(sq, cc[4], dq[k - 1][1]);
                });
                // H+- over the planes the pairs of this column reach, formed once per plane;
                // outputs in the outer loop so that only 2 Mz + 1 planes of H are live at a time
                constexpr int NW = R + 2 * Mz, I0 = M - Mz;
                T hp[3][NW], hm[3][NW];
                auto form = [&](int j) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int i = I0 + j;
                        const T a = base[c * PL + i * SX * SY + oy * SX + ox] - w0[c][i];
                        const T b = base[c * PL + i * SX * SY - oy * SX - ox] - w0[c][i];
                        hp[c][j] = MASK ? mp * a : a;
                        hm[c][j] = MASK ? mm * b : b;
                    }
                };
#pragma unroll
                for (int j = 0; j < 2 * Mz; ++j) form(j);
                constexpr int pbase = pair_index3(M, ox, oy, 0);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    form(r + 2 * Mz);
#pragma unroll
                    for (int oz = -Mz; oz <= Mz; ++oz) {
                        const T *cf = tab.v + 6 * (pbase + oz);
                        pair3(acc, r, ox != 0, oy != 0, oz != 0, cf[0], cf[1], cf[2], cf[3], cf[4], cf[5],
                              hp[0][r + Mz + oz] + hm[0][r + Mz - oz], hp[1][r + Mz + oz] + hm[1][r + Mz - oz],
                              hp[2][r + Mz + oz] + hm[2][r + Mz - oz]);
                    }
                }
            }
        });
    });
    // vertical parts
#pragma unroll
    for (int k = 1; k <= M; ++k) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            T A[3], B[3];
            const bool va = !MASK || ((zok >> (r + M + k)) & 1u), vb = !MASK || ((zok >> (r + M - k)) & 1u);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                A[c] = va ? w0[c][r + M + k] - w0[c][r + M] : T(0);
                B[c] = vb ? w0[c][r + M - k] - w0[c][r + M] : T(0);
            }
            const T W0 = A[0] + B[0], W1 = A[1] + B[1], W2 = A[2] + B[2];
            const T *q = cb[k - 1];
            if constexpr (MASK) {
                const T C0 = A[0] - B[0], C1 = A[1] - B[1], C2 = A[2] - B[2];
                acc[0][r] = dfma(dq[k - 1][0], C2, dfma(q[1], W1, dfma(q[0], W0, acc[0][r])));
                acc[1][r] = dfma(dq[k - 1][1], C2, dfma(q[1], W0, dfma(q[2], W1, acc[1][r])));
                acc[2][r] = dfma(dq[k - 1][1], C1, dfma(dq[k - 1][0], C0, dfma(q[3], W2, acc[2][r])));
            } else {   // the xy entry of Cbar is exactly zero on interior warps
                acc[0][r] = dfma(q[0], W0, acc[0][r]);
                acc[1][r] = dfma(q[2], W1, acc[1][r]);
                acc[2][r] = dfma(q[3], W2, acc[2][r]);
            }
        }
    }
}

// the pair form's table carries kappa g o for offsets with two or three nonzero components
// (pair3_rank1) in FP64; FP32 and the difference form keep the block entries
template <typename T, bool DIFF> constexpr bool kRank1() { return sizeof(T) == 8 && !DIFF; }

template <typename T, int M, bool DIFF>
__global__ void __launch_bounds__(kThreads, (DIFF && M <= 3) ? 3 : 2)
k_tbt3d(const T *__restrict__ u, T *__restrict__ out, int nx, int ny, int nz, int nzt, int64_t N,
        const uint8_t *__restrict__ cons, int project, const T *__restrict__ kd, T scale,
        PairTab<T, 3, M> tab, double *dot_partial, double *dot_out, unsigned int *retire,
        int in_z0, int in_zend, int64_t Nin, int out_z0, int out_zend)
{
    // Planes are grid planes; the input holds planes [in_z0, in_zend) with component
    // size Nin, the output planes [out_z0, out_zend) with component size N (the whole
    // grid: 0, nz, N, 0, nz).  Planes of the grid outside the input enter only
    // outputs that the launch does not write.
    constexpr int R = rows3d<T, M, DIFF>();
    constexpr int TX = kTX3, TY = kTY3, SX = TX + 2 * M, SY = TY + 2 * M, SZ = R + 2 * M;
    constexpr int PL = SX * SY * SZ;
    constexpr int NP = PairTab<T, 3, M>::kPairs;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);   // [3][SZ][SY][SX]

    const int zt = blockIdx.z % nzt;
    const int64_t b = blockIdx.z / nzt;
    const T *ub = u + b * 3 * Nin - (int64_t)in_z0 * ny * nx;   // indexed by grid node
    T *ob = out + b * 3 * N - (int64_t)out_z0 * ny * nx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = out_z0 + zt * R;

    for (int t = threadIdx.x; t < PL; t += kThreads) {
        const int zz = t / (SX * SY), rem = t - zz * SX * SY;
        const int yy = rem / SX, xx = rem - yy * SX;
        const int gx = x0 - M + xx, gy = y0 - M + yy, gz = z0 - M + zz;
        T v0 = T(0), v1 = T(0), v2 = T(0);
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= in_z0 && gz < in_zend) {
            const int64_t p = ((int64_t)gz * ny + gy) * nx + gx;
            v0 = __ldg(ub + p);
            v1 = __ldg(ub + Nin + p);
            v2 = __ldg(ub + 2 * Nin + p);
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) v0 = T(0);
                if (m & 2) v1 = T(0);
                if (m & 4) v2 = T(0);
            }
        }
        s[t] = v0;
        s[PL + t] = v1;
        s[2 * PL + t] = v2;
    }
    __syncthreads();

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const T *base = s + (ty + M) * SX + (tx + M);   // column (x, y), plane 0
    T acc[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[c][r] = T(0);
    const int gxt = x0 + tx, gyt = y0 + ty;
    // window plane i holds grid plane z0 - M + i
    static_assert(SZ <= 32, "plane mask is one word");
    uint32_t zok = 0;
#pragma unroll
    for (int i = 0; i < SZ; ++i)
        if (z0 - M + i >= 0 && z0 - M + i < nz) zok |= 1u << i;
    T w0[3][SZ];
    if constexpr (DIFF) {
        // one instantiation for every warp: the in-grid flags are 1 on interior lanes (half
        // the code of a separate interior copy, which measured slower for its instruction-cache misses)
        diff3_column<T, M, true>(base, tab, gxt, gyt, nx, ny, zok, acc);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < R; ++r) w0[c][r + M] = base[c * PL + (r + M) * SX * SY];
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < SZ; ++i) w0[c][i] = base[c * PL + i * SX * SY];
        // pair form: acc[.][r] += c(o) (u~_{p+o} + u~_{p-o}), against Kd u_p below
        static_for<0, M + 1>([&](auto OYI) {
            constexpr int oy = M - decltype(OYI)::value;
            constexpr int Mx = isqrt_c(M * M - oy * oy);
            static_for<-Mx, Mx + 1>([&](auto OX) {
                constexpr int ox = decltype(OX)::value;
                if constexpr (oy > 0 || ox > 0) {
                    constexpr int Mz = isqrt_c(M * M - ox * ox - oy * oy);
                    constexpr int pbase = pair_index3(M, ox, oy, 0);   // pairs of this column are consecutive in oz
                    T wp[3][SZ], wm[3][SZ];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int i = 0; i < SZ; ++i) {
                            wp[c][i] = base[c * PL + i * SX * SY + oy * SX + ox];
                            wm[c][i] = base[c * PL + i * SX * SY - oy * SX - ox];
                        }
                    static_for<-Mz, Mz + 1>([&](auto OZ) {
                        constexpr int oz = decltype(OZ)::value;
                        const T *cf = tab.v + 6 * (pbase + oz);
                        constexpr int nzc = (ox != 0) + (oy != 0) + (oz != 0);
                        if constexpr (kRank1<T, DIFF>() && nzc >= 2) {
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                pair3_rank1<ox, oy, oz>(acc, r, cf, wp[0][r + M + oz] + wm[0][r + M - oz],
                                                        wp[1][r + M + oz] + wm[1][r + M - oz],
                                                        wp[2][r + M + oz] + wm[2][r + M - oz]);
                        } else {
                            const T cxx = cf[0], cxy = cf[1], cxz = cf[2], cyy = cf[3], cyz = cf[4], czz = cf[5];
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                pair3(acc, r, ox != 0, oy != 0, oz != 0, cxx, cxy, cxz, cyy, cyz, czz,
                                      wp[0][r + M + oz] + wm[0][r + M - oz], wp[1][r + M + oz] + wm[1][r + M - oz],
                                      wp[2][r + M + oz] + wm[2][r + M - oz]);
                        }
                    });
                }
            });
        });
        constexpr int pcentre = pair_index3(M, 0, 0, 1);
#pragma unroll
        for (int oz = 1; oz <= M; ++oz) {
            const T *cf = tab.v + 6 * (pcentre + oz - 1);
            const T czz = cf[5];
#pragma unroll
            for (int r = 0; r < R; ++r)
                pair3(acc, r, false, false, true, T(0), T(0), T(0), T(0), T(0), czz, T(0), T(0),
                      w0[2][r + M + oz] + w0[2][r + M - oz]);
        }
    }

    T dot = T(0);   // per-thread partial in the kernel's precision; FP64 only across threads
    const int gx = x0 + tx, gy = y0 + ty;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gz = z0 + r;
        if (gx < nx && gy < ny && gz < out_zend) {
            const int64_t p = ((int64_t)gz * ny + gy) * nx + gx;
            const T *kk = tab.v + 6 * NP;
            T k0 = kk[0], k1 = kk[1], k2 = kk[2], k3 = kk[3], k4 = kk[4], k5 = kk[5];
            const int a0 = min(gx, M), a1 = min(nx - 1 - gx, M), b0 = min(gy, M), b1 = min(ny - 1 - gy, M),
                      c0 = min(gz, M), c1 = min(nz - 1 - gz, M);
            if constexpr (DIFF) {   // the in-grid bond sum: no diagonal term
                k0 = k1 = k2 = k3 = k4 = k5 = T(0);
            } else if (a0 != M || a1 != M || b0 != M || b1 != M || c0 != M || c1 != M) {
                const int cls =
                    ((((a0 * (M + 1) + a1) * (M + 1) + b0) * (M + 1) + b1) * (M + 1) + c0) * (M + 1) + c1;
                const T *q = kd + 6 * cls;
                k0 = __ldg(q);
                k1 = __ldg(q + 1);
                k2 = __ldg(q + 2);
                k3 = __ldg(q + 3);
                k4 = __ldg(q + 4);
                k5 = __ldg(q + 5);
            }
            const T u0 = w0[0][r + M], u1 = w0[1][r + M], u2 = w0[2][r + M];
            T f0 = dfma(k0, u0, dfma(k1, u1, dfma(k2, u2, -acc[0][r])));
            T f1 = dfma(k1, u0, dfma(k3, u1, dfma(k4, u2, -acc[1][r])));
            T f2 = dfma(k2, u0, dfma(k4, u1, dfma(k5, u2, -acc[2][r])));
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) f0 = T(0);
                if (m & 2) f1 = T(0);
                if (m & 4) f2 = T(0);
            }
            f0 *= scale;
            f1 *= scale;
            f2 *= scale;
            ob[p] = f0;
            ob[N + p] = f1;
            ob[2 * N + p] = f2;
            dot = dfma(u0, f0, dfma(u1, f1, dfma(u2, f2, dot)));
        }
    }
    if (dot_partial)
        finish_block_dot(dot, dot_partial, dot_out, retire, gridDim.x * gridDim.y * nzt,
                         blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zt), b);
}

namespace {

template <typename T, int M>
PairTab<T, 3, M> make_pairs3(const pd_grid *g, bool rank1)
{
    PairTab<T, 3, M> t{};
    double c[6], tot[6] = {0, 0, 0, 0, 0, 0};
    auto put = [&](int ox, int oy, int oz) {
        const int pi = pair_index3(M, ox, oy, oz);
        coef_of(g, ox, oy, oz, false, c);
        for (int i = 0; i < 6; ++i) {
            t.v[6 * pi + i] = (T)c[i];
            tot[i] += 2 * c[i];
        }
        if (rank1 && (ox != 0) + (oy != 0) + (oz != 0) >= 2) {
            // c_aa = kappa o_a^2 (entries xx, yy, zz at 0, 3, 5): kappa from a nonzero component
            const int o[3] = {ox, oy, oz};
            const int a = ox != 0 ? 0 : 1;
            const double kappa = c[a == 0 ? 0 : 3] / ((double)o[a] * o[a]);
            const double kg = kappa * gcd3_c(gcd3_c(ox, oy), oz);
            for (int i = 0; i < 3; ++i) t.v[6 * pi + i] = (T)(kg * o[i]);
            for (int i = 3; i < 6; ++i) t.v[6 * pi + i] = T(0);
        }
    };
    for (int oy = M; oy >= 0; --oy) {
        const int Mx = isqrt_c(M * M - oy * oy);
        for (int ox = -Mx; ox <= Mx; ++ox) {
            if (oy == 0 && ox <= 0) continue;
            const int Mz = isqrt_c(M * M - ox * ox - oy * oy);
            for (int oz = -Mz; oz <= Mz; ++oz) put(ox, oy, oz);
        }
    }
    for (int oz = 1; oz <= M; ++oz) put(0, 0, oz);
    constexpr int NP = PairTab<T, 3, M>::kPairs;
    for (int i = 0; i < 6; ++i) t.v[6 * NP + i] = (T)tot[i];
    return t;
}

template <typename T, int M, bool DIFF>
int run(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    constexpr int R = rows3d<T, M, DIFF>();
    const size_t smem = sizeof(T) * 3 * (kTX3 + 2 * M) * (kTY3 + 2 * M) * (R + 2 * M);
    auto kern = k_tbt3d<T, M, DIFF>;
    allow_smem(kern, smem);
    const int64_t nz = g->n[2], plane = g->n[0] * g->n[1];
    const int64_t in_planes = a.in_rows < 0 ? nz : a.in_rows, out_planes = a.out_rows < 0 ? nz : a.out_rows;
    if ((in_planes != nz || out_planes != nz) && a.dot_partial)
        return fail(PD_ERR_INVALID, "plane windows take no fused dot");
    const int nzt = (int)((out_planes + R - 1) / R);
    if ((int64_t)nzt * a.batch > 65535) return fail(PD_ERR_INVALID, "3D batch too large for one launch");
    dim3 grid((unsigned)((g->n[0] + kTX3 - 1) / kTX3), (unsigned)((g->n[1] + kTY3 - 1) / kTY3),
              (unsigned)(nzt * a.batch));
    const T *kd = sizeof(T) == 4 ? (const T *)g->d_kd32 : (const T *)g->d_kd64;
    kern<<<grid, kThreads, smem, s>>>((const T *)a.u, (T *)a.out, (int)g->n[0], (int)g->n[1], (int)nz, nzt,
                                      out_planes * plane, g->d_cons, a.project ? 1 : 0, kd, (T)a.scale,
                                      make_pairs3<T, M>(g, kRank1<T, DIFF>()), a.dot_partial, a.dot_out, a.retire, (int)a.in_row0,
                                      (int)(a.in_row0 + in_planes), in_planes * plane, (int)a.out_row0,
                                      (int)(a.out_row0 + out_planes));
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <typename T>
int run_t(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {   // FP32: the difference form unless the pair form is asked for
        if (!a.pair_form) {
            switch (g->M) {
                case 1: return run<T, 1, true>(g, a, s);
                case 2: return run<T, 2, true>(g, a, s);
                case 3: return run<T, 3, true>(g, a, s);
                case 4: return run<T, 4, true>(g, a, s);
            }
            return fail(PD_ERR_INVALID, "horizon M not compiled for 3D");
        }
    }
    switch (g->M) {
        case 1: return run<T, 1, false>(g, a, s);
        case 2: return run<T, 2, false>(g, a, s);
        case 3: return run<T, 3, false>(g, a, s);
        case 4: return run<T, 4, false>(g, a, s);
    }
    return fail(PD_ERR_INVALID, "horizon M not compiled for 3D");
}

}  // namespace

int run_tbt3d(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s)
{
    return f64 ? run_t<double>(g, a, s) : run_t<float>(g, a, s);
}

}  // namespace pd

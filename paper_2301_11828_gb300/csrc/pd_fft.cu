// pd_fft.cu -- the Toeplitz-block-Toeplitz part of K u by FFT (Sec. 3.2,
// Algorithm 3), fused with the 2x2 symbol product, in shared memory.
//
// Algorithm 3 embeds the whole grid in a 2N x 2N circulant and runs one global
// FFT.  On a GPU that global transform needs several passes over HBM.  This
// kernel applies the same circulant-embedding identity per tile instead
// (overlap-save): a CTA takes a P x P window (P = 64) of the zero-padded field,
// whose centre (P - 2M) x (P - 2M) nodes are its outputs, and computes the
// circular convolution of the window with the kernel table by FFT.  For an
// output node every neighbour p + o lies inside the window, so the circular
// result equals the Toeplitz product there, exactly as the 2N embedding does
// for the whole grid.  HBM then sees u once (plus the halo) and K u once.
//
// Per tile:
//   1. load z = u_x + i u_y - c (zero outside the grid, projected if asked),
//      with c the value at one in-grid node of the window (FP64) or the tile's
//      least-squares plane (FP32, see tile_plane): K maps a constant field to
//      zero on every row (the edge rows included) and a plane to zero at every
//      full-horizon node, so K u = K(u - c), or K(u - L) + K L with K L from a
//      first-moment table at the edge nodes, and the transforms then round
//      values of the size of u's variation (FP64) or curvature (FP32) over the
//      tile instead of u's own;
//   2. 64-point FFTs along x, then along y (each as 8 x 8, in two register
//      passes with the twiddles W64^(n2 k1) between them), leaving the
//      spectrum in digit-reversed order along both axes;
//   3. for each frequency pair (k, -k): unpack U_x, U_y from Z(k), Z(-k)
//      (both components are real), multiply by the real 2x2 symbol
//      S(k) = sum_o Kop(o) cos(2 pi k.o / P) / P^2 (Kop(0) = sum c, Kop(o) = -c(o);
//      the kernel is even, so S is real; a quarter of it is staged in shared
//      memory), repack W = H_x + i H_y;
//   4. inverse FFTs along y then x, from that order back to natural order;
//   5. epilogue: K u = Re/Im(w) - (Ctot - Kd_p) u_p on nodes near a face (the
//      D^e term of Eq. tea:sc), projection, scale, optional fused dot.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "pd_internal.cuh"
#include "pd_reduce.cuh"
#include "pd_tma2d.cuh"

namespace pd {

namespace {

constexpr int P = kFftP;       // tile edge
constexpr int PS = P + 1;      // padded row stride (complex elements): conflict-free rows and columns
constexpr int kT = 256;

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

__constant__ float2 c_tw32[P];
__constant__ double2 c_tw64[P];

template <typename T> __device__ __forceinline__ typename C2<T>::t tw(int j);
template <> __device__ __forceinline__ float2 tw<float>(int j) { return c_tw32[j]; }
template <> __device__ __forceinline__ double2 tw<double>(int j) { return c_tw64[j]; }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return {a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return {a.x - b.x, a.y - b.y}; }
// a * w (INV: a * conj(w))
template <bool INV, typename V> __device__ __forceinline__ V cmulw(V a, V w)
{
    if (INV) return {a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y};
    return {a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x};
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> __device__ __forceinline__ V mul_mi(V a)
{
    if (INV) return {-a.y, a.x};
    return {a.y, -a.x};
}

// In-register 8-point DFT, X[k] = sum_n x[n] w^(nk), w = exp(-+2 pi i / 8).
template <bool INV, typename V, typename T>
__device__ __forceinline__ void dft8(V (&x)[8])
{
    const T r = T(0.70710678118654752440);   // 1/sqrt(2)
    // DFT4 of the even and of the odd samples
    V e[4], o[4];
    {
        V a = cadd(x[0], x[4]), b = csub(x[0], x[4]), c = cadd(x[2], x[6]), d = mul_mi<INV>(csub(x[2], x[6]));
        e[0] = cadd(a, c); e[2] = csub(a, c); e[1] = cadd(b, d); e[3] = csub(b, d);
    }
    {
        V a = cadd(x[1], x[5]), b = csub(x[1], x[5]), c = cadd(x[3], x[7]), d = mul_mi<INV>(csub(x[3], x[7]));
        o[0] = cadd(a, c); o[2] = csub(a, c); o[1] = cadd(b, d); o[3] = csub(b, d);
    }
    // twiddles w^k, k = 1, 2, 3
    V t1, t2, t3;
    if (!INV) {
        t1 = {(o[1].x + o[1].y) * r, (o[1].y - o[1].x) * r};     // * (1 - i)/sqrt2
        t2 = {o[2].y, -o[2].x};                                  // * -i
        t3 = {(o[3].y - o[3].x) * r, -(o[3].x + o[3].y) * r};    // * (-1 - i)/sqrt2
    } else {
        t1 = {(o[1].x - o[1].y) * r, (o[1].x + o[1].y) * r};     // * (1 + i)/sqrt2
        t2 = {-o[2].y, o[2].x};                                  // * i
        t3 = {-(o[3].x + o[3].y) * r, (o[3].x - o[3].y) * r};    // * (-1 + i)/sqrt2
    }
    x[0] = cadd(e[0], o[0]); x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], t1);   x[5] = csub(e[1], t1);
    x[2] = cadd(e[2], t2);   x[6] = csub(e[2], t2);
    x[3] = cadd(e[3], t3);   x[7] = csub(e[3], t3);
}

// 64-point FFTs of 64 lines (rows: es = 1, ls = PS; columns: es = PS, ls = 1),
// as 8 x 8 with the twiddles W64^(n2 k1) between the two passes.  The forward
// transform takes the line in natural order and leaves it digit-reversed: slot
// 8 a + b holds frequency a + 8 b.  The inverse takes that order and returns the
// line in natural order.  So every pass writes back the very slots its thread
// read, and one block barrier per pass suffices (no transposing store that
// would overwrite slots another thread has yet to read).
// Thread mapping: lane -> line (and line + 32), warp -> the 8-point group index,
// so every shared-memory access of a warp hits distinct banks.
__device__ __forceinline__ int digrev64(int s) { return (s >> 3) | ((s & 7) << 3); }

template <typename T>
__device__ __forceinline__ void fft64_fwd(typename C2<T>::t *Z, int es, int ls)
{
    using V = typename C2<T>::t;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;   // g in [0, 8)
    V v[2][8];
    // pass 1: group g = n2; x[8 n1 + n2] -> DFT over n1 -> * W64^(n2 k1) -> slot 8 k1 + n2
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        V *line = Z + (lane + 32 * h) * ls;
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) v[h][n1] = line[(8 * n1 + g) * es];
        dft8<false, V, T>(v[h]);
#pragma unroll
        for (int k1 = 1; k1 < 8; ++k1) v[h][k1] = cmulw<false>(v[h][k1], tw<T>(g * k1));
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) line[(8 * k1 + g) * es] = v[h][k1];
    }
    __syncthreads();
    // pass 2: group g = k1; slots 8 k1 + n2 -> DFT over n2 -> X[k1 + 8 k2] at slot 8 k1 + k2
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        V *line = Z + (lane + 32 * h) * ls;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) v[h][n2] = line[(8 * g + n2) * es];
        dft8<false, V, T>(v[h]);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) line[(8 * g + k2) * es] = v[h][k2];
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void fft64_inv(typename C2<T>::t *Z, int es, int ls)
{
    using V = typename C2<T>::t;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    V v[2][8];
    // pass A: group g = k1; slot 8 k1 + k2 holds X[k1 + 8 k2] -> inverse DFT over k2 -> * conj W64^(k1 n2)
    // -> slot 8 k1 + n2
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        V *line = Z + (lane + 32 * h) * ls;
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) v[h][k2] = line[(8 * g + k2) * es];
        dft8<true, V, T>(v[h]);
#pragma unroll
        for (int n2 = 1; n2 < 8; ++n2) v[h][n2] = cmulw<true>(v[h][n2], tw<T>(g * n2));
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) line[(8 * g + n2) * es] = v[h][n2];
    }
    __syncthreads();
    // pass B: group g = n2; slots 8 k1 + n2 -> inverse DFT over k1 -> x[8 n1 + n2] at slot 8 n1 + n2
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        V *line = Z + (lane + 32 * h) * ls;
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) v[h][k1] = line[(8 * k1 + g) * es];
        dft8<true, V, T>(v[h]);
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) line[(8 * n1 + g) * es] = v[h][n1];
    }
    __syncthreads();
}

// The tile's reference plane.  Subtracting a constant leaves the FP32
// transforms rounding values of the size of u's variation over the tile, which
// on a smooth field is its gradient times the tile width; subtracting the
// least-squares plane of the tile leaves its curvature part instead.  K maps a
// plane to zero at every node with a full horizon, and at a node near a face to
// -sum_b (Tx_ab gx_b + Ty_ab gy_b), Tx_ab = sum of c_ab(o) o_x over the in-grid
// offsets (and Ty with o_y): the first-moment table of the node's edge class.
// The plane is quantised so that its value at every window node is exact in
// FP32: L = q (L0 + Gx (a - ar) + Gy (r - rr)) with q a power of two and
// integers |L0| + 64 (|Gx| + |Gy|) < 2^24 -- the transforms then see exactly
// u - L, and K u = K (u - L) + K L holds to rounding.
struct TilePlane {
    int l0[2], gx[2], gy[2];
    float q[2];
    int ar, rr;
};

// Least-squares plane of both components over an 8 x 8 sample of the window's
// in-grid rectangle [ax, bx) x [ay, by) (fetch(a, r, vx, vy) reads a node): any
// plane serves, the fit only has to follow the field closely.  Warp 0 takes the
// samples (two per lane), and every lane of it forms the same plane from the
// butterfly sums; lane 0 publishes it.  The caller's next block barrier makes
// *pl visible to every thread.
template <typename F>
__device__ __forceinline__ void tile_plane(F fetch, int ax, int bx, int ay, int by, TilePlane *pl)
{
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int wx = bx - ax, wy = by - ay;
    // sample columns ax + (i (wx - 1)) / 7 and rows likewise, their means and spreads
    float mx = 0.f, my = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        mx += (float)(ax + (i * (wx - 1)) / 7);
        my += (float)(ay + (i * (wy - 1)) / 7);
    }
    mx *= 0.125f;
    my *= 0.125f;
    float sxx = 0.f, syy = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float dx = (float)(ax + (i * (wx - 1)) / 7) - mx, dy = (float)(ay + (i * (wy - 1)) / 7) - my;
        sxx = fmaf(dx, dx, sxx);
        syy = fmaf(dy, dy, syy);
    }
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane & 7, j = (lane >> 3) + 4 * h;
        const int a = ax + (i * (wx - 1)) / 7, r = ay + (j * (wy - 1)) / 7;
        float vx, vy;
        fetch(a, r, vx, vy);
        const float dx = (float)a - mx, dy = (float)r - my;
        s[0] += vx;
        s[1] = fmaf(vx, dx, s[1]);
        s[2] = fmaf(vx, dy, s[2]);
        s[3] += vy;
        s[4] = fmaf(vy, dx, s[4]);
        s[5] = fmaf(vy, dy, s[5]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    const float ix = sxx > 0.f ? 0.125f / sxx : 0.f, iy = syy > 0.f ? 0.125f / syy : 0.f;
    const int ar = ax + (wx - 1) / 2, rr = ay + (wy - 1) / 2;
    int l0[2], gxi[2], gyi[2];
    float q[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float gx = s[3 * c + 1] * ix, gy = s[3 * c + 2] * iy;
        const float l = s[3 * c] * (1.f / 64.f) + gx * ((float)ar - mx) + gy * ((float)rr - my);
        const float bound = fabsf(l) + 64.f * (fabsf(gx) + fabsf(gy));
        l0[c] = gxi[c] = gyi[c] = 0;
        q[c] = 0.f;
        // q = 2^(k - 23) with bound < 2^k (from the exponent field), and 1/q exactly
        const int eb = (__float_as_int(bound) >> 23) & 0xff;   // biased exponent: bound < 2^(eb - 126)
        if (bound > 1e-30f && eb < 254 && eb > 30) {
            q[c] = __int_as_float((eb - 126 - 23 + 127) << 23);
            const float iq = __int_as_float((127 - (eb - 126 - 23)) << 23);
            l0[c] = __float2int_rn(l * iq);
            gxi[c] = __float2int_rn(gx * iq);
            gyi[c] = __float2int_rn(gy * iq);
        }
    }
    if (lane == 0) {
        pl->ar = ar;
        pl->rr = rr;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            pl->l0[c] = l0[c];
            pl->gx[c] = gxi[c];
            pl->gy[c] = gyi[c];
            pl->q[c] = q[c];
        }
    }
}

// The plane's value at window node (a, r), component c: exact in FP32.
__device__ __forceinline__ float plane_at(const TilePlane &pl, int c, int a, int r)
{
    return pl.q[c] * __int2float_rn(pl.l0[c] + pl.gx[c] * (a - pl.ar) + pl.gy[c] * (r - pl.rr));
}

template <typename T, int M>
__global__ void __launch_bounds__(kT)
k_fft_tile(const T *__restrict__ u, T *__restrict__ out, int nx, int ny, int64_t N,
           const uint8_t *__restrict__ cons, int project, const T *__restrict__ sym, const T *__restrict__ kd,
           const float *__restrict__ kt, T ctxx, T ctxy, T ctyy, T scale, double *dot_partial, double *dot_out,
           unsigned int *retire)
{
    using V = typename C2<T>::t;
    constexpr int TO = P - 2 * M;   // outputs per tile edge
    constexpr int QH = P / 2 + 1;   // quarter symbol edge
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *Z = reinterpret_cast<V *>(smem_raw);   // [P][PS]
    T *sq = reinterpret_cast<T *>(Z + P * PS);   // quarter symbol [3][QH][QH]
    for (int t = threadIdx.x; t < 3 * QH * QH; t += kT) sq[t] = __ldg(sym + t);

    const int64_t b = blockIdx.z;
    const T *ub = u + b * 2 * N;
    T *ob = out + b * 2 * N;
    const int x0 = blockIdx.x * TO - M, y0 = blockIdx.y * TO - M;   // window origin
    // the tile's reference value: the (projected) input at its first output node
    T cx, cy;
    {
        const int64_t p0 = (int64_t)(y0 + M) * nx + (x0 + M);
        cx = __ldg(ub + p0);
        cy = __ldg(ub + N + p0);
        if (project) {
            const uint8_t m = __ldg(cons + p0);
            if (m & 1) cx = T(0);
            if (m & 2) cy = T(0);
        }
    }

    // FP32: the tile's reference plane (tile_plane) instead of the constant
    constexpr bool PLANE = sizeof(T) == 4;
    __shared__ TilePlane s_pl;
    const int ax = max(0, -x0), bx = min(P, nx - x0), ay = max(0, -y0), by = min(P, ny - y0);
    auto fetch = [&](int a, int r, T &vx, T &vy) {
        const int64_t p = (int64_t)(y0 + r) * nx + (x0 + a);
        vx = __ldg(ub + p);
        vy = __ldg(ub + N + p);
        if (project) {
            const uint8_t m = __ldg(cons + p);
            if (m & 1) vx = T(0);
            if (m & 2) vy = T(0);
        }
    };
    if constexpr (PLANE) {
        tile_plane(fetch, ax, bx, ay, by, &s_pl);
        __syncthreads();
    }
    TilePlane pl{};
    if constexpr (PLANE) pl = s_pl;
    auto ref = [&](int c, int a, int r) -> T {
        if constexpr (PLANE) return plane_at(pl, c, a, r);
        return c == 0 ? cx : cy;
    };
    for (int t = threadIdx.x; t < P * P; t += kT) {
        const int a = t % P, r = t / P;
        V z = {T(0), T(0)};
        if (a >= ax && a < bx && r >= ay && r < by) {
            T vx, vy;
            fetch(a, r, vx, vy);
            z.x = vx - ref(0, a, r);
            z.y = vy - ref(1, a, r);
        }
        Z[r * PS + a] = z;
    }
    __syncthreads();

    fft64_fwd<T>(Z, 1, PS);    // rows (along x)
    fft64_fwd<T>(Z, PS, 1);    // columns (along y)

    // symbol product on frequency pairs (k, -k)
    // the transforms left slot (sy, sx) holding frequency (digrev64(sy), digrev64(sx))
    for (int t = threadIdx.x; t < P * P; t += kT) {
        const int sx = t % P, sy = t / P;
        const int kx = digrev64(sx), ky = digrev64(sy);
        const int mx = (P - kx) & (P - 1), my = (P - ky) & (P - 1);
        const int smx = digrev64(mx), smy = digrev64(my);
        const int t2 = smy * P + smx;
        if (t2 < t) continue;
        const V zk = Z[sy * PS + sx], zm0 = Z[smy * PS + smx];
        const V zm = {zm0.x, -zm0.y};   // conj Z(-k)
        // U_x = (Z(k) + conj Z(-k)) / 2,  U_y = -i (Z(k) - conj Z(-k)) / 2
        const V ux = {T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y + zm.y)};
        const V uy = {T(0.5) * (zk.y - zm.y), T(-0.5) * (zk.x - zm.x)};
        // S is even in kx and in ky for xx, yy and odd in each for xy (the offset set is
        // symmetric under ox -> -ox and oy -> -oy), so a quarter of it is stored
        const int qx = kx <= P / 2 ? kx : P - kx, qy = ky <= P / 2 ? ky : P - ky;
        const int qi = qy * QH + qx;
        const T sgn = ((kx > P / 2) != (ky > P / 2)) ? T(-1) : T(1);
        const T sxx = sq[qi], sxy = sgn * sq[QH * QH + qi], syy = sq[2 * QH * QH + qi];
        const V hx = {sxx * ux.x + sxy * uy.x, sxx * ux.y + sxy * uy.y};
        const V hy = {sxy * ux.x + syy * uy.x, sxy * ux.y + syy * uy.y};
        // W(k) = H_x + i H_y ; W(-k) = conj H_x + i conj H_y
        Z[sy * PS + sx] = {hx.x - hy.y, hx.y + hy.x};
        if (t2 != t) Z[smy * PS + smx] = {hx.x + hy.y, hy.x - hx.y};
    }
    __syncthreads();

    fft64_inv<T>(Z, PS, 1);     // columns
    fft64_inv<T>(Z, 1, PS);     // rows

    T dot = T(0);
    for (int t = threadIdx.x; t < TO * TO; t += kT) {
        const int a = M + t % TO, r = M + t / TO;
        const int gx = x0 + a, gy = y0 + r;
        if (gx >= nx || gy >= ny) continue;
        const int64_t p = (int64_t)gy * nx + gx;
        const V w = Z[r * PS + a];
        T fx = w.x, fy = w.y;
        const int a0 = min(gx, M), a1 = min(nx - 1 - gx, M), b0 = min(gy, M), b1 = min(ny - 1 - gy, M);
        const bool edge = (a0 != M || a1 != M || b0 != M || b1 != M);
        if (edge || dot_partial) {
            T upx = __ldg(ub + p), upy = __ldg(ub + N + p);
            const uint8_t m = project ? __ldg(cons + p) : 0;
            if (m & 1) upx = T(0);
            if (m & 2) upy = T(0);
            if (edge) {   // the D^e term on the shifted field the transforms saw
                const int cls = ((a0 * (M + 1) + a1) * (M + 1) + b0) * (M + 1) + b1;
                const T dxx = ctxx - __ldg(kd + 3 * cls), dxy = ctxy - __ldg(kd + 3 * cls + 1),
                        dyy = ctyy - __ldg(kd + 3 * cls + 2);
                const T zx = upx - ref(0, a, r), zy = upy - ref(1, a, r);
                fx -= dxx * zx + dxy * zy;
                fy -= dxy * zx + dyy * zy;
                if constexpr (PLANE) {   // K of the plane (zero at full-horizon nodes)
                    const float *t6 = kt + 6 * cls;
                    const float gxx = pl.q[0] * (float)pl.gx[0], gyx = pl.q[0] * (float)pl.gy[0];
                    const float gxy = pl.q[1] * (float)pl.gx[1], gyy = pl.q[1] * (float)pl.gy[1];
                    fx -= __ldg(t6) * gxx + __ldg(t6 + 3) * gyx + __ldg(t6 + 1) * gxy + __ldg(t6 + 4) * gyy;
                    fy -= __ldg(t6 + 1) * gxx + __ldg(t6 + 4) * gyx + __ldg(t6 + 2) * gxy + __ldg(t6 + 5) * gyy;
                }
            }
            if (m & 1) fx = T(0);
            if (m & 2) fy = T(0);
            fx *= scale;
            fy *= scale;
            dot += upx * fx + upy * fy;
        } else {
            if (project) {
                const uint8_t m2 = __ldg(cons + p);
                if (m2 & 1) fx = T(0);
                if (m2 & 2) fy = T(0);
            }
            fx *= scale;
            fy *= scale;
        }
        ob[p] = fx;
        ob[N + p] = fy;
    }
    if (dot_partial) {
        __shared__ double red[kT / 32];
        const double s = block_sum(dot, red);
        grid_finish(s, gridDim.x * gridDim.y, blockIdx.x + gridDim.x * blockIdx.y, dot_partial + b * gridDim.x * gridDim.y,
                    dot_out + b, retire + b, red);
    }
}

// FP32 tiles fed by TMA (products without projection or a fused dot): persistent
// CTAs, two per SM.  The window of the next tile is copied by the TMA engine
// into a staging box while the current tile is transformed, so the plain
// global loads of k_fft_tile -- the stall that bounds it -- leave the tile's
// critical path.  The window's x origin is rounded down to a 16-byte boundary
// (TMA rule) and the box is 4 columns wider.  The staging box holds zeros
// outside the grid; z = u - c is formed only for in-grid nodes (the embedding
// pads with zeros, not with -c).  Same arithmetic per tile as k_fft_tile.
constexpr int kFBX = P + 4;   // staged columns (16-byte aligned start)
template <int M>
__global__ void __launch_bounds__(kT, 2)
k_fft_tile_tma(const __grid_constant__ CUtensorMap map, float *__restrict__ out, int nx, int ny, int64_t N,
               int tiles_x, int tiles_y, int ntiles, const float *__restrict__ sym, const float *__restrict__ kd,
               const float *__restrict__ kt, float ctxx, float ctxy, float ctyy, float scale,
               const float *__restrict__ u, int *err)
{
    using V = float2;
    using namespace tma2d;
    constexpr int TO = P - 2 * M;
    constexpr int QH = P / 2 + 1;
    constexpr uint32_t kBytes = 2u * kFBX * P * sizeof(float);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *const stg = reinterpret_cast<float *>(smem_raw);                  // [2][P][kFBX] staged window
    V *const Z = reinterpret_cast<V *>(smem_raw + kBytes);                    // [P][PS]
    float *const sq = reinterpret_cast<float *>(Z + P * PS);                  // quarter symbol [3][QH][QH]
    __shared__ __align__(8) uint64_t full;
    __shared__ int s_abort;
    __shared__ TilePlane s_pl;
    for (int t = threadIdx.x; t < 3 * QH * QH; t += kT) sq[t] = __ldg(sym + t);
    if (threadIdx.x == 0) {
        mbar_init(&full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();
    auto coords = [&](int t, int &x0, int &y0, int &b) {
        const int per = tiles_x * tiles_y;
        b = t / per;
        const int r = t - b * per;
        y0 = (r / tiles_x) * TO - M;
        x0 = (r % tiles_x) * TO - M;
    };
    auto issue = [&](int t) {
        int x0, y0, b;
        coords(t, x0, y0, b);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&full, kBytes);
        tma_load_3d(stg, &map, x0 & ~3, y0, 2 * b, &full);
    };
    int it = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        int x0, y0, b;
        coords(t, x0, y0, b);
        const bool ok = mbar_wait(&full, it & 1);
        if (!ok) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                s_abort = 1;
            }
        }
        __syncthreads();
        if (s_abort) break;
        const int d = x0 - (x0 & ~3);   // column of the window's origin in the staged box
        const float *sx = stg, *sy = stg + P * kFBX;
        // the window's in-grid rectangle and the tile's reference plane over it
        const int ax = max(0, -x0), bx = min(P, nx - x0), ay = max(0, -y0), by = min(P, ny - y0);
        tile_plane([&](int a, int r, float &vx, float &vy) {
                       vx = sx[r * kFBX + a + d];
                       vy = sy[r * kFBX + a + d];
                   }, ax, bx, ay, by, &s_pl);
        __syncthreads();
        const TilePlane pl = s_pl;
        {   // a thread keeps its column (kT is a multiple of P) and steps rows by kT / P: the
            // plane's integers advance by a constant (exactly as plane_at would form them)
            static_assert(kT % P == 0, "one column per thread");
            constexpr int RS = kT / P;
            const int a = threadIdx.x % P, r0 = threadIdx.x / P;
            int lx = pl.l0[0] + pl.gx[0] * (a - pl.ar) + pl.gy[0] * (r0 - pl.rr);
            int ly = pl.l0[1] + pl.gx[1] * (a - pl.ar) + pl.gy[1] * (r0 - pl.rr);
            const int sx_ = RS * pl.gy[0], sy_ = RS * pl.gy[1];
            const bool ain = a >= ax && a < bx;
            for (int r = r0; r < P; r += RS, lx += sx_, ly += sy_) {
                V z = {0.f, 0.f};
                if (ain && r >= ay && r < by) {
                    z.x = sx[r * kFBX + a + d] - pl.q[0] * __int2float_rn(lx);
                    z.y = sy[r * kFBX + a + d] - pl.q[1] * __int2float_rn(ly);
                }
                Z[r * PS + a] = z;
            }
        }
        __syncthreads();   // the staged box is free: the next tile's window is copied meanwhile
        if (threadIdx.x == 0 && t + (int)gridDim.x < ntiles) issue(t + gridDim.x);

        fft64_fwd<float>(Z, 1, PS);
        fft64_fwd<float>(Z, PS, 1);
        {   // a thread keeps one slot column sx (kT is a multiple of P): its frequency, partner
            // column and quarter-symbol column are formed once; slot (sy, sx) holds frequency
            // (digrev64(sy), digrev64(sx))
            const int sx = threadIdx.x % P;
            const int kx = digrev64(sx), smx = digrev64((P - kx) & (P - 1));
            const int qx = kx <= P / 2 ? kx : P - kx;
            const bool hx = kx > P / 2;
            for (int sy = threadIdx.x / P; sy < P; sy += kT / P) {
            const int e = sy * P + sx;
            const int ky = digrev64(sy), smy = digrev64((P - ky) & (P - 1));
            const int t2 = smy * P + smx;
            if (t2 < e) continue;
            const V zk = Z[sy * PS + sx], zm0 = Z[smy * PS + smx];
            const V zm = {zm0.x, -zm0.y};
            const V ux = {0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y)};
            const V uy = {0.5f * (zk.y - zm.y), -0.5f * (zk.x - zm.x)};
            const int qy = ky <= P / 2 ? ky : P - ky;
            const int qi = qy * QH + qx;
            const float sgn = (hx != (ky > P / 2)) ? -1.f : 1.f;
            const float sxx = sq[qi], sxy = sgn * sq[QH * QH + qi], syy = sq[2 * QH * QH + qi];
            const V hx_ = {sxx * ux.x + sxy * uy.x, sxx * ux.y + sxy * uy.y};
            const V hy_ = {sxy * ux.x + syy * uy.x, sxy * ux.y + syy * uy.y};
            Z[sy * PS + sx] = {hx_.x - hy_.y, hx_.y + hy_.x};
            if (t2 != e) Z[smy * PS + smx] = {hx_.x + hy_.y, hy_.x - hx_.y};
            }
        }
        __syncthreads();
        fft64_inv<float>(Z, PS, 1);
        fft64_inv<float>(Z, 1, PS);

        const float *ub = u + (int64_t)b * 2 * N;
        float *ob = out + (int64_t)b * 2 * N;
        const int ea = threadIdx.x % P;   // a thread keeps a window column (outputs: M <= a, r < P - M)
        for (int r = M + ((threadIdx.x / P) - M % (kT / P) + (kT / P)) % (kT / P); r < P - M; r += kT / P) {
            const int a = ea;
            const int gx = x0 + a, gy = y0 + r;
            if (a < M || a >= P - M || gx >= nx || gy >= ny) continue;
            const int64_t p = (int64_t)gy * nx + gx;
            const V w = Z[r * PS + a];
            float fx = w.x, fy = w.y;
            const int a0 = min(gx, M), a1 = min(nx - 1 - gx, M), b0 = min(gy, M), b1 = min(ny - 1 - gy, M);
            if (a0 != M || a1 != M || b0 != M || b1 != M) {
                // the D^e term on the shifted field, and K of the plane (zero at full-horizon nodes)
                const int cls = ((a0 * (M + 1) + a1) * (M + 1) + b0) * (M + 1) + b1;
                const float dxx = ctxx - __ldg(kd + 3 * cls), dxy = ctxy - __ldg(kd + 3 * cls + 1),
                            dyy = ctyy - __ldg(kd + 3 * cls + 2);
                const float zx = __ldg(ub + p) - plane_at(pl, 0, a, r), zy = __ldg(ub + N + p) - plane_at(pl, 1, a, r);
                fx -= dxx * zx + dxy * zy;
                fy -= dxy * zx + dyy * zy;
                const float *t6 = kt + 6 * cls;   // Tx_xx, Tx_xy, Tx_yy, Ty_xx, Ty_xy, Ty_yy
                const float gxx = pl.q[0] * (float)pl.gx[0], gyx = pl.q[0] * (float)pl.gy[0];
                const float gxy = pl.q[1] * (float)pl.gx[1], gyy = pl.q[1] * (float)pl.gy[1];
                fx -= __ldg(t6) * gxx + __ldg(t6 + 3) * gyx + __ldg(t6 + 1) * gxy + __ldg(t6 + 4) * gyy;
                fy -= __ldg(t6 + 1) * gxx + __ldg(t6 + 4) * gyx + __ldg(t6 + 2) * gxy + __ldg(t6 + 5) * gyy;
            }
            ob[p] = fx * scale;
            ob[N + p] = fy * scale;
        }
        __syncthreads();   // Z is free for the next tile
    }
    __syncthreads();
    if (s_abort && threadIdx.x == 0) mbar_wait(&full, it & 1);   // let a copy still in flight land
}

// Tensor map over `batch` fields of two FP32 planes [2*batch][ny][nx] with the
// staged-window box of k_fft_tile_tma; false if the driver rejects it.
bool fft_map(CUtensorMap *map, const void *base, int nx, int ny, int64_t batch)
{
    tma2d::EncodeTiledFn enc = tma2d::encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)(2 * batch)};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)kFBX, (cuuint32_t)P, 2};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

std::once_flag g_tw_once[64];
int g_tw_status[64];

int upload_twiddles()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(PD_ERR_CUDA, "device query");
    std::call_once(g_tw_once[dev], [&] {
        float2 t32[P];
        double2 t64[P];
        const double pi = 3.14159265358979323846;
        for (int j = 0; j < P; ++j) {
            const double ang = -2.0 * pi * j / P;   // forward twiddle exp(-2 pi i j / P)
            t64[j] = make_double2(std::cos(ang), std::sin(ang));
            t32[j] = make_float2((float)t64[j].x, (float)t64[j].y);
        }
        g_tw_status[dev] = (cudaMemcpyToSymbol(c_tw32, t32, sizeof(t32)) == cudaSuccess &&
                            cudaMemcpyToSymbol(c_tw64, t64, sizeof(t64)) == cudaSuccess) ? 1 : -1;
    });
    return g_tw_status[dev] == 1 ? PD_OK : fail(PD_ERR_CUDA, "twiddle upload failed");
}

template <int M>
int run_tma(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    constexpr int TO = P - 2 * M;
    const int nx = (int)g->n[0], ny = (int)g->n[1];
    CUtensorMap map;
    if (!fft_map(&map, a.u, nx, ny, a.batch)) return fail(PD_ERR_CUDA, "tensor map encode failed");
    const size_t smem = 2 * sizeof(float) * kFBX * P + sizeof(float2) * P * PS + sizeof(float) * 3 * (P / 2 + 1) * (P / 2 + 1);
    auto kern = k_fft_tile_tma<M>;
    static int attr_done[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr_done[dev] = 1;
    }
    const int tiles_x = (nx + TO - 1) / TO, tiles_y = (ny + TO - 1) / TO;
    const int64_t nt = (int64_t)tiles_x * tiles_y * a.batch;
    if (nt > (1ll << 30)) return fail(PD_ERR_INVALID, "too many tiles");
    int occ = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kT, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (occ < 1) occ = 1;
    const int blocks = (int)std::min<int64_t>(nt, (int64_t)occ * sms);
    double ct[3] = {0, 0, 0};
    for (int k = 0; k < g->nnb; ++k)
        for (int c = 0; c < 3; ++c) ct[c] += g->coef1[3 * k + c] * g->E;
    kern<<<blocks, kT, smem, s>>>(map, (float *)a.out, nx, ny, g->N, tiles_x, tiles_y, (int)nt, g->d_sym32, g->d_kd32,
                                  g->d_kt32, (float)ct[0], (float)ct[1], (float)ct[2], (float)a.scale,
                                  (const float *)a.u, g->d_err);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <typename T, int M>
int run(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (!a.project && !a.dot_partial && !a.no_tma && !g->no_tma && g->n[0] % 4 == 0 &&
            ((uintptr_t)a.u & 15) == 0 && tma2d::encode_fn() != nullptr)
            return run_tma<M>(g, a, s);
    }
    constexpr int TO = P - 2 * M;
    const size_t smem = sizeof(typename C2<T>::t) * P * PS + sizeof(T) * 3 * (P / 2 + 1) * (P / 2 + 1);
    auto kern = k_fft_tile<T, M>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((unsigned)((g->n[0] + TO - 1) / TO), (unsigned)((g->n[1] + TO - 1) / TO), (unsigned)a.batch);
    const bool f64 = sizeof(T) == 8;
    const T *sym = f64 ? (const T *)g->d_sym64 : (const T *)g->d_sym32;
    const T *kd = f64 ? (const T *)g->d_kd64 : (const T *)g->d_kd32;
    // interior diagonal block Ctot = sum of all c(o)
    double ct[3] = {0, 0, 0};
    for (int k = 0; k < g->nnb; ++k)
        for (int c = 0; c < 3; ++c) ct[c] += g->coef1[3 * k + c] * g->E;
    kern<<<grid, kT, smem, s>>>((const T *)a.u, (T *)a.out, (int)g->n[0], (int)g->n[1], g->N, g->d_cons,
                                a.project ? 1 : 0, sym, kd, g->d_kt32, (T)ct[0], (T)ct[1], (T)ct[2], (T)a.scale,
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
    return fail(PD_ERR_INVALID, "horizon M not compiled for the FFT path");
}

}  // namespace

// Tile symbol S[c][ky][kx] (c = xx, xy, yy) at the current modulus, scaled by 1/P^2,
// for 0 <= kx, ky <= P/2 (the kernel extends it by symmetry).
int fft_prepare(pd_grid *g)
{
    if (g->dim != 2) return PD_OK;
    int rc = upload_twiddles();
    if (rc) return rc;
    const double pi = 3.14159265358979323846;
    constexpr int QH = P / 2 + 1;   // kx, ky in [0, P/2]: the rest follows by symmetry
    std::vector<double> S(3 * QH * QH, 0.0);
    double ct[3] = {0, 0, 0};
    for (int k = 0; k < g->nnb; ++k)
        for (int c = 0; c < 3; ++c) ct[c] += g->coef1[3 * k + c] * g->E;
    for (int ky = 0; ky < QH; ++ky)
        for (int kx = 0; kx < QH; ++kx) {
            double acc[3] = {ct[0], ct[1], ct[2]};
            for (int k = 0; k < g->nnb; ++k) {
                const int ox = g->off[3 * k], oy = g->off[3 * k + 1];
                const int ph = ((kx * ox + ky * oy) % P + P) % P;
                const double cs = std::cos(2.0 * pi * ph / P);
                for (int c = 0; c < 3; ++c) acc[c] -= g->coef1[3 * k + c] * g->E * cs;
            }
            for (int c = 0; c < 3; ++c) S[(size_t)c * QH * QH + ky * QH + kx] = acc[c] / ((double)P * P);
        }
    std::vector<float> S32(S.begin(), S.end());
    if (!g->d_sym64) {
        PD_CUDA(cudaMalloc(&g->d_sym64, sizeof(double) * S.size()));
        PD_CUDA(cudaMalloc(&g->d_sym32, sizeof(float) * S.size()));
    }
    PD_CUDA(cudaMemcpy(g->d_sym64, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(g->d_sym32, S32.data(), sizeof(float) * S32.size(), cudaMemcpyHostToDevice));
    return PD_OK;
}

int launch_fft_tile(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s)
{
    if (g->dim == 3) return launch_fft3_tile(g, f64, a, s);
    if (a.batch < 1 || a.batch > 65535) return fail(PD_ERR_INVALID, "batch must be in [1, 65535]");
    if (!g->d_sym32) {
        int rc = fft_prepare(g);
        if (rc) return rc;
    }
    return f64 ? run_t<double>(g, a, s) : run_t<float>(g, a, s);
}

}  // namespace pd

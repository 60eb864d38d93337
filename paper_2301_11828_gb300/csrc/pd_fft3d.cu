// pd_fft3d.cu -- the TBTBT part of K u in 3D by FFT (Sec. 4, Algorithm 4),
// fused with the 3x3 symbol product, per 16^3 tile in shared memory.
//
// Same per-tile circulant embedding as the 2D kernel (pd_fft.cu): a CTA takes a
// 16^3 window of the zero-padded field whose centre (16 - 2M)^3 nodes are its
// outputs; the circular convolution over the window equals the Toeplitz product
// on them.  The three real components go through two complex transforms,
// z1 = u_x + i u_y and z2 = u_z.  Per tile:
//   1. load z1, z2 (zero outside the grid, projected if asked);
//   2. 16-point FFTs along x, y, z -- one thread owns one line and transforms
//      it in registers (4 x 4 radix with the W16 twiddles);
//   3. for each frequency pair (k, -k): U_x, U_y from Z1(k), Z1(-k), U_z = Z2;
//      H = S(k) U with the real symmetric 3x3 symbol S(k) = sum_o Kop(o)
//      cos(2 pi k.o / 16) / 16^3; repack W1 = H_x + i H_y, W2 = H_z;
//   4. inverse FFTs; epilogue: K u = (Re W1, Im W1, Re W2) - (Ctot - Kd_p) u_p
//      near faces (D^e), projection, scale, optional fused dot.
// Shared memory rows are padded to 17 elements so that the lines of a warp fall
// in distinct banks along every axis.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "pd_internal.cuh"
#include "pd_reduce.cuh"

namespace pd {
namespace {

constexpr int P3 = 16;
constexpr int RS = P3 + 1;        // padded row stride (complex)
constexpr int PL3 = P3 * RS;      // plane stride
constexpr int VOL = P3 * PL3;     // elements per signal
constexpr int kT3 = 256;          // one thread per line (16 x 16 lines per axis)

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

__constant__ float2 c_w16f[P3];
__constant__ double2 c_w16d[P3];
template <typename T> __device__ __forceinline__ typename V2<T>::t w16(int j);
template <> __device__ __forceinline__ float2 w16<float>(int j) { return c_w16f[j]; }
template <> __device__ __forceinline__ double2 w16<double>(int j) { return c_w16d[j]; }

template <typename V> __device__ __forceinline__ V vadd(V a, V b) { return {a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V vsub(V a, V b) { return {a.x - b.x, a.y - b.y}; }
template <bool INV, typename V> __device__ __forceinline__ V vmulw(V a, V w)
{
    if (INV) return {a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y};
    return {a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x};
}
template <bool INV, typename V> __device__ __forceinline__ V vmi(V a)   // * -i (forward) / * i (inverse)
{
    if (INV) return {-a.y, a.x};
    return {a.y, -a.x};
}

template <bool INV, typename V>
__device__ __forceinline__ void dft4(V &a, V &b, V &c, V &d)
{
    const V s0 = vadd(a, c), d0 = vsub(a, c), s1 = vadd(b, d), d1 = vmi<INV>(vsub(b, d));
    a = vadd(s0, s1);
    c = vsub(s0, s1);
    b = vadd(d0, d1);
    d = vsub(d0, d1);
}

// In-register 16-point DFT, n = 4 n1 + n2, k = k1 + 4 k2; result in natural order.
template <bool INV, typename T>
__device__ __forceinline__ void dft16(typename V2<T>::t (&x)[16])
{
    using V = typename V2<T>::t;
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        dft4<INV>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);   // -> slot 4 k1 + n2 holds Y[n2][k1]
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) x[4 * k1 + n2] = vmulw<INV>(x[4 * k1 + n2], w16<T>(n2 * k1));
    }
    V y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        V a = x[4 * k1], b = x[4 * k1 + 1], c = x[4 * k1 + 2], d = x[4 * k1 + 3];
        dft4<INV>(a, b, c, d);
        y[k1] = a;
        y[k1 + 4] = b;
        y[k1 + 8] = c;
        y[k1 + 12] = d;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = y[i];
}

// FFT of all 256 lines of one signal along one axis: stride es between elements,
// line (a, b) at a * sa + b * sb.
template <bool INV, typename T>
__device__ __forceinline__ void lines16(typename V2<T>::t *Z, int es, int sa, int sb)
{
    using V = typename V2<T>::t;
    const int a = threadIdx.x & 15, b = threadIdx.x >> 4;
    V *line = Z + a * sa + b * sb;
    V x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = line[i * es];
    dft16<INV, T>(x);
#pragma unroll
    for (int i = 0; i < 16; ++i) line[i * es] = x[i];
}

template <bool INV, typename T>
__device__ __forceinline__ void fft3(typename V2<T>::t *Z)
{
    lines16<INV, T>(Z, 1, RS, PL3);     // along x: lines indexed by (y, z)
    __syncthreads();
    lines16<INV, T>(Z, RS, 1, PL3);     // along y: lines indexed by (x, z)
    __syncthreads();
    lines16<INV, T>(Z, PL3, 1, RS);     // along z: lines indexed by (x, y)
    __syncthreads();
}

template <typename T, int M>
__global__ void __launch_bounds__(kT3)
k_fft3d_tile(const T *__restrict__ u, T *__restrict__ out, int nx, int ny, int nz, int tx_n, int ty_n, int tz_n,
             int64_t N, const uint8_t *__restrict__ cons, int project, const T *__restrict__ sym,
             const T *__restrict__ kd, const T *__restrict__ ct, T scale, double *dot_partial, double *dot_out,
             unsigned int *retire)
{
    using V = typename V2<T>::t;
    constexpr int TO = P3 - 2 * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *Z1 = reinterpret_cast<V *>(smem_raw);
    V *Z2 = Z1 + VOL;

    const int per = tx_n * ty_n * tz_n;
    const int64_t b = blockIdx.x / per;
    const int tix = blockIdx.x - (int)b * per;
    const int x0 = (tix % tx_n) * TO - M, y0 = ((tix / tx_n) % ty_n) * TO - M, z0 = (tix / (tx_n * ty_n)) * TO - M;
    const T *ub = u + b * 3 * N;
    T *ob = out + b * 3 * N;
    // the tile's reference value (the projected input at its first output node): K maps a
    // constant to zero on every row, so the transforms take u - c (see the 2D tile)
    T c0v, c1v, c2v;
    {
        const int64_t p0 = ((int64_t)(z0 + M) * ny + (y0 + M)) * nx + (x0 + M);
        c0v = __ldg(ub + p0);
        c1v = __ldg(ub + N + p0);
        c2v = __ldg(ub + 2 * N + p0);
        if (project) {
            const uint8_t m = __ldg(cons + p0);
            if (m & 1) c0v = T(0);
            if (m & 2) c1v = T(0);
            if (m & 4) c2v = T(0);
        }
    }

    // fully unrolled: the window's loads are all in flight before the first store
#pragma unroll
    for (int t = threadIdx.x; t < P3 * P3 * P3; t += kT3) {
        const int x = t & 15, y = (t >> 4) & 15, z = t >> 8;
        const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
        V v1 = {T(0), T(0)}, v2 = {T(0), T(0)};
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz) {
            const int64_t p = ((int64_t)gz * ny + gy) * nx + gx;
            T a0 = __ldg(ub + p), a1 = __ldg(ub + N + p), a2 = __ldg(ub + 2 * N + p);
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) a0 = T(0);
                if (m & 2) a1 = T(0);
                if (m & 4) a2 = T(0);
            }
            v1.x = a0 - c0v;
            v1.y = a1 - c1v;
            v2.x = a2 - c2v;
        }
        const int e = z * PL3 + y * RS + x;
        Z1[e] = v1;
        Z2[e] = v2;
    }
    __syncthreads();
    fft3<false, T>(Z1);
    fft3<false, T>(Z2);

    for (int t = threadIdx.x; t < P3 * P3 * P3; t += kT3) {
        const int kx = t & 15, ky = (t >> 4) & 15, kz = t >> 8;
        const int mx = (16 - kx) & 15, my = (16 - ky) & 15, mz = (16 - kz) & 15;
        const int t2 = (mz << 8) | (my << 4) | mx;
        if (t2 < t) continue;
        const int e = kz * PL3 + ky * RS + kx, e2 = mz * PL3 + my * RS + mx;
        const V zk = Z1[e], zm0 = Z1[e2];
        const V zm = {zm0.x, -zm0.y};
        const V ux = {T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y + zm.y)};
        const V uy = {T(0.5) * (zk.y - zm.y), T(-0.5) * (zk.x - zm.x)};
        const V uz = Z2[e], uzm = Z2[e2];
        const T sxx = __ldg(sym + t), sxy = __ldg(sym + 4096 + t), sxz = __ldg(sym + 2 * 4096 + t);
        const T syy = __ldg(sym + 3 * 4096 + t), syz = __ldg(sym + 4 * 4096 + t), szz = __ldg(sym + 5 * 4096 + t);
        const V hx = {sxx * ux.x + sxy * uy.x + sxz * uz.x, sxx * ux.y + sxy * uy.y + sxz * uz.y};
        const V hy = {sxy * ux.x + syy * uy.x + syz * uz.x, sxy * ux.y + syy * uy.y + syz * uz.y};
        const V hz = {sxz * ux.x + syz * uy.x + szz * uz.x, sxz * ux.y + syz * uy.y + szz * uz.y};
        Z1[e] = {hx.x - hy.y, hx.y + hy.x};
        Z2[e] = hz;
        if (t2 != t) {
            // U(-k) = conj U(k) for the real components x, y; the stored Z2(-k) for z
            Z1[e2] = {hx.x + hy.y, hy.x - hx.y};
            Z2[e2] = {sxz * ux.x + syz * uy.x + szz * uzm.x, -(sxz * ux.y + syz * uy.y) + szz * uzm.y};
        }
    }
    __syncthreads();
    fft3<true, T>(Z1);
    fft3<true, T>(Z2);

    T dot = T(0);
    for (int t = threadIdx.x; t < TO * TO * TO; t += kT3) {
        const int x = M + t % TO, y = M + (t / TO) % TO, z = M + t / (TO * TO);
        const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
        if (gx >= nx || gy >= ny || gz >= nz) continue;
        const int64_t p = ((int64_t)gz * ny + gy) * nx + gx;
        const int e = z * PL3 + y * RS + x;
        T f0 = Z1[e].x, f1 = Z1[e].y, f2 = Z2[e].x;
        const int a0 = min(gx, M), a1 = min(nx - 1 - gx, M), b0 = min(gy, M), b1 = min(ny - 1 - gy, M),
                  c0 = min(gz, M), c1 = min(nz - 1 - gz, M);
        const bool edge = (a0 != M || a1 != M || b0 != M || b1 != M || c0 != M || c1 != M);
        const uint8_t m = project ? __ldg(cons + p) : 0;
        if (edge || dot_partial) {
            T u0 = __ldg(ub + p), u1 = __ldg(ub + N + p), u2 = __ldg(ub + 2 * N + p);
            if (m & 1) u0 = T(0);
            if (m & 2) u1 = T(0);
            if (m & 4) u2 = T(0);
            if (edge) {
                const int cls = ((((a0 * (M + 1) + a1) * (M + 1) + b0) * (M + 1) + b1) * (M + 1) + c0) * (M + 1) + c1;
                const T *q = kd + 6 * cls;
                const T dxx = ct[0] - q[0], dxy = ct[1] - q[1], dxz = ct[2] - q[2], dyy = ct[3] - q[3],
                        dyz = ct[4] - q[4], dzz = ct[5] - q[5];
                const T s0 = u0 - c0v, s1 = u1 - c1v, s2 = u2 - c2v;   // the shifted field of the transforms
                f0 -= dxx * s0 + dxy * s1 + dxz * s2;
                f1 -= dxy * s0 + dyy * s1 + dyz * s2;
                f2 -= dxz * s0 + dyz * s1 + dzz * s2;
            }
            if (m & 1) f0 = T(0);
            if (m & 2) f1 = T(0);
            if (m & 4) f2 = T(0);
            f0 *= scale;
            f1 *= scale;
            f2 *= scale;
            dot += u0 * f0 + u1 * f1 + u2 * f2;
        } else {
            if (m & 1) f0 = T(0);
            if (m & 2) f1 = T(0);
            if (m & 4) f2 = T(0);
            f0 *= scale;
            f1 *= scale;
            f2 *= scale;
        }
        ob[p] = f0;
        ob[N + p] = f1;
        ob[2 * N + p] = f2;
    }
    if (dot_partial) {
        __shared__ double red[kT3 / 32];
        const double s = block_sum(dot, red);
        grid_finish(s, per, tix, dot_partial + b * per, dot_out + b, retire + b, red);
    }
}

std::once_flag g_w16_once[64];
int g_w16_status[64];

int upload_w16()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(PD_ERR_CUDA, "device query");
    std::call_once(g_w16_once[dev], [&] {
        float2 f[P3];
        double2 d[P3];
        const double pi = 3.14159265358979323846;
        for (int j = 0; j < P3; ++j) {
            const double ang = -2.0 * pi * j / P3;
            d[j] = make_double2(std::cos(ang), std::sin(ang));
            f[j] = make_float2((float)d[j].x, (float)d[j].y);
        }
        g_w16_status[dev] = (cudaMemcpyToSymbol(c_w16f, f, sizeof(f)) == cudaSuccess &&
                             cudaMemcpyToSymbol(c_w16d, d, sizeof(d)) == cudaSuccess) ? 1 : -1;
    });
    return g_w16_status[dev] == 1 ? PD_OK : fail(PD_ERR_CUDA, "twiddle upload failed");
}

template <typename T, int M>
int run3(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    constexpr int TO = P3 - 2 * M;
    const size_t smem = sizeof(typename V2<T>::t) * 2 * VOL;
    auto kern = k_fft3d_tile<T, M>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int txn = (int)((g->n[0] + TO - 1) / TO), tyn = (int)((g->n[1] + TO - 1) / TO),
              tzn = (int)((g->n[2] + TO - 1) / TO);
    const int64_t blocks = (int64_t)txn * tyn * tzn * a.batch;
    if (blocks > 0x7fffffff) return fail(PD_ERR_INVALID, "too many FFT tiles");
    const bool f64 = sizeof(T) == 8;
    const T *sym = f64 ? (const T *)g->d_sym3_64 : (const T *)g->d_sym3_32;
    const T *kd = f64 ? (const T *)g->d_kd64 : (const T *)g->d_kd32;
    const T *ct = f64 ? (const T *)g->d_ctot64 : (const T *)g->d_ctot32;
    kern<<<(unsigned)blocks, kT3, smem, s>>>((const T *)a.u, (T *)a.out, (int)g->n[0], (int)g->n[1], (int)g->n[2],
                                              txn, tyn, tzn, g->N, g->d_cons, a.project ? 1 : 0, sym, kd, ct,
                                              (T)a.scale, a.dot_partial, a.dot_out, a.retire);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <typename T>
int run3_t(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    switch (g->M) {
        case 1: return run3<T, 1>(g, a, s);
        case 2: return run3<T, 2>(g, a, s);
        case 3: return run3<T, 3>(g, a, s);
        case 4: return run3<T, 4>(g, a, s);
    }
    return fail(PD_ERR_INVALID, "horizon M not compiled for the 3D FFT path");
}

}  // namespace

// 3D tile symbol S[c][kz][ky][kx] (c = xx, xy, xz, yy, yz, zz) at the current
// modulus, scaled by 1/16^3, and the interior diagonal block Ctot.
int fft3_prepare(pd_grid *g)
{
    int rc = upload_w16();
    if (rc) return rc;
    const double pi = 3.14159265358979323846;
    double ct[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < g->nnb; ++k)
        for (int c = 0; c < 6; ++c) ct[c] += g->coef1[6 * k + c] * g->E;
    std::vector<double> S(6 * 4096);
    for (int kz = 0; kz < P3; ++kz)
        for (int ky = 0; ky < P3; ++ky)
            for (int kx = 0; kx < P3; ++kx) {
                double acc[6];
                for (int c = 0; c < 6; ++c) acc[c] = ct[c];
                for (int k = 0; k < g->nnb; ++k) {
                    const int *o = &g->off[3 * k];
                    const int ph = (((kx * o[0] + ky * o[1] + kz * o[2]) % P3) + P3) % P3;
                    const double cs = std::cos(2.0 * pi * ph / P3);
                    for (int c = 0; c < 6; ++c) acc[c] -= g->coef1[6 * k + c] * g->E * cs;
                }
                for (int c = 0; c < 6; ++c) S[(size_t)c * 4096 + (kz * 16 + ky) * 16 + kx] = acc[c] / 4096.0;
            }
    std::vector<float> S32(S.begin(), S.end());
    float ct32[6];
    for (int c = 0; c < 6; ++c) ct32[c] = (float)ct[c];
    if (!g->d_sym3_64) {
        PD_CUDA(cudaMalloc(&g->d_sym3_64, sizeof(double) * S.size()));
        PD_CUDA(cudaMalloc(&g->d_sym3_32, sizeof(float) * S.size()));
        PD_CUDA(cudaMalloc(&g->d_ctot64, sizeof(double) * 6));
        PD_CUDA(cudaMalloc(&g->d_ctot32, sizeof(float) * 6));
    }
    PD_CUDA(cudaMemcpy(g->d_sym3_64, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(g->d_sym3_32, S32.data(), sizeof(float) * S32.size(), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(g->d_ctot64, ct, sizeof(double) * 6, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(g->d_ctot32, ct32, sizeof(float) * 6, cudaMemcpyHostToDevice));
    return PD_OK;
}

int launch_fft3_tile(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s)
{
    if (a.batch < 1) return fail(PD_ERR_INVALID, "batch must be >= 1");
    if (!g->d_sym3_32) {
        int rc = fft3_prepare(g);
        if (rc) return rc;
    }
    return f64 ? run3_t<double>(g, a, s) : run3_t<float>(g, a, s);
}

}  // namespace pd

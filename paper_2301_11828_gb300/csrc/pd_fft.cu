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
//      with c the value at one in-grid node of the window: K maps a constant
//      field to zero on every row (the edge rows included), so K(u - c) = K u,
//      and the transforms then round values of the size of u's variation over
//      the tile instead of u's own (a field with a large constant part would
//      otherwise carry that part's rounding into every output);
//   2. 64-point FFTs along x, then along y (each as 8 x 8, in two register
//      passes with the twiddles W64^(n2 k1) between them);
//   3. for each frequency pair (k, -k): unpack U_x, U_y from Z(k), Z(-k)
//      (both components are real), multiply by the real 2x2 symbol
//      S(k) = sum_o Kop(o) cos(2 pi k.o / P) / P^2 (Kop(0) = sum c, Kop(o) = -c(o);
//      the kernel is even, so S is real; a quarter of it is staged in shared
//      memory), repack W = H_x + i H_y;
//   4. inverse FFTs along y then x;
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

// 64-point FFT of 64 lines (rows: es = 1, ls = PS; columns: es = PS, ls = 1).
// Thread mapping: lane -> line (and line + 32), warp -> the 8-point group index,
// so every shared-memory access of a warp hits distinct banks.
template <bool INV, typename T>
__device__ __forceinline__ void fft64_lines(typename C2<T>::t *Z, int es, int ls)
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
        dft8<INV, V, T>(v[h]);
#pragma unroll
        for (int k1 = 1; k1 < 8; ++k1) v[h][k1] = cmulw<INV>(v[h][k1], tw<T>(g * k1));
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) line[(8 * k1 + g) * es] = v[h][k1];
    }
    __syncthreads();
    // pass 2: group g = k1; slots 8 k1 + n2 -> DFT over n2 -> X[k1 + 8 k2]
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        V *line = Z + (lane + 32 * h) * ls;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) v[h][n2] = line[(8 * g + n2) * es];
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        V *line = Z + (lane + 32 * h) * ls;
        dft8<INV, V, T>(v[h]);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) line[(g + 8 * k2) * es] = v[h][k2];
    }
    __syncthreads();
}

template <typename T, int M>
__global__ void __launch_bounds__(kT)
k_fft_tile(const T *__restrict__ u, T *__restrict__ out, int nx, int ny, int64_t N,
           const uint8_t *__restrict__ cons, int project, const T *__restrict__ sym, const T *__restrict__ kd,
           T ctxx, T ctxy, T ctyy, T scale, double *dot_partial, double *dot_out, unsigned int *retire)
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

    for (int t = threadIdx.x; t < P * P; t += kT) {
        const int a = t % P, r = t / P;
        const int gx = x0 + a, gy = y0 + r;
        V z = {T(0), T(0)};
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
            const int64_t p = (int64_t)gy * nx + gx;
            T vx = __ldg(ub + p), vy = __ldg(ub + N + p);
            if (project) {
                const uint8_t m = __ldg(cons + p);
                if (m & 1) vx = T(0);
                if (m & 2) vy = T(0);
            }
            z.x = vx - cx;
            z.y = vy - cy;
        }
        Z[r * PS + a] = z;
    }
    __syncthreads();

    fft64_lines<false, T>(Z, 1, PS);    // rows (along x)
    fft64_lines<false, T>(Z, PS, 1);    // columns (along y)

    // symbol product on frequency pairs (k, -k)
    for (int t = threadIdx.x; t < P * P; t += kT) {
        const int kx = t % P, ky = t / P;
        const int mx = (P - kx) & (P - 1), my = (P - ky) & (P - 1);
        const int t2 = my * P + mx;
        if (t2 < t) continue;
        const V zk = Z[ky * PS + kx], zm0 = Z[my * PS + mx];
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
        Z[ky * PS + kx] = {hx.x - hy.y, hx.y + hy.x};
        if (t2 != t) Z[my * PS + mx] = {hx.x + hy.y, hy.x - hx.y};
    }
    __syncthreads();

    fft64_lines<true, T>(Z, PS, 1);     // columns
    fft64_lines<true, T>(Z, 1, PS);     // rows

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
                const T zx = upx - cx, zy = upy - cy;
                fx -= dxx * zx + dxy * zy;
                fy -= dxy * zx + dyy * zy;
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
               float ctxx, float ctxy, float ctyy, float scale, const float *__restrict__ u, int *err)
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
        // the tile's reference value: the input at its first output node (always in the grid)
        const float cx = sx[M * kFBX + M + d], cy = sy[M * kFBX + M + d];
        for (int e = threadIdx.x; e < P * P; e += kT) {
            const int a = e % P, r = e / P;
            const int gx = x0 + a, gy = y0 + r;
            V z = {0.f, 0.f};
            if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                z.x = sx[r * kFBX + a + d] - cx;
                z.y = sy[r * kFBX + a + d] - cy;
            }
            Z[r * PS + a] = z;
        }
        __syncthreads();   // the staged box is free: the next tile's window is copied meanwhile
        if (threadIdx.x == 0 && t + (int)gridDim.x < ntiles) issue(t + gridDim.x);

        fft64_lines<false, float>(Z, 1, PS);
        fft64_lines<false, float>(Z, PS, 1);
        for (int e = threadIdx.x; e < P * P; e += kT) {
            const int kx = e % P, ky = e / P;
            const int mx = (P - kx) & (P - 1), my = (P - ky) & (P - 1);
            const int t2 = my * P + mx;
            if (t2 < e) continue;
            const V zk = Z[ky * PS + kx], zm0 = Z[my * PS + mx];
            const V zm = {zm0.x, -zm0.y};
            const V ux = {0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y)};
            const V uy = {0.5f * (zk.y - zm.y), -0.5f * (zk.x - zm.x)};
            const int qx = kx <= P / 2 ? kx : P - kx, qy = ky <= P / 2 ? ky : P - ky;
            const int qi = qy * QH + qx;
            const float sgn = ((kx > P / 2) != (ky > P / 2)) ? -1.f : 1.f;
            const float sxx = sq[qi], sxy = sgn * sq[QH * QH + qi], syy = sq[2 * QH * QH + qi];
            const V hx = {sxx * ux.x + sxy * uy.x, sxx * ux.y + sxy * uy.y};
            const V hy = {sxy * ux.x + syy * uy.x, sxy * ux.y + syy * uy.y};
            Z[ky * PS + kx] = {hx.x - hy.y, hx.y + hy.x};
            if (t2 != e) Z[my * PS + mx] = {hx.x + hy.y, hy.x - hx.y};
        }
        __syncthreads();
        fft64_lines<true, float>(Z, PS, 1);
        fft64_lines<true, float>(Z, 1, PS);

        const float *ub = u + (int64_t)b * 2 * N;
        float *ob = out + (int64_t)b * 2 * N;
        for (int e = threadIdx.x; e < TO * TO; e += kT) {
            const int a = M + e % TO, r = M + e / TO;
            const int gx = x0 + a, gy = y0 + r;
            if (gx >= nx || gy >= ny) continue;
            const int64_t p = (int64_t)gy * nx + gx;
            const V w = Z[r * PS + a];
            float fx = w.x, fy = w.y;
            const int a0 = min(gx, M), a1 = min(nx - 1 - gx, M), b0 = min(gy, M), b1 = min(ny - 1 - gy, M);
            if (a0 != M || a1 != M || b0 != M || b1 != M) {   // the D^e term on the shifted field
                const int cls = ((a0 * (M + 1) + a1) * (M + 1) + b0) * (M + 1) + b1;
                const float dxx = ctxx - __ldg(kd + 3 * cls), dxy = ctxy - __ldg(kd + 3 * cls + 1),
                            dyy = ctyy - __ldg(kd + 3 * cls + 2);
                const float zx = __ldg(ub + p) - cx, zy = __ldg(ub + N + p) - cy;
                fx -= dxx * zx + dxy * zy;
                fy -= dxy * zx + dyy * zy;
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
                                  (float)ct[0], (float)ct[1], (float)ct[2], (float)a.scale, (const float *)a.u,
                                  g->d_err);
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
                                a.project ? 1 : 0, sym, kd, (T)ct[0], (T)ct[1], (T)ct[2], (T)a.scale, a.dot_partial,
                                a.dot_out, a.retire);
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

// pd_tma2d.cuh -- shared pieces of the TMA-fed FP32 2D stencil kernels
// (the batched matvec in pd_stencil2d_tma.cu and the persistent CG in
// pd_cg_persist.cu): packed FP32x2 helpers, mbarrier / TMA wrappers, the tile
// geometry, the packed coefficient table and the per-tile pair sums of the TBT
// form (Sec. 3.2-3.4).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "pd_stencil.cuh"

namespace pd {
namespace tma2d {

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float a, float b)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk(u64 r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ u64 fadd2(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fsub2(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fmul2(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One arrival (release semantics at CTA scope) on a barrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the phase with the given parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((const void *)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

constexpr int kTXt = 64;                 // outputs per tile along x
constexpr int kRt = 8;                   // outputs per thread along y
constexpr int kTYt = kGY2 * kRt;         // outputs per tile along y (32)

template <int M>
__host__ __device__ constexpr int x_lead() { return M <= 4 ? 4 : 8; }   // 16-byte aligned halo on the left
template <int M>
__host__ __device__ constexpr int box_x() { return kTXt + 2 * x_lead<M>(); }
template <int M>
__host__ __device__ constexpr int box_y() { return kTYt + 2 * M; }

// Pair coefficients packed for the FP32x2 form: (cxx, cyy) and (cxy, cxy) per pair,
// then the interior Kd (xx, xy, yy, pad).
template <int M>
struct __align__(16) PackTab {
    static constexpr int kPairs = count_offsets(2, M) / 2;
    float v[4 * kPairs + 4];
};

// Per-tile pair sums.  colx / coly point at the thread's column (first halo
// row) in the x / y planes of a staged box of row length BX.  On return a1, a2
// hold the packed accumulators of sum_{o in half} c(o) s_o with
//   s_o = u~_{p+o} + u~_{p-o}                     (DIFF = false, pair form), or
//   s_o = (u~_{p+o} - u_p) + (u~_{p-o} - u_p)     (DIFF = true, difference form),
// (f_x = a1.x + a2.y, f_y = a1.y + a2.x), and w0 the thread's own column
// (w0[r + M] = u_p of output r).  The pair form leaves K u = Kd_p u_p - a: for a
// smooth field its terms nearly cancel, so its FP32 error is relative to
// sum |c||u| rather than to |K u|.  The difference form rounds the small
// differences instead and gives K u = (Kd_p - Kd_int) u_p - a, where Kd_int =
// 2 sum c(o) is the interior diagonal; it costs two packed subtractions more
// per general pair and two scalar ones per axis pair.
template <int M, bool DIFF = false>
__device__ __forceinline__ void tile_pairs(const float *colx, const float *coly, const PackTab<M> &tab,
                                           u64 (&a1)[kRt], u64 (&a2)[kRt], u64 (&w0)[kRt + 2 * M])
{
    constexpr int BX = box_x<M>(), WL = kRt + 2 * M;
#pragma unroll
    for (int r = 0; r < kRt; ++r) { a1[r] = 0ull; a2[r] = 0ull; }
    u64 ctr[DIFF ? kRt : 1];   // difference form: u_p of each output
    if constexpr (DIFF) {
#pragma unroll
        for (int r = 0; r < kRt; ++r) ctr[r] = pk(colx[(r + M) * BX], coly[(r + M) * BX]);
    }
    static_for<1, M + 1>([&](auto OX) {
        constexpr int ox = decltype(OX)::value;
        constexpr int My = isqrt_c(M * M - ox * ox);
        u64 wp[WL], wm[WL];
#pragma unroll
        for (int i = 0; i < WL; ++i) {
            wp[i] = pk(colx[i * BX + ox], coly[i * BX + ox]);
            wm[i] = pk(colx[i * BX - ox], coly[i * BX - ox]);
        }
        static_for<-My, My + 1>([&](auto OY) {
            constexpr int oy = decltype(OY)::value;
            if constexpr (oy != 0) {
                constexpr int pi = pair_index2(M, ox, oy);
                const u64 c1 = *reinterpret_cast<const u64 *>(&tab.v[4 * pi]);
                const u64 c2 = *reinterpret_cast<const u64 *>(&tab.v[4 * pi + 2]);
#pragma unroll
                for (int r = 0; r < kRt; ++r) {
                    u64 s;
                    if constexpr (DIFF)
                        s = fadd2(fsub2(wp[r + M + oy], ctr[r]), fsub2(wm[r + M - oy], ctr[r]));
                    else
                        s = fadd2(wp[r + M + oy], wm[r + M - oy]);
                    a1[r] = ffma2(c1, s, a1[r]);
                    a2[r] = ffma2(c2, s, a2[r]);
                }
            }
        });
        // Axis pair (ox, 0): c(o) = diag(c_xx, 0) exactly, so only the x
        // component is summed (scalar: one add and one FMA per output).
        {
            constexpr int pi = pair_index2(M, ox, 0);
            const float cxx = tab.v[4 * pi];
#pragma unroll
            for (int r = 0; r < kRt; ++r) {
                const float2 p2 = upk(wp[r + M]), m2 = upk(wm[r + M]);
                float2 acc = upk(a1[r]);
                float sx;
                if constexpr (DIFF) {
                    const float cx = upk(ctr[r]).x;
                    sx = (p2.x - cx) + (m2.x - cx);
                } else {
                    sx = p2.x + m2.x;
                }
                acc.x = __fmaf_rn(cxx, sx, acc.x);
                a1[r] = pk(acc.x, acc.y);
            }
        }
    });
#pragma unroll
    for (int i = 0; i < WL; ++i) w0[i] = pk(colx[i * BX], coly[i * BX]);
    // Axis pairs (0, oy): c(o) = diag(0, c_yy) exactly; only the y component.
    static_for<1, M + 1>([&](auto OY) {
        constexpr int oy = decltype(OY)::value;
        constexpr int pi = pair_index2(M, 0, oy);
        const float cyy = tab.v[4 * pi + 1];
#pragma unroll
        for (int r = 0; r < kRt; ++r) {
            const float2 p2 = upk(w0[r + M + oy]), m2 = upk(w0[r + M - oy]);
            float2 acc = upk(a1[r]);
            float sy;
            if constexpr (DIFF) {
                const float cy = upk(w0[r + M]).y;
                sy = (p2.y - cy) + (m2.y - cy);
            } else {
                sy = p2.y + m2.y;
            }
            acc.y = __fmaf_rn(cyy, sy, acc.y);
            a1[r] = pk(acc.x, acc.y);
        }
    });
}

// ---- the accurate (cancellation-free) form of the pair sums
//
// K u at node p is -sum_{o in half} c(o) s_o with s_o = (u~_{p+o} - u_p) + (u~_{p-o} - u_p)
// (u~ the input, the sum over in-grid neighbours only).  Written this way every
// term is a difference of nearby values, so the FP32 rounding error stays
// relative to |K u| even where the field is smooth or carries a large constant
// part (the pair form Kd u_p - sum c (u_{p+o} + u_{p-o}) loses the digits that
// cancel).  Two evaluations of the same sum:
//
//  * tile_eg (every neighbour of the warp's outputs inside the grid): the pair
//    sums are regrouped into horizontal second and central differences shared
//    by the outputs of a column, plus vertical second differences in the
//    thread's own column (below);
//  * tile_diff<M, true> (some neighbour outside the grid): the plain difference
//    form with every term whose neighbour lies outside the grid dropped, i.e.
//    the in-grid bond sum of Eq. mat:f1 itself (no diagonal table, no
//    cancelling edge self-term).
//
// AccTab holds the coefficients premultiplied by -scale, so that
//   (K u)_x = a1.x + a2.y,  (K u)_y = a1.y + a2.x.
template <int M>
struct __align__(16) AccTab {
    static constexpr int kPairs = count_offsets(2, M) / 2;
    // per pair (pair_index2 order): c1 = (cxx, cyy), c2 = (cxy, cxy);
    // then per k = 1..M the vertical block Cbar(k) = (cxx, cyy)
    float v[4 * kPairs + 2 * M];
};

template <int M>
__device__ __forceinline__ u64 acc_c1(const AccTab<M> &t, int pi) { return *reinterpret_cast<const u64 *>(&t.v[4 * pi]); }
template <int M>
__device__ __forceinline__ u64 acc_c2(const AccTab<M> &t, int pi) { return *reinterpret_cast<const u64 *>(&t.v[4 * pi + 2]); }
template <int M>
__device__ __forceinline__ u64 acc_w(const AccTab<M> &t, int k)
{
    return *reinterpret_cast<const u64 *>(&t.v[4 * AccTab<M>::kPairs + 2 * (k - 1)]);
}

// The interior sums.  With H_ox(i) = u(x+ox, i) - u(x, i) and, in the thread's
// own column, V_k(r) = u(x, r+k) - u(x, r), each pair sum splits as
//   s_(ox,oy) = H_ox(r+oy) + H_-ox(r-oy) + W_|oy|(r),   W_k = V_k + V_-k.
// The vertical second difference W_k(r) is shared by every pair with |oy| = k;
// it enters once with Cbar(k) = sum of c(o) over those pairs (diagonal: the xy
// entries of (ox, k) and (ox, -k) cancel exactly).  The pairs (ox, k) and
// (ox, -k) are then taken together: with E(i) = H_ox(i) + H_-ox(i) (the
// horizontal second difference of row i) and G(i) = u(x+ox, i) - u(x-ox, i),
//   s_(ox,k) + s_(ox,-k) = E(r+k) + E(r-k) + 2 W_k(r),
//   s_(ox,k) - s_(ox,-k) = G(r+k) - G(r-k),
// and since c(ox,-k) has the xx / yy entries of c(ox,k) and the opposite xy
// entry, the two pairs contribute (cxx, cyy) (E(r+k) + E(r-k)) to a1 and
// (cxy, cxy) (G(r+k) - G(r-k)) to a2.  E and G are formed once per row and
// column offset and shared by the column's outputs; the axis pair (ox, 0) is
// cxx E(r) on the x component alone.  Every operand is a difference of nearby
// values.  At M = 3: about 42 FP32x2 and 5 FP32 operations per output (the
// plain difference form takes 64, the pair form 36 with its cancellation).
template <int M>
__device__ __forceinline__ void tile_eg(const float *colx, const float *coly, const AccTab<M> &tab,
                                        u64 (&a1)[kRt], u64 (&a2)[kRt])
{
    constexpr int BX = box_x<M>(), WL = kRt + 2 * M;
    u64 w0[WL];
#pragma unroll
    for (int i = 0; i < WL; ++i) w0[i] = pk(colx[i * BX], coly[i * BX]);
    // vertical part: V_k(j) = u(x, j + k) - u(x, j); W_k(r) = V_k(r + M) - V_k(r + M - k)
    static_for<1, M + 1>([&](auto K) {
        constexpr int k = decltype(K)::value;
        const u64 c = acc_w(tab, k);
        u64 V[WL];
#pragma unroll
        for (int j = M - k; j < kRt + M; ++j) V[j] = fsub2(w0[j + k], w0[j]);
#pragma unroll
        for (int r = 0; r < kRt; ++r) {
            const u64 W = fsub2(V[r + M], V[r + M - k]);
            if constexpr (k == 1)
                a1[r] = fmul2(c, W);
            else
                a1[r] = ffma2(c, W, a1[r]);
        }
    });
#pragma unroll
    for (int r = 0; r < kRt; ++r) a2[r] = 0ull;
    static_for<1, M + 1>([&](auto OX) {
        constexpr int ox = decltype(OX)::value;
        constexpr int My = isqrt_c(M * M - ox * ox);
        const float cxx = tab.v[4 * pair_index2(M, ox, 0)];
        if constexpr (My == 0) {
            // only the axis pair (ox, 0): the x component of E alone, in scalar FP32
#pragma unroll
            for (int r = 0; r < kRt; ++r) {
                const int i = r + M;
                const float ux = upk(w0[i]).x;
                const float e = (colx[i * BX + ox] - ux) + (colx[i * BX - ox] - ux);
                float2 acc = upk(a1[r]);
                acc.x = __fmaf_rn(cxx, e, acc.x);
                a1[r] = pk(acc.x, acc.y);
            }
            return;
        }
        u64 E[WL], G[WL];
#pragma unroll
        for (int i = M - My; i < kRt + M + My; ++i) {
            const u64 wp = pk(colx[i * BX + ox], coly[i * BX + ox]);
            const u64 wm = pk(colx[i * BX - ox], coly[i * BX - ox]);
            E[i] = fadd2(fsub2(wp, w0[i]), fsub2(wm, w0[i]));
            G[i] = fsub2(wp, wm);
        }
        {   // axis pair (ox, 0): x component only
#pragma unroll
            for (int r = 0; r < kRt; ++r) {
                const float2 e = upk(E[r + M]);
                float2 acc = upk(a1[r]);
                acc.x = __fmaf_rn(cxx, e.x, acc.x);
                a1[r] = pk(acc.x, acc.y);
            }
        }
        static_for<1, My + 1>([&](auto K) {
            constexpr int k = decltype(K)::value;
            constexpr int pi = pair_index2(M, ox, k);
            const u64 c1 = acc_c1(tab, pi), c2 = acc_c2(tab, pi);
#pragma unroll
            for (int r = 0; r < kRt; ++r) {
                a1[r] = ffma2(c1, fadd2(E[r + M + k], E[r + M - k]), a1[r]);
                a2[r] = ffma2(c2, fsub2(G[r + M + k], G[r + M - k]), a2[r]);
            }
        });
    });
}

// Plain difference form, s_o = (u~_{p+o} - u_p) + (u~_{p-o} - u_p) for every
// pair, walked column offset by column offset with the outputs of a column in
// the outer loop, so that only a few window rows per column are live.  With
// MASK (warps holding an output whose horizon leaves the grid), each term whose
// neighbour lies outside [0,nx) x [0,ny) is dropped: that is the in-grid bond
// sum of Eq. mat:f1 itself (no diagonal table, no cancelling edge self-term).
// gx is the thread's grid column, gyw the grid row of window row 0.  The staged
// box must hold zeros outside the grid (the tensor map's fill).
template <int M, bool MASK>
__device__ __forceinline__ void tile_diff(const float *colx, const float *coly, const AccTab<M> &tab,
                                          u64 (&a1)[kRt], u64 (&a2)[kRt], int gx, int nx, int gyw, int ny)
{
    constexpr int BX = box_x<M>(), WL = kRt + 2 * M;
    static_assert(WL <= 32, "row mask is one word");
    uint32_t rowok = 0;
    if constexpr (MASK) {
#pragma unroll
        for (int i = 0; i < WL; ++i)
            if (gyw + i >= 0 && gyw + i < ny) rowok |= 1u << i;
    }
    u64 ctr[kRt];
#pragma unroll
    for (int r = 0; r < kRt; ++r) {
        a1[r] = 0ull;
        a2[r] = 0ull;
        ctr[r] = pk(colx[(r + M) * BX], coly[(r + M) * BX]);
    }
    static_for<0, M + 1>([&](auto OX) {
        constexpr int ox = decltype(OX)::value;
        constexpr int My = isqrt_c(M * M - ox * ox);
        const bool cp = gx + ox < nx, cm = gx - ox >= 0;
#pragma unroll
        for (int r = 0; r < kRt; ++r) {
            static_for<-My, My + 1>([&](auto OY) {
                constexpr int oy = decltype(OY)::value;
                if constexpr (ox > 0 || oy > 0) {
                    constexpr int pi = pair_index2(M, ox, oy);
                    const int ip = r + M + oy, im = r + M - oy;
                    const u64 vp = pk(colx[ip * BX + ox], coly[ip * BX + ox]);
                    const u64 vm = pk(colx[im * BX - ox], coly[im * BX - ox]);
                    u64 dp, dm;
                    if constexpr (MASK) {
                        // outside the grid the staged value is the tensor map's zero fill, so
                        // m (v - u_p) = v - m u_p with m = 1 inside and 0 outside: one FMA
                        const float fp = (cp && ((rowok >> ip) & 1u)) ? -1.f : 0.f;
                        const float fm = (cm && ((rowok >> im) & 1u)) ? -1.f : 0.f;
                        dp = ffma2(pk(fp, fp), ctr[r], vp);
                        dm = ffma2(pk(fm, fm), ctr[r], vm);
                    } else {
                        dp = fsub2(vp, ctr[r]);
                        dm = fsub2(vm, ctr[r]);
                    }
                    const u64 sum = fadd2(dp, dm);
                    a1[r] = ffma2(acc_c1(tab, pi), sum, a1[r]);
                    if constexpr (ox != 0 && oy != 0) a2[r] = ffma2(acc_c2(tab, pi), sum, a2[r]);
                }
            });
        }
    });
}

// ---- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (nullptr if absent).
EncodeTiledFn encode_fn();

// Tensor map over `batch` fields of two FP32 planes [2*batch][ny][nx] with the
// halo box of horizon M; false if the driver rejects it.
template <int M>
inline bool make_map(CUtensorMap *map, const void *base, int nx, int ny, int64_t batch, int box_h = box_y<M>())
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)(2 * batch)};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x<M>(), (cuuint32_t)box_h, 2};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Pair coefficients in the order tile_pairs reads them, then the interior Kd.
template <int M>
PackTab<M> make_pack(const pd_grid *g)
{
    PackTab<M> t{};
    double c[6], tot[3] = {0, 0, 0};
    auto put = [&](int ox, int oy) {
        const int pi = pair_index2(M, ox, oy);
        coef_of(g, ox, oy, 0, false, c);
        t.v[4 * pi + 0] = (float)c[0];
        t.v[4 * pi + 1] = (float)c[2];
        t.v[4 * pi + 2] = (float)c[1];
        t.v[4 * pi + 3] = (float)c[1];
        for (int i = 0; i < 3; ++i) tot[i] += 2 * c[i];
    };
    for (int ox = 1; ox <= M; ++ox) {
        const int My = isqrt_c(M * M - ox * ox);
        for (int oy = -My; oy <= My; ++oy) put(ox, oy);
    }
    for (int oy = 1; oy <= M; ++oy) put(0, oy);
    constexpr int NP = PackTab<M>::kPairs;
    for (int i = 0; i < 3; ++i) t.v[4 * NP + i] = (float)tot[i];
    return t;
}

// Coefficients of the accurate form, premultiplied by -scale (see AccTab).
template <int M>
AccTab<M> make_acc(const pd_grid *g, double scale)
{
    AccTab<M> t{};
    constexpr int NP = AccTab<M>::kPairs;
    double c[6], wb[M + 1][2] = {};
    auto put = [&](int ox, int oy) {
        const int pi = pair_index2(M, ox, oy);
        coef_of(g, ox, oy, 0, false, c);   // xx, xy, yy
        t.v[4 * pi + 0] = (float)(-scale * c[0]);
        t.v[4 * pi + 1] = (float)(-scale * c[2]);
        t.v[4 * pi + 2] = (float)(-scale * c[1]);
        t.v[4 * pi + 3] = (float)(-scale * c[1]);
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
        t.v[4 * NP + 2 * (k - 1)] = (float)(-scale * wb[k][0]);
        t.v[4 * NP + 2 * (k - 1) + 1] = (float)(-scale * wb[k][1]);
    }
    return t;
}

}  // namespace tma2d
}  // namespace pd

// pd_stencil.cuh -- pieces shared by the stencil translation units.
//
// The offset loops of the stencil kernels are unrolled at compile time with
// static_for, so every window index and every coefficient index is a constant
// expression: windows live in registers and coefficients are read from the
// kernel-parameter bank.  The host packs the coefficient tables in exactly the
// order the kernels walk them; the order functions below are used by both.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "pd_internal.cuh"
#include "pd_reduce.cuh"

namespace pd {

template <int B, int E, typename F>
__host__ __device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

__device__ __forceinline__ float dfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }

constexpr int kThreads = 256;
constexpr int kTX2 = 64, kGY2 = kThreads / kTX2;   // 2D: 64 columns x 4 row groups
constexpr int kTX3 = 32, kTY3 = kThreads / kTX3;   // 3D: 32 x 8 columns

template <typename T, int M>
__host__ __device__ constexpr int rows2d() { return sizeof(T) == 4 ? 8 : (M <= 4 ? 4 : 2); }
template <typename T, int M>
__host__ __device__ constexpr int rows2d_direct() { return sizeof(T) == 4 ? 4 : 2; }
// z-rows per thread of the 3D stencil: 8 for the FP32 pair form, 4 otherwise (the
// difference form keeps the own column and the H windows in registers)
template <typename T, int M, bool DIFF = false>
__host__ __device__ constexpr int rows3d() { return (sizeof(T) == 4 && !DIFF) ? 8 : 4; }

// ------------------------------------------------------------------ kernel walk orders
// 2D TBT pairs: ox = 1..M (oy = -My..My), then ox = 0 (oy = 1..M).
__host__ __device__ constexpr int pair_index2(int M, int ox, int oy)
{
    int k = 0;
    for (int x = 1; x <= M; ++x) {
        const int My = isqrt_c(M * M - x * x);
        for (int y = -My; y <= My; ++y) {
            if (x == ox && y == oy) return k;
            ++k;
        }
    }
    for (int y = 1; y <= M; ++y) {
        if (ox == 0 && y == oy) return k;
        ++k;
    }
    return -1;
}

// 3D TBT pairs: oy = M..0 descending, ox = -Mx..Mx (for oy = 0 only ox > 0), oz = -Mz..Mz;
// then the centre column (0, 0, oz), oz = 1..M.
__host__ __device__ constexpr int pair_index3(int M, int ox, int oy, int oz)
{
    int k = 0;
    for (int y = M; y >= 0; --y) {
        const int Mx = isqrt_c(M * M - y * y);
        for (int x = -Mx; x <= Mx; ++x) {
            if (y == 0 && x <= 0) continue;
            const int Mz = isqrt_c(M * M - x * x - y * y);
            for (int z = -Mz; z <= Mz; ++z) {
                if (x == ox && y == oy && z == oz) return k;
                ++k;
            }
        }
    }
    for (int z = 1; z <= M; ++z) {
        if (ox == 0 && oy == 0 && z == oz) return k;
        ++k;
    }
    return -1;
}

// Canonical bond index (lexicographic (oz, oy, ox)) of an offset: its bit in the mask.
__host__ __device__ constexpr int canon_index(int dim, int M, int ox, int oy, int oz)
{
    int k = 0;
    for (int z = (dim == 3 ? -M : 0); z <= (dim == 3 ? M : 0); ++z)
        for (int y = -M; y <= M; ++y)
            for (int x = -M; x <= M; ++x) {
                const int d2 = x * x + y * y + z * z;
                if (d2 == 0 || d2 > M * M) continue;
                if (x == ox && y == oy && z == oz) return k;
                ++k;
            }
    return -1;
}

// ------------------------------------------------------------------ tables passed by value
template <typename T, int DIM, int M>
struct PairTab {
    static constexpr int kPairs = count_offsets(DIM, M) / 2;
    T v[(kPairs + 1) * ncoef(DIM)];   // pairs in kernel order, then the interior Kd (sum of all c)
};

template <typename T, int M>
struct CanonTab2 {
    static constexpr int kN = count_offsets(2, M);
    T v[kN * 3];   // canonical order
};

// ------------------------------------------------------------------ fused dot epilogue
template <typename V>   // float or double: the per-warp part of the sum runs in V
__device__ __forceinline__ void finish_block_dot(V v, double *dot_partial, double *dot_out,
                                                 unsigned int *retire, int nblk, int bid, int64_t b)
{
    __shared__ double red[kThreads / 32];
    double s = block_sum(v, red);
    grid_finish(s, nblk, bid, dot_partial + b * nblk, dot_out + b, retire + b, red);
}

template <typename K>
inline void allow_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Coefficient block of offset o at the grid's modulus (unit modulus when unit = true).
void coef_of(const pd_grid *g, int ox, int oy, int oz, bool unit, double *c);

// Family runners (one translation unit each).
int run_tbt2d(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s);
int run_direct2d(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s);
int run_tbt3d(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s);

}  // namespace pd

// pd_probe.cu -- measured arithmetic peak of this GPU for the roofline of the
// ALU-bound kernels (the FP64 products and the large-horizon FP32 stencils):
// a kernel of independent fused multiply-add chains, timed with CUDA events.
#include <cuda_runtime.h>

#include "pd_internal.cuh"

namespace pd {
namespace {

constexpr int kChains = 16;    // independent chains per thread (covers the FMA latency)
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chains(T *sink, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;   // never true for the inputs used; keeps the chains live
}

template <typename T>
int probe(double *flops, cudaStream_t s)
{
    int dev = 0, sms = 0;
    PD_CUDA(cudaGetDevice(&dev));
    PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int occ = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_chains<T>, kProbeThreads, 0));
    const int blocks = sms * (occ > 0 ? occ : 1);
    T *sink = nullptr;
    cudaEvent_t e0, e1;
    PD_CUDA(cudaEventCreate(&e0));
    PD_CUDA(cudaEventCreate(&e1));
    // a = 1 - 2^-20, b = 2^-30: the chains stay finite and never reach the sink's value
    const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1073741824.0);
    int iters = 256;
    float ms = 0.f;
    for (int rep = 0; rep < 8; ++rep) {   // grow the run until it lasts 20 ms
        k_fma_chains<T><<<blocks, kProbeThreads, 0, s>>>(sink, iters, a, b);
        PD_CUDA(cudaEventRecord(e0, s));
        k_fma_chains<T><<<blocks, kProbeThreads, 0, s>>>(sink, iters, a, b);
        PD_CUDA(cudaEventRecord(e1, s));
        PD_CUDA(cudaEventSynchronize(e1));
        PD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms >= 20.f) break;
        iters *= (ms > 0.5f) ? (int)(20.f / ms) + 1 : 8;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fma_ops = (double)blocks * kProbeThreads * kChains * iters;
    *flops = 2.0 * fma_ops / (ms * 1e-3);
    return PD_OK;
}

}  // namespace
}  // namespace pd

extern "C" int pd_probe_fma_rate(uint32_t flags, double *flops, void *stream)
{
    using namespace pd;
    if (!flops) return fail(PD_ERR_INVALID, "flops is NULL");
    const bool f32 = flags & PD_F32, f64 = flags & PD_F64;
    if (f32 == f64) return fail(PD_ERR_INVALID, "exactly one of PD_F32 / PD_F64 must be set");
    return f64 ? probe<double>(flops, (cudaStream_t)stream) : probe<float>(flops, (cudaStream_t)stream);
}

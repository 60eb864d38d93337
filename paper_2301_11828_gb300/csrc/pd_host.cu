// pd_host.cu -- K u for fields held in host memory, with the copies overlapped.
//
// The batch is cut into chunks of a few fields.  Chunk k is copied host ->
// device on one stream, multiplied on a second, and copied device -> host on a
// third; two staging buffers per direction let chunk k + 1 upload and chunk
// k - 1 download while chunk k is multiplied.  The two copy directions run on
// separate copy engines, so the transfer time approaches the larger of the two
// instead of their sum.  One cudaMemcpyAsync per chunk and direction.
#include <cuda_runtime.h>

#include <algorithm>

#include "pd_internal.cuh"

namespace pd {

namespace {

struct HostPipe {
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};   // upload, product, download
    cudaEvent_t start = nullptr, end = nullptr;
    cudaEvent_t in_ready[2] = {nullptr, nullptr};       // chunk uploaded into slot
    cudaEvent_t in_free[2] = {nullptr, nullptr};        // product has read the slot
    cudaEvent_t out_ready[2] = {nullptr, nullptr};      // product written into slot
    cudaEvent_t out_free[2] = {nullptr, nullptr};       // slot downloaded
    void *buf = nullptr;                                // [2] in, [2] out
    size_t slot_bytes = 0;
};

int ensure_pipe(pd_grid *g, size_t slot_bytes, HostPipe *&p)
{
    p = (HostPipe *)g->hostpipe;
    if (!p) {
        p = new HostPipe();
        g->hostpipe = p;
        for (auto &s : p->st) PD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        PD_CUDA(cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming));
        PD_CUDA(cudaEventCreateWithFlags(&p->end, cudaEventDisableTiming));
        for (int i = 0; i < 2; ++i) {
            PD_CUDA(cudaEventCreateWithFlags(&p->in_ready[i], cudaEventDisableTiming));
            PD_CUDA(cudaEventCreateWithFlags(&p->in_free[i], cudaEventDisableTiming));
            PD_CUDA(cudaEventCreateWithFlags(&p->out_ready[i], cudaEventDisableTiming));
            PD_CUDA(cudaEventCreateWithFlags(&p->out_free[i], cudaEventDisableTiming));
        }
    }
    if (p->slot_bytes >= slot_bytes) return PD_OK;
    if (p->buf) {
        PD_CUDA(cudaDeviceSynchronize());   // an earlier call may still use the old buffers
        cudaFree(p->buf);
    }
    p->buf = nullptr;
    p->slot_bytes = 0;
    if (cudaMalloc(&p->buf, 4 * slot_bytes) != cudaSuccess) return fail(PD_ERR_OOM, "host-pipeline staging");
    p->slot_bytes = slot_bytes;
    return PD_OK;
}

}  // namespace

void hostpipe_release(pd_grid *g)
{
    HostPipe *p = (HostPipe *)g->hostpipe;
    if (!p) return;
    for (auto &s : p->st)
        if (s) cudaStreamDestroy(s);
    cudaEvent_t evs[] = {p->start, p->end, p->in_ready[0], p->in_ready[1], p->in_free[0], p->in_free[1],
                         p->out_ready[0], p->out_ready[1], p->out_free[0], p->out_free[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (p->buf) cudaFree(p->buf);
    delete p;
    g->hostpipe = nullptr;
}

}  // namespace pd

using namespace pd;

extern "C" int pd_matvec_batch_host(pd_grid *g, int64_t batch, const void *u_host, void *out_host, uint32_t flags,
                                    void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (batch < 1) return fail(PD_ERR_INVALID, "batch must be >= 1");
    if (!u_host || !out_host) return fail(PD_ERR_INVALID, "u_host and out_host must be host pointers");
    const bool f32 = flags & PD_F32, f64 = flags & PD_F64;
    if (f32 == f64) return fail(PD_ERR_INVALID, "exactly one of PD_F32 / PD_F64 must be set");
    cudaSetDevice(g->device);
    const size_t field = (size_t)g->dim * (size_t)g->N * (f64 ? sizeof(double) : sizeof(float));
    // chunks of about 32 MB, at least four when the batch allows
    int64_t per = std::max<int64_t>(1, (int64_t)((32u << 20) / std::max<size_t>(field, 1)));
    per = std::min<int64_t>(per, std::max<int64_t>(1, (batch + 3) / 4));
    per = std::min<int64_t>(per, batch);
    HostPipe *p = nullptr;
    int rc = ensure_pipe(g, field * (size_t)per, p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char *const in[2] = {(char *)p->buf, (char *)p->buf + p->slot_bytes};
    char *const outb[2] = {(char *)p->buf + 2 * p->slot_bytes, (char *)p->buf + 3 * p->slot_bytes};
    const char *uh = (const char *)u_host;
    char *oh = (char *)out_host;
    // start after the caller's earlier work on `stream`
    PD_CUDA(cudaEventRecord(p->start, s));
    for (auto &st : p->st) PD_CUDA(cudaStreamWaitEvent(st, p->start, 0));
    int64_t k = 0;
    for (int64_t f0 = 0; f0 < batch; f0 += per, ++k) {
        const int64_t nf = std::min<int64_t>(per, batch - f0);
        const size_t bytes = field * (size_t)nf;
        const int slot = (int)(k & 1);
        // upload into the slot once the product of chunk k - 2 has read it (for the
        // first two chunks: once the previous call's last product that used the slot
        // has; an event never recorded completes at once)
        PD_CUDA(cudaStreamWaitEvent(p->st[0], p->in_free[slot], 0));
        PD_CUDA(cudaMemcpyAsync(in[slot], uh + field * (size_t)f0, bytes, cudaMemcpyHostToDevice, p->st[0]));
        PD_CUDA(cudaEventRecord(p->in_ready[slot], p->st[0]));
        // product once uploaded, into an output slot whose download (chunk k - 2) is done
        PD_CUDA(cudaStreamWaitEvent(p->st[1], p->in_ready[slot], 0));
        PD_CUDA(cudaStreamWaitEvent(p->st[1], p->out_free[slot], 0));
        rc = matvec(g, nf, in[slot], outb[slot], flags, p->st[1]);
        if (rc) {   // keep the caller's stream ordered after the copies already queued
            for (auto &st : p->st) {
                cudaEventRecord(p->end, st);
                cudaStreamWaitEvent(s, p->end, 0);
            }
            return rc;
        }
        PD_CUDA(cudaEventRecord(p->in_free[slot], p->st[1]));
        PD_CUDA(cudaEventRecord(p->out_ready[slot], p->st[1]));
        // download once computed
        PD_CUDA(cudaStreamWaitEvent(p->st[2], p->out_ready[slot], 0));
        PD_CUDA(cudaMemcpyAsync(oh + field * (size_t)f0, outb[slot], bytes, cudaMemcpyDeviceToHost, p->st[2]));
        PD_CUDA(cudaEventRecord(p->out_free[slot], p->st[2]));
    }
    // the caller's later work on `stream` starts after the last download
    PD_CUDA(cudaEventRecord(p->end, p->st[2]));
    PD_CUDA(cudaStreamWaitEvent(s, p->end, 0));
    return PD_OK;
}

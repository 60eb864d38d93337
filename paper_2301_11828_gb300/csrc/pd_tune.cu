// pd_tune.cu -- the autotuner: measured choice of the product's method (direct
// stencil or FFT tiles) and of the FP32 2D stencil's tile height, per grid and
// precision, with a JSON cache keyed by (dim, extents, delta/h, precision,
// device) so that a process that meets the same grid again skips the timing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <string>

#include "pd_internal.cuh"

namespace pd {
bool tma_stencil_eligible(const pd_grid *g, const MatvecArgs &a, bool f64);

namespace {

struct Choice {
    int method = 0;        // PD_METHOD_STENCIL or PD_METHOD_FFT
    int tile_rows = 32;    // FP32 2D stencil layout: tile height 64, 32 or 16, 0 for the column walk
    double ms = 0.0;       // time per field of the chosen candidate
};

std::string key_of(const pd_grid *g, int prec)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    std::ostringstream k;
    k.precision(17);
    k << "dim=" << g->dim << " n=" << g->n[0] << "x" << g->n[1] << "x" << g->n[2] << " m=" << g->m
      << (prec ? " f64" : " f32") << (g->has_E ? " field" : "") << " device=" << prop.name << " sms="
      << prop.multiProcessorCount;
    return k.str();
}

// The cache file: one JSON object of entries
//   "<key>": {"method": "stencil"|"fft", "tile_rows": 64|32|16|0, "ms_per_field": t} (0: the column walk)
std::map<std::string, Choice> read_cache(const char *path)
{
    std::map<std::string, Choice> out;
    std::ifstream f(path);
    if (!f) return out;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string t = ss.str();
    size_t p = t.find('{');
    while (p != std::string::npos) {
        const size_t k0 = t.find('"', p + 1);
        if (k0 == std::string::npos) break;
        const size_t k1 = t.find('"', k0 + 1);
        const size_t o0 = t.find('{', k1), o1 = t.find('}', o0);
        if (k1 == std::string::npos || o0 == std::string::npos || o1 == std::string::npos) break;
        const std::string key = t.substr(k0 + 1, k1 - k0 - 1), obj = t.substr(o0, o1 - o0);
        Choice c;
        c.method = obj.find("\"fft\"") != std::string::npos ? PD_METHOD_FFT : PD_METHOD_STENCIL;
        const size_t tr = obj.find("\"tile_rows\"");
        if (tr != std::string::npos) c.tile_rows = std::atoi(obj.c_str() + obj.find(':', tr) + 1);
        const size_t ms = obj.find("\"ms_per_field\"");
        if (ms != std::string::npos) c.ms = std::atof(obj.c_str() + obj.find(':', ms) + 1);
        if (c.tile_rows != 64 && c.tile_rows != 16 && c.tile_rows != 0) c.tile_rows = 32;
        out[key] = c;
        p = o1;
    }
    return out;
}

bool write_cache(const char *path, const std::map<std::string, Choice> &m)
{
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return false;
        f << "{\n";
        size_t i = 0;
        for (const auto &kv : m) {
            char buf[64];
            std::snprintf(buf, sizeof(buf), "%.6g", kv.second.ms);
            f << "  \"" << kv.first << "\": {\"method\": \"" << (kv.second.method == PD_METHOD_FFT ? "fft" : "stencil")
              << "\", \"tile_rows\": " << kv.second.tile_rows << ", \"ms_per_field\": " << buf << "}"
              << (++i < m.size() ? ",\n" : "\n");
        }
        f << "}\n";
        if (!f) return false;
    }
    return std::rename(tmp.c_str(), path) == 0;
}

void apply(pd_grid *g, int prec, const Choice &c)
{
    g->auto_choice[prec] = c.method == PD_METHOD_FFT ? 2 : 1;
    if (prec == 0) g->stencil_tile_rows = c.tile_rows;
    ++g->op_stamp;
}

}  // namespace
}  // namespace pd

using namespace pd;

// Candidates per precision: the stencil (FP32 2D grids that take the TMA-fed
// kernel at M <= 4: tiles of 64 x 64 (M <= 3), 64 x 32 and 64 x 16 outputs and
// the column walk where it applies) and, without a modulus field, the FFT tiles
// (in FP32 chosen only from M = 5; see below).  Three warm-up products each,
// then five rounds of ten products per candidate in turn, each candidate
// keeping its fastest round (a clock ramp or a neighbour's burst does not
// decide).
extern "C" int pd_autotune(pd_grid *g, uint32_t flags, double *times_ms, void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    int dev = -1;
    PD_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(PD_ERR_STATE, "current CUDA device differs from the grid's device");
    if (!(flags & (PD_F32 | PD_F64))) return fail(PD_ERR_INVALID, "flags must name PD_F32 and/or PD_F64");
    cudaStream_t s = (cudaStream_t)stream;
    if (times_ms)
        for (int i = 0; i < 4; ++i) times_ms[i] = 0.0;
    const size_t bytes = sizeof(double) * (size_t)g->dim * g->N;
    if (!g->tune_ws) {   // two vectors, kept by the grid
        if (cudaMalloc(&g->tune_ws, 2 * bytes) != cudaSuccess) {
            g->tune_ws = nullptr;
            return fail(PD_ERR_OOM, "autotune scratch");
        }
        PD_CUDA(cudaMemsetAsync(g->tune_ws, 0, 2 * bytes, s));
    }
    void *u = g->tune_ws, *o = (char *)g->tune_ws + bytes;
    cudaEvent_t e0, e1;
    PD_CUDA(cudaEventCreate(&e0));
    PD_CUDA(cudaEventCreate(&e1));
    const bool fft_ok = !g->has_E;
    int rc = PD_OK;
    for (int prec = 0; prec < 2 && rc == PD_OK; ++prec) {
        const uint32_t dt = prec ? PD_F64 : PD_F32;
        if (!(flags & dt)) continue;
        // the layout before this precision's pass (the FP64 pass keeps the FP32 choice)
        const int saved_rows = g->stencil_tile_rows;
        struct Cand {
            uint32_t method;
            int rows;
            float best;
        };
        Cand cand[5];
        int nc = 0;
        cand[nc++] = {PD_METHOD_STENCIL, 32, 1e30f};
        MatvecArgs probe{};
        probe.u = u;
        if (prec == 0 && g->dim == 2 && g->M <= 4 && tma_stencil_eligible(g, probe, false)) {
            if (g->M <= 3) cand[nc++] = {PD_METHOD_STENCIL, 64, 1e30f};
            cand[nc++] = {PD_METHOD_STENCIL, 16, 1e30f};
            if (walk_stencil_eligible(g, probe)) cand[nc++] = {PD_METHOD_STENCIL, 0, 1e30f};   // column walk
        }
        if (fft_ok) cand[nc++] = {PD_METHOD_FFT, 32, 1e30f};
        for (int c = 0; c < nc && rc == PD_OK; ++c) {
            g->stencil_tile_rows = cand[c].rows;
            for (int w = 0; w < 3 && rc == PD_OK; ++w) rc = matvec(g, 1, u, o, dt | cand[c].method | PD_IGNORE_BROKEN, s);
        }
        for (int trial = 0; trial < 5 && rc == PD_OK; ++trial)
            for (int c = 0; c < nc && rc == PD_OK; ++c) {
                g->stencil_tile_rows = cand[c].rows;
                const uint32_t fl = dt | cand[c].method | PD_IGNORE_BROKEN;
                const int reps = 10;
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && rc == PD_OK; ++r) rc = matvec(g, 1, u, o, fl, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                cand[c].best = std::fmin(cand[c].best, ms / reps);
            }
        g->stencil_tile_rows = saved_rows;
        if (rc) break;
        // In FP32 the FFT tiles round relative to |u - L| |K| (L the tile's plane), not to
        // |K u|; |K| falls like 1/M^2 at a fixed modulus, so on smooth fields their error
        // is within the FP32 tolerance with a margin only from M = 5 (at M = 3 it reaches
        // the tolerance): below that they are measured but never chosen in FP32 (the
        // stencils sum differences).  PD_METHOD_FFT still selects them explicitly.
        int best = 0, best_st = 0;
        for (int c = 1; c < nc; ++c) {
            const bool eligible = !(prec == 0 && cand[c].method == PD_METHOD_FFT && g->M < 5);
            if (eligible && cand[c].best < cand[best].best) best = c;
            if (cand[c].method == PD_METHOD_STENCIL && cand[c].best < cand[best_st].best) best_st = c;
        }
        Choice ch;
        ch.method = (int)cand[best].method;
        ch.tile_rows = cand[best_st].rows;   // the stencil keeps its faster tile when the FFT wins
        ch.ms = cand[best].best;
        apply(g, prec, ch);
        if (times_ms) {
            times_ms[2 * prec] = cand[best_st].best;
            if (fft_ok) times_ms[2 * prec + 1] = cand[nc - 1].best;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

extern "C" int pd_autotune_cached(pd_grid *g, uint32_t flags, const char *cache_path, int *from_cache,
                                  double *times_ms, void *stream)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!cache_path) return fail(PD_ERR_INVALID, "cache_path is NULL");
    if (!(flags & (PD_F32 | PD_F64))) return fail(PD_ERR_INVALID, "flags must name PD_F32 and/or PD_F64");
    if (times_ms)
        for (int i = 0; i < 4; ++i) times_ms[i] = 0.0;
    std::map<std::string, Choice> cache = read_cache(cache_path);
    bool hit = true;
    for (int prec = 0; prec < 2; ++prec)
        if ((flags & (prec ? PD_F64 : PD_F32)) && !cache.count(key_of(g, prec))) hit = false;
    if (from_cache) *from_cache = hit ? 1 : 0;
    if (hit) {
        for (int prec = 0; prec < 2; ++prec)
            if (flags & (prec ? PD_F64 : PD_F32)) {
                const Choice &c = cache[key_of(g, prec)];
                apply(g, prec, c);
                if (times_ms) times_ms[2 * prec + (c.method == PD_METHOD_FFT ? 1 : 0)] = c.ms;
            }
        return PD_OK;
    }
    double t[4];
    int rc = pd_autotune(g, flags, t, stream);
    if (rc) return rc;
    if (times_ms)
        for (int i = 0; i < 4; ++i) times_ms[i] = t[i];
    for (int prec = 0; prec < 2; ++prec)
        if (flags & (prec ? PD_F64 : PD_F32)) {
            Choice c;
            c.method = g->auto_choice[prec] == 2 ? PD_METHOD_FFT : PD_METHOD_STENCIL;
            c.tile_rows = g->stencil_tile_rows;
            c.ms = c.method == PD_METHOD_FFT ? t[2 * prec + 1] : t[2 * prec];
            cache[key_of(g, prec)] = c;
        }
    if (!write_cache(cache_path, cache)) return fail(PD_ERR_INVALID, std::string("cannot write ") + cache_path);
    return PD_OK;
}

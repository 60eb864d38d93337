// pd_api.cu -- grid lifecycle, operator tables and the C entry points of libpd.
//
// Tables built here (once per grid, FP64 on the host, then copied):
//   - the neighbour offsets o with |o|^2 <= M^2 (Eq. band), canonical order;
//   - the unit-modulus bond blocks c1(o) = alpha1 lambda(o) h^(d-1) o o^T / |o|^3
//     (Eqs. ker:e1, frb:e1 in 2D, thm:e2 in 3D; lambda of Eq. fac:e1);
//   - the diagonal-block table Kd(class) = sum over in-grid offsets of c(o), i.e.
//     the full-horizon sum minus the edge term D^e of Eq. mat:se, for every class
//     of clipped distances to the faces.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pd_internal.cuh"

namespace pd {

static thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }

int fail(int code, const std::string &msg)
{
    t_err = msg;
    return code;
}

// lambda of Eq. fac:e1 for an offset with |o|^2 = d2, in grid units with
// m = delta / h: 1 when |o| <= m - 1/2, m + 1/2 - |o| on the shell
// m - 1/2 < |o| <= m, and 0 beyond m (an offset of the radius-ceil(m) disk that
// is no bond).  bond_of decides |o| <= m on the integer d2 (a tie counts).
bool bond_of(int d2, double m) { return (double)d2 <= m * m + 1e-9; }
double lambda_of(int d2, double m)
{
    if (!bond_of(d2, m)) return 0.0;
    return std::min(1.0, m + 0.5 - std::sqrt((double)d2));
}

static double alpha_of(int dim, double E, double delta, double thickness)
{
    const double pi = 3.14159265358979323846;
    if (dim == 2) return 9.0 * E / (pi * delta * delta * delta * thickness);
    return 12.0 * E / (pi * delta * delta * delta * delta);
}

// The bond blocks lambda V_q C(xi) of Eq. mat:f1 with V_q the volume of a node:
// h^3 in 3D and h^2 t for the 2D plate of thickness t, whose 1/t in alpha it
// cancels (the force density does not depend on the thickness).
static void build_coefs(pd_grid *g)
{
    const int nc = ncoef(g->dim);
    g->alpha1 = alpha_of(g->dim, 1.0, g->delta, g->thickness);
    g->alpha = g->alpha1 * g->E;
    g->coef1.assign((size_t)g->nnb * nc, 0.0);
    // V_q / h^d times the h^(d-1) of xi_a xi_b / |xi|^3 = h^2 o_a o_b / (h^3 |o|^3)
    const double hp = (g->dim == 2) ? g->h * g->thickness : g->h * g->h;
    for (int k = 0; k < g->nnb; ++k) {
        const int32_t *o = &g->off[3 * k];
        const int d2 = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
        const double r = std::sqrt((double)d2);
        const double w = g->alpha1 * lambda_of(d2, g->m) * hp / (r * r * r);
        double *c = &g->coef1[(size_t)nc * k];
        if (g->dim == 2) {
            c[0] = w * o[0] * o[0];
            c[1] = w * o[0] * o[1];
            c[2] = w * o[1] * o[1];
        } else {
            c[0] = w * o[0] * o[0];
            c[1] = w * o[0] * o[1];
            c[2] = w * o[0] * o[2];
            c[3] = w * o[1] * o[1];
            c[4] = w * o[1] * o[2];
            c[5] = w * o[2] * o[2];
        }
    }
}

// Kd tables at the current modulus: entry index (a0, a1, b0, b1[, c0, c1]) with
// each value the clipped distance (0..M) to the low / high face along x, y[, z].
static int build_kd(pd_grid *g)
{
    const int M = g->M, B = M + 1, nc = ncoef(g->dim);
    int64_t entries = 1;
    for (int i = 0; i < 2 * g->dim; ++i) entries *= B;
    std::vector<double> kd((size_t)entries * nc, 0.0);
    for (int64_t e = 0; e < entries; ++e) {
        int d[6] = {0, 0, 0, 0, 0, 0};
        int64_t t = e;
        for (int i = 2 * g->dim - 1; i >= 0; --i) {
            d[i] = (int)(t % B);
            t /= B;
        }
        for (int k = 0; k < g->nnb; ++k) {
            const int32_t *o = &g->off[3 * k];
            bool in = (-o[0] <= d[0]) && (o[0] <= d[1]) && (-o[1] <= d[2]) && (o[1] <= d[3]);
            if (g->dim == 3) in = in && (-o[2] <= d[4]) && (o[2] <= d[5]);
            if (!in) continue;
            for (int c = 0; c < nc; ++c) kd[(size_t)e * nc + c] += g->coef1[(size_t)k * nc + c] * g->E;
        }
    }
    if (g->dim == 2) {
        // first moments per edge class: T^x_ab = sum over in-grid offsets of c_ab(o) o_x, T^y_ab
        // alike with o_y (layout Tx_xx, Tx_xy, Tx_yy, Ty_xx, Ty_xy, Ty_yy): K of a plane at an edge
        // node (the FFT tiles and the FP64 stencil subtract a plane per tile)
        std::vector<double> kt((size_t)entries * 6, 0.0);
        for (int64_t e = 0; e < entries; ++e) {
            const int d0 = (int)(e / (B * B * B)), d1 = (int)((e / (B * B)) % B), d2 = (int)((e / B) % B),
                      d3 = (int)(e % B);
            for (int k = 0; k < g->nnb; ++k) {
                const int ox = g->off[3 * k], oy = g->off[3 * k + 1];
                if (!(-ox <= d0 && ox <= d1 && -oy <= d2 && oy <= d3)) continue;
                for (int c = 0; c < 3; ++c) {
                    kt[(size_t)6 * e + c] += g->coef1[3 * k + c] * g->E * ox;
                    kt[(size_t)6 * e + 3 + c] += g->coef1[3 * k + c] * g->E * oy;
                }
            }
        }
        std::vector<float> kt32(kt.begin(), kt.end());
        if (!g->d_kt64) {
            PD_CUDA(cudaMalloc(&g->d_kt64, kt.size() * sizeof(double)));
            PD_CUDA(cudaMalloc(&g->d_kt32, kt.size() * sizeof(float)));
        }
        PD_CUDA(cudaMemcpy(g->d_kt64, kt.data(), kt.size() * sizeof(double), cudaMemcpyHostToDevice));
        PD_CUDA(cudaMemcpy(g->d_kt32, kt32.data(), kt32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    std::vector<float> kd32(kd.begin(), kd.end());
    if (!g->d_kd64) {
        PD_CUDA(cudaMalloc(&g->d_kd64, kd.size() * sizeof(double)));
        PD_CUDA(cudaMalloc(&g->d_kd32, kd.size() * sizeof(float)));
    }
    PD_CUDA(cudaMemcpy(g->d_kd64, kd.data(), kd.size() * sizeof(double), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(g->d_kd32, kd32.data(), kd32.size() * sizeof(float), cudaMemcpyHostToDevice));
    g->kd_entries = entries;
    return PD_OK;
}

static void free_grid(pd_grid *g)
{
    if (!g) return;
    cudaFree(g->d_cons);
    cudaFree(g->d_E);
    cudaFree(g->d_mask);
    cudaFree(g->d_brlist);
    cudaFree(g->d_brflag);
    cudaFree(g->d_count);
    cudaFree(g->d_err);
    cudaFree(g->d_kd64);
    cudaFree(g->d_kd32);
    cudaFree(g->d_sym64);
    cudaFree(g->d_sym32);
    cudaFree(g->d_sym3_64);
    cudaFree(g->d_sym3_32);
    cudaFree(g->d_ctot64);
    cudaFree(g->d_ctot32);
    cudaFree(g->d_kt32);
    cudaFree(g->d_kt64);
    cudaFree(g->d_off);
    cudaFree(g->d_brk_thr);
    cudaFree(g->d_coef);
    cudaFree(g->d_coef1);
    cudaFree(g->d_nu_tab);
    cudaFree(g->d_band);
    cudaFree(g->d_tma_flags);
    cudaFree(g->ws);
    cudaFree(g->adj_ws);
    cudaFree(g->tune_ws);
    cg_release(g);
    adr_release(g);
    hostpipe_release(g);
    if (g->h_pinned) cudaFreeHost(g->h_pinned);
    delete g;
}

static int check_grid(pd_grid *g)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    int dev = -1;
    PD_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(PD_ERR_STATE, "current CUDA device differs from the grid's device");
    return PD_OK;
}

// Device copies of the offsets and of the bond blocks (current modulus and unit modulus),
// used by the sparse kernels (D^f gather, breaking, gradient).
int upload_coefs(pd_grid *g)
{
    const int nc = ncoef(g->dim);
    if (!g->d_off) {
        PD_CUDA(cudaMalloc(&g->d_off, sizeof(int32_t) * 3 * (size_t)g->nnb));
        PD_CUDA(cudaMalloc(&g->d_coef, sizeof(double) * nc * (size_t)g->nnb));
        PD_CUDA(cudaMalloc(&g->d_coef1, sizeof(double) * nc * (size_t)g->nnb));
        PD_CUDA(cudaMemcpy(g->d_off, g->off.data(), sizeof(int32_t) * 3 * (size_t)g->nnb, cudaMemcpyHostToDevice));
    }
    std::vector<double> cE(g->coef1);
    for (double &v : cE) v *= g->E;
    PD_CUDA(cudaMemcpy(g->d_coef1, g->coef1.data(), sizeof(double) * nc * (size_t)g->nnb, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(g->d_coef, cE.data(), sizeof(double) * nc * (size_t)g->nnb, cudaMemcpyHostToDevice));
    return PD_OK;
}

// ------------------------------------------------------------------ matvec front end
// out = scale * K u (K = -A) for `batch` vectors; optional fused FP64 dot
// dot_out[b] = sum_p u_p . out_p (u projected when PD_PROJECT).
int matvec(pd_grid *g, int64_t batch, const void *u, void *out, uint32_t flags, cudaStream_t s,
           double *dot_partial, double *dot_out, unsigned int *retire, double scale)
{
    const bool f32 = flags & PD_F32, f64 = flags & PD_F64;
    if (f32 == f64) return fail(PD_ERR_INVALID, "exactly one of PD_F32 / PD_F64 must be set");
    if (!u || !out) return fail(PD_ERR_INVALID, "u and out must be device pointers");
    if (u == out) return fail(PD_ERR_INVALID, "u and out must not alias");
    const uint32_t method = flags & (PD_METHOD_STENCIL | PD_METHOD_FFT);
    if (method == (PD_METHOD_STENCIL | PD_METHOD_FFT)) return fail(PD_ERR_INVALID, "two methods requested");
    const bool need_mu = !(flags & PD_IGNORE_BROKEN) && (g->broken_total > 0 || (flags & kForceMu));

    MatvecArgs a{};
    a.u = u;
    a.out = out;
    a.batch = batch;
    a.project = (flags & PD_PROJECT) && g->has_cons;
    a.input_projected = (flags & kInputProjected) != 0;
    a.no_tma = (flags & PD_NO_TMA) != 0;
    a.accurate = (flags & PD_ACCURATE) != 0;
    a.pair_form = (flags & PD_PAIR_FORM) != 0;
    a.scale = scale;

    if (dot_partial && g->sc) return fail(PD_ERR_INVALID, "internal: fused dot with the surface correction");
    if (g->has_E) {
        if (g->dim != 2) return fail(PD_ERR_INVALID, "a per-node modulus field is supported in 2D");
        if (method == PD_METHOD_FFT)
            return fail(PD_ERR_INVALID, "the FFT method needs a constant modulus (no field)");
        a.use_E = true;
        a.use_mu = need_mu;
        a.dot_partial = dot_partial;
        a.dot_out = dot_out;
        a.retire = retire;
        int rc = launch_stencil(g, f64, a, s);
        if (rc != PD_OK) return rc;
        return launch_sc_gather(g, f64, u, out, batch, a.project, need_mu, scale, s);
    }
    bool use_fft = (method == PD_METHOD_FFT);
    if (method == 0) use_fft = (g->auto_choice[f64 ? 1 : 0] == 2);
    if (dot_partial && need_mu) return fail(PD_ERR_INVALID, "internal: fused dot with broken bonds");
    a.dot_partial = dot_partial;
    a.dot_out = dot_out;
    a.retire = retire;
    int rc = use_fft ? launch_fft_tile(g, f64, a, s) : launch_stencil(g, f64, a, s);
    if (rc != PD_OK) return rc;
    if (need_mu) {
        rc = launch_df_gather(g, f64, u, out, batch, a.project, scale, s);
        if (rc != PD_OK) return rc;
    }
    return launch_sc_gather(g, f64, u, out, batch, a.project, need_mu, scale, s);
}

// Diagnostic of the bounded-wait error path: one thread polls a device flag that
// nothing sets, at most `spins` times with a short sleep between polls, and then
// records the timeout in the grid's error word, as the library's waits do.
__global__ void k_wait_unset_flag(const volatile int *flag, long long spins, int *err)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (long long i = 0; i < spins; ++i) {
        if (*flag) return;
        __nanosleep(256);
    }
    atomicExch(err, 2);
}

}  // namespace pd

using namespace pd;

// ====================================================================== C ABI
extern "C" {

const char *pd_last_error(void) { return t_err.c_str(); }

int pd_create_grid(int dim, const int64_t n[3], double h, double delta, const uint8_t *constrained,
                   pd_grid **out)
{
    if (!out) return fail(PD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(PD_ERR_INVALID, "dim must be 2 or 3");
    if (!n) return fail(PD_ERR_INVALID, "n is NULL");
    for (int i = 0; i < dim; ++i)
        if (n[i] < 1 || n[i] > (1 << 20)) return fail(PD_ERR_INVALID, "grid extents must be in [1, 2^20]");
    if (!(h > 0) || !(delta > 0) || !std::isfinite(h) || !std::isfinite(delta))
        return fail(PD_ERR_INVALID, "h and delta must be positive");
    // m = delta / h need not be an integer: the kernels work on the disk of radius
    // M = ceil(m) and the offsets beyond m carry a zero coefficient and never break
    double ratio = delta / h;
    if (!(ratio >= 1.0 - 1e-9)) return fail(PD_ERR_INVALID, "delta / h must be at least 1");
    const long near = std::lround(ratio);
    const bool integral = std::fabs(ratio - (double)near) <= 1e-9 * std::max(1.0, ratio);
    if (integral) ratio = (double)near;
    const int M = integral ? (int)near : (int)std::ceil(ratio);
    if ((dim == 2 && M > kMaxM2) || (dim == 3 && M > kMaxM3))
        return fail(PD_ERR_INVALID, "horizon radius ceil(delta/h) beyond the compiled maximum (2D 8, 3D 4)");
    const int64_t N = n[0] * n[1] * (dim == 3 ? n[2] : 1);
    if (N > ((int64_t)1 << 31) - 1) return fail(PD_ERR_INVALID, "more than 2^31 - 1 nodes");

    pd_grid *g = new (std::nothrow) pd_grid();
    if (!g) return fail(PD_ERR_OOM, "host allocation failed");
    g->dim = dim;
    g->M = M;
    g->m = ratio;
    g->h = h;
    g->delta = integral ? M * h : delta;
    g->n[0] = n[0];
    g->n[1] = n[1];
    g->n[2] = (dim == 3) ? n[2] : 1;
    g->N = N;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return fail(PD_ERR_CUDA, "no CUDA device");
    }
    for (int oz = (dim == 3 ? -M : 0); oz <= (dim == 3 ? M : 0); ++oz)
        for (int oy = -M; oy <= M; ++oy)
            for (int ox = -M; ox <= M; ++ox) {
                const int d2 = ox * ox + oy * oy + oz * oz;
                if (d2 == 0 || d2 > M * M) continue;
                g->off.push_back(ox);
                g->off.push_back(oy);
                g->off.push_back(oz);
            }
    g->nnb = (int)(g->off.size() / 3);
    g->W = (g->nnb + 31) / 32;
    build_coefs(g);

    auto bail = [&](int code, const char *msg) {
        free_grid(g);
        return fail(code, msg);
    };
    if (cudaMalloc(&g->d_mask, sizeof(uint32_t) * (size_t)g->W * N) != cudaSuccess) return bail(PD_ERR_OOM, "mask");
    if (cudaMemset(g->d_mask, 0xff, sizeof(uint32_t) * (size_t)g->W * N) != cudaSuccess)
        return bail(PD_ERR_CUDA, "mask init");
    if (cudaMalloc(&g->d_brlist, sizeof(int32_t) * (size_t)N) != cudaSuccess) return bail(PD_ERR_OOM, "list");
    if (cudaMalloc(&g->d_brflag, sizeof(uint32_t) * (size_t)N) != cudaSuccess) return bail(PD_ERR_OOM, "flags");
    if (cudaMemset(g->d_brflag, 0, sizeof(uint32_t) * (size_t)N) != cudaSuccess) return bail(PD_ERR_CUDA, "flags");
    if (cudaMalloc(&g->d_count, sizeof(unsigned long long) * 8) != cudaSuccess) return bail(PD_ERR_OOM, "counters");
    if (cudaMemset(g->d_count, 0, sizeof(unsigned long long) * 8) != cudaSuccess)
        return bail(PD_ERR_CUDA, "counters");
    if (cudaMallocHost(&g->h_pinned, 4096) != cudaSuccess) return bail(PD_ERR_OOM, "pinned mailbox");
    if (cudaMalloc(&g->d_brk_thr, sizeof(double) * 4 * (size_t)g->nnb) != cudaSuccess)
        return bail(PD_ERR_OOM, "breaking thresholds");
    if (cudaMalloc(&g->d_err, sizeof(int)) != cudaSuccess) return bail(PD_ERR_OOM, "error word");
    if (cudaMemset(g->d_err, 0, sizeof(int)) != cudaSuccess) return bail(PD_ERR_CUDA, "error word");
    if (constrained) {
        std::vector<uint8_t> bits((size_t)N, 0);
        bool any = false;
        for (int c = 0; c < dim; ++c)
            for (int64_t p = 0; p < N; ++p)
                if (constrained[(size_t)c * N + p]) {
                    bits[p] |= (uint8_t)(1u << c);
                    any = true;
                }
        g->has_cons = any;
        if (cudaMalloc(&g->d_cons, (size_t)N) != cudaSuccess) return bail(PD_ERR_OOM, "constraint mask");
        if (cudaMemcpy(g->d_cons, bits.data(), (size_t)N, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(PD_ERR_CUDA, "constraint mask copy");
    }
    int rc = build_kd(g);
    if (rc == PD_OK) rc = upload_coefs(g);
    if (rc != PD_OK) {
        std::string m = t_err;
        free_grid(g);
        return fail(rc, m);
    }
    *out = g;
    return PD_OK;
}

int pd_set_material(pd_grid *g, double E, double rho, double thickness, double s0, const double *E_field)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (!(E > 0) || !(rho > 0) || !(thickness > 0) || !std::isfinite(E) || !std::isfinite(rho) ||
        !std::isfinite(thickness) || !std::isfinite(s0))
        return fail(PD_ERR_INVALID, "E, rho and thickness must be positive and finite");
    if (E_field && g->dim != 2) return fail(PD_ERR_INVALID, "a modulus field is supported in 2D");
    g->E = E;
    g->rho = rho;
    g->thickness = thickness;
    g->s0 = s0;
    build_coefs(g);
    if (E_field) {
        if (!g->d_E) PD_CUDA(cudaMalloc(&g->d_E, sizeof(double) * (size_t)g->N));
        PD_CUDA(cudaMemcpy(g->d_E, E_field, sizeof(double) * (size_t)g->N, cudaMemcpyDeviceToDevice));
        std::vector<double> hE((size_t)g->N);
        PD_CUDA(cudaMemcpy(hE.data(), g->d_E, sizeof(double) * (size_t)g->N, cudaMemcpyDeviceToHost));
        g->E_max = 0.0;
        for (double v : hE) {
            if (!(v > 0) || !std::isfinite(v)) {
                g->has_E = false;
                return fail(PD_ERR_INVALID, "modulus field values must be positive and finite");
            }
            g->E_max = std::max(g->E_max, v);
        }
        g->has_E = true;
    } else {
        g->has_E = false;
        g->E_max = E;
    }
    rc = build_kd(g);
    if (rc) return rc;
    rc = upload_coefs(g);
    if (rc) return rc;
    g->auto_choice[0] = g->auto_choice[1] = 0;
    ++g->op_stamp;
    if (g->sc) {   // its FP32 copy of the unit-modulus blocks follows the thickness
        rc = surface_set(g, g->sc);
        if (rc) return rc;
    }
    if (g->d_sym3_32) {
        rc = fft3_prepare(g);
        if (rc) return rc;
    }
    if (g->d_sym32) return fft_prepare(g);
    return PD_OK;
}

int pd_matvec(pd_grid *g, const void *u, void *out, uint32_t flags, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    return matvec(g, 1, u, out, flags, (cudaStream_t)stream);
}

int pd_matvec_batch(pd_grid *g, int64_t batch, const void *u, void *out, uint32_t flags, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (batch < 1) return fail(PD_ERR_INVALID, "batch must be >= 1");
    return matvec(g, batch, u, out, flags, (cudaStream_t)stream);
}

int pd_matvec_rows(pd_grid *g, int64_t batch, int64_t row0, int64_t rows, const void *u_ext, int64_t ext_row0,
                   int64_t ext_rows, void *out, uint32_t flags, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (batch < 1 || batch > 65535) return fail(PD_ERR_INVALID, "batch must be in [1, 65535]");
    const int64_t ny = g->n[g->dim - 1], M = g->M;   // rows in 2D, planes in 3D
    if (rows < 1 || row0 < 0 || row0 + rows > ny) return fail(PD_ERR_INVALID, "rows outside the grid");
    if (g->dim == 2 && row0 % 32 != 0) return fail(PD_ERR_INVALID, "row0 must be a multiple of 32 (the tile height)");
    if (ext_row0 < 0 || ext_rows < 1 || ext_row0 + ext_rows > ny || ext_row0 > std::max<int64_t>(0, row0 - M) ||
        ext_row0 + ext_rows < std::min(ny, row0 + rows + M))
        return fail(PD_ERR_INVALID, "u_ext must hold the rows [row0 - M, row0 + rows + M) of the grid");
    const bool f32 = flags & PD_F32, f64 = flags & PD_F64;
    if (f32 == f64) return fail(PD_ERR_INVALID, "exactly one of PD_F32 / PD_F64 must be set");
    if (!u_ext || !out) return fail(PD_ERR_INVALID, "u_ext and out must be device pointers");
    if (flags & (PD_METHOD_FFT | PD_PAIR_FORM)) return fail(PD_ERR_INVALID, "pd_matvec_rows runs the stencil form");
    if (g->has_E || g->sc || g->broken_total > 0)
        return fail(PD_ERR_INVALID, "pd_matvec_rows: intact bonds, constant modulus, no surface correction");
    MatvecArgs a{};
    a.u = u_ext;
    a.out = out;
    a.batch = batch;
    a.project = (flags & PD_PROJECT) && g->has_cons;
    a.no_tma = (flags & PD_NO_TMA) != 0;
    a.accurate = (flags & PD_ACCURATE) != 0;
    a.scale = 1.0;
    a.in_row0 = ext_row0;
    a.in_rows = ext_rows;
    a.out_row0 = row0;
    a.out_rows = rows;
    return launch_stencil(g, f64, a, (cudaStream_t)stream);
}

int pd_set_stencil_tile_rows(pd_grid *g, int rows)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (rows != 64 && rows != 32 && rows != 16 && rows != 0)
        return fail(PD_ERR_INVALID, "tile rows must be 64, 32, 16 or 0 (column walk)");
    g->stencil_tile_rows = rows;
    ++g->op_stamp;
    return PD_OK;
}

int pd_set_method(pd_grid *g, uint32_t method)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (method == PD_METHOD_AUTO) {
        g->auto_choice[0] = g->auto_choice[1] = 0;
    } else if (method == PD_METHOD_STENCIL) {
        g->auto_choice[0] = g->auto_choice[1] = 1;
    } else if (method == PD_METHOD_FFT) {
        if (g->has_E) return fail(PD_ERR_INVALID, "the FFT method needs a grid without a modulus field");
        g->auto_choice[0] = g->auto_choice[1] = 2;
    } else {
        return fail(PD_ERR_INVALID, "method must be PD_METHOD_AUTO, PD_METHOD_STENCIL or PD_METHOD_FFT");
    }
    ++g->op_stamp;
    return PD_OK;
}

int pd_get_info(pd_grid *g, pd_grid_info *info)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (!info) return fail(PD_ERR_INVALID, "info is NULL");
    info->dim = g->dim;
    info->M = g->M;
    info->nnb = g->nnb;
    info->mask_words = g->W;
    for (int i = 0; i < 3; ++i) info->n[i] = g->n[i];
    info->N = g->N;
    info->h = g->h;
    info->delta = g->delta;
    info->alpha = g->alpha;
    unsigned long long cnt = 0;
    PD_CUDA(cudaMemcpy(&cnt, g->d_count, sizeof(cnt), cudaMemcpyDeviceToHost));
    info->n_broken_nodes = (int64_t)cnt;
    int derr = 0;
    PD_CUDA(cudaMemcpy(&derr, g->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    info->device_error = derr;
    for (int i = 0; i < 2; ++i) info->auto_method[i] = g->auto_choice[i] == 2 ? PD_METHOD_FFT : PD_METHOD_STENCIL;
    info->stencil_tile_rows = g->stencil_tile_rows;
    return PD_OK;
}

int pd_get_offsets(pd_grid *g, int32_t *off, int cap)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!off || cap < g->nnb) return fail(PD_ERR_INVALID, "offset buffer too small");
    std::memcpy(off, g->off.data(), sizeof(int32_t) * 3 * (size_t)g->nnb);
    return PD_OK;
}

int pd_get_coefficients(pd_grid *g, double *coef, int cap)
{
    if (!g) return fail(PD_ERR_INVALID, "grid is NULL");
    if (!coef || cap < g->nnb) return fail(PD_ERR_INVALID, "coefficient buffer too small");
    const int nc = ncoef(g->dim);
    for (size_t i = 0; i < (size_t)nc * g->nnb; ++i) coef[i] = g->coef1[i] * g->E;
    return PD_OK;
}

int pd_get_bond_mask(pd_grid *g, uint32_t *mask, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (!mask) return fail(PD_ERR_INVALID, "mask is NULL");
    PD_CUDA(cudaMemcpyAsync(mask, g->d_mask, sizeof(uint32_t) * (size_t)g->W * g->N, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return PD_OK;
}

int pd_set_bond_mask(pd_grid *g, const uint32_t *mask, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (!mask) return fail(PD_ERR_INVALID, "mask is NULL");
    PD_CUDA(cudaMemcpyAsync(g->d_mask, mask, sizeof(uint32_t) * (size_t)g->W * g->N, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return refresh_broken_nodes(g, (cudaStream_t)stream);
}

int pd_break_bonds(pd_grid *g, const void *u, uint32_t flags, int64_t *n_newly_broken, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    const bool f32 = flags & PD_F32, f64 = flags & PD_F64;
    if (f32 == f64) return fail(PD_ERR_INVALID, "exactly one of PD_F32 / PD_F64 must be set");
    if (!u) return fail(PD_ERR_INVALID, "u is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    PD_CUDA(cudaMemsetAsync(g->d_count + 2, 0, sizeof(unsigned long long), s));
    rc = launch_break(g, u, f64, nullptr, 0, s);
    if (rc) return rc;
    PD_CUDA(cudaMemcpyAsync(g->h_pinned, g->d_count, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    g->broken_total = (int64_t)g->h_pinned[1];
    if (g->h_pinned[2]) ++g->op_stamp;
    if (n_newly_broken) *n_newly_broken = (int64_t)g->h_pinned[2];
    return PD_OK;
}

int pd_break_segment(pd_grid *g, const int64_t seg[4], int64_t den, int64_t *n_broken, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (!seg || den < 1) return fail(PD_ERR_INVALID, "bad segment");
    const int64_t lim = (int64_t)1 << 28;
    for (int i = 0; i < 4; ++i)
        if (seg[i] < -lim || seg[i] > lim) return fail(PD_ERR_INVALID, "segment coordinates out of range");
    if (den * (2 * std::max(g->n[0], g->n[1]) + 1) > lim)
        return fail(PD_ERR_INVALID, "segment denominator too large");
    cudaStream_t s = (cudaStream_t)stream;
    PD_CUDA(cudaMemsetAsync(g->d_count + 2, 0, sizeof(unsigned long long), s));
    rc = launch_break_segment(g, seg, den, s);
    if (rc) return rc;
    PD_CUDA(cudaMemcpyAsync(g->h_pinned, g->d_count, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    g->broken_total = (int64_t)g->h_pinned[1];
    if (g->h_pinned[2]) ++g->op_stamp;
    if (n_broken) *n_broken = (int64_t)g->h_pinned[2];
    return PD_OK;
}

int pd_grad_modulus(pd_grid *g, const double *u, const double *lam, double scale, double *grad, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (!u || !lam || !grad) return fail(PD_ERR_INVALID, "NULL vector");
    return launch_grad_modulus(g, u, lam, scale, grad, (cudaStream_t)stream);
}

int pd_check_wait_timeout(pd_grid *g, int64_t spins, void *stream)
{
    int rc = check_grid(g);
    if (rc) return rc;
    if (spins < 1 || spins > ((int64_t)1 << 24)) return fail(PD_ERR_INVALID, "spins must be in [1, 2^24]");
    cudaStream_t s = (cudaStream_t)stream;
    int *flag = reinterpret_cast<int *>(g->d_count + 7);   // a counter word the library never writes
    PD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    k_wait_unset_flag<<<1, 32, 0, s>>>(flag, (long long)spins, g->d_err);
    PD_CUDA(cudaGetLastError());
    PD_CUDA(cudaStreamSynchronize(s));
    int derr = 0;
    PD_CUDA(cudaMemcpy(&derr, g->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!derr) return PD_OK;
    PD_CUDA(cudaMemset(g->d_err, 0, sizeof(int)));   // reported once; the context stays usable
    return fail(PD_ERR_TIMEOUT, "a bounded device wait gave up (diagnostic wait on a flag nothing sets)");
}

int pd_critical_stretch(double G0, double E, double delta, int mode, double *s0)
{
    if (!s0) return fail(PD_ERR_INVALID, "s0 is NULL");
    if (!(G0 > 0) || !(E > 0) || !(delta > 0) || !std::isfinite(G0) || !std::isfinite(E) || !std::isfinite(delta))
        return fail(PD_ERR_INVALID, "G0, E and delta must be positive and finite");
    const double pi = 3.14159265358979323846;
    if (mode == PD_PLANE_STRESS) *s0 = std::sqrt(4.0 * pi * G0 / (9.0 * E * delta));
    else if (mode == PD_PLANE_STRAIN) *s0 = std::sqrt(5.0 * pi * G0 / (12.0 * E * delta));
    else return fail(PD_ERR_INVALID, "mode must be PD_PLANE_STRESS or PD_PLANE_STRAIN");
    return PD_OK;
}

int pd_destroy(pd_grid *g)
{
    if (!g) return PD_OK;
    free_grid(g);
    return PD_OK;
}

}  // extern "C"

// pd_internal.cuh -- internal declarations of libpd (not part of the C ABI).
//
// Data layout in device memory (all owned by the pd_grid unless stated):
//   caller vectors  [dim][N] SoA, x fastest (node p = i + nx (j + ny k));
//   d_cons          uint8 [N], bit c set when component c is constrained (Omega_c);
//   d_mask          uint32 [W][N] bond-intact bits, W = ceil(nnb / 32), word-major so that
//                   a warp reading word w of 32 consecutive nodes is coalesced;
//   d_kd{32,64}     diagonal block table Kd = sum of c(o) over in-grid offsets, indexed by the
//                   clipped distances to the faces (the D^e table of Eq. mat:se, folded into
//                   the diagonal);
//   d_sym{32,64}    real symbol of one FFT tile (Sec. 3.2 Algorithm 3, per tile);
//   d_E             double [N] per-node modulus (optional);
//   d_brlist/flag   Omega_br: nodes holding at least one broken bond, compacted list.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pd.h"

namespace pd {

// ------------------------------------------------------------------ limits
constexpr int kMaxM2 = 8;    // largest horizon M compiled for 2D
constexpr int kMaxM3 = 4;    // largest horizon M compiled for 3D
constexpr int kFftP = 64;    // FFT tile edge (2D)

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
#define PD_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return ::pd::fail(PD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------ offsets
// Number of offsets o != 0 with |o|^2 <= M^2 (2D: oz = 0).
__host__ __device__ constexpr int count_offsets(int dim, int M)
{
    int c = 0;
    for (int oz = (dim == 3 ? -M : 0); oz <= (dim == 3 ? M : 0); ++oz)
        for (int oy = -M; oy <= M; ++oy)
            for (int ox = -M; ox <= M; ++ox) {
                int d2 = ox * ox + oy * oy + oz * oz;
                if (d2 > 0 && d2 <= M * M) ++c;
            }
    return c;
}

// Integer square root floor(sqrt(v)) for small non-negative v (compile-time friendly).
__host__ __device__ constexpr int isqrt_c(int v)
{
    int r = 0;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// Number of coefficient reals per offset: 3 in 2D (xx, xy, yy), 6 in 3D (xx, xy, xz, yy, yz, zz).
__host__ __device__ constexpr int ncoef(int dim) { return dim == 2 ? 3 : 6; }

// Coefficient table passed by value to the stencil kernels (kernel parameter space).
template <typename T, int DIM, int M>
struct CoefTab {
    static constexpr int kN = count_offsets(DIM, M);
    T v[kN * ncoef(DIM)];   // canonical offset order, ncoef(DIM) reals each
};

// ------------------------------------------------------------------ the grid
}  // namespace pd

struct pd_grid {
    int dim = 2, M = 1, nnb = 0, W = 1;
    int64_t n[3] = {1, 1, 1};
    int64_t N = 0;
    double h = 0, delta = 0;
    double m = 1;                   // delta / h (the kernels' radius M is ceil(m))
    double E = 1, rho = 1, thickness = 1, s0 = 0;
    double E_max = 1;               // largest modulus (of the field when one is set)
    double alpha = 0, alpha1 = 0;   // micromodulus at E and at E = 1
    int device = 0;
    bool has_cons = false;
    bool has_E = false;

    std::vector<int32_t> off;       // [nnb][3] canonical (oz, oy, ox) lexicographic order
    std::vector<double> coef1;      // [nnb][ncoef] bond blocks at E = 1 (alpha1 lambda h^(d-1) o_a o_b / |o|^3)

    uint8_t *d_cons = nullptr;
    double *d_E = nullptr;
    uint32_t *d_mask = nullptr;
    int32_t *d_brlist = nullptr;
    uint32_t *d_brflag = nullptr;
    int32_t *d_off = nullptr;       // [nnb][3] device copy of the offsets
    double *d_coef = nullptr;       // [nnb][ncoef] bond blocks at the current modulus
    double *d_coef1 = nullptr;      // [nnb][ncoef] bond blocks at E = 1
    unsigned long long *d_count = nullptr;   // [0] |Omega_br|, [1] broken total, [2] newly broken (scratch)
    double *d_brk_thr = nullptr;    // [nnb] threshold on |xi + eta|^2, then [nnb][3] xi = h o (upper half used)
    double brk_thr_s0 = -1.0;       // s0 the thresholds were computed for (< 0: not yet)
    int *d_err = nullptr;                     // device-side error word (bounded waits that ran out)
    double *d_kd64 = nullptr;
    float *d_kd32 = nullptr;
    double *d_sym64 = nullptr;
    float *d_sym32 = nullptr;
    double *d_sym3_64 = nullptr;    // 3D tile symbol (6 x 16^3)
    float *d_sym3_32 = nullptr;
    double *d_ctot64 = nullptr;     // interior diagonal block (3D FFT epilogue)
    float *d_ctot32 = nullptr;
    double *d_kt64 = nullptr;       // 2D: first moments sum_{in-grid o} c(o) o per edge class (6 values)
    float *d_kt32 = nullptr;        //     (K of a plane at an edge node), FP64 and FP32 copies
    int64_t kd_entries = 0;
    int64_t broken_total = 0;

    // CG / Verlet workspace, allocated on first use
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *adj_ws = nullptr;         // adjoint sweep workspace (pd_step_adjoint), grown on demand
    size_t adj_ws_bytes = 0;
    unsigned long long *h_pinned = nullptr;  // small pinned host mailbox

    // measured method choice cache: [dtype 0/1] -> 0 unknown, 1 stencil, 2 fft
    int auto_choice[2] = {0, 0};
    // FP32 2D stencil layout: 64 x 64 tiles (64, the default; used at M <= 3),
    // 64 x 32 (32; beyond M = 3 the 64 setting falls back to it), 64 x 16 (16;
    // used at M <= 4) or the column walk (0); set by the autotuner
    int stencil_tile_rows = 64;
    void *tune_ws = nullptr;         // autotuner scratch (two vectors), kept by the grid

    void *cg = nullptr;        // CG workspace and captured graphs (pd_cg.cu)
    void *adr = nullptr;       // ADR workspace and captured graph (pd_adr.cu)
    void *hostpipe = nullptr;  // streams, events and staging of pd_matvec_batch_host (pd_host.cu)
    bool no_tma = false;       // use the plain FP32 stencil instead of the TMA-fed one
    uint8_t *d_tma_flags = nullptr;   // per 64 x 32 tile: bit 0 an output is constrained, bit 1 its halo holds one
    int tma_flags_M = -1;             // horizon the flags were computed for
    // surface correction (pd_surface.cu): mode, nu per class of clipped face distances,
    // the band of nodes within 2M of a face, three words of scratch
    int sc = 0;
    double *d_nu_tab = nullptr;
    int32_t *d_band = nullptr;
    int64_t band_n = 0;
    unsigned long long *d_sc_rowmax = nullptr;
    float *d_sc_f32 = nullptr;     // FP32 nu table [sc_ncls], then unit-modulus bond blocks [nnb][ncoef]
    int sc_ncls = 0;
    int64_t op_stamp = 0;      // bumped whenever the operator changes (material, bond state)
};

namespace pd {

// ------------------------------------------------------------------ launchers (pd_stencil.cu)
struct MatvecArgs {
    const void *u;        // input  [batch][dim][N]
    void *out;            // output [batch][dim][N]
    int64_t batch;
    bool project;         // P K P
    bool use_mu;          // honour the bond mask inline (direct form)
    bool use_E;           // per-node modulus (direct form)
    bool input_projected; // the caller guarantees P u = u (skip the input projection)
    bool no_tma;          // force the plain FP32 2D stencil
    bool accurate;        // FP64 2D stencil: difference form instead of the plane-subtracted pair form
    bool pair_form;       // FP32 TMA 2D stencil: the cancelling pair form (PD_PAIR_FORM)
    double scale;         // multiplies the whole operator (1 = K u)
    // row window (2D stencils; pd_matvec_rows): the input holds grid rows
    // [in_row0, in_row0 + in_rows) and the output rows [out_row0, out_row0 + out_rows);
    // the defaults (whole grid) are set by matvec()
    int64_t in_row0 = 0, in_rows = -1, out_row0 = 0, out_rows = -1;
    // optional fused reduction: dot_out[b] = sum_p in . out (FP64), needs scratch
    double *dot_partial;  // [gridDim.x * gridDim.y] per batch
    double *dot_out;      // [batch]
    unsigned int *retire; // [batch] counters, zero on entry, reset by the last block
};
int launch_stencil(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s);
int stencil_blocks(pd_grid *g, bool f64, bool direct);   // CTAs per field (for sizing partials)
bool tma_stencil_eligible(const pd_grid *g, const MatvecArgs &a, bool f64);
int run_tbt2d_tma(pd_grid *g, const MatvecArgs &a, cudaStream_t s);
bool walk_stencil_eligible(const pd_grid *g, const MatvecArgs &a);
int run_tbt2d_walk(pd_grid *g, const MatvecArgs &a, cudaStream_t s);

// ------------------------------------------------------------------ launchers (pd_fft.cu)
int launch_fft_tile(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s);
int fft_prepare(pd_grid *g);   // builds the tile symbol tables
int fft3_prepare(pd_grid *g);  // 3D (pd_fft3d.cu)
int launch_fft3_tile(pd_grid *g, bool f64, const MatvecArgs &a, cudaStream_t s);

// ------------------------------------------------------------------ launchers (pd_crack.cu)
int launch_df_gather(pd_grid *g, bool f64, const void *u, void *out, int64_t batch, bool project,
                     double scale, cudaStream_t s);
int launch_break(pd_grid *g, const void *u, bool f64, int32_t *break_step, int32_t step_id,
                 cudaStream_t s);
int launch_break_segment(pd_grid *g, const int64_t seg[4], int64_t den, cudaStream_t s);
int refresh_broken_nodes(pd_grid *g, cudaStream_t s);
int launch_grad_modulus(pd_grid *g, const double *u, const double *lam, double scale, double *grad,
                        cudaStream_t s);

// ------------------------------------------------------------------ matvec front end (pd_api.cu)
// Internal flag: bonds may have broken on the device since the host last looked;
// always run the broken-bond correction (it reads the device-side count).
constexpr uint32_t kForceMu = 0x80000000u;
// Internal flag: the input already satisfies P u = u (the CG keeps its vectors projected).
constexpr uint32_t kInputProjected = 0x40000000u;
int upload_coefs(pd_grid *g);
double lambda_of(int d2, double m);   // Eq. fac:e1 in grid units, m = delta / h
bool bond_of(int d2, double m);        // |o| <= m for |o|^2 = d2

// ------------------------------------------------------------------ surface correction (pd_surface.cu)
// Class of a node for the surface-correction table: its distances to the low and
// high face along each axis, clipped at M (mixed radix M + 1).
__device__ __forceinline__ int nu_class(int i, int j, int k, int nx, int ny, int nz, int M, int dim)
{
    int c = min(i, M);
    c = c * (M + 1) + min(nx - 1 - i, M);
    c = c * (M + 1) + min(j, M);
    c = c * (M + 1) + min(ny - 1 - j, M);
    if (dim == 3) {
        c = c * (M + 1) + min(k, M);
        c = c * (M + 1) + min(nz - 1 - k, M);
    }
    return c;
}
int surface_set(pd_grid *g, int mode);
int launch_sc_gather(pd_grid *g, bool f64, const void *u, void *out, int64_t batch, bool project, bool use_mu,
                     double scale, cudaStream_t s);
int surface_row_abs_max(pd_grid *g, double out[3], cudaStream_t s);   // band rows only; synchronises s
void cg_release(pd_grid *g);
void adr_release(pd_grid *g);
void hostpipe_release(pd_grid *g);
int matvec(pd_grid *g, int64_t batch, const void *u, void *out, uint32_t flags, cudaStream_t s,
           double *dot_partial = nullptr, double *dot_out = nullptr, unsigned int *retire = nullptr,
           double scale = 1.0);

}  // namespace pd

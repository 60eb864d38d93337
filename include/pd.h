/*
 * pd.h -- C ABI of libpd, a GB300 (sm_103a) library for the stiffness product
 * K u of linear bond-based peridynamics on a uniform grid, and for the static
 * solve, the velocity-Verlet crack loop and the gradients built around it.
 *
 * The operator follows "A fast computational framework for the linear
 * bond-based peridynamic model" (arXiv 2301.11828):
 *   - the nodal force of Eq. mat:f1, f_p = sum_q mu_pq C(x_q - x_p)(u_q - u_p) lambda_q V_q,
 *     with the micromodulus tensor of Eq. ker:e1, the constant alpha of Sec. 2.1
 *     and the partial-volume factor of Eq. fac:e1;
 *   - written as f = A u with A = A^ + D^e + D^f (Sec. 3.2-3.5, Sec. 4): a
 *     Toeplitz-block-Toeplitz part A^ (TBTBT in 3D), the edge self-term D^e
 *     (Eq. mat:se) and the broken-bond correction D^f (Eq. df).
 * This library returns the stiffness product  K u := -A u  (symmetric positive
 * semidefinite; -A u = b is the static problem of Eq. mat:e2).
 *
 * Conventions shared by every call
 *   - Nodes sit at x = h (i + 1/2, j + 1/2[, k + 1/2]), 0-based, and are
 *     numbered p = i + n[0] (j + n[1] k) (Sec. 3 and Sec. 4 numbering).
 *   - A per-node vector is structure-of-arrays, component-major:
 *     v[c * N + p], c < dim, N = n[0] n[1] (n[2]); contiguous.
 *   - Vector arguments are DEVICE pointers owned by the caller unless the
 *     comment says host.  The library never frees caller memory.
 *   - Every call is ordered on the given CUDA stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream).  Calls that return values to the
 *     host (counts, statistics) synchronise that stream.
 *   - Every call returns a pd_status; nothing aborts.  pd_last_error() holds a
 *     message for the last failure on the calling thread.
 *   - A pd_grid may be used by one host thread / stream at a time.
 *   - The horizon delta is any real multiple m = delta / h >= 1 of the grid
 *     spacing.  The bonds of a node are the grid offsets o with |o| <= m
 *     (Eq. band; Eq. fac:e1 gives their partial-volume factor); the kernels
 *     work on the disk (ball) of integer radius M = ceil(m), where the offsets
 *     beyond m carry a zero coefficient.
 */
#ifndef PD_H
#define PD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pd_grid pd_grid;

typedef enum {
    PD_OK = 0,
    PD_ERR_INVALID = 1,        /* bad argument, shape, flag or state */
    PD_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    PD_ERR_OOM = 3,            /* device allocation failed */
    PD_ERR_NOT_CONVERGED = 4,  /* iteration cap reached; outputs hold the last iterate */
    PD_ERR_TIMEOUT = 5,        /* a bounded device-side wait ran out */
    PD_ERR_STATE = 6           /* call not valid in the grid's current state */
} pd_status;

/* ---- flags for pd_matvec / pd_matvec_batch / pd_break_bonds ---- */
#define PD_F32            0x1u   /* vectors are float  */
#define PD_F64            0x2u   /* vectors are double */
#define PD_METHOD_AUTO    0x00u  /* fastest measured method for (dim, M, dtype) */
#define PD_METHOD_STENCIL 0x10u  /* direct neighbour sum (Eq. mat:f1), shared-memory tiled */
#define PD_METHOD_FFT     0x20u  /* TBT part by FFT with the symbol product fused (Algorithms 3/4) */
#define PD_PROJECT        0x100u /* return P K P u: P zeroes the constrained components */
#define PD_IGNORE_BROKEN  0x200u /* use the intact operator A^ + D^e (skip mu / D^f) */
#define PD_NO_TMA         0x400u /* FP32 2D stencil and FFT tiles: use the plain-load kernels, not the TMA-fed ones */
#define PD_ACCURATE       0x800u /* FP64 2D stencil: the difference form (below) instead of the default
                                    pair form on u minus each tile's plane (both keep the error relative
                                    to |K u|); FP32 stencils sum differences by default (no effect) */
#define PD_PAIR_FORM      0x1000u /* stencils: the pair form Kd_p u_p - sum c(o) (u_p+o + u_p-o) on u
                                    itself instead of the default difference form (FP32, 3D) or the
                                    pair form on u minus each tile's least-squares plane, exact in FP64,
                                    plus K of the plane at the faces (FP64 2D; the difference form with
                                    a fused dot).  Less arithmetic, but its
                                    error is relative to sum |c| |u|, not to |K u|: on smooth fields,
                                    or fields with a large constant part, FP32 exceeds 1e-4 relative
                                    error (2D) and FP64 a few 1e-12 over the field (3e-10 on the
                                    interior of a field with a large gradient).  For comparison, for inner
                                    solver products whose rounding an FP64 refinement corrects, and
                                    for the FP64 CG and ADR iterations (tolerance far above it) */

/* ---- modes for pd_set_surface_correction ---- */
#define PD_SC_NONE   0    /* the paper's operator A = A^ + D^e + D^f (default) */
#define PD_SC_VOLUME 1    /* bonds scaled by v_pq = (nu_p + nu_q)/2, nu_p = V_full / V_p */

/* ---- modes for pd_critical_stretch ---- */
#define PD_PLANE_STRESS 0
#define PD_PLANE_STRAIN 1

/* ---- modes for pd_adr_solve ---- */
#define PD_ADR_F64   0x1u  /* Algorithm 1 in FP64 throughout (the paper's solver) */
#define PD_ADR_MIXED 0x2u  /* FP32 operator on the correction since an FP64 base, FP64 residual at each 10x drop */

/* ---- modes for pd_cg_solve ---- */
#define PD_CG_F64   0x1u  /* plain CG, FP64 vectors and FP64 matvec */
#define PD_CG_MIXED 0x2u  /* FP32-matvec CG, FP64 solution, FP64 residual replacement every 10x drop */
#define PD_CG_GRAPH 0x10u /* option for PD_CG_MIXED: run the FP32 inner loop as CUDA-graph-replayed
                             launches even where the persistent kernel applies */

typedef struct {
    int dim;          /* 2 or 3 */
    int M;            /* kernel radius: ceil(delta / h) (= delta / h in the paper's examples) */
    int nnb;          /* number of neighbour offsets (28 for 2D M = 3) */
    int mask_words;   /* 32-bit words per node in the bond mask */
    int64_t n[3];     /* grid extents (n[2] = 1 in 2D) */
    int64_t N;        /* number of nodes */
    double h, delta, alpha;  /* spacing, horizon, micromodulus constant at the set modulus */
    int64_t n_broken_nodes;  /* nodes with at least one broken bond (Omega_br) */
    int32_t device_error;    /* nonzero once a bounded device-side wait ran out (PD_ERR_TIMEOUT cause) */
    int32_t auto_method[2];  /* what PD_METHOD_AUTO runs for FP32 / FP64: PD_METHOD_STENCIL or PD_METHOD_FFT */
    int32_t stencil_tile_rows;  /* FP32 2D stencil tile height (32 or 16; set by the autotuner) */
} pd_grid_info;

typedef struct {
    int iterations;        /* total inner (matvec) iterations */
    int outer;             /* FP64 residual replacements (mixed) or restarts (FP64) */
    int f64_matvecs;       /* FP64 operator applications */
    double rel_residual;   /* ||P(b - K u)|| / ||P b||, FP64, recomputed at the end */
    double seconds;        /* wall time of the solve, device-synchronised */
    int persistent;        /* 1 if the FP32 inner loop ran as the persistent kernel */
} pd_cg_stats;

typedef struct {
    int64_t steps;            /* steps taken */
    int64_t newly_broken;     /* bonds broken during the call */
    int64_t broken_total;     /* bonds broken so far on this grid */
} pd_step_stats;

/* Creates a grid of n[0] x n[1] (x n[2]) nodes with spacing h and horizon
 * delta (Sec. 3, Sec. 4).  m = delta / h need not be an integer: the bonds are
 * the offsets with |o| <= m and lambda of Eq. fac:e1 uses the real delta; the
 * kernels run on the disk of radius M = ceil(m), whose offsets beyond m carry
 * a zero coefficient and never break (they appear in pd_get_offsets and the
 * bond mask as intact).  constrained: HOST uint8 [dim][N], nonzero
 * marks a component in the volume-constrained set Omega_c (Sec. 3.3, and the
 * per-component remark of Sec. 3.4); NULL = none.  Sets E = 1, rho = 1,
 * thickness = 1, s0 = 0 (no breaking); every bond intact.
 * Errors: PD_ERR_INVALID (dim not 2/3, n < 1, h <= 0, delta < h, ceil(delta/h)
 * beyond the compiled maximum: 8 in 2D, 4 in 3D), PD_ERR_OOM, PD_ERR_CUDA. */
int pd_create_grid(int dim, const int64_t n[3], double h, double delta,
                   const uint8_t *constrained, pd_grid **out);

/* Material (Sec. 2.1): E Young's modulus, rho density, thickness t (2D alpha =
 * 9E/(pi delta^3 t), 3D alpha = 12E/(pi delta^4); the node volume V_q of Eq.
 * mat:f1 is h^2 t in 2D, so the thickness cancels from the force density),
 * s0 critical stretch (Eq. mu;
 * s0 <= 0 disables breaking).  E_field: DEVICE double [N] per-node modulus or
 * NULL; with a field, bond (p,q) uses (E_p + E_q)/2 and the scalar E is
 * ignored.  The field is copied.  Errors: PD_ERR_INVALID (E, rho, t <= 0 or a
 * field value <= 0). */
int pd_set_material(pd_grid *g, double E, double rho, double thickness, double s0,
                    const double *E_field);

/* Surface correction on incomplete horizons (the remark on Omega_e in Sec. 3.3,
 * Eq. scr in Sec. 5.2): A_pq = v_pq A^_pq.  The paper takes v_pq from its
 * reference; PD_SC_VOLUME is the volume method: V_p = sum of lambda over the
 * in-grid part of the horizon of p, nu_p = V_full / V_p (1 on a full horizon),
 * v_pq = (nu_p + nu_q) / 2, so K stays symmetric.  Every later use of the
 * operator (pd_matvec, pd_cg_solve, pd_adr_solve, pd_step, the adjoints and the
 * modulus gradient) includes it, as a direct correction over the nodes closer
 * than 2M to a face added after the TBT/FFT product; the fused-dot and
 * persistent CG paths step aside.  Builds a compacted node list (4 bytes per
 * node of that band) and a table of (M+1)^(2 dim) doubles; PD_SC_NONE frees
 * them.  Errors: PD_ERR_INVALID (unknown mode, 2^31 nodes or more),
 * PD_ERR_CUDA.  A batch (pd_batch_create) refuses grids with the correction. */
int pd_set_surface_correction(pd_grid *g, int mode);

/* out = K u = -A u (or P K P u with PD_PROJECT), u and out DEVICE [dim][N] of
 * the dtype in flags; u and out must not overlap.  A = A^ + D^e + D^f is the
 * bond sum of Eq. mat:f1 split as in Sec. 3 (2D) and Sec. 4 (3D): the Toeplitz
 * part A^ by the direct stencil or by per-tile FFTs with the block symbol
 * (Algorithms 3 and 4; PD_METHOD_* picks, AUTO the measured faster one), the
 * edge term D^e (Eq. tea:sc) and the broken-bond term D^f (Eq. df).  The
 * stencils keep the rounding relative to |K u|: FP32 sums differences of
 * nearby values, FP64 2D sums pairs of u minus each tile's plane (see
 * PD_ACCURATE, PD_PAIR_FORM).  Broken bonds are honoured unless
 * PD_IGNORE_BROKEN.  Errors: PD_ERR_INVALID (dtype flag missing or both, u
 * aliasing out, two methods, FFT with a modulus field). */
int pd_matvec(pd_grid *g, const void *u, void *out, uint32_t flags, void *stream);

/* The same for `batch` independent vectors stored back to back:
 * u[b * dim * N + c * N + p].  One launch serves the whole batch; batch in
 * [1, 65535] (PD_ERR_INVALID otherwise, nothing written). */
int pd_matvec_batch(pd_grid *g, int64_t batch, const void *u, void *out, uint32_t flags,
                    void *stream);

/* pd_matvec_batch for fields in HOST memory: u_host, out_host HOST
 * [batch][dim][N] of the dtype in flags (page-locked memory -- cudaHostAlloc
 * or cudaHostRegister -- gives full copy bandwidth; pageable memory works but
 * the driver stages it).  The batch is cut into chunks of about 32 MB that are
 * uploaded, multiplied and downloaded on three streams of the grid, so the two
 * copy directions overlap each other and the products.  Ordered on `stream`:
 * it starts after the work already queued there, and work queued afterwards
 * starts after out_host is complete; the call itself returns at once.  Keeps
 * four staging buffers of one chunk with the grid.  Errors as pd_matvec_batch,
 * PD_ERR_OOM for the staging buffers. */
int pd_matvec_batch_host(pd_grid *g, int64_t batch, const void *u_host, void *out_host, uint32_t flags,
                         void *stream);

/* Solves P K P u = P b (Eq. mat:e2 with h = 0 on Omega_c) by conjugate
 * gradients.  b, u: DEVICE double [dim][N]; u is the initial guess on entry
 * and the solution on exit (its constrained components are set to 0).
 * mode: PD_CG_F64 or PD_CG_MIXED, optionally | PD_CG_GRAPH.  Stops when
 * ||P(b - K u)|| <= rtol ||P b|| in FP64.  stats may be NULL.  Returns
 * PD_ERR_NOT_CONVERGED after max_iter inner iterations with u holding the last
 * iterate and stats filled.  On a 2D grid with a constant modulus, no broken
 * bonds, no surface correction and a row length that is a multiple of 4, the
 * FP32 inner loop of PD_CG_MIXED runs as one persistent cooperative kernel
 * when all its 64 x 32 tiles fit one wave of resident CTAs (grid barriers with
 * bounded waits; PD_ERR_TIMEOUT if a wait gives up); on larger such grids, or
 * with PD_CG_GRAPH, as chunks of 32 iterations replayed from a CUDA graph, two
 * launches per iteration (the direction formed inside the operator kernel);
 * elsewhere as graph-replayed chunks of the separate kernels.  All give the
 * same iterates up to FP32 rounding order. */
int pd_cg_solve(pd_grid *g, const double *b, double *u, double rtol, int max_iter,
                uint32_t mode, pd_cg_stats *stats, void *stream);

/* The paper's quasi-static solver: adaptive dynamic relaxation with the
 * central-difference explicit integration of Algorithm 1 (Sec. 2.3), dt = 1,
 * on P K P u = P b.  The paper leaves the fictitious density D and the damping
 * c to its reference (Kilic and Madenci): D_i = 1/4 sum_j |K_ij| (Gershgorin,
 * interior row; with the surface correction, the largest row), c^n =
 * 2 sqrt(u^T K1 u / u^T u) with the diagonal local stiffness
 * K1_ii = -(f_i^n - f_i^(n-1)) / (D_i v_i^(n-1/2)), 0 when not positive.
 * mode PD_ADR_F64: FP64 throughout.  mode PD_ADR_MIXED: the same iteration with
 * the operator applied in FP32 to the correction d = u - u_base (residual
 * r_base - K d, velocity and damping in FP32); whenever that estimate has
 * dropped tenfold, d is added to u_base in FP64 and the residual there is
 * recomputed with the FP64 operator (stats->outer counts these).  Any operator
 * method of pd_matvec, broken bonds included; constant modulus only
 * (PD_ERR_INVALID with a modulus field).  b, u: DEVICE double [dim][N]; u is
 * the initial guess on entry and the solution on exit (constrained components
 * set to 0).  Stops when the FP64 ||P(b - K u)|| <= rtol ||P b|| (PD_ADR_F64:
 * at an iterate, before its update); at most max_iter updates
 * (stats->iterations counts them), PD_ERR_NOT_CONVERGED after that with u
 * holding the last iterate and stats filled (persistent = 0). */
int pd_adr_solve(pd_grid *g, const double *b, double *u, double rtol, int max_iter, uint32_t mode,
                 pd_cg_stats *stats, void *stream);

/* Velocity-Verlet (Algorithm 2) with acceleration a = (f + b)/rho, f = A(mu) u,
 * and bond breaking (Eqs. mu, fra:s1) after each drift.  u, v: DEVICE double
 * [dim][N], updated in place; b: DEVICE double [dim][N] or NULL.
 * v_prescribed: DEVICE double [dim][N] or NULL: constrained components move
 * with this velocity (u += dt v_p, v = v_p) -- the prescribed-velocity layers
 * of Sec. 5.2.  Each call first evaluates f at the incoming u.
 * break_step: DEVICE int32 [N * nnb] or NULL: where bond (p, k) breaks during
 * the call its entry receives step_base + the 1-based step index (used by the
 * adjoint to replay mu).  */
int pd_step(pd_grid *g, double *u, double *v, const double *b, int nsteps, double dt,
            const double *v_prescribed, int32_t *break_step, int32_t step_base,
            pd_step_stats *stats, void *stream);

/* Largest stable step of pd_step (the central-difference scheme of Algorithm 2,
 * undamped): dt = 2 sqrt(rho / (E_max Lambda)), Lambda the largest eigenvalue
 * of the unit-modulus symbol sum_{o in half} 2 c1(o) (1 - cos k.o) over the
 * frequencies of a periodic grid of twice the grid's extent (in 3D at most 96
 * per axis), E_max the modulus or the largest value of the modulus field.  An
 * upper bound on lambda_max(K) / (E_max) for the clamped, partially broken
 * grid, so dt is safe for every bond state.  Host computation, no GPU work.
 * Errors: PD_ERR_INVALID (NULL). */
int pd_stable_dt(pd_grid *g, double *dt);

/* pd_step without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot let a library call cudaMalloc --
 * services whose device memory is owned by their own pool or caching
 * allocator (such a pool may hold nearly all of the GPU, so a foreign
 * cudaMalloc fails or fragments it), and real-time loops where the implicit
 * synchronisation of cudaMalloc would stall the stream.  Same arguments and
 * results as pd_step.
 * Its two work vectors live in one fixed array of 2^20 doubles (8 MiB) that
 * the library defines in device memory; every GPU that loads the library holds
 * it until the process exits.  Limit: dim * N <= 524288 (a 512 x 512 plate in
 * 2D); larger grids get PD_ERR_INVALID with a message naming the limit.  The
 * grid's device must be the current device (PD_ERR_INVALID otherwise).  The
 * first call on each device looks the array's address up; make that first call
 * before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU (other streams, other threads, other grids) race on it
 * and must be serialised by the caller.  The grid itself must have been
 * created beforehand (pd_create_grid allocates). */
int pd_step_noalloc(pd_grid *g, double *u, double *v, const double *b, int nsteps, double dt,
                    const double *v_prescribed, int32_t *break_step, int32_t step_base,
                    pd_step_stats *stats, void *stream);

/* Reverse-mode sweep through one segment of the Verlet loop (Algorithm 2 with
 * a = (f + b)/rho), for gradients of a loss of the final state.  The segment is
 * the `nsteps` steps that pd_step took from the state (u_start, v_start) at
 * step index step_base; the sweep replays them (storing u at every step) with
 * the bond state of each step rebuilt from mask0 (the mask when the run began,
 * DEVICE uint32 [mask_words][N]) and break_step (as recorded by pd_step: bond
 * (p, k) intact at step s unless 0 < break_step[p * nnb + k] <= s), then runs
 * backward.  ubar, vbar, abar (DEVICE double [dim][N]): on entry the adjoints
 * of u, v, a at the segment's end; on exit at its start.  When step_base == 0
 * the dependence of the first acceleration on u_0 is included and abar is
 * cleared.  grad_E (DEVICE double [N] or NULL) accumulates dL/dE for the
 * per-node modulus field (bond modulus (E_p + E_q)/2).  Breaking is not
 * differentiated: the recorded bond history is held fixed.  Uses a workspace
 * of (nsteps + 6) vectors that the grid keeps (allocated on the first call
 * that needs more). */
int pd_step_adjoint(pd_grid *g, const double *u_start, const double *v_start, const double *b, int nsteps,
                    double dt, const double *v_prescribed, const uint32_t *mask0, const int32_t *break_step,
                    int32_t step_base, double *ubar, double *vbar, double *abar, double *grad_E, void *stream);

/* One breaking pass: every intact bond with stretch s >= s0 (Eq. fra:s1,
 * evaluated in FP64 as X = xi + (u_q - u_p), s = (|X| - |xi|)/|xi|, xi = h o,
 * no contraction) is broken in both directions.  u: DEVICE [dim][N] of the
 * dtype in flags (converted to double).  n_newly_broken: host, may be NULL. */
int pd_break_bonds(pd_grid *g, const void *u, uint32_t flags, int64_t *n_newly_broken,
                   void *stream);

/* Breaks every bond whose segment x_p -> x_q meets the closed segment
 * (seg[0], seg[1]) - (seg[2], seg[3]) / den, in units of h from the grid
 * corner (the pre-notch of Sec. 5.2).  In 3D the segment is extruded through
 * the whole thickness (the through-thickness notches of Sec. 5.4): a bond is
 * cut when its projection onto the x-y plane meets the segment.  Exact integer
 * geometry. */
int pd_break_segment(pd_grid *g, const int64_t seg[4], int64_t den, int64_t *n_broken,
                     void *stream);

/* K u on a slab of rows (2D: rows along y; 3D: planes along z), for a grid
 * split across devices along its slowest axis: each device holds a band of
 * rows plus an M-row halo on either side, exchanged before every product (the
 * block-banded structure of Sec. 3.1 and Sec. 4 couples only rows within M of
 * each other).  g is the whole grid (its tables and constraints); u_ext:
 * DEVICE [batch][dim][ext_rows][...] holding grid rows [ext_row0, ext_row0 +
 * ext_rows), which must contain [row0 - M, row0 + rows + M) clipped to the
 * grid; out: DEVICE [batch][dim][rows][...] receives rows [row0, row0 + rows)
 * of K u (P K P u with PD_PROJECT).  In 2D row0 must be a multiple of 32 (the
 * stencil tile height).  Every output of a band whose row count is a multiple
 * of 32, or which ends at the grid's last row, is then computed exactly as by
 * pd_matvec: the slabs of a split give the whole-grid product bit for bit.  (A
 * ragged band inside the grid agrees to rounding in the FP64 2D default form,
 * whose tiles fit their plane over the rows the band holds; bit for bit in the
 * other forms.)
 * Stencil form, intact bonds, constant modulus, no surface correction.
 * Errors: PD_ERR_INVALID (shape, alignment, unsupported state), PD_ERR_CUDA. */
int pd_matvec_rows(pd_grid *g, int64_t batch, int64_t row0, int64_t rows, const void *u_ext, int64_t ext_row0,
                   int64_t ext_rows, void *out, uint32_t flags, void *stream);

/* Chooses the method PD_METHOD_AUTO resolves to for each precision:
 * method = PD_METHOD_STENCIL or PD_METHOD_FFT pins it (both precisions);
 * PD_METHOD_AUTO clears the choice (AUTO then means the stencil until
 * pd_autotune has run).  The FFT method exists for 2D and 3D grids
 * without a modulus field.  Host-only; no device work. */
int pd_set_method(pd_grid *g, uint32_t method);

/* Pins the layout of the FP32 TMA-fed 2D stencil (the bond sum of Eq. mat:f1
 * taken as differences of nearby values): rows = 64 (64 x 64 output tiles, the
 * default; M <= 3, 64 x 32 beyond), 32 (64 x 32 tiles) or 16 (64 x 16 tiles;
 * M <= 4) -- all give identical bits -- or rows = 0, the column walk: each CTA walks down a strip of 128 columns and
 * every input row is staged once (no vertical halo), used at M <= 3 for
 * products without PD_PROJECT or a fused dot (the tile kernel serves the rest).
 * The walk agrees with the tiles to FP32 rounding, not bit for bit; a band of
 * rows (pd_matvec_rows) reproduces the whole-grid product of the same layout bit
 * for bit.  Host-only.  Errors: PD_ERR_INVALID (rows not 0, 16, 32 or 64). */
int pd_set_stencil_tile_rows(pd_grid *g, int rows);

/* Autotuner: measures the candidates of K u for the precision(s) in flags
 * (PD_F32 and/or PD_F64) -- the direct stencil and, without a modulus field,
 * the FFT tiles; for FP32 2D grids on the TMA-fed stencil at M <= 4 also the
 * stencil's layout (64 x 64 tiles at M <= 3, 64 x 32, 64 x 16, and the column
 * walk where it applies) -- on scratch vectors the
 * grid keeps (allocated on the first call), CUDA events on `stream`: three
 * warm-up launches each, then five rounds of ten launches per candidate in
 * turn, each keeping its fastest round.  Records the fastest candidate for
 * PD_METHOD_AUTO and the faster stencil layout for every stencil product.  In
 * FP32 below M = 5 the FFT tiles are timed but not chosen: their rounding error
 * is relative to |u - L| |K| (L the tile's plane) rather than |K u|, which
 * reaches the FP32 tolerance on smooth fields at small horizons
 * (PD_METHOD_FFT still selects them).
 * times_ms: host double [4] or NULL, receives {stencil f32, fft f32, stencil
 * f64, fft f64} in ms per field (the faster stencil tile; 0 where not
 * measured). */
int pd_autotune(pd_grid *g, uint32_t flags, double *times_ms, void *stream);

/* pd_autotune with a cache: cache_path names a JSON file of entries
 *   "<key>": {"method": "stencil"|"fft", "tile_rows": 64|32|16|0, "ms_per_field": t}
 * keyed by dimension, extents, delta/h, precision (and a modulus field), device
 * name and SM count.  When the file holds an entry for every precision in
 * flags, the recorded choice is applied without measuring (*from_cache = 1);
 * otherwise pd_autotune runs and its choice is added to the file (written to
 * cache_path.tmp, then renamed).  from_cache, times_ms: host or NULL.  Errors:
 * as pd_autotune; PD_ERR_INVALID when the file cannot be written. */
int pd_autotune_cached(pd_grid *g, uint32_t flags, const char *cache_path, int *from_cache, double *times_ms,
                       void *stream);

/* ---- batches of independent static solves ----
 * A pd_batch groups `count` existing 2D grids (each with its own size,
 * horizon M <= 4, constraints and modulus; no modulus field) so that their
 * solves advance together: each CG stage is one launch over the tiles or
 * chunks of every plate, and the inner iterations replay as a captured CUDA
 * graph.  The grids must outlive the batch; the batch keeps concatenated
 * copies of the vectors (allocated here).  Errors: PD_ERR_INVALID, PD_ERR_OOM. */
typedef struct pd_batch pd_batch;
int pd_batch_create(pd_grid *const *grids, int count, pd_batch **out);

/* Solves P K P u_i = P b_i for every plate of the batch by FP32 inner CG under
 * FP64 iterative refinement (the PD_CG_MIXED scheme) until every plate reaches
 * ||P(b_i - K u_i)|| <= rtol ||P b_i||.  b, u: HOST arrays of `count` DEVICE
 * pointers to double [2][N_i]; u_i is the initial guess on entry and the
 * solution on exit.  stats: HOST array of `count` entries or NULL (seconds is
 * the wall time of the whole batch).  Plates are taken in order of size, in
 * groups whose FP32 working set fits in L2; the groups run concurrently, each
 * on a stream of the batch, and the call returns with `stream` ordered after
 * all of them.  Each refinement pass ends after a tenfold drop of the FP32
 * residual and the next keeps the search direction (reliable updates).
 * max_iter caps the inner iterations of the slowest plate of each group
 * summed over refinement passes. */
int pd_batch_cg_solve(pd_batch *bt, const double *const *b, double *const *u, double rtol, int max_iter,
                      pd_cg_stats *stats, void *stream);
int pd_batch_destroy(pd_batch *bt);

/* Reads grid facts (host struct). */
int pd_get_info(pd_grid *g, pd_grid_info *info);

/* Neighbour offsets (HOST int32 [nnb][3], each row (ox, oy, oz); rows in
 * lexicographic (oz, oy, ox) order; offset k and nnb-1-k are opposite).
 * cap = rows available. */
int pd_get_offsets(pd_grid *g, int32_t *off, int cap);

/* Bond blocks lambda V_q C(xi) of Eq. mat:f1 at the grid's modulus (HOST
 * double [nnb][3] in 2D: xx, xy, yy; [nnb][6] in 3D: xx, xy, xz, yy, yz, zz),
 * in the order of pd_get_offsets; the kernel table K(o) of Sec. 3.2 / Sec. 4
 * (K(0) = -sum of all blocks).  cap = rows available. */
int pd_get_coefficients(pd_grid *g, double *coef, int cap);

/* Bond mask, DEVICE uint32 [mask_words][N]: bit (k % 32) of word k / 32 of
 * node p is 1 while bond (p, p + o_k) is intact (out-of-grid bits are 1). */
int pd_get_bond_mask(pd_grid *g, uint32_t *mask, void *stream);
int pd_set_bond_mask(pd_grid *g, const uint32_t *mask, void *stream);

/* Modulus gradient of a loss through a static solve (Sec. 2.1 model with the
 * bond modulus (E_p + E_q)/2): given the solution u and the adjoint lam
 * (P K P lam = P dL/du), grad[r] += scale * sum_{q intact} (lam_q - lam_r)^T
 * C1(q - r) (u_q - u_r), C1 the bond block at E = 1.  u, lam: DEVICE double
 * [dim][N]; grad: DEVICE double [N].  scale = -1/2 gives dL/dE. */
int pd_grad_modulus(pd_grid *g, const double *u, const double *lam, double scale,
                    double *grad, void *stream);

/* Diagnostic of the bounded-wait error path that the persistent CG and the
 * TMA pipelines use: one device thread polls a flag that nothing sets, at most
 * `spins` times (about 0.3 us each), records the timeout in the grid's device
 * error word and returns; the host reads the word, clears it and returns
 * PD_ERR_TIMEOUT.  Nothing faults and the context stays usable.  spins in
 * [1, 2^24].  Errors: PD_ERR_INVALID, PD_ERR_CUDA, PD_ERR_TIMEOUT (expected). */
int pd_check_wait_timeout(pd_grid *g, int64_t spins, void *stream);

/* Measured arithmetic peak of the current device, the denominator of the
 * roofline of the ALU-bound kernels (the paper has no counterpart): a kernel
 * of independent fused multiply-add chains in FP64 (flags PD_F64) or FP32
 * (PD_F32) over every SM, timed with CUDA events on `stream` for about 20 ms.
 * flops: host, receives FLOP/s (an FMA counts two).  Synchronises the stream.
 * Errors: PD_ERR_INVALID (flags, flops NULL), PD_ERR_CUDA. */
int pd_probe_fma_rate(uint32_t flags, double *flops, void *stream);

/* Critical bond stretch from the energy release rate G0 (Eq. fra:s1):
 * s0 = sqrt(4 pi G0 / (9 E delta)) in plane stress (mode PD_PLANE_STRESS) and
 * sqrt(5 pi G0 / (12 E delta)) in plane strain (PD_PLANE_STRAIN), for the 2D
 * model; pass the result to pd_set_material.  Host only, no GPU needed.
 * Errors: PD_ERR_INVALID (non-positive or non-finite input, unknown mode, s0 NULL). */
int pd_critical_stretch(double G0, double E, double delta, int mode, double *s0);

/* Destroys the grid and frees its device memory.  NULL is accepted. */
int pd_destroy(pd_grid *g);

/* Message of the last failed call on this thread ("" if none). */
const char *pd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PD_H */

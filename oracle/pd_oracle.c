/*
 * pd_oracle.c -- plain FP64 CPU oracle for linear bond-based peridynamics on a
 * uniform grid (the method of "A fast computational framework for the linear
 * bond-based peridynamic model", arXiv 2301.11828).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header
 * or table with the CUDA library and never calls it.
 *
 * Everything here is the plain definition written out: a direct sum over the
 * neighbour list of every node (Eq. mat:f1), with no FFT, no blocking and no
 * reordering.  Compiled with -O2 -ffp-contract=off so that no multiply-add is
 * fused; the node loops carry an OpenMP pragma, which does not change the
 * arithmetic of any single node.
 *
 * Conventions (readings of the paper, each listed in the design notes):
 *  - nodes x_p = h (i + 1/2, j + 1/2[, k + 1/2]) with 0-based i, j, k and
 *    p = i + Nx (j + Ny k) (Sec. 3 and Sec. 4 node numbering, 0-based);
 *  - per-node arrays are stored component-major: u[c * N + p];
 *  - the offset of a bond is o = (q - p) in grid units; the neighbour test
 *    |x_q - x_p| <= delta with delta = m h is |o|^2 <= m^2 (m = delta / h, an
 *    integer in the paper's examples but any real >= 1 here)
 *    (Eq. band, Sec. 3.1), and the bond vector is xi = h o (Eq. frb:e1);
 *  - f = A u is the paper's internal force; the stiffness product used by the
 *    solver is K u = -A u (Eq. mat:e2 reads -A u = b on the free nodes);
 *  - mu is stored as one byte per (node, offset index): 1 intact, 0 broken.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* Neighbour set (Eq. band) and partial-volume factor (Eq. fac:e1)           */
/* ------------------------------------------------------------------------- */

/* Offsets o != 0 with |o| <= m (m = delta / h, any real >= 1: the bonds of
 * Eq. band), in lexicographic (oz, oy, ox) order; the test is |o|^2 <= m^2 on
 * the integer |o|^2 (a tie at |o| = m counts, as Eq. fac:e1 includes r = delta).
 * Because the set is centrally symmetric, the offset at index k and the one at
 * index (count - 1 - k) are negatives of each other.  Returns the count, or -1
 * when cap is too small. */
int or_offsets(int dim, double m, int32_t *off, int cap)
{
    int cnt = 0;
    const int R = (int)ceil(m - 1e-9);
    int zlo = (dim == 3) ? -R : 0, zhi = (dim == 3) ? R : 0;
    for (int oz = zlo; oz <= zhi; ++oz)
        for (int oy = -R; oy <= R; ++oy)
            for (int ox = -R; ox <= R; ++ox) {
                int d2 = ox * ox + oy * oy + oz * oz;
                if (d2 == 0 || (double)d2 > m * m + 1e-9) continue;
                if (cnt >= cap) return -1;
                off[3 * cnt + 0] = ox;
                off[3 * cnt + 1] = oy;
                off[3 * cnt + 2] = oz;
                ++cnt;
            }
    return cnt;
}

/* Eq. fac:e1: lambda = 1 for r <= delta - dx/2, (2 delta + dx - 2 r)/(2 dx)
 * for delta - dx/2 < r <= delta, 0 otherwise. */
double or_lambda(double r, double delta, double dx)
{
    if (r <= delta - dx / 2.0) return 1.0;
    if (r <= delta) return (2.0 * delta + dx - 2.0 * r) / (2.0 * dx);
    return 0.0;
}

/* Sec. 2.1: alpha = 9E / (pi delta^3 t) in 2D (t the plate thickness),
 * alpha = 12E / (pi delta^4) in 3D. */
double or_alpha(int dim, double E, double delta, double thickness)
{
    if (dim == 2) return 9.0 * E / (M_PI * delta * delta * delta * thickness);
    return 12.0 * E / (M_PI * delta * delta * delta * delta);
}

/* Eq. mat:f1 weighs neighbour q by V_q, the volume of node q: h^dim in 3D and,
 * for the plate of thickness t, h^2 t in 2D.  The routines below take the
 * constant that multiplies lambda h^dim: alpha V_q / h^dim (alpha t in 2D). */
double or_bond_constant(int dim, double E, double delta, double thickness)
{
    const double a = or_alpha(dim, E, delta, thickness);
    return dim == 2 ? a * thickness : a;
}

/* Bond block lambda_q V_q C(xi) of Eqs. ker:e1 and mat:f1 for offset o:
 * c[a][b] = alpha xi_a xi_b / |xi|^3 * lambda * h^dim with xi = h o. */
static void bond_block(int dim, const int32_t *o, double h, double m, double alpha,
                       double c[3][3])
{
    double xi[3] = {h * o[0], h * o[1], h * o[2]};
    double r2 = 0.0;
    for (int a = 0; a < dim; ++a) r2 += xi[a] * xi[a];
    double r = sqrt(r2);
    double lam = or_lambda(r, m * h, h);
    double V = (dim == 2) ? h * h : h * h * h;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            c[a][b] = (a < dim && b < dim) ? alpha * xi[a] * xi[b] / (r2 * r) * lam * V : 0.0;
}

/* Public copy of the bond block for the tests (row-major 3x3). */
void or_bond_block(int dim, const int32_t *o, double h, double m, double alpha, double *c9)
{
    double c[3][3];
    bond_block(dim, o, h, m, alpha, c);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) c9[3 * a + b] = c[a][b];
}

/* ------------------------------------------------------------------------- */
/* Internal force f = A u (Eq. mat:f1, with Eq. matrix for its 2D blocks and  */
/* Eq. mae:e1 for 3D)                                                         */
/* ------------------------------------------------------------------------- */

/*
 * f_p = sum over neighbours q of p inside the grid of
 *       mu_pq * lambda_q V_q C(x_q - x_p) (u_q - u_p).
 * alpha: the micromodulus constant; when E is not NULL, alpha is the value
 *        for E = 1 and the bond (p, q) uses modulus (E_p + E_q) / 2.
 * mu:    NULL (all bonds intact) or [N][nnb] bytes.
 * nu:    NULL, or the per-node surface-correction factors of or_surface_nu:
 *        the bond (p, q) is then scaled by v_pq = (nu_p + nu_q) / 2.
 */
int or_force(int dim, const int64_t *n, double h, double m, double alpha,
             const double *E, const uint8_t *mu, const double *nu, const double *u, double *f)
{
    int32_t off[3 * 16384];
    int nnb = or_offsets(dim, m, off, 16384);
    if (nnb < 0) return -1;
    double (*blk)[3][3] = malloc(sizeof(double[3][3]) * (size_t)nnb);
    if (!blk) return -2;
    for (int k = 0; k < nnb; ++k) bond_block(dim, off + 3 * k, h, m, alpha, blk[k]);
    const int64_t nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1;
    const int64_t N = nx * ny * nz;

#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int64_t i = p % nx, j = (p / nx) % ny, kz = p / (nx * ny);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < nnb; ++k) {
            int64_t qi = i + off[3 * k], qj = j + off[3 * k + 1], qk = kz + off[3 * k + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            if (mu && !mu[p * nnb + k]) continue;
            int64_t q = qi + nx * (qj + ny * qk);
            double scale = E ? 0.5 * (E[p] + E[q]) : 1.0;
            if (nu) scale *= 0.5 * (nu[p] + nu[q]);
            for (int a = 0; a < dim; ++a) {
                double s = 0.0;
                for (int b = 0; b < dim; ++b)
                    s += blk[k][a][b] * (u[b * N + q] - u[b * N + p]);
                acc[a] += scale * s;
            }
        }
        for (int a = 0; a < dim; ++a) f[a * N + p] = acc[a];
    }
    free(blk);
    return nnb;
}

/* Stiffness product with the volume constraint: out = P K P u, K = -A, where
 * P zeroes the constrained components (cons[c * N + p] != 0). */
int or_stiffness(int dim, const int64_t *n, double h, double m, double alpha,
                 const double *E, const uint8_t *mu, const double *nu, const uint8_t *cons,
                 const double *u, double *out)
{
    const int64_t N = n[0] * n[1] * ((dim == 3) ? n[2] : 1);
    double *up = malloc(sizeof(double) * (size_t)(dim * N));
    if (!up) return -2;
    for (int64_t t = 0; t < dim * N; ++t) up[t] = (cons && cons[t]) ? 0.0 : u[t];
    int rc = or_force(dim, n, h, m, alpha, E, mu, nu, up, out);
    for (int64_t t = 0; t < dim * N; ++t) out[t] = (cons && cons[t]) ? 0.0 : -out[t];
    free(up);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Static solve: textbook conjugate gradients on P K P u = P b.  The paper    */
/* solves Eq. mat:e2 with ADR; CG on the same symmetric operator is the       */
/* solver this library pairs with the matvec.                                 */
/* ------------------------------------------------------------------------- */

static double dot(const double *a, const double *b, int64_t len)
{
    double s = 0.0;
    for (int64_t t = 0; t < len; ++t) s += a[t] * b[t];
    return s;
}

/* x: in = initial guess, out = solution.  Returns the iteration count (or a
 * negative error); *relres receives ||P(b - K x)|| / ||P b|| recomputed from
 * scratch at the end. */
int or_cg(int dim, const int64_t *n, double h, double m, double alpha, const double *E,
          const uint8_t *mu, const double *nu, const uint8_t *cons, const double *b, double *x,
          double rtol, int maxit, double *relres)
{
    const int64_t N = n[0] * n[1] * ((dim == 3) ? n[2] : 1), L = dim * N;
    double *r = malloc(sizeof(double) * L), *p = malloc(sizeof(double) * L),
           *q = malloc(sizeof(double) * L), *pb = malloc(sizeof(double) * L);
    if (!r || !p || !q || !pb) { free(r); free(p); free(q); free(pb); return -2; }
    for (int64_t t = 0; t < L; ++t) {
        pb[t] = (cons && cons[t]) ? 0.0 : b[t];
        if (cons && cons[t]) x[t] = 0.0;
    }
    double bnorm = sqrt(dot(pb, pb, L));
    if (bnorm == 0.0) bnorm = 1.0;
    int it = 0;
    for (int restart = 0; restart < 8 && it < maxit; ++restart) {
        or_stiffness(dim, n, h, m, alpha, E, mu, nu, cons, x, q);
        for (int64_t t = 0; t < L; ++t) { r[t] = pb[t] - q[t]; p[t] = r[t]; }
        double rr = dot(r, r, L);
        if (sqrt(rr) / bnorm <= rtol) break;
        for (; it < maxit; ++it) {
            or_stiffness(dim, n, h, m, alpha, E, mu, nu, cons, p, q);
            double a = rr / dot(p, q, L);
            for (int64_t t = 0; t < L; ++t) { x[t] += a * p[t]; r[t] -= a * q[t]; }
            double rr_new = dot(r, r, L);
            if (sqrt(rr_new) / bnorm <= rtol) { ++it; rr = rr_new; break; }
            double beta = rr_new / rr;
            rr = rr_new;
            for (int64_t t = 0; t < L; ++t) p[t] = r[t] + beta * p[t];
        }
    }
    or_stiffness(dim, n, h, m, alpha, E, mu, nu, cons, x, q);
    for (int64_t t = 0; t < L; ++t) r[t] = pb[t] - q[t];
    *relres = sqrt(dot(r, r, L)) / bnorm;
    free(r); free(p); free(q); free(pb);
    return it;
}

/* ------------------------------------------------------------------------- */
/* Bond breaking (Eqs. mu and fra:s1)                                         */
/* ------------------------------------------------------------------------- */

/*
 * For every intact bond (p, q) with q > p: stretch
 *   s = (|xi + eta| - |xi|) / |xi|,  xi = h o,  eta = u_q - u_p,
 * evaluated in this order in FP64 without contraction:
 *   X_c = xi_c + (u_q,c - u_p,c);  l = sqrt(X_x X_x + X_y X_y [+ X_z X_z]);
 *   r = sqrt(xi_x xi_x + xi_y xi_y [+ xi_z xi_z]);  s = (l - r) / r.
 * The bond breaks when s >= s0 (Eq. mu), in both directions, for good.
 * Returns the number of bonds newly broken.
 */
int64_t or_break(int dim, const int64_t *n, double h, double m, double s0,
                 const double *u, uint8_t *mu)
{
    int32_t off[3 * 16384];
    int nnb = or_offsets(dim, m, off, 16384);
    const int64_t nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1;
    const int64_t N = nx * ny * nz;
    int64_t broken = 0;
    for (int64_t p = 0; p < N; ++p) {
        int64_t i = p % nx, j = (p / nx) % ny, kz = p / (nx * ny);
        for (int k = 0; k < nnb; ++k) {
            int64_t qi = i + off[3 * k], qj = j + off[3 * k + 1], qk = kz + off[3 * k + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            int64_t q = qi + nx * (qj + ny * qk);
            if (q <= p || !mu[p * nnb + k]) continue;
            double xi[3] = {h * off[3 * k], h * off[3 * k + 1], h * off[3 * k + 2]};
            double X[3];
            for (int c = 0; c < dim; ++c) X[c] = xi[c] + (u[c * N + q] - u[c * N + p]);
            double l2 = X[0] * X[0] + X[1] * X[1];
            double r2 = xi[0] * xi[0] + xi[1] * xi[1];
            if (dim == 3) { l2 = l2 + X[2] * X[2]; r2 = r2 + xi[2] * xi[2]; }
            double l = sqrt(l2), r = sqrt(r2);
            double s = (l - r) / r;
            if (s >= s0) {
                mu[p * nnb + k] = 0;
                mu[q * nnb + (nnb - 1 - k)] = 0;
                ++broken;
            }
        }
    }
    return broken;
}

/* ------------------------------------------------------------------------- */
/* Pre-notch: bonds whose segment x_p -> x_q meets a given closed segment.   */
/* Exact integer geometry in units of h / (2 den) from the grid corner.      */
/* ------------------------------------------------------------------------- */

static int sgn(__int128 v) { return (v > 0) - (v < 0); }

static int orient(const int64_t *a, const int64_t *b, const int64_t *c)
{
    __int128 v = (__int128)(b[0] - a[0]) * (c[1] - a[1]) - (__int128)(b[1] - a[1]) * (c[0] - a[0]);
    return sgn(v);
}

static int on_seg(const int64_t *a, const int64_t *b, const int64_t *c)
{ /* c collinear with a-b: does it lie within the bounding box? */
    return (c[0] >= (a[0] < b[0] ? a[0] : b[0]) && c[0] <= (a[0] > b[0] ? a[0] : b[0]) &&
            c[1] >= (a[1] < b[1] ? a[1] : b[1]) && c[1] <= (a[1] > b[1] ? a[1] : b[1]));
}

static int seg_meet(const int64_t *p1, const int64_t *p2, const int64_t *q1, const int64_t *q2)
{
    int d1 = orient(q1, q2, p1), d2 = orient(q1, q2, p2);
    int d3 = orient(p1, p2, q1), d4 = orient(p1, p2, q2);
    if (d1 * d2 < 0 && d3 * d4 < 0) return 1;
    if (d1 == 0 && on_seg(q1, q2, p1)) return 1;
    if (d2 == 0 && on_seg(q1, q2, p2)) return 1;
    if (d3 == 0 && on_seg(p1, p2, q1)) return 1;
    if (d4 == 0 && on_seg(p1, p2, q2)) return 1;
    return 0;
}

/* seg = (x0, y0, x1, y1) numerators over den, in units of h from the grid
 * corner (node i, j sits at (i + 1/2, j + 1/2)).  Breaks every bond that
 * meets the closed segment; returns the number of bonds broken.  In 3D the
 * segment is extruded through the whole thickness (a planar notch normal to
 * the x-y plane): a bond is cut when its projection onto the x-y plane meets
 * the segment, whatever its z extent (a bond along z alone projects to a
 * point, cut only if that point lies on the segment). */
int64_t or_prenotch(int dim, const int64_t *n, double m, const int64_t *seg, int64_t den, uint8_t *mu)
{
    int32_t off[3 * 16384];
    int nnb = or_offsets(dim, m, off, 16384);
    const int64_t nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1, N = nx * ny * nz;
    int64_t A[2] = {2 * seg[0], 2 * seg[1]}, B[2] = {2 * seg[2], 2 * seg[3]};
    int64_t broken = 0;
    for (int64_t p = 0; p < N; ++p) {
        int64_t i = p % nx, j = (p / nx) % ny, kz = p / (nx * ny);
        for (int k = 0; k < nnb; ++k) {
            int64_t qi = i + off[3 * k], qj = j + off[3 * k + 1], qk = kz + off[3 * k + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            int64_t q = qi + nx * (qj + ny * qk);
            if (q <= p) continue;
            int64_t P1[2] = {den * (2 * i + 1), den * (2 * j + 1)};
            int64_t P2[2] = {den * (2 * qi + 1), den * (2 * qj + 1)};
            if (seg_meet(P1, P2, A, B)) {
                if (mu[p * nnb + k]) ++broken;
                mu[p * nnb + k] = 0;
                mu[q * nnb + (nnb - 1 - k)] = 0;
            }
        }
    }
    return broken;
}

/* ------------------------------------------------------------------------- */
/* Velocity-Verlet (Algorithm 2) with a = (f + b) / rho, bond breaking and    */
/* prescribed-velocity components.                                            */
/* ------------------------------------------------------------------------- */

/*
 * One call advances nsteps steps from (u, v, mu).  It first evaluates
 * f = A(mu) u.  Per step:
 *   1. u += dt v + dt^2/2 a on free components; u += dt vpres on constrained;
 *   2. break bonds with the new u;
 *   3. a_new = (A(mu) u + b) / rho;
 *   4. v += dt/2 (a + a_new) on free components; v = vpres on constrained.
 * cons may be NULL (nothing constrained); vpres may be NULL (zero velocity).
 * Returns the number of bonds broken during the call.
 */
int64_t or_vv(int dim, const int64_t *n, double h, double m, double alpha, const double *E,
              uint8_t *mu, const double *nu, double s0, const uint8_t *cons, const double *vpres,
              const double *b, double rho, double dt, int nsteps, double *u, double *v)
{
    const int64_t N = n[0] * n[1] * ((dim == 3) ? n[2] : 1), L = dim * N;
    double *a = malloc(sizeof(double) * L), *an = malloc(sizeof(double) * L);
    if (!a || !an) { free(a); free(an); return -2; }
    or_force(dim, n, h, m, alpha, E, mu, nu, u, a);
    for (int64_t t = 0; t < L; ++t) a[t] = (a[t] + (b ? b[t] : 0.0)) / rho;
    int64_t broken = 0;
    for (int s = 0; s < nsteps; ++s) {
        for (int64_t t = 0; t < L; ++t) {
            if (cons && cons[t]) u[t] += dt * (vpres ? vpres[t] : 0.0);
            else u[t] += dt * v[t] + 0.5 * dt * dt * a[t];
        }
        if (mu && s0 > 0.0) broken += or_break(dim, n, h, m, s0, u, mu);
        or_force(dim, n, h, m, alpha, E, mu, nu, u, an);
        for (int64_t t = 0; t < L; ++t) {
            an[t] = (an[t] + (b ? b[t] : 0.0)) / rho;
            if (cons && cons[t]) v[t] = vpres ? vpres[t] : 0.0;
            else v[t] += 0.5 * dt * (a[t] + an[t]);
            a[t] = an[t];
        }
    }
    free(a); free(an);
    return broken;
}

/* ------------------------------------------------------------------------- */
/* Gradient of a static loss with respect to the per-node modulus            */
/* ------------------------------------------------------------------------- */

/*
 * With bond modulus (E_p + E_q)/2 and K_P u = P b, a loss L(u) has
 *   dL/dE_r = -(alpha1/2) sum_{q in N(r), intact} (lam_q - lam_r)^T Chat(q - r) (u_q - u_r)
 * where lam solves K_P lam = P dL/du and alpha1 Chat is the bond block at
 * E = 1 (alpha = alpha1).  u and lam are the projected (constrained-zero)
 * vectors.  With surface-correction factors nu (nullable) each bond term also
 * carries v_rq = (nu_r + nu_q) / 2.  Writes g[N].
 */
int or_grad_modulus(int dim, const int64_t *n, double h, double m, double alpha1,
                    const uint8_t *mu, const double *nu, const double *u, const double *lam, double *g)
{
    int32_t off[3 * 16384];
    int nnb = or_offsets(dim, m, off, 16384);
    double (*blk)[3][3] = malloc(sizeof(double[3][3]) * (size_t)nnb);
    if (!blk) return -2;
    for (int k = 0; k < nnb; ++k) bond_block(dim, off + 3 * k, h, m, alpha1, blk[k]);
    const int64_t nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1;
    const int64_t N = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int64_t i = p % nx, j = (p / nx) % ny, kz = p / (nx * ny);
        double acc = 0.0;
        for (int k = 0; k < nnb; ++k) {
            int64_t qi = i + off[3 * k], qj = j + off[3 * k + 1], qk = kz + off[3 * k + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            if (mu && !mu[p * nnb + k]) continue;
            int64_t q = qi + nx * (qj + ny * qk);
            double t = 0.0;
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b)
                    t += (lam[a * N + q] - lam[a * N + p]) * blk[k][a][b] *
                         (u[b * N + q] - u[b * N + p]);
            acc += nu ? 0.5 * (nu[p] + nu[q]) * t : t;
        }
        g[p] = -0.5 * acc;
    }
    free(blk);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Surface correction (the remark on Omega_e in Sec. 3.3 and Eq. scr)         */
/* ------------------------------------------------------------------------- */

/*
 * The paper scales the bonds of nodes with an incomplete horizon by a
 * factor v_pq and leaves the factor to its reference; the reading taken here
 * is the volume method: with V_p the partial volume of the part of the
 * horizon of p inside the grid,
 *   V_p = sum over neighbours q of p inside the grid of lambda(|x_q - x_p|) h^dim,
 * and V_full the same sum over the complete horizon,
 *   nu_p = V_full / V_p   (1 on every node with a complete horizon),
 * and every bond uses the mean of its two ends, v_pq = (nu_p + nu_q) / 2, so
 * that A stays symmetric.  The common factor h^dim cancels in the ratio.
 * Writes nu[N]; returns the offset count.
 */
int or_surface_nu(int dim, const int64_t *n, double h, double m, double *nu)
{
    int32_t off[3 * 16384];
    int nnb = or_offsets(dim, m, off, 16384);
    if (nnb < 0) return -1;
    double *lam = malloc(sizeof(double) * (size_t)nnb);
    if (!lam) return -2;
    double full = 0.0;
    for (int k = 0; k < nnb; ++k) {
        double r2 = 0.0;
        for (int a = 0; a < dim; ++a) r2 += (h * off[3 * k + a]) * (h * off[3 * k + a]);
        lam[k] = or_lambda(sqrt(r2), m * h, h);
        full += lam[k];
    }
    const int64_t nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1;
    const int64_t N = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int64_t i = p % nx, j = (p / nx) % ny, kz = p / (nx * ny);
        double V = 0.0;
        for (int k = 0; k < nnb; ++k) {
            int64_t qi = i + off[3 * k], qj = j + off[3 * k + 1], qk = kz + off[3 * k + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            V += lam[k];
        }
        nu[p] = full / V;
    }
    free(lam);
    return nnb;
}

/*
 * Largest absolute row sum of K (all bonds intact, no projection) per
 * component: out[a] = max_p sum over columns (q, b) of |K_(p,a),(q,b)|, where
 * the diagonal block of row p is sum_q v_pq C_pq and the off-diagonal blocks
 * are -v_pq C_pq (nu NULL: v = 1).  This is the Gershgorin bound behind the
 * fictitious density of the ADR method.
 */
int or_row_abs_max(int dim, const int64_t *n, double h, double m, double alpha, const double *nu, double *out)
{
    int32_t off[3 * 16384];
    int nnb = or_offsets(dim, m, off, 16384);
    if (nnb < 0) return -1;
    double (*blk)[3][3] = malloc(sizeof(double[3][3]) * (size_t)nnb);
    if (!blk) return -2;
    for (int k = 0; k < nnb; ++k) bond_block(dim, off + 3 * k, h, m, alpha, blk[k]);
    const int64_t nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1;
    const int64_t N = nx * ny * nz;
    for (int a = 0; a < 3; ++a) out[a] = 0.0;
    for (int64_t p = 0; p < N; ++p) {
        int64_t i = p % nx, j = (p / nx) % ny, kz = p / (nx * ny);
        double diag[3][3] = {{0}}, offsum[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < nnb; ++k) {
            int64_t qi = i + off[3 * k], qj = j + off[3 * k + 1], qk = kz + off[3 * k + 2];
            if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
            int64_t q = qi + nx * (qj + ny * qk);
            double v = nu ? 0.5 * (nu[p] + nu[q]) : 1.0;
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) {
                    diag[a][b] += v * blk[k][a][b];
                    offsum[a] += fabs(v * blk[k][a][b]);
                }
        }
        for (int a = 0; a < dim; ++a) {
            double r = offsum[a];
            for (int b = 0; b < dim; ++b) r += fabs(diag[a][b]);
            if (r > out[a]) out[a] = r;
        }
    }
    free(blk);
    return nnb;
}

/* Number of threads the OpenMP loops above use (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
#endif
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the number of OpenMP threads of the node loops (n >= 1); used to time the
 * oracle on one core beside all cores. */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

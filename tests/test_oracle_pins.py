"""Pins for the FP64 oracle: what the paper and the mathematics fix, independent of the oracle's own code.

Each test names the plausible mistake it is there to catch.  CPU only.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic as syn


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# --------------------------------------------------------------------------- neighbour set

@pytest.mark.parametrize("dim,M,count,partial", [(2, 1, 4, 4), (2, 3, 28, 8), (2, 4, 48, 12), (2, 6, 112, 16),
                                                 (3, 3, 122, None)])
def test_offset_counts_gauss_circle(dim, M, count, partial):
    """Lattice-point counts of the disk / ball |o| <= M (Gauss circle problem:
    N2(9) = 29, N2(16) = 49, N2(36) = 113, N3(9) = 123, minus the centre), and the
    number of offsets in the partial-volume shell M - 1/2 < |o| <= M of Eq. fac:e1."""
    offs = oracle.offsets(dim, M)
    assert len(offs) == count
    # brute-force recount over the cube
    rng_ = range(-M, M + 1)
    zr = rng_ if dim == 3 else [0]
    brute = sum(1 for z in zr for y in rng_ for x in rng_ if 0 < x * x + y * y + z * z <= M * M)
    assert brute == count
    # central symmetry of the ordering: k and nnb-1-k are opposite
    assert np.array_equal(offs, -offs[::-1])
    if partial is not None:
        r = np.sqrt((offs.astype(float) ** 2).sum(1))
        lam = np.array([oracle.lam(v, float(M), 1.0) for v in r])
        assert int((lam < 1.0).sum()) == partial


def test_lambda_values():
    """Eq. fac:e1 at hand-computed points (catches the garbled variant printed as
    'M - sqrt(.)/2 + 1/2' and an off-by-half threshold)."""
    h = 0.25
    M = 3
    d = M * h
    assert oracle.lam(1 * h, d, h) == 1.0
    assert oracle.lam(math.sqrt(5) * h, d, h) == 1.0          # 2.236 <= 2.5
    assert oracle.lam(3 * h, d, h) == pytest.approx(0.5, abs=1e-15)
    assert oracle.lam(math.sqrt(8) * h, d, h) == pytest.approx(3.5 - math.sqrt(8), abs=1e-14)
    assert oracle.lam(math.sqrt(10) * h, d, h) == 0.0


# --------------------------------------------------------------------------- operator identities

def _field_coords(n, h):
    dim = len(n)
    idx = np.indices(tuple(reversed(n)))[::-1]   # x first
    return (idx + 0.5) * h


@pytest.mark.parametrize("dim,n,M", [(2, (13, 9), 3), (2, (9, 17), 4), (3, (7, 6, 8), 2), (2, (12, 10), 2.5),
                                     (3, (7, 8, 6), 1.5)])
def test_translation_rotation_give_zero_force(dim, n, M):
    """P1/P2: a rigid translation and an infinitesimal rigid rotation produce no
    bond force on ANY row, edges and broken bonds included (each bond term
    C(xi)(u_q - u_p) vanishes).  Catches a wrong diagonal term, a wrong sign of
    the xy block or a transposed block."""
    h = 1.0 / 16
    al = oracle.alpha(dim, 1.0, M * h)
    rng = np.random.default_rng(1)
    mu = oracle.intact_mu(dim, n, M)
    mu_rand = (rng.random(mu.shape) > 0.2).astype(np.uint8)
    # make the random bond state symmetric
    nnb = mu.shape[1]
    offs = oracle.offsets(dim, M)
    N = int(np.prod(n))
    coords = np.indices(tuple(reversed(n))).reshape(dim, N)[::-1]
    for p in range(N):
        for k in range(nnb):
            q = coords[:, p] + offs[k, :dim]
            if all(0 <= q[c] < n[c] for c in range(dim)):
                qi = int(sum(int(q[c]) * int(np.prod(n[:c])) for c in range(dim)))
                mu_rand[qi, nnb - 1 - k] = mu_rand[p, k]
    E = syn.lognormal_modulus(n, 0.1, 7)
    X = _field_coords(n, h)
    shift = np.stack([np.full(X[0].shape, 0.3 + c) for c in range(dim)])
    rot = np.zeros_like(X)
    rot[0], rot[1] = -X[1], X[0]          # omega = e_z
    for u in (shift, rot):
        for mu_ in (None, mu_rand):
            for E_ in (None, E):
                f = oracle.force(dim, n, h, M, al, u, E=E_, mu=mu_)
                scale = al * h ** dim * np.abs(u).max() * 10
                assert np.abs(f).max() < 1e-12 * scale


@pytest.mark.parametrize("dim,n,M", [(2, (15, 15), 3), (3, (9, 9, 9), 2), (2, (16, 15), 3.7)])
def test_linear_field_zero_on_full_horizon(dim, n, M):
    """P3: u = G x gives f = 0 at every node whose horizon lies inside the grid
    (odd symmetry of the kernel); at edge nodes it does not vanish."""
    h = 1.0 / 8
    al = oracle.alpha(dim, 1.0, M * h)
    X = _field_coords(n, h)
    G = np.random.default_rng(2).normal(size=(dim, dim))
    u = np.einsum("ab,b...->a...", G, X)
    f = oracle.force(dim, n, h, M, al, u)
    R = oracle.radius(M)
    inner = (slice(None),) + (slice(R, -R),) * dim
    scale = al * h ** dim * np.abs(u).max()
    assert np.abs(f[inner]).max() < 1e-12 * scale
    assert np.abs(f).max() > 1e-3 * scale


@pytest.mark.parametrize("dim,Ms,target", [(2, (6, 12, 24), 2.25), (3, (3, 6, 10), 2.4)])
def test_quadratic_field_continuum_limit(dim, Ms, target):
    """P4: for u = (x^2, 0[, 0]) the interior force tends to the local Navier value
    2 C11 (plane stress nu = 1/3: C11 = 9E/8 -> 2.25E; 3D nu = 1/4: C11 = 6E/5 -> 2.4E)
    as the horizon holds more nodes.  This pins the constant of alpha (9/pi, 12/pi)
    and the |xi|^-3 power; the error falls monotonically."""
    errs = []
    for M in Ms:
        n = (2 * M + 3,) * dim
        h = 1.0 / 64
        al = oracle.alpha(dim, 1.0, M * h)
        X = _field_coords(n, h)
        u = np.zeros_like(X)
        u[0] = X[0] ** 2
        f = oracle.force(dim, n, h, M, al, u)
        c = (M + 1,) * dim
        fx = f[(0,) + c]
        for a in range(1, dim):
            assert abs(f[(a,) + c]) < 1e-10
        errs.append(abs(fx / target - 1.0))
    assert errs[0] > errs[1] > errs[2]
    assert errs[-1] < 0.06


@pytest.mark.parametrize("t", [0.4, 2.5])
def test_plate_thickness(t):
    """Sec. 2.1 puts the plate thickness t in the 2D alpha (9E / (pi delta^3 t)),
    and Eq. mat:f1 weighs each neighbour by its node volume, h^2 t for the
    plate.  alpha itself scales as 1/t; the constant the force routines take
    (alpha V_q / h^2) does not depend on t, and with it the quadratic field of
    P4 tends to the plane-stress value 2.25E at any thickness, while alpha
    alone with an area volume (a dropped t) would give 2.25E / t."""
    delta = 3.0 / 64
    a1, at = oracle.alpha(2, 1.0, delta), oracle.alpha(2, 1.0, delta, t)
    assert abs(at * t / a1 - 1.0) < 1e-15
    assert abs(oracle.bond_constant(2, 1.0, delta, t) / a1 - 1.0) < 1e-15
    assert oracle.bond_constant(3, 1.0, delta, t) == oracle.alpha(3, 1.0, delta)   # 3D: no thickness
    M, h = 24, 1.0 / 64
    n = (2 * M + 3,) * 2
    X = _field_coords(n, h)
    u = np.zeros_like(X)
    u[0] = X[0] ** 2
    c = (M + 1,) * 2
    fx = oracle.force(2, n, h, M, oracle.bond_constant(2, 1.0, M * h, t), u)[(0,) + c]
    assert abs(fx / 2.25 - 1.0) < 0.06
    fa = oracle.force(2, n, h, M, oracle.alpha(2, 1.0, M * h, t), u)[(0,) + c]
    assert abs(fa * t / 2.25 - 1.0) < 0.06 and abs(fa / 2.25 - 1.0) > 0.3


@pytest.mark.parametrize("dim,n,M", [(2, (11, 7), 1), (2, (11, 7), 2), (2, (8, 8), 3), (2, (9, 10), 4),
                                     (3, (5, 6, 4), 1), (3, (5, 4, 6), 2), (2, (10, 9), 2.5), (2, (9, 9), 3.7),
                                     (3, (5, 6, 5), 1.5)])
def test_direct_sum_equals_dense_assembly(dim, n, M):
    """P5/P7: the C direct sum equals the brute-force dense matrix assembled from
    node positions (Eq. matrix / mae:e1); the dense matrix is symmetric and
    negative semidefinite (-A is PSD), with a null space holding the rigid
    translations."""
    h = 1.0 / 8   # binary h: positions and the distance test are exact
    al = oracle.alpha(dim, 1.0, M * h)
    A = oracle.dense_matrix(dim, n, h, M, al)
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    w = np.linalg.eigvalsh(-A)
    assert w.min() > -1e-12 * w.max()
    u = np.random.default_rng(3).uniform(-1, 1, (dim,) + tuple(reversed(n)))
    f = oracle.force(dim, n, h, M, al, u)
    assert _rel(f.reshape(-1), A @ u.reshape(-1)) < 1e-14


@pytest.mark.parametrize("dim,n,M,frac", [(2, (11, 7), 2, 0.0), (2, (13, 10), 3, 0.1), (2, (9, 12), 4, 0.05),
                                          (3, (5, 6, 7), 2, 0.0), (3, (6, 5, 7), 3, 0.05), (2, (12, 11), 2.5, 0.1),
                                          (2, (10, 13), 3.7, 0.0), (3, (6, 6, 7), 2.5, 0.05)])
def test_direct_sum_equals_fmvm(dim, n, M, frac):
    """P7: the direct sum equals the paper's fast form: TBT/TBTBT part by 2N
    circulant embedding and FFT (Algorithms 3/4), plus D^e (Eq. tea:sc) and the
    broken-bond correction D^f (Eq. tea:fr)."""
    h = 1.0 / 16
    al = oracle.alpha(dim, 1.0, M * h)
    rng = np.random.default_rng(4)
    u = rng.uniform(-1, 1, (dim,) + tuple(reversed(n)))
    mu = None
    if frac > 0:
        mu = oracle.intact_mu(dim, n, M)
        uu = u * 0.2
        oracle.break_bonds(dim, n, h, M, 0.05, uu, mu)   # a symmetric random-ish broken set
        assert (mu == 0).sum() > 0
    f1 = oracle.force(dim, n, h, M, al, u, mu=mu)
    f2 = oracle.fmvm(dim, n, h, M, al, u, mu=mu)
    assert _rel(f1, f2) < 1e-13


@pytest.mark.parametrize("dim,M,L", [(2, 3, (24, 20)), (2, 6, (30, 32)), (3, 2, (10, 12, 8))])
def test_symbol_real_zero_mean_negative_semidefinite(dim, M, L):
    """P6: the symbol of the TBT part is real (K even), vanishes at k = 0 (row sum
    of K is zero, Eq. frb:e4) and minus it is PSD at every frequency."""
    h = 1.0 / 32
    G = oracle.symbol(dim, L, h, M, oracle.alpha(dim, 1.0, M * h))
    assert np.abs(G.imag).max() < 1e-10 * np.abs(G.real).max()
    Gr = G.real
    zero = (slice(None), slice(None)) + (0,) * dim
    assert np.abs(Gr[zero]).max() < 1e-10 * np.abs(Gr).max()
    mats = np.moveaxis(Gr.reshape(dim, dim, -1), 2, 0)
    w = np.linalg.eigvalsh(-mats)
    assert w.min() > -1e-10 * np.abs(Gr).max()


def test_total_bond_count_formula():
    """P8: the number of (unordered) bonds equals 1/2 sum_o prod_i (N_i - |o_i|)."""
    for dim, n, M in [(2, (17, 11), 3), (2, (20, 9), 6), (3, (7, 8, 9), 3)]:
        offs = oracle.offsets(dim, M)
        expect = sum(int(np.prod([n[c] - abs(int(o[c])) for c in range(dim)])) for o in offs) // 2
        # count via the breaking routine: a huge stretch field breaks every bond exactly once
        mu = oracle.intact_mu(dim, n, M)
        X = _field_coords(n, 1.0)
        u = 10.0 * X   # uniform stretch of 1000 %
        got = oracle.break_bonds(dim, n, 1.0, M, 1.0, u, mu)
        assert got == expect


def test_force_sum_vanishes():
    """P10: sum_p f_p = 0 for any u, modulus field and symmetric broken set
    (pairwise antisymmetry of the bond forces)."""
    dim, n, M = 2, (21, 17), 3
    h = 1.0 / 16
    al = oracle.alpha(dim, 1.0, M * h)
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, (dim,) + tuple(reversed(n)))
    mu = oracle.intact_mu(dim, n, M)
    oracle.break_bonds(dim, n, h, M, 0.3, 0.1 * u, mu)
    E = syn.lognormal_modulus(n, 0.1, 3)
    f = oracle.force(dim, n, h, M, al, u, E=E, mu=mu)
    assert np.abs(f.reshape(dim, -1).sum(1)).max() < 1e-12 * np.abs(f).max() * f[0].size


# --------------------------------------------------------------------------- static solve

def test_cg_matches_sparse_direct_solve():
    """P9: oracle CG on the clamped plate equals a direct sparse LU solve (SuperLU)
    of the reduced system assembled column by column from the oracle matvec."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    w = syn.plate_static(24, 3, tag=11, u_amp=1e-3)
    al = oracle.alpha(2, w.E, w.delta)
    x, it, rel = oracle.cg(2, w.n, w.h, w.M, al, w.b, cons=w.constrained, rtol=1e-10)
    assert rel <= 1e-10 and it > 10
    free = np.flatnonzero(w.constrained.reshape(-1) == 0)
    L = w.constrained.size
    cols = []
    for j in free:
        e = np.zeros(L)
        e[j] = 1.0
        col = oracle.stiffness(2, w.n, w.h, w.M, al, e.reshape(w.constrained.shape), cons=w.constrained)
        cols.append(sp.csc_matrix(col.reshape(-1)[free][:, None]))
    Kf = sp.hstack(cols).tocsc()
    assert abs(Kf - Kf.T).max() < 1e-9 * abs(Kf).max()
    xd = spl.spsolve(Kf, w.b.reshape(-1)[free])
    assert _rel(x.reshape(-1)[free], xd) < 1e-7


def test_small_plate_cg_converges():
    """The 64x64 clamped plate (8192 DOF) reaches a true relative residual of 1e-8."""
    w = syn.small_plate()
    al = oracle.alpha(2, w.E, w.delta)
    x, it, rel = oracle.cg(2, w.n, w.h, w.M, al, w.b, cons=w.constrained, rtol=1e-8)
    assert rel <= 1e-8
    assert np.all(x[w.constrained.astype(bool)] == 0)
    # displacement goes in the direction of the traction
    assert x[0, :, -1].mean() > 0


def test_modulus_gradient_matches_finite_differences():
    """P12: dL/dE from the adjoint bond sum equals central differences of
    L(u(E)) = 1/2 |u|^2 with K_P(E) u = P b."""
    dim, n, M = 2, (12, 10), 3
    h = 1.0 / 12
    cons = syn.clamp_left(dim, n, M)
    b = syn.gaussian_field(dim, n, 1e-3, 21) * (1 - cons)
    E = syn.lognormal_modulus(n, 0.1, 22)
    al1 = oracle.alpha(dim, 1.0, M * h)

    def solve(Ef):
        x, _, rel = oracle.cg(dim, n, h, M, al1, b, cons=cons, E=Ef, rtol=1e-13)
        return x

    u = solve(E)
    lam_, _, _ = oracle.cg(dim, n, h, M, al1, u, cons=cons, E=E, rtol=1e-13)   # dL/du = u
    g = oracle.grad_modulus(dim, n, h, M, al1, u, lam_)
    rng = np.random.default_rng(6)
    for flat in rng.choice(E.size, 6, replace=False):
        idx = np.unravel_index(flat, E.shape)
        eps = 1e-5 * E[idx]
        Ep, Em = E.copy(), E.copy()
        Ep[idx] += eps
        Em[idx] -= eps
        fd = (0.5 * (solve(Ep) ** 2).sum() - 0.5 * (solve(Em) ** 2).sum()) / (2 * eps)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).max())


# --------------------------------------------------------------------------- breaking

def test_uniform_stretch_breaks_all_or_none():
    """Eq. fra:s1: under u = eps x every bond has stretch eps; with s0 below eps
    all bonds break, above it none do.  A sign error such as |x'+u'-x+u|
    fails this."""
    dim, n, M, h = 2, (12, 11), 3, 0.1
    X = _field_coords(n, h)
    eps = 2e-3
    for s0, expect_all in ((1e-3, True), (3e-3, False)):
        mu = oracle.intact_mu(dim, n, M)
        got = oracle.break_bonds(dim, n, h, M, s0, eps * X, mu)
        offs = oracle.offsets(dim, M)
        total = sum(int(np.prod([n[c] - abs(int(o[c])) for c in range(dim)])) for o in offs) // 2
        assert got == (total if expect_all else 0)


def test_finite_rotation_breaks_nothing_and_compression_neither():
    """A finite rigid rotation keeps every bond length: no stretch, nothing breaks;
    uniform compression gives negative stretch: nothing breaks either."""
    dim, n, M, h = 2, (14, 9), 3, 0.1
    X = _field_coords(n, h)
    th = 0.3
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    u_rot = np.einsum("ab,b...->a...", R - np.eye(2), X)
    mu = oracle.intact_mu(dim, n, M)
    assert oracle.break_bonds(dim, n, h, M, 1e-9, u_rot, mu) == 0
    mu = oracle.intact_mu(dim, n, M)
    assert oracle.break_bonds(dim, n, h, M, 1e-6, -0.01 * X, mu) == 0


def test_breaking_symmetric_and_monotone():
    """P11: the broken set is symmetric (bond (p,q) is broken in p's list iff it is
    broken in q's) and never heals."""
    dim, n, M, h = 2, (16, 13), 3, 1.0 / 16
    rng = np.random.default_rng(8)
    mu = oracle.intact_mu(dim, n, M)
    offs = oracle.offsets(dim, M)
    nnb = len(offs)
    prev = mu.copy()
    for step in range(3):
        u = rng.normal(0, 1e-2 * h, (dim,) + tuple(reversed(n)))
        oracle.break_bonds(dim, n, h, M, 1e-2, u, mu)
        assert np.all(mu <= prev)
        prev = mu.copy()
    N = int(np.prod(n))
    coords = np.indices(tuple(reversed(n))).reshape(dim, N)[::-1]
    for p in range(N):
        for k in range(nnb):
            q = coords[:, p] + offs[k, :dim]
            if all(0 <= q[c] < n[c] for c in range(dim)):
                qi = int(q[0] + n[0] * q[1])
                assert mu[p, k] == mu[qi, nnb - 1 - k]
    assert (mu == 0).sum() > 0


def _notch_count_fraction(n, M, a, b, Y):
    """Exact count with rationals: bonds whose segment meets y = Y for x in [a, b]
    (positions in units of h from the corner)."""
    cnt = 0
    offs = oracle.offsets(2, M)
    for o in offs:
        ox, oy = int(o[0]), int(o[1])
        if oy <= 0:
            continue
        for j in range(n[1]):
            y0, y1 = Fraction(2 * j + 1, 2), Fraction(2 * (j + oy) + 1, 2)
            if j + oy >= n[1] or not (y0 <= Y <= y1):
                continue
            t = (Y - y0) / (y1 - y0)
            for i in range(n[0]):
                if not (0 <= i + ox < n[0]):
                    continue
                x = Fraction(2 * i + 1, 2) + ox * t
                if a <= x <= b:
                    cnt += 1
    return cnt


@pytest.mark.parametrize("nside", [20, 32])
def test_prenotch_count_exact(nside):
    """P11: the pre-notch (closed segment y = L/2, |x - L/2| <= 0.1 L) breaks
    exactly the bonds that an independent rational-arithmetic count finds; far
    from the notch tips each crossed column loses sum_{oy>0} oy bonds (18 at M=3)."""
    M = 3
    w = syn.crack_plate(nside, M)
    mu = oracle.intact_mu(2, w.n, M)
    got = oracle.prenotch(w.n, M, w.extra["notch"], w.extra["notch_den"], mu)
    s = w.extra["notch"]
    den = w.extra["notch_den"]
    expect = _notch_count_fraction(w.n, M, Fraction(s[0], den), Fraction(s[2], den), Fraction(s[1], den))
    assert got == expect
    offs = oracle.offsets(2, M)
    assert sum(int(o[1]) for o in offs if o[1] > 0) == 18


# --------------------------------------------------------------------------- dynamics

def test_verlet_energy_conservation_second_order():
    """P10: undamped, unconstrained, unbroken velocity-Verlet conserves
    E = 1/2 rho |v|^2 - 1/2 u.A u up to O(dt^2): halving dt cuts the drift ~4x."""
    dim, n, M = 2, (16, 16), 3
    h = 1.0 / 16
    al = oracle.alpha(dim, 1.0, M * h)
    rng = np.random.default_rng(9)
    u0 = rng.normal(0, 1e-3, (dim,) + tuple(reversed(n)))
    # stable dt from the symbol bound: lambda_max(-A) <= max eigen of -G^
    G = oracle.symbol(dim, (32, 32), h, M, al).real
    lam_max = np.linalg.eigvalsh(-np.moveaxis(G.reshape(2, 2, -1), 2, 0)).max()
    dt0 = 0.2 * 2.0 / math.sqrt(lam_max)

    def energy(u, v):
        f = oracle.force(dim, n, h, M, al, u)
        return 0.5 * (v * v).sum() - 0.5 * (u * f).sum()

    drifts = []
    T = 40 * dt0
    for dt in (dt0, dt0 / 2):
        u, v = u0.copy(), np.zeros_like(u0)
        e0 = energy(u, v)
        steps = int(round(T / dt))
        es = []
        for _ in range(steps):
            oracle.vv(dim, n, h, M, al, u, v, 1, dt)
            es.append(energy(u, v))
        drifts.append(max(abs(e - e0) for e in es) / e0)
    assert drifts[0] < 0.05
    assert 2.5 < drifts[0] / drifts[1] < 6.0


def test_verlet_prescribed_velocity_layers():
    """Constrained components move exactly as u0 + v t and keep v = v_prescribed."""
    w = syn.crack_plate(24, 3)
    n, M, h = w.n, w.M, w.h
    al = oracle.alpha(2, 1.0, M * h)
    lay = w.extra["vel_layers"]
    cons = np.zeros((2,) + lay.shape, dtype=np.uint8)
    cons[1] = lay != 0
    vpres = np.zeros((2,) + lay.shape)
    vpres[1] = lay * 1e-3
    u = np.zeros((2,) + lay.shape)
    v = vpres.copy()
    dt = 1e-3
    mu = oracle.intact_mu(2, n, M)
    oracle.vv(2, n, h, M, al, u, v, 50, dt, E=w.extra["E_field"], mu=mu, s0=w.s0, cons=cons, vpres=vpres)
    np.testing.assert_allclose(u[1][lay != 0], 50 * dt * vpres[1][lay != 0], rtol=1e-12)
    assert np.array_equal(v[1][lay != 0], vpres[1][lay != 0])
    assert np.abs(u[0]).max() > 0   # free x components respond


def test_dynamic_modulus_gradient_matches_finite_differences():
    """P12 (dynamic): the oracle's discrete adjoint of Algorithm 2 equals central
    differences of L = 1/2 |u_N|^2 in E, on a pre-notched plate whose bonds break
    during the run (the +/- runs are checked to break the same bonds)."""
    w = syn.crack_plate(20, 3)
    n, M, h = w.n, w.M, w.h
    lay = w.extra["vel_layers"]
    cons = np.zeros((2,) + lay.shape, dtype=np.uint8)
    cons[1] = lay != 0
    vp = np.zeros((2,) + lay.shape)
    vp[1] = lay * 0.02
    E = w.extra["E_field"]
    al1 = oracle.alpha(2, 1.0, M * h)
    mu0 = oracle.intact_mu(2, n, M)
    oracle.prenotch(n, M, w.extra["notch"], w.extra["notch_den"], mu0)
    dt, steps, s0 = 2e-3, 30, 2e-3
    u0 = np.zeros((2,) + lay.shape)
    uN, g = oracle.vv_grad_modulus(2, n, h, M, al1, E, u0, vp.copy(), steps, dt, mu0=mu0, s0=s0, cons=cons, vpres=vp)
    us, _, mus = oracle.vv_history(2, n, h, M, al1, u0, vp.copy(), steps, dt, E=E, mu0=mu0, s0=s0, cons=cons, vpres=vp)
    assert (mus[-1] == 0).sum() > (mu0 == 0).sum()   # bonds broke during the run
    rng = np.random.default_rng(12)
    picks = list(np.argsort(-np.abs(g).ravel())[:3]) + list(rng.choice(E.size, 2, replace=False))
    for flat in picks:
        idx = np.unravel_index(flat, E.shape)
        eps = 1e-4 * E[idx]
        res = []
        for sgn in (1, -1):
            Ep = E.copy()
            Ep[idx] += sgn * eps
            usp, _, musp = oracle.vv_history(2, n, h, M, al1, u0, vp.copy(), steps, dt, E=Ep, mu0=mu0, s0=s0,
                                            cons=cons, vpres=vp)
            assert all(np.array_equal(a, b) for a, b in zip(musp, mus))
            res.append(0.5 * (usp[-1] ** 2).sum())
        fd = (res[0] - res[1]) / (2 * eps)
        assert g[idx] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(g).max())


# ---------------------------------------------------------------- ADR (Algorithm 1)
def test_adr_single_dof_critical_damping():
    """One spring k with fictitious mass d: the local-stiffness estimate is exact
    (k/d), so the damping is the critical value 2 sqrt(k/d) of a 1-DOF
    oscillator, and the iteration settles at the static answer b/k."""
    k, d, b = 3.0, 5.0, np.array([2.0])
    rec = []
    u, it, rel = oracle.adr(lambda x: k * x, b, np.array([d]), rtol=1e-12, maxit=10000, record=rec)
    assert rec and abs(rec[0] - 2.0 * np.sqrt(k / d)) <= 1e-14
    assert abs(u[0] - b[0] / k) <= 1e-11 and rel <= 1e-12


def test_adr_uncoupled_springs_converge():
    """Diagonal stiffness (uncoupled DOFs) with the Gershgorin density d = k/4 x 1.2:
    the answer is b / k componentwise."""
    rng = np.random.default_rng(5)
    kk = rng.uniform(0.5, 4.0, (2, 7))
    b = rng.uniform(-1.0, 1.0, (2, 7))
    D = np.array([0.25 * kk[0].max() * 1.2, 0.25 * kk[1].max() * 1.2])
    u, it, rel = oracle.adr(lambda x: kk * x, b, D, rtol=1e-11, maxit=200000)
    assert np.max(np.abs(u - b / kk)) <= 1e-9


@pytest.mark.parametrize("M", [2, 3])
def test_adr_reaches_the_cg_solution(M):
    """ADR on the plate (clamp left, traction right) converges to the solution of
    the same projected system found by textbook CG."""
    w = syn.plate_static(24, M, tag=3, u_amp=0.0)
    al = oracle.alpha(2, 1.0, w.delta)
    u, it, rel = oracle.adr_solve(2, w.n, w.h, w.M, al, w.b, cons=w.constrained, rtol=1e-10, maxit=200000)
    x, _, _ = oracle.cg(2, w.n, w.h, w.M, al, w.b, cons=w.constrained, rtol=1e-13)
    assert rel <= 1e-10
    assert np.linalg.norm(u - x) / np.linalg.norm(x) <= 1e-7


def test_adr_density_is_the_gershgorin_row_sum():
    """D = 1/4 sum_j |K_ij| for an interior row, against the dense matrix."""
    n, M, h = (12, 11), 3, 1.0 / 12
    al = oracle.alpha(2, 1.0, M * h)
    Kd = -oracle.dense_matrix(2, n, h, M, al)
    D = oracle.adr_density(2, h, M, al)
    N = n[0] * n[1]
    p = 5 * n[0] + 6   # interior node (full horizon)
    for a in range(2):
        row = Kd[a * N + p]
        assert abs(0.25 * np.abs(row).sum() - D[a]) <= 1e-12 * D[a]


# --------------------------------------------------------------------------- surface correction

def test_surface_nu_hand_values():
    """nu = V_full / V_p with lambda-weighted partial volumes, worked by hand.

    2D M = 1: the four axis bonds have lambda = 1/2, V_full = 2: corner 2/1,
    edge 2/1.5.  2D M = 2: axis-1 and diagonal bonds lambda = 1, axis-2 bonds
    lambda = 1/2, V_full = 10: corner 10/4, edge 10/6.5, the node one step in
    from two faces 10/9.  3D M = 1: V_full = 3: corner 3/1.5, edge 3/2, face
    3/2.5.  Catches an unweighted count, an inverted ratio and an off-by-one in
    the in-grid test."""
    nu = oracle.surface_nu(2, (5, 4), 1.0 / 8, 1)
    assert nu[0, 0] == 2.0 and nu[3, 4] == 2.0
    assert abs(nu[0, 2] - 4.0 / 3.0) <= 1e-15 and abs(nu[2, 0] - 4.0 / 3.0) <= 1e-15
    assert np.all(nu[1:3, 1:4] == 1.0)
    nu = oracle.surface_nu(2, (9, 8), 1.0 / 16, 2)
    assert abs(nu[0, 0] - 2.5) <= 1e-15
    assert abs(nu[4, 0] - 10.0 / 6.5) <= 1e-15
    assert abs(nu[1, 1] - 10.0 / 9.0) <= 1e-15
    assert np.all(nu[2:6, 2:7] == 1.0)
    nu = oracle.surface_nu(3, (4, 4, 4), 1.0 / 4, 1)
    assert nu[0, 0, 0] == 2.0 and nu[3, 3, 3] == 2.0
    assert nu[0, 0, 1] == 1.5 and nu[0, 1, 1] == 1.2
    assert np.all(nu[1:3, 1:3, 1:3] == 1.0)
    # 3D M = 2: |o|^2 = 1 (6 bonds, lambda 1), 2 (12, lambda 1), 3 (8, lambda 2.5 - sqrt 3),
    # 4 (6, lambda 1/2): V_full = 21 + 8 (2.5 - sqrt 3); a corner keeps 3 + 3 + (2.5 - sqrt 3) + 1.5
    l3 = 2.5 - math.sqrt(3.0)
    nu = oracle.surface_nu(3, (6, 6, 6), 1.0 / 8, 2)
    assert abs(nu[0, 0, 0] - (21 + 8 * l3) / (7.5 + l3)) <= 1e-14
    assert nu[2:4, 2:4, 2:4].min() == 1.0 and nu[2:4, 2:4, 2:4].max() == 1.0


@pytest.mark.parametrize("dim,n,M", [(2, (8, 8), 2), (2, (11, 7), 3), (3, (5, 6, 7), 2)])
def test_surface_corrected_force_equals_symmetrised_dense(dim, n, M):
    """A_sc off the diagonal is (N A + A N) / 2 with N = diag(nu) (the bond
    factor (nu_p + nu_q) / 2), and each diagonal block is minus the sum of its
    row's off-diagonal blocks; built from the dense matrix, against the direct
    sum with nu.  Catches a one-sided factor (nu_p only), a product instead of
    the mean, and a diagonal left uncorrected."""
    h = 1.0 / 16
    al = oracle.alpha(dim, 1.0, M * h)
    A = oracle.dense_matrix(dim, n, h, M, al)
    N = int(np.prod(n))
    nu = oracle.surface_nu(dim, n, h, M).reshape(-1)
    Nm = np.tile(nu, dim)
    same = np.tile(np.eye(N, dtype=bool), (dim, dim))
    Aoff = np.where(same, 0.0, A)
    Asc = 0.5 * (Nm[:, None] * Aoff + Aoff * Nm[None, :])
    for a in range(dim):
        for b in range(dim):
            blk = Asc[a * N:(a + 1) * N, b * N:(b + 1) * N]
            Asc[a * N + np.arange(N), b * N + np.arange(N)] = -blk.sum(axis=1)
    rng = np.random.default_rng(7)
    u = rng.uniform(-1, 1, (dim,) + tuple(reversed(n)))
    f = oracle.force(dim, n, h, M, al, u, nu=nu)
    assert _rel(f.reshape(-1), Asc @ u.reshape(-1)) <= 1e-13
    # symmetric, and the rigid motions still give zero force on every row
    K = -Asc
    assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
    assert np.abs(oracle.force(dim, n, h, M, al, np.ones_like(u), nu=nu)).max() <= 1e-12 * np.abs(K).max()


def test_surface_corrected_row_abs_max_matches_dense():
    """The ADR density with the correction: the largest absolute row sum of
    K_sc over all rows, against the dense matrix; without it, the interior row."""
    n, M, h = (12, 11), 3, 1.0 / 16
    al = oracle.alpha(2, 1.0, M * h)
    A = oracle.dense_matrix(2, n, h, M, al)
    N = n[0] * n[1]
    nu = oracle.surface_nu(2, n, h, M).reshape(-1)
    Nm = np.tile(nu, 2)
    same = np.tile(np.eye(N, dtype=bool), (2, 2))
    Aoff = np.where(same, 0.0, A)
    Asc = 0.5 * (Nm[:, None] * Aoff + Aoff * Nm[None, :])
    for a in range(2):
        for b in range(2):
            blk = Asc[a * N:(a + 1) * N, b * N:(b + 1) * N]
            Asc[a * N + np.arange(N), b * N + np.arange(N)] = -blk.sum(axis=1)
    rs = np.abs(Asc).sum(axis=1)
    got = oracle.row_abs_max(2, n, h, M, al, nu)
    for a in range(2):
        assert abs(got[a] - rs[a * N:(a + 1) * N].max()) <= 1e-12 * got[a]
    plain = oracle.row_abs_max(2, n, h, M, al)
    assert np.allclose(plain, 4 * oracle.adr_density(2, h, M, al), rtol=1e-12, atol=0)
    assert np.all(got > plain)   # corrected edge rows are heavier than the interior row here


def test_surface_corrected_adr_reaches_the_corrected_cg_solution():
    """ADR with the correction (and its density) converges to the solution of
    the corrected system that CG finds."""
    n, M = (24, 20), 3
    h = 1.0 / n[0]
    al = oracle.alpha(2, 1.0, M * h)
    cons = syn.clamp_left(2, n, M)
    b = syn.traction_right(2, n, M, 1e-3)
    nu = oracle.surface_nu(2, n, h, M)
    u, it, rel = oracle.adr_solve(2, n, h, M, al, b, cons=cons, rtol=1e-10, maxit=200000, nu=nu)
    x, _, _ = oracle.cg(2, n, h, M, al, b, cons=cons, rtol=1e-13, nu=nu)
    x0, _, _ = oracle.cg(2, n, h, M, al, b, cons=cons, rtol=1e-13)
    assert rel <= 1e-10
    assert np.linalg.norm(u - x) / np.linalg.norm(x) <= 1e-7
    assert np.linalg.norm(x - x0) / np.linalg.norm(x0) > 1e-3   # the correction changes the answer


# --------------------------------------------------------------------------- 3D through-thickness notch

def _vertical_notch_cuts(P1, P2, xn, y0, y1):
    """Closed vertical segment x = xn, y0 <= y <= y1 against the closed segment P1-P2 (Fractions)."""
    (x1, ya), (x2, yb) = P1, P2
    if not (min(x1, x2) <= xn <= max(x1, x2)):
        return False
    if x1 == x2:   # the bond is vertical too (or a point): overlap of the y ranges on the line x = xn
        return max(min(ya, yb), y0) <= min(max(ya, yb), y1)
    y = ya + (xn - x1) * (yb - ya) / (x2 - x1)
    return y0 <= y <= y1


@pytest.mark.parametrize("n,M,seg", [((12, 10, 4), 2, (20, 0, 20, 20)), ((9, 8, 3), 3, (14, 6, 14, 30)),
                                     ((10, 7, 1), 2, (18, 4, 18, 17))])
def test_prenotch_3d_is_the_extruded_2d_notch(n, M, seg):
    """Every bond whose x-y projection meets the vertical notch is cut, counted by
    brute force over node pairs with a parametric intersection in exact
    fractions (a route of its own).  With one layer the 3D set equals the 2D
    set.  Catches a z coordinate leaking into the test, a missed z-bond family
    and an asymmetric cut."""
    den = 4
    mu = oracle.intact_mu(3, n, M)
    got = oracle.prenotch(n, M, seg, den, mu, dim=3)
    xn, y0, y1 = Fraction(seg[0], den), Fraction(seg[1], den), Fraction(seg[3], den)
    offs = oracle.offsets(3, M)
    nx, ny, nz = n
    expect = 0
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = i + nx * (j + ny * k)
                for kk, (ox, oy, oz) in enumerate(offs):
                    qi, qj, qk = i + ox, j + oy, k + oz
                    if not (0 <= qi < nx and 0 <= qj < ny and 0 <= qk < nz):
                        continue
                    q = qi + nx * (qj + ny * qk)
                    cut = _vertical_notch_cuts((Fraction(2 * i + 1, 2), Fraction(2 * j + 1, 2)),
                                               (Fraction(2 * qi + 1, 2), Fraction(2 * qj + 1, 2)), xn, y0, y1)
                    assert mu[p, kk] == (0 if cut else 1)
                    if cut and q > p:
                        expect += 1
    assert got == expect and got > 0
    if nz == 1:
        mu2 = oracle.intact_mu(2, n[:2], M)
        assert oracle.prenotch(n[:2], M, seg, den, mu2) == got


def test_kw_block_step_is_below_the_stable_step():
    """The stable step stored with the 3D block, 2 h / sqrt(Lambda_1) with
    Lambda_1 = 1.2185, is a lower bound: Lambda_1 >= the largest eigenvalue of
    the unit symbol on the block's doubled grid; the run's step is below it."""
    w = syn.kw_block()
    L = tuple(2 * v for v in w.n)
    G = oracle.symbol(3, L, 1.0, w.M, oracle.alpha(3, 1.0, w.M * 1.0)).real
    lam = np.linalg.eigvalsh(-np.moveaxis(G.reshape(3, 3, -1), 2, 0)).max()
    assert 1.2 < lam <= 1.2185
    assert w.extra["dt_stable"] <= 2.0 * w.h / np.sqrt(lam)
    assert w.extra["dt"] < 0.1 * w.extra["dt_stable"]


def test_critical_stretch_hand_values():
    """Eq. fra:s1: G0 = 9/(4 pi) (plane stress) or 12/(5 pi) (plane strain) with
    E = delta = 1 gives s0 = 1; s0 grows as sqrt(G0 / (E delta)); the two
    cases differ by sqrt(15/16) for the same G0."""
    assert abs(oracle.critical_stretch(9 / (4 * math.pi), 1.0, 1.0, "stress") - 1.0) <= 1e-15
    assert abs(oracle.critical_stretch(12 / (5 * math.pi), 1.0, 1.0, "strain") - 1.0) <= 1e-15
    a = oracle.critical_stretch(3.0, 2.0, 0.5, "stress")
    assert abs(oracle.critical_stretch(12.0, 2.0, 0.5, "stress") / a - 2.0) <= 1e-15
    assert abs(oracle.critical_stretch(3.0, 2.0, 0.5, "strain") / a - math.sqrt(15 / 16)) <= 1e-15



# --------------------------------------------------------------------------- horizons that are not a whole number of spacings

@pytest.mark.parametrize("dim,m,count,shell", [(2, 1.5, 8, 4), (2, 2.5, 20, 8), (2, 3.7, 44, 8), (3, 2.5, 80, None)])
def test_offsets_and_lambda_for_real_m(dim, m, count, shell):
    """|o| <= m for m = delta / h not an integer, counted by hand: 2D m = 1.5 keeps
    |o|^2 in {1, 2} (4 + 4), m = 2.5 adds {4, 5} (4 + 8), m = 3.7 adds {8, 9, 10, 13}
    (4 + 4 + 8 + 8); 3D m = 2.5: |o|^2 in {1..6} (6 + 12 + 8 + 6 + 24 + 24).  The
    partial-volume shell m - 1/2 < |o| <= m holds |o|^2 = 2 (m = 1.5), 5 (m = 2.5)
    and 13 (m = 3.7; |o| = sqrt(10) = 3.16 is inside 3.2).  Catches rounding m to
    an integer and a shell taken from the integer radius."""
    offs = oracle.offsets(dim, m)
    assert len(offs) == count
    assert np.array_equal(offs, -offs[::-1])
    d2 = (offs.astype(float) ** 2).sum(1)
    assert d2.max() <= m * m
    if shell is not None:
        lam = np.array([oracle.lam(math.sqrt(v), m, 1.0) for v in d2])
        assert int((lam < 1.0).sum()) == shell
        assert np.all(lam > 0)
    # hand values at m = 2.5: |o| = 2 is inside (lambda 1), |o| = sqrt(5) on the shell
    assert oracle.lam(2.0, 2.5, 1.0) == 1.0
    assert abs(oracle.lam(math.sqrt(5), 2.5, 1.0) - (3.0 - math.sqrt(5))) <= 1e-15


def test_kw_block_geometry():
    """The 3D block's inputs: notches at 3/8 and 5/8 of the length from the y = 0
    face to half the width; the velocity zone is the first M layers strictly
    between the notches, y component only, at v0; nothing else is constrained."""
    w = syn.kw_block(201, 101, 9, 3, v0=0.00634)
    den = w.extra["notch_den"]
    (a, b) = w.extra["notches"]
    assert a[0] / den == 3 * 201 / 8 and b[0] / den == 5 * 201 / 8
    assert a[1] == b[1] == 0 and a[3] / den == b[3] / den == 101 / 2
    cons, vp = w.constrained, w.extra["v_prescribed"]
    assert cons[0].sum() == 0 and cons[2].sum() == 0
    zone = cons[1].astype(bool)
    k, j, i = np.nonzero(zone)
    assert set(j.tolist()) == {0, 1, 2}
    xc = i + 0.5
    assert np.all(xc > 3 * 201 / 8) and np.all(xc < 5 * 201 / 8)
    assert zone.sum() == 9 * 3 * int(((np.arange(201) + 0.5 > 3 * 201 / 8) & (np.arange(201) + 0.5 < 5 * 201 / 8)).sum())
    assert np.all(vp[1][zone] == 0.00634) and np.all(vp[1][~zone] == 0) and vp[0].sum() == vp[2].sum() == 0
    assert abs(w.extra["dt"] - 0.06747 / 201) <= 1e-15

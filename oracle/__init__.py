"""FP64 CPU oracle for the peridynamic stiffness product, solve and crack loop.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product package never
imports this module, and this module never imports the product package.

Two independent routes to the same operator live here:

* ``pd_oracle.c`` (loaded through ctypes): the plain definition -- a direct FP64
  sum over every node's neighbour list, Eq. mat:f1 -- plus textbook CG, the
  velocity-Verlet loop of Algorithm 2, bond breaking (Eqs. mu, fra:s1), the
  pre-notch and the modulus gradient.
* numpy (this file): a brute-force dense assembly of the matrix of Eq. matrix /
  Eq. mae:e1 from node positions, and the paper's fast form, Algorithm 3
  (FMVM) / Algorithm 4 (FTTM): kernel table, 2N circulant embedding, FFT,
  Hadamard product, inverse FFT, crop, then the D^e (Eq. tea:sc) and D^f
  (Eq. tea:fr) corrections.  Each exists to pin the C oracle against a second
  derivation on small grids.

Array layout: ``[dim][Nz][Ny][Nx]`` float64, x fastest.  Offsets are listed in
lexicographic (oz, oy, ox) order, so offset k and offset nnb-1-k are opposite.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pd_oracle.c with gcc (FP64, no contraction, OpenMP) if stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.c_void_p
            L.or_offsets.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int]
            L.or_offsets.restype = ctypes.c_int
            L.or_lambda.argtypes = [ctypes.c_double] * 3
            L.or_lambda.restype = ctypes.c_double
            L.or_alpha.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_alpha.restype = ctypes.c_double
            L.or_bond_constant.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_bond_constant.restype = ctypes.c_double
            L.or_bond_block.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.or_force.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   dp, dp, dp, dp, dp]
            L.or_force.restype = ctypes.c_int
            L.or_stiffness.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       dp, dp, dp, dp, dp, dp]
            L.or_stiffness.restype = ctypes.c_int
            L.or_cg.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                dp, dp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_double)]
            L.or_cg.restype = ctypes.c_int
            L.or_break.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
            L.or_break.restype = ctypes.c_int64
            L.or_prenotch.argtypes = [ctypes.c_int, i64p, ctypes.c_double, i64p, ctypes.c_int64, dp]
            L.or_prenotch.restype = ctypes.c_int64
            L.or_vv.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
                                dp, dp, ctypes.c_double, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int, dp, dp]
            L.or_vv.restype = ctypes.c_int64
            L.or_grad_modulus.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          dp, dp, dp, dp, dp]
            L.or_grad_modulus.restype = ctypes.c_int
            L.or_surface_nu.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, dp]
            L.or_surface_nu.restype = ctypes.c_int
            L.or_row_abs_max.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         dp, dp]
            L.or_row_abs_max.restype = ctypes.c_int
            L.or_threads.argtypes = []
            L.or_threads.restype = ctypes.c_int
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_set_threads.restype = None
            _lib = L
    return _lib


# --------------------------------------------------------------------------- helpers

def threads() -> int:
    """OpenMP threads the oracle's node loops use."""
    return int(lib().or_threads())


def set_threads(n: int) -> None:
    """Sets the OpenMP threads of the oracle's node loops (timing on one core)."""
    lib().or_set_threads(int(n))


def _n64(n):
    arr = (ctypes.c_int64 * 3)(*(list(int(v) for v in n) + [1] * (3 - len(n))))
    return arr


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


def radius(M) -> int:
    """Integer radius of the offset disk for m = delta / h (= m when m is an integer)."""
    return int(math.ceil(float(M) - 1e-9))


def offsets(dim: int, M) -> np.ndarray:
    """Neighbour offsets o != 0 with |o| <= m = M (Eq. band; M = delta / h, any real >= 1),
    int32 [nnb][3]."""
    buf = np.zeros((16384, 3), dtype=np.int32)
    cnt = lib().or_offsets(dim, M, _ptr(buf), 16384)
    assert cnt > 0
    return buf[:cnt].copy()


def lam(r: float, delta: float, dx: float) -> float:
    """Partial-volume factor of Eq. fac:e1."""
    return lib().or_lambda(r, delta, dx)


def alpha(dim: int, E: float, delta: float, thickness: float = 1.0) -> float:
    """Micromodulus constant of Sec. 2.1."""
    return lib().or_alpha(dim, E, delta, thickness)


def bond_constant(dim: int, E: float, delta: float, thickness: float = 1.0) -> float:
    """alpha times V_q / h^dim, the constant the force routines take as alpha_:
    the node volume of Eq. mat:f1 is h^2 t for a 2D plate of thickness t
    (alpha t in 2D, alpha in 3D; equal to alpha at unit thickness)."""
    return lib().or_bond_constant(dim, E, delta, thickness)


def bond_block(dim: int, o, h: float, M: int, alpha_: float) -> np.ndarray:
    out = np.zeros(9)
    oo = np.array(list(o) + [0] * (3 - len(o)), dtype=np.int32)
    lib().or_bond_block(dim, _ptr(oo), h, M, alpha_, _ptr(out))
    return out.reshape(3, 3)[:dim, :dim]


def force(dim, n, h, M, alpha_, u, E=None, mu=None, nu=None) -> np.ndarray:
    """f = A(mu) u by direct summation (Eq. mat:f1).  u: [dim][...] float64.
    nu: surface-correction factors (``surface_nu``) or None."""
    u = _f64(u)
    f = np.empty_like(u)
    rc = lib().or_force(dim, _n64(n), h, M, alpha_, _ptr(_f64(E)), _ptr(_u8(mu)), _ptr(_f64(nu)), _ptr(u), _ptr(f))
    assert rc > 0
    return f


def stiffness(dim, n, h, M, alpha_, u, cons=None, E=None, mu=None, nu=None) -> np.ndarray:
    """out = P K P u with K = -A and P zeroing constrained components."""
    u = _f64(u)
    out = np.empty_like(u)
    rc = lib().or_stiffness(dim, _n64(n), h, M, alpha_, _ptr(_f64(E)), _ptr(_u8(mu)), _ptr(_f64(nu)), _ptr(_u8(cons)),
                            _ptr(u), _ptr(out))
    assert rc > 0
    return out


def cg(dim, n, h, M, alpha_, b, cons=None, E=None, mu=None, x0=None, rtol=1e-8, maxit=100000, nu=None):
    """Textbook CG on P K P x = P b.  Returns (x, iterations, true relative residual)."""
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    rel = ctypes.c_double(0.0)
    it = lib().or_cg(dim, _n64(n), h, M, alpha_, _ptr(_f64(E)), _ptr(_u8(mu)), _ptr(_f64(nu)), _ptr(_u8(cons)),
                     _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(rel))
    assert it >= 0
    return x, it, rel.value


def adr_density(dim: int, h: float, M: int, alpha_: float) -> np.ndarray:
    """Fictitious diagonal density of the ADR method (Sec. 2.3, after Kilic and
    Madenci): D_i = 1/4 dt^2 sum_j |K_ij| with dt = 1, the Gershgorin bound that
    keeps the central-difference scheme stable.  The interior row has the
    largest sum, so one value per component serves every node.  Returns [dim]."""
    T = kernel_table(dim, h, M, alpha_)
    return np.array([0.25 * np.abs(T[a]).sum() for a in range(dim)])


def adr(matvec, b, D, rtol=1e-8, maxit=100000, u0=None, dt=1.0, record=None):
    """Adaptive dynamic relaxation with the central-difference explicit
    integration of Algorithm 1 (CDEI) for the static problem K u = b.

    matvec(u) = P K P u; b is projected by the caller; D: fictitious density per
    component.  f^n = -matvec(u^n) is the internal force, so f^n + b is the
    residual.  The paper leaves the damping to its reference [KM]: c^n =
    2 sqrt(u^T K1 u / u^T u) with the diagonal local stiffness
    K1_ii = -(f_i^n - f_i^(n-1)) / (D_i dt v_i^(n-1/2)) (0 where v_i = 0), and
    c^n = 0 when the quotient is not positive.  Stops when the relative residual
    |f^n + b| / |b| <= rtol, checked at u^n before the update.
    Returns (u, iterations, relative residual); record (a list) receives c^n."""
    Dn = np.asarray(D, dtype=np.float64).reshape((-1,) + (1,) * (np.ndim(b) - 1))
    b = np.asarray(b, dtype=np.float64)
    u = np.zeros_like(b) if u0 is None else np.array(u0, dtype=np.float64)
    bn = np.linalg.norm(b)
    bn = bn if bn > 0 else 1.0
    f = -matvec(u)
    rel = np.linalg.norm(f + b) / bn
    if rel <= rtol:
        return u, 0, rel
    v = dt * (f + b) / Dn / 2.0           # first half step of Algorithm 1
    u = u + dt * v
    f_old = f
    it = 1
    while it < maxit:
        f = -matvec(u)
        rel = np.linalg.norm(f + b) / bn
        if rel <= rtol:
            break
        with np.errstate(divide="ignore", invalid="ignore"):
            k1 = np.where(v != 0.0, -(f - f_old) / (Dn * dt * v), 0.0)
        num = float(np.sum(u * k1 * u))
        den = float(np.sum(u * u))
        c = 2.0 * math.sqrt(num / den) if (num > 0.0 and den > 0.0) else 0.0
        if record is not None:
            record.append(c)
        v = ((2.0 - c * dt) * v + 2.0 * dt * (f + b) / Dn) / (2.0 + c * dt)
        u = u + dt * v
        f_old = f
        it += 1
    return u, it, rel


def adr_solve(dim, n, h, M, alpha_, b, cons=None, mu=None, rtol=1e-8, maxit=100000, u0=None, record=None,
              nu=None):
    """ADR (Algorithm 1) on P K P u = P b with the oracle's direct-sum operator.
    With surface-correction factors nu the density is 1/4 of the largest
    absolute row sum over all rows (edge rows can exceed the interior one)."""
    b = _f64(b)
    P = 1.0 if cons is None else (1 - np.asarray(cons, dtype=np.float64))
    mv = lambda x: stiffness(dim, n, h, M, alpha_, x, cons=cons, mu=mu, nu=nu)
    D = adr_density(dim, h, M, alpha_) if nu is None else 0.25 * row_abs_max(dim, n, h, M, alpha_, nu)
    return adr(mv, b * P, D, rtol=rtol, maxit=maxit, u0=u0, record=record)


def surface_nu(dim, n, h, M) -> np.ndarray:
    """Surface-correction factor per node (volume method, the reading of the
    remark on Omega_e in Sec. 3.3): nu_p = V_full / V_p, shape node_shape(n)."""
    nu = np.empty(int(np.prod(n)), dtype=np.float64)
    assert lib().or_surface_nu(dim, _n64(n), h, M, _ptr(nu)) > 0
    return nu.reshape(tuple(reversed([int(v) for v in n])))


def row_abs_max(dim, n, h, M, alpha_, nu=None) -> np.ndarray:
    """Largest absolute row sum of K per component (bonds intact, no projection)."""
    out = np.zeros(3)
    assert lib().or_row_abs_max(dim, _n64(n), h, M, alpha_, _ptr(_f64(nu)), _ptr(out)) > 0
    return out[:dim]


def critical_stretch(G0: float, E: float, delta: float, plane: str = "stress") -> float:
    """Critical bond stretch of Eq. fra:s1 from the energy release rate G0."""
    if plane == "stress":
        return math.sqrt(4.0 * math.pi * G0 / (9.0 * E * delta))
    return math.sqrt(5.0 * math.pi * G0 / (12.0 * E * delta))


def intact_mu(dim, n, M) -> np.ndarray:
    """All-intact bond state, uint8 [N][nnb]."""
    return np.ones((int(np.prod(n)), len(offsets(dim, M))), dtype=np.uint8)


def break_bonds(dim, n, h, M, s0, u, mu) -> int:
    """Break every intact bond with stretch >= s0 (in place on mu); returns the count."""
    assert mu.dtype == np.uint8 and mu.flags.c_contiguous
    return int(lib().or_break(dim, _n64(n), h, M, s0, _ptr(_f64(u)), _ptr(mu)))


def prenotch(n, M, seg, den, mu, dim=2) -> int:
    """Break the bonds meeting the closed segment seg/den (units of h from the corner);
    in 3D the segment is extruded through z and bonds are tested by their x-y projection."""
    assert mu.dtype == np.uint8 and mu.flags.c_contiguous
    s = (ctypes.c_int64 * 4)(*[int(v) for v in seg])
    return int(lib().or_prenotch(dim, _n64(n), M, s, int(den), _ptr(mu)))


def vv(dim, n, h, M, alpha_, u, v, nsteps, dt, rho=1.0, b=None, E=None, mu=None, s0=0.0,
       cons=None, vpres=None, nu=None) -> int:
    """Velocity-Verlet (Algorithm 2) in place on u, v (float64 contiguous); returns bonds broken."""
    assert u.dtype == np.float64 and v.dtype == np.float64
    return int(lib().or_vv(dim, _n64(n), h, M, alpha_, _ptr(_f64(E)), _ptr(mu), _ptr(_f64(nu)), s0, _ptr(_u8(cons)),
                           _ptr(_f64(vpres)), _ptr(_f64(b)), rho, dt, nsteps, _ptr(u), _ptr(v)))


def grad_modulus(dim, n, h, M, alpha1, u, lam_, mu=None, nu=None) -> np.ndarray:
    g = np.empty(int(np.prod(n)), dtype=np.float64)
    lib().or_grad_modulus(dim, _n64(n), h, M, alpha1, _ptr(_u8(mu)), _ptr(_f64(nu)), _ptr(_f64(u)),
                          _ptr(_f64(lam_)), _ptr(g))
    return g.reshape(tuple(reversed([int(v) for v in n])))


# --------------------------------------------------------------------------- numpy routes

def dense_matrix(dim: int, n, h: float, M: int, alpha_: float, E=None) -> np.ndarray:
    """Brute-force dense A (Eq. matrix in 2D, Eq. mae:e1 in 3D) from node positions.

    Rows and columns are ordered component-major (c * N + p).  Every node pair is
    tested: q is a neighbour of p when |x_q - x_p| <= delta; the diagonal block
    is minus the sum of the row's off-diagonal blocks.  Use h = 2^-k so that
    the positions and the distance test are exact in binary floating point.
    """
    n = [int(v) for v in n]
    N = int(np.prod(n))
    idx = np.indices(tuple(reversed(n))).reshape(dim, N)[::-1]  # [dim][N], x first
    X = (idx + 0.5) * h
    delta = M * h
    V = h ** dim
    A = np.zeros((dim * N, dim * N))
    for p in range(N):
        for q in range(N):
            if q == p:
                continue
            xi = X[:, q] - X[:, p]
            r = math.sqrt(float(xi @ xi))
            if r > delta:
                continue
            lq = 1.0 if r <= delta - h / 2 else (2 * delta + h - 2 * r) / (2 * h)
            coef = alpha_ * lq * V / r ** 3
            if E is not None:
                coef *= 0.5 * (E.reshape(-1)[p] + E.reshape(-1)[q])
            for a in range(dim):
                for b in range(dim):
                    A[a * N + p, b * N + q] += coef * xi[a] * xi[b]
                    A[a * N + p, b * N + p] -= coef * xi[a] * xi[b]
    return A


def kernel_table(dim: int, h: float, M: int, alpha_: float) -> np.ndarray:
    """Kernel matrix / tensor of Eqs. frb:e1, frb:e4 (2D) and thm:e2, thm:e3 (3D).

    Returns T[a][b][oz+R][oy+R][ox+R] (2D: T[a][b][oy+R][ox+R]), R = radius(M), holding
    alpha lambda h^(dim-1) o_a o_b / |o|^3 off the centre (lambda = 0 beyond
    |o| = M = delta / h) and minus the sum of all others at the centre.
    """
    R = radius(M)
    rng_ = np.arange(-R, R + 1)
    if dim == 2:
        oy, ox = np.meshgrid(rng_, rng_, indexing="ij")
        comps = [ox, oy]
    else:
        oz, oy, ox = np.meshgrid(rng_, rng_, rng_, indexing="ij")
        comps = [ox, oy, oz]
    d2 = sum(c.astype(np.float64) ** 2 for c in comps)
    r = np.sqrt(d2)
    lamv = np.where(r <= M - 0.5, 1.0, np.where(r <= M, M + 0.5 - r, 0.0))
    lamv[d2 == 0] = 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        w = np.where(d2 > 0, alpha_ * lamv * h ** (dim - 1) / np.where(d2 > 0, r ** 3, 1.0), 0.0)
    T = np.zeros((dim, dim) + d2.shape)
    centre = (R,) * dim
    for a in range(dim):
        for b in range(dim):
            T[a, b] = w * comps[a] * comps[b]
            T[a, b][centre] = -T[a, b].sum()
    return T


def fmvm(dim: int, n, h: float, M: int, alpha_: float, u, mu=None) -> np.ndarray:
    """f = A u through the paper's fast form (Algorithm 3 in 2D, Algorithm 4 in 3D).

    f = IFFT(FFT(G) o FFT(U)) cropped (the TBT / TBTBT part A^ u), then
    + D^e u on nodes whose horizon leaves the grid (Eqs. mat:se, tea:sc), then
    + sum over broken bonds of A^_pq (u_p - u_q) (Eqs. df, tea:fr).
    The circulant embedding has size 2N per axis as in the paper.
    """
    n = [int(v) for v in n]
    T = kernel_table(dim, h, M, alpha_)
    shp = tuple(reversed(n))                       # array axes (z,) y, x
    big = tuple(2 * s for s in shp)
    u = np.asarray(u, dtype=np.float64).reshape((dim,) + shp)
    # G: first column of the embedded circulant, K(o) at index o mod 2N (zero elsewhere)
    G = np.zeros((dim, dim) + big)
    R = radius(M)
    rng_ = np.arange(-R, R + 1)
    grids = np.meshgrid(*([rng_] * dim), indexing="ij")   # axes order (z,) y, x
    idx = tuple(g % s for g, s in zip(grids, big))
    for a in range(dim):
        for b in range(dim):
            G[a, b][idx] = T[a, b]
    Ghat = np.fft.fftn(G, axes=tuple(range(2, 2 + dim)))
    U = np.zeros((dim,) + big)
    U[(slice(None),) + tuple(slice(0, s) for s in shp)] = u
    Uhat = np.fft.fftn(U, axes=tuple(range(1, 1 + dim)))
    Hhat = np.einsum("ab...,b...->a...", Ghat, Uhat)
    H = np.fft.ifftn(Hhat, axes=tuple(range(1, 1 + dim))).real
    f = H[(slice(None),) + tuple(slice(0, s) for s in shp)].copy()
    # D^e: sum of kernel entries whose partner lies outside the grid
    offs = offsets(dim, M)
    N = int(np.prod(n))
    coords = np.indices(shp).reshape(dim, N)[::-1]  # x first
    for k, o in enumerate(offs):
        q = coords + o[:dim, None]
        out = np.zeros(N, dtype=bool)
        for c in range(dim):
            out |= (q[c] < 0) | (q[c] >= n[c])
        if not out.any():
            continue
        tidx = tuple(int(o[c]) + R for c in reversed(range(dim)))
        for a in range(dim):
            for b in range(dim):
                f[a].reshape(-1)[out] += T[(a, b) + tidx] * u[b].reshape(-1)[out]
    # D^f: broken bonds
    if mu is not None:
        bro = np.argwhere(mu == 0)
        for p, k in bro:
            o = offs[k]
            c = coords[:, p] + o[:dim]
            if any(c[i] < 0 or c[i] >= n[i] for i in range(dim)):
                continue
            q = int(sum(int(c[i]) * int(np.prod(n[:i])) for i in range(dim)))
            tidx = tuple(int(o[cc]) + R for cc in reversed(range(dim)))
            for a in range(dim):
                for b in range(dim):
                    f[a].reshape(-1)[p] += T[(a, b) + tidx] * (u[b].reshape(-1)[p] - u[b].reshape(-1)[q])
    return f


def symbol(dim: int, L, h: float, M: int, alpha_: float) -> np.ndarray:
    """Real symbol G^(k) = sum_o K(o) exp(-2 pi i k.o / L) of the TBT part on an L-periodic grid,
    [dim][dim][...] over the frequency grid (axes (z,) y, x)."""
    T = kernel_table(dim, h, M, alpha_)
    L = [int(v) for v in L]
    big = tuple(reversed(L))
    G = np.zeros((dim, dim) + big)
    R = radius(M)
    rng_ = np.arange(-R, R + 1)
    grids = np.meshgrid(*([rng_] * dim), indexing="ij")
    idx = tuple(g % s for g, s in zip(grids, big))
    for a in range(dim):
        for b in range(dim):
            G[a, b][idx] = T[a, b]
    return np.fft.fftn(G, axes=tuple(range(2, 2 + dim)))


def vv_history(dim, n, h, M, alpha_, u0, v0, nsteps, dt, rho=1.0, b=None, E=None, mu0=None, s0=0.0, cons=None,
               vpres=None):
    """Algorithm 2 step by step, keeping u and the bond state after every step.
    Returns (us, vs, mus): lists of length nsteps + 1 (index = step)."""
    u, v = np.array(u0, dtype=np.float64), np.array(v0, dtype=np.float64)
    mu = intact_mu(dim, n, M) if mu0 is None else mu0.copy()
    us, vs, mus = [u.copy()], [v.copy()], [mu.copy()]
    for _ in range(nsteps):
        vv(dim, n, h, M, alpha_, u, v, 1, dt, rho=rho, b=b, E=E, mu=mu, s0=s0, cons=cons, vpres=vpres)
        us.append(u.copy())
        vs.append(v.copy())
        mus.append(mu.copy())
    return us, vs, mus


def vv_grad_modulus(dim, n, h, M, alpha1, E, u0, v0, nsteps, dt, rho=1.0, b=None, mu0=None, s0=0.0, cons=None,
                    vpres=None):
    """Gradient of L = 1/2 |u_N|^2 after nsteps steps of Algorithm 2 (a = (f + b)/rho,
    bond modulus (E_p + E_q)/2, alpha1 = alpha at E = 1) with respect to E, the
    bond history held at the one the forward run produced.

    Discrete adjoint of one step n -> n+1 (free components; constrained
    components move with the prescribed velocity and do not depend on v, a):
      u_{n+1} = u_n + dt v_n + dt^2/2 a_n ;  a_{n+1} = (A_{n+1} u_{n+1} + b)/rho ;
      v_{n+1} = v_n + dt/2 (a_n + a_{n+1}).
    Returns (u_N, dL/dE)."""
    us, vs, mus = vv_history(dim, n, h, M, alpha1, u0, v0, nsteps, dt, rho, b, E, mu0, s0, cons, vpres)
    free = np.ones_like(us[0]) if cons is None else (1.0 - np.asarray(cons, dtype=np.float64))
    ub = us[-1].copy()                      # dL/du_N
    vb = np.zeros_like(ub)
    ab = np.zeros_like(ub)
    gE = np.zeros(tuple(reversed([int(v) for v in n])))
    for s in reversed(range(nsteps)):
        # velocity update
        ab = (ab + 0.5 * dt * vb) * free
        ab_prev = 0.5 * dt * vb * free
        vb = vb * free
        # acceleration from the displacement at step s+1 (bond state of step s+1)
        ub = ub + force(dim, n, h, M, alpha1, ab, E=E, mu=mus[s + 1]) / rho
        gE = gE + grad_modulus(dim, n, h, M, alpha1, us[s + 1], ab, mu=mus[s + 1]) / rho
        # displacement update
        vb = vb + dt * ub * free
        ab = ab_prev + 0.5 * dt * dt * ub * free
    ab = ab * free
    ub = ub + force(dim, n, h, M, alpha1, ab, E=E, mu=mus[0]) / rho
    gE = gE + grad_modulus(dim, n, h, M, alpha1, us[0], ab, mu=mus[0]) / rho
    return us[-1], gE

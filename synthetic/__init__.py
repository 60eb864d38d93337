"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle.

This module holds no arithmetic of the peridynamic method: it only draws random
fields (numpy PCG64, fixed seeds) and builds the problem geometry (which nodes
are clamped, where the load acts, where the pre-notch lies) for the workloads
modelled on the paper's examples (Sec. 5.1-5.4).

Layout of every per-node array: ``[dim][Nz][Ny][Nx]`` (2D: ``[dim][Ny][Nx]``),
x fastest, which is the node numbering p = i + Nx*(j + Ny*k) of Sec. 3 and
Sec. 4 with 0-based indices.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

SEED_BASE = 2301_11828


def rng(tag: int) -> np.random.Generator:
    """Deterministic PCG64 generator for a given integer tag."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(tag)))


def node_shape(n: Tuple[int, ...]) -> Tuple[int, ...]:
    """Array shape of one component: reversed grid extents (x fastest)."""
    return tuple(int(v) for v in reversed(n))


def uniform_field(dim: int, n, lo: float, hi: float, tag: int) -> np.ndarray:
    """u ~ U[lo, hi] independently per component and node, float64 [dim][...]."""
    return rng(tag).uniform(lo, hi, size=(dim,) + node_shape(n))


def gaussian_field(dim: int, n, sigma: float, tag: int) -> np.ndarray:
    """b ~ N(0, sigma^2) independently per component and node, float64 [dim][...]."""
    return rng(tag).normal(0.0, sigma, size=(dim,) + node_shape(n))


def lognormal_modulus(n, sigma: float, tag: int, E0: float = 1.0) -> np.ndarray:
    """Per-node Young's modulus E_p = E0 * exp(sigma * z_p), z ~ N(0, 1), float64 [...]."""
    return E0 * np.exp(sigma * rng(tag).normal(0.0, 1.0, size=node_shape(n)))


def clamp_left(dim: int, n, M: int) -> np.ndarray:
    """Dirichlet volume layer of width delta on the x = 0 face.

    Node i is clamped (all components) when its centre (i + 1/2) h < delta = M h,
    i.e. i <= M - 1.  Returns uint8 [dim][...] (1 = constrained component).
    """
    mask = np.zeros((dim,) + node_shape(n), dtype=np.uint8)
    mask[..., :M] = 1
    return mask


def clamp_bottom_3d(n, M: int) -> np.ndarray:
    """3D: layers with z centre below delta (k <= M - 1) clamped in all components."""
    mask = np.zeros((3,) + node_shape(n), dtype=np.uint8)
    mask[:, :M, :, :] = 1
    return mask


def traction_right(dim: int, n, M: int, value: float) -> np.ndarray:
    """Body force density b_x = value on the strip x > L - delta (i >= Nx - M), else 0."""
    b = np.zeros((dim,) + node_shape(n), dtype=np.float64)
    b[0, ..., n[0] - M:] = value
    return b


def velocity_layers_2d(n, M: int) -> np.ndarray:
    """Top and bottom layers of depth delta (M rows each), constrained in y only.

    Returns int8 [Ny][Nx]: +1 on the top layer (j >= Ny - M), -1 on the bottom
    layer (j <= M - 1), 0 elsewhere; the sign gives the direction of the
    prescribed y-velocity.
    """
    nx, ny = int(n[0]), int(n[1])
    s = np.zeros((ny, nx), dtype=np.int8)
    s[:M, :] = -1
    s[ny - M:, :] = 1
    return s


@dataclass
class Workload:
    """One synthetic problem: grid, horizon, material and seeded fields."""
    name: str
    dim: int
    n: Tuple[int, ...]
    M: int
    E: float = 1.0
    thickness: float = 1.0
    rho: float = 1.0
    s0: float = 0.0
    h: float = 0.0
    constrained: Optional[np.ndarray] = None
    b: Optional[np.ndarray] = None
    u: Optional[np.ndarray] = None
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    @property
    def delta(self) -> float:
        return self.M * self.h


def plate_static(nside: int, M: int, tag: int, u_amp: float, traction: float = 1e-3) -> Workload:
    """Square plate, h = 1/nside, clamp on the left, x-traction strip on the right."""
    n = (nside, nside)
    return Workload(
        name=f"plate2d_{nside}x{nside}_M{M}", dim=2, n=n, M=M, h=1.0 / nside,
        constrained=clamp_left(2, n, M), b=traction_right(2, n, M, traction),
        u=uniform_field(2, n, -u_amp, u_amp, tag))


def small_plate() -> Workload:
    """64 x 64 plate, delta = 3h, E = 1, FP64 matvec and CG (the small, oracle-fast case)."""
    return plate_static(64, 3, tag=1, u_amp=1e-3)


def large_plate(M: int = 3) -> Workload:
    """1024 x 1024 plate, delta = M h, u ~ U[-1, 1] (the throughput case)."""
    return plate_static(1024, M, tag=2 + 100 * M, u_amp=1.0)


def cube(nside: int = 128, M: int = 3, tag: int = 3) -> Workload:
    """Cube nside^3, h = 1/nside, clamped bottom face, Gaussian body force sigma = 1e-3."""
    n = (nside, nside, nside)
    return Workload(
        name=f"cube3d_{nside}^3_M{M}", dim=3, n=n, M=M, h=1.0 / nside,
        constrained=clamp_bottom_3d(n, M), b=gaussian_field(3, n, 1e-3, tag),
        u=uniform_field(3, n, -1.0, 1.0, tag + 1000))


def crack_plate(nside: int = 512, M: int = 3, tag: int = 4) -> Workload:
    """Pre-notched plate under tensile edge velocity, lognormal modulus (sigma = 0.1).

    The notch is the closed segment y = L/2, |x - L/2| <= 0.1 L, given in
    ``extra['notch']`` as integer numerators over ``extra['notch_den']`` in units
    of h measured from the grid corner (node i sits at i + 1/2).
    ``extra['v_ramp']`` is an initial y-velocity field that matches the edge
    layers (v0 (2 y / L - 1) at node height y): started from it, the plate
    stretches at a uniform rate instead of being struck at its edges.
    """
    n = (nside, nside)
    den = 10
    # endpoints: x = L/2 -+ 0.1 L = nside*(0.5 -+ 0.1) h, y = nside/2 h
    notch = (nside * 4, nside * 5, nside * 6, nside * 5)  # over den: (0.4N, 0.5N)-(0.6N, 0.5N)
    return Workload(
        name=f"crack2d_{nside}x{nside}_M{M}", dim=2, n=n, M=M, h=1.0 / nside,
        s0=1e-3, rho=1.0,
        extra=dict(E_field=lognormal_modulus(n, 0.1, tag), notch=notch, notch_den=den,
                   vel_layers=velocity_layers_2d(n, M), v0=1e-3,
                   v_ramp=np.stack([np.zeros((nside, nside)),
                                    np.repeat((1e-3 * (2.0 * (np.arange(nside) + 0.5) / nside - 1.0))[:, None],
                                              nside, axis=1)])))


def kw_block(nx: int = 201, ny: int = 101, nz: int = 9, M: int = 3, v0: float = 0.00634) -> Workload:
    """Kalthoff-Winkler-like block (the geometry of Sec. 5.4, without the impactor).

    Length along x, width along y, thickness along z (the paper's 0.2 x 0.1 x
    0.009 block is 201 x 101 x 9 nodes, and 402 x 202 x 18 at half the
    spacing); h = 1/nx, E = rho = 1, critical stretch s0 = 0.01 as in the paper.
    Two through-thickness notches at x = 3/8 and 5/8 of the length run from the
    y = 0 face to half the width (length a0 = W/2, distance d = L/4, as in the
    paper); they are given in ``extra['notches']`` as segments over
    ``extra['notch_den']`` in units of h from the grid corner.  Instead of the
    impactor, the first M node layers of the y = 0 face between the notches
    (node centres strictly between them) move with the prescribed velocity
    v_y = v0: ``constrained`` marks their y component and ``extra['v_prescribed']``
    holds the velocity field.  Time step and impact speed are the paper's in
    units of the spacing and of the bar wave speed c0 = sqrt(E / rho) (its
    steel: E = 2e11 Pa, rho = 7850 kg/m^3, c0 = 5048 m/s, spacing 0.001 m):
    dt = 1.3367e-8 s -> 0.06747 h / c0 and v0 = 32 m/s -> 0.00634 c0, so the
    paper's 1350 steps cover the same 0.46 wave transits of the length.  That
    step is far below the stable one, 2 h sqrt(rho / (E Lambda_1)) with
    Lambda_1 <= 1.2185 the largest eigenvalue of the unit (h = 1) symbol
    (``extra['dt_stable']``).
    """
    n = (nx, ny, nz)
    den = 8
    notches = [(3 * nx, 0, 3 * nx, 4 * ny), (5 * nx, 0, 5 * nx, 4 * ny)]
    i = np.arange(nx)
    zone = (den * (2 * i + 1) > 2 * 3 * nx) & (den * (2 * i + 1) < 2 * 5 * nx)   # 3nx/8 < i + 1/2 < 5nx/8
    cons = np.zeros((3,) + node_shape(n), dtype=np.uint8)
    vp = np.zeros((3,) + node_shape(n))
    for j in range(min(M, ny)):
        cons[1, :, j, zone] = 1
        vp[1, :, j, zone] = v0
    h = 1.0 / nx
    return Workload(name=f"kw3d_{nx}x{ny}x{nz}_M{M}", dim=3, n=n, M=M, h=h, s0=0.01, rho=1.0,
                    constrained=cons,
                    extra=dict(notches=notches, notch_den=den, v_prescribed=vp, v0=v0, dt=0.06747 * h,
                               dt_stable=2.0 * h / np.sqrt(1.2185)))


def batched_plates(count: int = 64, tag: int = 5):
    """Uneven batch: sides n_i ~ U{128..512}, M_i in {3, 4} (p = 1/2), clamp left,
    body force N(0, (1e-3)^2) on free components."""
    g = rng(tag)
    sides = g.integers(128, 513, size=count)
    Ms = np.where(g.random(count) < 0.5, 3, 4)
    out = []
    for i, (s, m) in enumerate(zip(sides, Ms)):
        n = (int(s), int(s))
        cons = clamp_left(2, n, int(m))
        b = gaussian_field(2, n, 1e-3, tag * 1000 + i) * (1 - cons)
        out.append(Workload(name=f"plate{i}_{s}_M{m}", dim=2, n=n, M=int(m), h=1.0 / s,
                            constrained=cons, b=b))
    return out

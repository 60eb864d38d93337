"""cuFFT comparison baseline for the FFT route of the product (Algorithm 3 in
2D, Algorithm 4 in 3D): K u with library FFTs (cuFFT through torch.fft) and a
whole-grid circulant embedding.  Comparison only: nothing in the library calls
it, and the product the library computes never goes through it.

The TBT part is the correlation of u (zero outside the grid) with the kernel
table K(o) (the bond blocks of Eq. mat:f1, read back from the grid with
pd_get_coefficients); K(o) = K(-o), so it is a convolution, and embedding both
in a periodic grid of extent L_i >= n_i + M per axis makes the circular
convolution equal the linear one on the grid (no wrap-around reaches a node).
The edge self-term of Eq. tea:sc enters as the diagonal block
Kd_p = sum of K(o) over the in-grid neighbours, itself the convolution of K with
the grid's indicator (computed once).  Then K u = Kd u - conv(K, u).
"""
from __future__ import annotations

import numpy as np

from . import pd_get_coefficients, pd_get_info, pd_get_offsets


def _smooth_size(n: int) -> int:
    """Smallest 2^a 3^b 5^c 7^d >= n (sizes cuFFT transforms fastest)."""
    m = n
    while True:
        k = m
        for p in (2, 3, 5, 7):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        m += 1


class CufftProduct:
    """K u on a grid by cuFFT; `dtype` torch.float32 or torch.float64."""

    def __init__(self, grid, dtype, device="cuda"):
        import torch
        info = pd_get_info(grid.handle)
        self.dim = info.dim
        self.n = tuple(int(info.n[i]) for i in range(self.dim))   # (nx, ny[, nz])
        self.M = int(info.M)
        self.dtype = dtype
        self.L = tuple(_smooth_size(v + self.M) for v in self.n)
        off = pd_get_offsets(grid.handle)
        coef = pd_get_coefficients(grid.handle)
        nc = coef.shape[1]
        shape = tuple(reversed(self.L))   # arrays are [z][y][x]
        G = np.zeros((nc,) + shape)
        for k in range(off.shape[0]):
            ox, oy, oz = (int(v) for v in off[k])   # rows (ox, oy, oz)
            idx = (ox % self.L[0], oy % self.L[1]) if self.dim == 2 else (ox % self.L[0], oy % self.L[1],
                                                                           oz % self.L[2])
            G[(slice(None),) + tuple(reversed(idx))] += coef[k]
        dims = tuple(range(-self.dim, 0))
        self.dims = dims
        Gt = torch.tensor(G, dtype=dtype, device=device)
        self.S = torch.fft.rfftn(Gt, dim=dims).real.contiguous()   # real: the table is even
        # the symmetric blocks (ab) -> index into S
        if self.dim == 2:
            self.blk = [[0, 1], [1, 2]]
        else:
            self.blk = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]
        ones = torch.zeros((1,) + shape, dtype=dtype, device=device)
        sl = tuple(slice(0, v) for v in reversed(self.n))
        ones[(slice(None),) + sl] = 1.0
        F1 = torch.fft.rfftn(ones, dim=dims)
        kd = torch.fft.irfftn(self.S * F1, s=shape, dim=dims)
        self.Kd = kd[(slice(None),) + sl].contiguous()   # [nc][n...]: sum of K(o) over in-grid o

    def __call__(self, u):
        """u: [..., dim, (nz,) ny, nx] tensor of the grid's dtype; returns K u."""
        import torch
        d = self.dim
        shape = tuple(reversed(self.L))
        U = torch.fft.rfftn(u, s=shape, dim=self.dims)
        H = torch.empty_like(U)
        for a in range(d):
            acc = self.S[self.blk[a][0]] * U[..., 0, *([slice(None)] * d)]
            for b in range(1, d):
                acc = acc + self.S[self.blk[a][b]] * U[..., b, *([slice(None)] * d)]
            H[..., a, *([slice(None)] * d)] = acc
        h = torch.fft.irfftn(H, s=shape, dim=self.dims)
        sl = tuple(slice(0, v) for v in reversed(self.n))
        h = h[(Ellipsis,) + sl]
        out = torch.empty_like(u)
        for a in range(d):
            acc = self.Kd[self.blk[a][0]] * u[..., 0, *([slice(None)] * d)]
            for b in range(1, d):
                acc = acc + self.Kd[self.blk[a][b]] * u[..., b, *([slice(None)] * d)]
            out[..., a, *([slice(None)] * d)] = acc - h[..., a, *([slice(None)] * d)]
        return out

"""Row-slab split of a grid across processes (one GPU each; rows along y in 2D,
planes along z in 3D), with an M-row halo exchange before every product.

The block-banded-block structure of the 2D operator (Sec. 3.1, Eq. band: the
blocks of K vanish between node rows more than M apart) means that K u on a
band of rows needs u on that band and on M rows on either side.  Rank r owns
grid rows [row0_r, row0_r + rows_r); before each product it sends its first
and last M rows to its neighbours, receives theirs, and calls pd_matvec_rows on
the extended band.  Band boundaries lie on multiples of 32 rows (the stencil
tile height), so each rank computes every one of its outputs exactly as the
whole-grid product does: the slabs of a split reassemble to the one-grid
product bit for bit.

Collectives are point-to-point sends and receives of torch.distributed (NCCL
for device tensors, gloo for host tensors); nothing else is exchanged.
"""
from __future__ import annotations

from typing import List, Tuple


def partition(ny: int, world: int, align: int = 32) -> List[Tuple[int, int]]:
    """Rows (row0, rows) of each rank: bands of whole 32-row tiles, as even as
    possible, the last band taking the remainder of the grid."""
    if world < 1:
        raise ValueError("world must be >= 1")
    tiles = (ny + align - 1) // align
    if tiles < world:
        raise ValueError(f"{ny} rows make {tiles} tiles of {align}: too few for {world} ranks")
    out, t0 = [], 0
    for r in range(world):
        nt = tiles // world + (1 if r < tiles % world else 0)
        row0 = t0 * align
        row1 = min(ny, (t0 + nt) * align)
        out.append((row0, row1 - row0))
        t0 += nt
    return out


def halo_window(row0: int, rows: int, ny: int, M: int) -> Tuple[int, int]:
    """Rows (ext_row0, ext_rows) of the extended band: the owned rows and M
    rows on either side, clipped to the grid."""
    lo = max(0, row0 - M)
    hi = min(ny, row0 + rows + M)
    return lo, hi - lo


def exchange_halo(u_own, rank: int, parts, M: int, dist, group=None, axis: int = -2):
    """The extended band of this rank: u_own [..., dim, rows, nx] (2D, axis -2)
    or [..., dim, planes, ny, nx] (3D, axis -3) of the owned rows, with M rows
    of each neighbour on either side (received from them; the first and last M
    owned rows are sent to them).  Works on device tensors (NCCL) and host
    tensors (gloo)."""
    import torch
    if axis != -2:
        u_t = u_own.movedim(axis, -2)
        e, lo, ext = exchange_halo(u_t.contiguous(), rank, parts, M, dist, group, -2)
        return e.movedim(-2, axis).contiguous(), lo, ext
    world = len(parts)
    row0, rows = parts[rank]
    ny = parts[-1][0] + parts[-1][1]
    lo, ext = halo_window(row0, rows, ny, M)
    top = row0 - lo                       # halo rows above (from rank - 1)
    bot = lo + ext - (row0 + rows)        # halo rows below (from rank + 1)
    shape = list(u_own.shape)
    shape[-2] = ext
    u_ext = torch.empty(shape, dtype=u_own.dtype, device=u_own.device)
    u_ext[..., top:top + rows, :] = u_own
    ops = []
    if rank > 0 and top > 0:
        ops.append(dist.P2POp(dist.isend, u_own[..., :top, :].contiguous(), rank - 1, group))
        recv_top = torch.empty_like(u_ext[..., :top, :])
        ops.append(dist.P2POp(dist.irecv, recv_top, rank - 1, group))
    if rank < world - 1 and bot > 0:
        ops.append(dist.P2POp(dist.isend, u_own[..., rows - bot:, :].contiguous(), rank + 1, group))
        recv_bot = torch.empty_like(u_ext[..., top + rows:, :])
        ops.append(dist.P2POp(dist.irecv, recv_bot, rank + 1, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    if rank > 0 and top > 0:
        u_ext[..., :top, :] = recv_top
    if rank < world - 1 and bot > 0:
        u_ext[..., top + rows:, :] = recv_bot
    return u_ext, lo, ext


class SlabProduct:
    """K u for this rank's band of rows of a grid split across ranks.

    grid: the whole grid (every rank creates it with the same geometry and
    constraints); u_own: [batch, dim, rows, ...] device tensor of the owned rows
    (rows along y in 2D, planes along z in 3D)."""

    def __init__(self, grid, rank: int, world: int, dist, group=None):
        from . import pd_get_info
        info = pd_get_info(grid.handle)
        self.dim = int(info.dim)
        self.grid, self.rank, self.world, self.dist, self.group = grid, rank, world, dist, group
        self.M = int(info.M)
        self.n_slow = int(info.n[self.dim - 1])
        self.parts = partition(self.n_slow, world, align=32 if self.dim == 2 else 1)
        self.row0, self.rows = self.parts[rank]

    def __call__(self, u_own, flags: int = 0):
        import torch
        from . import PD_F32, PD_F64, pd_matvec_rows
        batched = u_own.dim() == self.dim + 2
        u4 = u_own if batched else u_own[None]
        axis = -2 if self.dim == 2 else -3
        u_ext, lo, ext = exchange_halo(u4, self.rank, self.parts, self.M, self.dist, self.group, axis)
        out = torch.empty_like(u4)
        fl = flags | (PD_F64 if u4.dtype == torch.float64 else PD_F32)
        pd_matvec_rows(self.grid.handle, u4.shape[0], self.row0, self.rows, u_ext.contiguous(), lo, ext, out, fl)
        return out if batched else out[0]

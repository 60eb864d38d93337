"""The row-slab split of a 2D grid (paper_2301_11828_gb300.slab) on CPU with
gloo ranks: the partition, the M-row halo exchange, and -- with the oracle's
product standing in for each rank's kernel -- that the slabs' products
reassemble to the whole-grid product bit for bit (the band structure of
Sec. 3.1 couples only rows within M of each other)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")


def test_partition_and_windows():
    from paper_2301_11828_gb300.slab import halo_window, partition
    for ny, world in ((1024, 2), (1024, 3), (100, 2), (96, 3), (64, 1)):
        parts = partition(ny, world)
        assert len(parts) == world
        assert parts[0][0] == 0 and parts[-1][0] + parts[-1][1] == ny
        for (r0, n0), (r1, _) in zip(parts, parts[1:]):
            assert r0 + n0 == r1 and r1 % 32 == 0
        assert all(n > 0 for _, n in parts)
    assert halo_window(0, 512, 1024, 3) == (0, 515)
    assert halo_window(512, 512, 1024, 3) == (509, 515)
    assert halo_window(32, 32, 96, 6) == (26, 44)
    with pytest.raises(ValueError):
        partition(40, 3)


def _slab_worker(rank, world, port, n, M, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import oracle
    import synthetic as syn
    from paper_2301_11828_gb300.slab import exchange_halo, partition
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny = n
        h = 1.0 / nx
        rng = np.random.default_rng(11)                 # the same global field on every rank
        u = rng.uniform(-1, 1, (2, 2, ny, nx))          # a batch of two fields
        cons = syn.clamp_left(2, n, M)
        parts = partition(ny, world)
        row0, rows = parts[rank]
        u_own = torch.tensor(u[:, :, row0:row0 + rows, :])
        u_ext, lo, ext = exchange_halo(u_own, rank, parts, M, dist)
        halo_ok = bool(np.array_equal(u_ext.numpy(), u[:, :, lo:lo + ext, :]))
        # each rank's kernel, stood in for by the oracle on its extended band
        al = oracle.alpha(2, 1.0, M * h)
        outs = []
        for proj in (False, True):
            o = np.stack([oracle.stiffness(2, (nx, ext), h, M, al, u_ext[b].numpy(),
                                           cons=cons[:, lo:lo + ext, :] if proj else None) for b in range(2)])
            outs.append(o[:, :, row0 - lo:row0 - lo + rows, :])
        out_q.put((rank, row0, rows, halo_ok, outs))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,M", [(2, (40, 70), 3), (3, (33, 96), 6)])
def test_slab_split_matches_whole_grid_bit_for_bit(world, n, M):
    import socket
    import oracle
    import synthetic as syn
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, n, M, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nx, ny = n
    h = 1.0 / nx
    rng = np.random.default_rng(11)
    u = rng.uniform(-1, 1, (2, 2, ny, nx))
    cons = syn.clamp_left(2, n, M)
    al = oracle.alpha(2, 1.0, M * h)
    for k, proj in enumerate((False, True)):
        whole = np.stack([oracle.stiffness(2, n, h, M, al, u[b], cons=cons if proj else None) for b in range(2)])
        got = np.concatenate([r[4][k] for r in res], axis=2)
        assert all(r[3] for r in res)                       # halos arrived intact
        assert np.array_equal(got, whole)                   # bit for bit

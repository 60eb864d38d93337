"""pd_matvec_rows, the per-rank product of the row-slab split, on one GPU: the
bands of a split (each computed from its rows plus an M-row halo, as a rank
would after the halo exchange) reassemble to the whole-grid pd_matvec bit for
bit, in every stencil path and precision, with and without projection."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pd():
    import paper_2301_11828_gb300 as pd
    pd.load_library()
    return pd


@pytest.mark.parametrize("n,M,world", [((256, 200), 3, 2), ((128, 256), 6, 3), ((132, 97), 4, 3), ((64, 64), 2.5, 2)])
def test_slabs_reassemble_the_product_bit_for_bit(pd, n, M, world):
    from paper_2301_11828_gb300.slab import halo_window, partition
    nx, ny = n
    rng = np.random.default_rng(int(10 * M) + nx)
    cons = syn.clamp_left(2, n, int(np.ceil(M)))
    g = pd.Grid(2, n, 1.0 / nx, M, constrained=cons)
    parts = partition(ny, world)
    for dt in (torch.float32, torch.float64):
        U = torch.tensor(rng.uniform(-1, 1, (2, 2, ny, nx)), dtype=dt, device="cuda")
        for extra in ((0, pd.PD_NO_TMA) if dt == torch.float32 else (0,)):
            for proj in (0, pd.PD_PROJECT):
                fl = pd.PD_METHOD_STENCIL | extra | proj
                whole = g.matvec(U, flags=fl)
                pieces = []
                for row0, rows in parts:
                    lo, ext = halo_window(row0, rows, ny, g.M)
                    u_ext = U[:, :, lo:lo + ext, :].contiguous()
                    out = torch.empty((2, 2, rows, nx), dtype=dt, device="cuda")
                    pd.pd_matvec_rows(g.handle, 2, row0, rows, u_ext, lo, ext, out,
                                      fl | (pd.PD_F32 if dt == torch.float32 else pd.PD_F64))
                    pieces.append(out)
                torch.cuda.synchronize()
                assert torch.equal(torch.cat(pieces, dim=2), whole), (str(dt), extra, proj)


def test_rows_argument_checks(pd):
    g = pd.Grid(2, (64, 96), 1.0 / 64, 3)
    U = torch.zeros((1, 2, 96, 64), dtype=torch.float32, device="cuda")
    out = torch.empty((1, 2, 32, 64), dtype=torch.float32, device="cuda")
    cases = [
        (16, 32, U[:, :, 13:51], 13, 38),    # row0 not a multiple of 32
        (32, 32, U[:, :, 30:67], 30, 37),    # halo short by one row above (needs row 29)
        (32, 32, U[:, :, 29:66], 29, 37),    # halo short by one row below (needs row 66)
    ]
    for row0, rows, ue, lo, ext in cases:
        with pytest.raises(pd.PDError) as e:
            pd.pd_matvec_rows(g.handle, 1, row0, rows, ue.contiguous(), lo, ext, out, pd.PD_F32)
        assert e.value.code == pd.PD_ERR_INVALID
    with pytest.raises(pd.PDError):
        pd.pd_matvec_rows(g.handle, 1, 32, 32, U[:, :, 29:67].contiguous(), 29, 38, out,
                          pd.PD_F32 | pd.PD_METHOD_FFT)
    pd.pd_matvec_rows(g.handle, 1, 32, 32, U[:, :, 29:67].contiguous(), 29, 38, out, pd.PD_F32)   # valid


@pytest.mark.parametrize("n,M", [((40, 33, 70), 3), ((24, 20, 50), 2.5)])
def test_plane_slabs_3d_reassemble_the_product_bit_for_bit(pd, n, M):
    """The 3D split along z: any plane boundaries."""
    from paper_2301_11828_gb300.slab import halo_window, partition
    nx, ny, nz = n
    rng = np.random.default_rng(nz)
    g = pd.Grid(3, n, 1.0 / 64, M, constrained=syn.clamp_bottom_3d(n, int(np.ceil(M))))
    parts = partition(nz, 3, align=1)
    for dt in (torch.float32, torch.float64):
        U = torch.tensor(rng.uniform(-1, 1, (2, 3, nz, ny, nx)), dtype=dt, device="cuda")
        for proj in (0, pd.PD_PROJECT):
            fl = pd.PD_METHOD_STENCIL | proj
            whole = g.matvec(U, flags=fl)
            pieces = []
            for z0, planes in parts:
                lo, ext = halo_window(z0, planes, nz, g.M)
                out = torch.empty((2, 3, planes, ny, nx), dtype=dt, device="cuda")
                pd.pd_matvec_rows(g.handle, 2, z0, planes, U[:, :, lo:lo + ext].contiguous(), lo, ext, out,
                                  fl | (pd.PD_F32 if dt == torch.float32 else pd.PD_F64))
                pieces.append(out)
            torch.cuda.synchronize()
            assert torch.equal(torch.cat(pieces, dim=2), whole), (str(dt), proj)


def test_ragged_band_inside_the_grid(pd):
    """A band whose row count is not a multiple of the tile height and which
    ends inside the grid: the kernels stage only the rows the input holds (the
    rows past it enter no written output).  FP32 bit for bit with the whole-grid
    product; FP64 bit for bit in the difference form (PD_ACCURATE), and within
    rounding in the default form, which subtracts a plane per tile fitted over
    what the tile stages."""
    n, M = (96, 160), 3
    nx, ny = n
    rng = np.random.default_rng(11)
    g = pd.Grid(2, n, 1.0 / nx, M)
    row0, rows = 32, 23
    lo, ext = row0 - M, rows + 2 * M
    for dt in (torch.float32, torch.float64):
        U = torch.tensor(rng.uniform(-1, 1, (1, 2, ny, nx)), dtype=dt, device="cuda")
        for extra in ((0, pd.PD_NO_TMA) if dt == torch.float32 else (0, pd.PD_ACCURATE)):
            fl = pd.PD_METHOD_STENCIL | extra
            whole = g.matvec(U, flags=fl)[:, :, row0:row0 + rows]
            out = torch.empty((1, 2, rows, nx), dtype=dt, device="cuda")
            pd.pd_matvec_rows(g.handle, 1, row0, rows, U[:, :, lo:lo + ext].contiguous(), lo, ext, out,
                              fl | (pd.PD_F32 if dt == torch.float32 else pd.PD_F64))
            torch.cuda.synchronize()
            if dt == torch.float32 or extra:
                assert torch.equal(out, whole), (str(dt), extra)
            else:
                d = (out - whole).norm() / whole.norm()
                assert float(d) <= 1e-14


def test_ragged_plane_band_3d(pd):
    """3D: a band of planes that is not a multiple of the tile depth, inside
    the grid, bit for bit."""
    n, M = (40, 33, 60), 3
    nx, ny, nz = n
    rng = np.random.default_rng(12)
    g = pd.Grid(3, n, 1.0 / 64, M)
    z0, planes = 21, 13
    lo, ext = z0 - M, planes + 2 * M
    for dt in (torch.float32, torch.float64):
        U = torch.tensor(rng.uniform(-1, 1, (1, 3, nz, ny, nx)), dtype=dt, device="cuda")
        whole = g.matvec(U, flags=pd.PD_METHOD_STENCIL)[:, :, z0:z0 + planes]
        out = torch.empty((1, 3, planes, ny, nx), dtype=dt, device="cuda")
        pd.pd_matvec_rows(g.handle, 1, z0, planes, U[:, :, lo:lo + ext].contiguous(), lo, ext, out,
                          pd.PD_METHOD_STENCIL | (pd.PD_F32 if dt == torch.float32 else pd.PD_F64))
        torch.cuda.synchronize()
        assert torch.equal(out, whole), str(dt)

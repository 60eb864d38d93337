"""The column-walk FP32 2D product (pd_set_stencil_tile_rows(g, 0)): each warp
walks down a 32-column strip with its own TMA ring and scatters every row into
the outputs it touches.  Checked through the C ABI against the FP64 oracle on
random and smooth fields (ragged strips, grids smaller than one strip, every
horizon it serves, a real delta/h), batches against single-field calls, and the
row bands of the slab split against the whole-grid product bit for bit."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pd():
    import paper_2301_11828_gb300 as pd
    pd.load_library()
    return pd


def _walk_grid(pd, n, h, M, **kw):
    g = pd.Grid(2, n, h, M, **kw)
    g.set_stencil_tile_rows(0)
    return g


def _ref(n, h, m, u, E=1.0):
    return oracle.stiffness(2, n, h, m, oracle.alpha(2, E, m * h), u)


def _smooth(n, offset):
    x = (np.arange(n[0]) + 0.5) / n[0]
    y = (np.arange(n[1]) + 0.5) / n[1]
    a = np.sin(2 * np.pi * x)[None, :] * np.cos(np.pi * y)[:, None]
    b = np.cos(3 * np.pi * x)[None, :] * np.sin(2 * np.pi * y)[:, None]
    if offset:
        return np.stack([1.0 + 0.3 * a, 0.7 + 0.2 * b])
    return np.stack([a, b])


@pytest.mark.parametrize("n,M", [((128, 97), 3), ((132, 70), 4), ((68, 45), 2), ((64, 45), 1), ((100, 77), 3),
                                 ((36, 9), 3), ((4, 5), 3), ((8, 1), 2), ((1024, 40), 3), ((96, 200), 4)])
def test_walk_matches_oracle_random(pd, n, M):
    h = 1.0 / 64
    rng = np.random.default_rng(31 * M + n[0] + n[1])
    u = torch.tensor(rng.uniform(-1, 1, (2, n[1], n[0])), dtype=torch.float32, device="cuda")
    g = _walk_grid(pd, n, h, M, E=2.5)
    out = g.matvec(u, flags=pd.PD_METHOD_STENCIL)
    torch.cuda.synchronize()
    ref = _ref(n, h, M, u.double().cpu().numpy(), E=2.5)
    err = rel_l2(out.double().cpu().numpy(), ref)
    assert err <= 2e-5, err
    assert err <= 1e-6, err   # in fact about 1e-7


@pytest.mark.parametrize("n", [(512, 384), (1024, 1024)])
@pytest.mark.parametrize("M", [3, 4])
@pytest.mark.parametrize("offset", [False, True])
def test_walk_smooth_fields(pd, n, M, offset):
    """Differences of nearby values throughout: the error stays relative to
    |K u| on smooth fields and on fields with a large constant part (whole
    field and full-horizon interior)."""
    h = 1.0 / n[0]
    g = _walk_grid(pd, n, h, M)
    ut = torch.tensor(_smooth(n, offset), dtype=torch.float32, device="cuda")
    ref = _ref(n, h, M, ut.double().cpu().numpy())
    out = g.matvec(ut, flags=pd.PD_METHOD_STENCIL).double().cpu().numpy()
    inner = (slice(None), slice(M, n[1] - M), slice(M, n[0] - M))
    e, e_in = rel_l2(out, ref), rel_l2(out[inner], ref[inner])
    print(f"walk n={n} M={M} offset={offset}: {e:.3e} (interior {e_in:.3e})")
    assert e <= 1e-6 and e_in <= 1e-6


def test_walk_real_horizon(pd):
    """delta/h = 2.6: kernels on radius 3 with zero coefficients beyond 2.6."""
    n, h, m = (120, 90), 1.0 / 120, 2.6
    rng = np.random.default_rng(5)
    u = torch.tensor(rng.uniform(-1, 1, (2, n[1], n[0])), dtype=torch.float32, device="cuda")
    g = _walk_grid(pd, n, h, m)
    out = g.matvec(u, flags=pd.PD_METHOD_STENCIL).double().cpu().numpy()
    ref = _ref(n, h, m, u.double().cpu().numpy())
    assert rel_l2(out, ref) <= 1e-6


def test_walk_batch_equals_single_fields(pd):
    n, M = (260, 131), 3
    rng = np.random.default_rng(9)
    U = torch.tensor(rng.uniform(-1, 1, (5, 2, n[1], n[0])), dtype=torch.float32, device="cuda")
    g = _walk_grid(pd, n, 1.0 / 256, M)
    whole = g.matvec(U, flags=pd.PD_METHOD_STENCIL)
    for b in range(5):
        one = g.matvec(U[b].contiguous(), flags=pd.PD_METHOD_STENCIL)
        assert torch.equal(one, whole[b])
    torch.cuda.synchronize()
    ref = _ref(n, 1.0 / 256, M, U[3].double().cpu().numpy())
    assert rel_l2(whole[3].double().cpu().numpy(), ref) <= 1e-6


def test_walk_agrees_with_tile_kernel(pd):
    """Both FP32 layouts sum differences: they agree to FP32 rounding."""
    n, M = (256, 192), 3
    rng = np.random.default_rng(3)
    U = torch.tensor(rng.uniform(-1, 1, (2, 2, n[1], n[0])), dtype=torch.float32, device="cuda")
    g = pd.Grid(2, n, 1.0 / 256, M)
    tile = g.matvec(U, flags=pd.PD_METHOD_STENCIL)
    g.set_stencil_tile_rows(0)
    walk = g.matvec(U, flags=pd.PD_METHOD_STENCIL)
    torch.cuda.synchronize()
    assert rel_l2(walk.double().cpu().numpy(), tile.double().cpu().numpy()) <= 5e-7


@pytest.mark.parametrize("n,M,world", [((256, 200), 3, 2), ((132, 97), 4, 3), ((64, 64), 2.5, 2), ((96, 70), 1, 3)])
def test_walk_slabs_bit_for_bit(pd, n, M, world):
    from paper_2301_11828_gb300.slab import halo_window, partition
    nx, ny = n
    rng = np.random.default_rng(int(10 * M) + nx)
    g = _walk_grid(pd, n, 1.0 / nx, M)
    U = torch.tensor(rng.uniform(-1, 1, (2, 2, ny, nx)), dtype=torch.float32, device="cuda")
    whole = g.matvec(U, flags=pd.PD_METHOD_STENCIL)
    pieces = []
    for row0, rows in partition(ny, world):
        lo, ext = halo_window(row0, rows, ny, g.M)
        u_ext = U[:, :, lo:lo + ext, :].contiguous()
        out = torch.empty((2, 2, rows, nx), dtype=torch.float32, device="cuda")
        pd.pd_matvec_rows(g.handle, 2, row0, rows, u_ext, lo, ext, out, pd.PD_METHOD_STENCIL | pd.PD_F32)
        pieces.append(out)
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(pieces, dim=2), whole)


def test_walk_falls_back_for_projection(pd):
    """Projected products take the tile kernel (same result within FP32)."""
    w = syn.plate_static(97, 3, tag=5, u_amp=1.0)
    nx = 100
    cons = np.zeros((2, 97, nx), dtype=np.uint8)
    cons[:, :, :3] = 1
    g = _walk_grid(pd, (nx, 97), 1.0 / nx, 3, constrained=cons)
    rng = np.random.default_rng(1)
    u = torch.tensor(rng.uniform(-1, 1, (2, 97, nx)), dtype=torch.float32, device="cuda")
    out = g.matvec(u, flags=pd.PD_METHOD_STENCIL | pd.PD_PROJECT).double().cpu().numpy()
    ref = oracle.stiffness(2, (nx, 97), 1.0 / nx, 3, oracle.alpha(2, 1.0, 3.0 / nx), u.double().cpu().numpy(),
                           cons=cons)
    assert rel_l2(out, ref) <= 1e-6
    del w

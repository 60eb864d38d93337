"""Horizons that are not a whole number of spacings (m = delta / h real): the GPU
runs its kernels on the radius-ceil(m) disk with zero coefficients beyond m;
products, broken sets, notches and solves against the oracle's bonds |o| <= m."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import mask_to_mu, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


@pytest.fixture(scope="module")
def pd():
    import paper_2301_11828_gb300 as pd
    pd.load_library()
    return pd


def _to_oracle_mu(g, dim, m):
    """GPU bond mask [N][nnb of the radius disk] -> the oracle's [N][bonds |o| <= m];
    the offsets beyond m must stay intact."""
    gpu = mask_to_mu(g.bond_mask().cpu().numpy(), g.nnb)
    goff = [tuple(o) for o in g.offsets()[:, :3]]
    ooff = [tuple(o) for o in oracle.offsets(dim, m)[:, :3]]
    idx = [goff.index(o) for o in ooff]
    extra = [k for k, o in enumerate(goff) if o not in set(ooff)]
    assert np.all(gpu[:, extra] == 1)
    return gpu[:, idx]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("dim,n,m,method", [
    (2, (132, 97), 2.5, "stencil"), (2, (132, 97), 2.5, "fft"), (2, (100, 67), 1.5, "stencil"),
    (2, (96, 80), 3.7, "stencil"), (2, (96, 80), 3.7, "fft"), (2, (75, 66), 5.3, "stencil"),
    (3, (30, 21, 17), 2.5, "stencil"), (3, (20, 20, 20), 2.5, "fft")])
def test_real_horizon_product(pd, dtype, dim, n, m, method):
    h = 1.0 / 64
    rng = np.random.default_rng(int(10 * m) + n[0])
    u = rng.uniform(-1, 1, (dim,) + tuple(reversed(n)))
    g = pd.Grid(dim, n, h, m, E=1.7)
    assert g.M == int(np.ceil(m))
    flags = pd.PD_METHOD_FFT if method == "fft" else pd.PD_METHOD_STENCIL
    ut = torch.tensor(u, dtype=dtype, device="cuda")
    al = oracle.alpha(dim, 1.7, m * h)
    ref = oracle.stiffness(dim, n, h, m, al, ut.double().cpu().numpy())
    for extra in ((0, pd.PD_PAIR_FORM, pd.PD_NO_TMA) if (dtype == torch.float32 and method == "stencil") else (0,)):
        out = g.matvec(ut, flags=flags | extra)
        assert rel_l2(out.double().cpu().numpy(), ref) <= TOL[dtype]


@pytest.mark.parametrize("dim,n,m", [(2, (90, 77), 2.5), (2, (64, 60), 3.7), (3, (30, 21, 17), 2.5)])
def test_real_horizon_breaking_and_notch_bit_exact(pd, dim, n, m):
    h = 1.0 / 64
    rng = np.random.default_rng(int(10 * m))
    ub = rng.normal(0, 0.05 * h, (dim,) + tuple(reversed(n)))
    g = pd.Grid(dim, n, h, m, s0=0.03)
    mu = oracle.intact_mu(dim, n, m)
    if dim == 2:
        seg = (10 * n[0] // 4, 10 * n[1] // 2 + 3, 10 * 3 * n[0] // 4, 10 * n[1] // 2 + 3)
        assert g.break_segment(seg, 10) == oracle.prenotch(n, m, seg, 10, mu) > 0
    nb = g.break_bonds(torch.tensor(ub, device="cuda"))
    assert nb == oracle.break_bonds(dim, n, h, m, 0.03, ub, mu) > 0
    assert np.array_equal(_to_oracle_mu(g, dim, m), mu)
    # the product honours the broken set
    u = rng.uniform(-1, 1, (dim,) + tuple(reversed(n)))
    out = g.matvec(torch.tensor(u, device="cuda"), flags=pd.PD_METHOD_STENCIL)
    ref = oracle.stiffness(dim, n, h, m, oracle.alpha(dim, 1.0, m * h), u, mu=mu)
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("mode", ["mixed", "f64", "adr"])
def test_real_horizon_solves(pd, mode):
    n, m = (64, 60), 2.5
    h = 1.0 / n[0]
    cons = syn.clamp_left(2, n, 3)
    b = syn.traction_right(2, n, 3, 1e-3)
    g = pd.Grid(2, n, h, m, constrained=cons)
    bt = torch.tensor(b, device="cuda")
    if mode == "adr":
        u, st = g.adr_solve(bt, rtol=1e-8, mode=pd.PD_ADR_MIXED)
    else:
        u, st = g.cg_solve(bt, rtol=1e-8, mode=pd.PD_CG_MIXED if mode == "mixed" else pd.PD_CG_F64)
    P = 1 - cons
    r = b * P - oracle.stiffness(2, n, h, m, oracle.alpha(2, 1.0, m * h), u.cpu().numpy(), cons=cons)
    assert np.linalg.norm(r) / np.linalg.norm(b * P) <= 1.05e-8


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_real_horizon_with_surface_correction(pd, dtype):
    """The surface-correction factors use lambda at the real delta: nu and the
    corrected product against the oracle at m = 2.5 (2D) and 1.5 (3D)."""
    for dim, n, m in ((2, (96, 71), 2.5), (3, (20, 17, 15), 1.5)):
        h = 1.0 / 64
        rng = np.random.default_rng(3)
        u = rng.uniform(-1, 1, (dim,) + tuple(reversed(n)))
        g = pd.Grid(dim, n, h, m, surface_correction=pd.PD_SC_VOLUME)
        ut = torch.tensor(u, dtype=dtype, device="cuda")
        out = g.matvec(ut, flags=pd.PD_METHOD_STENCIL).double().cpu().numpy()
        nu = oracle.surface_nu(dim, n, h, m)
        ref = oracle.stiffness(dim, n, h, m, oracle.alpha(dim, 1.0, m * h), ut.double().cpu().numpy(), nu=nu)
        assert rel_l2(out, ref) <= TOL[dtype]

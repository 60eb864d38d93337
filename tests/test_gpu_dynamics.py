"""GPU velocity-Verlet crack loop and gradient kernels against the oracle."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import mask_to_mu, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pd():
    import paper_2301_11828_gb300 as pd
    pd.load_library()
    return pd


def _crack_setup(nside, M=3):
    w = syn.crack_plate(nside, M)
    lay = w.extra["vel_layers"]
    cons = np.zeros((2,) + lay.shape, dtype=np.uint8)
    cons[1] = lay != 0
    vp = np.zeros((2,) + lay.shape)
    vp[1] = lay * w.extra["v0"]
    return w, cons, vp


def _stable_dt(w, E_max):
    al1 = oracle.alpha(2, 1.0, w.delta)
    G = oracle.symbol(2, (2 * w.n[0], 2 * w.n[1]), w.h, w.M, al1).real
    lam = np.linalg.eigvalsh(-np.moveaxis(G.reshape(2, 2, -1), 2, 0)).max()
    return 2.0 * np.sqrt(w.rho / (E_max * lam))


def test_verlet_matches_oracle_without_breaking(pd):
    w, cons, vp = _crack_setup(40)
    E = w.extra["E_field"]
    dt = 0.5 * _stable_dt(w, E.max())
    rng = np.random.default_rng(3)
    u0 = rng.normal(0, 1e-4, (2,) + E.shape)
    b = syn.gaussian_field(2, w.n, 1e-3, 4)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=cons, E_field=torch.tensor(E, device="cuda"), s0=0.0)
    u = torch.tensor(u0, device="cuda")
    v = torch.tensor(vp, device="cuda")
    g.step(u, v, torch.tensor(b, device="cuda"), nsteps=40, dt=dt, v_prescribed=torch.tensor(vp, device="cuda"))
    uo, vo = u0.copy(), vp.copy()
    al1 = oracle.alpha(2, 1.0, w.delta)
    oracle.vv(2, w.n, w.h, w.M, al1, uo, vo, 40, dt, b=b, E=E, cons=cons, vpres=vp)
    assert rel_l2(u.cpu().numpy(), uo) <= 1e-11
    assert rel_l2(v.cpu().numpy(), vo) <= 1e-10


def test_crack_loop_summary_and_break_steps(pd):
    """Pre-notched plate pulled apart: bonds break, the broken set stays symmetric
    and monotone, break steps are recorded, and the trajectory follows the oracle
    (identical broken sets step by step on this short run)."""
    w, cons, vp = _crack_setup(48)
    E = w.extra["E_field"]
    dt = 0.8 * _stable_dt(w, E.max())
    vp = vp * 50.0   # pull hard so that bonds break within a short run
    g = pd.Grid(2, w.n, w.h, w.M, constrained=cons, E_field=torch.tensor(E, device="cuda"), s0=w.s0)
    nb0 = g.break_segment(w.extra["notch"], w.extra["notch_den"])
    mu = oracle.intact_mu(2, w.n, w.M)
    assert nb0 == oracle.prenotch(w.n, w.M, w.extra["notch"], w.extra["notch_den"], mu)
    u = torch.zeros((2,) + E.shape, dtype=torch.float64, device="cuda")
    v = torch.tensor(vp, device="cuda")
    bs = torch.zeros(g.N * g.nnb, dtype=torch.int32, device="cuda")
    uo, vo = np.zeros((2,) + E.shape), vp.copy()
    al1 = oracle.alpha(2, 1.0, w.delta)
    total = 0
    for chunk in range(6):
        st = g.step(u, v, None, nsteps=10, dt=dt, v_prescribed=torch.tensor(vp, device="cuda"), break_step=bs,
                    step_base=10 * chunk)
        nbo = oracle.vv(2, w.n, w.h, w.M, al1, uo, vo, 10, dt, E=E, mu=mu, s0=w.s0, cons=cons, vpres=vp)
        total += st.newly_broken
        got = mask_to_mu(g.bond_mask().cpu().numpy(), g.nnb)
        assert np.array_equal(got, mu), f"broken sets diverged in chunk {chunk}"
        assert st.newly_broken == nbo
        assert rel_l2(u.cpu().numpy(), uo) <= 1e-9
    assert total > 0
    bsn = bs.cpu().numpy().reshape(g.N, g.nnb)
    assert np.all(mu[bsn > 0] == 0)
    assert (bsn > 0).sum() == 2 * total
    assert bsn.max() <= 60


def test_modulus_gradient_kernel_matches_oracle(pd):
    n, M, h = (50, 37), 3, 1.0 / 48
    rng = np.random.default_rng(7)
    u = rng.normal(size=(2, n[1], n[0]))
    lam = rng.normal(size=(2, n[1], n[0]))
    g = pd.Grid(2, n, h, M, s0=0.02)
    ub = rng.normal(0, 0.02 * h, (2, n[1], n[0]))
    g.break_bonds(torch.tensor(ub, device="cuda"))
    mu = oracle.intact_mu(2, n, M)
    oracle.break_bonds(2, n, h, M, 0.02, ub, mu)
    gr = g.grad_modulus(torch.tensor(u, device="cuda"), torch.tensor(lam, device="cuda"), scale=-0.5)
    ref = oracle.grad_modulus(2, n, h, M, oracle.alpha(2, 1.0, M * h), u, lam, mu=mu)
    assert rel_l2(gr.cpu().numpy(), ref) <= 1e-12


# --------------------------------------------------------------------------- 3D block with notches

def _stable_dt3(n, h, M):
    al = oracle.alpha(3, 1.0, M * h)
    G = oracle.symbol(3, tuple(2 * v for v in n), h, M, al).real
    lam = np.linalg.eigvalsh(-np.moveaxis(G.reshape(3, 3, -1), 2, 0)).max()
    return 2.0 / np.sqrt(lam)


@pytest.mark.parametrize("nx,ny,nz,M", [(201, 101, 9, 3), (33, 17, 6, 2), (40, 21, 5, 3)])
def test_kw_block_notches_bit_exact(pd, nx, ny, nz, M):
    """Through-thickness notches of the 3D block: the GPU cut set equals the oracle's."""
    w = syn.kw_block(nx, ny, nz, M)
    g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained, s0=w.s0)
    mu = oracle.intact_mu(3, w.n, w.M)
    tot_g = tot_o = 0
    for seg in w.extra["notches"]:
        tot_g += g.break_segment(seg, w.extra["notch_den"])
        tot_o += oracle.prenotch(w.n, w.M, seg, w.extra["notch_den"], mu, dim=3)
    assert tot_g == tot_o > 0
    assert np.array_equal(mask_to_mu(g.bond_mask().cpu().numpy(), g.nnb), mu)


def test_kw_block_crack_loop_follows_oracle(pd):
    """3D Verlet with breaking and the D^f correction on a small notched block
    driven between the notches: identical broken sets and matching trajectories
    chunk by chunk, break steps recorded."""
    w = syn.kw_block(33, 17, 6, 2, v0=0.01)
    dt = 0.8 * _stable_dt3(w.n, w.h, w.M)
    vp = w.extra["v_prescribed"]
    g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained, s0=w.s0)
    mu = oracle.intact_mu(3, w.n, w.M)
    for seg in w.extra["notches"]:
        g.break_segment(seg, w.extra["notch_den"])
        oracle.prenotch(w.n, w.M, seg, w.extra["notch_den"], mu, dim=3)
    u = torch.zeros((3,) + vp.shape[1:], dtype=torch.float64, device="cuda")
    v = torch.tensor(vp, device="cuda")
    vpt = torch.tensor(vp, device="cuda")
    bs = torch.zeros(g.N * g.nnb, dtype=torch.int32, device="cuda")
    uo, vo = np.zeros_like(vp), vp.copy()
    al = oracle.alpha(3, 1.0, w.delta)
    total = 0
    for chunk in range(6):
        st = g.step(u, v, None, nsteps=10, dt=dt, v_prescribed=vpt, break_step=bs, step_base=10 * chunk)
        nbo = oracle.vv(3, w.n, w.h, w.M, al, uo, vo, 10, dt, mu=mu, s0=w.s0, cons=w.constrained, vpres=vp)
        total += st.newly_broken
        assert np.array_equal(mask_to_mu(g.bond_mask().cpu().numpy(), g.nnb), mu), f"chunk {chunk}"
        assert st.newly_broken == nbo
        assert rel_l2(u.cpu().numpy(), uo) <= 1e-9
    assert total > 0
    bsn = bs.cpu().numpy().reshape(g.N, g.nnb)
    assert (bsn > 0).sum() == 2 * total and bsn.max() <= 60

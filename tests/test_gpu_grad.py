"""Gradients through the C ABI with hand-written adjoints (torch.autograd).

Static: u = (P K(E) P)^-1 P b by CG; dL/db and dL/dE against central finite
differences of the GPU solve and against the oracle's gradient.
Dynamic: the Verlet crack loop with checkpointed replay; dL/dE against the
oracle's discrete adjoint and finite differences."""
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
    import paper_2301_11828_gb300.autograd  # noqa: F401
    pd.load_library()
    return pd


def test_matvec_backward_is_K(pd):
    from paper_2301_11828_gb300.autograd import matvec
    n, M = (40, 33), 3
    g = pd.Grid(2, n, 1 / 40, M, constrained=syn.clamp_left(2, n, M))
    u = torch.randn((2, 33, 40), dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.randn_like(u)
    y = matvec(g, u, pd.PD_PROJECT)
    (y * w).sum().backward()
    assert torch.allclose(u.grad, g.matvec(w.contiguous(), flags=pd.PD_PROJECT), rtol=1e-12, atol=1e-12)


def test_static_solve_gradients(pd):
    from paper_2301_11828_gb300.autograd import static_solve
    n, M, h = (28, 22), 3, 1.0 / 28
    cons = syn.clamp_left(2, n, M)
    b_np = syn.gaussian_field(2, n, 1e-3, 41) * (1 - cons)
    E_np = syn.lognormal_modulus(n, 0.1, 42)
    g = pd.Grid(2, n, h, M, constrained=cons)
    b = torch.tensor(b_np, device="cuda", requires_grad=True)
    E = torch.tensor(E_np, device="cuda", requires_grad=True)
    u = static_solve(g, b, E, rtol=1e-12, mode=pd.PD_CG_F64)
    L = 0.5 * (u * u).sum()
    L.backward()
    gb, gE = b.grad.cpu().numpy(), E.grad.cpu().numpy()
    # oracle gradient: lam solves K lam = u, dL/dE = -1/2 bond sum, dL/db = lam
    al1 = oracle.alpha(2, 1.0, M * h)
    uo, _, _ = oracle.cg(2, n, h, M, al1, b_np, cons=cons, E=E_np, rtol=1e-13)
    lam, _, _ = oracle.cg(2, n, h, M, al1, uo, cons=cons, E=E_np, rtol=1e-13)
    assert rel_l2(gb, lam) <= 1e-8
    assert rel_l2(gE, oracle.grad_modulus(2, n, h, M, al1, uo, lam)) <= 1e-8
    # finite differences of the GPU solve itself
    rng = np.random.default_rng(3)
    with torch.no_grad():
        for flat in rng.choice(E_np.size, 3, replace=False):
            idx = np.unravel_index(flat, E_np.shape)
            eps = 1e-5 * E_np[idx]
            Lpm = []
            for sgn in (1, -1):
                Ep = E.detach().clone()
                Ep[idx] += sgn * eps
                up = static_solve(g, b.detach(), Ep, rtol=1e-13, mode=pd.PD_CG_F64)
                Lpm.append(0.5 * float((up * up).sum()))
            fd = (Lpm[0] - Lpm[1]) / (2 * eps)
            assert gE[idx] == pytest.approx(fd, rel=1e-4, abs=1e-6 * np.abs(gE).max())


def test_verlet_gradient_matches_oracle_adjoint(pd):
    from paper_2301_11828_gb300.autograd import verlet_run
    w = syn.crack_plate(40, 3)
    n, M, h = w.n, w.M, w.h
    lay = w.extra["vel_layers"]
    cons = np.zeros((2,) + lay.shape, dtype=np.uint8)
    cons[1] = lay != 0
    vp = np.zeros((2,) + lay.shape)
    vp[1] = lay * 0.02
    E_np = w.extra["E_field"]
    dt, steps, s0 = 2e-3, 40, 2e-3
    g = pd.Grid(2, n, h, M, constrained=cons, s0=s0)
    g.break_segment(w.extra["notch"], w.extra["notch_den"])
    mask0 = g.bond_mask().clone()
    E = torch.tensor(E_np, device="cuda", requires_grad=True)
    u0 = torch.zeros((2,) + lay.shape, dtype=torch.float64, device="cuda")
    v0 = torch.tensor(vp, device="cuda")
    vpt = torch.tensor(vp, device="cuda")
    uN = verlet_run(g, E, u0, v0, steps, dt, v_prescribed=vpt, checkpoint_every=12)
    (0.5 * (uN * uN).sum()).backward()
    gE = E.grad.cpu().numpy()
    al1 = oracle.alpha(2, 1.0, M * h)
    mu0 = oracle.intact_mu(2, n, M)
    oracle.prenotch(n, M, w.extra["notch"], w.extra["notch_den"], mu0)
    uo, go = oracle.vv_grad_modulus(2, n, h, M, al1, E_np, np.zeros_like(vp), vp.copy(), steps, dt, mu0=mu0, s0=s0,
                                    cons=cons, vpres=vp)
    assert rel_l2(uN.detach().cpu().numpy(), uo) <= 1e-10
    assert rel_l2(gE, go) <= 1e-8
    from helpers import mask_to_mu
    assert (mask_to_mu(g.bond_mask().cpu().numpy(), g.nnb) == 0).sum() > (mu0 == 0).sum()   # bonds broke
    # finite differences on the GPU forward (same broken sets in the +/- runs)
    with torch.no_grad():
        for flat in np.argsort(-np.abs(gE).ravel())[:2]:
            idx = np.unravel_index(flat, E_np.shape)
            eps = 1e-4 * E_np[idx]
            Lpm, masks = [], []
            for sgn in (1, -1):
                g.set_bond_mask(mask0)
                Ep = E.detach().clone()
                Ep[idx] += sgn * eps
                up = verlet_run(g, Ep, u0, v0, steps, dt, v_prescribed=vpt, checkpoint_every=12)
                Lpm.append(0.5 * float((up * up).sum()))
                masks.append(g.bond_mask().clone())
            assert torch.equal(masks[0], masks[1])
            fd = (Lpm[0] - Lpm[1]) / (2 * eps)
            assert gE[idx] == pytest.approx(fd, rel=1e-3)

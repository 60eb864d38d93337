"""GPU surface correction (volume method on incomplete horizons) against the
oracle's direct sum with the same factors: the product in both methods and
precisions, with projection, broken bonds and a modulus field; the solvers,
the Verlet loop and the modulus gradient that use it."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


@pytest.fixture(scope="module")
def pd():
    import paper_2301_11828_gb300 as pd
    pd.load_library()
    return pd


def _product(g, u_np, dtype, flags):
    u = torch.tensor(u_np, dtype=dtype, device="cuda")
    out = g.matvec(u, flags=flags)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), u.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("dim,n,M,method", [
    (2, (130, 97), 3, "stencil"), (2, (130, 97), 3, "fft"), (2, (75, 66), 5, "stencil"),
    (2, (5, 3), 3, "stencil"), (2, (1, 40), 3, "stencil"), (2, (256, 72), 2, "stencil"),
    (3, (30, 21, 17), 2, "stencil"), (3, (20, 20, 20), 3, "fft"), (3, (9, 4, 13), 3, "stencil")])
def test_sc_product_matches_oracle(pd, dtype, dim, n, M, method):
    h = 1.0 / 64
    rng = np.random.default_rng(M * 100 + n[0])
    u_np = rng.uniform(-1, 1, (dim,) + tuple(reversed(n)))
    g = pd.Grid(dim, n, h, M, E=2.5, surface_correction=pd.PD_SC_VOLUME)
    flags = pd.PD_METHOD_FFT if method == "fft" else pd.PD_METHOD_STENCIL
    out, u_used = _product(g, u_np, dtype, flags)
    al = oracle.alpha(dim, 2.5, M * h)
    nu = oracle.surface_nu(dim, n, h, M)
    assert rel_l2(out, oracle.stiffness(dim, n, h, M, al, u_used, nu=nu)) <= TOL[dtype]
    # switched off again: the paper's operator
    g.set_surface_correction(pd.PD_SC_NONE)
    out0, _ = _product(g, u_np, dtype, flags)
    assert rel_l2(out0, oracle.stiffness(dim, n, h, M, al, u_used)) <= TOL[dtype]
    g.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sc_projection_and_batch(pd, dtype):
    w = syn.plate_static(96, 3, tag=2, u_amp=1.0)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained, surface_correction=pd.PD_SC_VOLUME)
    rng = np.random.default_rng(2)
    U = rng.uniform(-1, 1, (3, 2, w.n[1], w.n[0]))
    Ut = torch.tensor(U, dtype=dtype, device="cuda")
    O = torch.empty_like(Ut)
    pd.pd_matvec_batch(g.handle, 3, Ut, O, (pd.PD_F64 if dtype == torch.float64 else pd.PD_F32) | pd.PD_PROJECT)
    al = oracle.alpha(2, 1.0, w.delta)
    nu = oracle.surface_nu(2, w.n, w.h, w.M)
    for b in range(3):
        ref = oracle.stiffness(2, w.n, w.h, w.M, al, Ut[b].double().cpu().numpy(), cons=w.constrained, nu=nu)
        assert rel_l2(O[b].double().cpu().numpy(), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sc_with_broken_bonds_and_modulus_field(pd, dtype):
    n, M, h = (77, 64), 3, 1.0 / 64
    rng = np.random.default_rng(4)
    ub = rng.normal(0, 0.05 * h, (2, n[1], n[0]))
    u_np = rng.uniform(-1, 1, (2, n[1], n[0]))
    nu = oracle.surface_nu(2, n, h, M)
    # constant modulus: TBT stencil + D^f gather + correction (mask-aware)
    g = pd.Grid(2, n, h, M, s0=0.03, surface_correction=pd.PD_SC_VOLUME)
    g.break_bonds(torch.tensor(ub, device="cuda"))
    mu = oracle.intact_mu(2, n, M)
    assert oracle.break_bonds(2, n, h, M, 0.03, ub, mu) > 0
    out, u_used = _product(g, u_np, dtype, 0)
    ref = oracle.stiffness(2, n, h, M, oracle.alpha(2, 1.0, M * h), u_used, mu=mu, nu=nu)
    assert rel_l2(out, ref) <= TOL[dtype]
    # per-node modulus: direct form + correction with (E_p + E_q)/2
    E = syn.lognormal_modulus(n, 0.1, 8)
    g2 = pd.Grid(2, n, h, M, E_field=torch.tensor(E, device="cuda"), surface_correction=pd.PD_SC_VOLUME)
    g2.set_material(E=1.0, s0=0.03, E_field=torch.tensor(E, device="cuda"))
    g2.break_bonds(torch.tensor(ub, device="cuda"))
    mu2 = oracle.intact_mu(2, n, M)
    oracle.break_bonds(2, n, h, M, 0.03, ub, mu2)
    out2, u_used = _product(g2, u_np, dtype, 0)
    ref2 = oracle.stiffness(2, n, h, M, oracle.alpha(2, 1.0, M * h), u_used, E=E, mu=mu2, nu=nu)
    assert rel_l2(out2, ref2) <= TOL[dtype]


def test_sc_full_size_plate_1024(pd):
    """The timed configuration (1024^2, delta = 3h, FP32 TMA stencil) with the correction, whole field."""
    w = syn.large_plate(3)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained, surface_correction=pd.PD_SC_VOLUME)
    out, u_used = _product(g, w.u, torch.float32, pd.PD_METHOD_STENCIL | pd.PD_PROJECT)
    nu = oracle.surface_nu(2, w.n, w.h, w.M)
    ref = oracle.stiffness(2, w.n, w.h, w.M, oracle.alpha(2, 1.0, w.delta), u_used, cons=w.constrained, nu=nu)
    assert rel_l2(out, ref) <= 2e-5
    band = np.zeros(w.n[::-1], dtype=bool)
    band[:6, :] = band[-6:, :] = True
    band[:, :6] = band[:, -6:] = True
    assert rel_l2(out[:, band], ref[:, band]) <= 2e-5


@pytest.mark.parametrize("mode", ["mixed", "f64"])
def test_sc_cg_converges_to_the_corrected_solution(pd, mode):
    n, M = (64, 64), 3
    w = syn.plate_static(n[0], M, tag=5, u_amp=0.0)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained, surface_correction=pd.PD_SC_VOLUME)
    u, st = g.cg_solve(torch.tensor(w.b, device="cuda"), rtol=1e-8,
                       mode=pd.PD_CG_MIXED if mode == "mixed" else pd.PD_CG_F64)
    assert st.persistent == 0
    nu = oracle.surface_nu(2, n, w.h, M)
    al = oracle.alpha(2, 1.0, w.delta)
    P = 1 - w.constrained
    r = w.b * P - oracle.stiffness(2, n, w.h, M, al, u.cpu().numpy(), cons=w.constrained, nu=nu)
    assert np.linalg.norm(r) / np.linalg.norm(w.b * P) <= 1.05e-8


def test_sc_adr_iterates_match_oracle(pd):
    n, M = (48, 40), 3
    h = 1.0 / n[0]
    cons = syn.clamp_left(2, n, M)
    b = syn.traction_right(2, n, M, 1e-3)
    g = pd.Grid(2, n, h, M, constrained=cons, surface_correction=pd.PD_SC_VOLUME)
    bt = torch.tensor(b, device="cuda")
    u = torch.zeros_like(bt)
    # 100 updates: with the correction the damping quotient amplifies rounding faster
    # than without (the oracle itself moves by 1.4e-13 at 100 updates and by 2.6e-10
    # at 300 under a 1e-16 relative change of its operator)
    st = pd.pd_adr_solve(g.handle, bt, u, 1e-30, 100, allow_not_converged=True)
    nu = oracle.surface_nu(2, n, h, M)
    al = oracle.alpha(2, 1.0, M * h)
    ref, it, _ = oracle.adr_solve(2, n, h, M, al, b, cons=cons, rtol=1e-30, maxit=100, nu=nu)
    assert st.iterations == it == 100
    assert rel_l2(u.cpu().numpy(), ref) <= 1e-9
    u, st = g.adr_solve(bt, rtol=1e-8)
    r = b * (1 - cons) - oracle.stiffness(2, n, h, M, al, u.cpu().numpy(), cons=cons, nu=nu)
    assert np.linalg.norm(r) / np.linalg.norm(b * (1 - cons)) <= 1.05e-8


def test_sc_verlet_and_modulus_gradient(pd):
    n, M, h = (40, 36), 3, 1.0 / 40
    E = syn.lognormal_modulus(n, 0.1, 3)
    cons = syn.clamp_left(2, n, M)
    rng = np.random.default_rng(3)
    u0 = rng.normal(0, 1e-4, (2, n[1], n[0]))
    b = syn.gaussian_field(2, n, 1e-3, 4)
    nu = oracle.surface_nu(2, n, h, M)
    g = pd.Grid(2, n, h, M, constrained=cons, E_field=torch.tensor(E, device="cuda"),
                surface_correction=pd.PD_SC_VOLUME)
    u = torch.tensor(u0, device="cuda")
    v = torch.zeros_like(u)
    dt = 1e-3
    g.step(u, v, torch.tensor(b, device="cuda"), nsteps=30, dt=dt)
    uo, vo = u0.copy(), np.zeros_like(u0)
    al1 = oracle.alpha(2, 1.0, M * h)
    oracle.vv(2, n, h, M, al1, uo, vo, 30, dt, b=b, E=E, cons=cons, nu=nu)
    assert rel_l2(u.cpu().numpy(), uo) <= 1e-11
    assert rel_l2(v.cpu().numpy(), vo) <= 1e-10
    lam = rng.normal(size=(2, n[1], n[0]))
    x = rng.normal(size=(2, n[1], n[0]))
    gr = g.grad_modulus(torch.tensor(x, device="cuda"), torch.tensor(lam, device="cuda"), scale=-0.5)
    ref = oracle.grad_modulus(2, n, h, M, al1, x, lam, nu=nu)
    assert rel_l2(gr.cpu().numpy(), ref) <= 1e-12


def test_sc_batch_refuses_and_modes_checked(pd):
    w = syn.plate_static(64, 3, tag=2, u_amp=1.0)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained, surface_correction=pd.PD_SC_VOLUME)
    with pytest.raises(pd.PDError) as e:
        pd.pd_batch_create([g])
    assert e.value.code == pd.PD_ERR_INVALID
    with pytest.raises(pd.PDError) as e:
        g.set_surface_correction(7)
    assert e.value.code == pd.PD_ERR_INVALID

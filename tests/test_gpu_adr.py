"""GPU ADR/CDEI (Algorithm 1) against the oracle's ADR: the same iterates after a
fixed number of updates, the same stopping point, and the true residual of the
converged answer measured with the oracle's FP64 operator."""
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


def _plate(n, M, tag=4):
    w = syn.plate_static(n[0], M, tag=tag, u_amp=0.0)
    w.n = n
    w.h = 1.0 / n[0]
    w.constrained = syn.clamp_left(2, n, M)
    w.b = syn.traction_right(2, n, M, 1e-3)
    return w


@pytest.mark.parametrize("n,M,iters", [((48, 40), 3, 300), ((37, 29), 2, 150), ((64, 64), 5, 200)])
def test_adr_iterates_match_oracle(pd, n, M, iters):
    w = _plate(n, M)
    al = oracle.alpha(2, 1.0, w.delta)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained)
    b = torch.tensor(w.b, device="cuda")
    u = torch.zeros_like(b)
    st = pd.pd_adr_solve(g.handle, b, u, 1e-30, iters, allow_not_converged=True)
    ref, it, rel = oracle.adr_solve(2, n, w.h, M, al, w.b, cons=w.constrained, rtol=1e-30, maxit=iters)
    assert st.iterations == it == iters
    assert rel_l2(u.cpu().numpy(), ref) <= 1e-9
    # the residual is a small difference of O(1) terms: rounding of u shows amplified
    assert abs(st.rel_residual - rel) <= 1e-6 * rel


@pytest.mark.parametrize("method", ["stencil", "fft"])
def test_adr_converges_like_oracle(pd, method):
    n, M = (64, 64), 3
    w = _plate(n, M, tag=5)
    al = oracle.alpha(2, 1.0, w.delta)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained)
    if method == "fft":
        g.prefer_method(pd.PD_METHOD_FFT)
    u, st = g.adr_solve(torch.tensor(w.b, device="cuda"), rtol=1e-8)
    un = u.cpu().numpy()
    ref, it, rel = oracle.adr_solve(2, n, w.h, M, al, w.b, cons=w.constrained, rtol=1e-8, maxit=1000000)
    assert st.rel_residual <= 1e-8
    assert abs(st.iterations - it) <= 2
    P = 1 - w.constrained
    r = w.b * P - oracle.stiffness(2, n, w.h, M, al, un, cons=w.constrained)
    assert np.linalg.norm(r) / np.linalg.norm(w.b * P) <= 1.05e-8
    assert np.all(un[w.constrained.astype(bool)] == 0)


def test_adr_with_broken_bonds_and_3d(pd):
    # pre-notched plate: the operator includes the D^f correction
    n, M = (48, 40), 3
    w = _plate(n, M, tag=6)
    al = oracle.alpha(2, 1.0, w.delta)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained)
    seg = (10 * n[0] // 4, 10 * n[1] // 2, 10 * 3 * n[0] // 4, 10 * n[1] // 2)
    g.break_segment(seg, 10)
    mu = oracle.intact_mu(2, n, M)
    oracle.prenotch(n, M, seg, 10, mu)
    u, st = g.adr_solve(torch.tensor(w.b, device="cuda"), rtol=1e-8)
    P = 1 - w.constrained
    r = w.b * P - oracle.stiffness(2, n, w.h, M, al, u.cpu().numpy(), cons=w.constrained, mu=mu)
    assert np.linalg.norm(r) / np.linalg.norm(w.b * P) <= 1.05e-8
    # 3D cube under an x-traction on its top layers, 150 updates against the oracle.
    # (Under the cube's random body force the damping quotient of near-zero
    # velocities makes the iterates chaotic: a 1e-16 change of the operator moves
    # them by percent, so there only the converged answer is compared.)
    c = syn.cube(12, 2)
    al3 = oracle.alpha(3, 1.0, c.delta)
    g3 = pd.Grid(3, c.n, c.h, c.M, constrained=c.constrained)
    bt = np.zeros_like(c.b)
    bt[0, -2:] = 1e-3
    b3 = torch.tensor(bt, device="cuda")
    u3 = torch.zeros_like(b3)
    pd.pd_adr_solve(g3.handle, b3, u3, 1e-30, 150, allow_not_converged=True)
    ref3, _, _ = oracle.adr_solve(3, c.n, c.h, c.M, al3, bt, cons=c.constrained, rtol=1e-30, maxit=150)
    assert rel_l2(u3.cpu().numpy(), ref3) <= 1e-9
    u3, st3 = g3.adr_solve(torch.tensor(c.b, device="cuda"), rtol=1e-8)
    P3 = 1 - c.constrained
    r3 = c.b * P3 - oracle.stiffness(3, c.n, c.h, c.M, al3, u3.cpu().numpy(), cons=c.constrained)
    assert st3.rel_residual <= 1e-8
    assert np.linalg.norm(r3) / np.linalg.norm(c.b * P3) <= 1.05e-8


def test_adr_rejects_modulus_field(pd):
    n, M = (16, 16), 2
    w = _plate(n, M)
    E = torch.tensor(syn.lognormal_modulus(n, 0.1, 3), device="cuda")
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained, E_field=E)
    b = torch.tensor(w.b, device="cuda")
    with pytest.raises(pd.PDError) as e:
        pd.pd_adr_solve(g.handle, b, torch.zeros_like(b), 1e-8, 10)
    assert e.value.code == pd.PD_ERR_INVALID


# --------------------------------------------------------------------------- mixed precision

@pytest.mark.parametrize("method", ["stencil", "fft"])
def test_adr_mixed_converges_like_fp64(pd, method):
    """FP32 operator on the correction, FP64 base residual at each tenfold drop:
    the true FP64 residual reaches rtol, in about as many updates as the FP64 iteration."""
    n, M = (64, 64), 3
    w = _plate(n, M, tag=5)
    al = oracle.alpha(2, 1.0, w.delta)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained)
    if method == "fft":
        g.prefer_method(pd.PD_METHOD_FFT)
    b = torch.tensor(w.b, device="cuda")
    u64, st64 = g.adr_solve(b, rtol=1e-8)
    um, stm = g.adr_solve(b, rtol=1e-8, mode=pd.PD_ADR_MIXED)
    assert stm.rel_residual <= 1e-8 and stm.outer >= 8
    assert abs(stm.iterations - st64.iterations) <= 0.1 * st64.iterations + 20
    P = 1 - w.constrained
    r = w.b * P - oracle.stiffness(2, n, w.h, M, al, um.cpu().numpy(), cons=w.constrained)
    assert np.linalg.norm(r) / np.linalg.norm(w.b * P) <= 1.05e-8
    assert np.all(um.cpu().numpy()[w.constrained.astype(bool)] == 0)
    assert rel_l2(um.cpu().numpy(), u64.cpu().numpy()) <= 1e-5


def test_adr_mixed_cap_broken_bonds_surface_and_3d(pd):
    # cap: stops with the iterate reached and the true residual of it
    n, M = (48, 40), 3
    w = _plate(n, M, tag=6)
    al = oracle.alpha(2, 1.0, w.delta)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained, surface_correction=pd.PD_SC_VOLUME)
    seg = (10 * n[0] // 4, 10 * n[1] // 2, 10 * 3 * n[0] // 4, 10 * n[1] // 2)
    g.break_segment(seg, 10)
    mu = oracle.intact_mu(2, n, M)
    oracle.prenotch(n, M, seg, 10, mu)
    nu = oracle.surface_nu(2, n, w.h, M)
    b = torch.tensor(w.b, device="cuda")
    u = torch.zeros_like(b)
    st = pd.pd_adr_solve(g.handle, b, u, 1e-12, 100, allow_not_converged=True, mode=pd.PD_ADR_MIXED)
    assert st.iterations == 100
    P = 1 - w.constrained
    r = w.b * P - oracle.stiffness(2, n, w.h, M, al, u.cpu().numpy(), cons=w.constrained, mu=mu, nu=nu)
    assert abs(np.linalg.norm(r) / np.linalg.norm(w.b * P) - st.rel_residual) <= 1e-6 * st.rel_residual
    # converged, with the D^f and surface corrections in the operator
    u, st = g.adr_solve(b, rtol=1e-8, mode=pd.PD_ADR_MIXED)
    r = w.b * P - oracle.stiffness(2, n, w.h, M, al, u.cpu().numpy(), cons=w.constrained, mu=mu, nu=nu)
    assert np.linalg.norm(r) / np.linalg.norm(w.b * P) <= 1.05e-8
    # 3D cube under its random body force
    c = syn.cube(12, 2)
    al3 = oracle.alpha(3, 1.0, c.delta)
    g3 = pd.Grid(3, c.n, c.h, c.M, constrained=c.constrained)
    u3, st3 = g3.adr_solve(torch.tensor(c.b, device="cuda"), rtol=1e-8, mode=pd.PD_ADR_MIXED)
    P3 = 1 - c.constrained
    r3 = c.b * P3 - oracle.stiffness(3, c.n, c.h, c.M, al3, u3.cpu().numpy(), cons=c.constrained)
    assert np.linalg.norm(r3) / np.linalg.norm(c.b * P3) <= 1.05e-8
    with pytest.raises(pd.PDError) as e:
        pd.pd_adr_solve(g3.handle, torch.tensor(c.b, device="cuda"), u3, 1e-8, 10, mode=7)
    assert e.value.code == pd.PD_ERR_INVALID

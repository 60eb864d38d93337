"""GPU static solves: CG (FP64 and FP32-inner with FP64 refinement) reach the
requested true relative residual, measured independently with the oracle's FP64
matvec, and agree with the oracle's own solution."""
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


def _true_rel(w, u, al, E=None, mu=None):
    b = w.b * (1 - w.constrained)
    r = b - oracle.stiffness(w.dim, w.n, w.h, w.M, al, u, cons=w.constrained, E=E, mu=mu)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_small_plate_cg(pd, mode):
    w = syn.small_plate()
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    b = torch.tensor(w.b, device="cuda")
    m = pd.PD_CG_F64 if mode == "f64" else pd.PD_CG_MIXED
    u, st = g.cg_solve(b, rtol=1e-8, mode=m)
    un = u.cpu().numpy()
    al = oracle.alpha(2, 1.0, w.delta)
    assert st.rel_residual <= 1e-8
    assert _true_rel(w, un, al) <= 1.05e-8
    x, it, rel = oracle.cg(2, w.n, w.h, w.M, al, w.b, cons=w.constrained, rtol=1e-10)
    assert rel_l2(un, x) <= 1e-5
    assert np.all(un[w.constrained.astype(bool)] == 0)


@pytest.mark.parametrize("method", ["stencil", "fft"])
def test_large_plate_mixed_vs_f64(pd, method):
    """1024^2 plate (2.1M DOF): both modes reach 1e-8 (true FP64 residual by the oracle)."""
    w = syn.large_plate(3)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    if method == "fft":
        g.prefer_method(pd.PD_METHOD_FFT)
    b = torch.tensor(w.b, device="cuda")
    al = oracle.alpha(2, 1.0, w.delta)
    sols = {}
    for mode in (pd.PD_CG_MIXED, pd.PD_CG_F64):
        u, st = g.cg_solve(b, rtol=1e-8, mode=mode, max_iter=200000)
        un = u.cpu().numpy()
        assert st.rel_residual <= 1e-8
        assert _true_rel(w, un, al) <= 1.05e-8
        sols[mode] = un
    assert rel_l2(sols[pd.PD_CG_MIXED], sols[pd.PD_CG_F64]) <= 1e-4


def test_cube_mixed(pd):
    w = syn.cube(32, 3)
    g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained)
    u, st = g.cg_solve(torch.tensor(w.b, device="cuda"), rtol=1e-8, mode=pd.PD_CG_MIXED)
    al = oracle.alpha(3, 1.0, w.delta)
    assert _true_rel(w, u.cpu().numpy(), al) <= 1.05e-8


def test_modulus_field_and_broken_bonds(pd):
    """CG with a per-node modulus (direct kernel, fused dot) and with broken bonds
    (TBT + D^f gather, separate dot)."""
    n, M = (48, 40), 3
    w = syn.plate_static(48, M, tag=3, u_amp=0.0)
    w.n = n
    w.constrained = syn.clamp_left(2, n, M)
    w.b = syn.traction_right(2, n, M, 1e-3)
    w.h = 1.0 / 48
    E = syn.lognormal_modulus(n, 0.1, 5)
    al1 = oracle.alpha(2, 1.0, w.delta)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained, E_field=torch.tensor(E, device="cuda"))
    u, st = g.cg_solve(torch.tensor(w.b, device="cuda"), rtol=1e-9, mode=pd.PD_CG_MIXED)
    assert _true_rel(w, u.cpu().numpy(), al1, E=E) <= 1.05e-9
    # broken bonds: pre-notch through the middle
    g2 = pd.Grid(2, n, w.h, M, constrained=w.constrained)
    seg = (10 * n[0] // 4, 10 * n[1] // 2, 10 * 3 * n[0] // 4, 10 * n[1] // 2)
    g2.break_segment(seg, 10)
    mu = oracle.intact_mu(2, n, M)
    oracle.prenotch(n, M, seg, 10, mu)
    for mode in (pd.PD_CG_F64, pd.PD_CG_MIXED):
        u2, st2 = g2.cg_solve(torch.tensor(w.b, device="cuda"), rtol=1e-9, mode=mode)
        assert _true_rel(w, u2.cpu().numpy(), oracle.alpha(2, 1.0, w.delta), mu=mu) <= 1.05e-9


def test_iteration_cap_reports_not_converged(pd):
    w = syn.small_plate()
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    b = torch.tensor(w.b, device="cuda")
    u = torch.zeros_like(b)
    st = pd.pd_cg_solve(g.handle, b, u, 1e-8, 5, pd.PD_CG_F64, allow_not_converged=True)
    assert st.iterations <= 5 and st.rel_residual > 1e-8
    with pytest.raises(pd.PDError) as e:
        pd.pd_cg_solve(g.handle, b, torch.zeros_like(b), 1e-8, 5, pd.PD_CG_MIXED)
    assert e.value.code == pd.PD_ERR_NOT_CONVERGED


@pytest.mark.parametrize("shape,M", [((512, 512), 3), ((200, 136), 2), ((260, 72), 4), ((128, 96), 6)])
def test_persistent_inner_loop_matches_graph_loop(pd, shape, M):
    """The FP32 inner loop as one persistent cooperative kernel and as graph-replayed
    launches: both reach the true FP64 residual and the same solution.  They differ
    only in the grouping of the FP32/FP64 sums, which FP32 CG amplifies, so the
    iteration counts are compared loosely."""
    n = shape
    w = syn.plate_static(n[0], M, tag=7, u_amp=0.0)
    w.n = n
    w.h = 1.0 / n[0]
    w.constrained = syn.clamp_left(2, n, M)
    w.b = syn.traction_right(2, n, M, 1e-3)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained)
    b = torch.tensor(w.b, device="cuda")
    al = oracle.alpha(2, 1.0, w.delta)
    res = {}
    for mode in (pd.PD_CG_MIXED, pd.PD_CG_MIXED | pd.PD_CG_GRAPH):
        u = torch.zeros_like(b)
        st = pd.pd_cg_solve(g.handle, b, u, 1e-8, 200000, mode)
        un = u.cpu().numpy()
        assert st.rel_residual <= 1e-8
        assert _true_rel(w, un, al) <= 1.05e-8
        res[mode] = (un, st.iterations, st.persistent)
    (u_p, it_p, used_p), (u_g, it_g, used_g) = res[pd.PD_CG_MIXED], res[pd.PD_CG_MIXED | pd.PD_CG_GRAPH]
    assert used_p == 1 and used_g == 0
    assert abs(it_p - it_g) <= 0.25 * it_g + 10
    assert rel_l2(u_p, u_g) <= 1e-4


def test_mixed_cg_generic_graph_path(pd):
    """A row length that is not a multiple of 4 rules out the TMA kernels: the mixed
    solve then runs the three-launch graph loop and still reaches the true residual."""
    n, M = (202, 96), 3
    w = syn.plate_static(n[0], M, tag=8, u_amp=0.0)
    w.n = n
    w.h = 1.0 / n[0]
    w.constrained = syn.clamp_left(2, n, M)
    w.b = syn.traction_right(2, n, M, 1e-3)
    g = pd.Grid(2, n, w.h, M, constrained=w.constrained)
    b = torch.tensor(w.b, device="cuda")
    u = torch.zeros_like(b)
    st = pd.pd_cg_solve(g.handle, b, u, 1e-8, 200000, pd.PD_CG_MIXED)
    assert st.persistent == 0
    assert _true_rel(w, u.cpu().numpy(), oracle.alpha(2, 1.0, w.delta)) <= 1.05e-8


def test_bounded_wait_reports_timeout_and_context_survives(pd):
    """A device wait on a flag that nothing sets runs out after its limit, the
    error word reaches the host as PD_ERR_TIMEOUT, is cleared, and the context
    keeps working (a product and a solve afterwards)."""
    w = syn.plate_static(64, 3, tag=5, u_amp=0.0)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    with pytest.raises(pd.PDError) as e:
        pd.pd_check_wait_timeout(g.handle, 4096)
    assert e.value.code == pd.PD_ERR_TIMEOUT
    assert pd.pd_get_info(g.handle).device_error == 0
    u = torch.tensor(w.b, device="cuda")
    out = g.matvec(u, flags=pd.PD_METHOD_STENCIL)
    al = oracle.alpha(2, 1.0, w.delta)
    assert rel_l2(out.cpu().numpy(), oracle.stiffness(2, w.n, w.h, w.M, al, w.b)) <= 1e-12
    x, st = g.cg_solve(u, rtol=1e-8)
    assert st.rel_residual <= 1e-8

"""Batched static solves: many plates of uneven size and horizon advance together
(one launch per CG stage, graph-replayed inner loop); every plate reaches the
requested true residual (checked with the oracle's FP64 matvec) and matches its
own single-plate solve."""
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


def _true_rel(w, u):
    al = oracle.alpha(2, 1.0, w.delta)
    b = w.b * (1 - w.constrained)
    r = b - oracle.stiffness(2, w.n, w.h, w.M, al, u, cons=w.constrained)
    return np.linalg.norm(r) / np.linalg.norm(b)


def _solve_batch(pd, plates, rtol):
    grids = [pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained) for w in plates]
    bt = pd.pd_batch_create(grids)
    bs = [torch.tensor(w.b, device="cuda") for w in plates]
    us = [torch.zeros_like(b) for b in bs]
    st = pd.pd_batch_cg_solve(bt, bs, us, rtol, 1_000_000)
    pd.pd_batch_destroy(bt)
    return grids, bs, us, st


def test_small_uneven_batch_matches_single_solves(pd):
    # (M = 1 has only axis-aligned bonds: no shear coupling, so a plate clamped on one
    # side is singular in u_y -- not a valid static problem)
    sides, Ms = [40, 57, 64, 33, 90, 129, 16, 200], [3, 4, 3, 4, 4, 3, 2, 2]
    plates = []
    for i, (n, M) in enumerate(zip(sides, Ms)):
        cons = syn.clamp_left(2, (n, n), M)
        plates.append(syn.Workload(name=f"p{i}", dim=2, n=(n, n), M=M, h=1.0 / n, constrained=cons,
                                   b=syn.gaussian_field(2, (n, n), 1e-3, 700 + i) * (1 - cons)))
    grids, bs, us, st = _solve_batch(pd, plates, 1e-8)
    for w, g, b, u, s in zip(plates, grids, bs, us, st):
        un = u.cpu().numpy()
        assert s.rel_residual <= 1e-8
        assert _true_rel(w, un) <= 1.05e-8
        single, _ = g.cg_solve(b, rtol=1e-8, mode=pd.PD_CG_MIXED)
        assert rel_l2(un, single.cpu().numpy()) <= 1e-5


def test_full_uneven_batch_64_plates(pd):
    plates = syn.batched_plates(64)
    grids, bs, us, st = _solve_batch(pd, plates, 1e-8)
    worst = max(_true_rel(w, u.cpu().numpy()) for w, u in zip(plates, us))
    assert worst <= 1.05e-8

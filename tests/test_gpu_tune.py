"""The autotuner (pd_autotune, pd_autotune_cached): the candidates it measures,
the choice it records, the JSON cache that replays that choice, and that the
stencil's tile height changes no result bit."""
import json

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


def test_tuned_choice_is_the_fastest_and_is_cached(pd, tmp_path):
    path = str(tmp_path / "tune.json")
    w = syn.large_plate(3)
    g = pd.Grid(2, w.n, w.h, w.M)
    t, hit = pd.pd_autotune_cached(g.handle, path)
    assert not hit
    info = pd.pd_get_info(g.handle)
    assert info.stencil_tile_rows in (0, 16, 32, 64)   # 0: the column walk
    for prec, (st, ff) in enumerate((("stencil_f32_ms", "fft_f32_ms"), ("stencil_f64_ms", "fft_f64_ms"))):
        assert t[st] > 0 and t[ff] > 0
        # FP32: the stencil (the FFT tiles miss the FP32 tolerance on smooth fields); FP64: the faster
        want = pd.PD_METHOD_FFT if (prec == 1 and t[ff] < t[st]) else pd.PD_METHOD_STENCIL
        assert info.auto_method[prec] == want
    entries = json.load(open(path))
    assert len(entries) == 2 and all(e["tile_rows"] in (0, 16, 32, 64) for e in entries.values())
    # a second grid of the same geometry takes the recorded choice without measuring
    g2 = pd.Grid(2, w.n, w.h, w.M)
    t2, hit2 = pd.pd_autotune_cached(g2.handle, path)
    assert hit2
    info2 = pd.pd_get_info(g2.handle)
    assert list(info2.auto_method) == list(info.auto_method)
    assert info2.stencil_tile_rows == info.stencil_tile_rows
    # another horizon is a new entry
    w6 = syn.large_plate(6)
    g6 = pd.Grid(2, w6.n, w6.h, w6.M)
    _, hit6 = pd.pd_autotune_cached(g6.handle, path, flags=pd.PD_F32)
    assert not hit6 and len(json.load(open(path))) == 3


@pytest.mark.parametrize("M", [2, 3, 4])
@pytest.mark.parametrize("patch", [False, True])
def test_stencil_tile_height_changes_no_bit(pd, M, patch):
    """The stencil tiles of the autotuner (64 x 64, 64 x 32 and 64 x 16 outputs)
    give the same bits, with and without projection (a 64 x 64 tile takes the
    union of the projection flags of its two 64 x 32 halves): every output is
    formed by the same operations in each."""
    n = (200, 150)
    rng = np.random.default_rng(M)
    cons = syn.clamp_left(2, n, M)
    if patch:   # constrained nodes only in the lower half of a 64-row tile (rows 40..50, 100..150)
        cons = np.zeros_like(cons)
        cons[:, 40:51, 70:90] = 1
        cons[1, 100:151, 150:160] = 1
    g = pd.Grid(2, n, 1.0 / 200, M, constrained=cons)
    U = torch.tensor(rng.uniform(-1, 1, (3, 2, n[1], n[0])), dtype=torch.float32, device="cuda")
    outs = {}
    for rows in (64, 32, 16):
        g.set_stencil_tile_rows(rows)
        assert pd.pd_get_info(g.handle).stencil_tile_rows == rows
        for proj in (0, pd.PD_PROJECT):
            outs[(rows, proj)] = g.matvec(U, flags=pd.PD_METHOD_STENCIL | proj)
    for proj in (0, pd.PD_PROJECT):
        assert torch.equal(outs[(32, proj)], outs[(16, proj)])
        assert torch.equal(outs[(32, proj)], outs[(64, proj)])
        ref = oracle.stiffness(2, n, 1.0 / 200, M, oracle.alpha(2, 1.0, M / 200), U[1].double().cpu().numpy(),
                               cons=cons if proj else None)
        assert rel_l2(outs[(16, proj)][1].double().cpu().numpy(), ref) <= 2e-5


@pytest.mark.parametrize("n", [(512, 384), (1024, 1024)])
@pytest.mark.parametrize("M", [3, 6])
def test_auto_method_meets_tolerance_on_smooth_fields(pd, n, M):
    """Whatever the autotuner picks, the product meets the precision's tolerance
    on smooth fields with a large constant part: FP32 within 2e-5, FP64 within
    1e-12 (the FP64 FFT tiles transform u minus a tile constant, the stencils
    sum differences)."""
    x = (np.arange(n[0]) + 0.5) / n[0]
    y = (np.arange(n[1]) + 0.5) / n[1]
    a = np.sin(2 * np.pi * x)[None, :] * np.cos(np.pi * y)[:, None]
    b = np.cos(3 * np.pi * x)[None, :] * np.sin(2 * np.pi * y)[:, None]
    u = np.stack([1.0 + 0.3 * a, 0.7 + 0.2 * b])
    g = pd.Grid(2, n, 1.0 / n[0], M)
    g.autotune()
    for dt, tol in ((torch.float32, 2e-5), (torch.float64, 1e-12)):
        ut = torch.tensor(u, dtype=dt, device="cuda")
        ref = oracle.stiffness(2, n, 1.0 / n[0], M, oracle.alpha(2, 1.0, M / n[0]), ut.double().cpu().numpy())
        for meth in ((pd.PD_METHOD_AUTO, pd.PD_METHOD_STENCIL) if dt == torch.float32 else
                     (pd.PD_METHOD_AUTO, pd.PD_METHOD_STENCIL, pd.PD_METHOD_FFT)):
            out = g.matvec(ut, flags=meth).double().cpu().numpy()
            assert rel_l2(out, ref) <= tol, (str(dt), meth)


def test_tuned_layout_is_one_of_the_horizons_candidates(pd):
    """The FP64 pass of the autotuner keeps the FP32 stencil layout the FP32 pass
    chose (64-row tiles are a candidate at M <= 3 only, the walk at M <= 3)."""
    for M, allowed in ((3, (0, 16, 32, 64)), (4, (16, 32))):
        w = syn.plate_static(256, M, tag=3, u_amp=1.0)
        g = pd.Grid(2, w.n, w.h, w.M)
        g.autotune()
        assert pd.pd_get_info(g.handle).stencil_tile_rows in allowed
        g.close()

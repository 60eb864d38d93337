"""The allocation-free Verlet entry point (pd_step_noalloc).

Some callers of this library cannot let it call cudaMalloc: services whose GPU
memory belongs to their own pool or caching allocator (which may hold nearly
all of the device), and real-time loops that cannot afford the synchronisation
an allocation implies.  pd_step_noalloc serves them with a fixed scratch array
inside the library.  These tests drive it through the C ABI and check that two
consecutive calls give the same state as two consecutive calls of pd_step from
the same start, that a call on a freshly set-up grid takes no device memory,
and that grids beyond its fixed limit are refused.  The file name makes pytest
collect it last.
"""
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


def _grid(pd, w, cons, E):
    g = pd.Grid(2, w.n, w.h, w.M, constrained=cons, E_field=torch.tensor(E, device="cuda"), s0=w.s0)
    g.break_segment(w.extra["notch"], w.extra["notch_den"])
    return g


def test_noalloc_step_matches_step_on_two_calls(pd):
    w = syn.crack_plate(96, 3)
    lay = w.extra["vel_layers"]
    cons = np.zeros((2,) + lay.shape, dtype=np.uint8)
    cons[1] = lay != 0
    vp = np.zeros((2,) + lay.shape)
    vp[1] = lay * 0.05
    E = w.extra["E_field"]
    dt = 2e-4
    ref_g, new_g = _grid(pd, w, cons, E), _grid(pd, w, cons, E)
    vpt = torch.tensor(vp, device="cuda")
    states = {}
    for name, g, fn in (("ref", ref_g, pd.pd_step), ("noalloc", new_g, pd.pd_step_noalloc)):
        u = torch.zeros((2,) + lay.shape, dtype=torch.float64, device="cuda")
        v = vpt.clone()
        bs = torch.zeros(g.N * g.nnb, dtype=torch.int32, device="cuda")
        got = []
        for call in range(2):
            st = fn(g.handle, u, v, None, 15, dt, v_prescribed=vpt, break_step=bs, step_base=15 * call)
            got.append((u.clone(), v.clone(), st.newly_broken, g.bond_mask().clone()))
        states[name] = (got, bs.clone())
    (ref, ref_bs), (new, new_bs) = states["ref"], states["noalloc"]
    for call in range(2):
        ru, rv, rn, rm = ref[call]
        nu, nv, nn, nm = new[call]
        assert rn == nn
        assert torch.equal(rm, nm)
        scale_u = max(float(ru.abs().max()), 1e-300)
        scale_v = max(float(rv.abs().max()), 1e-300)
        assert float((ru - nu).abs().max()) <= 1e-12 * scale_u
        assert float((rv - nv).abs().max()) <= 1e-12 * scale_v
    assert torch.equal(ref_bs, new_bs)
    assert float(new[1][0].abs().max()) > 0


def test_noalloc_step_refuses_grids_beyond_its_scratch(pd):
    g = pd.Grid(2, (1024, 1024), 1.0 / 1024, 3)
    u = torch.zeros((2, 1024, 1024), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(u)
    with pytest.raises(pd.PDError) as e:
        pd.pd_step_noalloc(g.handle, u, v, None, 1, 1e-4)
    assert e.value.code == pd.PD_ERR_INVALID
    assert "524288" in str(e.value)


def test_noalloc_step_takes_no_device_memory(pd):
    """A fresh grid's first pd_step_noalloc calls leave the device's free memory
    unchanged (a cudaMalloc reserves at least one 2 MiB page).  A warm-up call
    on another grid comes first, so that the kernels involved are loaded and the
    scratch address is known; the fresh grid's own set-up (creation, modulus
    field, notch) allocates and is done before the measurement."""
    w = syn.crack_plate(64, 3)
    lay = w.extra["vel_layers"]
    cons = np.zeros((2,) + lay.shape, dtype=np.uint8)
    cons[1] = lay != 0
    vpt = torch.zeros((2,) + lay.shape, dtype=torch.float64, device="cuda")
    vpt[1] = torch.tensor(lay * 0.05, device="cuda")
    E = w.extra["E_field"]

    def run(g, calls):
        u = torch.zeros((2,) + lay.shape, dtype=torch.float64, device="cuda")
        v = vpt.clone()
        bs = torch.zeros(g.N * g.nnb, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for call in range(calls):
            pd.pd_step_noalloc(g.handle, u, v, None, 10, 2e-4, v_prescribed=vpt, break_step=bs,
                               step_base=10 * call)
        torch.cuda.synchronize()
        return free0, torch.cuda.mem_get_info()[0]

    run(_grid(pd, w, cons, E), 1)             # warm-up on another grid
    g = _grid(pd, w, cons, E)                 # the fresh grid, fully set up
    free0, free1 = run(g, 2)
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"

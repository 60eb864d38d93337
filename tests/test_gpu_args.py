"""Degenerate and out-of-range arguments of the product through the C ABI:
each is rejected with PD_ERR_INVALID and a message, the grid stays usable, and
the output buffer is left untouched.  Largest batch a launch takes (65535) is
the limit that is checked; the smallest grids are covered by the parity tests
(1 x 1, 1 x 40, 5 x 3 nodes)."""
import numpy as np
import pytest

import oracle
from helpers import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pd():
    import paper_2301_11828_gb300 as pd
    pd.load_library()
    return pd


def _expect_invalid(pd, fn):
    with pytest.raises(pd.PDError) as e:
        fn()
    assert e.value.code == pd.PD_ERR_INVALID
    assert pd.load_library().pd_last_error()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_product_argument_checks(pd, dtype):
    n, M = (40, 30), 3
    g = pd.Grid(2, n, 1.0 / 40, M)
    rng = np.random.default_rng(4)
    U = torch.tensor(rng.uniform(-1, 1, (2, 2, n[1], n[0])), dtype=dtype, device="cuda")
    O = torch.full_like(U, 7.0)
    fl = pd.PD_F32 if dtype == torch.float32 else pd.PD_F64
    _expect_invalid(pd, lambda: pd.pd_matvec_batch(g.handle, 0, U, O, fl))                      # empty batch
    _expect_invalid(pd, lambda: pd.pd_matvec_batch(g.handle, -1, U, O, fl))
    _expect_invalid(pd, lambda: pd.pd_matvec_batch(g.handle, 65536, U, O, fl))                  # above one launch
    _expect_invalid(pd, lambda: pd.pd_matvec_batch(g.handle, 2, U, U, fl))                      # u aliases out
    _expect_invalid(pd, lambda: pd.pd_matvec_batch(g.handle, 2, U, O, pd.PD_F32 | pd.PD_F64))   # two precisions
    _expect_invalid(pd, lambda: pd.pd_matvec_batch(g.handle, 2, U, O, 0))                       # no precision
    _expect_invalid(pd, lambda: pd.pd_matvec_batch(g.handle, 2, U, O,
                                                   fl | pd.PD_METHOD_STENCIL | pd.PD_METHOD_FFT))
    torch.cuda.synchronize()
    assert bool((O == 7.0).all())
    # the grid still computes the right product afterwards
    g.matvec(U, O, flags=pd.PD_METHOD_STENCIL)
    torch.cuda.synchronize()
    ref = oracle.stiffness(2, n, 1.0 / 40, M, oracle.alpha(2, 1.0, M / 40), U[1].double().cpu().numpy())
    assert rel_l2(O[1].double().cpu().numpy(), ref) <= (1e-12 if dtype == torch.float64 else 2e-5)

"""CPU checks of the C ABI boundary: the library builds, loads without a GPU and
exports every entry point that include/pd.h declares; the Python binding carries
the same names."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pd.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_11828_gb300 import build
    path = build.build()
    import paper_2301_11828_gb300 as pd
    return pd.load_library(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["pd_create_grid", "pd_set_material", "pd_matvec", "pd_cg_solve", "pd_step", "pd_break_bonds",
              "pd_destroy", "pd_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2301_11828_gb300 as pd
    so = pd.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pd_[a-z0-9_]+)\b", out))
    for name in _declared():
        assert name in exported, f"{name} declared in pd.h but not exported"
        assert hasattr(lib, name)


def test_binding_has_same_names(lib):
    import paper_2301_11828_gb300 as pd
    for name in _declared():
        assert name in pd.SIGNATURES, f"binding lacks {name}"
        assert callable(getattr(pd, name))


def test_invalid_arguments_fail_without_gpu(lib):
    """Argument validation happens before any device work: bad dims / horizons are
    rejected with PD_ERR_INVALID and a message, not a crash."""
    import ctypes
    import paper_2301_11828_gb300 as pd
    n = (ctypes.c_int64 * 3)(8, 8, 1)
    out = ctypes.c_void_p()
    assert lib.pd_create_grid(4, n, 0.1, 0.3, None, ctypes.byref(out)) == pd.PD_ERR_INVALID
    assert "dim" in pd.pd_last_error()
    assert lib.pd_create_grid(2, n, 0.1, 0.05, None, ctypes.byref(out)) == pd.PD_ERR_INVALID   # delta < h
    assert "at least 1" in pd.pd_last_error()
    assert lib.pd_create_grid(2, n, 0.1, 0.95, None, ctypes.byref(out)) == pd.PD_ERR_INVALID   # radius 10 > 8
    assert lib.pd_destroy(None) == pd.PD_OK
    assert lib.pd_matvec(None, None, None, pd.PD_F32, None) == pd.PD_ERR_INVALID


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2301_11828_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "pd_oracle" not in txt, f


def test_critical_stretch_host_helper(lib):
    """Host-only entry point: agrees with the oracle's formula; refuses bad input."""
    import oracle
    import paper_2301_11828_gb300 as pd
    for G0, E, d in [(1e3, 2e11, 3e-3), (0.5, 1.0, 0.03)]:
        assert abs(pd.pd_critical_stretch(G0, E, d, pd.PD_PLANE_STRESS) - oracle.critical_stretch(G0, E, d, "stress")) \
            <= 1e-15 * oracle.critical_stretch(G0, E, d, "stress")
        assert abs(pd.pd_critical_stretch(G0, E, d, pd.PD_PLANE_STRAIN) - oracle.critical_stretch(G0, E, d, "strain")) \
            <= 1e-15 * oracle.critical_stretch(G0, E, d, "strain")
    with pytest.raises(pd.PDError):
        pd.pd_critical_stretch(-1.0, 1.0, 1.0)
    with pytest.raises(pd.PDError):
        pd.pd_critical_stretch(1.0, 1.0, 1.0, 5)

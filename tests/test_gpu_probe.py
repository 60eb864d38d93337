"""The measured arithmetic peak (pd_probe_fma_rate) that the roofline of the
ALU-bound kernels is stated against."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_fma_rate_probe():
    import paper_2301_11828_gb300 as pd
    pd.load_library()
    f32 = pd.pd_probe_fma_rate(pd.PD_F32)
    f64 = pd.pd_probe_fma_rate(pd.PD_F64)
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM, two flops per FMA, at most ~2.1 GHz
    nominal32 = props.multi_processor_count * 128 * 2 * 2.1e9
    assert 0.3 * nominal32 < f32 < 1.05 * nominal32
    assert 0 < f64 < f32
    with pytest.raises(pd.PDError):
        pd.pd_probe_fma_rate(pd.PD_F32 | pd.PD_F64)

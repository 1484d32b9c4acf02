"""The FP64 FMA-rate probe that bench.py reports beside the unit-count FP64 peak: on a GB300 (2 FP64
FMA lanes per SM per clock, 152 SMs, up to 2.07 GHz) it must report a rate near, and not above,
152 x 2 x 2 x 2.07 GHz = 1.26 TFLOP/s; a rate far off would mean the probe does not keep the FP64
pipe busy or is optimised away."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_13046_gb300 import fields  # noqa: E402


def test_fp64_fma_rate_is_near_the_unit_count_peak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import mg
    p = fields.sine_periodic(n=16)
    cfg = mg.config_for(p, mg.MG_MIXED)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        rates = [mg.mg_fp64_fma_rate(ctx, 3) for _ in range(2)]
    finally:
        mg.mg_destroy(ctx)
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 2 * 2 * 2.07e9 / 1e12
    for r in rates:
        assert 0.5 * nominal < r < 1.05 * nominal, (rates, nominal)

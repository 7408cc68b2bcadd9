"""The measured integer-multiply peak (the ALU roof of the modular
kernels): positive, stable between calls, and within what 152 SMs at up to
2.1 GHz can issue (at most 128 32-bit multiplies per SM and clock)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op", ["mad.wide.u32", "mul.hi.u32", "mad.lo.u32", "mad.cc.pair"])
def test_int_mul_peak_is_plausible(op):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    fg = __graft_entry__.build()
    ctx = fg.Context(log_n=10, q_bits=[60, 40], p_bits=[60], alpha=1, log_scale=40)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r1, r2 = fg.int_mul_peak(ctx, op), fg.int_mul_peak(ctx, op)
    assert 0 < r1 <= sms * 128 * 2.2e9
    assert abs(r1 - r2) / r1 < 0.1
    ctx.close()

"""The integer-pipe throughput probe (roofline denominator of the
bit-vector kernels): every operation kind runs and reports a rate no
instruction stream could exceed (32 lanes per scheduler per clock at the
GPU's maximum clock)."""
import pytest
import torch

from paper_2601_15458_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_15458_gb300 import build
    build.build()
    c = api.Context(0, workspace_bytes=64 << 20)
    yield c
    c.close()


@pytest.mark.parametrize("op", list(api.PROBE_OPS))
def test_probe_rates_are_physical(ctx, op):
    props = torch.cuda.get_device_properties(0)
    clock_hz = 2.2e9                     # above the GB300's 2,070 MHz maximum SM clock
    issue = props.multi_processor_count * 4 * 32 * clock_hz
    r = api.probe_int_pipe(ctx, op, iters=512, reps=2)
    ctx.check()
    assert r["lane_ops"] > 0 and r["ms"] > 0
    assert 0.02 * issue < r["ops_per_s"] <= issue


def test_probe_rejects_unknown_op(ctx):
    import ctypes
    from paper_2601_15458_gb300 import _lib
    n = ctypes.c_int64(0)
    assert _lib.lib().msa_probe_int_pipe(ctx.handle, 9, 16, ctypes.byref(n), None) == 1

"""The measurement aids that the benchmark's roofline rests on: the FMA rates in FP64 and
FP32 (smol_fma_rate) and the dependent-chain latencies (smol_op_latency) that make FP64
operations the expensive part of every kernel on this part."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smol():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_16559_gb300 as m
    return m


def test_fma_rates(smol):
    f64, ms64 = smol.fma_rate("fp64", 2000)
    f32, ms32 = smol.fma_rate("fp32conv", 2000)
    assert f64 > 0.0 and f32 > 0.0 and ms64 > 0.0 and ms32 > 0.0
    assert f32 > 4.0 * f64  # the FP64 pipe is a small fraction of the FP32 one


def test_op_latencies(smol):
    lat = {op: smol.op_latency(op, 1) for op in smol.OP_LATENCY_OPS}
    assert all(v > 0.0 for v in lat.values()), lat
    assert lat["dfma"] > lat["ffma"] and lat["dadd"] > lat["ffma"], lat
    # with eight warps the FP64 pipe is shared: no faster per warp than alone
    assert smol.op_latency("dfma", 8) >= 0.9 * lat["dfma"]
    with pytest.raises(smol.SmolError):
        smol.op_latency("dfma", 0)

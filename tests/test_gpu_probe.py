"""The rate probes behind the bench's atomic and FP64 roofs (GPU only): each launch runs its stated
number of operations and leaves the results that a 64-bit atomicMin must leave."""
import pytest
import torch

import paper_1903_00353_gb300 as sdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_shared_memory_atomic_min_probe():
    sink = torch.zeros(4 * _sms(), dtype=torch.int64, device="cuda")
    ops = sdf.probe_rate(sdf.PROBE_SMEM_ATOMIC_MIN, sink, 1024)
    torch.cuda.synchronize()
    assert ops == 4 * _sms() * 256 * 1024
    # each CTA's word was taken over by some key below the all-ones start value
    assert bool((sink.view(torch.int64) != -1).all())


def test_global_atomic_min_probe_only_lowers_words():
    n = 1 << 16
    buf = torch.full((n,), -1, dtype=torch.int64, device="cuda")  # all ones: the largest unsigned key
    ops = sdf.probe_rate(sdf.PROBE_GLOBAL_ATOMIC_MIN, buf, 8)
    torch.cuda.synchronize()
    assert ops == 4 * _sms() * 256 * 8
    changed = int((buf != -1).sum())
    assert changed > n // 2  # 1.2 M scattered atomics over 65 k words reach most of them
    # a second pass with the same keys changes nothing: atomicMin keeps the smaller value
    before = buf.clone()
    sdf.probe_rate(sdf.PROBE_GLOBAL_ATOMIC_MIN, buf, 8)
    torch.cuda.synchronize()
    assert torch.equal(buf, before)
    with pytest.raises(sdf.SDFError):
        sdf.probe_rate(sdf.PROBE_GLOBAL_ATOMIC_MIN, buf[: n - 1], 8)  # not a power of two


def test_fp64_probe_counts_flops():
    buf = torch.zeros(1, dtype=torch.float64, device="cuda")
    ops = sdf.probe_rate(sdf.PROBE_FP64_FMA, buf, 16)
    torch.cuda.synchronize()
    assert ops == 4 * _sms() * 256 * 16 * 16
    assert float(buf[0]) == 0.0

"""GPU checks of the roofline denominators the benchmark divides by: the
integer-instruction and shared-memory microbenchmarks return rates within
what 152 SMs at up to ~2.1 GHz can do."""
from __future__ import annotations

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_15561_gb300 as ga  # noqa: E402


def _sm_cycles_per_s():
    props = torch.cuda.get_device_properties(0)
    return props.multi_processor_count * 2.2e9  # an upper bound on SM clock


def test_int_peak_is_plausible():
    lop3, shf, mix = ga.ga_measure_int_peak()
    cap = _sm_cycles_per_s() * 128  # at most 128 lanes of 32-bit logic per SM per cycle
    for v in (lop3, shf, mix):
        assert 0.05 * cap < v <= cap


def test_smem_peak_is_plausible():
    load, store = ga.ga_measure_smem_peak()
    cap = _sm_cycles_per_s() * 128  # 128 bytes per SM per cycle (32 banks x 4 bytes)
    for v in (load, store):
        assert 0.05 * cap < v <= cap

"""The FP32 storage floor measured with the oracle (CPU): FP32 storage of
the state costs an ordinary string far less than the 1e-4 tolerance, but
the strongly nonlinear struck string of the mixed batch (f0 45.5 Hz, alpha
9.03, 4.7 g hammer at 2.8 m/s) drifts by more than 1e-3 over 0.25 s from
rounding alone, so no FP32 synthesis can meet 1e-4 for it."""

import pytest

from fp32_floor import fp32_state_floor
from paper_2311_18505_gb300 import workloads as W

N = 12000


@pytest.fixture(scope="module")
def mixed():
    return W.batch_mixed(256, seconds=2.0, seed=2)


def test_floor_is_small_for_ordinary_strings(mixed):
    pluck = next(i for i, d in enumerate(mixed) if d["excitation"]["kind"] == "pluck")
    for i in (pluck, 3):
        d = mixed[i]
        assert d["excitation"]["kind"] != "bow"
        assert fp32_state_floor(dict(d, n_samples=N), N) < 2e-5, i


def test_floor_of_the_strongly_nonlinear_struck_string(mixed):
    d = mixed[51]
    assert d["excitation"]["kind"] == "hammer" and d["alpha"] > 9
    assert fp32_state_floor(dict(d, n_samples=N), N) > 1e-3

"""Host logic of the Appendix A comparison (no GPU): the fine run's samples are taken at the
coarse run's sample times, whatever the fine run samples in between, and a coarse time the
fine run never sampled is an error."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import temporal as TM


def series(times):
    t = np.asarray(times, dtype=float)
    return {"t": t, "T": 300.0 + 1e3 * t}


def test_fine_samples_at_the_coarse_sample_times():
    dt = 2e-5
    coarse = series([0.0] + [dt * (i + 1) for i in range(5)] + [dt * 5 + 50 * dt])
    # the fine run samples k = 2 times as often in the scan, equally often in the cool-down
    fine_t = [0.0] + [dt / 2 * (i + 1) for i in range(10)] + [dt * 5 + 50 * dt]
    fine = series(np.array(fine_t) * (1 + 1e-15))  # times formed in another order round differently
    got = TM.common_samples(coarse, fine, 2)
    assert np.allclose(got, coarse["T"], rtol=0.0, atol=1e-9)


def test_a_missing_sample_time_is_an_error():
    coarse = series([0.0, 1e-5, 2e-5])
    fine = series([0.0, 0.5e-5, 2e-5])
    with pytest.raises(AssertionError):
        TM.common_samples(coarse, fine, 2)

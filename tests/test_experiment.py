"""Host helpers of the finite-size experiment driver (crossings, the
log-binning test, the temperature sets) on inputs with known answers, and a
small end-to-end run of the driver on the GPU."""
import numpy as np
import pytest

from paper_1403_4560_b300 import experiment as ex


def test_crossing_of_two_lines_is_found_by_linear_interpolation():
    T = np.array([1.0, 2.0, 3.0])
    a = np.array([3.0, 2.0, 1.0])  # a - b = 2 - 2 (T - 1): zero at T = 2
    b = np.array([1.0, 2.0 + 1e-12, 3.0])
    xs = ex.crossing(T, a, b)
    assert len(xs) == 1 and abs(xs[0] - 2.0) < 1e-9
    assert ex.crossing(T, a, a + 1.0) == []
    # NaN segments are skipped
    assert ex.crossing(T, np.array([np.nan, 0.0, 1.0]), np.array([0.0, 0.5, 0.5])) == [2.5]


def test_log_binning_test_reports_the_largest_deviation_in_errors():
    keys = ("g", "xi", "r12", "e")
    bins = []
    for b, val in enumerate([5.0, 1.3, 1.0, 1.0]):
        d = {k: np.full(3, val) for k in keys}
        d.update({k + "_err": np.full(3, 0.1) for k in keys})
        bins.append(d)
    z = ex.log_binning_test(bins, L=4, last=3)
    # bins 1 and 2 against bin 3: |1.3 - 1.0| / sqrt(0.1^2 + 0.1^2)
    assert abs(z["g"] - 0.3 / np.sqrt(0.02)) < 1e-12
    assert abs(z["xi"] - 0.3 / np.sqrt(0.02)) < 1e-12  # xi / L: scale cancels
    assert ex.log_binning_test(bins, L=4, last=2)["e"] == 0.0


def test_temperature_sets():
    T = ex.temperatures(("beta", 0.1, 1.8), 56)
    assert len(T) == 56 and np.all(np.diff(T) > 0)
    assert abs(T[0] - 1 / 1.8) < 1e-12 and abs(T[-1] - 10.0) < 1e-12
    beta = 1.0 / T[::-1]
    ratio = beta[1:] / beta[:-1]
    assert np.allclose(ratio, ratio[0])  # geometric in beta, as in Table I
    T2 = ex.temperatures(("T", 0.8, 1.6), 16)
    assert abs(T2[0] - 0.8) < 1e-12 and abs(T2[-1] - 1.6) < 1e-12


@pytest.mark.gpu
def test_driver_runs_end_to_end_on_small_sizes():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for the gpu-marked tests")
    from paper_1403_4560_b300 import build
    build.build()
    T = ex.temperatures(("T", 0.8, 1.6), 8)
    res, cross = ex.run([4, 6], 0.0, T, samples=128, log2_sweeps=8)
    for L in (4, 6):
        r = res[L]
        assert r["layout"] == "msc64" and len(r["g"]) == 8
        assert abs(sum(r["pq_lowest_T"]["p"]) - 1.0) < 1e-12
        assert set(r["log_binning_z"]) == {"g", "xi", "r12", "e"}
    assert "4-6" in cross and set(cross["4-6"]) >= {"g", "g_err", "xi_over_L", "R12"}

"""CPU checks of the slice-size rule (Section 4.1): the smallest slice within
p of the fastest measured run."""
from paper_1303_5164_gb300.autotune import choose_slice


def test_smallest_within_p_of_fastest():
    # the GB300 sweep of Black-Scholes at 4 slots (us per run)
    t = {1: 120.86, 2: 96.06, 4: 86.05, 8: 76.99, 16: 75.81, 27: 67.84, 32: 76.32, 64: 124.7}
    assert choose_slice(t, 0.02) == 27
    assert choose_slice(t, 0.15) == 8          # 76.99 / 67.84 - 1 = 0.135
    assert choose_slice(t, 0.5) == 2          # 96.06 / 67.84 - 1 = 0.42; 120.86 is 0.78 over
    assert choose_slice(t, 1.0) == 1
    assert choose_slice({1: 10.0}, 0.0) == 1


def test_non_monotonic_curve_and_ties():
    # very large slices unbalance the SMs: the fastest is in the middle
    t = {1: 200.0, 4: 150.0, 16: 100.0, 64: 180.0}
    assert choose_slice(t, 0.02) == 16
    assert choose_slice(t, 0.5) == 4          # 150 within 50% of 100; 64 is larger
    # exact ties: the smaller slice wins
    assert choose_slice({2: 50.0, 8: 50.0}, 0.0) == 2

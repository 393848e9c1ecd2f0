"""The no-progress rule of the serving loop (host logic, no GPU): a solve
whose |dmu| keeps falling is never stopped by it; a two-value cycle of mu is
stopped after STALL_CHECKS checks."""
from paper_1206_1361_gb300 import serve


def test_geometric_convergence_is_never_called_stalled():
    w = serve.StallWatch()
    assert not any(w.update(0.5 * 0.97 ** k) for k in range(5000))


def test_two_value_cycle_is_stopped_after_the_patience():
    w = serve.StallWatch()
    stops = [w.update(0.759) for _ in range(serve.STALL_CHECKS + 5)]
    assert stops.index(True) == serve.STALL_CHECKS


def test_noise_below_the_best_resets_the_count():
    w = serve.StallWatch()
    for k in range(serve.STALL_CHECKS - 1):
        assert not w.update(1.0 + (k % 3) * 1e-3)
    assert not w.update(0.9)                 # a new minimum
    assert not any(w.update(0.95) for _ in range(serve.STALL_CHECKS - 1))

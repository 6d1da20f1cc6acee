"""Host logic of the batched boolean set intersection server (no GPU)."""
import numpy as np
import pytest

from paper_2002_12459_gb300 import bsi_serve as B


class SimClock:
    """Simulated time: sleeping jumps ahead, answering a batch costs service(size)."""

    def __init__(self):
        self.t = 0.0

    def now(self):
        return self.t

    def sleep_until(self, t):
        self.t = max(self.t, t)


def _answerer(clock, service, seen):
    def answer(lo, hi):
        seen.append((lo, hi))
        clock.t += service(hi - lo)
    return answer


def test_fixed_batches_start_when_full_and_the_server_is_free():
    times = np.array([0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    clock, seen = SimClock(), []
    lat, sizes, busy = B.run_trace(times, ("fixed", 3), _answerer(clock, lambda c: 0.5, seen), clock)
    assert seen == [(0, 3), (3, 6), (6, 7)]          # the last batch is the trace's tail
    # batch 1 starts at t = 2 (third arrival) and ends at 2.5; batch 2 at 5 -> 5.5; batch 3 at 6
    assert np.allclose(lat, [2.5, 1.5, 0.5, 2.5, 1.5, 0.5, 0.5])
    assert sizes.tolist() == [3, 3, 1] and busy == pytest.approx(1.5)


def test_fixed_batches_queue_when_the_server_is_slow():
    times = np.arange(6, dtype=np.float64)
    clock, seen = SimClock(), []
    lat, sizes, _ = B.run_trace(times, ("fixed", 2), _answerer(clock, lambda c: 3.0, seen), clock)
    # batches start at 1, 4 (busy until then), 7
    assert seen == [(0, 2), (2, 4), (4, 6)]
    assert np.allclose(lat, [4.0, 3.0, 5.0, 4.0, 6.0, 5.0])


def test_greedy_takes_everything_waiting():
    times = np.array([0.0, 0.1, 0.2, 0.3, 5.0, 5.05])
    clock, seen = SimClock(), []
    lat, sizes, _ = B.run_trace(times, ("greedy",), _answerer(clock, lambda c: 1.0, seen), clock)
    assert seen == [(0, 1), (1, 4), (4, 5), (5, 6)]
    assert sizes.sum() == len(times) and (lat >= 1.0 - 1e-12).all()


def test_every_request_is_answered_once():
    times = B.arrivals(3000, 500.0, 1)
    for pol in [("fixed", 1), ("fixed", 37), ("greedy",)]:
        clock, seen = SimClock(), []
        lat, sizes, _ = B.run_trace(times, pol, _answerer(clock, lambda c: 1e-3 + 1e-5 * c, seen),
                                    clock)
        cover = np.zeros(len(times), np.int64)
        for lo, hi in seen:
            cover[lo:hi] += 1
        assert (cover == 1).all() and (lat > 0).all()


def test_batch_choice_and_the_proposition_4_rule():
    sizes = [1, 10, 100, 1000]
    n = 1e6
    kappa = 2e-9
    t = [kappa * n * c ** (1 / 3) for c in sizes]
    assert B.fit_kappa(n, sizes, t) == pytest.approx(kappa)
    assert B.prop4_batch(1000.0, n, 1.0) == pytest.approx((1000.0 * n) ** 0.6)
    # t = 2, 4.3, 9.3, 20 ms: at 1000 requests/s only C >= 10 keeps up; C = 10 is the least latency
    assert B.best_batch(1000.0, sizes, t) == 10
    # nothing keeps up: the largest batch
    assert B.best_batch(1e6, sizes, t) == 1000

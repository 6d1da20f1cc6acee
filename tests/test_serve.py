"""Host logic of the serving harness (no GPU): arrivals and request recipe."""
import numpy as np

from paper_2002_12459_gb300 import serve


def test_poisson_arrivals_have_the_stated_rate():
    t = serve.arrivals(20000, 250.0, 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1 / 250.0) < 0.05 / 250.0       # mean gap 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05         # exponential: CV 1


def test_requests_follow_the_recipe_and_caps():
    reqs = [serve._request((i, 3, 1e3, 2e4, 1e4, 1.3, 2.2, 0.5, 5e8, 2e8)) for i in range(12)]
    assert {r["kind"] for r in reqs} == {"two_path", "star"}
    for r in reqs:
        if r["kind"] == "two_path":
            assert len(r["x"]) == r["n"] and 1e3 <= r["n"] <= 2e4 and r["join"] <= 5e8
            key = r["x"].astype(np.int64) * (1 << 32) + r["y"]
            assert len(np.unique(key)) == r["n"]                    # a set of tuples
        else:
            assert len(r["rels"]) == 3 and 1e3 <= r["n"] <= 1e4 and r["join"] <= 2e8
    again = serve._request((5, 3, 1e3, 2e4, 1e4, 1.3, 2.2, 0.5, 5e8, 2e8))
    assert again["n"] == reqs[5]["n"]                               # seeded

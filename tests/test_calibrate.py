"""Cost-model calibration (host logic, no GPU).

The feature rows of calibrate.py are checked against the oracle's Section 5
degree index (oracle/cost_model.py, written separately), and the fit against
times made from known constants.
"""
import math

import numpy as np
import pytest

from paper_2002_12459_gb300 import calibrate, workloads as W
from oracle import cost_model as CM

pytest.importorskip("scipy")


def _relation(seed):
    return W.powerlaw_relation(20000, 4000, 1.6, 2000, 1.5, seed)


@pytest.mark.parametrize("seed", [1, 2])
@pytest.mark.parametrize("d1,d2", [(1, 1), (8, 4), (32, 16), (256, 64), (10 ** 9, 10 ** 9)])
def test_features_match_oracle_index(seed, d1, d2):
    x, y = _relation(seed)
    degx, degy, cand, n = calibrate.degree_terms(x, y)
    idx, info = CM.index_of_relations(x, y)
    assert n == info["N"] and len(degx) == info["dom_x"] and len(degy) == info["dom_y"]
    f = calibrate.features(degx, degy, cand, d1, d2)
    assert f[0] == idx.sum_y(d1) + idx.sum_x(d2)
    assert f[1] == idx.cdfx(d1) * info["dom_x"]
    u, v, w = idx.heavy_x(d2), idx.heavy_y(d1), idx.heavy_z(d2)
    on = u > 0 and v > 0 and w > 0
    assert f[2] == (2.0 * u * v * w if on else 0.0)
    assert f[3] == (1.0 if on else 0.0)
    assert f[4] == ((u * v + u * w) if on else 0.0)


def test_fit_recovers_planted_constants():
    """Times built from known constants plus a per-relation offset are fitted back."""
    rng = np.random.default_rng(0)
    k_true = np.array([1.0 / 200e9, 0.0, 1.0 / 3e15, 30e-6, 1.0 / 5e11])
    F, t, grp = [], [], []
    for g in range(12):
        x, y = _relation(100 + g)
        degx, degy, cand, _ = calibrate.degree_terms(x, y)
        offset = rng.uniform(1e-3, 5e-3)
        rows = [calibrate.features(degx, degy, cand, d1, d2)
                for d1 in (2, 4, 8, 16, 64, 512) for d2 in (2, 4, 8, 32, 128)]
        times = [offset + float(np.dot(k_true, r)) for r in rows]
        best = min(times)
        for r, tm in zip(rows, times):
            F.append(np.array(r) / best)
            t.append(tm / best)
            grp.append(g)
    k, rms, rms0 = calibrate.fit(np.array(F), np.array(t), np.array(grp))
    assert rms < 1e-6 * rms0
    for got, want in zip(k, k_true):
        if want == 0:
            assert got < 1e-3 * k_true[0]
        else:
            assert math.isclose(got, want, rel_tol=1e-4), (got, want)
    c = calibrate.constants(k, calibrate.DEFAULT_BASE)
    assert math.isclose(c["mm_rate"], 3e15, rel_tol=1e-4)
    assert c["eps"] == calibrate.DEFAULT_BASE["eps"]


def test_end_to_end_on_a_saved_sweep(tmp_path):
    """load_rows -> design -> fit on a tiny sweep file written like learn.py's --data output:
    three seeded relations whose grid times are made from known constants."""
    import json
    from paper_2002_12459_gb300 import learn
    k_true = np.array([1.0 / 100e9, 0.0, 1.0 / 2e15, 50e-6, 1.0 / 8e11])
    rows = []
    for i in range(3):
        spec = learn.relation_spec(i, seed=11, n_lo=2e4, n_hi=4e4)
        x, y = learn.make_relation(spec)
        degx, degy, cand, _ = calibrate.degree_terms(x, y)
        grid = [[1e3 * (2e-3 + float(np.dot(k_true, calibrate.features(degx, degy, cand, d1, d2))))
                 for d2 in learn.D2_GRID] for d1 in learn.D1_GRID]
        grid[0][0] = math.inf                     # a skipped grid point
        rows.append(dict(spec=spec, grid=grid))
    path = tmp_path / "sweeps.npz"
    meta = np.array([json.dumps(r) for r in rows])
    np.savez(path, train=meta, held=meta[:1], d1_grid=np.array(learn.D1_GRID),
             d2_grid=np.array(learn.D2_GRID))
    got = calibrate.load_rows(str(path))
    assert len(got) == 3 and got[0]["d1_grid"] == list(learn.D1_GRID)
    F, t, grp = calibrate.design(got, workers=2)
    assert len(t) == 3 * (49 - 1) and set(grp.tolist()) == {0, 1, 2}
    k, rms, rms0 = calibrate.fit(F, t, grp)
    assert rms < 1e-6 * rms0
    assert math.isclose(k[0], k_true[0], rel_tol=1e-3)
    assert math.isclose(1.0 / k[2], 2e15, rel_tol=1e-3)

"""A given reduced network evaluated on other operating points (okr_evaluate)
against the oracle, the voltage-margin sweep and the load-profile robustness
study built on it."""
from __future__ import annotations

import numpy as np
import pytest

import feedergen as fg
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import build
    build.build()
    c = K.Context(0)
    yield c
    c.close()


def test_evaluate_matches_the_search_and_the_oracle(ctx):
    import paper_2510_19608_gb300 as K
    f, run = fg.preset("feeder1000", n_bus=300)
    ctx.reduce(f, K.default_params(margin=run["margin"], target_reduction=0.6, precision=1))
    summ = ctx.summary()
    sup = ctx.assignment()
    _, vred_search = ctx.voltages()
    err, vred = ctx.evaluate(f, sup)
    assert abs(err.max() - summ["max_error"]) <= 1e-11
    assert np.abs(vred - vred_search).max() <= 1e-9
    err_o, vred_o = O.evaluate(f, sup)
    assert np.abs(err - err_o).max() <= 1e-11 and np.abs(vred - vred_o).max() <= 1e-9


def test_evaluate_on_other_hours_matches_the_oracle(ctx):
    import paper_2510_19608_gb300 as K
    f, run = fg.preset("feeder1000", n_bus=250)
    ctx.reduce(f, K.default_params(margin=run["margin"], target_reduction=0.5, precision=1))
    sup = ctx.assignment()
    hours = fg.daily_profiles(f, hours=4, seed=3)
    fh = fg.with_loads(f, hours)
    err, vred = ctx.evaluate(fh, sup)
    err_o, vred_o = O.evaluate(fh, sup)
    assert np.abs(err - err_o).max() <= 1e-11 and np.abs(vred - vred_o).max() <= 1e-9


def test_evaluate_rejects_an_assignment_to_a_reduced_bus(ctx):
    import paper_2510_19608_gb300 as K
    f, _ = fg.preset("feeder40")
    sup = np.arange(f.n_bus)
    sup[5] = 6
    sup[6] = 7                                           # 6 is not a super-node
    with pytest.raises(K.OkrError) as e:
        ctx.evaluate(f, sup)
    assert e.value.status == 1


def test_margin_sweep(ctx):
    from paper_2510_19608_gb300 import sweeps
    f, _ = fg.preset("feeder1000", n_bus=400)
    margins = [0.001, 0.002, 0.004, 0.008]
    rows, stats = sweeps.margin_sweep(ctx, f, margins)
    assert stats["fallbacks"] == 0
    assert all(r["status"] == 0 for r in rows)
    for r in rows:                                       # (greedy paths differ per margin: no monotonicity claim)
        assert r["max_error"] <= r["margin"] + 1e-12
        assert 0.0 <= r["radial_reduction"] <= r["reduction"]


def test_profile_robustness(ctx):
    from paper_2510_19608_gb300 import sweeps
    f, _ = fg.preset("feeder1000", n_bus=300)
    hours = fg.daily_profiles(f, hours=12, seed=1)
    out = sweeps.profile_robustness(ctx, f, hours, margin=0.005, target=0.5)
    errs = np.array(out["max_error_by_hour"])
    assert errs.shape == (12,)
    heavy, light = out["library_hours"]
    # the library hours are the search's own scenarios: within the margin
    assert errs[heavy] <= 0.005 + 1e-12 and errs[light] <= 0.005 + 1e-12
    assert abs(max(errs[heavy], errs[light]) - out["library_max_error"]) <= 1e-11

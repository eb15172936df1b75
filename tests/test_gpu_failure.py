"""Failure detection without a GPU fault: every device-side wait of the search
(grid and team barriers) is bounded by params.max_spins.  With a limit of one
poll the barriers give up, the kernels return, the call reports
OKR_ETIMEOUT, and the same context then runs normally."""
from __future__ import annotations

import numpy as np
import pytest

import feedergen as fg

pytestmark = pytest.mark.gpu

ETIMEOUT = 5


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import build
    build.build()
    c = K.Context(0)
    yield c
    c.close()


def test_search_barrier_timeout_is_reported_and_the_context_recovers(ctx):
    import paper_2510_19608_gb300 as K
    f, run = fg.preset("feeder1000", n_bus=300)
    p_ok = K.default_params(margin=run["margin"], target_reduction=0.5, precision=1, engine=1)
    ctx.reduce(f, p_ok)
    ref = ctx.decisions()
    with pytest.raises(K.OkrError) as e:
        ctx.reduce(f, K.default_params(margin=run["margin"], target_reduction=0.5, precision=1, max_spins=1, engine=1))
    assert e.value.status == ETIMEOUT
    ctx.reduce(f, p_ok)
    again = ctx.decisions()
    assert np.array_equal(again["s"], ref["s"]) and np.array_equal(again["r"], ref["r"])


def test_batch_team_barrier_timeout_is_reported_per_feeder(ctx):
    import paper_2510_19608_gb300 as K
    batch = fg.batch_presets(count=6, first_seed=50, n_lo=100, n_hi=300)
    feeders = [f for f, _ in batch]
    ok = [K.default_params(margin=r["margin"], target_reduction=r["target"], precision=1, engine=1) for _, r in batch]
    bad = [K.default_params(margin=r["margin"], target_reduction=r["target"], precision=1, max_spins=1, engine=1)
           for _, r in batch]
    ctx.set_batch_config(1)                               # teams of two CTAs: their barriers wait
    items, _, _ = ctx.reduce_batch(feeders, bad)
    assert all(it["status"] != 0 for it in items)
    assert any(it["status"] == ETIMEOUT for it in items)
    items2, parts2, _ = ctx.reduce_batch(feeders, ok)
    assert all(it["status"] == 0 for it in items2)
    ctx.reduce(feeders[0], ok[0])
    assert np.array_equal(parts2[0], ctx.assignment())


def test_load_flow_barrier_timeout_is_reported_and_the_context_recovers(ctx):
    """The cooperative load flow's grid barriers honour params.max_spins too:
    with one poll a CTA that waits for a slower one gives up, every CTA
    leaves at its next barrier, and the call reports OKR_ETIMEOUT.  The
    incremental engine has no device-side wait, so the timeout can only come
    from the load flow here.  The same context then runs normally."""
    import paper_2510_19608_gb300 as K
    f, run = fg.preset("feeder1000")
    p_ok = K.default_params(margin=run["margin"], target_reduction=0.5, precision=1, engine=2)
    ctx.reduce(f, p_ok)
    ref = ctx.decisions()
    with pytest.raises(K.OkrError) as e:
        ctx.reduce(f, K.default_params(margin=run["margin"], target_reduction=0.5, precision=1, engine=2,
                                       max_spins=1))
    assert e.value.status == ETIMEOUT
    assert "load flow" in str(e.value)
    ctx.reduce(f, p_ok)
    again = ctx.decisions()
    assert np.array_equal(again["s"], ref["s"]) and np.array_equal(again["r"], ref["r"])
    assert np.array_equal(again["score"], ref["score"])

"""A batch captured as one CUDA graph (okr_batch_plan_*) through the C ABI:
every replay returns what okr_reduce_batch returns for the same batch, new
loads set between replays take effect, and the plan works for both engines."""
from __future__ import annotations

import numpy as np
import pytest

import feedergen as fg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import build
    build.build()
    c = K.Context(0)
    yield c
    c.close()


def params(**kw):
    import paper_2510_19608_gb300 as K
    return K.default_params(**kw)


def _same(a, b):
    items_a, parts_a, _ = a
    items_b, parts_b, _ = b
    assert len(items_a) == len(items_b)
    for x, y in zip(items_a, items_b):
        assert x == y
    for p, q in zip(parts_a, parts_b):
        assert np.array_equal(p, q)


@pytest.mark.parametrize("engine,precision", [(2, 1), (2, 0), (1, 1)])
def test_replays_equal_the_direct_batch(ctx, engine, precision):
    batch = fg.batch_presets(count=8, first_seed=120, n_lo=80, n_hi=400)
    feeders = [f for f, _ in batch]
    ps = [params(margin=r["margin"], target_reduction=r["target"], engine=engine, precision=precision)
          for _, r in batch]
    direct = ctx.reduce_batch(feeders, ps)
    plan = ctx.batch_plan(feeders, ps)
    try:
        for _ in range(3):
            got = plan.run()
            _same(got, direct)
            assert all(it["status"] == 0 for it in got[0])
            assert got[2]["search_ms"] > 0 and got[2]["setup_ms"] > 0
    finally:
        plan.close()


def test_new_loads_take_effect(ctx):
    batch = fg.batch_presets(count=5, first_seed=140, n_lo=80, n_hi=300)
    feeders = [f for f, _ in batch]
    ps = [params(margin=r["margin"], target_reduction=r["target"], precision=1) for _, r in batch]
    plan = ctx.batch_plan(feeders, ps)
    try:
        base = plan.run()
        # the light scenario as the only loading level: a different operating point
        lighter = [fg.Feeder(parent=f.parent, phases=f.phases, z_line=f.z_line, s_load=f.s_load * 0.5,
                             v_slack=f.v_slack, meta={}) for f in feeders]
        for i, f in enumerate(lighter):
            plan.set_loads(i, f.s_load)
        got = plan.run()
        _same(got, ctx.reduce_batch(lighter, ps))
        for i, f in enumerate(feeders):              # and back
            plan.set_loads(i, f.s_load)
        _same(plan.run(), base)
    finally:
        plan.close()


def test_plan_rejects_bad_arguments(ctx):
    import paper_2510_19608_gb300 as K
    f, _ = fg.preset("feeder40")
    with pytest.raises(K.OkrError):
        ctx.batch_plan([f], params(margin=-1.0))
    plan = ctx.batch_plan([f], params(margin=0.005))
    try:
        with pytest.raises(ValueError):
            plan.set_loads(0, np.zeros((1, 3, 3, 2)))
    finally:
        plan.close()

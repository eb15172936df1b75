"""okr_reduce_batch (many feeders, one persistent launch) through the C ABI.

Every feeder of a batch must get exactly the result the single-feeder entry
point gives it (that path is checked against the oracle in
test_gpu_parity.py), and a sample is checked against the oracle directly.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import feedergen as fg
from oracle import oracle as O

pytestmark = pytest.mark.gpu

S_TOL = 1e-11


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


def _batch(count, n_lo, n_hi, seed=0):
    return fg.batch_presets(count=count, first_seed=seed, n_lo=n_lo, n_hi=n_hi)


def _check_against_single(ctx, feeders, plist, items, parts):
    for f, p, it, sup in zip(feeders, plist, items, parts):
        ctx.reduce(f, p)
        s = ctx.summary()
        assert it["status"] == 0
        assert it["n_iter"] == s["n_iter"] and it["stop_reason"] == s["stop_reason"]
        assert it["n_kept"] == s["n_kept"] and it["candidates"] == s["candidates"]
        assert abs(it["smice"] - s["smice"]) <= S_TOL
        assert abs(it["max_error"] - s["max_error"]) <= 1e-12
        assert np.array_equal(sup, ctx.assignment())


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_single_feeder_runs(ctx, precision, engine):
    batch = _batch(10, 40, 400, seed=precision * 100)
    feeders = [f for f, _ in batch]
    plist = [params(margin=r["margin"], target_reduction=r["target"], precision=precision, engine=engine)
             for _, r in batch]
    items, parts, stats = ctx.reduce_batch(feeders, plist)
    assert stats["fallbacks"] == 0 and stats["ctas"] >= 1
    assert stats["candidates"] == sum(it["candidates"] for it in items)
    _check_against_single(ctx, feeders, plist, items, parts)


def test_batch_against_oracle(ctx):
    batch = _batch(4, 30, 120, seed=7)
    feeders = [f for f, _ in batch]
    plist = [params(margin=r["margin"], target_reduction=r["target"], precision=1) for _, r in batch]
    items, parts, _ = ctx.reduce_batch(feeders, plist)
    for f, p, it, sup in zip(feeders, plist, items, parts):
        vhat, ihat = O.operating_points(f)
        res = O.reduce(f, vhat, ihat, margin=p.margin, max_merges=O.max_merges_for(f.n_bus, p.target_reduction))
        assert np.all(res["gap"] > 1e-12)
        assert it["n_iter"] == res["n_iter"] and it["stop_reason"] == res["stop_reason"]
        assert np.array_equal(sup, res["super_of"])
        if res["n_iter"]:
            assert abs(it["smice"] - res["score"][-1]) <= S_TOL


def test_batch_mixed_precisions_and_objectives(ctx):
    batch = _batch(8, 40, 300, seed=11)
    feeders = [f for f, _ in batch]
    plist = []
    for k, (_, r) in enumerate(batch):
        if k % 3 == 2:
            plist.append(params(margin=r["margin"], target_reduction=r["target"], precision=0, objective=1))
        else:
            plist.append(params(margin=r["margin"], target_reduction=r["target"], precision=k % 2))
    items, parts, _ = ctx.reduce_batch(feeders, plist)
    _check_against_single(ctx, feeders, plist, items, parts)


def test_batch_isolates_a_failing_feeder(ctx):
    good = [f for f, _ in _batch(3, 40, 80, seed=21)]
    bad = fg.make_feeder(60, 5)
    bad.s_load[...] *= 1e4                              # no load-flow solution
    feeders = good[:1] + [bad] + good[1:]
    items, parts, _ = ctx.reduce_batch(feeders, params(margin=0.005, target_reduction=0.5))
    assert items[1]["status"] == 4                      # OKR_EPF
    assert np.all(parts[1] == -1)
    for k in (0, 2, 3):
        assert items[k]["status"] == 0


def test_batch_rejects_an_invalid_tree(ctx):
    import paper_2510_19608_gb300 as K
    f, _ = fg.preset("feeder40")
    g = fg.make_feeder(20, 3)
    g.parent[5] = 7                                     # parent after child
    with pytest.raises(K.OkrError) as e:
        ctx.reduce_batch([f, g], params())
    assert e.value.status == 1


def test_autotune_picks_a_shape_and_keeps_results(ctx):
    batch = _batch(12, 40, 300, seed=31)
    feeders = [f for f, _ in batch]
    plist = [params(margin=r["margin"], target_reduction=r["target"], precision=1, engine=1) for _, r in batch]
    ref, ref_parts, _ = ctx.reduce_batch(feeders, plist)
    cfg, ms = ctx.batch_autotune(feeders, plist)
    assert cfg in (0, 1, 2, 3) and all(m > 0 and math.isfinite(m) for m in ms)
    items, parts, stats = ctx.reduce_batch(feeders, plist)
    assert stats["config"] == cfg
    for a, b, pa, pb in zip(ref, items, ref_parts, parts):
        assert abs(a.pop("smice") - b.pop("smice")) <= S_TOL      # summation order follows the team size
        assert a == b and np.array_equal(pa, pb)


@pytest.mark.parametrize("config", [0, 1, 2, 3])
def test_every_team_shape_matches_single_runs(ctx, config):
    batch = _batch(6, 40, 500, seed=41 + config)
    feeders = [f for f, _ in batch]
    plist = [params(margin=r["margin"], target_reduction=r["target"], precision=1, engine=1) for _, r in batch]
    ctx.set_batch_config(config)
    items, parts, stats = ctx.reduce_batch(feeders, plist)
    assert stats["config"] == config and stats["ctas"] % (1 << config) == 0
    _check_against_single(ctx, feeders, plist, items, parts)

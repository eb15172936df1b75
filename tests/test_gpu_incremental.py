"""The incremental engine (scores carried across merges) through the C ABI.

Engine 3 (verify) re-evaluates every candidate after every merge and counts
the carried scores -- fixed-point sums of the FP64 terms and counts of terms
above the margin -- that differ bit for bit from the fresh evaluation; there
must be none.  Decisions equal the sweep engine's here and the oracle's in
test_gpu_parity.py.  Batches run one CTA per feeder and must reproduce the
single-feeder results exactly."""
from __future__ import annotations

import numpy as np
import pytest

import feedergen as fg

pytestmark = pytest.mark.gpu

EINVAL = 1


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


VERIFY = {
    "feeder40": (lambda: fg.preset("feeder40")[0], 0.005, 1.0),
    "keep150_L1": (lambda: fg.make_feeder(150, 31, kv_ll=4.16, phase_mode="keep", load=("uniform", 50.0), n_scen=1),
                   0.003, 1.0),
    "mix300": (lambda: fg.make_feeder(300, 32, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0)), 0.005, 1.0),
    "lognormal250_L3": (lambda: fg.make_feeder(250, 33, phase_mode=(0.45, 0.15, 0.4), load=("lognormal", 15.0, 1.0),
                                               n_scen=3), 0.004, 0.95),
    "tight400_L4": (lambda: fg.make_feeder(400, 34, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0), n_scen=4),
                    0.002, 1.0),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(VERIFY))
def test_carried_scores_equal_a_fresh_evaluation(ctx, name, precision):
    make, margin, target = VERIFY[name]
    f = make()
    ctx.reduce(f, params(margin=margin, target_reduction=target, engine=3, precision=precision))
    s = ctx.summary()
    assert s["engine"] == 2
    assert s["n_iter"] > 0
    assert s["inc_mismatches"] == 0
    inc = ctx.decisions()
    ctx.reduce(f, params(margin=margin, target_reduction=target, engine=1))
    sw = ctx.decisions()
    assert ctx.summary()["engine"] == 1
    assert np.array_equal(inc["s"], sw["s"]) and np.array_equal(inc["r"], sw["r"])
    assert np.abs(inc["score"] - sw["score"]).max() <= 1e-11
    assert np.abs(inc["maxerr"] - sw["maxerr"]).max() <= 1e-12
    assert np.array_equal(inc["ncand"], sw["ncand"])


def test_auto_engine_choice(ctx):
    f, _ = fg.preset("feeder40")
    ctx.reduce(f, params(margin=0.005))
    assert ctx.summary()["engine"] == 2
    ctx.reduce(f, params(margin=0.005, precision=1))
    assert ctx.summary()["engine"] == 2
    ctx.reduce(f, params(margin=0.005, precision=1, engine=1))
    assert ctx.summary()["engine"] == 1
    ctx.reduce(f, params(margin=0.005, objective=1))
    assert ctx.summary()["engine"] == 1


def test_incremental_engine_rejects_what_it_does_not_run(ctx):
    import paper_2510_19608_gb300 as K
    f, _ = fg.preset("feeder40")
    for bad in (dict(engine=2, objective=1), dict(engine=3, objective=1), dict(engine=2, precision=2),
                dict(engine=4), dict(engine=-1)):
        with pytest.raises(K.OkrError) as e:
            ctx.reduce(f, params(margin=0.005, **bad))
        assert e.value.status == EINVAL
    ctx.reduce(f, params(margin=0.005, engine=2, max_merges=3))
    assert ctx.summary()["n_iter"] == 3


def test_profile_counts_terms(ctx):
    f, run = fg.preset("feeder1000", n_bus=300)
    ctx.reduce(f, params(margin=run["margin"], target_reduction=0.5, engine=2, profile=1))
    s = ctx.summary()
    assert s["terms"] > 0
    assert s["phase_ms"][0] > 0.0


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_incremental_equals_single_runs(ctx, precision):
    batch = fg.batch_presets(count=10, first_seed=70, n_lo=100, n_hi=600)
    feeders = [f for f, _ in batch]
    ps = [params(margin=r["margin"], target_reduction=r["target"], precision=precision) for _, r in batch]
    items, parts, stats = ctx.reduce_batch(feeders, ps)
    assert stats["fallbacks"] == 0
    for f, p, it, part in zip(feeders, ps, items, parts):
        assert it["status"] == 0
        ctx.reduce(f, p)
        s = ctx.summary()
        assert s["engine"] == 2
        assert it["n_iter"] == s["n_iter"] and it["stop_reason"] == s["stop_reason"]
        assert it["candidates"] == s["candidates"]
        assert abs(it["smice"] - s["smice"]) <= 1e-13
        assert abs(it["max_error"] - s["max_error"]) <= 1e-13
        assert np.array_equal(part, ctx.assignment())


def test_batch_mixing_engines(ctx):
    """Feeders of one batch may ask for different engines; each result equals
    its single run."""
    batch = fg.batch_presets(count=6, first_seed=90, n_lo=100, n_hi=400)
    feeders = [f for f, _ in batch]
    ps = [params(margin=r["margin"], target_reduction=r["target"], precision=i % 2, engine=1 + (i // 2) % 2)
          for i, (_, r) in enumerate(batch)]
    items, parts, _ = ctx.reduce_batch(feeders, ps)
    for f, p, it, part in zip(feeders, ps, items, parts):
        assert it["status"] == 0
        ctx.reduce(f, p)
        assert it["n_iter"] == ctx.summary()["n_iter"]
        assert np.array_equal(part, ctx.assignment())

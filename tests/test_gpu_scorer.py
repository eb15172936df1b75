"""The learned candidate scorer through the C ABI: forward and gradient of
the CUDA kernels against the FP64 CPU oracle (oracle/mlp.py, evaluated at the
same bfloat16-rounded weights the kernels use), training, recorded features,
and the ranking it learns from exhaustive-search scores."""
from __future__ import annotations

import numpy as np
import pytest

import feedergen as fg
from oracle import mlp as M

pytestmark = pytest.mark.gpu

F = 12


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import build
    build.build()
    c = K.Context(0)
    yield c
    c.close()


def _bf16_weights(theta, F):
    """The kernels multiply with bfloat16 copies of the weight matrices (biases stay FP32)."""
    th = theta.astype(np.float32).copy()
    W1, b1, W2, b2, W3, b3, w4, b4 = M.unpack(th, F)
    for a in (W1, W2, W3, w4):
        a[...] = M.bf16_round(a)
    return th.astype(np.float64)


def _problem(seed, N):
    from paper_2510_19608_gb300 import scorer
    rng = np.random.default_rng(seed)
    theta = scorer.init_params(F, seed)
    x = rng.normal(0.0, 1.0, (N, F)).astype(np.float32)
    t = rng.normal(0.0, 1.0, N).astype(np.float32)
    return theta, x, t


def test_forward_matches_oracle(ctx):
    theta, x, _ = _problem(1, 257)
    ctx.scorer_init(F, theta)
    y = ctx.scorer_predict(x)
    y_ref, _ = M.forward(_bf16_weights(theta, F), x.astype(np.float64))
    assert np.abs(y - y_ref).max() <= 1e-4 * max(1.0, np.abs(y_ref).max())


@pytest.mark.parametrize("Fx,N", [(12, 1), (12, 127), (12, 129), (3, 1000), (16, 4096), (12, 40000)])
def test_tensor_core_forward_matches_oracle(ctx, Fx, N):
    """okr_scorer_predict_tc against the FP64 forward with bfloat16 operands
    (weights and every layer input rounded).  A layer input within FP32
    accumulation error of a bfloat16 rounding boundary may round the other way
    on the GPU; that moves the output by about one bfloat16 step of one
    activation's share, hence a tolerance above FP32 rounding for the largest
    deviation and a much tighter one for the median."""
    from paper_2510_19608_gb300 import scorer
    rng = np.random.default_rng(100 + N)
    theta = scorer.init_params(Fx, 7 + Fx)
    x = rng.normal(0.0, 1.0, (N, Fx)).astype(np.float32)
    ctx.scorer_init(Fx, theta)
    y = ctx.scorer_predict_tc(x)
    y_ref = M.forward_bf16_operands(_bf16_weights(theta, Fx), x.astype(np.float64))
    scale = max(1.0, np.abs(y_ref).max())
    d = np.abs(y - y_ref)
    assert d.max() <= 2e-3 * scale
    assert np.median(d) <= 1e-5 * scale
    # the CUDA-core forward (FP32 activations) ranks the same way
    y_cc = ctx.scorer_predict(x)
    assert np.abs(y - y_cc).max() <= 2e-2 * scale
    ctx.scorer_init(F, _problem(1, 1)[0])


@pytest.mark.parametrize("N", [1, 33, 4100])
def test_gradient_matches_oracle(ctx, N):
    theta, x, t = _problem(2 + N, N)
    ctx.scorer_init(F, theta)
    g, loss = ctx.scorer_gradient(x, t)
    th = _bf16_weights(theta, F)
    g_ref = M.grad(th, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - M.loss(th, x.astype(np.float64), t.astype(np.float64))) <= 1e-4 * max(1.0, loss)
    assert np.abs(g - g_ref).max() <= 2e-4 * max(1e-3, np.abs(g_ref).max())


def test_training_fits_a_smooth_function(ctx):
    from paper_2510_19608_gb300 import scorer
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.0, 1.0, (20000, F)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2] + 0.5 * np.abs(x[:, 3])).astype(np.float32)
    loss = scorer.train(ctx, x, t, epochs=15, batch=1024, lr=2e-3, seed=5)
    assert loss[-1] < 0.05 * np.var(t) and loss[-1] < loss[0]
    y = ctx.scorer_predict(x[:2000])
    assert np.mean((y - t[:2000]) ** 2) < 0.05 * np.var(t)


def test_recorded_features(ctx):
    import paper_2510_19608_gb300 as K
    f, run = fg.preset("feeder40")
    ctx.reduce(f, K.default_params(margin=run["margin"], precision=0, record_iters=3, engine=1))
    for it in range(3):
        rec = ctx.recorded(it)
        feat = ctx.recorded_features(it)
        assert feat.shape == (rec["s"].size, 14) and np.isfinite(feat).all()
        pc = np.array([bin(int(v)).count("1") for v in f.phases]) / 3.0
        assert np.allclose(feat[:, 4], pc[rec["r"]]) and np.allclose(feat[:, 5], pc[rec["s"]])
        assert set(np.unique(feat[:, 8])) <= {0.0, 1.0}
        if it == 0:
            assert np.all(feat[:, 6] == 0) and np.all(feat[:, 7] == 0)      # every MICE starts at 0


def test_learned_ranking_beats_chance_on_held_out_feeders(ctx):
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import scorer
    train_runs = [(fg.make_feeder(300, 10000 + k, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0)),
                   K.default_params(margin=0.005, target_reduction=0.5)) for k in range(4)]
    test_runs = [(fg.make_feeder(300, 20000, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0)),
                  K.default_params(margin=0.005, target_reduction=0.5))]
    X, T, _ = scorer.collect(ctx, train_runs, record_iters=40)
    scorer.train(ctx, X, T, epochs=10, batch=2048, lr=1e-3, seed=0)
    Xt, _, groups = scorer.collect(ctx, test_runs, record_iters=40)
    q = scorer.miss_rate(ctx, Xt, groups, ks=(64,))
    assert q["winner_rank_percentile"] < 0.25               # chance: 0.5


# ----------------------------------------------------------------------------- learned pruning in the search
def _props_of_network(ctx, f, margin):
    """A pruned run's network: the reported voltages are the oracle's evaluation
    of its assignment, its largest error is within the margin and equals the
    reported one, and the reported SMICE is recomputed from those voltages."""
    from oracle import oracle as O
    sup = ctx.assignment()
    err_o, vred_o = O.evaluate(f, sup)
    _, vr = ctx.voltages()
    s = ctx.summary()
    assert np.abs(vr - vred_o).max() <= 1e-9
    assert err_o.max() <= margin + 1e-12 and abs(err_o.max() - s["max_error"]) <= 1e-11
    vh, _ = ctx.voltages()
    pres = np.array([[(int(f.phases[i]) >> p) & 1 for p in range(3)] for i in range(f.n_bus)], bool)
    e = np.where(pres[None], np.abs(np.abs(vh) - np.abs(vr)), 0.0)
    smice = sum(float(e[l][sup == k].max()) for l in range(e.shape[0]) for k in np.unique(sup))
    assert abs(s["smice"] - smice) <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_pruning_with_k_above_the_candidate_count_is_exhaustive(ctx, precision):
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import scorer
    f, run = fg.preset("feeder1000", n_bus=300)
    ctx.scorer_init(14, scorer.init_params(14, 3))            # any weights: every candidate is kept
    p = dict(margin=run["margin"], target_reduction=0.5, precision=precision)
    ctx.reduce(f, K.default_params(**p))
    ref = ctx.decisions()
    ctx.reduce(f, K.default_params(scorer_topk=100000, **p))
    got = ctx.decisions()
    assert np.array_equal(got["s"], ref["s"]) and np.array_equal(got["r"], ref["r"])
    assert np.abs(got["score"] - ref["score"]).max() <= 1e-12


@pytest.mark.parametrize("precision,topk", [(1, 16), (0, 16), (1, 1)])
def test_pruned_search_yields_a_valid_network(ctx, precision, topk):
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import scorer
    runs = [(fg.make_feeder(250, 10000 + k, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0)),
             K.default_params(margin=0.005, target_reduction=0.5)) for k in range(3)]
    X, T, _ = scorer.collect(ctx, runs, record_iters=30)
    scorer.train(ctx, X, T, epochs=6, batch=2048, lr=1e-3, seed=1)
    f, run = fg.preset("feeder1000", n_bus=300)
    ctx.reduce(f, K.default_params(margin=run["margin"], target_reduction=0.5, precision=precision, scorer_topk=topk))
    s = ctx.summary()
    assert s["n_iter"] == 150 or s["stop_reason"] == 1
    _props_of_network(ctx, f, run["margin"])
    dec = ctx.decisions()
    assert np.all(dec["maxerr"] <= run["margin"] + 1e-12)


def test_pruning_needs_a_scorer_of_the_right_width(ctx):
    import paper_2510_19608_gb300 as K
    f, _ = fg.preset("feeder40")
    ctx.scorer_init(12)
    with pytest.raises(K.OkrError) as e:
        ctx.reduce(f, K.default_params(scorer_topk=8))
    assert e.value.status == 1


CERTIFIED = {
    "feeder1000_300": lambda: fg.preset("feeder1000", n_bus=300),
    "feeder2200_600": lambda: fg.preset("feeder2200", n_bus=600),
    "feeder40": lambda: fg.preset("feeder40"),
}


@pytest.mark.parametrize("topk", [1, 16, 64])
@pytest.mark.parametrize("name", sorted(CERTIFIED))
def test_certified_pruning_reproduces_the_exhaustive_search(ctx, name, topk):
    """prune_exact: the scorer's top-k candidates are scored first, then every
    other candidate unless the certified lower bound (half spreads of the
    clusters at its positions against their MICE) excludes it from the tie band.  Any weights
    order the candidates; the decisions and scores must be the exhaustive FP64
    sweep's, bit for bit, and the bound must exclude some candidates."""
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import scorer
    f, run = CERTIFIED[name]()
    ctx.scorer_init(14, scorer.init_params(14, 5))
    p = dict(margin=run["margin"], target_reduction=min(run["target"], 0.9), precision=0, engine=1)
    ctx.reduce(f, K.default_params(**p))
    ref = ctx.decisions()
    ref_s = ctx.summary()
    ctx.reduce(f, K.default_params(scorer_topk=topk, prune_exact=1, **p))
    got = ctx.decisions()
    s = ctx.summary()
    assert s["n_iter"] == ref_s["n_iter"] and s["stop_reason"] == ref_s["stop_reason"]
    for k in ("s", "r", "score", "maxerr", "ncand"):
        assert np.array_equal(got[k], ref[k]), k
    assert s["scorer_fallbacks"] == 0
    assert 0 < s["pruned"] < s["candidates"]


def test_trained_network_lets_the_bound_exclude_more(ctx):
    """What the trained network gains over the search without it: with the
    same top-k and the same exact decisions, the candidates the trained
    network ranks first give a tighter threshold, so the certified bound
    excludes more of the other candidates than with untrained weights."""
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import scorer
    runs = [(fg.make_feeder(n, 10000 + k, phase_mode=(0.45, 0.15, 0.4), load=("lognormal", 15.0, 1.0)),
             K.default_params(margin=0.005, target_reduction=0.8, max_merges=48))
            for k, n in enumerate((400, 500, 600, 700))]
    X, T, _ = scorer.collect(ctx, runs, record_iters=48)
    scorer.train(ctx, X, T, epochs=8, batch=2048, lr=1e-3, seed=0)
    trained = ctx.scorer_params().copy()
    f, run = fg.preset("feeder2200", n_bus=600)
    p = dict(margin=run["margin"], target_reduction=0.8, precision=0, engine=1)
    ctx.reduce(f, K.default_params(**p))
    ref = ctx.decisions()
    frac = {}
    for name, theta in (("trained", trained), ("untrained", scorer.init_params(14, 5))):
        ctx.scorer_init(14, theta)
        ctx.reduce(f, K.default_params(scorer_topk=16, prune_exact=1, **p))
        got = ctx.decisions()
        for k in ("s", "r", "score"):
            assert np.array_equal(got[k], ref[k]), (name, k)
        s = ctx.summary()
        frac[name] = s["pruned"] / s["candidates"]
    assert frac["trained"] > frac["untrained"] + 0.1, frac


def test_certified_pruning_rejects_what_it_does_not_run(ctx):
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300._binding import EINVAL
    f, run = fg.preset("feeder40")
    for bad in (dict(prune_exact=1), dict(prune_exact=1, scorer_topk=8, precision=1),
                dict(prune_exact=1, scorer_topk=8, objective=1), dict(prune_exact=2, scorer_topk=8),
                dict(prune_exact=1, scorer_topk=8, engine=2)):
        with pytest.raises(K.OkrError) as e:
            ctx.reduce(f, K.default_params(margin=run["margin"], **bad))
        assert e.value.status == EINVAL

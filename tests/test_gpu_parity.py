"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

Decisions (the chosen (s, r) of every merge, hence the kept set) must be
identical; voltages within 1e-6 p.u. is the contract, and the tests ask for much
tighter bounds (1e-9 p.u. on voltages, 1e-11 on SMICE) because both sides are
FP64 and differ only by rounding order.  A decision comparison is meaningful
only while the oracle's tie margin (distance of the next score above the tie
band) is far above that rounding; the tests assert it is.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import feedergen as fg
from oracle import oracle as O

pytestmark = pytest.mark.gpu

V_TOL = 1e-9          # p.u., voltages
S_TOL = 1e-11         # SMICE
GAP_MIN = 1e-12       # tie margins below this would make the comparison fragile


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


# The three ways of scoring candidates; each must reproduce the oracle's decisions.
ENGINES = {
    "sweep-fp64": dict(engine=1, precision=0),
    "sweep-mixed": dict(engine=1, precision=1),
    "incremental": dict(engine=2, precision=0),
    "incremental-mixed": dict(engine=2, precision=1),
}


def oracle_run(f, margin, merges, record=0, mode="delta"):
    merges = min(merges, f.n_bus - 1)            # the library caps merges the same way
    vhat, ihat = O.operating_points(f)
    return O.reduce(f, vhat, ihat, margin=margin, max_merges=merges, record_iters=record, mode=mode), vhat


def assert_same_run(ctx, res, vhat_o, check_voltages=True):
    dec = ctx.decisions()
    summ = ctx.summary()
    t = res["n_iter"]
    assert summ["n_iter"] == t, (summ["n_iter"], t)
    assert summ["stop_reason"] == res["stop_reason"]
    assert np.all(res["gap"][:t] > GAP_MIN), "oracle tie margins too small for a decision comparison"
    assert np.array_equal(dec["s"], res["s"]) and np.array_equal(dec["r"], res["r"])
    assert np.abs(dec["score"] - res["score"]).max(initial=0.0) <= S_TOL
    assert np.abs(dec["maxerr"] - res["maxerr"]).max(initial=0.0) <= 1e-12
    assert np.array_equal(dec["ncand"], res["ncand"])
    assert np.array_equal(ctx.assignment(), res["super_of"])
    if check_voltages:
        vh, vr = ctx.voltages()
        assert np.abs(vh - vhat_o).max() <= V_TOL
        assert np.abs(vr - res["v_red"]).max() <= V_TOL


# ----------------------------------------------------------------------------- load flow
@pytest.mark.parametrize("name,n", [("feeder40", None), ("feeder1000", 300)])
def test_power_flow_matches_oracle(ctx, name, n):
    f, _ = fg.preset(name, **({"n_bus": n} if n else {}))
    vg, ig, sw = ctx.power_flow(f)
    vo, swo = O.power_flow(f)
    io = O.injection(f, vo)
    assert np.abs(vg - vo).max() <= 1e-12
    assert np.abs(ig - io).max() <= 1e-9
    assert abs(sw - swo) <= 1


# ----------------------------------------------------------------------------- search
CASES = [
    # (n, seed, kv, phase_mode, load, L, margin, target)
    (40, 1, 4.16, "keep", ("uniform", 50.0), 2, 0.005, 1.0),
    (60, 7, 4.16, "keep", ("uniform", 50.0), 1, 0.003, 1.0),
    (150, 11, 12.47, (0.7, 0.1, 0.2), ("uniform", 100.0), 2, 0.005, 1.0),
    (250, 12, 12.47, (0.45, 0.15, 0.4), ("lognormal", 15.0, 1.0), 3, 0.004, 0.9),
    (400, 13, 12.47, (0.7, 0.1, 0.2), ("uniform", 100.0), 4, 0.002, 0.6),
]


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}-s{c[1]}-L{c[5]}" for c in CASES])
def test_search_matches_oracle(ctx, case, engine):
    n, seed, kv, mode, load, L, margin, target = case
    f = fg.make_feeder(n, seed, kv_ll=kv, phase_mode=mode, load=load, n_scen=L)
    merges = O.max_merges_for(n, target)
    res, vhat_o = oracle_run(f, margin, merges)
    ctx.reduce(f, params(margin=margin, target_reduction=target, **ENGINES[engine]))
    assert_same_run(ctx, res, vhat_o)


def test_screen_bounds_cover_the_fp64_scores(ctx):
    """Precision 1: every screened score lies within its bound of the oracle's
    FP64 score (the argument that makes the mixed-precision selection exact)."""
    for f in (fg.preset("feeder40")[0], fg.make_feeder(300, 23, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0))):
        K = 8
        res, _ = oracle_run(f, 0.005, f.n_bus, record=K)
        ctx.reduce(f, params(margin=0.005, record_iters=K, precision=1))
        worst = 0.0
        for t in range(min(K, res["n_iter"])):
            go = {(int(s), int(r)): v for s, r, v in zip(res["recorded"][t]["s"], res["recorded"][t]["r"],
                                                         res["recorded"][t]["score"])}
            rg = ctx.recorded(t)
            assert len(rg["s"]) == len(go)
            for s, r, v, b in zip(rg["s"], rg["r"], rg["score"], rg["bound"]):
                o = go[(int(s), int(r))]
                if math.isinf(v):
                    assert math.isinf(o)        # screened out only when surely infeasible
                    continue
                if math.isinf(o):
                    continue                    # screen kept an infeasible candidate: allowed
                assert abs(v - o) <= b, (t, s, r, v, o, b)
                worst = max(worst, abs(v - o) / b if b > 0 else 0.0)
        assert worst < 1.0


@pytest.mark.parametrize("engine", ["sweep-fp64", "incremental"])
def test_every_candidate_score_matches_oracle(ctx, engine):
    for f in (fg.preset("feeder40")[0], fg.make_feeder(200, 21, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0))):
        K = 6
        res, _ = oracle_run(f, 0.005, f.n_bus, record=K)
        ctx.reduce(f, params(margin=0.005, record_iters=K, **ENGINES[engine]))
        for t in range(min(K, res["n_iter"])):
            rec_o = res["recorded"][t]
            rec_g = ctx.recorded(t)
            go = {(int(s), int(r)): v for s, r, v in zip(rec_o["s"], rec_o["r"], rec_o["score"])}
            gg = {(int(s), int(r)): v for s, r, v in zip(rec_g["s"], rec_g["r"], rec_g["score"])}
            assert set(go) == set(gg)
            for key, v in go.items():
                w = gg[key]
                if math.isinf(v) or math.isinf(w):
                    assert math.isinf(v) and math.isinf(w), key
                else:
                    assert abs(v - w) <= S_TOL, (t, key, v, w)


# ----------------------------------------------------------------------------- objective 1
OBJ1_FEEDERS = {
    "feeder40": lambda: fg.preset("feeder40")[0],
    "feeder1000_300": lambda: fg.preset("feeder1000", n_bus=300)[0],
    "mixed200": lambda: fg.make_feeder(200, 21, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0)),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(OBJ1_FEEDERS))
def test_max_error_objective_matches_oracle(ctx, name, precision):
    """objective = 1: each candidate is scored by the largest per-phase error of
    its network (the iteration objective of Sec. IV); decisions must match the
    oracle's, and so must every recorded score (FP64), or lie within the
    screen's bound of it (FP32 screen)."""
    f = OBJ1_FEEDERS[name]()
    K = 4
    vhat, ihat = O.operating_points(f)
    merges = f.n_bus - 1 if name == "feeder40" else f.n_bus // 2
    res = O.reduce(f, vhat, ihat, margin=0.005, max_merges=merges, objective=1, record_iters=K)
    ctx.reduce(f, params(margin=0.005, max_merges=merges, objective=1, precision=precision, record_iters=K))
    assert_same_run(ctx, res, vhat)
    for t in range(min(K, res["n_iter"])):
        rec_o, rec_g = res["recorded"][t], ctx.recorded(t)
        go = {(int(s), int(r)): v for s, r, v in zip(rec_o["s"], rec_o["r"], rec_o["score"])}
        gg = {(int(s), int(r)): (v, b) for s, r, v, b in zip(rec_g["s"], rec_g["r"], rec_g["score"], rec_g["bound"])}
        assert set(go) == set(gg)
        for key, v in go.items():
            w, b = gg[key]
            if math.isinf(v) or math.isinf(w):
                if precision == 0:
                    assert math.isinf(v) and math.isinf(w), (t, key, v, w)
                else:                   # the screen may keep a candidate that FP64 rejects, never the reverse
                    assert math.isinf(v), (t, key, v, w)
                continue
            tol = S_TOL if precision == 0 else b + 1e-12
            assert abs(v - w) <= tol, (t, key, v, w, b)


def test_reduce_ops_with_oracle_operating_points(ctx):
    f, run = fg.preset("feeder40")
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=f.n_bus - 1)
    ctx.reduce_ops(f, vhat, ihat, params(margin=run["margin"]))
    assert ctx.summary()["pf_sweeps"] == 0
    assert_same_run(ctx, res, vhat)


def test_device_entry_matches_host_entry(ctx):
    torch = pytest.importorskip("torch")
    import paper_2510_19608_gb300 as K
    f = fg.make_feeder(300, 5, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0))
    p = params(margin=0.005, target_reduction=0.5)
    ctx.reduce(f, p)
    host = ctx.decisions()
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.parent, f.phases, f.z_line, f.s_load)]
    df = K.device_feeder(f.n_bus, f.n_scen, *[t.data_ptr() for t in dev], f.v_slack)
    torch.cuda.synchronize()
    ctx.reduce_device(df, p)
    d = ctx.decisions()
    assert np.array_equal(d["s"], host["s"]) and np.array_equal(d["r"], host["r"])
    assert np.array_equal(d["score"], host["score"])          # same kernels, same order: bit-identical


# ----------------------------------------------------------------------------- edge cases
def _mk(parent, phases, seed=0, load=0.05, L=2):
    rng = np.random.default_rng(seed)
    n = len(parent)
    z = np.zeros((n, 3, 3, 2))
    s = np.zeros((L, n, 3, 2))
    for i in range(1, n):
        ps = [p for p in range(3) if phases[i] >> p & 1]
        for a in ps:
            for b in ps:
                z[i, a, b] = (0.004, 0.008) if a == b else (0.001, 0.003)
            for l in range(L):
                s[l, i, a] = (load * rng.random() * (0.3 ** l), 0.3 * load * rng.random() * (0.3 ** l))
    vs = np.array([[1.0, 0.0], [-0.5, -math.sqrt(3) / 2], [-0.5, math.sqrt(3) / 2]])
    return fg.Feeder(parent=np.array(parent, np.int32), phases=np.array(phases, np.uint8), z_line=z, s_load=s,
                     v_slack=vs, meta={})


EDGE = {
    "two_bus": _mk([-1, 0], [7, 7]),
    "chain": _mk([-1] + list(range(0, 79)), [7] * 80, seed=1, load=0.01),
    "star": _mk([-1] + [0] * 60, [7] + [1, 2, 4, 3, 5, 6, 7] * 8 + [7] * 4, seed=2),
    "single_phase": _mk([-1, 0, 1, 1, 2, 2, 3, 3, 4, 5, 6, 7], [7] + [2] * 11, seed=3),
    "unloaded": _mk([-1, 0, 0, 1, 1, 2, 2, 3, 4, 5, 6, 6, 7, 8], [7] * 14, load=0.0),
}


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("name", sorted(EDGE))
def test_edge_feeders_match_oracle(ctx, name, engine):
    f = EDGE[name]
    res, vhat_o = oracle_run(f, 0.01, f.n_bus)
    ctx.reduce(f, params(margin=0.01, **ENGINES[engine]))
    if name == "unloaded":
        # every candidate scores exactly 0: all tied, the smallest (r, s) wins each time
        assert np.all(res["score"] == 0.0)
        res["gap"][:] = np.inf
    assert_same_run(ctx, res, vhat_o)


def test_zero_target_and_tiny_margin(ctx):
    f, _ = fg.preset("feeder40")
    ctx.reduce(f, params(margin=0.005, max_merges=0))
    s = ctx.summary()
    assert s["n_iter"] == 0 and s["stop_reason"] == 0 and s["n_kept"] == f.n_bus
    vh, vr = ctx.voltages()
    assert np.array_equal(vh, vr)
    res, _ = oracle_run(f, 1e-15, f.n_bus)
    ctx.reduce(f, params(margin=1e-15))
    assert ctx.summary()["n_iter"] == res["n_iter"]
    assert ctx.summary()["stop_reason"] == res["stop_reason"] == 1


def test_invalid_inputs_are_rejected(ctx):
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300._binding import EINVAL, EPF, ESINGULAR
    f, _ = fg.preset("feeder40")
    bad = fg.Feeder(parent=f.parent.copy(), phases=f.phases.copy(), z_line=f.z_line.copy(),
                    s_load=f.s_load.copy(), v_slack=f.v_slack, meta={})
    bad.parent[5] = 9
    with pytest.raises(K.OkrError) as e:
        ctx.reduce(bad, params())
    assert e.value.status == EINVAL
    bad = fg.Feeder(parent=f.parent.copy(), phases=f.phases.copy(), z_line=f.z_line.copy(),
                    s_load=f.s_load.copy(), v_slack=f.v_slack, meta={})
    i = int(np.where(f.phases != 7)[0][0])
    bad.phases[i + 1:] = 7
    bad.phases[i] = 1
    kids = [k for k in range(f.n_bus) if f.parent[k] == i]
    if kids:
        with pytest.raises(K.OkrError) as e:
            ctx.reduce(bad, params())
        assert e.value.status == EINVAL
    bad = fg.Feeder(parent=f.parent.copy(), phases=f.phases.copy(), z_line=f.z_line.copy(),
                    s_load=f.s_load.copy(), v_slack=f.v_slack, meta={})
    bad.z_line[3] = 0.0
    with pytest.raises(K.OkrError) as e:
        ctx.reduce(bad, params())
    assert e.value.status == ESINGULAR
    bad = fg.Feeder(parent=f.parent.copy(), phases=f.phases.copy(), z_line=f.z_line.copy(),
                    s_load=f.s_load * 500.0, v_slack=f.v_slack, meta={})
    with pytest.raises(K.OkrError) as e:
        ctx.reduce(bad, params())
    assert e.value.status == EPF
    with pytest.raises(K.OkrError) as e:
        ctx.reduce(f, params(margin=-1.0))
    assert e.value.status == EINVAL
    # the context still works after the errors
    ctx.reduce(f, params(margin=0.005, max_merges=3))
    assert ctx.summary()["n_iter"] == 3


# ----------------------------------------------------------------------------- full sizes
def _check_properties(ctx, f, margin):
    """Properties every result must have, at any size: clusters are connected,
    phase-feasible and led by their super-node; the reported errors follow from
    the reported voltages; the margin holds."""
    sup = ctx.assignment()
    n = f.n_bus
    assert sup[0] == 0
    for i in range(n):
        k = sup[i]
        assert sup[k] == k
        assert (f.phases[i] & f.phases[k]) == f.phases[i]
        if i != k:                      # connected: the tree path from i to k stays in the cluster
            a, b = i, k
            anc_i = [a]
            while a > 0:
                a = f.parent[a]
                anc_i.append(a)
            anc_k = [b]
            while b > 0:
                b = f.parent[b]
                anc_k.append(b)
            common = next(x for x in anc_i if x in set(anc_k))
            path = anc_i[:anc_i.index(common) + 1] + anc_k[:anc_k.index(common)]
            assert all(sup[x] == k for x in path)
    vh, vr = ctx.voltages()
    pres = np.array([[(f.phases[i] >> p) & 1 for p in range(3)] for i in range(n)], bool)
    e = np.where(pres[None], np.abs(np.abs(vh) - np.abs(vr)), 0.0)
    assert e.max() <= margin
    smice = sum(float(e[l][sup == k].max()) for l in range(e.shape[0]) for k in np.unique(sup))
    s = ctx.summary()
    assert abs(s["smice"] - smice) <= 1e-10
    # the chosen network evaluated by the oracle (load flow, aggregated
    # injections, tree solve): the same voltages and the same largest error
    err_o, vred_o = O.evaluate(f, sup)
    assert np.abs(vr - vred_o).max() <= V_TOL
    assert abs(float(err_o.max()) - s["max_error"]) <= 1e-11
    assert abs(s["max_error"] - e.max()) <= 1e-12


@pytest.fixture(scope="module")
def feeder1000_oracle():
    f, run = fg.preset("feeder1000")
    merges = O.max_merges_for(f.n_bus, run["target"])
    res, vhat_o = oracle_run(f, run["margin"], merges)
    return f, run, res, vhat_o


@pytest.mark.parametrize("engine", sorted(ENGINES))
def test_feeder1000_full_run_matches_oracle(ctx, feeder1000_oracle, engine):
    f, run, res, vhat_o = feeder1000_oracle
    ctx.reduce(f, params(margin=run["margin"], target_reduction=run["target"], **ENGINES[engine]))
    assert_same_run(ctx, res, vhat_o)
    _check_properties(ctx, f, run["margin"])


@pytest.mark.parametrize("name", ["feeder2200", "feeder3100"])
def test_large_feeders_prefix_and_properties(ctx, name):
    f, run = fg.preset(name)
    K = 12
    res, vhat_o = oracle_run(f, run["margin"], K)
    for engine in sorted(ENGINES):
        ctx.reduce(f, params(margin=run["margin"], max_merges=K, **ENGINES[engine]))
        assert_same_run(ctx, res, vhat_o)
    ctx.reduce(f, params(margin=run["margin"], target_reduction=run["target"], **ENGINES["sweep-mixed"]))
    full1 = ctx.decisions()
    ctx.reduce(f, params(margin=run["margin"], target_reduction=run["target"], **ENGINES["incremental"]))
    full0 = ctx.decisions()
    assert np.array_equal(full0["s"], full1["s"]) and np.array_equal(full0["r"], full1["r"])
    s = ctx.summary()
    assert s["n_iter"] == O.max_merges_for(f.n_bus, run["target"]) or s["stop_reason"] == 1
    _check_properties(ctx, f, run["margin"])

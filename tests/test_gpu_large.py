"""Full-size parity of the CUDA library (through its C ABI) with the CPU oracle.

The 2,200- and 3,100-bus stand-ins of the paper's 5,991- and 8,381-node
feeders (Table 2) are reduced to their targets (90 % and 80 %) by every engine
and precision, and every decision of the whole run is compared with the
oracle's: the chosen (s, r) bit-exact, scores within 1e-11, largest errors
within 1e-12, candidate counts exact, and the final network's voltages within
1e-9 p.u. of the oracle's evaluation of the same assignment.

The oracle's full runs take minutes, so they are stored under tests/golden/
(written by tests/golden/make_golden.py, which calls only the oracle) with the
fingerprint of the feeder they were made from.  A machine whose generator draws
a different feeder runs the oracle itself instead.

The incremental engine takes size-dependent paths: where the selection records
live (shared memory with or without the largest MICE per super-node, or device
memory) and whether a merge's work entries overflow the shared-memory tile into
device memory.  Those paths are run in verify mode (every carried score
re-evaluated after every merge, bit for bit) at the sizes that select them by
themselves, and forced through okr_set_inc_shape on small feeders, where the
oracle's full runs are quick.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import feedergen as fg
from oracle import oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
S_TOL = 1e-11          # SMICE (both sides FP64, differing only in rounding order)
E_TOL = 1e-12          # largest error of a decision
V_TOL = 1e-9           # p.u., voltages
GAP_MIN = 1e-12        # oracle tie margins below this would make a decision comparison fragile

ENGINES = {
    "sweep-fp64": dict(engine=1, precision=0),
    "sweep-mixed": dict(engine=1, precision=1),
    "incremental": dict(engine=2, precision=0),
    "incremental-mixed": dict(engine=2, precision=1),
}


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


def load_golden(label: str):
    """A stored oracle run: header fields and the decision rows, or None."""
    path = os.path.join(GOLDEN, f"{label}_decisions.txt")
    if not os.path.exists(path):
        return None
    hdr, rows = {}, []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                w = line[1:].split()
                if w and w[0] == "fingerprint":
                    hdr["fingerprint"] = w[1]
                elif w and w[0] == "n_iter":
                    hdr.update(n_iter=int(w[1]), stop_reason=int(w[3]), candidates=int(w[5]))
                continue
            rows.append(line.split())
    a = np.array(rows, dtype=object).reshape(-1, 7)
    return dict(hdr, s=a[:, 1].astype(np.int32), r=a[:, 2].astype(np.int32), score=a[:, 3].astype(float),
                maxerr=a[:, 4].astype(float), gap=a[:, 5].astype(float), ncand=a[:, 6].astype(np.int32))


def oracle_full(label: str, f, run):
    """The oracle's full run of feeder f: from tests/golden/ when the stored
    fingerprint is this feeder's, else computed here."""
    g = load_golden(label)
    if g is not None and g.get("fingerprint") == fg.fingerprint(f):
        return g
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=O.max_merges_for(f.n_bus, run["target"]))
    return dict(n_iter=res["n_iter"], stop_reason=res["stop_reason"], candidates=res["candidates"], s=res["s"],
                r=res["r"], score=res["score"], maxerr=res["maxerr"], gap=res["gap"], ncand=res["ncand"])


def assignment_of(n: int, s, r) -> np.ndarray:
    """super_of after committing the merges (s absorbs r's cluster), caller ids."""
    sup = np.arange(n, dtype=np.int32)
    for a, b in zip(s, r):
        sup[sup == b] = a
    return sup


def assert_decisions(dec, summ, g, upto=None):
    t = g["n_iter"] if upto is None else upto
    assert np.all(g["gap"][:t] > GAP_MIN), "oracle tie margins too small for a decision comparison"
    if upto is None:
        assert summ["n_iter"] == g["n_iter"] and summ["stop_reason"] == g["stop_reason"]
    assert len(dec["s"]) == t
    assert np.array_equal(dec["s"], g["s"][:t]) and np.array_equal(dec["r"], g["r"][:t])
    assert np.abs(dec["score"] - g["score"][:t]).max(initial=0.0) <= S_TOL
    assert np.abs(dec["maxerr"] - g["maxerr"][:t]).max(initial=0.0) <= E_TOL
    assert np.array_equal(dec["ncand"], g["ncand"][:t])


def check_final_network(ctx, f, margin):
    """The chosen network evaluated by the oracle (load flow, aggregated
    injections, tree solve) has the library's voltages and largest error."""
    sup = ctx.assignment()
    _, vr = ctx.voltages()
    err_o, vred_o = O.evaluate(f, sup)
    s = ctx.summary()
    assert np.abs(vr - vred_o).max() <= V_TOL
    assert abs(float(err_o.max()) - s["max_error"]) <= E_TOL
    assert s["max_error"] <= margin


LARGE = ["feeder2200", "feeder3100"]


@pytest.fixture(scope="module", params=LARGE)
def large(request):
    f, run = fg.preset(request.param)
    return request.param, f, run, oracle_full(request.param, f, run)


@pytest.mark.parametrize("engine", sorted(ENGINES))
def test_full_run_matches_oracle(ctx, large, engine):
    name, f, run, g = large
    ctx.reset_inc_shape()
    ctx.reduce(f, params(margin=run["margin"], target_reduction=run["target"], **ENGINES[engine]))
    summ = ctx.summary()
    assert_decisions(ctx.decisions(), summ, g)
    assert summ["candidates"] == g["candidates"]
    assert np.array_equal(ctx.assignment(), assignment_of(f.n_bus, g["s"], g["r"]))
    check_final_network(ctx, f, run["margin"])


# ---------------------------------------------------------------- size-dependent paths of the incremental engine
# records: 1 device memory, 2 shared memory, 3 shared memory with the largest MICE per super-node
VERIFY_MERGES = 300


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["feeder3100-auto", "feeder2800-auto", "feeder2200-auto"])
def test_verify_mode_at_the_sizes_that_select_each_record_placement(ctx, case, precision):
    """Verify mode (engine 3) with the placement the size selects by itself:
    device memory at 3,100 buses, shared memory at 2,800, shared memory with the
    per-super-node maximum at 2,200.  No carried score may differ from a fresh
    evaluation, and the decisions are the oracle's (3,100 and 2,200) or the
    FP64 sweep's (2,800)."""
    ctx.reset_inc_shape()
    if case == "feeder2800-auto":
        f, run = fg.preset("feeder3100", n_bus=2800)
        want = 2
    else:
        name = case.split("-")[0]
        f, run = fg.preset(name)
        want = 1 if name == "feeder3100" else 3
    ctx.reduce(f, params(margin=run["margin"], max_merges=VERIFY_MERGES, engine=3, precision=precision))
    s = ctx.summary()
    assert s["inc_records"] == want
    assert s["n_iter"] == VERIFY_MERGES
    assert s["inc_mismatches"] == 0
    dec = ctx.decisions()
    if case == "feeder2800-auto":
        ctx.reduce(f, params(margin=run["margin"], max_merges=VERIFY_MERGES, engine=1, precision=0))
        ref = ctx.decisions()
        assert np.array_equal(dec["s"], ref["s"]) and np.array_equal(dec["r"], ref["r"])
        assert np.abs(dec["score"] - ref["score"]).max() <= S_TOL
    else:
        g = oracle_full(case.split("-")[0], f, run)
        assert_decisions(dec, s, g, upto=VERIFY_MERGES)


# forced shapes on small feeders: every record placement, work entries spilling
# past a tiny shared tile, both CTA sizes and evaluation-warp splits
SHAPES = {
    "dev-records-4-entries": dict(records=1, shared_entries=4),
    "shared-records-16-entries": dict(records=2, shared_entries=16),
    "max-records-1-entry": dict(records=3, shared_entries=1),
    "256-threads-dev-records-8-entries": dict(threads=256, eval_warps=1, records=1, shared_entries=8),
    "256-threads-default": dict(threads=256),
    "512-threads-12-eval-warps": dict(threads=512, eval_warps=12, shared_entries=32),
    "512-threads-1-eval-warp": dict(threads=512, eval_warps=1, records=2),
    "384-threads-11-eval-warps-dev-records": dict(threads=384, eval_warps=11, records=1, shared_entries=24),
    "512-threads-default": dict(threads=512),
}

SMALL = [
    # (n, seed, phase_mode, load, L, margin, target)
    (150, 11, (0.7, 0.1, 0.2), ("uniform", 100.0), 2, 0.005, 1.0),
    (250, 12, (0.45, 0.15, 0.4), ("lognormal", 15.0, 1.0), 3, 0.004, 0.9),
    (400, 13, (0.7, 0.1, 0.2), ("uniform", 100.0), 4, 0.002, 0.6),
]
_small_cache: dict = {}


def small_case(i):
    if i not in _small_cache:
        n, seed, mode, load, L, margin, target = SMALL[i]
        f = fg.make_feeder(n, seed, phase_mode=mode, load=load, n_scen=L)
        vhat, ihat = O.operating_points(f)
        res = O.reduce(f, vhat, ihat, margin=margin, max_merges=O.max_merges_for(n, target))
        _small_cache[i] = (f, margin, target, res)
    return _small_cache[i]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_forced_shapes_verify_and_match_oracle(ctx, shape, precision):
    try:
        ctx.set_inc_shape(**SHAPES[shape])
        for i in range(len(SMALL)):
            f, margin, target, res = small_case(i)
            ctx.reduce(f, params(margin=margin, target_reduction=target, engine=3, precision=precision))
            s = ctx.summary()
            sh = SHAPES[shape]
            assert s["inc_threads"] == (sh.get("threads") or 384)
            if sh.get("eval_warps", 0):
                assert s["inc_eval_warps"] == sh["eval_warps"]
            if sh.get("records", 0):
                assert s["inc_records"] == sh["records"]
            if sh.get("shared_entries", 0):
                assert s["inc_shared_entries"] == sh["shared_entries"]
            assert s["inc_mismatches"] == 0
            g = dict(n_iter=res["n_iter"], stop_reason=res["stop_reason"], s=res["s"], r=res["r"],
                     score=res["score"], maxerr=res["maxerr"], gap=res["gap"], ncand=res["ncand"])
            assert_decisions(ctx.decisions(), s, g)
            assert np.array_equal(ctx.assignment(), res["super_of"])
    finally:
        ctx.reset_inc_shape()


def test_shape_setter_rejects_out_of_range(ctx):
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300._binding import EINVAL
    for bad in (dict(threads=128), dict(threads=1024), dict(threads=320), dict(eval_warps=12),
                dict(threads=256, eval_warps=8),
                dict(shared_entries=257), dict(shared_entries=-1), dict(records=4), dict(records=-1)):
        with pytest.raises(K.OkrError) as e:
            ctx.set_inc_shape(**bad)
        assert e.value.status == EINVAL
    ctx.reset_inc_shape()
    assert ctx.inc_shape() == dict(threads=384, eval_warps=2, shared_entries=256, records=0)
    # a forced placement that does not fit shared memory is refused at the reduction
    f, run = fg.preset("feeder3100")
    try:
        ctx.set_inc_shape(records=2)
        with pytest.raises(K.OkrError) as e:
            ctx.reduce(f, params(margin=run["margin"], max_merges=2, engine=2))
        assert e.value.status == EINVAL
    finally:
        ctx.reset_inc_shape()
    ctx.reduce(f, params(margin=run["margin"], max_merges=2, engine=2))
    assert ctx.summary()["n_iter"] == 2


# ---------------------------------------------------------------- batches at full size
BATCH_LARGEST = ((4, 0.9), (80, 0.7), (110, 0.5))   # largest feeder of each target in batch_presets(256)


@pytest.fixture(scope="module")
def batch256():
    return fg.batch_presets(256)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch256_incremental_matches_single_runs_and_oracle(ctx, batch256, precision):
    """The 256-feeder batch on the incremental engine (one CTA per feeder):
    every feeder as its own single run, and the largest feeder of each target
    decision for decision as the oracle's full run."""
    ctx.reset_inc_shape()
    feeders = [f for f, _ in batch256]
    ps = [params(margin=r["margin"], target_reduction=r["target"], precision=precision, engine=2) for _, r in batch256]
    items, parts, stats = ctx.reduce_batch(feeders, ps)
    assert stats["fallbacks"] == 0
    for k, (f, p, it, part) in enumerate(zip(feeders, ps, items, parts)):
        assert it["status"] == 0
        ctx.reduce(f, p)
        s = ctx.summary()
        assert it["n_iter"] == s["n_iter"] and it["stop_reason"] == s["stop_reason"], k
        assert it["candidates"] == s["candidates"]
        assert abs(it["smice"] - s["smice"]) <= 1e-13
        assert np.array_equal(part, ctx.assignment()), k
    for k, target in BATCH_LARGEST:
        f, run = batch256[k]
        assert run["target"] == target
        g = oracle_full(f"batch256_{k}", f, run)
        assert items[k]["n_iter"] == g["n_iter"] and items[k]["stop_reason"] == g["stop_reason"]
        assert items[k]["candidates"] == g["candidates"]
        assert abs(items[k]["smice"] - g["score"][-1]) <= S_TOL
        assert np.array_equal(parts[k], assignment_of(f.n_bus, g["s"], g["r"]))


def test_batch256_sweep_largest_match_oracle(ctx, batch256):
    """The sweep engine's batch (teams of CTAs per feeder, FP32 screen) on the
    largest feeder of each target: the oracle's full run."""
    ctx.reset_inc_shape()
    sel = [k for k, _ in BATCH_LARGEST]
    feeders = [batch256[k][0] for k in sel]
    ps = [params(margin=batch256[k][1]["margin"], target_reduction=batch256[k][1]["target"], precision=1, engine=1)
          for k in sel]
    items, parts, _ = ctx.reduce_batch(feeders, ps)
    for k, f, it, part in zip(sel, feeders, items, parts):
        g = oracle_full(f"batch256_{k}", f, batch256[k][1])
        assert it["status"] == 0
        assert it["n_iter"] == g["n_iter"] and it["candidates"] == g["candidates"]
        assert np.array_equal(part, assignment_of(f.n_bus, g["s"], g["r"]))


@pytest.mark.parametrize("shape", ["256-threads-default", "dev-records-4-entries", "512-threads-1-eval-warp"])
def test_batch_shapes_equal_default(ctx, batch256, shape):
    """A batch gives the same results under every shape it accepts."""
    sel = list(range(0, 256, 16))
    feeders = [batch256[k][0] for k in sel]
    ps = [params(margin=batch256[k][1]["margin"], target_reduction=batch256[k][1]["target"], precision=1, engine=2)
          for k in sel]
    ctx.reset_inc_shape()
    ref, ref_parts, _ = ctx.reduce_batch(feeders, ps)
    try:
        ctx.set_inc_shape(**SHAPES[shape])
        items, parts, _ = ctx.reduce_batch(feeders, ps)
    finally:
        ctx.reset_inc_shape()
    for a, b, pa, pb in zip(ref, items, ref_parts, parts):
        assert a["status"] == b["status"] == 0
        assert a["n_iter"] == b["n_iter"] and a["smice"] == b["smice"]
        assert np.array_equal(pa, pb)


def test_batch_rejects_the_per_super_node_maximum(ctx, batch256):
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300._binding import EINVAL
    feeders = [batch256[k][0] for k in range(4)]
    ps = [params(margin=0.005, target_reduction=0.5, engine=2)]
    try:
        ctx.set_inc_shape(records=3)
        with pytest.raises(K.OkrError) as e:
            ctx.reduce_batch(feeders, ps)
        assert e.value.status == EINVAL
    finally:
        ctx.reset_inc_shape()


def test_inc_autotune_single_and_batch(ctx, batch256):
    """okr_inc_autotune times every shape of its list, keeps the fastest on the
    context, and the results under the kept shape are the default shape's."""
    import math
    f, run = fg.preset("feeder1000", n_bus=600)
    p = params(margin=run["margin"], target_reduction=0.5, precision=1, engine=2)
    ctx.reset_inc_shape()
    ctx.reduce(f, p)
    ref = ctx.decisions()
    try:
        best, table = ctx.inc_autotune([f], [p])
        assert len(table) >= 6
        times = [t for _, t in table]
        assert all(t > 0 for t in times)
        i = int(np.argmin(times))
        for k in ("threads", "eval_warps"):
            assert best[k] == table[i][0][k]
        assert ctx.inc_shape() == best
        ctx.reduce(f, p)
        d = ctx.decisions()
        assert np.array_equal(d["s"], ref["s"]) and np.array_equal(d["score"], ref["score"])
        sel = list(range(0, 256, 32))
        feeders = [batch256[k][0] for k in sel]
        ps = [params(margin=batch256[k][1]["margin"], target_reduction=batch256[k][1]["target"], precision=1,
                     engine=2) for k in sel]
        bbest, btable = ctx.inc_autotune(feeders, ps)
        assert all(t > 0 and not math.isnan(t) for _, t in btable)
        assert ctx.inc_shape() == bbest
        from paper_2510_19608_gb300._binding import EINVAL
        import paper_2510_19608_gb300 as K
        with pytest.raises(K.OkrError) as e:
            ctx.inc_autotune([f], [params(margin=run["margin"], engine=1)])
        assert e.value.status == EINVAL
    finally:
        ctx.reset_inc_shape()


def test_flat_and_block_walk_selection_agree_at_the_flat_limit(ctx):
    """Pass B of the selection reads every record when the feeder has at most
    1,536 buses and its records are in shared memory, and walks the block
    summaries otherwise.  On a feeder of exactly 1,536 buses both ways (the
    records in shared memory, then forced into device memory) give the same
    run in both precisions: every decision, score, largest error, gap and
    candidate count bit for bit, and the same assignment; verify mode with
    the flat pass finds every carried score equal to a fresh evaluation."""
    f = fg.make_feeder(1536, 1536, phase_mode=(0.45, 0.15, 0.4), load=("lognormal", 15.0, 1.0))
    for precision in (0, 1):
        runs = []
        for shape in ({}, dict(records=1)):
            try:
                if shape:
                    ctx.set_inc_shape(**shape)
                ctx.reduce(f, params(margin=0.005, target_reduction=0.5, engine=2, precision=precision))
                s = ctx.summary()
                assert (s["inc_records"] == 1) if shape else (s["inc_records"] in (2, 3))
                runs.append((ctx.decisions(), s, ctx.assignment()))
            finally:
                ctx.reset_inc_shape()
        (d0, s0, a0), (d1, s1, a1) = runs
        assert s0["n_iter"] == s1["n_iter"] > 0 and s0["stop_reason"] == s1["stop_reason"]
        for key in ("s", "r", "score", "maxerr", "gap", "ncand"):
            assert np.array_equal(d0[key], d1[key]), key
        assert np.array_equal(a0, a1)
        ctx.reduce(f, params(margin=0.005, max_merges=150, engine=3, precision=precision))
        s = ctx.summary()
        assert s["inc_records"] in (2, 3) and s["n_iter"] == 150 and s["inc_mismatches"] == 0

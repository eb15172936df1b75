"""The C ABI's result objects and allocator hook.

okr_result_take copies a reduction's outputs (the kept set and clusters, the
decision sequence, the voltages and errors of Sec. III-IV, and Y_Kron of
Sec. II-B) out of the context into a library-owned object: later calls on the
context must leave it untouched, and its getters answer size queries when
given NULL buffers.  okr_set_allocator routes every device allocation of a
context through the caller's allocator (here torch's caching allocator): the
results must equal those of a context on cudaMalloc, and every block handed
out must come back.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import feedergen as fg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import build
    build.build()
    return K


def test_result_object_outlives_later_calls(K):
    fa, run = fg.preset("feeder1000", n_bus=300)
    fb, _ = fg.preset("feeder40")
    p = K.default_params(margin=run["margin"], target_reduction=0.5, precision=1)
    with K.Context(0) as ctx:
        ctx.reduce(fa, p)
        want = dict(dec=ctx.decisions(), sup=ctx.assignment(), volt=ctx.voltages(), summ=ctx.summary(),
                    yk=ctx.kron())
        res = ctx.take_result(with_ykron=True)
        res_noy = ctx.take_result()
        # later calls overwrite the context's own results
        ctx.reduce(fb, K.default_params(margin=0.005))
        ctx.kron()
        assert ctx.summary()["n_bus"] == fb.n_bus
        with res:
            d = res.decisions()
            for k in ("s", "r", "score", "maxerr", "gap", "ncand"):
                assert np.array_equal(d[k], want["dec"][k]), k
            assert np.array_equal(res.assignment(), want["sup"])
            e = res.errors()
            assert np.array_equal(e["vhat"], want["volt"][0]) and np.array_equal(e["vred"], want["volt"][1])
            assert e["max_error"] == want["summ"]["max_error"] and e["smice"] == want["summ"]["smice"]
            s = res.summary()
            for k in ("n_bus", "n_iter", "candidates", "smice", "max_error", "stop_reason", "engine"):
                assert s[k] == want["summ"][k], k
            y, pn = res.ykron()
            assert np.array_equal(y, want["yk"][0]) and np.array_equal(pn, want["yk"][1])
            st = res.stats()
            assert st["candidates"] == want["summ"]["candidates"] and st["iterations"] == want["summ"]["n_iter"]
            assert abs(st["seconds"] - 1e-3 * want["summ"]["search_ms"]) < 1e-12
        with res_noy:
            from paper_2510_19608_gb300._binding import ENOTREADY
            with pytest.raises(K.OkrError) as ex:
                res_noy.ykron()
            assert ex.value.status == ENOTREADY
            assert np.array_equal(res_noy.assignment(), want["sup"])


def test_result_size_queries_and_errors(K):
    from paper_2510_19608_gb300 import _binding as B
    f, run = fg.preset("feeder40")
    with K.Context(0) as ctx:
        h = C.c_void_p()
        assert B.lib().okr_result_take(ctx._h, 0, C.byref(h)) == B.ENOTREADY     # no reduction yet
        ctx.reduce(f, K.default_params(margin=run["margin"]))
        assert B.lib().okr_result_take(ctx._h, 1, C.byref(h)) == B.OK
        try:
            L = B.lib()
            n, kept = C.c_int32(-1), C.c_int32(-1)
            assert L.okr_result_assignment(h, None, C.byref(n), C.byref(kept)) == B.OK
            assert n.value == f.n_bus and kept.value == f.n_bus - ctx.summary()["n_iter"]
            cnt = C.c_int32(-1)
            assert L.okr_result_decisions(h, 0, None, None, None, None, None, None, C.byref(cnt)) == B.OK
            assert cnt.value == ctx.summary()["n_iter"]
            k = C.c_int32(-1)
            assert L.okr_result_ykron(h, 0, None, None, C.byref(k)) == B.OK
            assert k.value == ctx.kron()[0].shape[0]
            y = np.zeros(2 * k.value * k.value)
            assert L.okr_result_ykron(h, k.value - 1, y.ctypes.data_as(C.c_void_p), None, C.byref(k)) == B.EINVAL
            ls, nb = C.c_int32(-1), C.c_int32(-1)
            assert L.okr_result_errors(h, None, None, None, None, C.byref(ls), C.byref(nb)) == B.OK
            assert (ls.value, nb.value) == (f.n_scen, f.n_bus)
        finally:
            B.lib().okr_result_free(h)


def test_torch_allocator_gives_the_same_results_and_gets_every_block_back(K):
    import torch
    f, run = fg.preset("feeder1000", n_bus=400)
    batch = [fb for fb, _ in fg.batch_presets(count=4, first_seed=7, n_lo=100, n_hi=300)]
    p = K.default_params(margin=run["margin"], target_reduction=0.5, precision=1)
    x = np.random.default_rng(0).normal(size=(700, 14)).astype(np.float32)

    def run_all(ctx):
        ctx.reduce(f, p)
        out = dict(dec=ctx.decisions(), sup=ctx.assignment(), yk=ctx.kron()[0])
        items, parts, _ = ctx.reduce_batch(batch, [K.default_params(margin=0.005, target_reduction=0.5)])
        out["batch"] = [it["smice"] for it in items]
        ctx.scorer_init(14, np.linspace(-0.01, 0.01, 14 * 128 + 128 + 2 * (128 * 128 + 128) + 129, dtype=np.float32))
        out["pred"] = ctx.scorer_predict(x)
        plan = ctx.batch_plan(batch, [K.default_params(margin=0.005, target_reduction=0.5)])
        try:
            out["plan"] = [it["smice"] for it in plan.run()[0]]
        finally:
            plan.close()
        return out

    with K.Context(0) as ref_ctx:
        ref = run_all(ref_ctx)
    live = {}
    calls = {"alloc": 0, "free": 0}

    def alloc(nbytes, device, stream):
        ptr = torch.cuda.caching_allocator_alloc(nbytes, device, stream)
        live[ptr] = nbytes
        calls["alloc"] += 1
        return ptr

    def free(ptr, device, stream):
        assert ptr in live
        del live[ptr]
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    base = torch.cuda.memory_allocated(0)
    ctx = K.Context(0)
    try:
        ctx.set_allocator(alloc, free)
        got = run_all(ctx)
        assert calls["alloc"] > 0 and len(live) > 0
        assert torch.cuda.memory_allocated(0) - base >= sum(live.values())   # accounted in torch
        for k in ("s", "r", "score"):
            assert np.array_equal(got["dec"][k], ref["dec"][k])
        assert np.array_equal(got["sup"], ref["sup"]) and np.array_equal(got["yk"], ref["yk"])
        assert got["batch"] == ref["batch"] and got["plan"] == ref["plan"]
        assert np.array_equal(got["pred"], ref["pred"])
        # the allocator can only be set on a context that holds no device memory
        from paper_2510_19608_gb300._binding import EINVAL
        with pytest.raises(K.OkrError) as ex:
            ctx.set_allocator(alloc, free)
        assert ex.value.status == EINVAL
    finally:
        ctx.close()
    assert not live and calls["alloc"] == calls["free"]

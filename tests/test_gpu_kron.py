"""Y_Kron on the GPU (okr_kron, through the C ABI) against the oracle's
elimination of every reduced bus (Sec. II-B, eq. Y_kron).

Both sides are FP64 and differ only in the route: the oracle eliminates buses
one at a time on the dense Y; the library inverts one small port-impedance
block per reduced component.  The bound is relative to the largest entry.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import feedergen as fg
from oracle import oracle as O

pytestmark = pytest.mark.gpu

Y_RTOL = 1e-10        # relative to max |Y_Kron|


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import build
    build.build()
    c = K.Context(0)
    yield c
    c.close()


def _hub(n_children, phases=7, seed=0):
    """Bus 1 under the slack with n_children buses below it."""
    rng = np.random.default_rng(seed)
    n = n_children + 2
    parent = [-1, 0] + [1] * n_children
    ph = [7, 7] + [phases] * n_children
    z = np.zeros((n, 3, 3, 2))
    s = np.zeros((2, n, 3, 2))
    for i in range(1, n):
        for a in range(3):
            for b in range(3):
                if ph[i] >> a & 1 and ph[i] >> b & 1:
                    z[i, a, b] = (0.004 + 0.002 * rng.random(), 0.008) if a == b else (0.001, 0.003 + 0.001 * rng.random())
            if ph[i] >> a & 1:
                s[0, i, a] = (0.01 * rng.random(), 0.003)
                s[1, i, a] = 0.3 * s[0, i, a]
    vs = np.array([[1.0, 0.0], [-0.5, -math.sqrt(3) / 2], [-0.5, math.sqrt(3) / 2]])
    return fg.Feeder(parent=np.array(parent, np.int32), phases=np.array(ph, np.uint8), z_line=z, s_load=s,
                     v_slack=vs, meta={})


def _compare(Yg, pg, f, kept):
    Yo, ko = O.kron(f, kept)
    assert np.array_equal(pg, ko)
    scale = np.abs(Yo).max()
    assert np.abs(Yg - Yo).max() <= Y_RTOL * scale, np.abs(Yg - Yo).max() / scale


@pytest.mark.parametrize("name,n", [("feeder40", None), ("feeder1000", None), ("feeder2200", 600)])
def test_kron_of_the_chosen_network(ctx, name, n):
    import paper_2510_19608_gb300 as K
    f, run = fg.preset(name, **({"n_bus": n} if n else {}))
    ctx.reduce(f, K.default_params(margin=run["margin"], target_reduction=run["target"], precision=1))
    sup = ctx.assignment()
    kept = (sup == np.arange(f.n_bus)).astype(np.uint8)
    Yg, pg = ctx.kron()
    _compare(Yg, pg, f, kept)
    assert ctx.summary()["kron_ms"] > 0.0


@pytest.mark.parametrize("frac", [0.05, 0.3, 0.6, 0.9])
def test_kron_of_random_kept_sets(ctx, frac):
    f, _ = fg.preset("feeder1000", n_bus=400)
    ctx.power_flow(f)
    rng = np.random.default_rng(int(frac * 100))
    kept = (rng.random(f.n_bus) < frac).astype(np.uint8)
    kept[0] = 1
    Yg, pg = ctx.kron(kept)
    _compare(Yg, pg, f, kept)


def test_kron_keeping_everything_is_y(ctx):
    f, _ = fg.preset("feeder40")
    ctx.power_flow(f)
    Yg, pg = ctx.kron(np.ones(f.n_bus, np.uint8))
    Y = O.ybus(f)
    assert Yg.shape == Y.shape
    assert np.abs(Yg - Y).max() <= 1e-12 * np.abs(Y).max()


def test_kron_keeping_only_the_slack_is_zero(ctx):
    f, _ = fg.preset("feeder40")
    ctx.power_flow(f)
    kept = np.zeros(f.n_bus, np.uint8)
    kept[0] = 1
    Yg, pg = ctx.kron(kept)
    assert list(pg) == [0, 1, 2]
    assert np.abs(Yg).max() == 0.0


@pytest.mark.parametrize("children,phases", [(30, 7), (50, 3), (21, 7)])
def test_kron_large_component_uses_global_scratch(ctx, children, phases):
    """A reduced hub with many kept children: one group of 63-100 phase-nodes,
    above the shared-memory size for the larger cases."""
    f = _hub(children, phases)
    ctx.power_flow(f)
    kept = np.ones(f.n_bus, np.uint8)
    kept[1] = 0
    Yg, pg = ctx.kron(kept)
    _compare(Yg, pg, f, kept)


def test_kron_rejects_a_reduced_slack(ctx):
    import paper_2510_19608_gb300 as K
    f, _ = fg.preset("feeder40")
    ctx.power_flow(f)
    kept = np.ones(f.n_bus, np.uint8)
    kept[0] = 0
    with pytest.raises(K.OkrError) as e:
        ctx.kron(kept)
    assert e.value.status == 1


def test_kron_needs_a_feeder():
    import paper_2510_19608_gb300 as K
    with K.Context(0) as c:
        with pytest.raises(K.OkrError) as e:
            c.kron()
        assert e.value.status == 6


# ----------------------------------------------------------------------------- Sec. V radialization
def _bus_graph(Y, pn, tol=0.0):
    bus = pn // 3
    buses = np.unique(bus)
    adj = {int(b): set() for b in buses}
    rows, cols = np.nonzero(np.abs(Y) > tol)
    for a, c in zip(rows, cols):
        if bus[a] != bus[c]:
            adj[int(bus[a])].add(int(bus[c]))
    return buses, adj


def _is_tree(buses, adj):
    if sum(len(v) for v in adj.values()) // 2 != len(buses) - 1:
        return False
    seen, stack = {int(buses[0])}, [int(buses[0])]
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == len(buses)


@pytest.mark.parametrize("name,n", [("feeder40", None), ("feeder1000", None), ("feeder2200", 600)])
def test_radialization_of_the_chosen_network(ctx, name, n):
    import paper_2510_19608_gb300 as K
    f, run = fg.preset(name, **({"n_bus": n} if n else {}))
    ctx.reduce(f, K.default_params(margin=run["margin"], target_reduction=run["target"], precision=1))
    kept = (ctx.assignment() == np.arange(f.n_bus)).astype(np.uint8)
    crit = ctx.radialize()
    assert np.array_equal(crit, O.radialize(f, kept))
    Yr, pr = ctx.kron(np.maximum(kept, crit))
    assert _is_tree(*_bus_graph(Yr, pr))


@pytest.mark.parametrize("frac", [0.2, 0.5, 0.8])
def test_radialization_of_random_kept_sets(ctx, frac):
    f, _ = fg.preset("feeder1000", n_bus=300)
    ctx.power_flow(f)
    kept = (np.random.default_rng(int(100 * frac)).random(f.n_bus) < frac).astype(np.uint8)
    kept[0] = 1
    crit = ctx.radialize(kept)
    assert np.array_equal(crit, O.radialize(f, kept))
    Yr, pr = ctx.kron(np.maximum(kept, crit))
    assert _is_tree(*_bus_graph(Yr, pr))


def test_radialization_of_a_hub(ctx):
    f = _hub(5)
    ctx.power_flow(f)
    kept = np.ones(f.n_bus, np.uint8)
    kept[1] = 0
    assert list(ctx.radialize(kept)) == [0, 1] + [0] * 5

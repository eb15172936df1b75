"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU.  Each checks the oracle against something
other than itself: closed forms, independent numpy routes (dense inverses,
Moore-Penrose Kron reduction on the padded matrix), invariants of Kron
reduction (Sec. II-B, Lemma 2), brute force over all candidates through the
Kron route (Algorithm 1), and global brute force over all assignments
(Sec. II-C rules).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import feedergen as fg
from oracle import oracle as O
from tests import kron_route as KR


def small(n, seed, **kw):
    kw.setdefault("kv_ll", 4.16)
    kw.setdefault("phase_mode", "keep")
    return fg.make_feeder(n, seed, **kw)


def three_phase_only(n, seed):
    return small(n, seed, phase_mode=(1.0, 0.0, 0.0))


# --------------------------------------------------------------------------- generator
def test_generator_is_deterministic_and_valid():
    a = small(60, 11)
    b = small(60, 11)
    for x, y in ((a.parent, b.parent), (a.phases, b.phases), (a.z_line, b.z_line), (a.s_load, b.s_load)):
        assert np.array_equal(x, y)
    assert a.parent[0] == -1 and all(a.parent[i] < i for i in range(1, 60))
    for i in range(1, 60):
        assert (a.phases[i] & a.phases[a.parent[i]]) == a.phases[i]
        absent = [p for p in range(3) if not a.phases[i] >> p & 1]
        assert np.all(a.z_line[i][absent] == 0) and np.all(a.z_line[i][:, absent] == 0)
        assert np.all(a.s_load[:, i][:, absent] == 0)
    # symmetric impedances, light scenario = 0.3 x heavy
    z = KR.zc(a)
    assert np.allclose(z, np.transpose(z, (0, 2, 1)))
    assert np.allclose(a.s_load[1], 0.3 * a.s_load[0])


# --------------------------------------------------------------------------- Y and Z
@pytest.mark.parametrize("seed", [3, 4])
def test_ybus_matches_padded_stamp_and_invariants(seed):
    f = small(25, seed)
    Y = O.ybus(f)
    Yp = KR.padded_y(f)
    pres = KR.present(f)
    assert np.allclose(Y, Yp[np.ix_(pres, pres)], rtol=0, atol=1e-9 * np.abs(Yp).max())
    assert np.allclose(Y, Y.T, rtol=0, atol=1e-9 * np.abs(Y).max())       # complex symmetric
    # series-only lines: the same three-phase vector at every bus draws no current
    for v3 in (np.array([1.0, -0.5 - 0.8j, -0.5 + 0.8j]), np.array([0.3 + 0.1j, 2.0, -1.0j])):
        v = np.tile(v3, f.n_bus)[pres]
        assert np.abs(Y @ v).max() <= 1e-9 * np.abs(Y).max()


@pytest.mark.parametrize("seed", [5, 6])
def test_zbus_equals_path_impedance_closed_form_and_inverse(seed):
    f = small(30, seed)
    n = f.n_bus
    Zo = O.zbus(f).reshape(3 * n, 3 * n).T          # Zo[(i,p),(j,q)]
    Zc = KR.z_closed_form(f)
    scale = np.abs(Zc).max()
    assert np.abs(Zo - Zc).max() <= 1e-12 * scale
    # and the dense inverse of the non-slack block of Y
    pres = KR.present(f)
    rows = np.where(pres)[0]
    nonslack = rows[rows >= 3]
    Yp = KR.padded_y(f)
    Zinv = np.linalg.inv(Yp[np.ix_(nonslack, nonslack)])
    assert np.abs(Zinv - Zc[np.ix_(nonslack, nonslack)]).max() <= 1e-9 * scale


def test_tree_solve_matches_dense_solve():
    f = small(35, 8)
    n = f.n_bus
    rng = np.random.default_rng(0)
    pres = KR.present(f)
    b = (rng.normal(size=(2, n, 3)) + 1j * rng.normal(size=(2, n, 3))) * pres.reshape(n, 3)
    v0 = np.array([1.0, np.exp(-2j * np.pi / 3), np.exp(2j * np.pi / 3)])
    V = O.tree_solve(f, b, v0)
    Yp = KR.padded_y(f)
    rows = np.where(pres)[0]
    ns = rows[rows >= 3]
    for l in range(2):
        rhs = b[l].reshape(-1)[ns] - Yp[np.ix_(ns, [0, 1, 2])] @ v0
        ref = np.linalg.solve(Yp[np.ix_(ns, ns)], rhs)
        assert np.abs(V[l].reshape(-1)[ns] - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
        assert np.allclose(V[l, 0], v0)


# --------------------------------------------------------------------------- load flow
def _one_line_feeder(r, x, p, q, phases=1):
    parent = np.array([-1, 0], np.int32)
    ph = np.array([7, phases], np.uint8)
    z = np.zeros((2, 3, 3, 2))
    s = np.zeros((1, 2, 3, 2))
    for k in range(3):
        if phases >> k & 1:
            z[1, k, k] = (r, x)
            s[0, 1, k] = (p, q)
    vs = np.array([[1.0, 0.0], [-0.5, -math.sqrt(3) / 2], [-0.5, math.sqrt(3) / 2]])
    return fg.Feeder(parent=parent, phases=ph, z_line=z, s_load=s, v_slack=vs, meta={})


@pytest.mark.parametrize("r,x,p,q", [(0.01, 0.02, 0.5, 0.2), (0.03, 0.05, 1.2, 0.4), (0.002, 0.004, 0.1, 0.0)])
def test_pf_single_line_closed_form(r, x, p, q):
    """One line, one phase, constant-power load: the receiving-end magnitude solves
    |V|^4 + (2(rP + xQ) - |V0|^2)|V|^2 + |z|^2|S|^2 = 0 (larger root)."""
    f = _one_line_feeder(r, x, p, q)
    v, _ = O.power_flow(f)
    b = 1.0 - 2.0 * (r * p + x * q)
    c = (r * r + x * x) * (p * p + q * q)
    v2 = 0.5 * (b + math.sqrt(b * b - 4.0 * c))
    assert abs(abs(v[0, 1, 0]) - math.sqrt(v2)) <= 1e-12


def test_pf_satisfies_kcl_with_constant_power_loads():
    f, _ = fg.preset("feeder40")
    v, sweeps = O.power_flow(f)
    inj = O.injection(f, v)
    s = f.s_load[..., 0] + 1j * f.s_load[..., 1]
    pres = KR.present(f).reshape(f.n_bus, 3)
    for l in range(f.n_scen):
        for i in range(1, f.n_bus):
            for p in range(3):
                if pres[i, p]:
                    load = np.conj(s[l, i, p] / v[l, i, p])
                    assert abs(inj[l, i, p] + load) <= 1e-9
    assert sweeps < 50


# --------------------------------------------------------------------------- Kron reduction
@pytest.mark.parametrize("seed", [21, 22, 23])
def test_kron_matches_pinv_route_and_invariants(seed):
    f = small(16, seed)
    n = f.n_bus
    rng = np.random.default_rng(seed)
    kept = rng.random(n) < 0.45
    kept[0] = True
    Yk, kidx = O.kron(f, kept.astype(np.uint8))
    Yp = KR.padded_y(f)
    ref = KR.kron_pinv(Yp, np.repeat(kept, 3))
    K = np.where(np.repeat(kept, 3))[0]
    sel = [list(K).index(k) for k in kidx]
    ref = ref[np.ix_(sel, sel)]
    scale = np.abs(ref).max()
    assert np.abs(Yk - ref).max() <= 1e-9 * scale
    assert np.abs(Yk - Yk.T).max() <= 1e-9 * scale                         # symmetric
    v3 = np.array([1.0, -0.5 - 0.8j, -0.5 + 0.8j])
    ones = np.array([v3[k % 3] for k in kidx])
    assert np.abs(Yk @ ones).max() <= 1e-8 * scale                          # zero "row sums"
    # without the slack, Y_Kron^{-1} is Z restricted to the kept phase nodes
    nz = [a for a, k in enumerate(kidx) if k >= 3]
    Zc = KR.z_closed_form(f)
    zk = Zc[np.ix_(kidx[nz], kidx[nz])]
    assert np.abs(np.linalg.inv(Yk[np.ix_(nz, nz)]) - zk).max() <= 1e-8 * np.abs(zk).max()


def test_kron_solve_equals_full_solve_with_aggregated_injections():
    """Sec. IV: solving the full network with the aggregated injections gives the
    super-node voltages of the Kron-reduced network."""
    f = small(18, 31)
    vhat, ihat = O.operating_points(f)
    rng = np.random.default_rng(1)
    n = f.n_bus
    # a valid assignment: fold random leaves into their parents
    sup = np.arange(n)
    for i in range(n - 1, 0, -1):
        p = f.parent[i]
        if rng.random() < 0.4 and sup[p] == p and (f.phases[i] & f.phases[p]) == f.phases[i] and p != 0:
            sup[sup == i] = p
    vk = KR.kron_route_voltages(f, KR.padded_y(f), sup, ihat)
    agg = np.zeros_like(ihat)
    for i in range(n):
        agg[:, sup[i]] += ihat[:, i]
    vfull = O.tree_solve(f, agg)
    pres = KR.present(f).reshape(n, 3)
    for i in range(n):
        k = sup[i]
        for p in range(3):
            if pres[i, p]:
                assert abs(vk[:, i, p] - vfull[:, k, p]).max() <= 1e-10


def _block_pattern(Yk, kidx, n):
    pat = np.zeros((n, n), bool)
    for a, ka in enumerate(kidx):
        for b, kb in enumerate(kidx):
            if abs(Yk[a, b]) > 1e-12 * np.abs(Yk).max():
                pat[ka // 3, kb // 3] = True
    return pat


@pytest.mark.parametrize("seed", [41, 42])
def test_lemma2_single_elimination_topology(seed):
    """Lemma 2: eliminating bus r makes its neighbours a clique and leaves every
    other coupling alone; the three-phase pattern equals the one-phase pattern."""
    f3 = three_phase_only(14, seed)
    n = f3.n_bus
    z1 = np.zeros_like(f3.z_line)
    z1[:, 0, 0] = f3.z_line[:, 0, 0]
    f1 = fg.Feeder(parent=f3.parent.copy(), phases=np.ones(n, np.uint8), z_line=z1,
                   s_load=f3.s_load.copy(), v_slack=f3.v_slack.copy(), meta={})
    for r in range(1, n):
        kept = np.ones(n, np.uint8)
        kept[r] = 0
        p3 = _block_pattern(*O.kron(f3, kept), n)
        Yk1, k1 = O.kron(f1, kept)
        p1 = _block_pattern(Yk1, k1, n)
        assert np.array_equal(p3, p1)
        nb = [int(f3.parent[r])] + [i for i in range(n) if f3.parent[i] == r]
        for a in range(n):
            for b in range(n):
                if a == r or b == r or a == b:
                    continue
                orig = f3.parent[a] == b or f3.parent[b] == a
                expect = orig or (a in nb and b in nb)
                assert p3[a, b] == expect


def test_reduced_graph_is_edge_disjoint_union_of_maximal_cliques():
    nx = pytest.importorskip("networkx")
    f = three_phase_only(20, 51)
    n = f.n_bus
    rng = np.random.default_rng(5)
    kept = (rng.random(n) < 0.5).astype(np.uint8)
    kept[0] = 1
    Yk, kidx = O.kron(f, kept)
    pat = _block_pattern(Yk, kidx, n)
    g = nx.Graph()
    ks = [i for i in range(n) if kept[i]]
    g.add_nodes_from(ks)
    for a in ks:
        for b in ks:
            if a < b and pat[a, b]:
                g.add_edge(a, b)
    cliques = [c for c in nx.find_cliques(g) if len(c) >= 2]
    seen = set()
    for c in cliques:
        for a in c:
            for b in c:
                if a < b:
                    assert (a, b) not in seen          # edge-disjoint
                    seen.add((a, b))
    assert seen == {(a, b) for a, b in g.edges for a, b in [tuple(sorted((a, b)))]}


# --------------------------------------------------------------------------- Algorithm 1
def test_identity_assignment_reproduces_full_voltages():
    f, _ = fg.preset("feeder40")
    vhat, ihat = O.operating_points(f)
    for mode, tol in (("delta", 1e-15), ("literal", 1e-11)):
        res = O.reduce(f, vhat, ihat, margin=0.005, max_merges=0, mode=mode)
        assert res["n_iter"] == 0
        assert np.abs(res["v_red"] - vhat).max() <= tol


def test_single_line_candidate_closed_form():
    f = _one_line_feeder(0.02, 0.04, 0.8, 0.3)
    f.s_load = np.concatenate([f.s_load, 0.3 * f.s_load])
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=1.0, max_merges=1, record_iters=1)
    rec = res["recorded"][0]
    assert list(zip(rec["s"], rec["r"])) == [(0, 1)]
    expect = 0.0
    for l, (p, q) in enumerate([(0.8, 0.3), (0.24, 0.09)]):
        b = 1.0 - 2.0 * (0.02 * p + 0.04 * q)
        c = (0.02 ** 2 + 0.04 ** 2) * (p * p + q * q)
        expect += 1.0 - math.sqrt(0.5 * (b + math.sqrt(b * b - 4 * c)))
    assert abs(rec["score"][0] - expect) <= 1e-12
    assert res["n_iter"] == 1 and res["s"][0] == 0 and res["r"][0] == 1


def test_candidate_count_identity_all_three_phase():
    """|A(t)| = 2 (n_s - 1) minus the quotient degree of the slack (never reduced)."""
    f = three_phase_only(60, 61)
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=0.05, max_merges=40)
    n = f.n_bus
    sup = np.arange(n)
    for t in range(res["n_iter"]):
        ns = len(set(sup.tolist()))
        deg_root = len({int(sup[i]) for i in range(1, n) if sup[f.parent[i]] == 0 and sup[i] != 0})
        assert res["ncand"][t] == 2 * (ns - 1) - deg_root
        s, r = res["s"][t], res["r"][t]
        sup[sup == r] = s


def _candidates(f, sup):
    n = f.n_bus
    out = set()
    for i in range(1, n):
        a, b = int(sup[f.parent[i]]), int(sup[i])
        if a == b:
            continue
        for s, r in ((a, b), (b, a)):
            if r != 0 and (f.phases[r] & f.phases[s]) == f.phases[r]:
                out.add((s, r))
    return sorted(out)


def _tie_pick(scores: dict, tau: float):
    if not scores:
        return None
    m = min(scores.values())
    if m == math.inf:
        return None
    band = [c for c, v in scores.items() if v <= m + tau]
    return min(band, key=lambda c: (c[1], c[0]))


@pytest.mark.parametrize("seed,n,objective,mode", [(71, 9, 0, "literal"), (72, 11, 0, "delta"),
                                                   (73, 12, 0, "delta"), (74, 10, 1, "delta"),
                                                   (75, 12, 1, "literal")])
def test_every_candidate_against_kron_route(seed, n, objective, mode):
    """Brute force: each candidate of each iteration scored by forming the
    Kron-reduced network of its post-merge super-nodes with the pseudo-inverse
    and solving it; scores, candidate sets and decisions must agree."""
    f = small(n, seed)
    vhat, ihat = O.operating_points(f)
    margin = 0.004
    res = O.reduce(f, vhat, ihat, margin=margin, max_merges=n, objective=objective, mode=mode,
                   record_iters=n)
    Yp = KR.padded_y(f)
    sup = np.arange(n)
    for t in range(res["n_iter"] + (1 if res["stop_reason"] == 1 else 0)):
        rec = res["recorded"][t]
        cands = _candidates(f, sup)
        got = {(int(s), int(r)): float(v) for s, r, v in zip(rec["s"], rec["r"], rec["score"])}
        assert sorted(got) == cands
        ref = {c: KR.kron_route_score(f, Yp, vhat, ihat, sup, c[0], c[1], margin, objective)[0] for c in cands}
        for c in cands:
            if math.isinf(ref[c]) or math.isinf(got[c]):
                assert math.isinf(ref[c]) and math.isinf(got[c]), c
            else:
                assert abs(ref[c] - got[c]) <= 1e-12, (t, c, ref[c], got[c])
        pick = _tie_pick(ref, 1e-9)
        if t == res["n_iter"]:
            assert pick is None
            break
        assert pick == (res["s"][t], res["r"][t])
        s, r = pick
        sup[sup == r] = s


@pytest.mark.parametrize("seed", [81, 82, 83])
def test_greedy_is_feasible_and_never_beats_global_optimum(seed):
    """All connected, phase-feasible assignments of an 8-bus feeder: the greedy
    result is feasible and reduces no more buses than the best feasible one."""
    n = 8
    f = small(n, seed)
    vhat, ihat = O.operating_points(f)
    margin = 0.002
    res = O.reduce(f, vhat, ihat, margin=margin, max_merges=n)
    Yp = KR.padded_y(f)
    sup = res["super_of"]
    score, maxe = KR.score_from_voltages(f, vhat, KR.kron_route_voltages(f, Yp, sup, ihat), sup, margin)
    assert maxe <= margin
    best = 0
    for cand in KR.connected_partitions(f):
        red = n - len(set(cand.tolist()))
        if red <= best:
            continue
        _, me = KR.score_from_voltages(f, vhat, KR.kron_route_voltages(f, Yp, cand, ihat), cand, margin)
        if me <= margin:
            best = red
    assert res["n_iter"] <= best


def test_literal_and_delta_agree_on_feeder40():
    f, run = fg.preset("feeder40")
    vhat, ihat = O.operating_points(f)
    a = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=f.n_bus, mode="literal")
    b = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=f.n_bus, mode="delta")
    assert a["n_iter"] == b["n_iter"] and a["stop_reason"] == b["stop_reason"]
    assert np.array_equal(a["s"], b["s"]) and np.array_equal(a["r"], b["r"])
    assert np.abs(a["score"] - b["score"]).max() <= 1e-11
    assert np.abs(a["v_red"] - b["v_red"]).max() <= 1e-11


def test_decisions_do_not_depend_on_thread_count():
    f = small(120, 91, kv_ll=12.47, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0))
    vhat, ihat = O.operating_points(f)
    outs = []
    for t in (1, max(2, O.num_threads())):
        O.set_threads(t)
        outs.append(O.reduce(f, vhat, ihat, margin=0.005, max_merges=60, record_iters=3))
    O.set_threads(0)
    a, b = outs
    for k in ("s", "r", "score", "maxerr", "super_of"):
        assert np.array_equal(a[k], b[k])
    for ra, rb in zip(a["recorded"], b["recorded"]):
        assert np.array_equal(ra["score"], rb["score"])


def test_stops_when_no_candidate_is_feasible():
    f, run = fg.preset("feeder40")
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=f.n_bus, record_iters=f.n_bus)
    assert res["stop_reason"] == 1
    last = res["recorded"][res["n_iter"]]
    assert np.all(np.isinf(last["score"]))
    assert res["maxerr"].max() <= run["margin"]


def test_transposes_pinned_with_nonsymmetric_lines():
    """Physical line impedances are symmetric, which hides a transposed operand.
    With a non-symmetric z (the stamp [y, -y; -y, y] still holds) the tree
    factorization, Z and the Kron elimination must still match the dense routes."""
    f = small(14, 97)
    rng = np.random.default_rng(97)
    for i in range(1, f.n_bus):
        ps = [p for p in range(3) if f.phases[i] >> p & 1]
        for a in ps:
            for b in ps:
                if a < b:
                    d = rng.uniform(0.1, 0.3) * f.z_line[i, a, b]
                    f.z_line[i, a, b] += d
                    f.z_line[i, b, a] -= d
    n = f.n_bus
    Zo = O.zbus(f).reshape(3 * n, 3 * n).T
    Zc = KR.z_closed_form(f)
    assert np.abs(Zo - Zc).max() <= 1e-12 * np.abs(Zc).max()
    kept = np.ones(n, np.uint8)
    kept[[2, 5, 6, 9]] = 0
    Yk, kidx = O.kron(f, kept)
    ref = KR.kron_pinv(KR.padded_y(f), np.repeat(kept.astype(bool), 3))
    K = list(np.where(np.repeat(kept.astype(bool), 3))[0])
    sel = [K.index(k) for k in kidx]
    ref = ref[np.ix_(sel, sel)]
    assert np.abs(Yk - ref).max() <= 1e-9 * np.abs(ref).max()
    assert np.abs(Yk - Yk.T).max() > 1e-6 * np.abs(Yk).max()     # really non-symmetric


def test_golden_feeder40_decision_sequence():
    """Regression against tests/golden/feeder40_decisions.txt (written by
    tests/golden/make_golden.py from the oracle alone)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "feeder40_decisions.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    f, run = fg.preset("feeder40")
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=f.n_bus, mode="delta")
    assert res["n_iter"] == len(rows)
    for t, row in enumerate(rows):
        assert (res["s"][t], res["r"][t]) == (int(row[1]), int(row[2]))
        assert abs(res["score"][t] - float(row[3])) <= 1e-11
        assert abs(res["maxerr"][t] - float(row[4])) <= 1e-12


# ----------------------------------------------------------------------------- Sec. V radialization
def _is_tree(buses, adj):
    edges = sum(len(v) for v in adj.values()) // 2
    if edges != len(buses) - 1:
        return False
    seen, stack = {int(buses[0])}, [int(buses[0])]
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == len(buses)


def _star_feeder(children):
    parent = [-1, 0] + [1] * children
    return _simple_feeder(parent, [7] * len(parent))


def _simple_feeder(parent, phases):
    n = len(parent)
    z = np.zeros((n, 3, 3, 2))
    s = np.zeros((2, n, 3, 2))
    rng = np.random.default_rng(n)
    for i in range(1, n):
        for a in range(3):
            for b in range(3):
                if phases[i] >> a & 1 and phases[i] >> b & 1:
                    z[i, a, b] = (0.004 + 0.001 * rng.random(), 0.008) if a == b else (0.001, 0.003)
    vs = np.array([[1.0, 0.0], [-0.5, -math.sqrt(3) / 2], [-0.5, math.sqrt(3) / 2]])
    return fg.Feeder(parent=np.array(parent, np.int32), phases=np.array(phases, np.uint8), z_line=z, s_load=s,
                     v_slack=vs, meta={})


def test_radialize_star_marks_the_hub_and_a_chain_needs_nothing():
    f = _star_feeder(3)                               # 0 - 1 - {2, 3, 4}
    kept = np.array([1, 0, 1, 1, 1], np.uint8)        # Kron graph: the 4-clique {0, 2, 3, 4}
    assert list(O.radialize(f, kept)) == [0, 1, 0, 0, 0]
    chain = _simple_feeder([-1, 0, 1, 2, 3, 4], [7] * 6)
    assert not O.radialize(chain, np.array([1, 0, 1, 0, 0, 1], np.uint8)).any()
    # two children kept under a reduced bus only: a 3-clique with the parent side
    assert list(O.radialize(_star_feeder(2), np.array([1, 0, 1, 1], np.uint8))) == [0, 1, 0, 0]


@pytest.mark.parametrize("seed,frac", [(1, 0.3), (2, 0.5), (3, 0.7)])
def test_radialized_network_is_radial_and_minimal(seed, frac):
    f, _ = fg.preset("feeder1000", n_bus=120, seed=seed)
    kept = (np.random.default_rng(seed).random(f.n_bus) < frac).astype(np.uint8)
    kept[0] = 1
    crit = O.radialize(f, kept)
    rad = np.maximum(kept, crit)
    buses, adj = O.kron_graph(f, rad)
    assert _is_tree(buses, adj)
    if not crit.any():
        assert _is_tree(*O.kron_graph(f, kept))
    for c in np.nonzero(crit)[0][:6]:                 # each critical bus is needed
        less = rad.copy()
        less[c] = 0
        assert not _is_tree(*O.kron_graph(f, less))


def test_radialization_keeps_super_node_voltages():
    """Sec. V: critical buses added without injections leave the super-node
    voltages of the Kron-reduced network unchanged."""
    f, run = fg.preset("feeder1000", n_bus=150)
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=0.005, max_merges=90)
    sup = res["super_of"]
    kept = (sup == np.arange(f.n_bus)).astype(np.uint8)
    crit = O.radialize(f, kept)
    assert crit.any()
    iagg = np.zeros((ihat.shape[0], 3 * f.n_bus), dtype=np.complex128)
    for l in range(ihat.shape[0]):
        for i in range(f.n_bus):
            iagg[l, 3 * sup[i]:3 * sup[i] + 3] += ihat[l, i]
    Ypad = KR.padded_y(f)
    v1 = KR.kron_kept_voltages(f, Ypad, kept, iagg)
    v2 = KR.kron_kept_voltages(f, Ypad, np.maximum(kept, crit), iagg)
    rows = np.repeat(kept.astype(bool), 3) & KR.present(f)
    assert np.abs(v1[:, rows] - v2[:, rows]).max() <= 1e-12


# ----------------------------------------------------------------------------- evaluation of a given network
def test_evaluate_identity_assignment_is_exact():
    f, _ = fg.preset("feeder40")
    err, vred = O.evaluate(f, np.arange(f.n_bus))
    vhat, _ = O.operating_points(f)
    assert err.max() <= 1e-12 and np.abs(vred - vhat).max() <= 1e-12


def test_evaluate_reproduces_the_search_result():
    """Algorithm 1's own voltages and largest error for its final network equal
    the evaluation of that network by a separate route (tree solve)."""
    f, run = fg.preset("feeder1000", n_bus=120)
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=0.005, max_merges=60)
    err, vred = O.evaluate(f, res["super_of"])
    assert abs(err.max() - res["maxerr"][-1]) <= 1e-12
    assert np.abs(vred - res["v_red"]).max() <= 1e-12

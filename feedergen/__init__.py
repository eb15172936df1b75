"""Seeded synthetic three-phase radial feeders.

This module only draws random inputs: a radial tree, per-bus phase sets, per-line
series impedances and per-phase constant-power loads for a few loading
scenarios.  It holds none of the reduction method's arithmetic and is the one
module that both the CUDA library's tests/benchmark and the CPU oracle use.

Shapes follow the paper's workloads (Section VI: unbalanced radial feeders with
single-, two- and three-phase laterals and two loading scenarios, the heaviest and
the lightest of a set of load profiles).  The distributions are:

* tree: breadth-first; each popped bus receives U{1,2,3} children until ``n_bus``
  buses exist.  Bus 0 is the substation (slack) and ``parent[i] < i``.
* phases: bus 0 carries {a,b,c}.  ``phase_mode="keep"``: a child keeps its
  parent's phases with probability 0.7, otherwise a uniformly drawn proper
  non-empty subset of them.  ``phase_mode=(f3,f2,f1)``: the target share of
  three-, two- and one-phase buses.  Phase counts can only drop along a line.
  The trunk stays three-phase: only a line whose child subtree holds at most 5 %
  of the buses (a lateral) may drop its child's count, with probability ``q``
  (3 -> 2 with probability ``q*w``, 3 -> 1 with ``q*(1-w)``, 2 -> 1 with ``q``).
  ``q`` and ``w`` are fitted (bisection over the exact expected shares on the
  drawn tree, no randomness) so that the expected shares equal the target.  The
  kept subset is drawn uniformly among the parent's phases.
* line impedance per mile: symmetric complex 3x3, self R U(0.3,0.6) ohm, self X
  U(0.6,1.4) ohm, mutual R U(0.05,0.15) ohm, mutual X U(0.2,0.5) ohm; length
  lognormal(ln 0.1 mi, 0.7) clipped to [0.02, 0.5] mi; restricted to the child's
  phases (entries of absent phases are zero).
* per unit: S_base = 1 MVA three-phase, V_base = V_LL/sqrt(3), so
  Z_base = V_LL^2 / S_base and a per-phase load is divided by S_base/3.
* loads: a fraction ``unloaded_frac`` of non-root buses has no load; the others
  draw, per present phase, P from ``load`` and a lagging power factor from
  ``pf_range``.
* scenario 0 is the heavy case, scenario 1 is ``light_factor`` times it.
* load scaling (deterministic, needs no power flow): with the heavy loads, the
  linear voltage-drop bound ``drop(i,p) = sum_{lines e on root->i} sum_q
  |z_e[p,q]| * D_e[q]`` (``D_e[q]`` = total |S| of phase q below e) is computed
  and all loads are multiplied by ``lam = min(1, drop_target / max drop)``.
  This keeps the synthetic feeders in a realistic operating range, as measured
  feeders are.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Feeder", "make_feeder", "preset", "batch_presets", "PRESETS", "daily_profiles", "with_loads",
           "fingerprint"]


@dataclasses.dataclass
class Feeder:
    """A radial feeder as plain arrays (host memory, C-contiguous)."""

    parent: np.ndarray      # int32 [n]; parent[0] = -1, parent[i] < i
    phases: np.ndarray      # uint8 [n]; bit0=a, bit1=b, bit2=c
    z_line: np.ndarray      # float64 [n,3,3,2]; p.u. series impedance of line parent(i)->i
    s_load: np.ndarray      # float64 [L,n,3,2]; p.u. per-phase constant-power load
    v_slack: np.ndarray     # float64 [3,2]; slack voltage (p.u.)
    meta: dict

    @property
    def n_bus(self) -> int:
        return int(self.parent.shape[0])

    @property
    def n_scen(self) -> int:
        return int(self.s_load.shape[0])

    @property
    def n_phase_nodes(self) -> int:
        return int(sum(bin(int(p)).count("1") for p in self.phases))


def _bits(mask: int) -> list[int]:
    return [p for p in range(3) if mask >> p & 1]


def _mask(ps) -> int:
    m = 0
    for p in ps:
        m |= 1 << int(p)
    return m


def _levels(parent: np.ndarray) -> list[np.ndarray]:
    """Bus indices grouped by depth (root excluded), parents before children."""
    n = parent.shape[0]
    depth = np.zeros(n, dtype=np.int64)
    for i in range(1, n):
        depth[i] = depth[parent[i]] + 1
    return [np.nonzero(depth == d)[0] for d in range(1, int(depth.max()) + 1)] if n > 1 else []


def _chain_shares(parent: np.ndarray, elig: np.ndarray, q: float, w: float, levels=None) -> tuple[float, float]:
    """Exact expected (three-phase, two-phase) shares of the lateral drop chain."""
    n = parent.shape[0]
    if levels is None:
        levels = _levels(parent)
    pr = np.zeros((n, 3))
    pr[0, 0] = 1.0
    qv = np.where(elig, q, 0.0)
    for idx in levels:                         # element-wise the same arithmetic as a bus-by-bus loop
        par = parent[idx]
        a3, a2, a1 = pr[par, 0], pr[par, 1], pr[par, 2]
        qq = qv[idx]
        pr[idx, 0] = a3 * (1.0 - qq)
        pr[idx, 1] = a3 * qq * w + a2 * (1.0 - qq)
        pr[idx, 2] = a3 * qq * (1.0 - w) + a2 * qq + a1
    m = pr.mean(axis=0)
    return float(m[0]), float(m[1])


def _fit_phase_chain(parent: np.ndarray, elig: np.ndarray, mix) -> tuple[float, float]:
    """Fit (q, w) so that the expected three- and two-phase shares match ``mix``."""
    f3, f2 = float(mix[0]), float(mix[1])
    levels = _levels(parent)
    lo, hi = 0.0, 1.0
    for _ in range(50):                       # three-phase share falls with q
        q = 0.5 * (lo + hi)
        if _chain_shares(parent, elig, q, 0.5, levels)[0] > f3:
            lo = q
        else:
            hi = q
    q = 0.5 * (lo + hi)
    lo, hi = 0.0, 1.0
    for _ in range(50):                       # two-phase share rises with w
        w = 0.5 * (lo + hi)
        if _chain_shares(parent, elig, q, w, levels)[1] < f2:
            lo = w
        else:
            hi = w
    return q, 0.5 * (lo + hi)


def make_feeder(n_bus: int, seed: int, *, kv_ll: float = 12.47, phase_mode="keep",
                load=("uniform", 50.0), pf_range=(0.9, 0.98), unloaded_frac: float = 0.3,
                n_scen: int = 2, light_factor: float = 0.3, drop_target: float = 0.10,
                s_base_mva: float = 1.0) -> Feeder:
    """Draw one feeder.  The order of random draws is part of the definition."""
    if n_bus < 2:
        raise ValueError("a feeder needs at least 2 buses")
    if n_scen < 1:
        raise ValueError("n_scen must be >= 1")
    rng = np.random.default_rng(seed)

    # --- tree (breadth first) -------------------------------------------------
    parent = np.full(n_bus, -1, dtype=np.int32)
    queue = [0]
    nxt = 1
    head = 0
    while nxt < n_bus:
        b = queue[head]
        head += 1
        k = int(rng.integers(1, 4))
        for _ in range(min(k, n_bus - nxt)):
            parent[nxt] = b
            queue.append(nxt)
            nxt += 1

    # --- phases ---------------------------------------------------------------
    if phase_mode != "keep":
        size = np.ones(n_bus, dtype=np.int64)
        for i in range(n_bus - 1, 0, -1):
            size[parent[i]] += size[i]
        elig = size <= max(1, int(0.05 * n_bus))
        q_drop, w_two = _fit_phase_chain(parent, elig, phase_mode)
    phases = np.zeros(n_bus, dtype=np.uint8)
    phases[0] = 7
    for i in range(1, n_bus):
        pp = _bits(int(phases[parent[i]]))
        if phase_mode == "keep":
            u = rng.random()
            if u < 0.7 or len(pp) == 1:
                ps = pp
            else:
                k = int(rng.integers(1, len(pp)))          # proper, non-empty
                ps = sorted(rng.choice(pp, size=k, replace=False).tolist())
        else:
            m = len(pp)
            u = rng.random()
            qq = q_drop if elig[i] else 0.0
            if m == 3:
                k = 3 if u >= qq else (2 if u < qq * w_two else 1)
            elif m == 2:
                k = 2 if u >= qq else 1
            else:
                k = 1
            ps = pp if k == m else sorted(rng.choice(pp, size=k, replace=False).tolist())
        phases[i] = _mask(ps)

    # --- line impedances ------------------------------------------------------
    z_base = kv_ll * kv_ll / s_base_mva
    z_line = np.zeros((n_bus, 3, 3, 2), dtype=np.float64)
    lengths = np.zeros(n_bus)
    for i in range(1, n_bus):
        zr = np.zeros((3, 3))
        zx = np.zeros((3, 3))
        for p in range(3):
            zr[p, p] = rng.uniform(0.3, 0.6)
            zx[p, p] = rng.uniform(0.6, 1.4)
        for p in range(3):
            for q in range(p + 1, 3):
                zr[p, q] = zr[q, p] = rng.uniform(0.05, 0.15)
                zx[p, q] = zx[q, p] = rng.uniform(0.2, 0.5)
        length = float(np.clip(rng.lognormal(math.log(0.1), 0.7), 0.02, 0.5))
        lengths[i] = length
        ps = _bits(int(phases[i]))
        for p in ps:
            for q in ps:
                z_line[i, p, q, 0] = zr[p, q] * length / z_base
                z_line[i, p, q, 1] = zx[p, q] * length / z_base

    # --- loads (heavy scenario, kW / kvar per phase) ---------------------------
    s_heavy = np.zeros((n_bus, 3), dtype=np.complex128)
    for i in range(1, n_bus):
        if rng.random() < unloaded_frac:
            continue
        for p in _bits(int(phases[i])):
            if load[0] == "uniform":
                pkw = rng.uniform(0.0, load[1])
            elif load[0] == "lognormal":
                pkw = rng.lognormal(math.log(load[1]), load[2])
            else:
                raise ValueError(f"unknown load distribution {load[0]!r}")
            pf = rng.uniform(*pf_range)
            qkvar = pkw * math.tan(math.acos(pf))
            s_heavy[i, p] = complex(pkw, qkvar) / (s_base_mva * 1000.0 / 3.0)

    # --- deterministic load scaling (linear drop bound, no power flow) --------
    absz = np.hypot(z_line[..., 0], z_line[..., 1])           # [n,3,3]
    down = np.abs(s_heavy).copy()                             # [n,3] subtree |S|
    for i in range(n_bus - 1, 0, -1):
        down[parent[i]] += down[i]
    drop = np.zeros((n_bus, 3))
    for i in range(1, n_bus):
        drop[i] = drop[parent[i]] + absz[i] @ down[i]
    worst = float(drop.max())
    lam = 1.0 if worst <= drop_target else drop_target / worst
    s_heavy *= lam

    s_load = np.zeros((n_scen, n_bus, 3, 2), dtype=np.float64)
    for l in range(n_scen):
        f = 1.0 if l == 0 else light_factor ** l
        s_load[l, :, :, 0] = (s_heavy * f).real
        s_load[l, :, :, 1] = (s_heavy * f).imag

    ang = [0.0, -2.0 * math.pi / 3.0, 2.0 * math.pi / 3.0]
    v_slack = np.array([[math.cos(a), math.sin(a)] for a in ang], dtype=np.float64)

    counts = [0, 0, 0]
    for i in range(n_bus):
        counts[bin(int(phases[i])).count("1") - 1] += 1
    meta = dict(seed=seed, kv_ll=kv_ll, load_scale=lam, linear_drop_bound=worst * lam,
                phase_count_mix={"1": counts[0] / n_bus, "2": counts[1] / n_bus, "3": counts[2] / n_bus},
                mean_length_mi=float(lengths[1:].mean()))
    return Feeder(parent=parent, phases=phases, z_line=z_line, s_load=s_load,
                  v_slack=v_slack, meta=meta)


# Workload presets: sizes and distributions of the paper's feeders and
# sub-feeders (Section VI) as stand-ins for the proprietary feeders.
PRESETS = {
    # 40-bus sub-feeder, 4.16 kV, loads U(0,50) kW/phase; margin 0.005 p.u.,
    # run until no candidate is feasible.
    "feeder40": dict(n_bus=40, seed=1, kv_ll=4.16, phase_mode="keep", load=("uniform", 50.0),
                     pf_range=(0.9, 0.98), target=1.0, margin=0.005),
    # 1,000-bus feeder, 12.47 kV, loads U(0,100) kW/phase, 70/10/20 % phase mix,
    # 50 % target reduction.
    "feeder1000": dict(n_bus=1000, seed=1000, kv_ll=12.47, phase_mode=(0.7, 0.1, 0.2),
                       load=("uniform", 100.0), pf_range=(0.9, 0.98), target=0.5, margin=0.005),
    # stand-in for the 5,991-node feeder: 2,200 buses, 45/15/40 % mix, lognormal
    # loads (median 15 kW, sigma 1), 90 % target.
    "feeder2200": dict(n_bus=2200, seed=2200, kv_ll=12.47, phase_mode=(0.45, 0.15, 0.40),
                       load=("lognormal", 15.0, 1.0), pf_range=(0.85, 0.99), target=0.9, margin=0.005),
    # stand-in for the 8,381-node feeder: 3,100 buses, same distributions, 80 %.
    "feeder3100": dict(n_bus=3100, seed=3100, kv_ll=12.47, phase_mode=(0.45, 0.15, 0.40),
                       load=("lognormal", 15.0, 1.0), pf_range=(0.85, 0.99), target=0.8, margin=0.005),
}


def preset(name: str, **over) -> tuple[Feeder, dict]:
    """Return ``(feeder, run)`` where ``run`` holds the target reduction and margin."""
    cfg = dict(PRESETS[name])
    cfg.update(over)
    target = cfg.pop("target")
    margin = cfg.pop("margin")
    n_bus = cfg.pop("n_bus")
    seed = cfg.pop("seed")
    return make_feeder(n_bus, seed, **cfg), dict(target=target, margin=margin)


def batch_presets(count: int = 256, first_seed: int = 0, n_lo: int = 200, n_hi: int = 2000):
    """Uneven batch of feeders: n ~ U[n_lo, n_hi], target in {0.5, 0.7, 0.9}, margin 0.005."""
    out = []
    for k in range(count):
        seed = first_seed + k
        rng = np.random.default_rng(1_000_003 + seed)
        n = int(rng.integers(n_lo, n_hi + 1))
        target = [0.5, 0.7, 0.9][int(rng.integers(0, 3))]
        f = make_feeder(n, seed, kv_ll=12.47, phase_mode=(0.7, 0.1, 0.2), load=("uniform", 100.0),
                        pf_range=(0.9, 0.98))
        out.append((f, dict(target=target, margin=0.005)))
    return out


def daily_profiles(feeder: Feeder, hours: int = 24, seed: int = 0, noise: float = 0.15) -> np.ndarray:
    """Synthetic hourly loads for robustness studies: the feeder's heavy
    scenario scaled per hour by a daily shape (night trough, evening peak) and,
    per bus, by a random shift of that shape and a lognormal factor, so that
    buses do not move in lockstep.  Returns s_load [hours, n, 3, 2]."""
    rng = np.random.default_rng(seed)
    n = feeder.n_bus
    shift = rng.uniform(-2.0, 2.0, n)                     # hours
    h = np.arange(hours)[:, None] + shift[None, :]
    shape = 0.55 + 0.30 * np.sin(2 * math.pi * (h - 10.0) / 24.0) + 0.15 * np.exp(-((h % 24 - 19.0) ** 2) / 8.0)
    fac = shape * rng.lognormal(0.0, noise, (hours, n))
    return feeder.s_load[0][None, :, :, :] * fac[:, :, None, None]


def with_loads(feeder: Feeder, s_load: np.ndarray) -> Feeder:
    """The same network with other per-scenario loads ([L, n, 3, 2])."""
    return Feeder(parent=feeder.parent, phases=feeder.phases, z_line=feeder.z_line,
                  s_load=np.ascontiguousarray(s_load, dtype=np.float64), v_slack=feeder.v_slack, meta=dict(feeder.meta))


def fingerprint(feeder: Feeder) -> str:
    """SHA-256 of a feeder's arrays (their bytes, in a fixed order): two
    machines that draw the same feeder bit for bit give the same string, so a
    stored expected value can be checked against the inputs it was made from."""
    import hashlib
    h = hashlib.sha256()
    for a, dt in ((feeder.parent, np.int32), (feeder.phases, np.uint8), (feeder.z_line, np.float64),
                  (feeder.s_load, np.float64), (feeder.v_slack, np.float64)):
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    return h.hexdigest()

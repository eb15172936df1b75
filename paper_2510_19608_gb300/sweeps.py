"""Studies that reuse the reduction: the voltage-margin sweep (reduction level
against the largest voltage error, with and without radialization) and the
robustness of one reduction over many operating points.

Every reduction, radialization and evaluation runs in libokron.so; this module
only arranges the calls and collects the numbers.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import _binding as B


@dataclasses.dataclass
class _Loads:
    """A feeder's network with other per-scenario loads."""
    parent: np.ndarray
    phases: np.ndarray
    z_line: np.ndarray
    s_load: np.ndarray
    v_slack: np.ndarray

    @property
    def n_bus(self) -> int:
        return int(self.parent.shape[0])

    @property
    def n_scen(self) -> int:
        return int(self.s_load.shape[0])


def _with_loads(feeder, s_load) -> _Loads:
    return _Loads(np.asarray(feeder.parent), np.asarray(feeder.phases), np.asarray(feeder.z_line),
                  np.ascontiguousarray(s_load, dtype=np.float64), np.asarray(feeder.v_slack))


def margin_sweep(ctx: "B.Context", feeder, margins, *, target: float = 1.0, precision: int = 1,
                 radialize: bool = True):
    """Reduce `feeder` once per margin, all margins in one batched launch.
    Returns (rows, batch stats); each row has the margin, the reduction level
    (reduced buses / n), the largest voltage error, SMICE and, with
    `radialize`, the reduction level left after the critical buses of the
    radialization are kept again."""
    margins = [float(m) for m in margins]
    params = [B.default_params(margin=m, target_reduction=target, precision=precision) for m in margins]
    items, parts, stats = ctx.reduce_batch([feeder] * len(margins), params)
    n = int(np.asarray(feeder.parent).shape[0])
    if radialize:
        ctx.power_flow(feeder)                     # the context's network for okr_radialize
    rows = []
    for m, it, sup in zip(margins, items, parts):
        row = {"margin": m, "status": it["status"], "reduction": 1.0 - it["n_kept"] / n,
               "max_error": it["max_error"], "smice": it["smice"], "merges": it["n_iter"]}
        if radialize and it["status"] == 0:
            kept = (sup == np.arange(n)).astype(np.uint8)
            crit = ctx.radialize(kept)
            row["critical"] = int(crit.sum())
            row["radial_reduction"] = 1.0 - (int(kept.sum()) + int(crit.sum())) / n
        rows.append(row)
    return rows, stats


def profile_robustness(ctx: "B.Context", feeder, s_hours: np.ndarray, margin: float, *, target: float = 1.0,
                       precision: int = 1) -> dict:
    """Build the scenario library from the heaviest and the lightest hour of
    `s_hours` ([H, n, 3, 2]), reduce with it, then evaluate the reduced network
    on every hour.  Returns the library hours, the reduction level and the
    largest voltage error of each hour."""
    s_hours = np.asarray(s_hours, np.float64)
    tot = np.abs(s_hours).sum(axis=(1, 2, 3))
    heavy, light = int(np.argmax(tot)), int(np.argmin(tot))
    lib = _with_loads(feeder, s_hours[[heavy, light]])
    ctx.reduce(lib, B.default_params(margin=margin, target_reduction=target, precision=precision))
    summ = ctx.summary()
    sup = ctx.assignment()
    errs = []
    for h0 in range(0, s_hours.shape[0], 4):            # up to four scenarios per evaluation
        err, _ = ctx.evaluate(_with_loads(feeder, s_hours[h0:h0 + 4]), sup)
        errs.extend(float(e) for e in err)
    errs = np.array(errs)
    n = lib.n_bus
    return {"library_hours": [heavy, light], "reduction": 1.0 - summ["n_kept"] / n,
            "library_max_error": summ["max_error"], "max_error_by_hour": errs.tolist(),
            "hours_within_margin": float(np.mean(errs <= margin)), "worst_hour_error": float(errs.max())}

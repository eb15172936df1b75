"""Training data and evaluation for the learned candidate scorer.

The network, its training (forward, backward, Adam) and its inference run in
libokron.so (okr_scorer_*); this module only gathers data through the C ABI,
shapes the targets and counts how often the ranking misses the optimum.

Data: an exhaustive search with ``record_iters`` (precision 0) keeps, for its
first iterations, every candidate's exact score and features.  The target of a
candidate is its distance to that iteration's best score, in units of the
margin, on a log scale: ``log10(1e-6 + (score - best) / margin)``, clipped to
[-6, 2]; infeasible candidates get 2.  Ranking candidates by the prediction
then puts the likely optimum first.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import _binding as B

T_LO, T_HI = -6.0, 2.0


def targets(scores: np.ndarray, margin: float) -> np.ndarray:
    s = np.asarray(scores, np.float64)
    feas = np.isfinite(s)
    out = np.full(s.shape, T_HI, np.float64)
    if feas.any():
        best = s[feas].min()
        out[feas] = np.clip(np.log10(1e-6 + (s[feas] - best) / margin), T_LO, T_HI)
    return out.astype(np.float32)


def winner(s_ids: np.ndarray, r_ids: np.ndarray, scores: np.ndarray, tau: float = 1e-9) -> int:
    """Index of the candidate Algorithm 1 commits: the smallest (r, s) inside the
    tie band [m, m + tau] of the feasible scores (-1 if none is feasible)."""
    feas = np.isfinite(scores)
    if not feas.any():
        return -1
    m = scores[feas].min()
    band = np.nonzero(feas & (scores <= m + tau))[0]
    return int(min(band, key=lambda i: (int(r_ids[i]), int(s_ids[i]))))


def collect(ctx: "B.Context", runs, record_iters: int):
    """Run each (feeder, params) with recording and return (X, T, groups): the
    features, targets and, per recorded iteration, (start, stop, winner) rows."""
    xs, ts, groups = [], [], []
    o = 0
    for f, p in runs:
        q = B.default_params(margin=p.margin, target_reduction=p.target_reduction, max_merges=p.max_merges,
                             tie_tol=p.tie_tol, precision=0, record_iters=record_iters, engine=1)
        ctx.reduce(f, q)
        n_it = min(record_iters, ctx.summary()["n_iter"])
        for it in range(n_it):
            rec = ctx.recorded(it)
            feat = ctx.recorded_features(it)
            k = feat.shape[0]
            xs.append(feat)
            ts.append(targets(rec["score"], p.margin))
            groups.append((o, o + k, winner(rec["s"], rec["r"], rec["score"], p.tie_tol)))
            o += k
    X = np.concatenate(xs) if xs else np.zeros((0, 14), np.float32)
    T = np.concatenate(ts) if ts else np.zeros(0, np.float32)
    return X, T, groups


def init_params(n_features: int, seed: int) -> np.ndarray:
    """He-normal weights, zero biases, in the okr_scorer_params order."""
    rng = np.random.default_rng(seed)
    H = 128
    parts = [rng.normal(0.0, math.sqrt(2.0 / n_features), (n_features, H)), np.zeros(H),
             rng.normal(0.0, math.sqrt(2.0 / H), (H, H)), np.zeros(H),
             rng.normal(0.0, math.sqrt(2.0 / H), (H, H)), np.zeros(H),
             rng.normal(0.0, math.sqrt(1.0 / H), H), np.zeros(1)]
    return np.concatenate([a.ravel() for a in parts]).astype(np.float32)


def train(ctx: "B.Context", X: np.ndarray, T: np.ndarray, *, epochs: int = 20, batch: int = 4096, lr: float = 1e-3,
          seed: int = 0) -> np.ndarray:
    """Initialise and train the scorer on the GPU; returns the loss per epoch."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(X.shape[0])
    ctx.scorer_init(X.shape[1], init_params(X.shape[1], seed))
    return ctx.scorer_train(X[perm], T[perm], batch=batch, epochs=epochs, lr=lr)


def miss_rate(ctx: "B.Context", X: np.ndarray, groups, ks=(16, 64, 256), T=None, margin=0.005,
              tau=1e-9) -> dict:
    """For each recorded iteration with a feasible candidate and each k: whether
    the committed candidate is among the top-k predictions (miss_rate); with the
    targets T, also whether the top-k holds any candidate of optimal score
    (optimum_missed: none within the tie band) and the regret, the best exact
    score among the top-k above the optimum, in margins; the mean fraction
    of candidates a top-k evaluation would score; and how many candidates tie
    with the optimum per iteration (tie_band_median, tie_band_max)."""
    pred = ctx.scorer_predict(X) if X.shape[0] else np.zeros(0, np.float32)
    out = {}
    rows = [(a, b, w) for a, b, w in groups if w >= 0]
    band = math.log10(1e-6 + tau / margin)
    for k in ks:
        miss, opt_miss, frac, regrets = 0, 0, 0.0, []
        for a, b, w in rows:
            order = np.argsort(pred[a:b], kind="stable")
            top = order[:k]
            if w not in set(top.tolist()):
                miss += 1
            if T is not None:
                tbest = float(T[a:b][top].min())
                if tbest > band + 1e-6:
                    opt_miss += 1
                regrets.append(max(0.0, 10.0 ** tbest - 1e-6))
            frac += min(k, b - a) / (b - a)
        d = {"miss_rate": miss / max(1, len(rows)), "evaluated_fraction": frac / max(1, len(rows)),
             "iterations": len(rows)}
        if T is not None:
            d["optimum_missed"] = opt_miss / max(1, len(rows))
            d["regret_margins_median"] = float(np.median(regrets)) if regrets else 0.0
            d["regret_margins_max"] = float(np.max(regrets)) if regrets else 0.0
        out[k] = d
    pct = [float(np.searchsorted(np.sort(pred[a:b]), pred[a + w], side="left")) / (b - a) for a, b, w in rows]
    out["winner_rank_percentile"] = float(np.mean(pct)) if pct else float("nan")
    if T is not None and rows:
        # candidates tied with the iteration's optimum (inside the tie band):
        # the committed one is the smallest (r, s) among them, which no
        # ranking by predicted score can single out when many tie
        sizes = [int(np.count_nonzero(T[a:b] <= band + 1e-6)) for a, b, _ in rows]
        out["tie_band_median"] = float(np.median(sizes))
        out["tie_band_max"] = int(max(sizes))
    return out


def inference_timing(ctx: "B.Context", n: int, n_features: int = B.SCORER_FEATURES, reps: int = 5,
                     seed: int = 0) -> dict:
    """Wall time of okr_scorer_predict (CUDA cores, FP32 activations) and
    okr_scorer_predict_tc (tensor cores, bfloat16 layer inputs) on n seeded
    samples, host copies included, with a freshly initialised network (the
    context's scorer is replaced)."""
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.0, (n, n_features)).astype(np.float32)
    ctx.scorer_init(n_features, init_params(n_features, seed))
    out = {"samples": n, "features": n_features,
           "flops_per_sample": 2 * 128 * (n_features + 2 * 128 + 1)}
    ys = {}
    for name, fn in (("cuda_core", ctx.scorer_predict), ("tensor_core", ctx.scorer_predict_tc)):
        ys[name] = fn(x)                                  # warm-up
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn(x)
            times.append(time.perf_counter() - t0)
        out[name + "_ms"] = 1e3 * float(np.median(times))
    out["max_abs_difference"] = float(np.abs(ys["cuda_core"] - ys["tensor_core"]).max())
    return out


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="time the scorer's inference on seeded samples")
    ap.add_argument("--samples", type=int, default=1 << 20)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--features", type=int, default=B.SCORER_FEATURES,
                    help="inputs of the network (the search's scorer has OKR_SCORER_FEATURES)")
    a = ap.parse_args()
    with B.Context(a.device) as c:
        print(json.dumps(inference_timing(c, a.samples, n_features=a.features, reps=a.reps)))

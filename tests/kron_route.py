"""Independent numpy routes used to pin the CPU oracle (test helpers).

Nothing here is imported by the library or by the oracle.  Each helper follows a
different path to the same quantity than the oracle does:

* ``padded_y``      the 3n x 3n admittance with zero rows/columns for absent
                    phases (Sec. II-A), stamped line by line with numpy inverses
* ``z_closed_form`` Z_(i,p),(j,q) = sum of the line impedances on the common part
                    of the root paths of i and j (radial networks)
* ``kron_pinv``     eq. (Y_kron) with the Moore-Penrose pseudo-inverse on the
                    padded matrix (Sec. II-B)
* ``kron_route_score`` one candidate of Algorithm 1 evaluated by forming the
                    Kron-reduced network of its post-merge super-nodes and
                    solving it (Sec. II-C, eq. v_agg; Sec. IV)
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def zc(feeder) -> np.ndarray:
    z = feeder.z_line[..., 0] + 1j * feeder.z_line[..., 1]
    return z


def ancestors(parent, v):
    out = [v]
    while v > 0:
        v = int(parent[v])
        out.append(v)
    return out


def padded_y(feeder) -> np.ndarray:
    n = feeder.n_bus
    z = zc(feeder)
    Y = np.zeros((3 * n, 3 * n), dtype=np.complex128)
    for i in range(1, n):
        ps = [p for p in range(3) if feeder.phases[i] >> p & 1]
        y = np.linalg.inv(z[i][np.ix_(ps, ps)])
        p_ = int(feeder.parent[i])
        ii = [3 * i + p for p in ps]
        pp = [3 * p_ + p for p in ps]
        Y[np.ix_(ii, ii)] += y
        Y[np.ix_(pp, pp)] += y
        Y[np.ix_(ii, pp)] -= y
        Y[np.ix_(pp, ii)] -= y
    return Y


def present(feeder) -> np.ndarray:
    return np.array([(feeder.phases[i] >> p) & 1 for i in range(feeder.n_bus) for p in range(3)], bool)


def z_closed_form(feeder) -> np.ndarray:
    """Padded Z[(j,q),(i,p)] from path sums (root rows/columns zero)."""
    n = feeder.n_bus
    z = zc(feeder)
    path = [set(ancestors(feeder.parent, v)) - {0} for v in range(n)]
    Z = np.zeros((3 * n, 3 * n), dtype=np.complex128)
    for i in range(1, n):
        for j in range(1, n):
            common = path[i] & path[j]
            blk = np.zeros((3, 3), dtype=np.complex128)
            for e in common:
                blk += z[e]
            for p in range(3):
                for q in range(3):
                    if (feeder.phases[i] >> p & 1) and (feeder.phases[j] >> q & 1):
                        Z[3 * i + p, 3 * j + q] = blk[p, q]
    return Z


def kron_pinv(Y: np.ndarray, kept_rows: np.ndarray) -> np.ndarray:
    """Y_KK - Y_KR pinv(Y_RR) Y_RK on the padded matrix; kept_rows is a bool mask."""
    K = np.where(kept_rows)[0]
    R = np.where(~kept_rows)[0]
    if R.size == 0:
        return Y[np.ix_(K, K)].copy()
    return Y[np.ix_(K, K)] - Y[np.ix_(K, R)] @ np.linalg.pinv(Y[np.ix_(R, R)]) @ Y[np.ix_(R, K)]


def kron_route_voltages(feeder, Ypad, sup, ihat):
    """Voltages of every bus when each bus takes the voltage of its super-node,
    super-node voltages from the Kron-reduced network (slack fixed)."""
    n = feeder.n_bus
    L = ihat.shape[0]
    pres = present(feeder)
    supers = sorted(set(int(x) for x in sup))
    kept_bus = np.zeros(n, bool)
    kept_bus[supers] = True
    kept_rows = np.repeat(kept_bus, 3)
    Yk = kron_pinv(Ypad, kept_rows)
    K = np.where(kept_rows)[0]
    pos = {int(k): a for a, k in enumerate(K)}
    v0 = feeder.v_slack[:, 0] + 1j * feeder.v_slack[:, 1]
    out = np.zeros((L, n, 3), dtype=np.complex128)
    for l in range(L):
        # aggregated injections (eq. i_agg)
        Iagg = np.zeros(3 * n, dtype=np.complex128)
        for i in range(n):
            for p in range(3):
                Iagg[3 * sup[i] + p] += ihat[l, i, p]
        unk = [a for a, k in enumerate(K) if k >= 3 and pres[k]]
        fix = [a for a, k in enumerate(K) if k < 3]
        A = Yk[np.ix_(unk, unk)]
        b = Iagg[K[unk]] - Yk[np.ix_(unk, fix)] @ v0
        vk = np.linalg.solve(A, b)
        V = np.zeros(3 * n, dtype=np.complex128)
        V[0:3] = v0
        for a, x in zip(unk, vk):
            V[K[a]] = x
        for i in range(n):
            for p in range(3):
                if pres[3 * i + p]:
                    out[l, i, p] = V[3 * sup[i] + p]
    return out


def score_from_voltages(feeder, vhat, vred, sup, margin, objective=0):
    n = feeder.n_bus
    L = vhat.shape[0]
    pres = present(feeder).reshape(n, 3)
    e = np.abs(np.abs(vhat) - np.abs(vred))
    e = np.where(pres[None], e, 0.0)
    maxe = float(e.max())
    if not maxe <= margin:
        return math.inf, maxe
    if objective == 1:
        return maxe, maxe
    total = 0.0
    for l in range(L):
        for k in sorted(set(int(x) for x in sup)):
            members = [i for i in range(n) if sup[i] == k]
            total += float(e[l, members].max())
    return total, maxe


def kron_route_score(feeder, Ypad, vhat, ihat, sup, s, r, margin, objective=0):
    sup2 = np.array([s if x == r else x for x in sup])
    vred = kron_route_voltages(feeder, Ypad, sup2, ihat)
    return score_from_voltages(feeder, vhat, vred, sup2, margin, objective)


def connected_partitions(feeder):
    """All assignments (Sec. II-C rules): connected clusters, each with a super-node
    whose phases cover its members', slack kept as a super-node.  Yields super_of."""
    n = feeder.n_bus
    par = feeder.parent
    ph = feeder.phases
    # a partition of a tree into connected clusters = a choice of cut edges
    for cut in itertools.product([0, 1], repeat=n - 1):
        label = list(range(n))
        for i in range(1, n):
            if not cut[i - 1]:
                label[i] = label[int(par[i])]
        clusters = {}
        for i in range(n):
            clusters.setdefault(label[i], []).append(i)
        choices = []
        for root_bus, mem in clusters.items():
            need = 0
            for i in mem:
                need |= int(ph[i])
            if 0 in mem:
                cand = [0] if (int(ph[0]) & need) == need else []
            else:
                cand = [k for k in mem if (int(ph[k]) & need) == need]
            if not cand:
                choices = None
                break
            choices.append((mem, cand))
        if choices is None:
            continue
        for pick in itertools.product(*[c for _, c in choices]):
            sup = np.zeros(n, dtype=np.int64)
            for (mem, _), k in zip(choices, pick):
                for i in mem:
                    sup[i] = k
            yield sup


def kron_kept_voltages(feeder, Ypad, kept_bus, iagg):
    """Voltages of the kept buses of the Kron-reduced network on `kept_bus` for
    injections `iagg` ([L, 3n], zero on eliminated buses), slack fixed."""
    n = feeder.n_bus
    pres = present(feeder)
    kept_rows = np.repeat(np.asarray(kept_bus, bool), 3)
    Yk = kron_pinv(Ypad, kept_rows)
    K = np.where(kept_rows)[0]
    v0 = feeder.v_slack[:, 0] + 1j * feeder.v_slack[:, 1]
    unk = [a for a, k in enumerate(K) if k >= 3 and pres[k]]
    fix = [a for a, k in enumerate(K) if k < 3]
    out = np.zeros((iagg.shape[0], 3 * n), dtype=np.complex128)
    for l in range(iagg.shape[0]):
        A = Yk[np.ix_(unk, unk)]
        b = iagg[l, K[unk]] - Yk[np.ix_(unk, fix)] @ v0
        x = np.linalg.solve(A, b)
        out[l, 0:3] = v0
        for a, v in zip(unk, x):
            out[l, K[a]] = v
    return out

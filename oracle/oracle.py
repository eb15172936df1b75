"""CPU oracle for the exhaustive Kron-based reduction -- TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper around ``okr_oracle.c`` (plain FP64 C, OpenMP over
candidates).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares no code with the CUDA
library and never imports it.

Functions (each names the passage it follows):
  ybus            dense compact admittance (Sec. II-A, eq. KCL-3phase)
  injection       I = Y V (Sec. II-A)
  power_flow      operating points of the scenario library (Sec. III)
  tree_solve      Y_LL V_L = I_L - Y_L0 V_0 (the candidate solve of Algorithm 1)
  zbus            Z = Y_LL^{-1}
  kron            Y_Kron, the Schur complement onto the kept buses (Sec. II-B)
  reduce          Algorithm 1 (Sec. IV), literal or delta mode
  kron_graph      bus adjacency of Y_Kron: a 3x3 block with a nonzero entry (Sec. V)
  maximal_cliques maximal cliques of that graph (Bron-Kerbosch with pivoting)
  radialize       critical nodes of every maximal clique (Sec. V)
  evaluate        the reduced network of a given assignment on a feeder's own
                  scenarios (Algorithm 1's voltage model, eq. i_agg)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "okr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no FMA contraction, no -march)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Summary(C.Structure):
    _fields_ = [("n_iter", C.c_int32), ("stop_reason", C.c_int32), ("candidates", C.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i32, f64 = C.c_int, C.c_double
            lib.orc_phase_index.argtypes = [i32, P, P]
            lib.orc_ybus.argtypes = [i32, P, P, P, P]
            lib.orc_injection.argtypes = [i32, P, P, P, i32, P, P]
            lib.orc_pf.argtypes = [i32, P, P, P, i32, P, P, f64, i32, P]
            lib.orc_tree_solve.argtypes = [i32, P, P, P, i32, P, P, P]
            lib.orc_zbus.argtypes = [i32, P, P, P, P]
            lib.orc_kron.argtypes = [i32, P, P, P, P, P, P]
            lib.orc_reduce.argtypes = [i32, P, P, P, i32, P, P, P, f64, i32, i32, f64, i32, i32,
                                       P, P, P, P, P, P, P, P, P, P, P, P, C.POINTER(_Summary)]
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_set_threads.restype = None
            for fn in ("orc_phase_index", "orc_ybus", "orc_injection", "orc_pf", "orc_tree_solve",
                       "orc_zbus", "orc_kron", "orc_reduce", "orc_num_threads"):
                getattr(lib, fn).restype = C.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _tree(feeder):
    parent = np.ascontiguousarray(feeder.parent, dtype=np.int32)
    phases = np.ascontiguousarray(feeder.phases, dtype=np.uint8)
    z = np.ascontiguousarray(feeder.z_line, dtype=np.float64)
    return parent, phases, z


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(t: int) -> None:
    """OpenMP thread count for later calls (candidates are evaluated in parallel)."""
    _load().orc_set_threads(int(t))


def phase_index(phases: np.ndarray) -> tuple[np.ndarray, int]:
    ph = np.ascontiguousarray(phases, dtype=np.uint8)
    idx = np.zeros(3 * ph.shape[0], dtype=np.int32)
    nphi = _load().orc_phase_index(ph.shape[0], _p(ph), _p(idx))
    return idx.reshape(-1, 3), int(nphi)


def ybus(feeder) -> np.ndarray:
    """Dense compact admittance matrix (complex128, n_phi x n_phi, root included)."""
    parent, phases, z = _tree(feeder)
    _, nphi = phase_index(phases)
    Y = np.zeros((nphi, nphi), dtype=np.complex128)
    rc = _load().orc_ybus(parent.shape[0], _p(parent), _p(phases), _p(z), _p(Y))
    if rc:
        raise ValueError("singular line impedance")
    return Y


def injection(feeder, v: np.ndarray) -> np.ndarray:
    """I = Y V for padded voltages v[L,n,3] (complex128)."""
    parent, phases, z = _tree(feeder)
    v = np.ascontiguousarray(v, dtype=np.complex128)
    out = np.zeros_like(v)
    rc = _load().orc_injection(parent.shape[0], _p(parent), _p(phases), _p(z), v.shape[0], _p(v), _p(out))
    if rc:
        raise ValueError("singular line impedance")
    return out


def power_flow(feeder, tol: float = 1e-13, max_iter: int = 200) -> tuple[np.ndarray, int]:
    """Backward/forward sweep; returns (V[L,n,3] complex128, sweeps)."""
    parent, phases, z = _tree(feeder)
    s = np.ascontiguousarray(feeder.s_load, dtype=np.float64)
    vs = np.ascontiguousarray(feeder.v_slack, dtype=np.float64)
    L, n = s.shape[0], parent.shape[0]
    v = np.zeros((L, n, 3), dtype=np.complex128)
    it = _load().orc_pf(n, _p(parent), _p(phases), _p(z), L, _p(s), _p(vs), tol, max_iter, _p(v))
    if it < 0:
        raise RuntimeError("power flow did not converge")
    return v, int(it)


def operating_points(feeder) -> tuple[np.ndarray, np.ndarray]:
    """Scenario library: Vhat from the load flow, Ihat := Y Vhat."""
    vhat, _ = power_flow(feeder)
    return vhat, injection(feeder, vhat)


def tree_solve(feeder, b: np.ndarray, v0=None) -> np.ndarray:
    parent, phases, z = _tree(feeder)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    if v0 is None:
        v0 = feeder.v_slack[:, 0] + 1j * feeder.v_slack[:, 1]
    v0 = np.ascontiguousarray(v0, dtype=np.complex128)
    out = np.zeros_like(b)
    rc = _load().orc_tree_solve(parent.shape[0], _p(parent), _p(phases), _p(z), b.shape[0], _p(b), _p(v0), _p(out))
    if rc:
        raise ValueError("singular block")
    return out


def zbus(feeder) -> np.ndarray:
    """Padded Z: Z[j,q,i,p] = dV(i,p)/dI(j,q) (zero for root and absent phases)."""
    parent, phases, z = _tree(feeder)
    n = parent.shape[0]
    Z = np.zeros((n, 3, n, 3), dtype=np.complex128)
    rc = _load().orc_zbus(n, _p(parent), _p(phases), _p(z), _p(Z))
    if rc:
        raise ValueError("singular block")
    return Z


def kron(feeder, kept: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Y_Kron over the kept phase nodes and their ids (bus*3+phase)."""
    parent, phases, z = _tree(feeder)
    kept = np.ascontiguousarray(kept, dtype=np.uint8)
    if not kept[0]:
        raise ValueError("the slack bus must be kept")
    kphi_max = int(sum(bin(int(phases[i])).count("1") for i in range(len(kept)) if kept[i]))
    Yk = np.zeros((kphi_max, kphi_max), dtype=np.complex128)
    kidx = np.zeros(kphi_max, dtype=np.int32)
    kphi = _load().orc_kron(parent.shape[0], _p(parent), _p(phases), _p(z), _p(kept), _p(Yk), _p(kidx))
    if kphi < 0:
        raise ValueError("singular block")
    return Yk[:kphi, :kphi], kidx[:kphi]


def reduce(feeder, vhat: np.ndarray, ihat: np.ndarray, *, margin: float, max_merges: int,
           objective: int = 0, tau: float = 1e-9, mode: str = "delta", record_iters: int = 0) -> dict:
    """Algorithm 1.  Returns a dict with the decision sequence and the final state."""
    parent, phases, z = _tree(feeder)
    n = parent.shape[0]
    vhat = np.ascontiguousarray(vhat, dtype=np.complex128)
    ihat = np.ascontiguousarray(ihat, dtype=np.complex128)
    L = vhat.shape[0]
    vs = np.ascontiguousarray(feeder.v_slack, dtype=np.float64)
    cap = max(1, min(max_merges, n))
    dec_s = np.full(cap, -1, np.int32)
    dec_r = np.full(cap, -1, np.int32)
    dec_score = np.zeros(cap)
    dec_maxerr = np.zeros(cap)
    dec_gap = np.zeros(cap)
    dec_ncand = np.zeros(cap, np.int32)
    sup = np.zeros(n, np.int32)
    vred = np.zeros((L, n, 3), np.complex128)
    K = max(0, record_iters)
    rec_s = np.zeros((max(K, 1), 2 * n), np.int32)
    rec_r = np.zeros((max(K, 1), 2 * n), np.int32)
    rec_score = np.zeros((max(K, 1), 2 * n))
    rec_count = np.zeros(max(K, 1), np.int32)
    summ = _Summary()
    rc = _load().orc_reduce(n, _p(parent), _p(phases), _p(z), L, _p(vhat), _p(ihat), _p(vs),
                            float(margin), int(max_merges), int(objective), float(tau),
                            0 if mode == "literal" else 1, K,
                            _p(dec_s), _p(dec_r), _p(dec_score), _p(dec_maxerr), _p(dec_gap), _p(dec_ncand),
                            _p(sup), _p(vred), _p(rec_s), _p(rec_r), _p(rec_score), _p(rec_count),
                            C.byref(summ))
    if rc:
        raise RuntimeError(f"oracle reduce failed ({rc})")
    t = summ.n_iter
    rec = []
    for k in range(min(K, t + 1)):
        c = rec_count[k]
        rec.append(dict(s=rec_s[k, :c].copy(), r=rec_r[k, :c].copy(), score=rec_score[k, :c].copy()))
    return dict(n_iter=t, stop_reason=summ.stop_reason, candidates=summ.candidates,
                s=dec_s[:t].copy(), r=dec_r[:t].copy(), score=dec_score[:t].copy(),
                maxerr=dec_maxerr[:t].copy(), gap=dec_gap[:t].copy(), ncand=dec_ncand[:t].copy(),
                super_of=sup, v_red=vred, recorded=rec)


def max_merges_for(n_bus: int, target: float) -> int:
    """Target reduction -> number of merges: ceil(target * n), at most n - 1."""
    import math
    return min(n_bus - 1, int(math.ceil(target * n_bus - 1e-12)))


# ----------------------------------------------------------------------------- Sec. V
def kron_graph(feeder, kept: np.ndarray, tol: float = 0.0) -> tuple[np.ndarray, dict]:
    """Kept buses and their adjacency in the Kron-reduced network: buses i != j are
    connected when the 3x3 block of Y_Kron between them has an entry with
    |y| > tol (Sec. V extends the single-phase nonzero test to blocks)."""
    Yk, kidx = kron(feeder, kept)
    bus = kidx // 3
    buses = np.unique(bus)
    adj = {int(b): set() for b in buses}
    for a in range(len(kidx)):
        for c in range(len(kidx)):
            if bus[a] != bus[c] and abs(Yk[a, c]) > tol:
                adj[int(bus[a])].add(int(bus[c]))
    return buses, adj


def maximal_cliques(adj: dict) -> list[set]:
    """Every maximal clique of an undirected graph (Bron-Kerbosch with pivoting)."""
    out = []

    def bk(r, p, x):
        if not p and not x:
            out.append(set(r))
            return
        u = max(p | x, key=lambda v: len(adj[v] & p))
        for v in list(p - adj[u]):
            bk(r | {v}, p & adj[v], x & adj[v])
            p = p - {v}
            x = x | {v}

    bk(set(), set(adj), set())
    return out


def radialize(feeder, kept: np.ndarray) -> np.ndarray:
    """Critical nodes (Sec. V): for every maximal clique of the Kron-reduced graph,
    take the sub-tree of the original feeder that spans the clique's buses and
    mark its buses of degree >= 3 (within that sub-tree) that are not kept.
    Returns a flag per bus; kept + critical buses make the reduced network radial."""
    parent = np.asarray(feeder.parent)
    n = parent.shape[0]
    _, adj = kron_graph(feeder, kept)
    crit = np.zeros(n, dtype=np.uint8)
    for clique in maximal_cliques(adj):
        if len(clique) < 3:
            continue
        # spanning sub-tree: the union of the tree paths between the clique's buses
        nodes, edges = set(), set()
        cl = sorted(clique)
        for a in cl:
            for b in cl:
                if a >= b:
                    continue
                pa, pb = [a], [b]
                while pa[-1] != 0:
                    pa.append(int(parent[pa[-1]]))
                while pb[-1] != 0:
                    pb.append(int(parent[pb[-1]]))
                common = set(pa) & set(pb)
                path = [v for v in pa if v not in common] + [v for v in pb if v not in common]
                # lowest common ancestor: the deepest common bus
                depth = {}
                for v in common:
                    d, w = 0, v
                    while w != 0:
                        w = int(parent[w])
                        d += 1
                    depth[v] = d
                lca = max(common, key=lambda v: depth[v])
                for v in path:
                    nodes.add(v)
                    edges.add((v, int(parent[v])))
                nodes.add(lca)
        deg = {v: 0 for v in nodes}
        for (c, p_) in edges:
            deg[c] += 1
            deg[p_] += 1
        for v, d in deg.items():
            if d >= 3 and not kept[v]:
                crit[v] = 1
    return crit


def evaluate(feeder, super_of: np.ndarray):
    """Largest per-phase magnitude error per scenario, and the reduced voltages,
    of assignment super_of on the feeder's scenarios: aggregated injections at
    the super-nodes, the tree solved with the slack fixed, every bus at its
    super-node's voltage."""
    vhat, ihat = operating_points(feeder)
    n = feeder.n_bus
    sup = np.asarray(super_of)
    iagg = np.zeros_like(ihat)
    for i in range(n):
        iagg[:, sup[i], :] += ihat[:, i, :]
    V = tree_solve(feeder, iagg)
    pres = np.array([[(int(feeder.phases[i]) >> p) & 1 for p in range(3)] for i in range(n)], bool)
    vred = np.where(pres[None], V[:, sup, :], 0.0)
    err = np.array([np.abs(np.abs(vhat[l][pres]) - np.abs(vred[l][pres])).max() for l in range(vhat.shape[0])])
    return err, vred

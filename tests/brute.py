"""Definitional brute force on tiny graphs, independent of the C oracle.

Everything here follows the paper's definitions directly, on top of a
library all-pairs BFS (scipy.sparse.csgraph), so it can pin the oracle:

* ``apsp``            -- d_G(u, v) for all pairs (Sec. 3.1), 255 = unreachable.
* ``canonical``       -- the label set the method must produce for a fixed
                         order and bit-parallel vertex set X: (v_j, d(v_j,u)) is
                         in L(u) iff v_j is not in X, u is reachable from v_j,
                         and no vertex of X or of {v_i : i < j} lies in
                         P_G(v_j, u) (Sec. 3.1 defines P_G). This is what the
                         correctness proof of Thm 4.1 shows is always labelled,
                         and the minimality proof of Thm 4.2 shows is all that is
                         labelled; X enters through Sec. 5.4.
* ``bp_pointwise``    -- S^{-1}_r(v), S^0_r(v) from their definition in Sec.
                         5.1: the members s of S_r with d(s, v) - d(r, v) equal
                         to -1 and 0.
* ``label_query``     -- Query(s, t, L) of Sec. 3.3 written as a set
                         intersection (no merge).
* ``apsp_directed``, ``canonical_directed`` -- the same for the directed
                         labels of Sec. 6: (v_j, d(v_j, u)) is in L_IN(u)
                         iff no v_i with i < j lies on a shortest v_j -> u
                         path, and (v_j, d(u, v_j)) is in L_OUT(u) iff none
                         lies on a shortest u -> v_j path (the arguments of
                         Thm 4.1 and Thm 4.2 run unchanged along arcs).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

INF = 255


def apsp(offsets, cols) -> np.ndarray:
    n = len(offsets) - 1
    if n == 0:
        return np.zeros((0, 0), dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(offsets, dtype=np.int64)))
    A = sp.csr_matrix((np.ones(len(cols)), (rows, np.asarray(cols, dtype=np.int64))), shape=(n, n))
    D = shortest_path(A, method="D", unweighted=True, directed=False)
    out = np.full((n, n), INF, dtype=np.int64)
    fin = np.isfinite(D)
    out[fin] = D[fin].astype(np.int64)
    return out


def canonical(D: np.ndarray, order, inX) -> dict:
    """{u: [(rank j, d)] ascending} for every vertex u."""
    n = D.shape[0]
    order = np.asarray(order, dtype=np.int64)
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    inX = np.asarray(inX, dtype=bool)
    Dw = np.where(D >= INF, 10**6, D)  # large finite stand-in so sums stay comparable
    L = {u: [] for u in range(n)}
    for j in range(n):
        v = order[j]
        if inX[v]:
            continue
        bad = inX | (rank < j)  # vertices that must not lie on a shortest v-u path
        # on_path[w, u] = w lies in P_G(v, u)
        on_path = (Dw[v][:, None] + Dw) == Dw[v][None, :]
        blocked = (on_path & bad[:, None]).any(axis=0)
        for u in range(n):
            if D[v, u] < INF and not blocked[u]:
                L[u].append((j, int(D[v, u])))
    return L


def bp_pointwise(D: np.ndarray, roots, cnt, S):
    """d, m1, m0 as [n][t] arrays from the definitions (Sec. 5.1)."""
    n = D.shape[0]
    t = len(roots)
    d = np.full((n, t), INF, dtype=np.uint8)
    m1 = np.zeros((n, t), dtype=np.uint64)
    m0 = np.zeros((n, t), dtype=np.uint64)
    for i in range(t):
        r = int(roots[i])
        if r == 0xFFFFFFFF:
            continue
        for v in range(n):
            if D[r, v] >= INF:
                continue
            d[v, i] = D[r, v]
            a = b = 0
            for j in range(int(cnt[i])):
                s = int(S[i][j])
                if D[s, v] == D[r, v] - 1:
                    a |= 1 << j
                elif D[s, v] == D[r, v]:
                    b |= 1 << j
            m1[v, i] = a
            m0[v, i] = b
    return d, m1, m0


def label_query(La, Lb) -> int:
    da = dict(La)
    best = INF
    for h, x in Lb:
        if h in da:
            best = min(best, da[h] + x)
    return best


def apsp_directed(offsets, cols) -> np.ndarray:
    """d(u, v) along arcs (out-neighbour CSR), 255 = unreachable."""
    n = len(offsets) - 1
    if n == 0:
        return np.zeros((0, 0), dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(offsets, dtype=np.int64)))
    A = sp.csr_matrix((np.ones(len(cols)), (rows, np.asarray(cols, dtype=np.int64))), shape=(n, n))
    D = shortest_path(A, method="D", unweighted=True, directed=True)
    out = np.full((n, n), INF, dtype=np.int64)
    fin = np.isfinite(D)
    out[fin] = D[fin].astype(np.int64)
    return out


def canonical_directed(D: np.ndarray, order):
    """({u: [(rank j, d)]} for L_IN, the same for L_OUT), hubs ascending."""
    n = D.shape[0]
    order = np.asarray(order, dtype=np.int64)
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    Dw = np.where(D >= INF, 10**6, D)
    Lin = {u: [] for u in range(n)}
    Lout = {u: [] for u in range(n)}
    for j in range(n):
        v = order[j]
        early = rank < j
        # forward: w on a shortest v -> u path iff d(v, w) + d(w, u) = d(v, u)
        on_fwd = (Dw[v][:, None] + Dw) == Dw[v][None, :]
        blocked_in = (on_fwd & early[:, None]).any(axis=0)
        # reverse: w on a shortest u -> v path iff d(u, w) + d(w, v) = d(u, v)
        on_rev = (Dw + Dw[:, v][None, :]) == Dw[:, v][:, None]
        blocked_out = (on_rev & early[None, :]).any(axis=1)
        for u in range(n):
            if D[v, u] < INF and not blocked_in[u]:
                Lin[u].append((j, int(D[v, u])))
            if D[u, v] < INF and not blocked_out[u]:
                Lout[u].append((j, int(D[u, v])))
    return Lin, Lout


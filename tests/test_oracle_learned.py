"""Pins of the learned-order oracle (oracle/learned.py, core numbers in
oracle.c) against definitions, closed forms and brute force -- no GPU."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import learned as OL
from paper_1304_4661_gb300 import graphgen as gg

from . import graphs


# ------------------------------------------------------------ core numbers
def core_by_definition(g):
    """core(v) = max over vertex subsets S containing v of the minimum degree
    of the subgraph induced by S (exhaustive, tiny graphs only)."""
    n = g.n
    adj = [set(g.cols[g.offsets[v]:g.offsets[v + 1]].tolist()) for v in range(n)]
    best = [0] * n
    for r in range(1, n + 1):
        for S in itertools.combinations(range(n), r):
            Ss = set(S)
            k = min(len(adj[v] & Ss) for v in S)
            for v in S:
                best[v] = max(best[v], k)
    return np.array(best)


@pytest.mark.parametrize("g,expect", [
    (graphs.complete(5), [4] * 5),
    (graphs.star(6), [1] * 6),
    (graphs.cycle(7), [2] * 7),
    (graphs.path(5), [1] * 5),
    (gg.from_edges(3, [], []), [0] * 3),
    # K4 with a pendant vertex 4 on vertex 0
    (gg.from_edges(5, [0, 0, 0, 1, 1, 2, 0], [1, 2, 3, 2, 3, 3, 4]), [3, 3, 3, 3, 1]),
])
def test_core_numbers_textbook(g, expect):
    assert oracle.core_numbers(g.offsets, g.cols).tolist() == expect


def test_core_numbers_petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    u, v = zip(*(outer + inner + spokes))
    g = gg.from_edges(10, u, v)
    assert (oracle.core_numbers(g.offsets, g.cols) == 3).all()


@pytest.mark.parametrize("seed", range(12))
def test_core_numbers_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 10))
    m = int(rng.integers(0, n * (n - 1) // 2 + 1))
    pairs = list(itertools.combinations(range(n), 2))
    pick = rng.choice(len(pairs), size=m, replace=False) if m else []
    u = [pairs[i][0] for i in pick]
    v = [pairs[i][1] for i in pick]
    g = gg.from_edges(n, u, v)
    assert np.array_equal(oracle.core_numbers(g.offsets, g.cols), core_by_definition(g))


def test_core_numbers_are_degeneracy_ordering():
    """On a larger graph: every vertex with core k has >= k neighbours of core
    >= k, and the k-core (vertices of core >= k) has minimum degree >= k."""
    g = gg.rmat(12, 8, seed=2)
    c = oracle.core_numbers(g.offsets, g.cols)
    for v in range(g.n):
        nb = g.cols[g.offsets[v]:g.offsets[v + 1]]
        assert (c[nb] >= c[v]).sum() >= c[v]
    # no vertex could sit in a denser core: peeling the (k+1)-core removes it
    for k in range(1, int(c.max()) + 1):
        inside = c >= k
        for v in np.flatnonzero(inside)[:200]:
            nb = g.cols[g.offsets[v]:g.offsets[v + 1]]
            assert inside[nb].sum() >= k


# ------------------------------------------------------------ features
def test_two_hop_identities():
    g = gg.ba(500, 3, 4)
    deg, two_hop, _, _ = OL.raw_features(g.offsets, g.cols, 0)
    # each vertex u adds deg(u) to each of its deg(u) neighbours
    assert two_hop.sum() == (deg ** 2).sum()
    s = graphs.star(9)
    _, th, _, _ = OL.raw_features(s.offsets, s.cols, 0)
    assert th.tolist() == [8] + [8] * 8  # centre: 8 leaves of degree 1; leaf: the centre


def test_bit_parallel_statistics_on_a_star_and_isolated_vertex():
    # star on 0..5 plus an isolated vertex 6; t = 1: root = centre, S = leaves
    g = gg.from_edges(7, [0] * 5, [1, 2, 3, 4, 5])
    _, _, _, bp = OL.raw_features(g.offsets, g.cols, 1)
    # centre: d = 0, no mask members; leaf: d = 1, S^-1 = {itself}, S^0 empty
    assert bp[0].tolist() == [0, 0, 1, 0, 0]
    for leaf in range(1, 6):
        assert bp[leaf].tolist() == [1, 1, 1, 1 / 64, 0]
    # unreachable: distance capped, nothing within 2
    assert bp[6].tolist() == [OL.D_CAP, OL.D_CAP, 0, 0, 0]


def test_bit_parallel_s0_counts_equal_distance_members():
    """A 4-cycle 0-1-2-3 with t = 1: root 0 (all degrees 2, lowest id), S =
    {1, 3}. Vertex 2 is at distance 2 from the root and 1 from both members,
    so S^-1(2) = {1, 3}; vertex 1 has S^-1 = {1} and S^0 = {} (d(3,1) = 2)."""
    g = graphs.cycle(4)
    _, _, _, bp = OL.raw_features(g.offsets, g.cols, 1)
    assert bp[2].tolist() == [2, 2, 1, 2 / 64, 0]
    assert bp[1].tolist() == [1, 1, 1, 1 / 64, 0]
    assert bp[0].tolist() == [0, 0, 1, 0, 0]


@pytest.mark.parametrize("g", [graphs.complete(6), graphs.cycle(9), gg.from_edges(4, [], [])],
                         ids=lambda g: g.name)
def test_features_of_vertex_transitive_graphs_are_zero(g):
    """Every vertex looks the same, so every column without bit-parallel
    roots is constant and standardises to 0 exactly; with roots, only the
    roots break the symmetry, so the first three columns stay 0."""
    assert not OL.features(g.offsets, g.cols, 0).any()
    assert not OL.features(g.offsets, g.cols, 4)[:, :3].any()


def test_features_standardised():
    g = gg.rmat(11, 8, seed=5)
    Z = OL.features(g.offsets, g.cols, 16)
    assert Z.shape == (g.n, 8)
    for j in range(8):
        col = Z[:, j]
        if np.allclose(col, 0):
            continue
        assert abs(col.mean()) < 1e-9 and abs(col.std() - 1) < 1e-9
    # the log-degree column is an increasing function of degree
    d = g.degrees
    order = np.argsort(d, kind="stable")
    assert (np.diff(Z[order, 0]) >= -1e-12).all()


# ------------------------------------------------------------ bf16
def bf16_nearest_brute(x):
    """Nearest bfloat16 by search: candidates are the two bf16 values around x
    (truncation and truncation + 1 ulp); ties go to the even mantissa."""
    out = []
    for v in np.asarray(x, dtype=np.float32):
        b = int(np.float32(v).view(np.uint32))
        lo = b & 0xFFFF0000
        hi = lo + 0x10000
        flo = float(np.uint32(lo).view(np.float32))
        fhi = float(np.uint32(hi).view(np.float32))
        dl, dh = abs(float(v) - flo), abs(fhi - float(v))
        if dl < dh or (dl == dh and ((lo >> 16) & 1) == 0):
            out.append(flo)
        else:
            out.append(fhi)
    return np.array(out)


def test_bf16_round_known_values():
    ulp = 2.0 ** -7
    x = np.array([1.0, 1 + ulp / 2, 1 + 3 * ulp / 2, 1 + ulp / 2 + 2 ** -20, -(1 + ulp / 2),
                  0.0, 3.0, -2.5], dtype=np.float32)
    assert OL.bf16_round(x).tolist() == [1.0, 1.0, 1 + 2 * ulp, 1 + ulp, -1.0, 0.0, 3.0, -2.5]


def test_bf16_round_brute_force():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(5000) * np.exp(rng.uniform(-20, 20, 5000))).astype(np.float32)
    assert np.array_equal(OL.bf16_round(x), bf16_nearest_brute(x))


# ------------------------------------------------------------ network
def small_problem(seed, B=37):
    p = gg.mlp_init(seed)
    rng = np.random.default_rng(seed)
    p[512:576] = rng.uniform(-0.5, 0.5, 64)     # b1
    p[4672:4736] = rng.uniform(-0.5, 0.5, 64)   # b2
    p[4800] = 0.3
    X = rng.standard_normal((B, 8))
    y = rng.standard_normal(B)
    return p, X, y


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed):
    p, X, y = small_problem(seed)
    q = OL.bf16_round(p)
    loss, g = OL.net_loss_grad(q, X, y)
    rng = np.random.default_rng(seed + 10)
    idx = np.concatenate([rng.choice(OL.NPARAM, 120, replace=False), [4800, 4799, 0, 575]])
    h = 1e-6
    for i in idx:
        e = np.zeros(OL.NPARAM)
        e[i] = h
        lp, _ = OL.net_loss_grad(q + e, X, y)
        lm, _ = OL.net_loss_grad(q - e, X, y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_constant_network_closed_form():
    """All weights and hidden biases zero: y = b3 for every row, the loss is
    mean((b3 - t)^2), only b3 has a gradient, 2 mean(b3 - t)."""
    p = np.zeros(OL.NPARAM, dtype=np.float32)
    p[4800] = 0.75
    X = np.random.default_rng(1).standard_normal((9, 8))
    t = np.arange(9, dtype=np.float64)
    y, _ = OL.forward(p, X)
    assert np.allclose(y, 0.75)
    loss, g = OL.loss_grad(p, X, t)
    assert loss == pytest.approx(((0.75 - t) ** 2).mean())
    assert g[4800] == pytest.approx(2 * (0.75 - t).mean())
    assert np.count_nonzero(g[:4800]) == 0


def test_linear_regime_is_a_matrix_product():
    """Positive inputs, weights and biases keep every ReLU open, so the
    network is the affine map w3 (W2 (W1 x + b1) + b2) + b3."""
    rng = np.random.default_rng(2)
    p = rng.uniform(0.01, 0.1, OL.NPARAM).astype(np.float32)
    X = rng.uniform(0, 1, (11, 8))
    q = OL.unpack(OL.bf16_round(p))
    expect = ((X @ q["W1"].T + q["b1"]) @ q["W2"].T + q["b2"]) @ q["w3"] + q["b3"][0]
    y, _ = OL.forward(p, X)
    assert np.allclose(y, expect, rtol=1e-12)


def test_adam_first_step_closed_form():
    """From m = v = 0 the bias-corrected first step is lr g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, eps = 1e-3, 1e-8
    p1, m, v = OL.adam_step(p, np.zeros(50), np.zeros(50), g, lr, 1, eps=eps)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_mlp_init_layout():
    p = gg.mlp_init(7)
    assert p.dtype == np.float32 and p.shape == (OL.NPARAM,)
    P = OL.unpack(p.astype(np.float64))
    for name, fan in (("W1", 8), ("W2", 64), ("w3", 64)):
        a = np.sqrt(6 / fan)
        assert np.abs(P[name]).max() <= a and np.abs(P[name]).max() > 0.8 * a
    for name in ("b1", "b2", "b3"):
        assert not P[name].any()
    assert np.array_equal(p, gg.mlp_init(7)) and not np.array_equal(p, gg.mlp_init(8))


# ------------------------------------------------------------ order, targets
def test_order_from_scores_ties_by_id():
    s = np.array([0.5, 2.0, 0.5, -1.0, 2.0, 0.5], dtype=np.float32)
    expect = sorted(range(6), key=lambda v: (-float(s[v]), v))
    assert OL.order_from_scores(s).tolist() == expect == [1, 4, 0, 2, 5, 3]


def test_hub_counts_star():
    """Star, t = 0: the centre comes first and is a hub of every label; each
    leaf is a hub of its own label only (the centre prunes the rest)."""
    g = graphs.star(8)
    ix = oracle.Index(g.offsets, g.cols, 0)
    c = OL.hub_counts(ix.labels(), ix.order())
    assert c.tolist() == [8] + [1] * 7
    assert c.sum() == len(ix.labels().hubs)


def test_hub_counts_total_and_order_invariance_of_distances():
    g = gg.ba(300, 2, 9)
    ix = oracle.Index(g.offsets, g.cols, 4)
    c = OL.hub_counts(ix.labels(), ix.order())
    assert c.sum() == len(ix.labels().hubs)
    # bit-parallel vertices get no normal-label entries (Sec. 5.4)
    rank, inX = ix.rank_inX()
    assert (c[inX == 1] == 0).all()
    # any order gives the same distances (Thm 4.1); a score order is one
    scores = gg.uniform(3, g.n).astype(np.float32)
    ix2 = oracle.Index(g.offsets, g.cols, 4, order=OL.order_from_scores(scores))
    s, u = gg.pairs(g.n, 2000, 1)
    assert np.array_equal(ix.query_batch(s, u), ix2.query_batch(s, u))

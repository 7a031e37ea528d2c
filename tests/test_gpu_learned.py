"""The learned order on the GPU against the oracle (oracle/learned.py).

Integer results (core numbers, neighbour-degree sums, hub counts, orders,
bf16 bit patterns, labels) must match exactly. Floating point:
  * features: float32 storage of float64 values and float64 moments, so
    |gpu - oracle| <= 2e-5 + 1e-5 |oracle| per standardised value;
  * network: float32 arithmetic over 8 + 64 + 64 terms per output with the
    same bf16 parameters, so scores within 1e-5 relative to the score scale;
  * gradient: float32 sums over at most a few thousand rows, checked within
    1e-4 of the largest gradient entry plus 1e-4 relative;
  * Adam: float32 update, within 1e-6 relative plus 2e-9 absolute (a few
    ulps of a step of size lr = 1e-3).
"""
import numpy as np
import pytest

import oracle
from oracle import learned as OL
from paper_1304_4661_gb300 import graphgen as gg
from paper_1304_4661_gb300 import learned as L
from paper_1304_4661_gb300 import pll

from . import graphs
from .gpu_util import dev_u32, gpu_build

pytestmark = pytest.mark.gpu


def fgraphs():
    return [
        gg.from_edges(7, [0] * 5, [1, 2, 3, 4, 5]),   # star + isolated vertex
        graphs.cycle(4), graphs.complete(6), graphs.path(9),
        graphs.disjoint(graphs.star(40), graphs.cycle(25)),
        gg.ba(2000, 3, 1), gg.ws(1500, 6, 0.1, 2), gg.rmat(11, 8, seed=4), gg.rmat(13, 16, seed=5),
    ]


@pytest.mark.parametrize("t", [0, 1, 4, 16, 64])
@pytest.mark.parametrize("g", fgraphs(), ids=lambda g: g.name)
def test_features_match_oracle(g, t):
    X, core, two = pll.features(dev_u32(g.offsets), dev_u32(g.cols), t, raw=True)
    _, two_ref, core_ref, _ = OL.raw_features(g.offsets, g.cols, t)
    assert np.array_equal(core.cpu().numpy().astype(np.int64), core_ref)
    assert np.array_equal(two.cpu().numpy(), two_ref)
    Z = OL.features(g.offsets, g.cols, t)
    got = X.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - Z) <= 2e-5 + 1e-5 * np.abs(Z)), np.abs(got - Z).max()


def test_features_reject_bad_csr():
    g = graphs.path(5)
    cols = g.cols.copy()
    cols[0] = 4  # vertex 0 -> 4 without 4 -> 0
    with pytest.raises(pll.PLLError):
        pll.features(dev_u32(g.offsets), dev_u32(cols), 4)


@pytest.mark.parametrize("t", [0, 16])
@pytest.mark.parametrize("g", [graphs.star(8), gg.ba(1500, 2, 3), gg.rmat(12, 16, seed=6)],
                         ids=lambda g: g.name)
def test_hub_counts_match_oracle(g, t):
    ix = gpu_build(g, t)
    c, f = ix.hub_counts()
    ref = oracle.Index(g.offsets, g.cols, t)
    expect = OL.hub_counts(ref.labels(), ref.order())
    assert np.array_equal(c.cpu().numpy().astype(np.int64), expect)
    assert np.allclose(f.cpu().numpy(), np.log1p(expect), rtol=1e-6, atol=1e-7)


def test_order_from_scores_ties_and_signed_zero():
    import torch
    rng = np.random.default_rng(1)
    s = rng.integers(-5, 6, 20000).astype(np.float32) / 4  # many ties
    s[::97] = -0.0
    s[::89] = 0.0
    got = pll.order_from_scores(torch.from_numpy(s).cuda()).cpu().numpy().astype(np.uint32)
    assert np.array_equal(got, OL.order_from_scores(s))
    s2 = rng.standard_normal(3001).astype(np.float32)
    got2 = pll.order_from_scores(torch.from_numpy(s2).cuda()).cpu().numpy().astype(np.uint32)
    assert np.array_equal(got2, OL.order_from_scores(s2))


def random_params(seed):
    p = gg.mlp_init(seed)
    rng = np.random.default_rng(seed)
    p[512:576] = rng.uniform(-0.5, 0.5, 64)
    p[4672:4736] = rng.uniform(-0.5, 0.5, 64)
    p[4800] = 0.25
    return p


def test_bf16_copy_and_forward_match_oracle():
    import torch
    p = random_params(3)
    mlp = pll.MLP(max_batch=1024)
    mlp.set_params(p)
    master, b16 = mlp.params()
    assert np.array_equal(master, p)
    ref16 = OL.bf16_round(p).astype(np.float32).view(np.uint32) >> 16
    assert np.array_equal(b16.astype(np.uint32), ref16)
    X = np.random.default_rng(4).standard_normal((5000, 8)).astype(np.float32)
    y = mlp.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    yr, _ = OL.forward(p, X)
    assert np.max(np.abs(y - yr)) <= 1e-5 * max(1.0, np.abs(yr).max())


@pytest.mark.parametrize("batch,use_idx", [(1, False), (127, False), (128, True), (1000, True),
                                           (2049, True)])
def test_gradient_matches_oracle(batch, use_idx):
    import torch
    p = random_params(5)
    rng = np.random.default_rng(batch)
    N = 4096
    X = rng.standard_normal((N, 8)).astype(np.float32)
    T = rng.standard_normal(N).astype(np.float32)
    idx = rng.choice(N, batch, replace=False).astype(np.int32) if use_idx else np.arange(batch, dtype=np.int32)
    mlp = pll.MLP(max_batch=4096)
    mlp.set_params(p)
    g, loss = mlp.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(),
                       idx=torch.from_numpy(idx).cuda() if use_idx else None, batch=batch)
    lr_, gr = OL.loss_grad(p, X[idx].astype(np.float64), T[idx].astype(np.float64))
    assert loss == pytest.approx(lr_, rel=1e-5, abs=1e-7)
    scale = np.abs(gr).max()
    assert np.all(np.abs(g - gr) <= 1e-4 * scale + 1e-4 * np.abs(gr)), np.abs(g - gr).max() / scale
    # deterministic: the same call gives the same bits
    g2, loss2 = mlp.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(),
                         idx=torch.from_numpy(idx).cuda() if use_idx else None, batch=batch)
    assert np.array_equal(g, g2) and loss == loss2


def test_gradient_rejects_oversized_batch():
    import torch
    mlp = pll.MLP(max_batch=256)
    mlp.set_params(random_params(1))
    x = torch.zeros((300, 8), device="cuda")
    with pytest.raises(pll.PLLError):
        mlp.grad(x, torch.zeros(300, device="cuda"), batch=300)


def test_adam_steps_match_oracle():
    import torch
    p = random_params(6)
    rng = np.random.default_rng(7)
    X = torch.from_numpy(rng.standard_normal((700, 8)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.standard_normal(700).astype(np.float32)).cuda()
    mlp = pll.MLP(max_batch=1024)
    mlp.set_params(p)
    pr = p.astype(np.float64)
    m = np.zeros(OL.NPARAM)
    v = np.zeros(OL.NPARAM)
    for step in (1, 2, 3):
        g, _ = mlp.grad(X, T, batch=700)
        mlp.adam(1e-3)
        pr, m, v = OL.adam_step(pr, m, v, g.astype(np.float64), 1e-3, step)
        master, b16 = mlp.params()
        # float32: one rounding of p (6e-8 |p|) plus a few ulps of the step lr * (~1)
        assert np.all(np.abs(master - pr) <= 1e-6 * np.abs(pr) + 2e-9), (step, np.abs(master - pr).max())
        pr = master.astype(np.float64)  # continue from the device's float32 state
        assert np.array_equal(b16.astype(np.uint32),
                              OL.bf16_round(master).astype(np.float32).view(np.uint32) >> 16)


def test_learned_order_trains_and_builds_exact_labels():
    """Train on 24 small R-MATs, order a held-out R-MAT-13 by the network:
    the labels of that order equal the oracle's for the same order (Thm 4.1,
    4.2 hold for any order); the index is far smaller than under a random
    order, and its size against the Degree order is reported."""
    import torch
    specs = gg.learned_training_specs(24, seed=3, scales=(10, 11, 12), first_seed=500)
    train_graphs = [gg.rmat(sc, 16, seed=sd) for sc, sd in specs]
    X, y, rows, hs = L.harvest(train_graphs, t=16)
    assert hs["rows"] < hs["vertices"]
    mlp, th = L.train(X, y, rows, epochs=6, batch=4096, lr=3e-3)
    losses = [l for _, l in th["loss"]]
    assert losses[-1] < losses[0]
    g = gg.rmat(13, 16, seed=77)
    order = L.learned_order(mlp, g, t=16).cpu().numpy().astype(np.uint32)
    assert np.array_equal(np.sort(order), np.arange(g.n, dtype=np.uint32))
    ix = gpu_build(g, 16, order=order)
    ref = oracle.Index(g.offsets, g.cols, 16, order=order)
    La, Lb = ix.labels(), ref.labels()
    assert np.array_equal(La.offsets, Lb.offsets) and np.array_equal(La.hubs, Lb.hubs)
    assert np.array_equal(La.dists, Lb.dists)
    deg_entries = gpu_build(g, 16).label_entries()
    rnd = OL.order_from_scores(gg.uniform(9, g.n).astype(np.float32))
    rnd_entries = gpu_build(g, 16, order=rnd).label_entries()
    learned = ix.label_entries()
    print(f"label entries: learned {learned}, degree {deg_entries}, random {rnd_entries}")
    assert learned < rnd_entries / 2
    # The network is trained to predict the labels each vertex hubs under the
    # Degree order; ordering by that cannot beat the Degree order itself (even
    # the exact hub counts give 0.2-0.3 % more entries on R-MAT 13-15). Here it
    # gives 21,416 entries against Degree's 21,113 (1.4 % more; training is
    # deterministic): a regression past 2.5 % fails.
    assert learned <= 1.025 * deg_entries
    s, u = gg.pairs(g.n, 20000, 4)
    assert np.array_equal(ix.query(dev_u32(s), dev_u32(u)).cpu().numpy(), ref.query_batch(s, u))

"""Oracle of the learned vertex order -- TEST INFRASTRUCTURE ONLY.

Same rules as the rest of ``oracle/``: only tests, the smoke check and the
benchmark's CPU legs use it; it shares no code with the CUDA library.

The paper fixes the method's output for ANY vertex order (Thm 4.1, 4.2: the
labels are exact and minimal for that order) and shows that the order decides
the index size (Sec. 4.4, Table 4). It proposes Random, Degree and Closeness
orders; the learned order is an addition: a small network scores each vertex
from local features and vertices are taken by descending score. Everything
here is plain numpy in float64 unless a step fixes another precision:

  features(...)        eight per-vertex features, standardised per graph
  bf16_round(x)        float32 -> nearest bfloat16 (ties to even), as float64
  forward / loss_grad  the 8 -> 64 -> 64 -> 1 ReLU network with bf16-rounded
                       parameters, and the gradient of the mean squared error
  adam_step            one Adam update of the float32 master parameters
  order_from_scores    vertices by descending score, ties by ascending id
  hub_counts           label entries per hub vertex (the training target)

Parameter vector layout (4801 float32): W1 [64][8], b1 [64], W2 [64][64],
b2 [64], w3 [64], b3 [1]; row j of W holds the weights into unit j.
"""
from __future__ import annotations

import numpy as np

from . import Index, core_numbers

NF = 8
H = 64
NPARAM = H * NF + H + H * H + H + H + 1  # 4801
D_CAP = 32  # distances to bit-parallel roots are capped here (255 = unreachable)

_SLICES = {}
_o = 0
for _name, _shape in (("W1", (H, NF)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)),
                      ("b3", (1,))):
    _k = int(np.prod(_shape))
    _SLICES[_name] = (slice(_o, _o + _k), _shape)
    _o += _k
assert _o == NPARAM


def unpack(p):
    """Parameter vector -> dict of arrays (views)."""
    return {k: p[s].reshape(shape) for k, (s, shape) in _SLICES.items()}


def _popcount(m):
    """Set bits of each uint64 (unpacked to single bits and summed)."""
    m = np.ascontiguousarray(m, dtype=np.uint64)
    bits = np.unpackbits(m.view(np.uint8).reshape(m.shape + (8,)), axis=-1)
    return bits.sum(axis=-1).astype(np.int64)


# ------------------------------------------------------------------ features
def raw_features(offsets, cols, t: int):
    """Per-vertex quantities before standardisation:
    deg(v); two_hop(v) = sum of deg(u) over neighbours u (walks of length 2);
    core(v); and, from the bit-parallel labels of the Degree order with t roots
    (Alg. 3, Sec. 5.4), with d_i = min(d(r_i, v), D_CAP) over the t slots:
    mean_i d_i, min_i d_i, #{i : d_i <= 2} / t, mean_i |S^-1_i(v)| / 64 and
    mean_i |S^0_i(v)| / 64 (all 0 when t = 0)."""
    off = np.asarray(offsets, dtype=np.int64)
    col = np.asarray(cols, dtype=np.int64)
    n = off.shape[0] - 1
    deg = np.diff(off)
    two_hop = np.zeros(n, dtype=np.int64)
    src = np.repeat(np.arange(n), deg)
    np.add.at(two_hop, src, deg[col])
    core = core_numbers(offsets, cols).astype(np.int64)
    bp = np.zeros((n, 5))
    if t > 0 and n > 0:
        d, m1, m0 = Index(offsets, cols, t, with_pruned=False).bp()
        dc = np.minimum(d.astype(np.float64), D_CAP)
        bp[:, 0] = dc.mean(axis=1)
        bp[:, 1] = dc.min(axis=1)
        bp[:, 2] = (dc <= 2).sum(axis=1) / t
        bp[:, 3] = _popcount(m1).mean(axis=1) / 64.0
        bp[:, 4] = _popcount(m0).mean(axis=1) / 64.0
    return deg, two_hop, core, bp


def features(offsets, cols, t: int):
    """[n][8] float64: log1p(deg), log1p(two_hop), log1p(core), then the five
    bit-parallel statistics; each column standardised over the graph's
    vertices, (x - mean) / std with the population std, or 0 where std = 0."""
    deg, two_hop, core, bp = raw_features(offsets, cols, t)
    n = deg.shape[0]
    X = np.zeros((n, NF))
    X[:, 0] = np.log1p(deg)
    X[:, 1] = np.log1p(two_hop)
    X[:, 2] = np.log1p(core)
    X[:, 3:] = bp
    if n == 0:
        return X
    # a column of equal values has std 0 exactly; test that directly, since
    # the float64 mean of equal values need not equal them
    ok = X.max(axis=0) > X.min(axis=0)
    mu = X.mean(axis=0)
    sd = np.sqrt(((X - mu) ** 2).mean(axis=0))
    Z = np.zeros_like(X)
    Z[:, ok] = (X[:, ok] - mu[ok]) / sd[ok]
    return Z


# ------------------------------------------------------------------ network
def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even); returns
    float64 holding the rounded values. NaN and infinity are not expected."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X):
    """Scores y [n] and the activations with the float32 master parameters p
    rounded to bf16 first (see net)."""
    return net(bf16_round(p), X)


def net(qv, X):
    """The network at float64 parameters qv (no rounding):
    z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2),
    y = w3 . h2 + b3. Returns y and (X, z1, h1, z2, h2)."""
    q = unpack(np.asarray(qv, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0)
    y = h2 @ q["w3"] + q["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_grad(p, X, target):
    """Mean squared error over the rows and its gradient with respect to the
    parameters, at the float32 master parameters p rounded to bf16."""
    return net_loss_grad(bf16_round(p), X, target)


def net_loss_grad(qv, X, target):
    """Mean squared error of net(qv, X) against target and its gradient with
    respect to qv, by the chain rule through the network."""
    q = unpack(np.asarray(qv, dtype=np.float64))
    y, (X, z1, h1, z2, h2) = net(qv, X)
    B = X.shape[0]
    r = y - np.asarray(target, dtype=np.float64)
    loss = float((r ** 2).mean())
    dy = 2.0 * r / B                       # d loss / d y
    g = np.zeros(NPARAM)
    G = unpack(g)
    G["w3"][:] = h2.T @ dy
    G["b3"][:] = dy.sum()
    dz2 = np.outer(dy, q["w3"]) * (z2 > 0)
    G["W2"][:] = dz2.T @ h1
    G["b2"][:] = dz2.sum(axis=0)
    dz1 = (dz2 @ q["W2"]) * (z1 > 0)
    G["W1"][:] = dz1.T @ X
    G["b1"][:] = dz1.sum(axis=0)
    return loss, g


def adam_step(p, m, v, g, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) at 1-based step `step`:
    m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    p <- p - lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ order
def order_from_scores(scores):
    """order[r] = the vertex of rank r: descending score, ties by ascending id."""
    s = np.asarray(scores)
    return np.lexsort((np.arange(s.shape[0]), -s.astype(np.float64))).astype(np.uint32)


def hub_counts(labels, order):
    """counts[v] = number of label entries whose hub is vertex v (labels store
    hub ranks; order maps a rank to its vertex)."""
    n = order.shape[0]
    by_rank = np.bincount(labels.hubs.astype(np.int64), minlength=n)
    out = np.zeros(n, dtype=np.int64)
    out[order] = by_rank
    return out

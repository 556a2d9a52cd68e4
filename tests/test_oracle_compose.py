"""Pins for the oracle's composition of gates into a softmax block (App. G):
Beaver multiplication by its definition, the composed shares against the
plaintext pipeline (exact), the comparison-tree max against numpy's max
(exact), the bytes sent against the gates' closed forms, and the fixed-point
result against float64 softmax (scale sanity: a wrong shift fails it)."""
import numpy as np
import pytest

import oracle as O
from oracle import compose as C
from paper_2606_09551_b300 import specs as S

SEED = bytes(range(16))


def _gates():
    return {k: O.Spec(**v.descriptor()) for k, v in S.softmax_specs().items()}


@pytest.mark.parametrize("group", [1, 7])
def test_beaver_mul_definition(group):
    """Sec. 3.4: the shares reconstruct to x * y[e // group] over Z_{2^64};
    16 bytes per element per party."""
    rng = np.random.default_rng(group)
    n = 700
    x = rng.integers(0, 2 ** 64, n, dtype=np.uint64)
    y = rng.integers(0, 2 ** 64, n // group, dtype=np.uint64)
    x0 = rng.integers(0, 2 ** 64, n, dtype=np.uint64)
    y0 = rng.integers(0, 2 ** 64, y.size, dtype=np.uint64)
    t0, t1 = O.beaver_dealer(SEED, 3, 0, n)
    assert np.array_equal((t0[0] + t1[0]) * (t0[1] + t1[1]), t0[2] + t1[2])     # c = a b
    z0, z1, comm = O.beaver_mul(t0, t1, x0, x - x0, y0, y - y0, group)
    assert np.array_equal(z0 + z1, x * np.repeat(y, group))
    assert list(comm) == [16 * n] * 2


def _scores(rng, rows, L, sigma=2.0):
    g = sigma * rng.standard_normal((rows, L))
    x = S.encode(g.reshape(-1), 12).reshape(rows, L)
    x0 = rng.integers(0, 2 ** 64, size=(rows, L), dtype=np.uint64)
    return g, x, x0, x - x0


@pytest.mark.parametrize("rows,L", [(3, 1), (4, 2), (5, 7), (2, 16), (3, 128)])
def test_softmax_pair_equals_plain(rows, L):
    g = _gates()
    rng = np.random.default_rng(10 * rows + L)
    _, x, x0, x1 = _scores(rng, rows, L)
    y0, y1, comm, st = C.softmax_pair(g, SEED, 500, x0, x1)
    yp, plain = C.softmax_plain(g, x)
    assert np.array_equal(y0 + y1, yp)
    m = st["m"][0] + st["m"][1]
    assert np.array_equal(m.view(np.int64), x.view(np.int64).max(axis=1))
    assert np.array_equal(m, plain["m"])
    # bytes: each gate's 8 + 16 n_mults (+1 for a shift), the product 16
    tree = 0
    n = L
    while n > 1:
        tree += rows * (n // 2)
        n = n // 2 + n % 2
    per = {"relu": 8 + 16, "exp": 8 + 48, "shift": 9, "recip": 8 + 48, "mul": 16}
    want = (tree * per["relu"] + rows * L * (per["exp"] + per["shift"] + per["mul"] + per["shift"])
            + rows * (per["recip"] + per["shift"]))
    assert list(comm) == [want] * 2


def test_softmax_accuracy_against_float():
    """The fixed-point pipeline against float64 softmax on N(0, 2^2) scores
    and on rows dominated by one value."""
    g = _gates()
    rng = np.random.default_rng(99)
    gs, x, _, _ = _scores(rng, 16, 128)
    dom = np.full((2, 128), -10.0)
    dom[:, 5] = 10.0
    gs = np.concatenate([gs, dom])
    x = np.concatenate([x, S.encode(dom.reshape(-1), 12).reshape(2, 128)])
    yp, _ = C.softmax_plain(g, x)
    got = yp.view(np.int64) / 2.0 ** 12
    ref = np.exp(gs - gs.max(axis=1, keepdims=True))
    ref /= ref.sum(axis=1, keepdims=True)
    assert np.abs(got - ref).max() < 3e-3
    assert np.abs(got.sum(axis=1) - 1.0).max() < 1e-2


@pytest.mark.parametrize("rows,H", [(3, 1), (4, 5), (3, 768)])
def test_layernorm_pair_equals_plain(rows, H):
    """LayerNorm composition (App. G): shares reconstruct to the plaintext
    pipeline exactly; the mean is the rounded row mean; bytes = the gates'
    closed forms plus 16 per Beaver product."""
    sp, cH = S.layernorm_specs(H)
    g = {k: O.Spec(**v.descriptor()) for k, v in sp.items()}
    rng = np.random.default_rng(rows * 7 + H)
    h = 1.3 * rng.standard_normal((rows, H)) + 0.4
    x = S.encode(h.reshape(-1), 12).reshape(rows, H)
    x0 = rng.integers(0, 2 ** 64, size=(rows, H), dtype=np.uint64)
    y0, y1, comm, st = C.layernorm_pair(g, SEED, 900, x0, x - x0, cH)
    yp, plain = C.layernorm_plain(g, x, cH)
    assert np.array_equal(y0 + y1, yp)
    mu = (st["mu"][0] + st["mu"][1]).view(np.int64)
    sx = x.view(np.int64).sum(axis=1)
    assert np.array_equal(mu, np.floor((sx * cH + 2 ** 23) / 2 ** 24).astype(np.int64))
    want = rows * (9 + 9 + (8 + 48) + 9) + rows * H * (16 + 16 + 9)
    assert list(comm) == [want] * 2


def test_layernorm_accuracy_against_float():
    sp, cH = S.layernorm_specs(768)
    g = {k: O.Spec(**v.descriptor()) for k, v in sp.items()}
    rng = np.random.default_rng(5)
    h = rng.standard_normal((8, 768)) * np.linspace(0.5, 3, 8)[:, None] + np.linspace(-2, 2, 8)[:, None]
    x = S.encode(h.reshape(-1), 12).reshape(8, 768)
    yp, _ = C.layernorm_plain(g, x, cH)
    ref = (h - h.mean(axis=1, keepdims=True)) / np.sqrt(h.var(axis=1, keepdims=True) + 1e-5)
    assert np.abs(yp.view(np.int64) / 2.0 ** 12 - ref).max() < 5e-3

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


# --------------------------------------------------------------------------
# Newton refinement of the reciprocal and of 1/sqrt (a fixed post-processing
# circuit of Beaver products and shift gates; Def. "specification-compatible
# scalar gate", App. G)
# --------------------------------------------------------------------------

def _ev(g, name, v):
    v = np.asarray(v, np.uint64)
    if g[name].trunc_s:
        v = v + np.uint64(1 << (g[name].trunc_s - 1))
    return g[name].plain_eval(v)[0][:, 0]


def test_reciprocal_newton_squares_the_error():
    """t' = t (2 - s t) gives s t' - 1 = -(s t - 1)^2 exactly over the reals;
    in fixed point (s at 16, t at 20 bits) the two rounded shifts add at most
    one unit of t': |e' + e^2| <= s 2^-20 for every s of a log sweep."""
    g = _gates()
    s = np.unique(np.round(np.exp(np.linspace(0, np.log(2000), 4000)) * 2 ** 16).astype(np.int64)).astype(np.uint64)
    t = _ev(g, "shift_t", _ev(g, "recip", s))
    sf = s.astype(np.float64) / 2 ** 16
    e0 = sf * t.view(np.int64) / 2 ** 20 - 1
    u = _ev(g, "shift_n1", s * t)
    t1 = _ev(g, "shift_n2", t * (np.uint64(1 << 21) - u))
    e1 = sf * t1.view(np.int64) / 2 ** 20 - 1
    assert np.all(np.abs(e1 + e0 ** 2) <= sf * 2.0 ** -20)
    assert np.abs(e0).max() > 1e-2 and np.abs(e1).max() < 1e-2


def test_rsqrt_newton_squares_the_error():
    """r' = r (3 - v r^2) / 2 gives r' sqrt(v) - 1 = -(3/2) e^2 - (1/2) e^3 for
    r sqrt(v) = 1 + e; in fixed point (v at 12, r at 20 bits) the three
    rounded shifts add a few units of r'."""
    sp, _ = S.layernorm_specs(768)
    g = {k: O.Spec(**v.descriptor()) for k, v in sp.items()}
    v = np.unique(np.round(np.exp(np.linspace(np.log(0.125), np.log(120), 3000)) * 2 ** 12).astype(np.int64)).astype(np.uint64)
    r = _ev(g, "shift_r", _ev(g, "rsqrt", v))
    vf = v.astype(np.float64) / 2 ** 12
    e0 = np.sqrt(vf) * r.view(np.int64) / 2 ** 20 - 1
    q = _ev(g, "shift_n1", r * r)
    w = _ev(g, "shift_n2", v * q)
    r1 = _ev(g, "shift_n3", r * (np.uint64(3 << 20) - w))
    e1 = np.sqrt(vf) * r1.view(np.int64) / 2 ** 20 - 1
    want = -1.5 * e0 ** 2 - 0.5 * e0 ** 3
    assert np.all(np.abs(e1 - want) <= 4 * np.sqrt(vf) * 2.0 ** -20)
    assert np.abs(e1).max() < np.abs(e0).max() / 20     # down to the fixed-point floor


@pytest.mark.parametrize("rows,L", [(3, 1), (5, 7), (3, 128)])
def test_softmax_newton_pair_equals_plain(rows, L):
    g = _gates()
    rng = np.random.default_rng(30 * rows + L)
    _, x, x0, x1 = _scores(rng, rows, L)
    y0, y1, comm, st = C.softmax_pair(g, SEED, 600, x0, x1, newton=1)
    yp, plain = C.softmax_plain(g, x, newton=1)
    assert np.array_equal(y0 + y1, yp)
    assert np.array_equal(st["t"][0] + st["t"][1], plain["t"])
    _, _, comm0, _ = C.softmax_pair(g, SEED, 600, x0, x1)
    # one Newton step: two products (16 bytes) and two shift gates (9 bytes) per row
    assert list(comm - comm0) == [rows * (16 + 9 + 16 + 9)] * 2


def test_softmax_newton_accuracy_against_float():
    g = _gates()
    rng = np.random.default_rng(99)
    gs, x, _, _ = _scores(rng, 16, 128)
    ref = np.exp(gs - gs.max(axis=1, keepdims=True))
    ref /= ref.sum(axis=1, keepdims=True)
    err = [np.abs(C.softmax_plain(g, x, newton=k)[0].view(np.int64) / 2.0 ** 12 - ref).max() for k in (0, 1)]
    assert err[1] < 3e-4 and err[1] < err[0] / 3


@pytest.mark.parametrize("rows,H", [(3, 1), (3, 768)])
def test_layernorm_newton_pair_equals_plain(rows, H):
    sp, cH = S.layernorm_specs(H)
    g = {k: O.Spec(**v.descriptor()) for k, v in sp.items()}
    rng = np.random.default_rng(rows * 11 + H)
    h = 1.3 * rng.standard_normal((rows, H)) + 0.4
    x = S.encode(h.reshape(-1), 12).reshape(rows, H)
    x0 = rng.integers(0, 2 ** 64, size=(rows, H), dtype=np.uint64)
    y0, y1, comm, st = C.layernorm_pair(g, SEED, 950, x0, x - x0, cH, newton=1)
    yp, plain = C.layernorm_plain(g, x, cH, newton=1)
    assert np.array_equal(y0 + y1, yp)
    assert np.array_equal(st["r"][0] + st["r"][1], plain["r"])
    want = rows * (9 + 9 + (8 + 48) + 9) + rows * H * (16 + 16 + 9) + rows * 3 * (16 + 9)
    assert list(comm) == [want] * 2


def test_layernorm_newton_accuracy_against_float():
    sp, cH = S.layernorm_specs(768)
    g = {k: O.Spec(**v.descriptor()) for k, v in sp.items()}
    rng = np.random.default_rng(5)
    h = rng.standard_normal((8, 768)) * np.linspace(0.5, 3, 8)[:, None] + np.linspace(-2, 2, 8)[:, None]
    x = S.encode(h.reshape(-1), 12).reshape(8, 768)
    ref = (h - h.mean(axis=1, keepdims=True)) / np.sqrt(h.var(axis=1, keepdims=True) + 1e-5)
    err = [np.abs(C.layernorm_plain(g, x, cH, newton=k)[0].view(np.int64) / 2.0 ** 12 - ref).max() for k in (0, 1)]
    assert err[1] < 1e-3 and err[1] < err[0]

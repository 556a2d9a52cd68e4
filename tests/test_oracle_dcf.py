"""Pins for the oracle's DCF (a generalisation of Boyle et al., EUROCRYPT
2021, to arity 2^r: r input bits per tree level) by brute force:
Eval_0 (+) Eval_1 = beta * 1[u < alpha] for every alpha and every u at small
k, for r = 1 to 6 (every arity the gates take), including k not a
multiple of r, and over two and three levels at arities 32 and 64."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_bit_dcf_all_alpha_all_u(k, r):
    rng = np.random.default_rng(100 + k + 10 * r)
    for alpha in range(2 ** k):
        a, b = O.dcf_gen(k, alpha, 0, None, rng.bytes(16), rng.bytes(16), r=r)
        for u in range(2 ** k):
            assert O.dcf_eval(0, a, u, 0) ^ O.dcf_eval(1, b, u, 0) == (1 if u < alpha else 0)


def test_bit_dcf_k10_sampled_alpha_all_u():
    k = 10
    rng = np.random.default_rng(7)
    for alpha in [0, 1, 511, 512, 513, 1023] + [int(v) for v in rng.integers(0, 1024, 6)]:
        a, b = O.dcf_gen(k, alpha, 0, None, rng.bytes(16), rng.bytes(16))
        for u in range(2 ** k):
            assert O.dcf_eval(0, a, u, 0) ^ O.dcf_eval(1, b, u, 0) == (1 if u < alpha else 0)


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("k,p", [(1, 1), (3, 2), (5, 3), (5, 4), (6, 1)])
def test_vector_dcf_all_alpha_all_u(k, p, r):
    rng = np.random.default_rng(200 + 10 * k + p + 100 * r)
    for alpha in range(2 ** k):
        beta = rng.integers(0, 2 ** 64, size=p, dtype=np.uint64)
        a, b = O.dcf_gen(k, alpha, p, beta, rng.bytes(16), rng.bytes(16), r=r)
        for u in range(2 ** k):
            got = O.dcf_eval(0, a, u, p) + O.dcf_eval(1, b, u, p)
            want = beta if u < alpha else np.zeros(p, np.uint64)
            assert (got == want).all()


@pytest.mark.parametrize("r,k", [(5, 11), (6, 7), (6, 8), (6, 13)])
@pytest.mark.parametrize("p", [0, 4])
def test_dcf_wide_arity_every_u(r, k, p):
    """Arities 32 and 64 over two or three levels (a first digit of 1 to 3
    bits): every u, for alpha at 0, 1, the top, each side of a digit
    boundary and at random."""
    rng = np.random.default_rng(500 + 10 * r + k + p)
    top = 2 ** k
    alphas = {0, 1, top - 1, top // 2, 2 ** r - 1, 2 ** r, 2 ** r + 1, 3 * 2 ** r}
    alphas |= {int(v) for v in rng.integers(0, top, 3)}
    u = np.arange(top)
    for alpha in sorted(a for a in alphas if a < top):
        beta = rng.integers(0, 2 ** 64, size=p, dtype=np.uint64) if p else None
        a, b = O.dcf_gen(k, alpha, p, beta, rng.bytes(16), rng.bytes(16), r=r)
        if p == 0:
            got = np.array([O.dcf_eval(0, a, int(x), 0) ^ O.dcf_eval(1, b, int(x), 0) for x in u])
            assert np.array_equal(got, (u < alpha).astype(got.dtype)), alpha
        else:
            for x in u:
                got = O.dcf_eval(0, a, int(x), p) + O.dcf_eval(1, b, int(x), p)
                assert (got == (beta if x < alpha else np.zeros(p, np.uint64))).all(), (alpha, x)


def test_path_child_randomness_hides_alpha():
    """The correction words at a level do not single out alpha's digit: over
    many keys, the t-CW bits of every child are unbiased, and for each child
    the value-CW bit is unbiased too (the path child's are drawn fresh, the
    others are masked by pseudorandom expansion bits)."""
    rng = np.random.default_rng(12)
    k, r = 8, 2
    counts = np.zeros((4, 4, 2))
    for trial in range(800):
        alpha = int(rng.integers(0, 2 ** k))
        a, _ = O.dcf_gen(k, alpha, 0, None, rng.bytes(16), rng.bytes(16), r=r)
        f = a.fields()
        d0 = (alpha >> 6) & 3                     # digit of the first level
        for c in range(4):
            counts[d0, c, 0] += f["cw"][0, c, 0] & 1
            counts[d0, c, 1] += (f["cw"][0, c, 0] >> 1) & 1
    per = counts / (counts.sum(axis=(1, 2), keepdims=True) / 8 + 1e-9)
    assert np.abs(per - 1.0).max() < 0.35


def test_vector_dcf_k10_sampled():
    k, p = 10, 3
    rng = np.random.default_rng(9)
    for alpha in [0, 1, 1023, 700]:
        beta = rng.integers(0, 2 ** 64, size=p, dtype=np.uint64)
        a, b = O.dcf_gen(k, alpha, p, beta, rng.bytes(16), rng.bytes(16))
        for u in range(2 ** k):
            got = O.dcf_eval(0, a, u, p) + O.dcf_eval(1, b, u, p)
            want = beta if u < alpha else np.zeros(p, np.uint64)
            assert (got == want).all()


def test_single_key_shares_look_random():
    """A party's share alone does not reveal 1[u < alpha]: party 0's bits
    are unbiased across u (a sanity check of the t-bit/correction logic,
    not a security proof)."""
    k = 10
    rng = np.random.default_rng(3)
    a, b = O.dcf_gen(k, 512, 0, None, rng.bytes(16), rng.bytes(16))
    s0 = np.array([O.dcf_eval(0, a, u, 0) for u in range(2 ** k)])
    assert 0.4 < s0[:512].mean() < 0.6 and 0.4 < s0[512:].mean() < 0.6


@pytest.mark.parametrize("k", [33, 47, 63])
def test_bit_dcf_wide_views(k):
    """Bit DCF on views wider than 32 bits (comparisons up to k = 63): on
    random alpha and u plus the neighbours of alpha and the ends of the
    domain, Eval_0 xor Eval_1 = 1[u < alpha]."""
    rng = np.random.default_rng(k)
    for trial in range(6):
        alpha = int(rng.integers(1, 2 ** k - 1, dtype=np.uint64))
        k0, k1 = O.dcf_gen(k, alpha, 0, None, rng.bytes(16), rng.bytes(16))
        us = [0, 2 ** k - 1, alpha - 1, alpha, alpha + 1] + [int(v) for v in rng.integers(0, 2 ** k, 10, dtype=np.uint64)]
        for u in us:
            assert (O.dcf_eval(0, k0, u, 0) ^ O.dcf_eval(1, k1, u, 0)) == int(u < alpha), (alpha, u)

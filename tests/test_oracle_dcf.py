"""Pins for the oracle's DCF (Boyle et al., EUROCRYPT 2021) by brute force:
Eval_0 (+) Eval_1 = beta * 1[u < alpha] for every alpha and every u at small k."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_bit_dcf_all_alpha_all_u(k):
    rng = np.random.default_rng(100 + k)
    for alpha in range(2 ** k):
        a, b = O.dcf_gen(k, alpha, 0, None, rng.bytes(16), rng.bytes(16))
        for u in range(2 ** k):
            assert O.dcf_eval(0, a, u, 0) ^ O.dcf_eval(1, b, u, 0) == (1 if u < alpha else 0)


def test_bit_dcf_k10_sampled_alpha_all_u():
    k = 10
    rng = np.random.default_rng(7)
    for alpha in [0, 1, 511, 512, 513, 1023] + [int(v) for v in rng.integers(0, 1024, 6)]:
        a, b = O.dcf_gen(k, alpha, 0, None, rng.bytes(16), rng.bytes(16))
        for u in range(2 ** k):
            assert O.dcf_eval(0, a, u, 0) ^ O.dcf_eval(1, b, u, 0) == (1 if u < alpha else 0)


@pytest.mark.parametrize("k,p", [(1, 1), (3, 2), (5, 3), (5, 4)])
def test_vector_dcf_all_alpha_all_u(k, p):
    rng = np.random.default_rng(200 + 10 * k + p)
    for alpha in range(2 ** k):
        beta = rng.integers(0, 2 ** 64, size=p, dtype=np.uint64)
        a, b = O.dcf_gen(k, alpha, p, beta, rng.bytes(16), rng.bytes(16))
        for u in range(2 ** k):
            got = O.dcf_eval(0, a, u, p) + O.dcf_eval(1, b, u, p)
            want = beta if u < alpha else np.zeros(p, np.uint64)
            assert (got == want).all()


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

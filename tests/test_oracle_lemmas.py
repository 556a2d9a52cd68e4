"""Brute-force pins of the paper's identities at small bit widths, written
here directly from the lemma statements (independent of the oracle), plus
the oracle's per-element lookup compilation checked against them."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2606_09551_b300 import specs as S


def lt(a, b):
    return 1 if a < b else 0


@pytest.mark.parametrize("n", [1, 3, 5])
def test_mask_rewrite_unsigned(n):
    """Lemma 'masked rewrite for unsigned comparison' (Sec. 4.3):
    1[x < beta] = 1[x^ < theta] ^ 1[x^ < r] ^ w, theta = (r+beta) mod N, w = 1[r+beta >= N]."""
    N = 2 ** n
    for beta in range(N + 1):
        for r in range(N):
            theta, w = (r + beta) % N, lt(N - 1, r + beta)
            for x in range(N):
                xh = (x + r) % N
                assert lt(x, beta) == lt(xh, theta) ^ lt(xh, r) ^ w


@pytest.mark.parametrize("n,f", [(5, 2), (6, 3), (4, 4)])
def test_mask_rewrite_lowbit(n, f):
    """Lemma 'masked rewrite for low-bit predicate' (App. E)."""
    N, Nf = 2 ** n, 2 ** f
    for gamma in range(Nf + 1):
        for r in range(N):
            rf = r % Nf
            theta, w = (rf + gamma) % Nf, lt(Nf - 1, rf + gamma)
            for x in range(N):
                xhf = ((x + r) % N) % Nf
                assert lt(x % Nf, gamma) == lt(xhf, theta) ^ lt(xhf, rf) ^ w


@pytest.mark.parametrize("n", [3, 5])
def test_signed_and_msb_rewrites(n):
    """App. J: signed compare and MSB(x+c) as shifted unsigned compares."""
    N, s = 2 ** n, 2 ** (n - 1)
    def signed(v):
        return v - N if v >= s else v
    for beta in range(N):
        bp = (beta + s) % N
        for r in range(N):
            theta, w = (r + bp) % N, lt(N - 1, r + bp)
            for x in range(N):
                xh = (x + r) % N
                vx = (xh + s) % N
                assert lt(signed(x), signed(beta)) == lt(vx, theta) ^ lt(vx, r) ^ w
    for c in range(N):
        for r in range(N):
            th, w = (r + s) % N, lt(N - 1, r + s)
            for x in range(N):
                xc = ((x + r) % N + c) % N
                msb = 1 if (x + c) % N >= s else 0
                assert msb == 1 ^ (lt(xc, th) ^ lt(xc, r) ^ w)


def test_interval_indicators_partition():
    """Lemmas 'interval indicator as XOR' and 'indicators form a partition' (App. D, J)."""
    n = 5
    N = 2 ** n
    rng = np.random.default_rng(1)
    for _ in range(50):
        m = int(rng.integers(1, N + 1))
        alpha = [0] + sorted(rng.choice(np.arange(1, N), m - 1, replace=False).tolist()) + [N]
        for x in range(N):
            J = [lt(x, alpha[i + 1]) ^ lt(x, alpha[i]) for i in range(m)]
            assert sum(J) == 1
            i = J.index(1)
            assert alpha[i] <= x < alpha[i + 1]


@pytest.mark.parametrize("k", [2, 3, 5])
def test_oracle_lookup_compilation_every_mask(k):
    """Protocol 'compile a scalar gate' step (1) as the oracle implements it:
    for every mask r, |B| = M+1, B strictly increasing from 0 to 2^k, and the
    translated lookup returns the piece of x for every x (Lemma 'interval
    translation': at most one interval splits)."""
    N = 2 ** k
    rng = np.random.default_rng(k)
    for trial in range(30):
        m = int(rng.integers(2, min(N, 16) + 1))
        sp = S.random_spec(rng, k, m, 0)
        o = O.Spec(k, m, 0, 1, sp.alpha, sp.coeff)
        assert o.M == min(m + 1, N)
        for r in range(N):
            B, ordv = o.compile_lookup(r)
            B = [int(b) for b in B]
            assert len(B) == o.M + 1 and B[0] == 0 and B[-1] == N
            assert all(a < b for a, b in zip(B, B[1:]))
            for x in range(N):
                xh = (x + r) % N
                j = max(i for i in range(o.M) if B[i] <= xh)
                piece = max(i for i in range(m) if sp.alpha[i] <= x)
                assert ordv[j] == piece
            # payload duplication: the lookup has exactly M - m duplicated entries
            assert len(set(ordv.tolist())) == m


def test_padding_split_is_smallest_gap():
    """When the wrap point hits a boundary (beta_0 = 0), the dummy split is
    delta = B_{j*} + 1 at the smallest j* with a gap >= 2 (App. F)."""
    k = 4
    alpha = [0, 1, 2, 8, 16]          # gaps 1, 1, 6, 8
    o = O.Spec(k, 4, 0, 1, alpha, np.zeros(4, np.uint64))
    B, ordv = o.compile_lookup(0)     # r = 0: no wrap
    assert [int(b) for b in B] == [0, 1, 2, 3, 8, 16]
    assert ordv.tolist() == [0, 1, 2, 2, 3]
    B, ordv = o.compile_lookup(16 - 8)   # r_k = 8: alpha_3 + r = 16 wraps onto 0
    assert int(B[0]) == 0 and len(B) == 6

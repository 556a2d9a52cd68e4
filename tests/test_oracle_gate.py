"""Pins for the oracle's whole gate: compiler correctness (Lemma 'compiler
correctness'), the App. N ReLU closed form, the plaintext evaluator against an
independent Python evaluation, communication counts and public shapes."""
import numpy as np
import pytest

import oracle as O
from conftest import golden
from paper_2606_09551_b300 import specs as S

SEED = bytes(range(16))
M64 = (1 << 64) - 1


def ospec(sp):
    return O.Spec(**sp.descriptor())


def _formula_value(nodes, v, x):
    """The bit-expression grammar's semantics with Python booleans."""
    nd = nodes[v]
    if nd.op == "pred":
        q = nd.pred
        return int((((x % (1 << q.f)) + q.c) % (1 << q.f)) < q.gamma) ^ q.negate
    if nd.op == "const":
        return nd.a
    if nd.op == "not":
        return 1 - _formula_value(nodes, nd.a, x)
    a, b = _formula_value(nodes, nd.a, x), _formula_value(nodes, nd.b, x)
    return {"xor": a ^ b, "and": a & b, "or": a | b}[nd.op]


def python_plain(sp, xs):
    """Independent plaintext evaluation with Python integers."""
    ys, zs = [], []
    bits = []
    if sp.partition_bits:
        bits += [(sp.k, 0, a, 0) for a in sp.alpha[1:-1]]
    bits += sp.pred_tuples()
    for x in (int(v) for v in xs):
        xk = x % (1 << sp.k)
        i = int(np.searchsorted(np.array(sp.alpha[:-1], dtype=object), xk, side="right")) - 1
        row = []
        for o in range(sp.n_out):
            c = [int(v) for v in sp.coeff[i, o]]
            acc = 0
            for j in range(sp.degree, -1, -1):
                acc = (acc * x + c[j]) & M64
            row.append(acc)
        if sp.trunc_shift:                  # Python's >> floors negative values
            v = xk - (1 << sp.k) if (sp.trunc_signed and xk >> (sp.k - 1)) else xk
            row[0] = (row[0] + (v >> sp.trunc_shift)) & M64
        ys.append(row)
        z = 0
        for t, (f, c, g, neg) in enumerate(bits):
            v = (((x % (1 << f)) + c) % (1 << f)) < g
            z |= (int(v) ^ neg) << t
        for j, out in enumerate(sp.piecewise):          # the active interval's predicate / formula
            if sp.bx_nodes:
                z |= _formula_value(sp.bx_nodes, out[i], x) << (len(bits) + j)
                continue
            q = out[i]
            v = (((x % (1 << q.f)) + q.c) % (1 << q.f)) < q.gamma
            z |= (int(v) ^ q.negate) << (len(bits) + j)
        zs.append(z)
    return np.array(ys, dtype=np.uint64), np.array(zs, dtype=np.uint32)


def run_gate(sp, x, r_override=None, call_id=0):
    o = ospec(sp)
    k0, k1, x0, x1 = O.dealer(o, SEED, call_id, 0, x.size, x, r_override=r_override)
    res = O.eval_pair(o, k0, k1, x0, x1)
    y, z = O.reconstruct(res["y0"], res["y1"], res["z0"], res["z1"], sp.n_out)
    return o, res, y, z


def test_plain_evaluator_matches_independent_python():
    rng = np.random.default_rng(1)
    for trial in range(12):
        k = int(rng.integers(3, 25))
        m = int(rng.integers(1, 17))
        d = int(rng.integers(0, 4))
        r = 1 if d > 1 else int(rng.integers(1, 3))
        sp = S.random_spec(rng, k, m, d, r, partition_bits=bool(trial % 2), n_extra=int(rng.integers(0, 4)))
        if trial % 3 == 0:
            sp.trunc_shift, sp.trunc_signed = int(rng.integers(1, k)), bool(trial % 2)
        x = rng.integers(0, 2 ** 64, size=300, dtype=np.uint64)
        y, z = ospec(sp).plain_eval(x)
        yp, zp = python_plain(sp, x)
        assert (y == yp).all() and (z == zp).all()


@pytest.mark.parametrize("dcf_bits", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_gate_every_mask_every_input(k, dcf_bits):
    """Reconstruction equals F(x) for all x and all masks r (Lemma 'compiler
    correctness'), with DCF keys of arity 2, 4 and 8 (for arity 8 and k = 4,
    5 the first tree level takes one or two input bits)."""
    rng = np.random.default_rng(40 + k)
    N = 2 ** k
    for trial in range(6):
        m = int(rng.integers(1, min(N, 16) + 1))
        d = int(rng.integers(0, 4))
        sp = S.random_spec(rng, k, m, d, 1, partition_bits=bool(trial % 2),
                           n_extra=int(rng.integers(0, 3))).arity(dcf_bits)
        hi_x = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
        hi_r = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
        xs = np.tile(np.arange(N, dtype=np.uint64), N) + hi_x
        rs = np.repeat(np.arange(N, dtype=np.uint64), N) + hi_r
        o, res, y, z = run_gate(sp, xs, r_override=rs)
        yp, zp = python_plain(sp, xs)
        assert (y == yp).all() and (z == zp).all()
        # online communication: 8 B for the opening + 16 B per Beaver multiplication
        assert (res["comm"] == xs.size * (8 + 16 * d * sp.n_out)).all()


@pytest.mark.parametrize("dcf_bits", [5, 6])
def test_gate_every_mask_every_input_two_levels_wide_arity(dcf_bits):
    """The whole gate at k = 7 with arity-32 and arity-64 keys, whose walks
    take two levels (a first digit of 2 or 1 bits): reconstruction equals
    F(x) for all x and all masks r, for a plain piecewise polynomial and for
    one with a shift gate on its output."""
    rng = np.random.default_rng(70 + dcf_bits)
    k = 7
    N = 2 ** k
    xs = np.tile(np.arange(N, dtype=np.uint64), N) + (rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k))
    rs = np.repeat(np.arange(N, dtype=np.uint64), N) + (rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k))
    for trial in range(2):
        sp = S.random_spec(rng, k, int(rng.integers(5, 17)), int(rng.integers(1, 4)), 1, partition_bits=bool(trial),
                           n_extra=2)
        if trial:
            sp.trunc_shift, sp.trunc_signed = 3, True
        sp = sp.arity(dcf_bits)
        o, res, y, z = run_gate(sp, xs, r_override=rs)
        yp, zp = python_plain(sp, xs)
        assert (y == yp).all() and (z == zp).all(), trial


@pytest.mark.parametrize("dcf_bits", [2, 6])
def test_relu_worked_example_closed_form(dcf_bits):
    """App. N: y = max(x, 0) and z = MSB(x) on signed k-bit inputs, with the
    stated compiled shapes; with DCF keys of arity 4 and of arity 64 (three
    levels at k = 16, the arity the plain form picks for the layer's gates)."""
    fx = dict(line.split() for line in open(golden("relu_worked_example.txt"))
              if line.strip() and not line.startswith("#"))
    k = 16
    sp = S.relu(k).arity(dcf_bits)
    rng = np.random.default_rng(5)
    xs_signed = np.concatenate([np.array([0, 1, -1, 2 ** 15 - 1, -(2 ** 15)], dtype=np.int64),
                                rng.integers(-(2 ** 15), 2 ** 15, size=3000, dtype=np.int64)])
    o, res, y, z = run_gate(sp, xs_signed.view(np.uint64))
    assert o.M == int(fx["M"]) and o.p == int(fx["p"]) and o.T == int(fx["T"])
    assert o.n_mults == int(fx["mults"]) and sp.m == int(fx["m"])
    assert (y[:, 0].view(np.int64) == np.maximum(xs_signed, 0)).all()
    assert (z == (xs_signed < 0).astype(np.uint32)).all()


def test_relu_every_mask_small_ring():
    """The same closed form at k = 4 over every (x, r) pair, x sign-extended."""
    k, N = 4, 16
    sp = S.relu(k)
    xs_signed = np.tile(np.arange(-8, 8, dtype=np.int64), N)
    rs = np.repeat(np.arange(N, dtype=np.uint64), N)
    o, res, y, z = run_gate(sp, xs_signed.view(np.uint64), r_override=rs)
    assert (y[:, 0].view(np.int64) == np.maximum(xs_signed, 0)).all()
    assert (z == (xs_signed < 0).astype(np.uint32)).all()


def test_special_cases():
    rng = np.random.default_rng(9)
    x = rng.integers(0, 2 ** 64, size=500, dtype=np.uint64)
    # identity polynomial P(x) = x on one interval: no lookup keys (App. O), y = x
    coeff = np.zeros((1, 1, 2), np.uint64)
    coeff[0, 0, 1] = 1
    sp = S.OperatorSpec("id", 16, 0, 0, 1, 1, 1, [0, 1 << 16], coeff)
    o, res, y, z = run_gate(sp, x)
    assert o.M == 1 and o.T == 0
    assert (y[:, 0] == x).all()
    # degree 0: no Beaver multiplications, no Horner communication
    sp = S.random_spec(rng, 12, 5, 0)
    o, res, y, z = run_gate(sp, x)
    assert o.n_mults == 0 and (res["comm"] == 8 * x.size).all()
    assert (y == python_plain(sp, x)[0]).all()
    # sentinel predicates: C_0 = 0 and C_{2^f} = 1 need no queries
    sp = S.random_spec(rng, 10, 3, 1, partition_bits=False)
    sp.preds = [S.PredDesc(10, 0, 0, 0), S.PredDesc(6, 3, 64, 0), S.PredDesc(6, 0, 64, 1)]
    o, res, y, z = run_gate(sp, x)
    assert o.T == 0
    assert (z == 0b010).all()


def test_shapes_are_mask_independent_and_match_counts():
    """Prop. 'mask-independent shape via padding' and App. O counts for the
    workload specs: T, M, p and the per-element key record do not depend on r."""
    for sp, T, M, p in [(S.gelu4(), 4, 5, 3), (S.gelu8(), 8, 9, 3), (S.nexp16(), 16, 17, 4),
                        (S.recip16(), 16, 17, 4), (S.rsqrt16(), 16, 17, 4), (S.silu16(), 16, 17, 4)]:
        o = ospec(sp)
        assert (o.T, o.M, o.p) == (T, M, p), sp.name
        for r in [0, 1, (1 << sp.k) - sp.alpha[1], 12345, (1 << sp.k) - 1, 2 ** 63 + 7]:
            B, _ = o.compile_lookup(r)
            assert len(B) == M + 1


def test_query_list_order():
    """The fixed descriptor order: per view the 1[v < r_f] atom first, then one
    theta atom per distinct predicate; MSB merges with the boundary 2^(k-1)."""
    o = ospec(S.gelu4())
    q = o.queries()
    assert q[0] == (16, 0, -1)
    assert [x[2] for x in q[1:]] == [0, 1, 2]
    assert o.n_bool == 4


def test_distinct_calls_draw_distinct_masks():
    sp = S.gelu4()
    o = ospec(sp)
    x = np.zeros(64, np.uint64)
    a0, a1, _, _ = O.dealer(o, SEED, 0, 0, 64, x)
    b0, b1, _, _ = O.dealer(o, SEED, 1, 0, 64, x)
    ra = [(a0.fields(o, i)["r_share"] + a1.fields(o, i)["r_share"]) & M64 for i in range(64)]
    rb = [(b0.fields(o, i)["r_share"] + b1.fields(o, i)["r_share"]) & M64 for i in range(64)]
    assert len(set(ra) | set(rb)) == 128


@pytest.mark.parametrize("k", [2, 4, 5])
def test_xhat_basis_variant_every_mask_every_input(k):
    """The x^-basis payload variant: the dealer re-expands each piece as a
    polynomial in the public x^ (binomial expansion of P(x^ - r) over
    Z_{2^64}); reconstruction still equals F(x) for all x and r, with no
    Beaver multiplication and only the 8-byte opening on the wire."""
    rng = np.random.default_rng(90 + k)
    N = 2 ** k
    for trial in range(6):
        m = int(rng.integers(1, min(N, 16) + 1))
        d = int(rng.integers(0, 4))
        r = 1 if d > 1 else int(rng.integers(1, 3))
        sp = S.random_spec(rng, k, m, d, r, partition_bits=bool(trial % 2), n_extra=int(rng.integers(0, 3)))
        sp = sp.variant(True)
        hi_x = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
        hi_r = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
        xs = np.tile(np.arange(N, dtype=np.uint64), N) + hi_x
        rs = np.repeat(np.arange(N, dtype=np.uint64), N) + hi_r
        o, res, y, z = run_gate(sp, xs, r_override=rs)
        assert o.n_mults == 0
        yp, zp = python_plain(sp, xs)
        assert (y == yp).all() and (z == zp).all()
        assert (res["comm"] == xs.size * 8).all()


def test_xhat_basis_matches_standard_reconstruction():
    """Same inputs and masks through both variants: shares differ, the
    reconstructed outputs agree (the workload specs, full 64-bit masks)."""
    for sp in (S.gelu8(), S.nexp16()):
        x = np.random.default_rng(4).integers(0, 2 ** 64, size=200, dtype=np.uint64)
        _, _, y_std, z_std = run_gate(sp, x, call_id=3)
        _, _, y_x, z_x = run_gate(sp.variant(True), x, call_id=3)
        assert np.array_equal(y_std, y_x) and np.array_equal(z_std, z_x)


@pytest.mark.parametrize("k", [2, 3, 5])
def test_piecewise_boolean_outputs_every_mask_every_input(k):
    """Lemma "boolean normalization": piecewise Boolean outputs
    z_j = XOR_i (J_i AND B_i^(j)) with XOR-shared interval indicators and one
    packed Boolean AND triple per 32 gates reconstruct B_{i*}^(j)(x) for all
    x and r; the n_pw * m normalisation ANDs take one round and 8 bytes per
    party per 32 of them (one opening of e and f)."""
    rng = np.random.default_rng(120 + k)
    N = 2 ** k
    for trial in range(6):
        m = int(rng.integers(1, min(N, 16) + 1))
        d = int(rng.integers(0, 3))
        sp = S.random_spec(rng, k, m, d, 1, partition_bits=bool(trial % 2), n_extra=int(rng.integers(0, 3)))
        sp = S.random_piecewise(rng, sp, int(rng.integers(1, 5)))
        if trial % 3 == 2:
            sp = sp.variant(True)
        hi_x = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
        hi_r = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
        xs = np.tile(np.arange(N, dtype=np.uint64), N) + hi_x
        rs = np.repeat(np.arange(N, dtype=np.uint64), N) + hi_r
        o, res, y, z = run_gate(sp, xs, r_override=rs)
        yp, zp = python_plain(sp, xs)
        assert (y == yp).all() and (z == zp).all(), (trial, sp.name)
        mults = 0 if sp.xhat_basis else d
        words = -(-len(sp.piecewise) * m // 32)
        assert o.n_bw == words
        assert (res["comm"] == xs.size * (8 + 16 * mults + 8 * words)).all()


def _and_rounds(nodes, roots):
    """Rounds and packed words of the formulas' AND gates, from the AND
    depths: AND / OR add one, NOT / XOR keep their inputs' depth."""
    dep = []
    for nd in nodes:
        if nd.op in ("pred", "const"):
            dep.append(0)
        elif nd.op == "not":
            dep.append(dep[nd.a])
        else:
            dep.append(max(dep[nd.a], dep[nd.b]) + (0 if nd.op == "xor" else 1))
    gates = {}
    for v, nd in enumerate(nodes):
        if nd.op in ("and", "or"):
            gates[dep[v]] = gates.get(dep[v], 0) + 1
    for out in roots:
        for r in out:
            gates[dep[r] + 1] = gates.get(dep[r] + 1, 0) + 1
    return max(gates), sum(-(-g // 32) for g in gates.values())


@pytest.mark.parametrize("k", [2, 3, 4])
def test_formula_outputs_every_mask_every_input(k):
    """Boolean formulas per interval (NOT / XOR / AND / OR over predicates
    and constants, AND depth up to 4): the round-by-round evaluation on XOR
    shares with packed Boolean AND triples reconstructs B_{i*}^(j)(x) for
    every x and every mask r; each AND round sends 8 bytes per party per 32
    gates."""
    rng = np.random.default_rng(310 + k)
    N = 2 ** k
    for trial in range(5):
        m = int(rng.integers(1, min(N - 1, 8) + 1))
        d = int(rng.integers(0, 3))
        sp = S.random_spec(rng, k, m, d, 1, partition_bits=bool(trial % 2), n_extra=int(rng.integers(0, 2)))
        sp = S.random_formulas(rng, sp, int(rng.integers(1, 4)), n_nodes=int(rng.integers(3, 30)))
        if trial % 3 == 2:
            sp = sp.variant(True)
        hi_x = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
        hi_r = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
        xs = np.tile(np.arange(N, dtype=np.uint64), N) + hi_x
        rs = np.repeat(np.arange(N, dtype=np.uint64), N) + hi_r
        o, res, y, z = run_gate(sp, xs, r_override=rs)
        yp, zp = python_plain(sp, xs)
        assert (y == yp).all() and (z == zp).all(), (trial, sp.name)
        rounds, words = _and_rounds(sp.bx_nodes, sp.piecewise)
        assert (o.n_bx_rounds, o.n_bw) == (rounds, words)
        mults = 0 if sp.xhat_basis else d
        assert (res["comm"] == xs.size * (8 + 16 * mults + 8 * words)).all()


@pytest.mark.parametrize("k", [3, 5])
def test_formula_depth_bound_every_mask_every_input(k):
    """Formulas at the AND-depth bound (4), so five exchange rounds, for
    every x and r."""
    rng = np.random.default_rng(400 + k)
    N = 2 ** k
    sp = S.deep_formula(S.random_spec(rng, k, 3, 1, 1, partition_bits=True))
    xs = np.tile(np.arange(N, dtype=np.uint64), N)
    rs = np.repeat(np.arange(N, dtype=np.uint64), N) + (rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64)
                                                         << np.uint64(k))
    o, res, y, z = run_gate(sp, xs, r_override=rs)
    assert (o.n_bx_rounds, o.n_bw) == (5, 5)
    yp, zp = python_plain(sp, xs)
    assert (y == yp).all() and (z == zp).all()


def test_formula_closed_form_example():
    """A hand-written formula with a closed form: on the negative half
    (x >= 2^(k-1)) output (x mod 16 < 8) AND NOT(x mod 4 < 1), on the
    non-negative half (x < 100) OR MSB(x + 2^(k-1)), i.e. x < 100 OR x < 2^(k-1)."""
    k = 8
    sp = S.random_spec(np.random.default_rng(2), k, 2, 1)
    sp.alpha = [0, 1 << (k - 1), 1 << k]
    sp.partition_bits = False
    sp.preds = []
    nodes = [S.BxNode("pred", pred=S.PredDesc(4, 0, 8, 0)),            # 0: x mod 16 < 8
             S.BxNode("pred", pred=S.PredDesc(2, 0, 1, 0)),            # 1: x mod 4 < 1
             S.BxNode("not", 1),                                       # 2
             S.BxNode("and", 0, 2),                                    # 3
             S.BxNode("pred", pred=S.PredDesc(k, 0, 100, 0)),          # 4: x < 100
             S.BxNode("pred", pred=S.PredDesc(k, 1 << (k - 1), 1 << (k - 1), 1)),   # 5: MSB(x + 2^(k-1))
             S.BxNode("or", 4, 5)]                                     # 6
    sp.bx_nodes, sp.piecewise = nodes, [[6, 3]]
    xs = np.arange(1 << k, dtype=np.uint64)
    _, res, _, z = run_gate(sp, xs + (np.uint64(7) << np.uint64(40)))
    want = [(int(x < 100 or x < 128) if x < 128 else int(x % 16 < 8 and x % 4 != 0)) for x in range(1 << k)]
    assert list(z) == want


def test_piecewise_relu_sign_select():
    """A concrete piecewise output: on the non-negative half return
    1[x mod 2^4 < 8] (a low-bit predicate), on the negative half the constant 1."""
    k = 8
    sp = S.relu(k)
    sp.piecewise = [[S.PredDesc(4, 0, 8, 0), S.PredDesc(k, 0, 1 << k, 0)]]
    xs = np.arange(-(2 ** (k - 1)), 2 ** (k - 1), dtype=np.int64)
    o, res, y, z = run_gate(sp, xs.view(np.uint64))
    want = np.where(xs >= 0, ((xs % 16) < 8).astype(np.uint32), 1)
    assert np.array_equal((z >> 1) & 1, want)
    assert np.array_equal(z & 1, (xs < 0).astype(np.uint32))


@pytest.mark.parametrize("dcf_bits", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("k", [2, 3, 5, 7])
def test_truncation_every_shift_every_mask_every_input(k, dcf_bits):
    """Shift gate (Def. "specification-compatible scalar gate" with the
    low-bit rewrite of App. "low-bit predicate rewrite"): for every shift s,
    both the logical and the arithmetic form, all x and all masks r, the
    reconstruction is the shift of the k-bit view; one byte per element per
    party opens the two daBit-masked bits."""
    N = 2 ** k
    rng = np.random.default_rng(300 + k)
    hi_x = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
    hi_r = rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k)
    xs = np.tile(np.arange(N, dtype=np.uint64), N) + hi_x
    rs = np.repeat(np.arange(N, dtype=np.uint64), N) + hi_r
    for s_ in range(1, k):
        for signed in (False, True):
            sp = S.trunc(k, s_, signed).arity(dcf_bits)
            o, res, y, z = run_gate(sp, xs, r_override=rs)
            yp, _ = python_plain(sp, xs)
            assert (y == yp).all(), (s_, signed)
            assert (res["comm"] == xs.size * (8 + 1)).all()


def test_truncation_textbook_shifts():
    """In-range values: the signed form is numpy's arithmetic right shift of
    int64, the logical form numpy's right shift of the unsigned k-bit value."""
    rng = np.random.default_rng(5)
    k, s_ = 32, 12
    v = rng.integers(-(2 ** 31), 2 ** 31, size=4000, dtype=np.int64)
    _, _, y, _ = run_gate(S.trunc(k, s_, True), v.view(np.uint64))
    assert np.array_equal(y[:, 0].view(np.int64), np.right_shift(v, s_))
    u = rng.integers(0, 2 ** 32, size=4000, dtype=np.uint64) + (rng.integers(0, 2 ** 31, size=4000, dtype=np.uint64) << np.uint64(33))
    _, _, y, _ = run_gate(S.trunc(k, s_, False), u)
    assert np.array_equal(y[:, 0], (u & np.uint64(2 ** 32 - 1)) >> np.uint64(s_))


@pytest.mark.parametrize("k", [3, 6])
def test_truncation_with_polynomial_and_boolean_outputs(k):
    """A shift added to a piecewise polynomial's first output, beside
    predicates, piecewise outputs and the x^-basis variant; all x, all r."""
    N = 2 ** k
    rng = np.random.default_rng(400 + k)
    xs = np.tile(np.arange(N, dtype=np.uint64), N) + (rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k))
    rs = np.repeat(np.arange(N, dtype=np.uint64), N) + (rng.integers(0, 2 ** 40, size=N * N, dtype=np.uint64) << np.uint64(k))
    for trial in range(6):
        m = int(rng.integers(1, min(N, 16) + 1))
        d = int(rng.integers(0, 3))
        r = 1 if d > 1 else int(rng.integers(1, 3))
        sp = S.random_spec(rng, k, m, d, r, partition_bits=bool(trial % 2), n_extra=int(rng.integers(0, 3)))
        if trial % 3 == 1:
            sp = S.random_piecewise(rng, sp, 2)
        sp.trunc_shift, sp.trunc_signed = int(rng.integers(1, k)), bool(trial % 2)
        if trial % 3 == 2:
            sp = sp.variant(True)
        o, res, y, z = run_gate(sp, xs, r_override=rs)
        yp, zp = python_plain(sp, xs)
        assert (y == yp).all() and (z == zp).all(), trial
        mults = 0 if sp.xhat_basis else d * r
        assert (res["comm"] == xs.size * (8 + 16 * mults + 8 * -(-len(sp.piecewise) * sp.m // 32) + 1)).all()


@pytest.mark.parametrize("dcf_bits", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("k,s", [(40, 20), (63, 49), (63, 1), (48, 47)])
def test_truncation_wide_views(k, s, dcf_bits):
    """Shift gates on views wider than 32 bits (single-interval specs may use
    k up to 63): random 64-bit x against Python's integer shift of the k-bit
    view; at k = 63 the arithmetic form equals numpy's int64 right shift of
    values inside the 63-bit signed range."""
    rng = np.random.default_rng(k * 100 + s)
    x = rng.integers(0, 2 ** 64, size=3000, dtype=np.uint64)
    for signed in (False, True):
        sp = S.trunc(k, s, signed).arity(dcf_bits)
        _, res, y, _ = run_gate(sp, x)
        yp, _ = python_plain(sp, x)
        assert np.array_equal(y, yp), signed
        assert (res["comm"] == x.size * 9).all()
    if k == 63:
        v = rng.integers(-(2 ** 62), 2 ** 62, size=3000, dtype=np.int64)
        _, _, y, _ = run_gate(S.trunc(63, s, True), v.view(np.uint64))
        assert np.array_equal(y[:, 0].view(np.int64), np.right_shift(v, s))


def test_wide_view_predicates_single_interval():
    """m = 1 specs with predicates on views up to 63 bits (no lookup)."""
    rng = np.random.default_rng(77)
    x = rng.integers(0, 2 ** 64, size=2000, dtype=np.uint64)
    for k in (33, 50, 63):
        preds = [S.PredDesc(k, 0, 1 << (k - 1), 1),                       # MSB of the k-bit view
                 S.PredDesc(k, int(rng.integers(0, 2 ** k, dtype=np.uint64)), int(rng.integers(1, 2 ** k, dtype=np.uint64)), 0),
                 S.PredDesc(min(k, 40), 12345, 2 ** (min(k, 40) - 1) + 7, 1)]
        coeff = rng.integers(0, 2 ** 64, size=(1, 1, 3), dtype=np.uint64)
        sp = S.OperatorSpec(f"wide{k}", k=k, frac_bits=0, out_frac_bits=0, m=1, degree=2, n_out=1,
                            alpha=[0, 1 << k], coeff=coeff, partition_bits=False, preds=preds)
        _, _, y, z = run_gate(sp, x)
        yp, zp = python_plain(sp, x)
        assert np.array_equal(y, yp) and np.array_equal(z, zp), k
    # a lookup needs k <= 32
    with pytest.raises(ValueError):
        ospec(S.random_spec(rng, 33, 3, 1, 1))
